// FP32 instantiation of the TENO7-ext kernels (FMA contraction on).
#include "teno7_kernels.cuh"

namespace t7 {
cudaError_t launch_stage1d_f32(const Stage1D &p, cudaStream_t s) { return launch_stage1d<float>(p, s); }
cudaError_t launch_alpha1d_f32(const Alpha1D &p, cudaStream_t s) { return launch_alpha1d<float>(p, s); }
cudaError_t launch_recon_f32(const Recon &p, cudaStream_t s) { return launch_recon<float>(p, s); }
}  // namespace t7
