// FP64 instantiation of the TENO7-ext kernels.  Built with -fmad=false so that
// each FP64 expression is evaluated operation by operation in source order.
#include "teno7_kernels.cuh"
#include "teno7_kernels2d.cuh"

namespace t7 {
cudaError_t launch_stage1d_f64(const Stage1D &p, cudaStream_t s) { return launch_stage1d<double>(p, s); }
cudaError_t launch_alpha1d_f64(const Alpha1D &p, cudaStream_t s) { return launch_alpha1d<double>(p, s); }
cudaError_t launch_recon_f64(const Recon &p, cudaStream_t s) { return launch_recon<double>(p, s); }
cudaError_t launch_stage2d_f64(const Stage2D &p, cudaStream_t s) { return launch_stage2d<double>(p, s); }
cudaError_t launch_alpha2d_f64(const Alpha2D &p, cudaStream_t s) { return launch_alpha2d<double>(p, s); }
cudaError_t launch_batch1d_f64(const Batch1D &p, cudaStream_t s) { return launch_batch1d<double>(p, s); }
}  // namespace t7
