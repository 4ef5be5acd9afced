// FP32 and mixed-precision slab mode of the 2D kernels (Stage2D.halo: padded
// arrays, global alphas from device doubles).  Its own translation unit, so
// that the whole-domain instantiations in teno7_f32.cu stay untouched and
// compile in parallel with these.
#include "teno7_kernels2d.cuh"

namespace t7 {
cudaError_t launch_stage2d_slab_f32(const Stage2D &p, cudaStream_t s) { return launch_stage2d<float, true>(p, s); }
cudaError_t launch_stage2d_slab_mixed(const Stage2D &p, cudaStream_t s) {
    return launch_stage2d_paired<double, true>(p, s);
}
cudaError_t launch_alpha2d_slab_f32(const Alpha2D &p, cudaStream_t s) { return launch_alpha2d<float, true>(p, s); }
}  // namespace t7
