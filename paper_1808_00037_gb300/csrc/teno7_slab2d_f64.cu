// FP64 slab mode of the 2D kernels (Stage2D.halo: padded arrays, global alphas
// from device doubles).  Its own translation unit, built with -fmad=false as
// teno7_f64.cu is, so that the whole-domain instantiations there stay
// untouched and compile in parallel with these.
#include "teno7_kernels2d.cuh"

namespace t7 {
cudaError_t launch_stage2d_slab_f64(const Stage2D &p, cudaStream_t s) { return launch_stage2d<double, true>(p, s); }
cudaError_t launch_alpha2d_slab_f64(const Alpha2D &p, cudaStream_t s) { return launch_alpha2d<double, true>(p, s); }
}  // namespace t7
