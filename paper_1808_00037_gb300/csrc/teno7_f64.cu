// FP64 instantiation of the TENO7-ext kernels.  Built with -fmad=false so that
// each FP64 expression is evaluated operation by operation in source order.
#include "teno7_kernels.cuh"
#include "teno7_kernels2d.cuh"
#include "teno7_adjoint.cuh"

namespace t7 {
cudaError_t launch_stage1d_f64(const Stage1D &p, cudaStream_t s) { return launch_stage1d<double>(p, s); }
cudaError_t launch_alpha1d_f64(const Alpha1D &p, cudaStream_t s) { return launch_alpha1d<double>(p, s); }
cudaError_t launch_recon_f64(const Recon &p, cudaStream_t s) { return launch_recon<double>(p, s); }
cudaError_t launch_stage2d_f64(const Stage2D &p, cudaStream_t s) { return launch_stage2d<double>(p, s); }
cudaError_t launch_alpha2d_f64(const Alpha2D &p, cudaStream_t s) { return launch_alpha2d<double>(p, s); }
cudaError_t launch_batch1d_f64(const Batch1D &p, cudaStream_t s) { return launch_batch1d<double>(p, s); }
cudaError_t launch_batch1d_alpha_f64(const Batch1D &p, double *a, cudaStream_t s) {
    return launch_batch1d_alpha<double>(p, a, s);
}
int batch1d_groups_f64(int group_warps) { return batch1d_groups<double>(group_warps); }
cudaError_t launch_rhs_adjoint1d_f64(const Adjoint1D &p, cudaStream_t s) { return launch_rhs_adjoint1d<double>(p, s); }
cudaError_t launch_combine_f64(void *out, const void *x, const void *y, const void *z, double c1, double c2,
                               double c3, size_t N, cudaStream_t s) {
    return launch_combine<double>(out, x, y, z, c1, c2, c3, N, s);
}
cudaError_t launch_combine2_f64(void *out1, void *out2, const void *x, const void *y, double a1, double b1,
                                double a2, double b2, size_t N, cudaStream_t s) {
    return launch_combine2<double>(out1, out2, x, y, a1, b1, a2, b2, N, s);
}
}  // namespace t7
