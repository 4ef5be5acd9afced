// FP32 instantiation of the TENO7-ext kernels (FMA contraction on).
#include "teno7_kernels.cuh"
#include "teno7_kernels2d.cuh"
#include "teno7_adjoint.cuh"

namespace t7 {
cudaError_t launch_stage1d_f32(const Stage1D &p, cudaStream_t s) { return launch_stage1d<float>(p, s); }
cudaError_t launch_stage1d_mixed(const Stage1D &p, cudaStream_t s) { return launch_stage1d_paired<double>(p, s); }
cudaError_t launch_alpha1d_f32(const Alpha1D &p, cudaStream_t s) { return launch_alpha1d<float>(p, s); }
cudaError_t launch_recon_f32(const Recon &p, cudaStream_t s) { return launch_recon<float>(p, s); }
cudaError_t launch_stage2d_f32(const Stage2D &p, cudaStream_t s) { return launch_stage2d<float>(p, s); }
cudaError_t launch_stage2d_mixed(const Stage2D &p, cudaStream_t s) { return launch_stage2d_paired<double>(p, s); }
cudaError_t launch_alpha2d_f32(const Alpha2D &p, cudaStream_t s) { return launch_alpha2d<float>(p, s); }
cudaError_t launch_batch1d_f32(const Batch1D &p, cudaStream_t s) { return launch_batch1d<float>(p, s); }
cudaError_t launch_batch1d_alpha_f32(const Batch1D &p, double *a, cudaStream_t s) {
    return launch_batch1d_alpha<float>(p, a, s);
}
int batch1d_groups_f32(int group_warps) { return batch1d_groups<float>(group_warps); }

// Self-test of the index check (t7_probe_index_check): one thread passes i
// through chk against [lo, hi) and writes the index an access would use; no
// memory is addressed by i.
__global__ void index_check_probe_kernel(int i, int lo, int hi, DevCtl *ctl, int *out) {
    out[0] = chk(ctl, i, lo, hi);
    out[1] = T7_CHECKED;
}
cudaError_t launch_index_check_probe(int i, int lo, int hi, DevCtl *ctl, int *out, cudaStream_t s) {
    index_check_probe_kernel<<<1, 1, 0, s>>>(i, lo, hi, ctl, out);
    return cudaGetLastError();
}
cudaError_t launch_rhs_adjoint1d_f32(const Adjoint1D &p, cudaStream_t s) { return launch_rhs_adjoint1d<float>(p, s); }
cudaError_t launch_combine_f32(void *out, const void *x, const void *y, const void *z, double c1, double c2,
                               double c3, size_t N, cudaStream_t s) {
    return launch_combine<float>(out, x, y, z, c1, c2, c3, N, s);
}
cudaError_t launch_combine2_f32(void *out1, void *out2, const void *x, const void *y, double a1, double b1,
                                double a2, double b2, size_t N, cudaStream_t s) {
    return launch_combine2<float>(out1, out2, x, y, a1, b1, a2, b2, N, s);
}
}  // namespace t7
