// Internal declarations shared by the translation units of libteno7 (the
// precision-specific kernel files and the C-ABI file).  Not installed.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace t7 {

enum { SYS_ADV = 0, SYS_EULER1D = 1, SYS_EULER2D = 2, SYS_BURGERS = 3 };
enum { BC_PERIODIC = 0, BC_ZG = 1 };
enum { ERR_NONPHYSICAL = 1, ERR_NONFINITE = 2, ERR_NOEXIST = 4, ERR_INDEX = 8 };

// Device-resident control block of a context.  amax[slot][dir] holds the bit
// pattern of a non-negative double (max characteristic speed) so that it can
// be reduced with atomicMax on unsigned 64-bit integers.
//
// The last CTA of every stage launch (and of the alpha kernel) finalizes the
// launch: it converts the freshly reduced alpha to float (alpha_f), clears the
// slot the next launch accumulates into, and at the end of an RK step advances
// t and computes the next CFL step, so that no CTA ever divides in FP64.
struct DevCtl {
    // alphas of slots 0-2 as the bits of non-negative doubles: [slot][0] 1D
    // global, [slot][0..1] 2D (x, y), [slot][0..2] 1D per characteristic field
    unsigned long long amax[3][3];
    double t, dt, t_end, cfl, dx, dy;
    float alpha_f[3][3];
    float dt_f, pad_f;
    int steps, max_steps, active, err;
    int err_index;
    unsigned blocks_done;
};

// Cells a warp tile of the 1D stage kernels updates (the stage launches'
// tile_lo / tile_hi count these tiles).
constexpr int TILE_CELLS = 29;

// One launch of the fused 1D stage kernel.
struct Stage1D {
    const void *Us;  // stage input state [m][n] (stencil reads)
    const void *U0;  // U^n (pointwise reads; stages 1 and 2 only)
    void *out;       // RK mode: stage output; RHS mode: dU/dt
    uint8_t *masks;  // RHS mode, nullable: [2][m][n+1]
    int n, sys, bc_lo, bc_hi;
    double dx, eps, CT, gamma, a;
    int rhs_mode;    // 1: write L(U) (and masks); 0: RK stage
    int stage;       // 0, 1, 2 (RK mode)
    double dt_fixed; // > 0: use it; otherwise the control block's dt
    DevCtl *ctl;
    int slot_in;     // alpha of Us
    // the same parameters rounded to float, for the FP32 kernels
    float f_dx, f_eps, f_CT, f_gamma, f_gm1, f_a, f_dt_fixed;
    int scheme;         // 0: TENO7-ext, 1: TENO5 baseline
    double *alpha_rec;  // nullable: receives alpha of the output state (RK mode)
    int tile_lo, tile_hi;  // warp tiles [tile_lo, tile_hi) of the domain (29 cells each; tile_hi <= 0: all)
    int partial;           // RK mode: one part of a stage split over several launches, not its last
    // Slab of a decomposed domain: Us, U0 and out are padded by HALO_CELLS
    // cells per side (row stride n + 2 HALO_CELLS, cell 0 at offset
    // HALO_CELLS); the stencils read the padding, which the caller has
    // filled, instead of applying the boundary condition
    int halo;
    const double *alpha_in;  // nullable: alpha of Us from this device value instead of the control block
    int alpha_mode;          // t7_alpha_mode: 1 = one alpha per characteristic field (1D Euler)
};

// Ghost cells per side of a slab (the stencil reach of the scheme, Eq. app:
// the RHS at cell i depends on cells i-4 .. i+4).
constexpr int HALO_CELLS = 4;

struct Alpha1D {
    const void *U;
    int n, sys;
    int stride;  // between conserved variables (0: n)
    double gamma, a;
    DevCtl *ctl;
    int slot;
    double *alpha_rec;  // nullable: receives the finished alpha
    int alpha_mode;     // 1: the three per-field alphas of 1D Euler into amax[slot][0..2]
};

// One stage of the 2D Euler system, dimension by dimension: the x sweep
// writes Lx(U) into R, the y sweep adds Ly(U) and applies the RK stage.
struct Stage2D {
    const void *Us;  // stage input [4][ny][nx]
    const void *U0;  // U^n (stages 1 and 2)
    void *out;       // RK mode: stage output; RHS mode: dU/dt (== R)
    void *R;         // x part of L(U), [4][ny][nx]
    uint8_t *masks;  // RHS mode, nullable: x faces [2][4][ny][nx+1], then y faces [2][4][nx][ny+1]
    int nx, ny;
    int bc[4];
    double dx, dy, eps_x, eps_y, CT, gamma;
    int rhs_mode, stage;
    double dt_fixed;
    DevCtl *ctl;
    int slot_in;
    float f_dx, f_dy, f_eps_x, f_eps_y, f_CT, f_gamma, f_gm1, f_dt_fixed;
    // Slab of a domain cut along y (the launch_*_slab_* entry points only):
    // Us, U0 and (RK mode) out hold HALO_CELLS padding rows per side
    // ([4][ny + 2 HALO_CELLS][nx]) and point at row 0, sv and svo are the
    // strides between conserved variables of Us / U0 and of out (R is always
    // [4][ny][nx]); the y stencils read the padding, which the caller has
    // filled, instead of applying the y boundary condition
    size_t sv, svo;
    int halo;
    const double *alpha_in;  // nullable: [2] alpha_x, alpha_y of Us instead of the control block's
    double *alpha_rec;       // nullable: receives [2] alpha_x, alpha_y of the output (RK mode)
};

struct Alpha2D {
    const void *U;
    int nx, ny;
    size_t stride;  // slab mode: between conserved variables
    double gamma;
    DevCtl *ctl;
    int slot;
    double *alpha_rec;  // nullable: receives [2] the finished alpha_x, alpha_y
};

// chk() on one index (teno7_f32.cu): out[0] = the index used, out[1] = T7_CHECKED
cudaError_t launch_index_check_probe(int i, int lo, int hi, DevCtl *ctl, int *out, cudaStream_t s);
cudaError_t launch_stage2d_f64(const Stage2D &p, cudaStream_t s);
cudaError_t launch_stage2d_f32(const Stage2D &p, cudaStream_t s);
cudaError_t launch_stage2d_mixed(const Stage2D &p, cudaStream_t s);  // FP64 state, FP32 reconstruction
cudaError_t launch_alpha2d_f64(const Alpha2D &p, cudaStream_t s);
cudaError_t launch_alpha2d_f32(const Alpha2D &p, cudaStream_t s);
// slab mode (halo, alpha_in, alpha_rec, sv / svo / stride honoured)
cudaError_t launch_stage2d_slab_f64(const Stage2D &p, cudaStream_t s);
cudaError_t launch_stage2d_slab_f32(const Stage2D &p, cudaStream_t s);
cudaError_t launch_stage2d_slab_mixed(const Stage2D &p, cudaStream_t s);
cudaError_t launch_alpha2d_slab_f64(const Alpha2D &p, cudaStream_t s);
cudaError_t launch_alpha2d_slab_f32(const Alpha2D &p, cudaStream_t s);

// A ragged batch of independent 1D Euler tubes, concatenated variable-major
// ([3][Ntot]); each tube runs its own SSP-RK3 loop to t_end inside one
// persistent launch.
struct Batch1D {
    void *U;                   // state, advanced in place
    void *W1, *W2;             // stage buffers, same layout
    const long long *offsets;  // device, ntubes + 1
    const double *dx;          // device, per tube
    const int *order;          // device, processing order
    int ntubes;
    long long Ntot;
    int bc_lo, bc_hi;
    double t_end, cfl, gamma, CT;
    int max_steps;
    int group_warps;           // warps per tube (1, 2, 4 or 8)
    int nbig;                  // the first nbig tubes of `order` run on whole CTAs (all 8 warps)
    int *queue;                // device work counters [2] (whole-CTA, then group tubes), zero before the launch
    int *steps_out;            // device, per tube
    double *t_out;             // device, per tube
    DevCtl *ctl;               // error word
};

cudaError_t launch_batch1d_f64(const Batch1D &p, cudaStream_t s);
cudaError_t launch_batch1d_f32(const Batch1D &p, cudaStream_t s);
// concurrent groups of `group_warps` warps the batch kernel runs (CTAs x groups per CTA)
int batch1d_groups_f64(int group_warps);
int batch1d_groups_f32(int group_warps);
// per-tube wave speed max(|u| + c) of p.U into alpha_out[ntubes] (device);
// reads p.U, p.offsets, p.ntubes, p.Ntot, p.gamma
cudaError_t launch_batch1d_alpha_f64(const Batch1D &p, double *alpha_out, cudaStream_t s);
cudaError_t launch_batch1d_alpha_f32(const Batch1D &p, double *alpha_out, cudaStream_t s);

// Discrete adjoint of the 1D Euler right-hand side (teno7_adjoint.cuh).
struct Adjoint1D;
cudaError_t launch_rhs_adjoint1d_f64(const Adjoint1D &p, cudaStream_t s);
cudaError_t launch_rhs_adjoint1d_f32(const Adjoint1D &p, cudaStream_t s);
cudaError_t launch_combine_f64(void *out, const void *x, const void *y, const void *z, double c1, double c2,
                               double c3, size_t N, cudaStream_t s);
cudaError_t launch_combine_f32(void *out, const void *x, const void *y, const void *z, double c1, double c2,
                               double c3, size_t N, cudaStream_t s);
// out1 = a1 x + b1 y; out2 (nullable) = a2 x + b2 y; x may be null
cudaError_t launch_combine2_f64(void *out1, void *out2, const void *x, const void *y, double a1, double b1,
                                double a2, double b2, size_t N, cudaStream_t s);
cudaError_t launch_combine2_f32(void *out1, void *out2, const void *x, const void *y, double a1, double b1,
                                double a2, double b2, size_t N, cudaStream_t s);

// Finalization done by the last CTA of a launch (see DevCtl).
enum { FIN_NONE = 0, FIN_ALPHA = 1, FIN_STEP = 2 };

struct Recon {
    const void *v;  // n + 8 values
    void *fhat;     // n + 1
    uint8_t *d3, *D5;
    int n, sign;
    double eps, CT;
    DevCtl *ctl;
};

cudaError_t launch_stage1d_f64(const Stage1D &p, cudaStream_t s);
cudaError_t launch_stage1d_f32(const Stage1D &p, cudaStream_t s);
cudaError_t launch_stage1d_mixed(const Stage1D &p, cudaStream_t s);  // FP64 state, FP32 reconstruction
cudaError_t launch_alpha1d_f64(const Alpha1D &p, cudaStream_t s);
cudaError_t launch_alpha1d_f32(const Alpha1D &p, cudaStream_t s);
cudaError_t launch_recon_f64(const Recon &p, cudaStream_t s);
cudaError_t launch_recon_f32(const Recon &p, cudaStream_t s);

// Control-block helpers (teno7_api.cu).
cudaError_t launch_ctl_begin(DevCtl *ctl, double t_end, double cfl, double dx, double dy, int max_steps,
                             cudaStream_t s);

}  // namespace t7
