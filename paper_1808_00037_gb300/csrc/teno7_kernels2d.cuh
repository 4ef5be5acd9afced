// teno7_kernels2d.cuh -- 2D Euler, dimension by dimension (L = Lx + Ly), with the
// TENO7-ext reconstruction of each direction in its own characteristic frame
// (Roe average of the two cells of the face; fields un-c, un, shear, un+c).
//
//   x sweep  warp tiles along rows, as the 1D kernels (lane = face; the FP32
//            state's kernel pairs two faces per lane in 61-cell tiles, as the
//            1D face-paired kernel); writes Lx(U) into R (coalesced along x).
//   y sweep  one CTA stages a block of 39 rows x 32 columns (29-row tile + halo)
//            in padded shared memory; each warp runs the lane = face logic down
//            4 of the columns, exchanging cutoff words and face fluxes by
//            __shfl along y; after a barrier the CTA adds Lx, applies the RK
//            stage and reduces max(|u|+c), max(|v|+c) in row-major order (the
//            FP32 state's kernel is persistent and copies the next block's
//            state in by cp.async while the current one computes).
//
// Templated on T; instantiated for FP64 (-fmad=false: the oracle's operation
// order, including the component permutation of the y frame) and FP32.
#pragma once
#include "teno7_kernels.cuh"

namespace t7 {

// Flat index y * nx + x of the cell a fault is reported at.  A face flag
// names the face's left (x sweep) or lower (y sweep) cell, clamped into the
// grid: x sweep flat_cell(y, j, nx), y sweep flat_cell(j, x, nx, ny).
__device__ __forceinline__ int flat_cell(int y, int x, int nx, int ny = 0x7fffffff) {
    x = x < 0 ? 0 : (x >= nx ? nx - 1 : x);
    y = y < 0 ? 0 : (y >= ny ? ny - 1 : y);
    return y * nx + x;
}

// Per-face state of one 2D sweep: characteristic projections of the 8 stencil
// cells, Roe state, cutoff word ('+' codes at bits 3k, '-' at 3(4+k)).
template <typename T>
struct Face2D {
    T qp[4][7], qm[4][7];
    T un, vt, c, Ht, q2;
    unsigned word;
    int flag;
};

// Rotated index of physical component c for sweep direction DIR (1 <-> 2 in y).
template <int DIR>
__device__ __forceinline__ constexpr int rot(int c) {
    return DIR == 0 ? c : (c == 1 ? 2 : (c == 2 ? 1 : c));
}

// Frame, projection and cutoff bits of one face.  pr(q, t): staged primitive q
// (0 normal velocity, 1 tangential velocity, 2 H, 3 sqrt(rho)) of local cell t;
// gp(c, t) / gm(c, t): physical component c of the split fluxes of local cell
// t; local cell t = 0 .. 7 is cell j-3+t of face j+1/2.
template <typename T, int DIR, typename PR, typename GP, typename GM>
__device__ __forceinline__ void face2d_bits(Face2D<T> &F, PR pr, GP gp, GM gm, T gm1, T eps, T CT, T kt) {
    const T unl = pr(0, 3), unr = pr(0, 4), utl = pr(1, 3), utr = pr(1, 4);
    const T Hl = pr(2, 3), Hr = pr(2, 4), sl = pr(3, 3), sr = pr(3, 4);
    F.un = (sl * unl + sr * unr) / (sl + sr);
    F.vt = (sl * utl + sr * utr) / (sl + sr);
    F.Ht = (sl * Hl + sr * Hr) / (sl + sr);
    F.q2 = T(0.5) * (F.un * F.un + F.vt * F.vt);
    const T c2 = gm1 * (F.Ht - F.q2);
    F.c = sq_root(c2);
    const T b1 = gm1 / c2;
    const T b2 = F.q2 * b1;
    const T un = F.un, vt = F.vt, c = F.c;
    const T Lr[4][4] = {
        {T(0.5) * (b2 + un / c), T(-0.5) * (b1 * un + T(1) / c), T(-0.5) * (b1 * vt), T(0.5) * b1},
        {T(1) - b2, b1 * un, b1 * vt, -b1},
        {-vt, T(0), T(1), T(0)},
        {T(0.5) * (b2 - un / c), T(-0.5) * (b1 * un - T(1) / c), T(-0.5) * (b1 * vt), T(0.5) * b1},
    };
    F.flag = (c2 > T(0)) ? 0 : (isfinite(c2) ? ERR_NONPHYSICAL : ERR_NONFINITE);
    F.word = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
#pragma unroll
        for (int t = 0; t < 7; t++) {
            // physical component order c = 0..3, L[k][c] = Lr[k][rot(c)]
            T sp = Lr[k][0] * gp(0, t);
            T sm = Lr[k][0] * gm(0, t + 1);
            sp = sp + Lr[k][rot<DIR>(1)] * gp(1, t);
            sm = sm + Lr[k][rot<DIR>(1)] * gm(1, t + 1);
            sp = sp + Lr[k][rot<DIR>(2)] * gp(2, t);
            sm = sm + Lr[k][rot<DIR>(2)] * gm(2, t + 1);
            sp = sp + Lr[k][3] * gp(3, t);
            sm = sm + Lr[k][3] * gm(3, t + 1);
            F.qp[k][t] = sp;
            F.qm[k][t] = sm;
        }
        const unsigned bp = cutoff_bits(F.qp[k][1], F.qp[k][2], F.qp[k][3], F.qp[k][4], F.qp[k][5], eps, CT, kt);
        const unsigned bm = cutoff_bits(F.qm[k][5], F.qm[k][4], F.qm[k][3], F.qm[k][2], F.qm[k][1], eps, CT, kt);
        F.word |= bp << (3 * k);
        F.word |= bm << (3 * (4 + k));
    }
}

// Selection, polynomial and back-projection of one face given the neighbours'
// words.  Writes the physical face flux fh[4] and (if D != nullptr) the Delta
// codes D[0..3] ('+') and D[4..7] ('-').
template <typename T, int DIR>
__device__ __forceinline__ void face2d_flux(Face2D<T> &F, unsigned wl, unsigned wr, const T *coef, T fh[4],
                                            int *D) {
    T f[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int Dp = pack_delta(wl >> (3 * k), F.word >> (3 * k), wr >> (3 * k));
        const int Dm = pack_delta(wr >> (3 * (4 + k)), F.word >> (3 * (4 + k)), wl >> (3 * (4 + k)));
        int mp = lut_select(Dp), mm = lut_select(Dm);
        if (mp == 15) {
            mp = 11;
            F.flag |= ERR_NOEXIST;
        }
        if (mm == 15) {
            mm = 11;
            F.flag |= ERR_NOEXIST;
        }
        const T *cp = coef + 7 * mp, *cm = coef + 7 * mm;
        const T fp = poly7(cp, F.qp[k][0], F.qp[k][1], F.qp[k][2], F.qp[k][3], F.qp[k][4], F.qp[k][5], F.qp[k][6]);
        const T fm = poly7(cm, F.qm[k][6], F.qm[k][5], F.qm[k][4], F.qm[k][3], F.qm[k][2], F.qm[k][1], F.qm[k][0]);
        f[k] = fp + fm;
        if (D) {
            D[k] = Dp;
            D[4 + k] = Dm;
        }
    }
    const T un = F.un, vt = F.vt, c = F.c, Ht = F.Ht, q2 = F.q2;
    // rotated right eigenvectors (columns un-c, un, shear, un+c), rows in rotated order
    const T Rr[4][4] = {
        {T(1), T(1), T(0), T(1)},
        {un - c, un, T(0), un + c},
        {vt, vt, T(1), vt},
        {Ht - un * c, q2, vt, Ht + un * c},
    };
#pragma unroll
    for (int cc = 0; cc < 4; cc++) {
        const int r = rot<DIR>(cc);
        T s = Rr[r][0] * f[0];
        s = s + Rr[r][1] * f[1];
        s = s + Rr[r][2] * f[2];
        s = s + Rr[r][3] * f[3];
        fh[cc] = s;
    }
}

// Per-cell primitives and split fluxes of one 2D state along DIR, in the
// oracle's expression order.  prim = (normal velocity, tangential velocity, H,
// sqrt(rho)).
template <typename T, int DIR>
__device__ __forceinline__ void cell2d(const T U[4], T gm1, T alpha, T prim[4], T gp[4], T gm[4]) {
    const T u = U[1] / U[0];
    const T v = U[2] / U[0];
    const T p = gm1 * (U[3] - T(0.5) * (U[1] * u + U[2] * v));
    T F[4];
    if (DIR == 0) {
        F[0] = U[1];
        F[1] = U[1] * u + p;
        F[2] = U[2] * u;
        F[3] = u * (U[3] + p);
        prim[0] = u;
        prim[1] = v;
    } else {
        F[0] = U[2];
        F[1] = U[1] * v;
        F[2] = U[2] * v + p;
        F[3] = v * (U[3] + p);
        prim[0] = v;
        prim[1] = u;
    }
    prim[2] = (U[3] + p) / U[0];
    prim[3] = sq_root(U[0]);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        gp[k] = T(0.5) * (F[k] + alpha * U[k]);
        gm[k] = T(0.5) * (F[k] - alpha * U[k]);
    }
}

// max(|u|+c) and max(|v|+c) of one cell; flags non-physical / non-finite.
// In FP32 every rounding is written out (no contraction left to the
// compiler), so that every instantiation of a kernel gives the same bits.
template <typename T>
__device__ __forceinline__ void wavespeed2d(const T U[4], T gm1, T gamma, T &sx, T &sy, int *flag) {
    const T u = U[1] / U[0];
    const T v = U[2] / U[0];
    T p, c;
    if constexpr (sizeof(T) == 4) {
        p = __fmul_rn(gm1, __fmaf_rn(-0.5f, __fmaf_rn(U[1], u, __fmul_rn(U[2], v)), U[3]));
        c = sqrtf(__fdiv_rn(__fmul_rn(gamma, p), U[0]));
    } else {
        p = gm1 * (U[3] - T(0.5) * (U[1] * u + U[2] * v));
        c = sq_root(gamma * p / U[0]);
    }
    // a non-finite cell is reported as such; a finite one needs rho > 0, p > 0
    if (!isfinite(U[0]) || !isfinite(U[1]) || !isfinite(U[2]) || !isfinite(U[3]))
        *flag |= ERR_NONFINITE;
    else if (!(U[0] > T(0)) || !(p > T(0)))
        *flag |= ERR_NONPHYSICAL;
    if constexpr (sizeof(T) == 4) {
        sx = __fadd_rn(fabsf(u), c);
        sy = __fadd_rn(fabsf(v), c);
    } else {
        sx = absval(u) + c;
        sy = absval(v) + c;
    }
}

template <typename T>
__device__ __forceinline__ T alpha_of(const DevCtl *ctl, int slot, int dir) {
    if constexpr (sizeof(T) == 8) {
        return __longlong_as_double((long long)ctl->amax[slot][dir]);
    } else {
        return ctl->alpha_f[slot][dir];
    }
}

// Slab mode of the 2D kernels (template argument HALO; see Stage2D.halo).
// The instantiations without it are the whole-domain kernels.
//
// Source row of staged row y of a y sweep: the grid's own rows as they are;
// rows outside it by the y boundary condition, or, in a slab, from the
// padding rows, those beyond the padding clamped into it (they feed only the
// polynomials of faces 0 and 31 of a tile, whose fluxes no updated cell uses).
template <bool HALO>
__device__ __forceinline__ int y_row(int y, const Stage2D &p) {
    if constexpr (HALO) {
        if (y < 0 || y >= p.ny)
            y = y < -HALO_CELLS ? -HALO_CELLS : (y >= p.ny + HALO_CELLS ? p.ny + HALO_CELLS - 1 : y);
        return chk(p.ctl, y, -HALO_CELLS, p.ny + HALO_CELLS);
    } else {
        if (y < 0 || y >= p.ny) y = ghost_map(y, p.ny, p.bc[2], p.bc[3]);
        return chk(p.ctl, y, 0, p.ny);
    }
}

// Offset of value (k, y, x) of a state array with variable stride sv (in a
// slab y may be negative: the padding rows precede row 0).
template <bool HALO>
__device__ __forceinline__ auto st_at(int k, size_t sv, int y, int nx, int x) {
    if constexpr (HALO) {
        return (ptrdiff_t)k * (ptrdiff_t)sv + (ptrdiff_t)y * nx + x;
    } else {
        return (size_t)k * sv + (size_t)y * nx + x;
    }
}

// alpha of the stage input in direction dir: the slab's global value, or the
// control block's
template <typename T, bool HALO>
__device__ __forceinline__ T alpha2d_in(const Stage2D &p, const DevCtl *ctl, int dir) {
    if constexpr (HALO) {
        return T(p.alpha_in[dir]);
    } else {
        return alpha_of<T>(ctl, p.slot_in, dir);
    }
}

// --------------------------------------------------------------------------
// x sweep: R = Lx(U), warp tiles of 29 cells along rows.
// --------------------------------------------------------------------------
template <typename T, bool HALO>
__global__ void __launch_bounds__(WPB * 32, 1) xsweep2d_kernel(const Stage2D p) {
    __shared__ T s_gp[WPB][4][WC];
    __shared__ T s_gm[WPB][4][WC];
    __shared__ T s_pr[WPB][4][WC];
    __shared__ T s_coef[WPB][92];
    DevCtl *ctl = p.ctl;
    const bool fixed = p.dt_fixed > 0.0;
    if (!p.rhs_mode && !fixed && !ctl->active) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = lane; q < 91; q += 32) s_coef[warp][q] = coef<T>(q);
    const T alpha = alpha2d_in<T, HALO>(p, ctl, 0);
    const T gm1 = pick<T>(p.gamma - 1.0, p.f_gm1);
    const T eps = pick<T>(p.eps_x, p.f_eps_x), CT = pick<T>(p.CT, p.f_CT);
    const T kt = keep_all_factor(CT);
    const T *Us = static_cast<const T *>(p.Us);
    T *R = static_cast<T *>(p.R);
    const int nx = p.nx, ny = p.ny;
    const size_t N = (size_t)nx * ny;
    const size_t sv = HALO ? p.sv : N;
    const int ntx = (nx + WT - 1) / WT;
    const long ntiles = (long)ntx * ny;
    T (*sgp)[WC] = s_gp[warp];
    T (*sgm)[WC] = s_gm[warp];
    T (*spr)[WC] = s_pr[warp];
    __syncwarp();
    for (long tile = (long)blockIdx.x * WPB + warp; tile < ntiles; tile += (long)gridDim.x * WPB) {
        const int y = (int)(tile / ntx);
        const int c0 = (int)(tile % ntx) * WT;
        const T *row = Us + (size_t)y * nx;
        for (int c = lane; c < WS; c += 32) {
            int gi = c0 - 5 + c;
            if (gi < 0 || gi >= nx) gi = ghost_map(gi, nx, p.bc[0], p.bc[1]);
            gi = chk(p.ctl, gi, 0, nx);
            T U[4], pr[4], gp[4], gm[4];
#pragma unroll
            for (int k = 0; k < 4; k++) U[k] = row[(size_t)k * sv + gi];
            cell2d<T, 0>(U, gm1, alpha, pr, gp, gm);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                spr[k][c] = pr[k];
                sgp[k][c] = gp[k];
                sgm[k][c] = gm[k];
            }
        }
        __syncwarp();
        const int j = c0 - 2 + lane;
        Face2D<T> F;
        face2d_bits<T, 0>(
            F, [&](int q, int t) { return spr[q][lane + t]; }, [&](int c, int t) { return sgp[c][lane + t]; },
            [&](int c, int t) { return sgm[c][lane + t]; }, gm1, eps, CT, kt);
        const unsigned wl = __shfl_up_sync(0xffffffffu, F.word, 1);
        const unsigned wr = __shfl_down_sync(0xffffffffu, F.word, 1);
        T fh[4];
        int D[8];
        face2d_flux<T, 0>(F, wl, wr, s_coef[warp], fh, D);
        const bool face_out = lane >= 1 && lane <= 30;
        if (p.rhs_mode && p.masks && face_out && j >= -1 && j <= nx - 1) {
#pragma unroll
            for (int sk = 0; sk < 8; sk++)
                p.masks[((size_t)sk * ny + y) * (nx + 1) + (j + 1)] = (uint8_t)D[sk];
        }
        if (F.flag && face_out && j >= -2 && j <= nx)
            latch_error(ctl, (F.flag & (ERR_NONPHYSICAL | ERR_NONFINITE)) | ((F.flag & ERR_NOEXIST) ? ERR_NONFINITE : 0),
                        flat_cell(y, j, nx));
        T fprev[4];
#pragma unroll
        for (int k = 0; k < 4; k++) fprev[k] = __shfl_up_sync(0xffffffffu, fh[k], 1);
        if (lane >= 2 && lane <= 30 && j < nx) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                T r;
                if constexpr (sizeof(T) == 8) {
                    r = (fprev[k] - fh[k]) / p.dx;
                } else {
                    r = (fprev[k] - fh[k]) * (1.f / p.f_dx);
                }
                R[(size_t)k * N + (size_t)y * nx + chk(p.ctl, j, 0, p.nx)] = r;
            }
        }
        __syncwarp();
    }
}

// --------------------------------------------------------------------------
// y sweep + RK stage.  Block (bx, by): columns 32 bx .. 32 bx + 31, cells of
// rows 29 by .. 29 by + 28.  Dynamic shared memory (T):
//   gp, gm, pr  [4][39][33] each; ry [4][29][33]; coef [92]; reductions.
// --------------------------------------------------------------------------
constexpr int YB_COLS = 32, YB_ROWS = WT, YB_STAGE = WS, YB_LD = 33;

template <typename T>
constexpr size_t ysweep_smem_bytes() {
    return sizeof(T) * (3 * 4 * YB_STAGE * YB_LD + 4 * YB_ROWS * YB_LD + 92) + 2 * WPB * sizeof(T);
}

template <typename T, bool HALO>
__global__ void __launch_bounds__(WPB * 32, 1) ysweep2d_kernel(const Stage2D p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    T *s_gp = sm;                                 // [4][39][33]
    T *s_gm = s_gp + 4 * YB_STAGE * YB_LD;        // [4][39][33]
    T *s_pr = s_gm + 4 * YB_STAGE * YB_LD;        // [4][39][33]
    T *s_ry = s_pr + 4 * YB_STAGE * YB_LD;        // [4][29][33]
    T *s_coef = s_ry + 4 * YB_ROWS * YB_LD;       // [92]
    T *s_red = s_coef + 92;                       // [2][WPB]
    auto at = [](T *base, int c, int r, int col) -> T & { return base[(c * YB_STAGE + r) * YB_LD + col]; };

    DevCtl *ctl = p.ctl;
    const bool fixed = p.dt_fixed > 0.0;
    if (!p.rhs_mode && !fixed && !ctl->active) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nx = p.nx, ny = p.ny;
    const size_t N = (size_t)nx * ny;
    const size_t sv = HALO ? p.sv : N, svo = HALO ? p.svo : N;
    const int x0 = blockIdx.x * YB_COLS, r0 = blockIdx.y * YB_ROWS;
    const T alpha = alpha2d_in<T, HALO>(p, ctl, 1);
    const T gamma = pick<T>(p.gamma, p.f_gamma), gm1 = pick<T>(p.gamma - 1.0, p.f_gm1);
    const T eps = pick<T>(p.eps_y, p.f_eps_y), CT = pick<T>(p.CT, p.f_CT);
    const T kt = keep_all_factor(CT);
    const T *Us = static_cast<const T *>(p.Us);
    for (int q = tid; q < 91; q += blockDim.x) s_coef[q] = coef<T>(q);

    // ---- stage rows r0-5 .. r0+33 of columns x0 .. x0+31 (coalesced along x)
    for (int idx = tid; idx < YB_STAGE * YB_COLS; idx += blockDim.x) {
        const int r = idx / YB_COLS, col = idx % YB_COLS, x = x0 + col;
        if (x >= nx) continue;
        int y = r0 - 5 + r;
        y = y_row<HALO>(y, p);
        T U[4], pr[4], gp[4], gm[4];
#pragma unroll
        for (int k = 0; k < 4; k++) U[k] = Us[st_at<HALO>(k, sv, y, nx, chk(p.ctl, x, 0, p.nx))];
        cell2d<T, 1>(U, gm1, alpha, pr, gp, gm);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            at(s_pr, k, r, col) = pr[k];
            at(s_gp, k, r, col) = gp[k];
            at(s_gm, k, r, col) = gm[k];
        }
    }
    __syncthreads();

    // ---- faces down the columns: warp w takes columns w, w+8, w+16, w+24
    for (int col = warp; col < YB_COLS; col += WPB) {
        const int x = x0 + col;
        if (x >= nx) break;
        const int j = r0 - 2 + lane;  // face j+1/2 along y
        Face2D<T> F;
        face2d_bits<T, 1>(
            F, [&](int q, int t) { return at(s_pr, q, lane + t, col); },
            [&](int c, int t) { return at(s_gp, c, lane + t, col); },
            [&](int c, int t) { return at(s_gm, c, lane + t, col); }, gm1, eps, CT, kt);
        const unsigned wl = __shfl_up_sync(0xffffffffu, F.word, 1);
        const unsigned wr = __shfl_down_sync(0xffffffffu, F.word, 1);
        T fh[4];
        int D[8];
        face2d_flux<T, 1>(F, wl, wr, s_coef, fh, D);
        const bool face_out = lane >= 1 && lane <= 30;
        if (p.rhs_mode && p.masks && face_out && j >= -1 && j <= ny - 1) {
            uint8_t *ym = p.masks + (size_t)8 * ny * (nx + 1);
#pragma unroll
            for (int sk = 0; sk < 8; sk++) ym[((size_t)sk * nx + x) * (ny + 1) + (j + 1)] = (uint8_t)D[sk];
        }
        if (F.flag && face_out && j >= -2 && j <= ny)
            latch_error(ctl, (F.flag & (ERR_NONPHYSICAL | ERR_NONFINITE)) | ((F.flag & ERR_NOEXIST) ? ERR_NONFINITE : 0),
                        flat_cell(j, x, nx, ny));
        T fprev[4];
#pragma unroll
        for (int k = 0; k < 4; k++) fprev[k] = __shfl_up_sync(0xffffffffu, fh[k], 1);
        if (lane >= 2 && lane <= 30) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                T r;
                if constexpr (sizeof(T) == 8) {
                    r = (fprev[k] - fh[k]) / p.dy;
                } else {
                    r = (fprev[k] - fh[k]) * (1.f / p.f_dy);
                }
                s_ry[(k * YB_ROWS + (lane - 2)) * YB_LD + col] = r;
            }
        }
    }
    __syncthreads();

    // ---- L = Lx + Ly, RK stage, wavespeeds (row-major, coalesced) -----------
    const T *R = static_cast<const T *>(p.R);
    const T *U0 = static_cast<const T *>(p.U0);
    T *out = static_cast<T *>(p.out);
    T dtT = T(0);
    if (!p.rhs_mode) {
        if constexpr (sizeof(T) == 8) {
            dtT = fixed ? p.dt_fixed : ctl->dt;
        } else {
            dtT = fixed ? p.f_dt_fixed : ctl->dt_f;
        }
    }
    T mx = T(0), my = T(0);
    for (int idx = tid; idx < YB_ROWS * YB_COLS; idx += blockDim.x) {
        const int r = idx / YB_COLS, col = idx % YB_COLS, x = x0 + col, y = r0 + r;
        if (x >= nx || y >= ny) continue;
        const size_t g = (size_t)chk(p.ctl, y, 0, p.ny) * nx + chk(p.ctl, x, 0, p.nx);
        T o[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const T rr = R[(size_t)k * N + g] + s_ry[(k * YB_ROWS + r) * YB_LD + col];
            if (p.rhs_mode) {
                out[(size_t)k * svo + g] = rr;
                continue;
            }
            const T us = Us[(size_t)k * sv + g];
            if (p.stage == 0) {
                o[k] = us + dtT * rr;
            } else if (p.stage == 1) {
                o[k] = T(0.75) * U0[(size_t)k * sv + g] + T(0.25) * (us + dtT * rr);
            } else {
                if constexpr (sizeof(T) == 8) {
                    o[k] = T(1.0 / 3.0) * U0[(size_t)k * sv + g] + T(2.0 / 3.0) * (us + dtT * rr);
                } else {
                    const T u0 = U0[(size_t)k * sv + g];
                    o[k] = fmaf(2.0f / 3.0f, (us + dtT * rr) - u0, u0);
                }
            }
            out[(size_t)k * svo + g] = o[k];
        }
        if (!p.rhs_mode) {
            int wflag = 0;
            T sx, sy;
            wavespeed2d<T>(o, gm1, gamma, sx, sy, &wflag);
            if (wflag) latch_error(ctl, wflag, (int)g);
            mx = fmax(mx, sx);
            my = fmax(my, sy);
        }
    }
    if (!p.rhs_mode) {
        mx = warp_max(mx);
        my = warp_max(my);
        if (lane == 0) {
            s_red[warp] = mx;
            s_red[WPB + warp] = my;
        }
        __syncthreads();
        if (tid == 0) {
            T vx = s_red[0], vy = s_red[WPB];
            for (int w = 1; w < WPB; w++) {
                vx = fmax(vx, s_red[w]);
                vy = fmax(vy, s_red[WPB + w]);
            }
            const int so = (p.stage + 1) % 3;
            atomicMax(&ctl->amax[so][0], (unsigned long long)__double_as_longlong((double)vx));
            atomicMax(&ctl->amax[so][1], (unsigned long long)__double_as_longlong((double)vy));
            finish_launch(ctl, so, (p.stage + 2) % 3, p.stage == 2 && !fixed, p.stage == 2 && !fixed, true,
                          HALO ? p.alpha_rec : nullptr);
        }
    }
}

// alpha (both directions) of a 2D state into ctl->amax[slot][0..1].
template <typename T, bool HALO>
__global__ void __launch_bounds__(256) alpha2d_kernel(const Alpha2D p) {
    __shared__ T s_red[2][8];
    const T *U = static_cast<const T *>(p.U);
    const T gamma = T(p.gamma), gm1 = T(p.gamma - 1.0);
    const size_t N = (size_t)p.nx * p.ny, sv = HALO ? p.stride : N;
    T mx = T(0), my = T(0);
    int flag = 0, first = 0x7fffffff;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        T Uc[4];
#pragma unroll
        for (int k = 0; k < 4; k++) Uc[k] = U[(size_t)k * sv + i];
        int f = 0;
        T sx, sy;
        wavespeed2d<T>(Uc, gm1, gamma, sx, sy, &f);
        if (f) {
            flag |= f;
            first = min(first, (int)i);
        }
        mx = fmax(mx, sx);
        my = fmax(my, sy);
    }
    if (flag) latch_error(p.ctl, flag, first);
    mx = warp_max(mx);
    my = warp_max(my);
    if ((threadIdx.x & 31) == 0) {
        s_red[0][threadIdx.x >> 5] = mx;
        s_red[1][threadIdx.x >> 5] = my;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        T vx = s_red[0][0], vy = s_red[1][0];
        for (int w = 1; w < 8; w++) {
            vx = fmax(vx, s_red[0][w]);
            vy = fmax(vy, s_red[1][w]);
        }
        atomicMax(&p.ctl->amax[p.slot][0], (unsigned long long)__double_as_longlong((double)vx));
        atomicMax(&p.ctl->amax[p.slot][1], (unsigned long long)__double_as_longlong((double)vy));
        finish_launch(p.ctl, p.slot, (p.slot + 1) % 3, false, true, true, HALO ? p.alpha_rec : nullptr);
    }
}

// ==========================================================================
// FP32 2D sweeps with paired splits (the 1D FP32 kernel's design, 4 fields).
// S is the state type: float, or double for the mixed-precision form (FP64
// state and x-part R, exact FP64 flux differences and RK combination).
//
// Per face the split fluxes of the 8 stencil cells are held in registers as
// pairs g[c][t] = (G+_c at cell j-3+t, G-_c at cell j+4-t); the four
// characteristic fields are then processed one at a time -- projection
// P_k[t] = sum_c L_kc g[c][t], cutoff codes, neighbour codes by shuffle,
// Delta, polynomial -- so that only one field's 7 pairs are live at once and
// the kernels fit two CTAs per SM.
// ==========================================================================

// Prims (normal velocity, tangential velocity, H, sqrt(rho)) and split fluxes
// of one cell along DIR, FP32.  Here and in face2d_f32 every rounding is
// written out (__fmaf_rn / __fmul_rn / __fadd_rn: nothing is left for the
// compiler to contract), so the whole-domain and slab instantiations of the
// sweeps, and any later change around them, give the same bits.
template <int DIR>
__device__ __forceinline__ void cell2d_f32(const float U[4], float gm1, float alpha, float pr[4], float gp[4],
                                           float gm[4]) {
    const float ri = rcp_approx(U[0]);
    const float u = __fmul_rn(U[1], ri), v = __fmul_rn(U[2], ri);
    const float p = __fmul_rn(gm1, __fmaf_rn(-0.5f, __fmaf_rn(U[1], u, __fmul_rn(U[2], v)), U[3]));
    const float ep = __fadd_rn(U[3], p);
    float F[4];
    if (DIR == 0) {
        F[0] = U[1];
        F[1] = __fmaf_rn(U[1], u, p);
        F[2] = __fmul_rn(U[2], u);
        F[3] = __fmul_rn(u, ep);
        pr[0] = u;
        pr[1] = v;
    } else {
        F[0] = U[2];
        F[1] = __fmul_rn(U[1], v);
        F[2] = __fmaf_rn(U[2], v, p);
        F[3] = __fmul_rn(v, ep);
        pr[0] = v;
        pr[1] = u;
    }
    pr[2] = __fmul_rn(ep, ri);
    pr[3] = __fmul_rn(U[0], rsqrtf(U[0]));
#pragma unroll
    for (int k = 0; k < 4; k++) {
        gp[k] = 0.5f * fmaf(alpha, U[k], F[k]);
        gm[k] = 0.5f * fmaf(-alpha, U[k], F[k]);
    }
}

// One face along DIR: frame, per-field projection / cutoff / Delta / polynomial,
// back-projection to the physical face flux fh[4].  pr(q, i), gp(c, i),
// gm(c, i) read staged index i (face j+1/2 <-> cells j-3+t at index lane+t).
// codes_p / codes_m receive the four fields' Delta codes (5 bits each).
template <int DIR, typename PR, typename GP, typename GM>
__device__ __forceinline__ void face2d_f32(float fh[4], unsigned &codes_p, unsigned &codes_m, int &flag, PR pr,
                                           GP gp, GM gm, const float (*s_cf)[8], float eps4, float CT, float kt,
                                           float gm1, int lane) {
    const float unl = pr(0, lane + 3), unr = pr(0, lane + 4), vtl = pr(1, lane + 3), vtr = pr(1, lane + 4);
    const float Hl = pr(2, lane + 3), Hr = pr(2, lane + 4), sl = pr(3, lane + 3), sr = pr(3, lane + 4);
    const float w = rcp_approx(__fadd_rn(sl, sr));
    const float un = __fmul_rn(__fmaf_rn(sl, unl, __fmul_rn(sr, unr)), w);
    const float vt = __fmul_rn(__fmaf_rn(sl, vtl, __fmul_rn(sr, vtr)), w);
    const float Ht = __fmul_rn(__fmaf_rn(sl, Hl, __fmul_rn(sr, Hr)), w);
    const float q2 = __fmul_rn(0.5f, __fmaf_rn(un, un, __fmul_rn(vt, vt)));
    const float c2 = __fmul_rn(gm1, __fadd_rn(Ht, -q2));
    const float rc = rsqrtf(c2);
    const float c = __fmul_rn(c2, rc);
    const float b1 = __fmul_rn(gm1, __fmul_rn(rc, rc)), b2 = __fmul_rn(q2, b1);
    if (!(c2 > 0.f)) flag |= isfinite(c2) ? ERR_NONPHYSICAL : ERR_NONFINITE;
    // rows of L in the rotated component order (rho, normal, tangential, E);
    // row 2 (shear) is (-vt, 0, 1, 0)
    const float b1u = __fmul_rn(b1, un), l02 = __fmul_rn(-0.5f, __fmul_rn(b1, vt)), l03 = __fmul_rn(0.5f, b1);
    const float L0[4] = {__fmul_rn(0.5f, __fmaf_rn(un, rc, b2)), __fmul_rn(-0.5f, __fadd_rn(b1u, rc)), l02, l03};
    const float L1[4] = {__fadd_rn(1.f, -b2), b1u, __fmul_rn(b1, vt), -b1};
    const float L3[4] = {__fmul_rn(0.5f, __fmaf_rn(-un, rc, b2)), __fmul_rn(-0.5f, __fadd_rn(b1u, -rc)), l02, l03};
    constexpr int CN = rot<DIR>(1), CT_ = rot<DIR>(2);  // physical index of the normal / tangential momentum
    float2 g[4][7];
#pragma unroll
    for (int t = 0; t < 7; t++)
#pragma unroll
        for (int cc = 0; cc < 4; cc++) g[cc][t] = make_float2(gp(cc, lane + t), gm(cc, lane + 7 - t));
    float f[4];
    codes_p = 0;
    codes_m = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        float2 P[7];
        if (k == 2) {
#pragma unroll
            for (int t = 0; t < 7; t++) P[t] = __ffma2_rn(f2(-vt), g[0][t], g[CT_][t]);
        } else {
            const float *Lk = k == 0 ? L0 : (k == 1 ? L1 : L3);
            // Lk is in rotated order: physical component cc takes Lk[rot(cc)]
            const float2 l0 = f2(Lk[0]), ln = f2(Lk[1]), lt = f2(Lk[2]), le = f2(Lk[3]);
#pragma unroll
            for (int t = 0; t < 7; t++) {
                float2 q = __fmul2_rn(l0, g[0][t]);
                q = __ffma2_rn(ln, g[CN][t], q);
                q = __ffma2_rn(lt, g[CT_][t], q);
                P[t] = __ffma2_rn(le, g[3][t], q);
            }
        }
        unsigned cp, cm;
        cutoff2(P[1], P[2], P[3], P[4], P[5], eps4, CT, kt, cp, cm);
        const unsigned word = (cp << 1) | (cm << 6);
        const unsigned wl = __shfl_up_sync(0xffffffffu, word, 1);
        const unsigned wr = __shfl_down_sync(0xffffffffu, word, 1);
        const unsigned dp = ((wl << 1) & 0x10u) | (word & 0x0Eu) | ((wr >> 1) & 0x01u);
        const unsigned dm = (((wr << 1) & 0x200u) | (word & 0x1C0u) | ((wl >> 1) & 0x20u)) >> 5;
        codes_p |= dp << (5 * k);
        codes_m |= dm << (5 * k);
        float2 s;
        if (dp == 31u && dm == 31u) {
            s = __fmul2_rn(f2(-1.f / 140.f), P[0]);
            s = __ffma2_rn(f2(5.f / 84.f), P[1], s);
            s = __ffma2_rn(f2(-101.f / 420.f), P[2], s);
            s = __ffma2_rn(f2(319.f / 420.f), P[3], s);
            s = __ffma2_rn(f2(107.f / 210.f), P[4], s);
            s = __ffma2_rn(f2(-19.f / 210.f), P[5], s);
            s = __ffma2_rn(f2(1.f / 105.f), P[6], s);
        } else {
            const float *cpp = s_cf[dp];
            const float *cmm = s_cf[dm];
            s = __fmul2_rn(make_float2(cpp[0], cmm[0]), P[0]);
#pragma unroll
            for (int t = 1; t < 7; t++) s = __ffma2_rn(make_float2(cpp[t], cmm[t]), P[t], s);
        }
        f[k] = __fadd_rn(s.x, s.y);
    }
    // back-projection: rotated rows (rho, normal, tangential, E) of R
    const float Fr0 = __fadd_rn(__fadd_rn(f[0], f[1]), f[3]);
    const float Fr1 = __fmaf_rn(__fadd_rn(un, c), f[3], __fmaf_rn(__fadd_rn(un, -c), f[0], __fmul_rn(un, f[1])));
    const float Fr2 = __fmaf_rn(vt, Fr0, f[2]);
    const float hm = __fmaf_rn(-un, c, Ht), hp = __fmaf_rn(un, c, Ht);
    const float Fr3 = __fmaf_rn(hp, f[3], __fmaf_rn(vt, f[2], __fmaf_rn(q2, f[1], __fmul_rn(hm, f[0]))));
    fh[0] = Fr0;
    fh[CN] = Fr1;
    fh[CT_] = Fr2;
    fh[3] = Fr3;
}

template <typename S, bool HALO>
__global__ void __launch_bounds__(WPB * 32, 2) xsweep2d_f32_kernel(const Stage2D p) {
    constexpr bool MIXED = sizeof(S) == 8;
    __shared__ float s_gp[WPB][4][WC];
    __shared__ float s_gm[WPB][4][WC];
    __shared__ float s_pr[WPB][4][WC];
    __shared__ __align__(16) float s_cf[32][8];
    DevCtl *ctl = p.ctl;
    const bool fixed = p.dt_fixed > 0.0;
    if (!p.rhs_mode && !fixed && !ctl->active) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    fill_delta_table(s_cf);
    const float alpha = alpha2d_in<float, HALO>(p, ctl, 0);
    const float gm1 = p.f_gm1, eps4 = 4.f * p.f_eps_x, CT = p.f_CT;
    const float kt = keep_all_factor(CT);
    const float idx = 1.f / p.f_dx;
    const double idxD = 1.0 / p.dx;
    const S *Us = static_cast<const S *>(p.Us);
    S *R = static_cast<S *>(p.R);
    const int nx = p.nx, ny = p.ny;
    const size_t N = (size_t)nx * ny;
    const size_t sv = HALO ? p.sv : N;
    const int ntx = (nx + WT - 1) / WT;
    const long ntiles = (long)ntx * ny;
    float (*sgp)[WC] = s_gp[warp];
    float (*sgm)[WC] = s_gm[warp];
    float (*spr)[WC] = s_pr[warp];
    __syncthreads();
    // one tile ahead, held in the state type and rounded to float only when
    // the tile is used (a mixed-precision load is then not waited for at once)
    S ua[4], ub[4];
    auto load_tile = [&](int y, int tx) {
        const int c0 = tx * WT;
        const S *row = Us + (size_t)y * nx;
        int ga = c0 - 5 + lane, gb = c0 - 5 + 32 + lane;
        if (ga < 0 || ga >= nx) ga = ghost_map(ga, nx, p.bc[0], p.bc[1]);
        if (gb < 0 || gb >= nx) gb = ghost_map(gb, nx, p.bc[0], p.bc[1]);
        ga = chk(p.ctl, ga, 0, nx);
        gb = chk(p.ctl, gb, 0, nx);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            ua[k] = row[(size_t)k * sv + ga];
            ub[k] = (lane < WS - 32) ? row[(size_t)k * sv + gb] : S(0);
        }
    };
    // the warp's tiles as row and tile column, stepped instead of divided out
    // of a tile index every tile (as in the paired x sweep)
    const long tstride = (long)gridDim.x * WPB, tile0 = (long)blockIdx.x * WPB + warp;
    const int step_y = (int)(tstride / ntx), step_x = (int)(tstride % ntx);
    auto next = [&](int &ty, int &tx) {
        ty += step_y;
        tx += step_x;
        if (tx >= ntx) {
            tx -= ntx;
            ty += 1;
        }
    };
    int ty = tile0 < ntiles ? (int)(tile0 / ntx) : ny, tx = tile0 < ntiles ? (int)(tile0 % ntx) : 0;
    if (ty < ny) load_tile(ty, tx);
    for (; ty < ny; next(ty, tx)) {
        const int y = ty;
        const int c0 = tx * WT;
        float cur[2][4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            cur[0][k] = to_f32(ua[k]);
            cur[1][k] = to_f32(ub[k]);
        }
        {
            int ty1 = ty, tx1 = tx;
            next(ty1, tx1);
            if (ty1 < ny) load_tile(ty1, tx1);
        }
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const int c = lane + 32 * r;
            if (c >= WS) break;
            float pr[4], gp[4], gm[4];
            cell2d_f32<0>(cur[r], gm1, alpha, pr, gp, gm);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                spr[k][c] = pr[k];
                sgp[k][c] = gp[k];
                sgm[k][c] = gm[k];
            }
        }
        __syncwarp();
        const int j = c0 - 2 + lane;
        float fh[4];
        unsigned cpk, cmk;
        int flag = 0;
        face2d_f32<0>(
            fh, cpk, cmk, flag, [&](int q, int i) { return spr[q][i]; }, [&](int cc, int i) { return sgp[cc][i]; },
            [&](int cc, int i) { return sgm[cc][i]; }, s_cf, eps4, CT, kt, gm1, lane);
        const bool face_out = lane >= 1 && lane <= 30;
        if (p.rhs_mode && p.masks && face_out && j >= -1 && j <= nx - 1) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                p.masks[((size_t)k * ny + y) * (nx + 1) + (j + 1)] = (uint8_t)((cpk >> (5 * k)) & 31u);
                p.masks[((size_t)(4 + k) * ny + y) * (nx + 1) + (j + 1)] = (uint8_t)((cmk >> (5 * k)) & 31u);
            }
        }
        if (flag && face_out && j >= -2 && j <= nx) latch_error(ctl, flag, flat_cell(y, j, nx));
        float fprev[4];
#pragma unroll
        for (int k = 0; k < 4; k++) fprev[k] = __shfl_up_sync(0xffffffffu, fh[k], 1);
        if (lane >= 2 && lane <= 30 && j < nx) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if constexpr (MIXED)
                    R[(size_t)k * N + (size_t)y * nx + chk(p.ctl, j, 0, p.nx)] = (to_f64(fprev[k]) - to_f64(fh[k])) * idxD;
                else
                    R[(size_t)k * N + (size_t)y * nx + chk(p.ctl, j, 0, p.nx)] = (fprev[k] - fh[k]) * idx;
            }
        }
        __syncwarp();
    }
}

template <typename S>
constexpr size_t ysweep_f32_smem_bytes() {
    return sizeof(float) * (3 * 4 * YB_STAGE * YB_LD) + sizeof(S) * (4 * YB_ROWS * YB_LD) +
           sizeof(float) * (32 * 8 + 2 * WPB);
}

template <typename S, bool HALO>
__global__ void __launch_bounds__(WPB * 32, 2) ysweep2d_f32_kernel(const Stage2D p) {
    constexpr bool MIXED = sizeof(S) == 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S *s_ry = reinterpret_cast<S *>(smem_raw);                                    // [4][29][33]
    float *s_gp = reinterpret_cast<float *>(smem_raw + sizeof(S) * 4 * YB_ROWS * YB_LD);  // [4][39][33]
    float *s_gm = s_gp + 4 * YB_STAGE * YB_LD;
    float *s_pr = s_gm + 4 * YB_STAGE * YB_LD;
    float(*s_cf)[8] = reinterpret_cast<float(*)[8]>(s_pr + 4 * YB_STAGE * YB_LD);  // [32][8]
    float *s_red = reinterpret_cast<float *>(s_cf + 32);                           // [2][WPB]
    auto at = [](const float *base, int c, int r, int col) -> float {
        return base[(c * YB_STAGE + r) * YB_LD + col];
    };

    DevCtl *ctl = p.ctl;
    const bool fixed = p.dt_fixed > 0.0;
    if (!p.rhs_mode && !fixed && !ctl->active) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nx = p.nx, ny = p.ny;
    const size_t N = (size_t)nx * ny;
    const size_t sv = HALO ? p.sv : N, svo = HALO ? p.svo : N;
    const int x0 = blockIdx.x * YB_COLS, r0 = blockIdx.y * YB_ROWS;
    const float alpha = alpha2d_in<float, HALO>(p, ctl, 1);
    const float gamma = p.f_gamma, gm1 = p.f_gm1, eps4 = 4.f * p.f_eps_y, CT = p.f_CT;
    const float kt = keep_all_factor(CT);
    const S *Us = static_cast<const S *>(p.Us);
    fill_delta_table(s_cf);

    // ---- stage rows r0-5 .. r0+33 of columns x0 .. x0+31 (coalesced along x);
    // all of a thread's loads are issued before any is used
    // (in the state type: a mixed-precision value is rounded to float only
    // when it is used)
    constexpr int NSTG = (YB_STAGE * YB_COLS + WPB * 32 - 1) / (WPB * 32);
    S Ust[NSTG][4];
#pragma unroll
    for (int sI = 0; sI < NSTG; sI++) {
        const int q = tid + sI * WPB * 32;
        const int r = q / YB_COLS, x = x0 + q % YB_COLS;
        if (q < YB_STAGE * YB_COLS && x < nx) {
            int y = r0 - 5 + r;
            y = y_row<HALO>(y, p);
#pragma unroll
            for (int k = 0; k < 4; k++) Ust[sI][k] = Us[st_at<HALO>(k, sv, y, nx, chk(p.ctl, x, 0, p.nx))];
        }
    }
#pragma unroll
    for (int sI = 0; sI < NSTG; sI++) {
        const int q = tid + sI * WPB * 32;
        const int r = q / YB_COLS, col = q % YB_COLS;
        if (q < YB_STAGE * YB_COLS && x0 + col < nx) {
            float uf[4], pr[4], gp[4], gm[4];
#pragma unroll
            for (int k = 0; k < 4; k++) uf[k] = to_f32(Ust[sI][k]);
            cell2d_f32<1>(uf, gm1, alpha, pr, gp, gm);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                s_pr[(k * YB_STAGE + r) * YB_LD + col] = pr[k];
                s_gp[(k * YB_STAGE + r) * YB_LD + col] = gp[k];
                s_gm[(k * YB_STAGE + r) * YB_LD + col] = gm[k];
            }
        }
    }
    __syncthreads();

    // ---- faces down the columns: warp w takes columns w, w+8, w+16, w+24
    const float idy = 1.f / p.f_dy;
    const double idyD = 1.0 / p.dy;
    for (int col = warp; col < YB_COLS; col += WPB) {
        const int x = x0 + col;
        if (x >= nx) break;
        const int j = r0 - 2 + lane;
        float fh[4];
        unsigned cpk, cmk;
        int flag = 0;
        face2d_f32<1>(
            fh, cpk, cmk, flag, [&](int q, int i) { return at(s_pr, q, i, col); },
            [&](int cc, int i) { return at(s_gp, cc, i, col); }, [&](int cc, int i) { return at(s_gm, cc, i, col); },
            s_cf, eps4, CT, kt, gm1, lane);
        const bool face_out = lane >= 1 && lane <= 30;
        if (p.rhs_mode && p.masks && face_out && j >= -1 && j <= ny - 1) {
            uint8_t *ym = p.masks + (size_t)8 * ny * (nx + 1);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                ym[((size_t)k * nx + x) * (ny + 1) + (j + 1)] = (uint8_t)((cpk >> (5 * k)) & 31u);
                ym[((size_t)(4 + k) * nx + x) * (ny + 1) + (j + 1)] = (uint8_t)((cmk >> (5 * k)) & 31u);
            }
        }
        if (flag && face_out && j >= -2 && j <= ny) latch_error(ctl, flag, flat_cell(j, x, nx, ny));
        float fprev[4];
#pragma unroll
        for (int k = 0; k < 4; k++) fprev[k] = __shfl_up_sync(0xffffffffu, fh[k], 1);
        if (lane >= 2 && lane <= 30) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if constexpr (MIXED)
                    s_ry[(k * YB_ROWS + (lane - 2)) * YB_LD + col] = (to_f64(fprev[k]) - to_f64(fh[k])) * idyD;
                else
                    s_ry[(k * YB_ROWS + (lane - 2)) * YB_LD + col] = (fprev[k] - fh[k]) * idy;
            }
        }
    }
    __syncthreads();

    // ---- L = Lx + Ly, RK stage, wavespeeds (row-major, coalesced) -----------
    const S *R = static_cast<const S *>(p.R);
    const S *U0 = static_cast<const S *>(p.U0);
    S *out = static_cast<S *>(p.out);
    const float dtF = p.rhs_mode ? 0.f : (fixed ? p.f_dt_fixed : ctl->dt_f);
    const double dtD = p.rhs_mode ? 0.0 : (fixed ? p.dt_fixed : ctl->dt);
    float mx = 0.f, my = 0.f;
    // EB cells per thread at a time, their loads issued before any is used
    constexpr int EB = MIXED ? 2 : 4;
    const bool use_u0 = !p.rhs_mode && p.stage > 0;
    for (int q0 = tid; q0 < YB_ROWS * YB_COLS; q0 += EB * WPB * 32) {
        S Rv[EB][4], Uv[EB][4], U0v[EB][4];
#pragma unroll
        for (int e = 0; e < EB; e++) {
            const int q = q0 + e * WPB * 32;
            const int r = q / YB_COLS, x = x0 + q % YB_COLS, y = r0 + r;
            if (q < YB_ROWS * YB_COLS && x < nx && y < ny) {
                const size_t gi = (size_t)chk(p.ctl, y, 0, p.ny) * nx + chk(p.ctl, x, 0, p.nx);
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    Rv[e][k] = R[(size_t)k * N + gi];
                    Uv[e][k] = p.rhs_mode ? S(0) : Us[(size_t)k * sv + gi];
                    U0v[e][k] = use_u0 ? U0[(size_t)k * sv + gi] : S(0);
                }
            }
        }
#pragma unroll
        for (int e = 0; e < EB; e++) {
            const int q = q0 + e * WPB * 32;
            const int r = q / YB_COLS, col = q % YB_COLS, x = x0 + col, y = r0 + r;
            if (!(q < YB_ROWS * YB_COLS && x < nx && y < ny)) continue;
            const size_t gi = (size_t)chk(p.ctl, y, 0, p.ny) * nx + chk(p.ctl, x, 0, p.nx);
            float of[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const S rr = Rv[e][k] + s_ry[(k * YB_ROWS + r) * YB_LD + col];
                if (p.rhs_mode) {
                    out[(size_t)k * svo + gi] = rr;
                    continue;
                }
                S o;
                if constexpr (MIXED) {
                    const double v = fma(dtD, (double)rr, (double)Uv[e][k]);
                    if (p.stage == 0)
                        o = v;
                    else if (p.stage == 1)
                        o = fma(0.75, (double)U0v[e][k], 0.25 * v);
                    else
                        o = fma(2.0 / 3.0, v, (1.0 / 3.0) * (double)U0v[e][k]);
                } else {
                    const float v = fmaf(dtF, (float)rr, (float)Uv[e][k]);
                    if (p.stage == 0) {
                        o = v;
                    } else if (p.stage == 1) {
                        o = fmaf(0.75f, (float)U0v[e][k], 0.25f * v);
                    } else {
                        const float u0 = (float)U0v[e][k];
                        o = fmaf(2.0f / 3.0f, v - u0, u0);
                    }
                }
                out[(size_t)k * svo + gi] = o;
                of[k] = to_f32(o);
            }
            if (!p.rhs_mode) {
                int wflag = 0;
                float sx, sy;
                wavespeed2d<float>(of, gm1, gamma, sx, sy, &wflag);
                if (wflag) latch_error(ctl, wflag, (int)gi);
                mx = fmaxf(mx, sx);
                my = fmaxf(my, sy);
            }
        }
    }
    if (!p.rhs_mode) {
        mx = warp_max(mx);
        my = warp_max(my);
        if (lane == 0) {
            s_red[warp] = mx;
            s_red[WPB + warp] = my;
        }
        __syncthreads();
        if (tid == 0) {
            float vx = s_red[0], vy = s_red[WPB];
            for (int w = 1; w < WPB; w++) {
                vx = fmaxf(vx, s_red[w]);
                vy = fmaxf(vy, s_red[WPB + w]);
            }
            const int so = (p.stage + 1) % 3;
            atomicMax(&ctl->amax[so][0], (unsigned long long)__double_as_longlong((double)vx));
            atomicMax(&ctl->amax[so][1], (unsigned long long)__double_as_longlong((double)vy));
            finish_launch(ctl, so, (p.stage + 2) % 3, p.stage == 2 && !fixed, p.stage == 2 && !fixed, true,
                          HALO ? p.alpha_rec : nullptr);
        }
    }
}

// --------------------------------------------------------------------------
// FP32 y sweep, persistent: each CTA walks blocks b = blockIdx.x, + gridDim.x,
// ... (32 columns x 29 rows, as ysweep2d_f32_kernel), and the raw state of
// its next block is copied into shared memory by cp.async while the current
// block's faces and epilogue compute, so the staging loads are not waited for
// in the block's critical path.  The per-cell and per-face arithmetic is that
// of ysweep2d_f32_kernel, so the results are the same bits.
// Dynamic shared memory: ry [4][29][33]; gp, gm, pr [4][39][33]; raw
// [4][39][32]; Delta table [32][8]; reductions [2][WPB].
// --------------------------------------------------------------------------
// (cp_async4, cp_async_commit, cp_async_wait_all: teno7_kernels.cuh)

// ==========================================================================
// FP32 2D faces in PAIRS (the 1D face-paired kernel's design, 4 fields): every
// float2 holds (face A, face B), the two splits run one after the other, and
// the fields go in two groups -- fields 0, 1, 3, which read all four
// components, and the shear field 2, which reads two -- so that one group's
// projections (7 pairs per field) are live at a time.  Every per-face
// operation is the one face2d_f32 performs, in the same order, so the results
// are the same bits.
//   pr(q, i)     primitive q of staged index i, as the pair (face A's cell,
//                face B's cell); cell j-3+t of face j+1/2 is staged index lane+t
//   gs(s, c, i)  split s (0: '+', 1: '-') of physical component c, likewise
//   WRAP         true: faces A and B of lane l are c0-2+l and c0+30+l of one
//                row, so face A of lane 31 and face B of lane 0 are
//                neighbours (the x sweep); false: A and B lie in two columns
// D[s][g] receives the Delta words of split s and field group g (A slots from
// bit 0, B slots SH bits higher, 5 bits per field, as in the 1D kernel).
// ==========================================================================
template <int G>
__device__ __forceinline__ unsigned pair_delta(unsigned word, int s, int lane, bool wrap) {
    constexpr int SH = 5 * G;
    constexpr unsigned MASK_A = (1u << SH) - 1u;
    const unsigned wl = __shfl_sync(0xffffffffu, word, (lane + 31) & 31);
    const unsigned wr = __shfl_sync(0xffffffffu, word, (lane + 1) & 31);
    // codes of each face's left and right neighbour faces, in its own slots
    const unsigned LW = (wrap && lane == 0) ? (wl & MASK_A) | (wl << SH) : wl;
    const unsigned RW = (wrap && lane == 31) ? (wr >> SH) | (wr & ~MASK_A) : wr;
    return s == 0 ? (((LW << 1) & SLOT_HI) | (word & SLOT_MID) | ((RW >> 1) & SLOT_LO))
                  : (((RW << 1) & SLOT_HI) | (word & SLOT_MID) | ((LW >> 1) & SLOT_LO));
}

// Table co2 polynomial of one field of both faces: the all-kept row as
// constants, any other row from the Delta-indexed table.
__device__ __forceinline__ float2 pair_poly(const float2 P[7], unsigned codeA, unsigned codeB,
                                            const float (*s_cf)[8]) {
    float2 v;
    if (codeA == 31u && codeB == 31u) {
        v = __fmul2_rn(f2(-1.f / 140.f), P[0]);
        v = __ffma2_rn(f2(5.f / 84.f), P[1], v);
        v = __ffma2_rn(f2(-101.f / 420.f), P[2], v);
        v = __ffma2_rn(f2(319.f / 420.f), P[3], v);
        v = __ffma2_rn(f2(107.f / 210.f), P[4], v);
        v = __ffma2_rn(f2(-19.f / 210.f), P[5], v);
        v = __ffma2_rn(f2(1.f / 105.f), P[6], v);
    } else {
        const float *cA = s_cf[codeA];
        const float *cB = s_cf[codeB];
        v = __fmul2_rn(make_float2(cA[0], cB[0]), P[0]);
#pragma unroll
        for (int t = 1; t < 7; t++) v = __ffma2_rn(make_float2(cA[t], cB[t]), P[t], v);
    }
    return v;
}

template <int DIR, bool WRAP, typename PR, typename GS>
__device__ __forceinline__ void face2d_pair(float2 fh[4], unsigned (&D)[2][2], int &flagA, int &flagB, PR pr,
                                            GS gs, const float (*s_cf)[8], float eps4, float CT, float kt,
                                            float gm1, int lane) {
    // ---- Roe frames of both faces (face2d_f32's roundings, packed)
    const float2 unl = pr(0, lane + 3), unr = pr(0, lane + 4), vtl = pr(1, lane + 3), vtr = pr(1, lane + 4);
    const float2 Hl = pr(2, lane + 3), Hr = pr(2, lane + 4), sl = pr(3, lane + 3), sr = pr(3, lane + 4);
    const float2 ssum = __fadd2_rn(sl, sr);
    const float2 w = make_float2(rcp_approx(ssum.x), rcp_approx(ssum.y));
    const float2 un = __fmul2_rn(__ffma2_rn(sl, unl, __fmul2_rn(sr, unr)), w);
    const float2 vt = __fmul2_rn(__ffma2_rn(sl, vtl, __fmul2_rn(sr, vtr)), w);
    const float2 Ht = __fmul2_rn(__ffma2_rn(sl, Hl, __fmul2_rn(sr, Hr)), w);
    const float2 q2 = __fmul2_rn(f2(0.5f), __ffma2_rn(un, un, __fmul2_rn(vt, vt)));
    const float2 c2 = __fmul2_rn(f2(gm1), __fadd2_rn(Ht, f2neg(q2)));
    const float2 rc = make_float2(rsqrtf(c2.x), rsqrtf(c2.y));
    if (!(c2.x > 0.f)) flagA |= isfinite(c2.x) ? ERR_NONPHYSICAL : ERR_NONFINITE;
    if (!(c2.y > 0.f)) flagB |= isfinite(c2.y) ? ERR_NONPHYSICAL : ERR_NONFINITE;
    // only un, vt, Ht, q2 and 1/c stay live through the splits: b1, b2 and c
    // are formed again where they are used (the same operations, the same bits)
    constexpr int CN = rot<DIR>(1), CT_ = rot<DIR>(2);  // physical index of the normal / tangential momentum
    float2 f[4];
#pragma unroll
    for (int s = 0; s < 2; s++) {
        // ---- fields 0, 1, 3
        {
            // rows of L of fields 0, 1, 3 in the rotated component order (rho,
            // normal, tangential, E), formed per split so that they are live
            // only here; field 2 (shear) is (-vt, 0, 1, 0)
            const float2 b1 = __fmul2_rn(f2(gm1), __fmul2_rn(rc, rc)), b2 = __fmul2_rn(q2, b1);
            const float2 b1u = __fmul2_rn(b1, un), l02 = __fmul2_rn(f2(-0.5f), __fmul2_rn(b1, vt));
            const float2 l03 = __fmul2_rn(f2(0.5f), b1);
            const float2 L[3][4] = {
                {__fmul2_rn(f2(0.5f), __ffma2_rn(un, rc, b2)), __fmul2_rn(f2(-0.5f), __fadd2_rn(b1u, rc)), l02, l03},
                {__fadd2_rn(f2(1.f), f2neg(b2)), b1u, __fmul2_rn(b1, vt), f2neg(b1)},
                {__fmul2_rn(f2(0.5f), __ffma2_rn(f2neg(un), rc, b2)),
                 __fmul2_rn(f2(-0.5f), __fadd2_rn(b1u, f2neg(rc))), l02, l03}};
            float2 P[3][7];
#pragma unroll
            for (int t = 0; t < 7; t++) {
                const int i = s == 0 ? lane + t : lane + 7 - t;
                const float2 g0 = gs(s, 0, i), gn = gs(s, CN, i), gt = gs(s, CT_, i), ge = gs(s, 3, i);
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    float2 q = __fmul2_rn(L[k][0], g0);
                    q = __ffma2_rn(L[k][1], gn, q);
                    q = __ffma2_rn(L[k][2], gt, q);
                    P[k][t] = __ffma2_rn(L[k][3], ge, q);
                }
            }
            bool keep_all = true;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float2 tau = tau_pair(P[k][1], P[k][2], P[k][3], P[k][4], P[k][5]);
                keep_all = keep_all && tau.x < kt * eps4 && tau.y < kt * eps4;
            }
            unsigned word = 0;
            if (keep_all) {
                word = (7u << 1) | (7u << 6) | (7u << 11) | (7u << 16) | (7u << 21) | (7u << 26);
            } else {
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    unsigned cA, cB;
                    cutoff2(P[k][1], P[k][2], P[k][3], P[k][4], P[k][5], eps4, CT, kt, cA, cB);
                    word |= (cA << (5 * k + 1)) | (cB << (15 + 5 * k + 1));
                }
            }
            const unsigned Dw = pair_delta<3>(word, s, lane, WRAP);
            D[s][0] = Dw;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float2 v = pair_poly(P[k], (Dw >> (5 * k)) & 31u, (Dw >> (15 + 5 * k)) & 31u, s_cf);
                const int fk = k == 2 ? 3 : k;
                f[fk] = s == 0 ? v : __fadd2_rn(f[fk], v);
            }
        }
        // ---- field 2 (shear)
        {
            float2 P[7];
#pragma unroll
            for (int t = 0; t < 7; t++) {
                const int i = s == 0 ? lane + t : lane + 7 - t;
                P[t] = __ffma2_rn(f2neg(vt), gs(s, 0, i), gs(s, CT_, i));
            }
            unsigned cA, cB;
            cutoff2(P[1], P[2], P[3], P[4], P[5], eps4, CT, kt, cA, cB);
            const unsigned Dw = pair_delta<1>((cA << 1) | (cB << 6), s, lane, WRAP);
            D[s][1] = Dw;
            const float2 v = pair_poly(P, Dw & 31u, (Dw >> 5) & 31u, s_cf);
            f[2] = s == 0 ? v : __fadd2_rn(f[2], v);
        }
    }
    // ---- back projection: rotated rows (rho, normal, tangential, E) of R
    const float2 c = __fmul2_rn(__fmul2_rn(f2(gm1), __fadd2_rn(Ht, f2neg(q2))), rc);
    const float2 Fr0 = __fadd2_rn(__fadd2_rn(f[0], f[1]), f[3]);
    const float2 Fr1 = __ffma2_rn(__fadd2_rn(un, c), f[3], __ffma2_rn(__fadd2_rn(un, f2neg(c)), f[0], __fmul2_rn(un, f[1])));
    const float2 Fr2 = __ffma2_rn(vt, Fr0, f[2]);
    const float2 hm = __ffma2_rn(f2neg(un), c, Ht), hp = __ffma2_rn(un, c, Ht);
    const float2 Fr3 =
        __ffma2_rn(hp, f[3], __ffma2_rn(vt, f[2], __ffma2_rn(q2, f[1], __fmul2_rn(hm, f[0]))));
    fh[0] = Fr0;
    fh[CN] = Fr1;
    fh[CT_] = Fr2;
    fh[3] = Fr3;
}

// Delta code (5 bits) of split s, field k of face h (0: A, 1: B) from face2d_pair's words.
__device__ __forceinline__ unsigned pair_code(const unsigned (&D)[2][2], int s, int k, int h) {
    const int g = k == 2 ? 1 : 0, slot = k == 3 ? 2 : (k == 2 ? 0 : k), SH = g == 0 ? 15 : 5;
    return (D[s][g] >> (5 * slot + (h ? SH : 0))) & 31u;
}

// --------------------------------------------------------------------------
// FP32 x sweep with paired faces: R = Lx(U).  Warp tile = WT2 = 61 cells of a
// row (cells c0 .. c0+60); lane l owns faces c0-2+l (A) and c0+30+l (B); the
// 71 cells c0-5 .. c0+65 are staged as pairs (cell i, cell i + 32), one tile
// ahead in registers.  FP32 state only.
// --------------------------------------------------------------------------
template <bool HALO>
__global__ void __launch_bounds__(WPB * 32, 2) xsweep2d_f32fp_kernel(const Stage2D p) {
    __shared__ float2 s_pr[WPB][4][WP2];
    __shared__ float2 s_gp[WPB][4][WP2];
    __shared__ float2 s_gm[WPB][4][WP2];
    __shared__ float s_raw[WPB][4][3 * 32];  // raw state of the next tile (cp.async)
    __shared__ __align__(16) float s_cf[32][8];
    DevCtl *ctl = p.ctl;
    const bool fixed = p.dt_fixed > 0.0;
    if (!p.rhs_mode && !fixed && !ctl->active) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    fill_delta_table(s_cf);
    const float alpha = alpha2d_in<float, HALO>(p, ctl, 0);
    const float gm1 = p.f_gm1, eps4 = 4.f * p.f_eps_x, CT = p.f_CT;
    const float kt = keep_all_factor(CT);
    const float idx = 1.f / p.f_dx;
    const float *Us = static_cast<const float *>(p.Us);
    float *R = static_cast<float *>(p.R);
    const int nx = p.nx, ny = p.ny;
    const size_t N = (size_t)nx * ny;
    const size_t sv = HALO ? p.sv : N;
    const int ntx = (nx + WT2 - 1) / WT2;
    const long ntiles = (long)ntx * ny;
    float2 (*spr)[WP2] = s_pr[warp];
    float2 (*sgp)[WP2] = s_gp[warp];
    float2 (*sgm)[WP2] = s_gm[warp];
    float (*sraw)[3 * 32] = s_raw[warp];
    __syncthreads();
    // raw state of the staged cells of a tile (rounds r = 0, 1, 2: cells
    // c0-5+32r+lane) into sraw by asynchronous copies, one tile ahead
    auto copy_tile = [&](int y, int tx) {
        const int c0 = tx * WT2;
        const float *row = Us + (size_t)y * nx;
        const bool inside = c0 >= 5 && c0 + WS2 - 5 <= nx;  // every staged cell in the row (warp-uniform)
#pragma unroll
        for (int r = 0; r < 3; r++) {
            if (lane + 32 * r >= WS2) break;
            int g = c0 - 5 + 32 * r + lane;
            if (!inside && (g < 0 || g >= nx)) g = ghost_map(g, nx, p.bc[0], p.bc[1]);
            g = chk(p.ctl, g, 0, nx);
#pragma unroll
            for (int k = 0; k < 4; k++) cp_async4(&sraw[k][32 * r + lane], &row[(size_t)k * sv + g]);
        }
        cp_async_commit();
    };
    // the warp's tiles (row-major, grid-stride) as row and tile column,
    // stepped by the stride's rows and columns instead of divided out of a
    // tile index every tile
    const long tstride = (long)gridDim.x * WPB, tile0 = (long)blockIdx.x * WPB + warp;
    const int step_y = (int)(tstride / ntx), step_x = (int)(tstride % ntx);
    auto next = [&](int &ty, int &tx) {
        ty += step_y;
        tx += step_x;
        if (tx >= ntx) {
            tx -= ntx;
            ty += 1;
        }
    };
    int ty = tile0 < ntiles ? (int)(tile0 / ntx) : ny, tx = tile0 < ntiles ? (int)(tile0 % ntx) : 0;
    if (ty < ny) copy_tile(ty, tx);
    for (; ty < ny; next(ty, tx)) {
        const int y = ty;
        const int c0 = tx * WT2;
        cp_async_wait_all();
        __syncwarp();
        float cur[3][4];
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int k = 0; k < 4; k++) cur[r][k] = (lane + 32 * r < WS2) ? sraw[k][32 * r + lane] : 0.f;
        __syncwarp();  // every lane has read sraw before the next tile's copies land in it
        {
            int ty1 = ty, tx1 = tx;
            next(ty1, tx1);
            if (ty1 < ny) copy_tile(ty1, tx1);
        }
        // primitives and split fluxes of the staged cells; after round r >= 1
        // lane l writes pair l + 32 (r - 1) = (round r - 1, round r)
        float vpr[2][4], vgp[2][4], vgm[2][4];
#pragma unroll
        for (int r = 0; r < 3; r++) {
            if (lane + 32 * r >= WS2) break;
            const int h = r & 1;
            cell2d_f32<0>(cur[r], gm1, alpha, vpr[h], vgp[h], vgm[h]);
            if (r == 0) continue;
            const int i = lane + 32 * (r - 1);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                spr[k][i] = make_float2(vpr[1 - h][k], vpr[h][k]);
                sgp[k][i] = make_float2(vgp[1 - h][k], vgp[h][k]);
                sgm[k][i] = make_float2(vgm[1 - h][k], vgm[h][k]);
            }
        }
        __syncwarp();
        float2 fh[4];
        unsigned D[2][2];
        int flagA = 0, flagB = 0;
        face2d_pair<0, true>(
            fh, D, flagA, flagB, [&](int q, int i) { return spr[q][i]; },
            [&](int s, int cc, int i) { return s == 0 ? sgp[cc][i] : sgm[cc][i]; }, s_cf, eps4, CT, kt, gm1, lane);
        const int jA = c0 - 2 + lane, jB = c0 + 30 + lane;  // faces, and the cells they update
        if (p.rhs_mode && p.masks) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int j = h == 0 ? jA : jB;
                if (!((h == 0 ? lane >= 1 : lane <= 30) && j >= -1 && j <= nx - 1)) continue;
#pragma unroll
                for (int s = 0; s < 2; s++)
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        p.masks[((size_t)(4 * s + k) * ny + y) * (nx + 1) + (j + 1)] = (uint8_t)pair_code(D, s, k, h);
            }
        }
        if (flagA && lane >= 1 && jA >= -2 && jA <= nx) latch_error(ctl, flagA, flat_cell(y, jA, nx));
        if (flagB && lane <= 30 && jB <= nx) latch_error(ctl, flagB, flat_cell(y, jB, nx));
        // flux difference: the left face of cell jA is lane l-1's A; of cell jB,
        // lane l-1's B (lane 0: lane 31's A)
        float2 fprev[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float xr = __shfl_sync(0xffffffffu, fh[k].x, (lane + 31) & 31);
            const float yr = __shfl_sync(0xffffffffu, fh[k].y, (lane + 31) & 31);
            fprev[k] = make_float2(xr, lane == 0 ? xr : yr);
        }
        const bool updA = lane >= 2 && jA < nx, updB = lane <= 30 && jB < nx;
        if (updA || updB) {
            float *Ry = R + (size_t)y * nx;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const float2 r = __fmul2_rn(__fadd2_rn(fprev[k], f2neg(fh[k])), f2(idx));
                if (updA) Ry[(size_t)k * N + chk(p.ctl, jA, 0, p.nx)] = r.x;
                if (updB) Ry[(size_t)k * N + chk(p.ctl, jB, 0, p.nx)] = r.y;
            }
        }
        __syncwarp();  // the next tile overwrites this warp's staging rows
    }
}


inline constexpr size_t ysweep_f32p_smem_bytes() {
    return sizeof(float) * (4 * YB_ROWS * YB_LD + 3 * 4 * YB_STAGE * YB_LD + 4 * YB_STAGE * YB_COLS + 32 * 8 +
                            2 * WPB);
}

template <typename S, bool HALO>  // S = float (the FP32 state) only
__global__ void __launch_bounds__(WPB * 32, 2) ysweep2d_f32p_kernel(const Stage2D p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *s_ry = reinterpret_cast<float *>(smem_raw);  // [4][29][33]
    float *s_gp = s_ry + 4 * YB_ROWS * YB_LD;            // [4][39][33]
    float *s_gm = s_gp + 4 * YB_STAGE * YB_LD;
    float *s_pr = s_gm + 4 * YB_STAGE * YB_LD;
    float *s_in = s_pr + 4 * YB_STAGE * YB_LD;           // [4][39][32] raw state of the block
    float(*s_cf)[8] = reinterpret_cast<float(*)[8]>(s_in + 4 * YB_STAGE * YB_COLS);
    float *s_red = reinterpret_cast<float *>(s_cf + 32);  // [2][WPB]
    auto at = [](const float *base, int c, int r, int col) -> float {
        return base[(c * YB_STAGE + r) * YB_LD + col];
    };

    DevCtl *ctl = p.ctl;
    const bool fixed = p.dt_fixed > 0.0;
    if (!p.rhs_mode && !fixed && !ctl->active) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nx = p.nx, ny = p.ny;
    const size_t N = (size_t)nx * ny;
    const size_t sv = HALO ? p.sv : N, svo = HALO ? p.svo : N;
    const int nbx = (nx + YB_COLS - 1) / YB_COLS, nblocks = nbx * ((ny + YB_ROWS - 1) / YB_ROWS);
    const float alpha = alpha2d_in<float, HALO>(p, ctl, 1);
    const float gamma = p.f_gamma, gm1 = p.f_gm1, eps4 = 4.f * p.f_eps_y, CT = p.f_CT;
    const float kt = keep_all_factor(CT);
    const float *Us = static_cast<const float *>(p.Us);
    const float *R = static_cast<const float *>(p.R);
    const float *U0 = static_cast<const float *>(p.U0);
    float *out = static_cast<float *>(p.out);
    const float idy = 1.f / p.f_dy;
    const float dtF = p.rhs_mode ? 0.f : (fixed ? p.f_dt_fixed : ctl->dt_f);
    const bool use_u0 = !p.rhs_mode && p.stage > 0;
    fill_delta_table(s_cf);
    // running max(|u|+c), max(|v|+c) of the CTA's output cells, as the bit
    // patterns of non-negative floats (ordered like the values)
    int *s_amax = reinterpret_cast<int *>(s_red);
    if (tid < 2) s_amax[tid] = 0;

    // rows r0-5 .. r0+33 of columns x0 .. x0+31 of block b into s_in (one
    // 4-byte asynchronous copy per value; rows outside the grid by y_row,
    // columns beyond it skipped)
    auto copy_block = [&](int b) {
        const int x0 = (b % nbx) * YB_COLS, r0 = (b / nbx) * YB_ROWS;
        const bool inside = r0 >= 5 && r0 + YB_STAGE - 5 <= ny;  // every staged row in the grid (CTA-uniform)
        for (int q = tid; q < YB_STAGE * YB_COLS; q += WPB * 32) {
            const int r = q / YB_COLS, col = q % YB_COLS, x = x0 + col;
            if (x >= nx) continue;
            int y = r0 - 5 + r;
            y = inside ? chk(p.ctl, y, 0, ny) : y_row<HALO>(y, p);
#pragma unroll
            for (int k = 0; k < 4; k++)
                cp_async4(&s_in[(k * YB_STAGE + r) * YB_COLS + col], &Us[st_at<HALO>(k, sv, y, nx, chk(p.ctl, x, 0, p.nx))]);
        }
        cp_async_commit();
    };

    int b = blockIdx.x;
    if (b < nblocks) copy_block(b);
    for (; b < nblocks; b += gridDim.x) {
        const int x0 = (b % nbx) * YB_COLS, r0 = (b / nbx) * YB_ROWS;
        cp_async_wait_all();
        __syncthreads();
        // ---- split fluxes and primitives of the staged cells
        for (int q = tid; q < YB_STAGE * YB_COLS; q += WPB * 32) {
            const int r = q / YB_COLS, col = q % YB_COLS;
            if (x0 + col >= nx) continue;
            float uf[4], pr[4], gp[4], gm[4];
#pragma unroll
            for (int k = 0; k < 4; k++) uf[k] = s_in[(k * YB_STAGE + r) * YB_COLS + col];
            cell2d_f32<1>(uf, gm1, alpha, pr, gp, gm);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                s_pr[(k * YB_STAGE + r) * YB_LD + col] = pr[k];
                s_gp[(k * YB_STAGE + r) * YB_LD + col] = gp[k];
                s_gm[(k * YB_STAGE + r) * YB_LD + col] = gm[k];
            }
        }
        __syncthreads();
        // the next block's raw state streams in while this one computes
        if (b + (int)gridDim.x < nblocks) copy_block(b + gridDim.x);

        // ---- faces down the columns: warp w takes columns w, w+8, w+16, w+24
        for (int col = warp; col < YB_COLS; col += WPB) {
            const int x = x0 + col;
            if (x >= nx) break;
            const int j = r0 - 2 + lane;
            float fh[4];
            unsigned cpk, cmk;
            int flag = 0;
            face2d_f32<1>(
                fh, cpk, cmk, flag, [&](int q, int i) { return at(s_pr, q, i, col); },
                [&](int cc, int i) { return at(s_gp, cc, i, col); },
                [&](int cc, int i) { return at(s_gm, cc, i, col); }, s_cf, eps4, CT, kt, gm1, lane);
            const bool face_out = lane >= 1 && lane <= 30;
            if (p.rhs_mode && p.masks && face_out && j >= -1 && j <= ny - 1) {
                uint8_t *ym = p.masks + (size_t)8 * ny * (nx + 1);
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    ym[((size_t)k * nx + x) * (ny + 1) + (j + 1)] = (uint8_t)((cpk >> (5 * k)) & 31u);
                    ym[((size_t)(4 + k) * nx + x) * (ny + 1) + (j + 1)] = (uint8_t)((cmk >> (5 * k)) & 31u);
                }
            }
            if (flag && face_out && j >= -2 && j <= ny) latch_error(ctl, flag, flat_cell(j, x, nx, ny));
            float fprev[4];
#pragma unroll
            for (int k = 0; k < 4; k++) fprev[k] = __shfl_up_sync(0xffffffffu, fh[k], 1);
            if (lane >= 2 && lane <= 30) {
#pragma unroll
                for (int k = 0; k < 4; k++) s_ry[(k * YB_ROWS + (lane - 2)) * YB_LD + col] = (fprev[k] - fh[k]) * idy;
            }
        }
        __syncthreads();

        // ---- L = Lx + Ly, RK stage, wavespeeds (row-major, coalesced)
        float mx = 0.f, my = 0.f;
        constexpr int EB = 2;  // (4 spills in the persistent loop)
        for (int q0 = tid; q0 < YB_ROWS * YB_COLS; q0 += EB * WPB * 32) {
            float Rv[EB][4], Uv[EB][4], U0v[EB][4];
#pragma unroll
            for (int e = 0; e < EB; e++) {
                const int q = q0 + e * WPB * 32;
                const int r = q / YB_COLS, x = x0 + q % YB_COLS, y = r0 + r;
                if (q < YB_ROWS * YB_COLS && x < nx && y < ny) {
                    const size_t gi = (size_t)chk(p.ctl, y, 0, p.ny) * nx + chk(p.ctl, x, 0, p.nx);
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        Rv[e][k] = R[(size_t)k * N + gi];
                        Uv[e][k] = p.rhs_mode ? 0.f : Us[(size_t)k * sv + gi];
                        U0v[e][k] = use_u0 ? U0[(size_t)k * sv + gi] : 0.f;
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < EB; e++) {
                const int q = q0 + e * WPB * 32;
                const int r = q / YB_COLS, col = q % YB_COLS, x = x0 + col, y = r0 + r;
                if (!(q < YB_ROWS * YB_COLS && x < nx && y < ny)) continue;
                const size_t gi = (size_t)chk(p.ctl, y, 0, p.ny) * nx + chk(p.ctl, x, 0, p.nx);
                float of[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const float rr = Rv[e][k] + s_ry[(k * YB_ROWS + r) * YB_LD + col];
                    if (p.rhs_mode) {
                        out[(size_t)k * svo + gi] = rr;
                        continue;
                    }
                    float o;
                    const float v = fmaf(dtF, rr, Uv[e][k]);
                    if (p.stage == 0) {
                        o = v;
                    } else if (p.stage == 1) {
                        o = fmaf(0.75f, U0v[e][k], 0.25f * v);
                    } else {
                        const float u0 = U0v[e][k];
                        o = fmaf(2.0f / 3.0f, v - u0, u0);
                    }
                    out[(size_t)k * svo + gi] = o;
                    of[k] = o;
                }
                if (!p.rhs_mode) {
                    int wflag = 0;
                    float sx, sy;
                    wavespeed2d<float>(of, gm1, gamma, sx, sy, &wflag);
                    if (wflag) latch_error(ctl, wflag, (int)gi);
                    mx = fmaxf(mx, sx);
                    my = fmaxf(my, sy);
                }
            }
        }
        if (!p.rhs_mode) {
            mx = warp_max(mx);
            my = warp_max(my);
            if (lane == 0) {
                atomicMax(&s_amax[0], __float_as_int(mx));
                atomicMax(&s_amax[1], __float_as_int(my));
            }
        }
        __syncthreads();  // s_ry and the staged arrays are rewritten by the next block
    }
    if (!p.rhs_mode) {
        __syncthreads();
        if (tid == 0) {
            const float vx = __int_as_float(s_amax[0]), vy = __int_as_float(s_amax[1]);
            const int so = (p.stage + 1) % 3;
            atomicMax(&ctl->amax[so][0], (unsigned long long)__double_as_longlong((double)vx));
            atomicMax(&ctl->amax[so][1], (unsigned long long)__double_as_longlong((double)vy));
            finish_launch(ctl, so, (p.stage + 2) % 3, p.stage == 2 && !fixed, p.stage == 2 && !fixed, true,
                          HALO ? p.alpha_rec : nullptr);
        }
    }
}

template <typename S, bool HALO = false>
cudaError_t launch_stage2d_paired(const Stage2D &p, cudaStream_t st) {
    const int ntx = (p.nx + WT - 1) / WT;
    long ntiles = (long)ntx * p.ny;
    long gx = (ntiles + WPB - 1) / WPB;
    // whole waves of 2 CTAs per SM (2D FP32 4.50 -> 4.58 Gcell-steps/s at 2048^2
    // with two waves instead of four)
    const long cap = (long)num_sms() * 2 * T7_WAVES_X2D;
    if (gx > cap) gx = cap;
    if constexpr (sizeof(S) == 4) {
        // FP32 state: paired faces, 61-cell tiles
        const long gx2 = ((long)((p.nx + WT2 - 1) / WT2) * p.ny + WPB - 1) / WPB;
        xsweep2d_f32fp_kernel<HALO><<<(int)(gx2 < cap ? gx2 : cap), WPB * 32, 0, st>>>(p);
    } else {
        xsweep2d_f32_kernel<S, HALO><<<(int)gx, WPB * 32, 0, st>>>(p);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if constexpr (sizeof(S) == 4) {
        // FP32 state: persistent CTAs (two per SM) with the next block prefetched
        const size_t smem = ysweep_f32p_smem_bytes();
        e = cudaFuncSetAttribute(ysweep2d_f32p_kernel<S, HALO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const long nb = (long)((p.nx + YB_COLS - 1) / YB_COLS) * ((p.ny + YB_ROWS - 1) / YB_ROWS);
        const long cap = (long)num_sms() * 2;
        ysweep2d_f32p_kernel<S, HALO><<<(int)(nb < cap ? nb : cap), WPB * 32, smem, st>>>(p);
        return cudaGetLastError();
    } else {
        // mixed precision (FP64 state): one block per CTA
        const size_t smem = ysweep_f32_smem_bytes<S>();
        e = cudaFuncSetAttribute(ysweep2d_f32_kernel<S, HALO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        dim3 grid((p.nx + YB_COLS - 1) / YB_COLS, (p.ny + YB_ROWS - 1) / YB_ROWS);
        ysweep2d_f32_kernel<S, HALO><<<grid, WPB * 32, smem, st>>>(p);
        return cudaGetLastError();
    }
}

template <typename T, bool HALO = false>
cudaError_t launch_stage2d(const Stage2D &p, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        return launch_stage2d_paired<float, HALO>(p, st);
    } else {
    const int ntx = (p.nx + WT - 1) / WT;
    long ntiles = (long)ntx * p.ny;
    long gx = (ntiles + WPB - 1) / WPB;
    const long cap = (long)num_sms() * 4;
    if (gx > cap) gx = cap;
    xsweep2d_kernel<T, HALO><<<(int)gx, WPB * 32, 0, st>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = ysweep_smem_bytes<T>();
    e = cudaFuncSetAttribute(ysweep2d_kernel<T, HALO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((p.nx + YB_COLS - 1) / YB_COLS, (p.ny + YB_ROWS - 1) / YB_ROWS);
    ysweep2d_kernel<T, HALO><<<grid, WPB * 32, smem, st>>>(p);
    return cudaGetLastError();
    }
}

template <typename T, bool HALO = false>
cudaError_t launch_alpha2d(const Alpha2D &p, cudaStream_t st) {
    long grid = ((long)p.nx * p.ny + 255) / 256;
    if (grid > num_sms() * 8) grid = num_sms() * 8;
    alpha2d_kernel<T, HALO><<<(int)grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace t7
