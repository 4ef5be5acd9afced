// teno7_kernels2d.cuh -- 2D Euler, dimension by dimension (L = Lx + Ly), with the
// TENO7-ext reconstruction of each direction in its own characteristic frame
// (Roe average of the two cells of the face; fields un-c, un, shear, un+c).
//
//   x sweep  warp tiles along rows, exactly as the 1D kernels (lane = face);
//            writes Lx(U) into R (coalesced along x).
//   y sweep  one CTA stages a block of 39 rows x 32 columns (29-row tile + halo)
//            in padded shared memory; each warp runs the lane = face logic down
//            4 of the columns, exchanging cutoff words and face fluxes by
//            __shfl along y; after a barrier the CTA adds Lx, applies the RK
//            stage and reduces max(|u|+c), max(|v|+c) in row-major order.
//
// Templated on T; instantiated for FP64 (-fmad=false: the oracle's operation
// order, including the component permutation of the y frame) and FP32.
#pragma once
#include "teno7_kernels.cuh"

namespace t7 {

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
__device__ __forceinline__ void face2d_bits(Face2D<T> &F, PR pr, GP gp, GM gm, T gm1, T eps, T CT) {
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
    F.flag = (c2 > T(0)) ? 0 : ERR_NONPHYSICAL;
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
        const unsigned bp = cutoff_bits(F.qp[k][1], F.qp[k][2], F.qp[k][3], F.qp[k][4], F.qp[k][5], eps, CT);
        const unsigned bm = cutoff_bits(F.qm[k][5], F.qm[k][4], F.qm[k][3], F.qm[k][2], F.qm[k][1], eps, CT);
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
template <typename T>
__device__ __forceinline__ void wavespeed2d(const T U[4], T gm1, T gamma, T &sx, T &sy, int *flag) {
    const T u = U[1] / U[0];
    const T v = U[2] / U[0];
    const T p = gm1 * (U[3] - T(0.5) * (U[1] * u + U[2] * v));
    const T c = sq_root(gamma * p / U[0]);
    if (!(U[0] > T(0)) || !(p > T(0))) *flag |= ERR_NONPHYSICAL;
    if (!isfinite(U[0]) || !isfinite(U[1]) || !isfinite(U[2]) || !isfinite(U[3])) *flag |= ERR_NONFINITE;
    sx = absval(u) + c;
    sy = absval(v) + c;
}

template <typename T>
__device__ __forceinline__ T alpha_of(const DevCtl *ctl, int slot, int dir) {
    if constexpr (sizeof(T) == 8) {
        return __longlong_as_double((long long)ctl->amax[slot][dir]);
    } else {
        return ctl->alpha_f[slot][dir];
    }
}

// --------------------------------------------------------------------------
// x sweep: R = Lx(U), warp tiles of 29 cells along rows.
// --------------------------------------------------------------------------
template <typename T>
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
    const T alpha = alpha_of<T>(ctl, p.slot_in, 0);
    const T gm1 = pick<T>(p.gamma - 1.0, p.f_gm1);
    const T eps = pick<T>(p.eps_x, p.f_eps_x), CT = pick<T>(p.CT, p.f_CT);
    const T *Us = static_cast<const T *>(p.Us);
    T *R = static_cast<T *>(p.R);
    const int nx = p.nx, ny = p.ny;
    const size_t N = (size_t)nx * ny;
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
            T U[4], pr[4], gp[4], gm[4];
#pragma unroll
            for (int k = 0; k < 4; k++) U[k] = row[(size_t)k * N + gi];
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
            [&](int c, int t) { return sgm[c][lane + t]; }, gm1, eps, CT);
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
            latch_error(ctl, (F.flag & ERR_NONPHYSICAL) | ((F.flag & ERR_NOEXIST) ? ERR_NONFINITE : 0), j);
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
                R[(size_t)k * N + (size_t)y * nx + j] = r;
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

template <typename T>
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
    const int x0 = blockIdx.x * YB_COLS, r0 = blockIdx.y * YB_ROWS;
    const T alpha = alpha_of<T>(ctl, p.slot_in, 1);
    const T gamma = pick<T>(p.gamma, p.f_gamma), gm1 = pick<T>(p.gamma - 1.0, p.f_gm1);
    const T eps = pick<T>(p.eps_y, p.f_eps_y), CT = pick<T>(p.CT, p.f_CT);
    const T *Us = static_cast<const T *>(p.Us);
    for (int q = tid; q < 91; q += blockDim.x) s_coef[q] = coef<T>(q);

    // ---- stage rows r0-5 .. r0+33 of columns x0 .. x0+31 (coalesced along x)
    for (int idx = tid; idx < YB_STAGE * YB_COLS; idx += blockDim.x) {
        const int r = idx / YB_COLS, col = idx % YB_COLS, x = x0 + col;
        if (x >= nx) continue;
        int y = r0 - 5 + r;
        if (y < 0 || y >= ny) y = ghost_map(y, ny, p.bc[2], p.bc[3]);
        T U[4], pr[4], gp[4], gm[4];
#pragma unroll
        for (int k = 0; k < 4; k++) U[k] = Us[(size_t)k * N + (size_t)y * nx + x];
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
            [&](int c, int t) { return at(s_gm, c, lane + t, col); }, gm1, eps, CT);
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
            latch_error(ctl, (F.flag & ERR_NONPHYSICAL) | ((F.flag & ERR_NOEXIST) ? ERR_NONFINITE : 0), j);
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
        const size_t g = (size_t)y * nx + x;
        T o[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const T rr = R[(size_t)k * N + g] + s_ry[(k * YB_ROWS + r) * YB_LD + col];
            if (p.rhs_mode) {
                out[(size_t)k * N + g] = rr;
                continue;
            }
            const T us = Us[(size_t)k * N + g];
            if (p.stage == 0) {
                o[k] = us + dtT * rr;
            } else if (p.stage == 1) {
                o[k] = T(0.75) * U0[(size_t)k * N + g] + T(0.25) * (us + dtT * rr);
            } else {
                if constexpr (sizeof(T) == 8) {
                    o[k] = T(1.0 / 3.0) * U0[(size_t)k * N + g] + T(2.0 / 3.0) * (us + dtT * rr);
                } else {
                    const T u0 = U0[(size_t)k * N + g];
                    o[k] = fmaf(2.0f / 3.0f, (us + dtT * rr) - u0, u0);
                }
            }
            out[(size_t)k * N + g] = o[k];
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
            finish_launch(ctl, so, (p.stage + 2) % 3, p.stage == 2 && !fixed, p.stage == 2 && !fixed, true);
        }
    }
}

// alpha (both directions) of a 2D state into ctl->amax[slot][0..1].
template <typename T>
__global__ void __launch_bounds__(256) alpha2d_kernel(const Alpha2D p) {
    __shared__ T s_red[2][8];
    const T *U = static_cast<const T *>(p.U);
    const T gamma = T(p.gamma), gm1 = T(p.gamma - 1.0);
    const size_t N = (size_t)p.nx * p.ny;
    T mx = T(0), my = T(0);
    int flag = 0, first = 0x7fffffff;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        T Uc[4];
#pragma unroll
        for (int k = 0; k < 4; k++) Uc[k] = U[(size_t)k * N + i];
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
        finish_launch(p.ctl, p.slot, (p.slot + 1) % 3, false, true, true);
    }
}

template <typename T>
cudaError_t launch_stage2d(const Stage2D &p, cudaStream_t st) {
    const int ntx = (p.nx + WT - 1) / WT;
    long ntiles = (long)ntx * p.ny;
    long gx = (ntiles + WPB - 1) / WPB;
    const long cap = (long)num_sms() * 4;
    if (gx > cap) gx = cap;
    xsweep2d_kernel<T><<<(int)gx, WPB * 32, 0, st>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = ysweep_smem_bytes<T>();
    e = cudaFuncSetAttribute(ysweep2d_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((p.nx + YB_COLS - 1) / YB_COLS, (p.ny + YB_ROWS - 1) / YB_ROWS);
    ysweep2d_kernel<T><<<grid, WPB * 32, smem, st>>>(p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_alpha2d(const Alpha2D &p, cudaStream_t st) {
    long grid = ((long)p.nx * p.ny + 255) / 256;
    if (grid > num_sms() * 8) grid = num_sms() * 8;
    alpha2d_kernel<T><<<(int)grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace t7
