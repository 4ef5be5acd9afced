// teno7_kernels.cuh -- CUDA kernels of the TENO7-ext hot path (arXiv:1808.00037),
// templated on the floating-point type.  Included by one translation unit per
// precision:
//   teno7_f64.cu  compiled with -fmad=false: every FP64 expression below is
//                 evaluated one IEEE operation at a time in the written order
//                 (the same order in which the CPU oracle states the method),
//                 so FP64 results and stencil masks are reproducible bit for bit;
//   teno7_f32.cu  FMA contraction on; the cutoff test uses an overflow-safe
//                 rescaled form (g_k / g_max)^6 because gamma_k = (1 + r)^6
//                 overflows FP32 near strong jumps.
//
// Tile design (1D).  One CTA of NT = 256 threads owns the faces j+1/2,
// j = s-2 .. s+253, one face per thread, and updates the TILE = 253 cells
// s .. s+252.  Per-cell data for cells s-5 .. s+257 (the face stencils plus
// halo) are staged once in shared memory: conserved variables, the global
// Lax-Friedrichs split fluxes G+- = (F +- alpha U)/2, and for the Euler system
// u, H and sqrt(rho) for the Roe average.  Each thread then
//   1. builds its face's Roe frame (L, R) and projects the 8 cells it needs
//      into characteristic fields, keeping q+ (7 cells) and q- (7 cells) per
//      field in registers;
//   2. computes the three cutoff bits of both splits of every field (Eqs.
//      smooth_expl, tau5, TENO1, norm, seclect) and publishes them as one
//      word in shared memory -- the "store the smoothness of the whole field
//      first" step of the paper, done per tile;
//   3. after a barrier, reads the neighbouring faces' words, forms Delta_i
//      (Eq. vec) for each split and field, looks the polynomial up (Table co3,
//      a 32 x 4-bit table held in two 64-bit immediates) and evaluates it
//      (Table co2, 7 taps, coefficients in shared memory);
//   4. back-projects with R and publishes the face flux; after a barrier the
//      cell threads take the flux difference (Eq. app), apply the SSP-RK3
//      stage, write the new state and reduce max(|u| + c) of it for the next
//      stage's alpha (one atomicMax per CTA).
#pragma once
#include <math.h>
#include <stdint.h>

#include "teno7_internal.h"

namespace t7 {

constexpr int NT = 256;         // faces (threads) per tile
constexpr int TILE = NT - 3;    // cells updated per tile
constexpr int HALO = 5;         // staged cells start at s - HALO
constexpr int NCELL = NT + 7;   // cells staged per tile
constexpr int NCP = NCELL + 1;  // padded row length in shared memory

// Table co3 as 32 four-bit entries (index = Delta with its first component in
// bit 4); 15 marks the pattern (*,0,0,0,*) that cannot occur for finite data.
constexpr unsigned long long LUT_LO = 0x14886ACC37BB6AFFull;  // Delta 0..15
constexpr unsigned long long LUT_HI = 0x02556A9937BB6AFFull;  // Delta 16..31

__device__ __forceinline__ int lut_select(int D) {
    unsigned long long w = (D & 16) ? LUT_HI : LUT_LO;
    return (int)((w >> (4 * (D & 15))) & 15ull);
}

// Delta_i from the three-bit codes of faces i-1/2 (dm), i+1/2 (d0), i+3/2 (dp)
// for the '+' split; the '-' split passes the neighbours swapped.
__device__ __forceinline__ int pack_delta(unsigned dm, unsigned d0, unsigned dp) {
    return (int)(((dm & 1u) << 4) | ((d0 & 1u) << 3) | (((d0 >> 1) & 1u) << 2) | (((d0 >> 2) & 1u) << 1) |
                 ((dp >> 2) & 1u));
}

// Table co2, coefficients on f_{i-3} .. f_{i+3}; each entry is the nearest
// double to the printed rational.
__device__ __forceinline__ double coef_f64(int idx) {
    switch (idx) {
        // clang-format off
        case 0: return -1.0/140.0; case 1: return 5.0/84.0; case 2: return -101.0/420.0; case 3: return 319.0/420.0;
        case 4: return 107.0/210.0; case 5: return -19.0/210.0; case 6: return 1.0/105.0;
        case 7: return 0.0; case 8: return 1.0/60.0; case 9: return -2.0/15.0; case 10: return 37.0/60.0;
        case 11: return 37.0/60.0; case 12: return -2.0/15.0; case 13: return 1.0/60.0;
        case 14: return -1.0/60.0; case 15: return 7.0/60.0; case 16: return -23.0/60.0; case 17: return 19.0/20.0;
        case 18: return 11.0/30.0; case 19: return -1.0/30.0; case 20: return 0.0;
        case 21: return 0.0; case 22: return 0.0; case 23: return -1.0/20.0; case 24: return 9.0/20.0;
        case 25: return 47.0/60.0; case 26: return -13.0/60.0; case 27: return 1.0/30.0;
        case 28: return 0.0; case 29: return 1.0/30.0; case 30: return -13.0/60.0; case 31: return 47.0/60.0;
        case 32: return 9.0/20.0; case 33: return -1.0/20.0; case 34: return 0.0;
        case 35: return -1.0/20.0; case 36: return 17.0/60.0; case 37: return -43.0/60.0; case 38: return 77.0/60.0;
        case 39: return 1.0/5.0; case 40: return 0.0; case 41: return 0.0;
        case 42: return 0.0; case 43: return 0.0; case 44: return 0.0; case 45: return 1.0/4.0;
        case 46: return 13.0/12.0; case 47: return -5.0/12.0; case 48: return 1.0/12.0;
        case 49: return 0.0; case 50: return 0.0; case 51: return -1.0/12.0; case 52: return 7.0/12.0;
        case 53: return 7.0/12.0; case 54: return -1.0/12.0; case 55: return 0.0;
        case 56: return 0.0; case 57: return 1.0/12.0; case 58: return -5.0/12.0; case 59: return 13.0/12.0;
        case 60: return 1.0/4.0; case 61: return 0.0; case 62: return 0.0;
        case 63: return -1.0/4.0; case 64: return 13.0/12.0; case 65: return -23.0/12.0; case 66: return 25.0/12.0;
        case 67: return 0.0; case 68: return 0.0; case 69: return 0.0;
        case 70: return 0.0; case 71: return 0.0; case 72: return 0.0; case 73: return 1.0/3.0;
        case 74: return 5.0/6.0; case 75: return -1.0/6.0; case 76: return 0.0;
        case 77: return 0.0; case 78: return 0.0; case 79: return -1.0/6.0; case 80: return 5.0/6.0;
        case 81: return 1.0/3.0; case 82: return 0.0; case 83: return 0.0;
        case 84: return 0.0; case 85: return 1.0/3.0; case 86: return -7.0/6.0; case 87: return 11.0/6.0;
        case 88: return 0.0; case 89: return 0.0; case 90: return 0.0;
        default: return 0.0;
        // clang-format on
    }
}

// --------------------------------------------------------------------------
// Five-point smoothness measure and cutoff bits (d0 | d1<<1 | d2<<2) of one
// window w0..w4 = f_{i-2} .. f_{i+2} in upwind order.
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned cutoff_bits(double w0, double w1, double w2, double w3, double w4, double eps,
                                                double CT) {
    // Eq. smooth_expl
    double s0a = w0 - 4.0 * w1 + 3.0 * w2;
    double s0b = w0 - 2.0 * w1 + w2;
    double s1a = w1 - w3;
    double s1b = w1 - 2.0 * w2 + w3;
    double s2a = 3.0 * w2 - 4.0 * w3 + w4;
    double s2b = w2 - 2.0 * w3 + w4;
    double b0 = 0.25 * (s0a * s0a) + (13.0 / 12.0) * (s0b * s0b);
    double b1 = 0.25 * (s1a * s1a) + (13.0 / 12.0) * (s1b * s1b);
    double b2 = 0.25 * (s2a * s2a) + (13.0 / 12.0) * (s2b * s2b);
    // Eq. tau5, Eq. TENO1 with C = 1, q = 6 (squared, squared again, times square)
    double tau = fabs(b0 - b2);
    double g0 = 1.0 + tau / (b0 + eps);
    double g1 = 1.0 + tau / (b1 + eps);
    double g2 = 1.0 + tau / (b2 + eps);
    double q0 = g0 * g0, q1 = g1 * g1, q2 = g2 * g2;
    double y0 = (q0 * q0) * q0, y1 = (q1 * q1) * q1, y2 = (q2 * q2) * q2;
    // Eqs. norm, seclect: delta = 0 iff chi < C_T
    double S = (y0 + y1) + y2;
    unsigned d0 = (y0 / S < CT) ? 0u : 1u;
    unsigned d1 = (y1 / S < CT) ? 0u : 1u;
    unsigned d2 = (y2 / S < CT) ? 0u : 1u;
    return d0 | (d1 << 1) | (d2 << 2);
}

__device__ __forceinline__ unsigned cutoff_bits(float w0, float w1, float w2, float w3, float w4, float eps,
                                                float CT) {
    float s0a = fmaf(3.f, w2, fmaf(-4.f, w1, w0));
    float s0b = fmaf(-2.f, w1, w0) + w2;
    float s1a = w1 - w3;
    float s1b = fmaf(-2.f, w2, w1) + w3;
    float s2a = fmaf(3.f, w2, fmaf(-4.f, w3, w4));
    float s2b = fmaf(-2.f, w3, w2) + w4;
    const float c13 = 13.f / 12.f;
    float b0 = fmaf(0.25f * s0a, s0a, c13 * s0b * s0b);
    float b1 = fmaf(0.25f * s1a, s1a, c13 * s1b * s1b);
    float b2 = fmaf(0.25f * s2a, s2a, c13 * s2b * s2b);
    float tau = fabsf(b0 - b2);
    float g0 = 1.f + __fdividef(tau, b0 + eps);
    float g1 = 1.f + __fdividef(tau, b1 + eps);
    float g2 = 1.f + __fdividef(tau, b2 + eps);
    // chi_k = g_k^6 / sum g^6 = x_k^6 / sum x^6 with x = g / g_max in (0, 1]
    float rg = __frcp_rn(fmaxf(g0, fmaxf(g1, g2)));
    float x0 = g0 * rg, x1 = g1 * rg, x2 = g2 * rg;
    x0 *= x0; x1 *= x1; x2 *= x2;
    float y0 = x0 * x0 * x0, y1 = x1 * x1 * x1, y2 = x2 * x2 * x2;
    float thr = CT * ((y0 + y1) + y2);
    return (y0 < thr ? 0u : 1u) | ((y1 < thr ? 0u : 1u) << 1) | ((y2 < thr ? 0u : 1u) << 2);
}

template <typename T>
__device__ __forceinline__ T poly7(const T *__restrict__ c, const T v0, const T v1, const T v2, const T v3,
                                   const T v4, const T v5, const T v6) {
    // sum in tap order, starting from the first product
    T s = c[0] * v0;
    s = s + c[1] * v1;
    s = s + c[2] * v2;
    s = s + c[3] * v3;
    s = s + c[4] * v4;
    s = s + c[5] * v5;
    s = s + c[6] * v6;
    return s;
}

template <typename T>
__device__ __forceinline__ T dv(T a, T b);
template <>
__device__ __forceinline__ double dv<double>(double a, double b) {
    return a / b;
}
template <>
__device__ __forceinline__ float dv<float>(float a, float b) {
    return __fdividef(a, b);
}

__device__ __forceinline__ double sq_root(double x) { return sqrt(x); }
__device__ __forceinline__ float sq_root(float x) { return sqrtf(x); }
__device__ __forceinline__ double absval(double x) { return fabs(x); }
__device__ __forceinline__ float absval(float x) { return fabsf(x); }

__device__ __forceinline__ int ghost_map(int l, int n, int bc_lo, int bc_hi) {
    if (l < 0) {
        if (bc_lo == BC_PERIODIC) {
            int r = l % n;
            return r < 0 ? r + n : r;
        }
        return 0;
    }
    if (l >= n) return bc_hi == BC_PERIODIC ? (l % n) : n - 1;
    return l;
}

__device__ __forceinline__ void latch_error(DevCtl *ctl, int flag, int index) {
    atomicOr(&ctl->err, flag);
    atomicMin(&ctl->err_index, index);
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Largest characteristic speed of one cell (1D systems) and its validity.
template <typename T, int SYS>
__device__ __forceinline__ T wavespeed1d(const T *Uc, T gm1, T gamma, T a, int *flag) {
    if (SYS == SYS_ADV) return absval(a);
    if (SYS == SYS_BURGERS) {
        if (!isfinite(Uc[0])) *flag |= ERR_NONFINITE;
        return absval(Uc[0]);
    }
    T u = Uc[1] / Uc[0];
    T p = gm1 * (Uc[2] - T(0.5) * Uc[1] * u);
    T c = sq_root(gamma * p / Uc[0]);
    if (!(Uc[0] > T(0)) || !(p > T(0))) *flag |= ERR_NONPHYSICAL;
    if (!isfinite(Uc[0]) || !isfinite(Uc[1]) || !isfinite(Uc[2])) *flag |= ERR_NONFINITE;
    return absval(u) + c;
}

// ==========================================================================
// Fused 1D stage kernel.  SYS in {SYS_ADV, SYS_BURGERS, SYS_EULER1D}.
// ==========================================================================
template <typename T, int SYS>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 ? 2 : 1)) stage1d_kernel(const Stage1D p) {
    constexpr int M = (SYS == SYS_EULER1D) ? 3 : 1;
    constexpr int NP = (SYS == SYS_EULER1D) ? 3 : 1;  // u, H, sqrt(rho)
    __shared__ T s_U[M][NCP];
    __shared__ T s_gp[M][NCP];
    __shared__ T s_gm[M][NCP];
    __shared__ T s_pr[NP][NCP];
    __shared__ T s_coef[91];
    __shared__ unsigned s_bits[NT];
    __shared__ T s_fh[M][NT];
    __shared__ double s_red[NT / 32];

    DevCtl *ctl = p.ctl;
    const int tid = threadIdx.x;
    const int n = p.n;
    const int s = blockIdx.x * TILE;

    // ---- time step of this stage -----------------------------------------
    const double alpha_d = __longlong_as_double((long long)ctl->amax[p.slot_in][0]);
    double dt = 0.0;
    if (!p.rhs_mode) {
        if (p.dt_fixed > 0.0) {
            dt = p.dt_fixed;
        } else if (p.stage == 0) {
            const double t = ctl->t, t_end = ctl->t_end;
            const bool active = (ctl->steps < ctl->max_steps) && (t < t_end);
            dt = (ctl->cfl * p.dx) / alpha_d;
            if (t + dt > t_end) dt = t_end - t;
            if (blockIdx.x == 0 && tid == 0) {
                ctl->dt = dt;
                ctl->active = active ? 1 : 0;
            }
            if (!active) return;
        } else {
            if (!ctl->active) return;
            dt = ctl->dt;
        }
        if (blockIdx.x == 0 && tid == 0) ctl->amax[(p.stage + 2) % 3][0] = 0ull;
    }

    const T gamma = T(p.gamma), gm1 = T(p.gamma - 1.0), a = T(p.a);
    const T alpha = T(alpha_d), eps = T(p.eps), CT = T(p.CT);
    const T *Us = static_cast<const T *>(p.Us);

    for (int q = tid; q < 91; q += NT) s_coef[q] = T(coef_f64(q));

    // ---- stage per-cell data: cells s-5 .. s+257 ---------------------------
    for (int c = tid; c < NCELL; c += NT) {
        const int gi = ghost_map(s - HALO + c, n, p.bc_lo, p.bc_hi);
        T U[M], F[M];
#pragma unroll
        for (int k = 0; k < M; k++) U[k] = Us[(size_t)k * n + gi];
        if (SYS == SYS_ADV) {
            F[0] = a * U[0];
        } else if (SYS == SYS_BURGERS) {
            F[0] = T(0.5) * U[0] * U[0];
        } else {
            T u = U[1] / U[0];
            T pr = gm1 * (U[2] - T(0.5) * U[1] * u);
            F[0] = U[1];
            F[1] = U[1] * u + pr;
            F[2] = u * (U[2] + pr);
            s_pr[0][c] = u;
            s_pr[NP > 1 ? 1 : 0][c] = (U[2] + pr) / U[0];
            s_pr[NP > 2 ? 2 : 0][c] = sq_root(U[0]);
        }
#pragma unroll
        for (int k = 0; k < M; k++) {
            s_U[k][c] = U[k];
            s_gp[k][c] = T(0.5) * (F[k] + alpha * U[k]);
            s_gm[k][c] = T(0.5) * (F[k] - alpha * U[k]);
        }
    }
    __syncthreads();

    // ---- face j+1/2, j = s-2+tid: frame, projection, cutoff bits ------------
    T L[M][M];
    T ut = T(0), cc = T(0), Ht = T(0);
    int flag = 0;
    if (SYS == SYS_EULER1D) {
        const T ul = s_pr[0][tid + 3], ur = s_pr[0][tid + 4];
        const T Hl = s_pr[NP > 1 ? 1 : 0][tid + 3], Hr = s_pr[NP > 1 ? 1 : 0][tid + 4];
        const T sl = s_pr[NP > 2 ? 2 : 0][tid + 3], sr = s_pr[NP > 2 ? 2 : 0][tid + 4];
        ut = (sl * ul + sr * ur) / (sl + sr);
        Ht = (sl * Hl + sr * Hr) / (sl + sr);
        const T c2 = gm1 * (Ht - T(0.5) * ut * ut);
        cc = sq_root(c2);
        const T b1 = gm1 / c2;
        const T b2 = T(0.5) * ut * ut * b1;
        L[0][0] = T(0.5) * (b2 + ut / cc);
        L[0][1 % M] = T(-0.5) * (b1 * ut + T(1) / cc);
        L[0][2 % M] = T(0.5) * b1;
        L[1 % M][0] = T(1) - b2;
        L[1 % M][1 % M] = b1 * ut;
        L[1 % M][2 % M] = -b1;
        L[2 % M][0] = T(0.5) * (b2 - ut / cc);
        L[2 % M][1 % M] = T(-0.5) * (b1 * ut - T(1) / cc);
        L[2 % M][2 % M] = T(0.5) * b1;
        if (!(c2 > T(0))) flag |= ERR_NONPHYSICAL;
    } else {
        L[0][0] = T(1);
    }

    T qp[M][7], qm[M][7];
    unsigned word = 0;
#pragma unroll
    for (int k = 0; k < M; k++) {
#pragma unroll
        for (int t = 0; t < 7; t++) {
            if (M == 1) {
                qp[k][t] = s_gp[0][tid + t];
                qm[k][t] = s_gm[0][tid + 1 + t];
            } else {
                T sp = L[k][0] * s_gp[0][tid + t];
                T sm = L[k][0] * s_gm[0][tid + 1 + t];
#pragma unroll
                for (int c = 1; c < M; c++) {
                    sp = sp + L[k][c] * s_gp[c][tid + t];
                    sm = sm + L[k][c] * s_gm[c][tid + 1 + t];
                }
                qp[k][t] = sp;
                qm[k][t] = sm;
            }
        }
        const unsigned bp = cutoff_bits(qp[k][1], qp[k][2], qp[k][3], qp[k][4], qp[k][5], eps, CT);
        const unsigned bm = cutoff_bits(qm[k][5], qm[k][4], qm[k][3], qm[k][2], qm[k][1], eps, CT);
        word |= bp << (3 * k);
        word |= bm << (3 * (M + k));
    }
    s_bits[tid] = word;
    __syncthreads();

    // ---- selection, polynomial, back-projection ----------------------------
    const int j = s - 2 + tid;  // this thread's face is j+1/2
    if (tid >= 1 && tid <= NT - 2) {
        const unsigned wl = s_bits[tid - 1], wr = s_bits[tid + 1];
        T f[M];
#pragma unroll
        for (int k = 0; k < M; k++) {
            const int Dp = pack_delta(wl >> (3 * k), word >> (3 * k), wr >> (3 * k));
            const int Dm = pack_delta(wr >> (3 * (M + k)), word >> (3 * (M + k)), wl >> (3 * (M + k)));
            int mp = lut_select(Dp), mm = lut_select(Dm);
            if (mp == 15) {
                mp = 11;
                flag |= ERR_NOEXIST;
            }
            if (mm == 15) {
                mm = 11;
                flag |= ERR_NOEXIST;
            }
            const T fp = poly7(s_coef + 7 * mp, qp[k][0], qp[k][1], qp[k][2], qp[k][3], qp[k][4], qp[k][5], qp[k][6]);
            const T fm = poly7(s_coef + 7 * mm, qm[k][6], qm[k][5], qm[k][4], qm[k][3], qm[k][2], qm[k][1], qm[k][0]);
            f[k] = fp + fm;
            if (p.rhs_mode && p.masks && j >= -1 && j <= n - 1) {
                p.masks[(size_t)(0 * M + k) * (n + 1) + (j + 1)] = (uint8_t)Dp;
                p.masks[(size_t)(1 * M + k) * (n + 1) + (j + 1)] = (uint8_t)Dm;
            }
        }
        if (SYS == SYS_EULER1D) {
            // R columns: eigenvectors of u-c, u, u+c at the Roe state
            const T R20 = Ht - ut * cc, R21 = T(0.5) * ut * ut, R22 = Ht + ut * cc;
            s_fh[0][tid] = f[0] + f[1 % M] + f[2 % M];
            s_fh[1 % M][tid] = (ut - cc) * f[0] + ut * f[1 % M] + (ut + cc) * f[2 % M];
            s_fh[2 % M][tid] = R20 * f[0] + R21 * f[1 % M] + R22 * f[2 % M];
        } else {
            s_fh[0][tid] = f[0];
        }
    }
    if (flag && j >= -2 && j <= n) latch_error(ctl, (flag & ERR_NONPHYSICAL) | ((flag & ERR_NOEXIST) ? ERR_NONFINITE : 0), j);
    __syncthreads();

    // ---- flux difference and RK stage ---------------------------------------
    const int i = j;  // cell i = j: faces i-1/2 (tid-1) and i+1/2 (tid)
    double ws = 0.0;
    if (tid >= 2 && tid <= NT - 2 && i < n) {
        T r[M];
        const T dxT = T(p.dx);
#pragma unroll
        for (int k = 0; k < M; k++) r[k] = (s_fh[k][tid - 1] - s_fh[k][tid]) / dxT;
        T *out = static_cast<T *>(p.out);
        if (p.rhs_mode) {
#pragma unroll
            for (int k = 0; k < M; k++) out[(size_t)k * n + i] = r[k];
        } else {
            const T dtT = T(dt);
            const T *U0 = static_cast<const T *>(p.U0);
            T o[M];
#pragma unroll
            for (int k = 0; k < M; k++) {
                const T us = s_U[k][tid + 3];
                if (p.stage == 0) {
                    o[k] = us + dtT * r[k];
                } else if (p.stage == 1) {
                    o[k] = T(0.75) * U0[(size_t)k * n + i] + T(0.25) * (us + dtT * r[k]);
                } else {
                    if constexpr (sizeof(T) == 8) {
                        o[k] = T(1.0 / 3.0) * U0[(size_t)k * n + i] + T(2.0 / 3.0) * (us + dtT * r[k]);
                    } else {
                        // in FP32, float(1/3) + float(2/3) = 1 + 6e-8 would grow the
                        // solution by that factor every step: use u0 + 2/3 (v - u0)
                        const T u0 = U0[(size_t)k * n + i];
                        o[k] = fmaf(2.0f / 3.0f, (us + dtT * r[k]) - u0, u0);
                    }
                }
                out[(size_t)k * n + i] = o[k];
            }
            int wflag = 0;
            ws = (double)wavespeed1d<T, SYS>(o, gm1, gamma, a, &wflag);
            if (wflag) latch_error(ctl, wflag, i);
        }
    }
    if (!p.rhs_mode) {
        ws = warp_max(ws);
        if ((tid & 31) == 0) s_red[tid >> 5] = ws;
        __syncthreads();
        if (tid < 32) {
            double v = tid < NT / 32 ? s_red[tid] : 0.0;
            v = warp_max(v);
            if (tid == 0) atomicMax(&ctl->amax[(p.stage + 1) % 3][0], (unsigned long long)__double_as_longlong(v));
        }
        if (p.stage == 2 && p.dt_fixed <= 0.0 && blockIdx.x == 0 && tid == 0) {
            ctl->t = ctl->t + dt;
            ctl->steps = ctl->steps + 1;
        }
    }
}

// alpha of a 1D state into ctl->amax[slot][0]; grid-stride, one atomic per CTA.
template <typename T, int SYS>
__global__ void __launch_bounds__(256) alpha1d_kernel(const Alpha1D p) {
    __shared__ double s_red[8];
    const T *U = static_cast<const T *>(p.U);
    const T gamma = T(p.gamma), gm1 = T(p.gamma - 1.0), a = T(p.a);
    constexpr int M = (SYS == SYS_EULER1D) ? 3 : 1;
    double m = 0.0;
    int flag = 0, first = 0x7fffffff;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += gridDim.x * blockDim.x) {
        T Uc[M];
#pragma unroll
        for (int k = 0; k < M; k++) Uc[k] = U[(size_t)k * p.n + i];
        int f = 0;
        double w = (double)wavespeed1d<T, SYS>(Uc, gm1, gamma, a, &f);
        if (f) {
            flag |= f;
            first = min(first, i);
        }
        m = fmax(m, w);
    }
    if (flag) latch_error(p.ctl, flag, first);
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < 8 ? s_red[threadIdx.x] : 0.0;
        v = warp_max(v);
        if (threadIdx.x == 0) atomicMax(&p.ctl->amax[p.slot][0], (unsigned long long)__double_as_longlong(v));
    }
}

// Scalar reconstruction of caller-padded values (t7_teno7_reconstruct).
template <typename T>
__global__ void __launch_bounds__(NT) recon_kernel(const Recon p) {
    __shared__ T s_v[NCP];
    __shared__ T s_coef[91];
    __shared__ unsigned s_bits[NT];
    const int tid = threadIdx.x, n = p.n;
    const int s = blockIdx.x * TILE;
    const T *v = static_cast<const T *>(p.v);
    const T eps = T(p.eps), CT = T(p.CT);
    for (int q = tid; q < 91; q += NT) s_coef[q] = T(coef_f64(q));
    for (int c = tid; c < NCELL; c += NT) {
        int l = s - HALO + c + 4;  // index into v (cell -4 is v[0])
        l = l < 0 ? 0 : (l > n + 7 ? n + 7 : l);
        s_v[c] = v[l];
    }
    __syncthreads();
    const int j = s - 2 + tid;
    unsigned bits;
    if (p.sign > 0)
        bits = cutoff_bits(s_v[tid + 1], s_v[tid + 2], s_v[tid + 3], s_v[tid + 4], s_v[tid + 5], eps, CT);
    else
        bits = cutoff_bits(s_v[tid + 6], s_v[tid + 5], s_v[tid + 4], s_v[tid + 3], s_v[tid + 2], eps, CT);
    s_bits[tid] = bits;
    if (p.d3 && j >= -2 && j <= n) p.d3[j + 2] = (uint8_t)bits;
    __syncthreads();
    if (tid >= 1 && tid <= NT - 2 && j >= -1 && j <= n - 1) {
        const unsigned wl = s_bits[tid - 1], wr = s_bits[tid + 1];
        int D, m;
        T f;
        if (p.sign > 0) {
            D = pack_delta(wl, bits, wr);
            m = lut_select(D);
            if (m == 15) {
                m = 11;
                latch_error(p.ctl, ERR_NONFINITE, j);
            }
            f = poly7(s_coef + 7 * m, s_v[tid], s_v[tid + 1], s_v[tid + 2], s_v[tid + 3], s_v[tid + 4], s_v[tid + 5],
                      s_v[tid + 6]);
        } else {
            D = pack_delta(wr, bits, wl);
            m = lut_select(D);
            if (m == 15) {
                m = 11;
                latch_error(p.ctl, ERR_NONFINITE, j);
            }
            f = poly7(s_coef + 7 * m, s_v[tid + 7], s_v[tid + 6], s_v[tid + 5], s_v[tid + 4], s_v[tid + 3],
                      s_v[tid + 2], s_v[tid + 1]);
        }
        static_cast<T *>(p.fhat)[j + 1] = f;
        if (p.D5) p.D5[j + 1] = (uint8_t)D;
    }
}

// ---------------------------------------------------------------- launchers --
template <typename T>
cudaError_t launch_stage1d(const Stage1D &p, cudaStream_t st) {
    const int grid = (p.n + TILE - 1) / TILE;
    switch (p.sys) {
        case SYS_ADV: stage1d_kernel<T, SYS_ADV><<<grid, NT, 0, st>>>(p); break;
        case SYS_BURGERS: stage1d_kernel<T, SYS_BURGERS><<<grid, NT, 0, st>>>(p); break;
        case SYS_EULER1D: stage1d_kernel<T, SYS_EULER1D><<<grid, NT, 0, st>>>(p); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_alpha1d(const Alpha1D &p, cudaStream_t st) {
    int grid = (p.n + 255) / 256;
    if (grid > 152 * 8) grid = 152 * 8;
    switch (p.sys) {
        case SYS_ADV: alpha1d_kernel<T, SYS_ADV><<<grid, 256, 0, st>>>(p); break;
        case SYS_BURGERS: alpha1d_kernel<T, SYS_BURGERS><<<grid, 256, 0, st>>>(p); break;
        case SYS_EULER1D: alpha1d_kernel<T, SYS_EULER1D><<<grid, 256, 0, st>>>(p); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_recon(const Recon &p, cudaStream_t st) {
    const int grid = (p.n + TILE - 1) / TILE;
    recon_kernel<T><<<grid, NT, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace t7
