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
// Tile design (1D).  The work unit is a warp tile: one warp owns the 32
// faces j+1/2, j = c0-2 .. c0+29, one face per lane, and updates the WT = 29
// cells c0 .. c0+28.  The 39 cells c0-5 .. c0+33 that those faces' stencils
// reach are staged in warp-private shared memory (conserved variables, the
// global Lax-Friedrichs split fluxes G+- = (F +- alpha U)/2 and, for the Euler
// system, u, H and sqrt(rho) for the Roe average), so no CTA-wide barrier is
// needed inside the loop; warps stride over tiles.  Each lane then
//   1. builds its face's Roe frame (L, R) and projects the cells it needs into
//      characteristic fields (q+ on cells j-3 .. j+3, q- on j-2 .. j+4);
//   2. computes the three cutoff bits of both splits of every field (Eqs.
//      smooth_expl, tau5, TENO1, norm, seclect) -- the paper's "measure the
//      smoothness of every face first" pass, kept per warp tile;
//   3. takes the neighbouring faces' bits by __shfl (faces i-1/2 and i+3/2 are
//      the adjacent lanes), forms Delta_i (Eq. vec) for each split and field,
//      selects the polynomial (Table co3) and evaluates it (Table co2, 7 taps);
//   4. back-projects with R; the face flux of lane l-1 arrives by __shfl, and
//      lanes 2..30 take the flux difference (Eq. app), apply the SSP-RK3 stage,
//      write the new state and fold max(|u| + c) of it into the next stage's
//      alpha (a warp/CTA reduction, one atomicMax per CTA).
// The FP32 kernels keep this structure with packed f32x2 arithmetic:
// stage1d_f32_kernel pairs the two splits of one face in a float2 (it runs the
// mixed precision form, the batch tubes and parted launches); stage1d_f32fp_kernel
// pairs two faces of a 61-cell tile (lane l: faces c0-2+l and c0+30+l) and runs
// the splits one after the other (whole-domain and slab launches of the FP32
// state).  Both give the same bits.
// Grids cover whole waves of each kernel's resident CTAs (stage_grid); the
// loads of a tile take the boundary map only where a staged cell lies outside
// the grid; every index formed for a global access passes through chk(),
// which the checked build (T7_CHECKED=1) turns into a bounds check.
#pragma once
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "teno7_internal.h"

namespace t7 {

// CTA tiles of the plain scalar reconstruction kernel (recon_kernel, the face
// values alone, without the flux difference), which exchanges cutoff words
// through shared memory; the stage kernels use the warp tiles described above.
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

// Table co2, coefficients on f_{i-3} .. f_{i+3}; each FP64 entry is the nearest
// double to the printed rational (FP32: that double rounded to float).
template <typename T>
__device__ __forceinline__ T coef(int idx) {
    switch (idx) {
        // clang-format off
        case 0: return T(-1.0/140.0); case 1: return T(5.0/84.0); case 2: return T(-101.0/420.0); case 3: return T(319.0/420.0);
        case 4: return T(107.0/210.0); case 5: return T(-19.0/210.0); case 6: return T(1.0/105.0);
        case 7: return T(0); case 8: return T(1.0/60.0); case 9: return T(-2.0/15.0); case 10: return T(37.0/60.0);
        case 11: return T(37.0/60.0); case 12: return T(-2.0/15.0); case 13: return T(1.0/60.0);
        case 14: return T(-1.0/60.0); case 15: return T(7.0/60.0); case 16: return T(-23.0/60.0); case 17: return T(19.0/20.0);
        case 18: return T(11.0/30.0); case 19: return T(-1.0/30.0); case 20: return T(0);
        case 21: return T(0); case 22: return T(0); case 23: return T(-1.0/20.0); case 24: return T(9.0/20.0);
        case 25: return T(47.0/60.0); case 26: return T(-13.0/60.0); case 27: return T(1.0/30.0);
        case 28: return T(0); case 29: return T(1.0/30.0); case 30: return T(-13.0/60.0); case 31: return T(47.0/60.0);
        case 32: return T(9.0/20.0); case 33: return T(-1.0/20.0); case 34: return T(0);
        case 35: return T(-1.0/20.0); case 36: return T(17.0/60.0); case 37: return T(-43.0/60.0); case 38: return T(77.0/60.0);
        case 39: return T(1.0/5.0); case 40: return T(0); case 41: return T(0);
        case 42: return T(0); case 43: return T(0); case 44: return T(0); case 45: return T(1.0/4.0);
        case 46: return T(13.0/12.0); case 47: return T(-5.0/12.0); case 48: return T(1.0/12.0);
        case 49: return T(0); case 50: return T(0); case 51: return T(-1.0/12.0); case 52: return T(7.0/12.0);
        case 53: return T(7.0/12.0); case 54: return T(-1.0/12.0); case 55: return T(0);
        case 56: return T(0); case 57: return T(1.0/12.0); case 58: return T(-5.0/12.0); case 59: return T(13.0/12.0);
        case 60: return T(1.0/4.0); case 61: return T(0); case 62: return T(0);
        case 63: return T(-1.0/4.0); case 64: return T(13.0/12.0); case 65: return T(-23.0/12.0); case 66: return T(25.0/12.0);
        case 67: return T(0); case 68: return T(0); case 69: return T(0);
        case 70: return T(0); case 71: return T(0); case 72: return T(0); case 73: return T(1.0/3.0);
        case 74: return T(5.0/6.0); case 75: return T(-1.0/6.0); case 76: return T(0);
        case 77: return T(0); case 78: return T(0); case 79: return T(-1.0/6.0); case 80: return T(5.0/6.0);
        case 81: return T(1.0/3.0); case 82: return T(0); case 83: return T(0);
        case 84: return T(0); case 85: return T(1.0/3.0); case 86: return T(-7.0/6.0); case 87: return T(11.0/6.0);
        case 88: return T(0); case 89: return T(0); case 90: return T(0);
        default: return T(0);
        // clang-format on
    }
}

// --------------------------------------------------------------------------
// Shortcut of the cutoff test.  If tau < kt (beta_min + eps), every
// g_k = 1 + tau / (beta_k + eps) lies in [1, 1 + kt), so
// chi_k = g_k^6 / sum_j g_j^6 >= 1 / (3 (1 + kt)^6).  With
// 1 + kt = 0.9 (3 C_T)^(-1/6) that bound is C_T / 0.9^6 = 1.88 C_T: every
// stencil is kept, and the divisions and powers need not be evaluated.  The
// 10% margin in g (1.9x in chi) is far above the rounding of either
// precision, so the bits are exactly the ones the full evaluation gives.
// kt = 0 (the shortcut never applies) when C_T >= 1/3.
// --------------------------------------------------------------------------
__device__ __forceinline__ double keep_all_factor(double CT) {
    return (CT > 0.0 && CT < 1.0 / 3.0) ? 0.9 * pow(3.0 * CT, -1.0 / 6.0) - 1.0 : 0.0;
}
__device__ __forceinline__ float keep_all_factor(float CT) {
    return (CT > 0.f && CT < 1.f / 3.f) ? 0.9f * powf(3.f * CT, -1.f / 6.f) - 1.f : 0.f;
}

// --------------------------------------------------------------------------
// Five-point smoothness measure and cutoff bits (d0 | d1<<1 | d2<<2) of one
// window w0..w4 = f_{i-2} .. f_{i+2} in upwind order; kt from keep_all_factor.
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned cutoff_bits(double w0, double w1, double w2, double w3, double w4, double eps,
                                                double CT, double kt) {
    // Eq. smooth_expl
    double s0a = w0 - 4.0 * w1 + 3.0 * w2;
    double s0b = w0 - 2.0 * w1 + w2;
    double s2a = 3.0 * w2 - 4.0 * w3 + w4;
    double s2b = w2 - 2.0 * w3 + w4;
    double b0 = 0.25 * (s0a * s0a) + (13.0 / 12.0) * (s0b * s0b);
    double b2 = 0.25 * (s2a * s2a) + (13.0 / 12.0) * (s2b * s2b);
    // Eq. tau5, Eq. TENO1 with C = 1, q = 6 (squared, squared again, times square)
    double tau = fabs(b0 - b2);
    // every stencil kept (see keep_all_factor); beta_min >= 0, so tau < kt eps
    // already suffices and beta_1 is not needed
    if (tau < kt * eps) return 7u;
    double s1a = w1 - w3;
    double s1b = w1 - 2.0 * w2 + w3;
    double b1 = 0.25 * (s1a * s1a) + (13.0 / 12.0) * (s1b * s1b);
    if (tau < kt * (fmin(fmin(b0, b1), b2) + eps)) return 7u;
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
                                                float CT, float kt) {
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
    // FP32 round-off floor of epsilon (2^-24 Q^2 / 12 for the unscaled beta;
    // see RO_FLOOR12 below)
    const float q = fmaxf(fmaxf(fabsf(w0), fabsf(w2)), fabsf(w4));
    eps = fmaxf(eps, (5.9604644775390625e-08f / 12.f) * (q * q));
    if (tau < kt * (fminf(fminf(b0, b1), b2) + eps)) return 7u;  // every stencil kept (see keep_all_factor)
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

// Checked build (compiled with T7_CHECKED=1; compute-sanitizer is not
// available to this project): every cell, row and column index a kernel forms
// for a global-memory access is tested against the extent of the array it
// addresses.  An index outside [lo, hi) is latched as ERR_INDEX with its value
// and replaced by lo, so that the access stays inside the buffer and the
// launch completes; the host reports T7_EINDEX.  In the release build
// (T7_CHECKED=0) chk is the identity and adds no instruction.
#ifndef T7_CHECKED
#define T7_CHECKED 0
#endif
__device__ __forceinline__ int chk(DevCtl *ctl, int i, int lo, int hi) {
#if T7_CHECKED
    if (i < lo || i >= hi) {
        latch_error(ctl, ERR_INDEX, i);
        return lo;
    }
#else
    (void)ctl;
    (void)lo;
    (void)hi;
#endif
    return i;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Largest characteristic speed of one cell (1D systems) and its validity.
// FP64 follows the oracle's expression order; FP32 uses fast reciprocals.
template <typename T, int SYS>
__device__ __forceinline__ T wavespeed1d(const T *Uc, T gm1, T gamma, T a, int *flag) {
    if (SYS == SYS_ADV) return absval(a);
    if (SYS == SYS_BURGERS) {
        if (!isfinite(Uc[0])) *flag |= ERR_NONFINITE;
        return absval(Uc[0]);
    }
    T u, p, c;
    if constexpr (sizeof(T) == 8) {
        u = Uc[1] / Uc[0];
        p = gm1 * (Uc[2] - T(0.5) * Uc[1] * u);
        c = sq_root(gamma * p / Uc[0]);
    } else {
        const float ri = __frcp_rn(Uc[0]);
        u = Uc[1] * ri;
        p = gm1 * (Uc[2] - 0.5f * Uc[1] * u);
        c = __fsqrt_rn(gamma * p * ri);
    }
    // a non-finite cell is reported as such; a finite one needs rho > 0, p > 0
    if (!isfinite(Uc[0]) || !isfinite(Uc[1]) || !isfinite(Uc[2]))
        *flag |= ERR_NONFINITE;
    else if (!(Uc[0] > T(0)) || !(p > T(0)))
        *flag |= ERR_NONPHYSICAL;
    return absval(u) + c;
}

// |u - c|, |u|, |u + c| of one 1D Euler cell (the characteristic speeds of
// fields 0, 1, 2, for per-field alphas), with wavespeed1d's operations and
// flags; the largest equals wavespeed1d's |u| + c bit for bit.
template <typename T>
__device__ __forceinline__ void wavespeeds1d(const T *Uc, T gm1, T gamma, T w[3], int *flag) {
    T u, p, c;
    if constexpr (sizeof(T) == 8) {
        u = Uc[1] / Uc[0];
        p = gm1 * (Uc[2] - T(0.5) * Uc[1] * u);
        c = sq_root(gamma * p / Uc[0]);
    } else {
        const float ri = __frcp_rn(Uc[0]);
        u = Uc[1] * ri;
        p = gm1 * (Uc[2] - 0.5f * Uc[1] * u);
        c = __fsqrt_rn(gamma * p * ri);
    }
    if (!isfinite(Uc[0]) || !isfinite(Uc[1]) || !isfinite(Uc[2]))
        *flag |= ERR_NONFINITE;
    else if (!(Uc[0] > T(0)) || !(p > T(0)))
        *flag |= ERR_NONPHYSICAL;
    w[0] = absval(u - c);
    w[1] = absval(u);
    w[2] = absval(u + c);
}

template <typename T>
__device__ __forceinline__ T pick(double d, float f) {
    if constexpr (sizeof(T) == 8) {
        return d;
    } else {
        return f;
    }
}

// Table co2 row 0 (the seventh-order polynomial) as immediates: the common
// smooth case avoids the shared-memory coefficient table.  Same values and
// summation order as the table path.
template <typename T>
__device__ __forceinline__ T poly_f0(T v0, T v1, T v2, T v3, T v4, T v5, T v6) {
    T s = T(-1.0 / 140.0) * v0;
    s = s + T(5.0 / 84.0) * v1;
    s = s + T(-101.0 / 420.0) * v2;
    s = s + T(319.0 / 420.0) * v3;
    s = s + T(107.0 / 210.0) * v4;
    s = s + T(-19.0 / 210.0) * v5;
    s = s + T(1.0 / 105.0) * v6;
    return s;
}

// --------------------------------------------------------------------------
// TENO5 baseline (the fifth-order TENO scheme the paper measures TENO7-ext
// against).  A face selects its polynomial from its OWN three cutoff bits --
// no neighbour faces -- among the seven rows of Table co1, polynomials on
// f_{i-2} .. f_{i+2} in upwind order.
// --------------------------------------------------------------------------
enum { SCH_TENO7EXT = 0, SCH_TENO5 = 1 };

// Table co1 row for the code d0 | d1<<1 | d2<<2 as eight 4-bit entries
// (7 = no cutoff bit set, which finite data cannot produce).
constexpr unsigned SEL5 = 0x01632457u;
__device__ __forceinline__ int sel5(unsigned code) { return (int)((SEL5 >> (4 * (code & 7u))) & 15u); }

// Table co1 coefficients, row-major [7][5]; FP64 entries are the nearest
// doubles to the printed rationals.
template <typename T>
__device__ __forceinline__ T coef5(int idx) {
    switch (idx) {
        // clang-format off
        case 0: return T(1.0/30.0); case 1: return T(-13.0/60.0); case 2: return T(47.0/60.0); case 3: return T(9.0/20.0); case 4: return T(-1.0/20.0);
        case 5: return T(0); case 6: return T(-1.0/9.0); case 7: return T(2.0/3.0); case 8: return T(1.0/2.0); case 9: return T(-1.0/18.0);
        case 10: return T(1.0/21.0); case 11: return T(-13.0/42.0); case 12: return T(41.0/42.0); case 13: return T(2.0/7.0); case 14: return T(0);
        case 15: return T(0); case 16: return T(0); case 17: return T(1.0/3.0); case 18: return T(5.0/6.0); case 19: return T(-1.0/6.0);
        case 20: return T(0); case 21: return T(-1.0/6.0); case 22: return T(5.0/6.0); case 23: return T(1.0/3.0); case 24: return T(0);
        case 25: return T(1.0/3.0); case 26: return T(-7.0/6.0); case 27: return T(11.0/6.0); case 28: return T(0); case 29: return T(0);
        case 30: return T(1.0/12.0); case 31: return T(-7.0/24.0); case 32: return T(17.0/24.0); case 33: return T(5.0/8.0); case 34: return T(-1.0/8.0);
        default: return T(0);
        // clang-format on
    }
}

template <typename T>
__device__ __forceinline__ T poly5(const T *__restrict__ c, const T v0, const T v1, const T v2, const T v3,
                                   const T v4) {
    T s = c[0] * v0;
    s = s + c[1] * v1;
    s = s + c[2] * v2;
    s = s + c[3] * v3;
    s = s + c[4] * v4;
    return s;
}

// --------------------------------------------------------------------------
// Last-CTA finalization of a launch (see DevCtl).  Called by thread 0 of every
// CTA after its atomicMax into amax[slot_out].
//   zero_slot    the slot the next launch accumulates into (cleared here)
//   end_of_step  advance t and steps by the step just taken
//   plan_step    compute active and the CFL step dt for the next RK step from
//                alpha(U^n) = amax[slot_out] (oracle's expression order)
// --------------------------------------------------------------------------
__device__ __forceinline__ void finish_launch(DevCtl *ctl, int slot_out, int zero_slot, bool end_of_step,
                                              bool plan_step, bool two_d = false, double *alpha_rec = nullptr,
                                              int nfield = 1) {
    __threadfence();
    const unsigned prev = atomicAdd(&ctl->blocks_done, 1u);
    if (prev != gridDim.x * gridDim.y - 1) return;
    __threadfence();
    const double a = __longlong_as_double((long long)atomicAdd(&ctl->amax[slot_out][0], 0ull));
    const double ay = (two_d || nfield > 1) ? __longlong_as_double((long long)atomicAdd(&ctl->amax[slot_out][1], 0ull))
                                            : 0.0;
    const double a2 = nfield > 2 ? __longlong_as_double((long long)atomicAdd(&ctl->amax[slot_out][2], 0ull)) : 0.0;
    ctl->alpha_f[slot_out][0] = (float)a;
    ctl->alpha_f[slot_out][1] = (float)ay;
    ctl->alpha_f[slot_out][2] = (float)a2;
    if (alpha_rec) {  // recorded for a later adjoint, or for a slab's all-reduce
        alpha_rec[0] = a;
        if (two_d) alpha_rec[1] = ay;
    }
    ctl->amax[zero_slot][0] = 0ull;
    ctl->amax[zero_slot][1] = 0ull;
    ctl->amax[zero_slot][2] = 0ull;
    if (end_of_step) {
        ctl->t = ctl->t + ctl->dt;
        ctl->steps = ctl->steps + 1;
    }
    if (plan_step) {
        const double t = ctl->t, t_end = ctl->t_end;
        const int active = (ctl->steps < ctl->max_steps) && (t < t_end);
        // CFL step in the oracle's expression order: 1D cfl dx / a, 2D cfl / (ax/dx + ay/dy); per-field
        // alphas: the largest of the three, which equals the global alpha
        const double a1d = nfield > 2 ? fmax(fmax(a, ay), a2) : a;
        double dt = two_d ? ctl->cfl / (a / ctl->dx + ay / ctl->dy) : (ctl->cfl * ctl->dx) / a1d;
        if (t + dt > t_end) dt = t_end - t;
        ctl->active = active;
        ctl->dt = dt;
        ctl->dt_f = (float)dt;
    }
    ctl->blocks_done = 0u;
}

// ==========================================================================
// Warp-tile sweep of one 1D problem (a whole domain, or one tube of a ragged
// batch), shared by the grid-wide stage kernels and the persistent batch
// kernel.  Warp tile w updates the WT = 29 cells c0 = 29 w .. c0 + 28; lane l
// owns the face j+1/2 with j = c0 - 2 + l (faces c0-2 .. c0+29) and stages
// cells c0-5+l (and c0+27+l for l < 7) in warp-private shared memory.
// Neighbouring faces' cutoff words and face fluxes travel by __shfl, so the
// loop has no CTA-wide barrier; lanes 1..30 produce face fluxes and lanes
// 2..30 update cells.  Returns this lane's max characteristic speed of the
// cells it wrote (RK mode).
// ==========================================================================
constexpr int WT = 29;   // cells updated per warp tile
constexpr int WS = 39;   // cells staged per warp tile
constexpr int WC = 40;   // padded row length
constexpr int WPB = 8;   // warps per CTA
static_assert(WT == TILE_CELLS, "the host's tile size must match the kernels'");

template <typename T>
struct TileArgs {
    const T *Us;     // stage input (stencil reads)
    const T *U0;     // U^n (pointwise reads; stages 1 and 2)
    T *out;          // RK: stage output; RHS: dU/dt
    uint8_t *masks;  // RHS only, nullable: [2][m][n+1]
    int n;           // cells
    size_t cs;       // stride between conserved variables (Us, U0)
    size_t cso;      // stride between conserved variables of out
    int bc_lo, bc_hi;
    double dx;
    float f_dx;
    T alpha, dtT, gamma, gm1, a, eps, CT;
    T alf[3];        // per-field alphas (1D Euler, the per-field alpha mode)
    double dtD;      // FP64 step (mixed precision: FP64 state, FP32 reconstruction)
    int rhs_mode, stage;
    int ebase;       // added to cell/face indices in error reports
    int halo;        // the arrays hold HALO_CELLS filled ghost cells per side (slab mode)
    DevCtl *ctl;
};

// Index of a staged cell l outside 0 .. n-1: the boundary condition, or in
// slab mode the caller-filled padding (cells beyond it are never used by an
// updated cell and are read clamped into it).
__device__ __forceinline__ int ghost_or_halo(int l, int n, int bc_lo, int bc_hi, int halo) {
    if (halo) return l < -HALO_CELLS ? -HALO_CELLS : (l > n + HALO_CELLS - 1 ? n + HALO_CELLS - 1 : l);
    return ghost_map(l, n, bc_lo, bc_hi);
}

// PF (1D Euler, TENO7-ext): per-field alphas A.alf -- each field's split values
// (L_k F +- alf[k] L_k U) / 2 from the staged flux (sgp) and state (sU), in the
// oracle's operation order; ws3 receives the output's three characteristic
// speed maxima (the function then returns 0).
template <typename T, int SYS, int SCH = SCH_TENO7EXT, bool PF = false>
__device__ __forceinline__ T tiles1d(const TileArgs<T> &A, T (*sU)[WC], T (*sgp)[WC], T (*sgm)[WC], T (*spr)[WC],
                                     const T *scoef, int tile0, int tstride, int tile_end = 0x7fffffff,
                                     T *ws3 = nullptr) {
    constexpr int M = (SYS == SYS_EULER1D) ? 3 : 1;
    constexpr int NP = (SYS == SYS_EULER1D) ? 3 : 1;  // u, H, sqrt(rho)
    constexpr bool F64 = sizeof(T) == 8;
    const int lane = threadIdx.x & 31;
    const T *Us = A.Us;
    const T *U0 = A.U0;
    T *out = A.out;
    const int n = A.n;
    const size_t cs = A.cs;
    const int ntiles = min((n + WT - 1) / WT, tile_end);  // tiles tile0, tile0 + tstride, ... below it
    const T alpha = A.alpha, dtT = A.dtT, gamma = A.gamma, gm1 = A.gm1, a = A.a, eps = A.eps, CT = A.CT;
    const T kt = keep_all_factor(CT);
    DevCtl *ctl = A.ctl;
    T wsmax = T(0);
    for (int tile = tile0; tile < ntiles; tile += tstride) {
        const int c0 = tile * WT;
        // ---- stage cells c0-5 .. c0+33 -----------------------------------
        for (int c = lane; c < WS; c += 32) {
            int gi = c0 - 5 + c;
            if (gi < 0 || gi >= n) gi = ghost_or_halo(gi, n, A.bc_lo, A.bc_hi, A.halo);
            gi = chk(ctl, gi, A.halo ? -HALO_CELLS : 0, n + (A.halo ? HALO_CELLS : 0));
            T U[M], F[M];
#pragma unroll
            for (int k = 0; k < M; k++) U[k] = Us[(size_t)k * cs + gi];
            if (SYS == SYS_ADV) {
                F[0] = a * U[0];
            } else if (SYS == SYS_BURGERS) {
                F[0] = T(0.5) * U[0] * U[0];
            } else {
                if constexpr (F64) {
                    T u = U[1] / U[0];
                    T pr = gm1 * (U[2] - T(0.5) * U[1] * u);
                    F[0] = U[1];
                    F[1] = U[1] * u + pr;
                    F[2] = u * (U[2] + pr);
                    spr[0][c] = u;
                    spr[NP > 1 ? 1 : 0][c] = (U[2] + pr) / U[0];
                    spr[NP > 2 ? 2 : 0][c] = sq_root(U[0]);
                } else {
                    const float ri = __frcp_rn(U[0]);
                    const float u = U[1] * ri;
                    const float pr = gm1 * (U[2] - 0.5f * U[1] * u);
                    F[0] = U[1];
                    F[1] = U[1] * u + pr;
                    F[2] = u * (U[2] + pr);
                    spr[0][c] = u;
                    spr[NP > 1 ? 1 : 0][c] = (U[2] + pr) * ri;
                    spr[NP > 2 ? 2 : 0][c] = __fsqrt_rn(U[0]);
                }
            }
#pragma unroll
            for (int k = 0; k < M; k++) {
                sU[k][c] = U[k];
                if constexpr (PF) {
                    sgp[k][c] = F[k];
                } else {
                    sgp[k][c] = T(0.5) * (F[k] + alpha * U[k]);
                    sgm[k][c] = T(0.5) * (F[k] - alpha * U[k]);
                }
            }
        }
        __syncwarp();

        // ---- face j+1/2: frame, projection, cutoff bits --------------------
        const int j = c0 - 2 + lane;
        T L[M][M];
        T ut = T(0), cc = T(0), Ht = T(0);
        int flag = 0;
        if (SYS == SYS_EULER1D) {
            const T ul = spr[0][lane + 3], ur = spr[0][lane + 4];
            const T Hl = spr[NP > 1 ? 1 : 0][lane + 3], Hr = spr[NP > 1 ? 1 : 0][lane + 4];
            const T sl = spr[NP > 2 ? 2 : 0][lane + 3], sr = spr[NP > 2 ? 2 : 0][lane + 4];
            if constexpr (F64) {
                // Roe average and eigenvectors in the oracle's operation order
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
                if (!(c2 > T(0))) flag |= isfinite(c2) ? ERR_NONPHYSICAL : ERR_NONFINITE;
            } else {
                const float w = __frcp_rn(sl + sr);
                ut = (sl * ul + sr * ur) * w;
                Ht = (sl * Hl + sr * Hr) * w;
                const float c2 = gm1 * (Ht - 0.5f * ut * ut);
                const float rc = rsqrtf(c2);  // 1/c
                cc = c2 * rc;
                const float b1 = gm1 * (rc * rc);
                const float b2 = 0.5f * ut * ut * b1;
                const float uc = ut * rc;
                L[0][0] = 0.5f * (b2 + uc);
                L[0][1 % M] = -0.5f * (b1 * ut + rc);
                L[0][2 % M] = 0.5f * b1;
                L[1 % M][0] = 1.f - b2;
                L[1 % M][1 % M] = b1 * ut;
                L[1 % M][2 % M] = -b1;
                L[2 % M][0] = 0.5f * (b2 - uc);
                L[2 % M][1 % M] = -0.5f * (b1 * ut - rc);
                L[2 % M][2 % M] = 0.5f * b1;
                if (!(c2 > 0.f)) flag |= isfinite(c2) ? ERR_NONPHYSICAL : ERR_NONFINITE;
            }
        } else {
            L[0][0] = T(1);
        }

        T qp[M][7], qm[M][7];
        unsigned word = 0;
#pragma unroll
        for (int k = 0; k < M; k++) {
#pragma unroll
            for (int t = 0; t < 7; t++) {
                if (SCH == SCH_TENO5 && (t == 0 || t == 6)) {  // five-point stencils
                    qp[k][t] = qm[k][t] = T(0);
                    continue;
                }
                if constexpr (PF) {
                    // '+' at cell lane+t, '-' at cell lane+1+t (forward order, as qm)
                    T lf = L[k][0] * sgp[0][lane + t], lu = L[k][0] * sU[0][lane + t];
                    T mf = L[k][0] * sgp[0][lane + 1 + t], mu = L[k][0] * sU[0][lane + 1 + t];
#pragma unroll
                    for (int c = 1; c < M; c++) {
                        lf = lf + L[k][c] * sgp[c][lane + t];
                        lu = lu + L[k][c] * sU[c][lane + t];
                        mf = mf + L[k][c] * sgp[c][lane + 1 + t];
                        mu = mu + L[k][c] * sU[c][lane + 1 + t];
                    }
                    qp[k][t] = T(0.5) * (lf + A.alf[k] * lu);
                    qm[k][t] = T(0.5) * (mf - A.alf[k] * mu);
                } else if (M == 1) {
                    qp[k][t] = sgp[0][lane + t];
                    qm[k][t] = sgm[0][lane + 1 + t];
                } else {
                    T sp = L[k][0] * sgp[0][lane + t];
                    T sm = L[k][0] * sgm[0][lane + 1 + t];
#pragma unroll
                    for (int c = 1; c < M; c++) {
                        sp = sp + L[k][c] * sgp[c][lane + t];
                        sm = sm + L[k][c] * sgm[c][lane + 1 + t];
                    }
                    qp[k][t] = sp;
                    qm[k][t] = sm;
                }
            }
            const unsigned bp = cutoff_bits(qp[k][1], qp[k][2], qp[k][3], qp[k][4], qp[k][5], eps, CT, kt);
            const unsigned bm = cutoff_bits(qm[k][5], qm[k][4], qm[k][3], qm[k][2], qm[k][1], eps, CT, kt);
            word |= bp << (3 * k);
            word |= bm << (3 * (M + k));
        }
        // ---- selection, polynomial, back-projection ------------------------
        const bool face_out = lane >= 1 && lane <= 30;
        T f[M];
        if constexpr (SCH == SCH_TENO5) {
            // TENO5: the face's own code picks a Table co1 row; '+' taps are
            // cells j-2 .. j+2, '-' taps cells j+3 .. j-1
#pragma unroll
            for (int k = 0; k < M; k++) {
                const unsigned bp = (word >> (3 * k)) & 7u, bm = (word >> (3 * (M + k))) & 7u;
                int rp = sel5(bp), rm = sel5(bm);
                if (rp == 7) {
                    rp = 0;
                    if (face_out) flag |= ERR_NOEXIST;
                }
                if (rm == 7) {
                    rm = 0;
                    if (face_out) flag |= ERR_NOEXIST;
                }
                const T fp = poly5(scoef + 5 * rp, qp[k][1], qp[k][2], qp[k][3], qp[k][4], qp[k][5]);
                const T fm = poly5(scoef + 5 * rm, qm[k][5], qm[k][4], qm[k][3], qm[k][2], qm[k][1]);
                f[k] = fp + fm;
                if (A.masks && face_out && j >= -1 && j <= n - 1) {
                    A.masks[(size_t)(0 * M + k) * (n + 1) + (j + 1)] = (uint8_t)bp;
                    A.masks[(size_t)(1 * M + k) * (n + 1) + (j + 1)] = (uint8_t)bm;
                }
            }
        } else {
        const unsigned wl = __shfl_up_sync(0xffffffffu, word, 1);
        const unsigned wr = __shfl_down_sync(0xffffffffu, word, 1);
#pragma unroll
        for (int k = 0; k < M; k++) {
            const int Dp = pack_delta(wl >> (3 * k), word >> (3 * k), wr >> (3 * k));
            const int Dm = pack_delta(wr >> (3 * (M + k)), word >> (3 * (M + k)), wl >> (3 * (M + k)));
            int mp = lut_select(Dp), mm = lut_select(Dm);
            if (mp == 15) {
                mp = 11;
                if (face_out) flag |= ERR_NOEXIST;
            }
            if (mm == 15) {
                mm = 11;
                if (face_out) flag |= ERR_NOEXIST;
            }
            T fp, fm;
            if (mp == 0)
                fp = poly_f0(qp[k][0], qp[k][1], qp[k][2], qp[k][3], qp[k][4], qp[k][5], qp[k][6]);
            else
                fp = poly7(scoef + 7 * mp, qp[k][0], qp[k][1], qp[k][2], qp[k][3], qp[k][4], qp[k][5], qp[k][6]);
            if (mm == 0)
                fm = poly_f0(qm[k][6], qm[k][5], qm[k][4], qm[k][3], qm[k][2], qm[k][1], qm[k][0]);
            else
                fm = poly7(scoef + 7 * mm, qm[k][6], qm[k][5], qm[k][4], qm[k][3], qm[k][2], qm[k][1], qm[k][0]);
            f[k] = fp + fm;
            if (A.masks && face_out && j >= -1 && j <= n - 1) {
                A.masks[(size_t)(0 * M + k) * (n + 1) + (j + 1)] = (uint8_t)Dp;
                A.masks[(size_t)(1 * M + k) * (n + 1) + (j + 1)] = (uint8_t)Dm;
            }
        }
        }  // TENO7-ext
        T fh[M];
        if (SYS == SYS_EULER1D) {
            // R columns: eigenvectors of u-c, u, u+c at the Roe state
            const T R20 = Ht - ut * cc, R21 = T(0.5) * ut * ut, R22 = Ht + ut * cc;
            fh[0] = f[0] + f[1 % M] + f[2 % M];
            fh[1 % M] = (ut - cc) * f[0] + ut * f[1 % M] + (ut + cc) * f[2 % M];
            fh[2 % M] = R20 * f[0] + R21 * f[1 % M] + R22 * f[2 % M];
        } else {
            fh[0] = f[0];
        }
        if (flag && face_out && j >= -2 && j <= n)
            latch_error(ctl, (flag & (ERR_NONPHYSICAL | ERR_NONFINITE)) | ((flag & ERR_NOEXIST) ? ERR_NONFINITE : 0),
                        A.ebase + j);

        // ---- flux difference and RK stage ----------------------------------
        T fprev[M];
#pragma unroll
        for (int k = 0; k < M; k++) fprev[k] = __shfl_up_sync(0xffffffffu, fh[k], 1);
        const int i = j;  // cell i: faces i-1/2 (lane-1) and i+1/2 (this lane)
        if (lane >= 2 && lane <= 30 && i < n) {
            const int ii = chk(ctl, i, 0, n);
            T r[M];
            if constexpr (F64) {
#pragma unroll
                for (int k = 0; k < M; k++) r[k] = (fprev[k] - fh[k]) / A.dx;
            } else {
                const float idx = __frcp_rn(A.f_dx);
#pragma unroll
                for (int k = 0; k < M; k++) r[k] = (fprev[k] - fh[k]) * idx;
            }
            if (A.rhs_mode) {
#pragma unroll
                for (int k = 0; k < M; k++) out[(size_t)k * A.cso + ii] = r[k];
            } else {
                T o[M];
#pragma unroll
                for (int k = 0; k < M; k++) {
                    const T us = sU[k][lane + 3];
                    if (A.stage == 0) {
                        o[k] = us + dtT * r[k];
                    } else if (A.stage == 1) {
                        o[k] = T(0.75) * U0[(size_t)k * cs + ii] + T(0.25) * (us + dtT * r[k]);
                    } else {
                        if constexpr (F64) {
                            o[k] = T(1.0 / 3.0) * U0[(size_t)k * cs + ii] + T(2.0 / 3.0) * (us + dtT * r[k]);
                        } else {
                            // in FP32, float(1/3) + float(2/3) = 1 + 6e-8 would grow the
                            // solution by that factor every step: use u0 + 2/3 (v - u0)
                            const T u0 = U0[(size_t)k * cs + ii];
                            o[k] = fmaf(2.0f / 3.0f, (us + dtT * r[k]) - u0, u0);
                        }
                    }
                    out[(size_t)k * A.cso + ii] = o[k];
                }
                int wflag = 0;
                if constexpr (PF) {
                    T w[3];
                    wavespeeds1d<T>(o, gm1, gamma, w, &wflag);
#pragma unroll
                    for (int q = 0; q < 3; q++) ws3[q] = fmax(ws3[q], w[q]);
                } else {
                    wsmax = fmax(wsmax, wavespeed1d<T, SYS>(o, gm1, gamma, a, &wflag));
                }
                if (wflag) latch_error(ctl, wflag, A.ebase + i);
            }
        }
        __syncwarp();  // the next tile overwrites this warp's staging rows
    }

    return wsmax;
}

// ==========================================================================
// Fused 1D stage kernel (grid-wide), SYS in {SYS_ADV, SYS_BURGERS, SYS_EULER1D}.
// ==========================================================================
template <typename T, int SYS, int SCH, bool PF = false>
__global__ void __launch_bounds__(WPB * 32, (sizeof(T) == 4 ? 2 : 1)) stage1d_kernel(const Stage1D p) {
    constexpr int M = (SYS == SYS_EULER1D) ? 3 : 1;
    constexpr int NP = (SYS == SYS_EULER1D) ? 3 : 1;
    __shared__ T s_U[WPB][M][WC];
    __shared__ T s_gp[WPB][M][WC];
    __shared__ T s_gm[WPB][M][WC];
    __shared__ T s_pr[WPB][NP][WC];
    __shared__ T s_coef[WPB][92];
    __shared__ T s_red[PF ? 3 : 1][WPB];

    DevCtl *ctl = p.ctl;
    const bool fixed = p.dt_fixed > 0.0;
    if (!p.rhs_mode && !fixed && !ctl->active) return;  // uniform: the run has ended
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (SCH == SCH_TENO5) {
        for (int q = lane; q < 35; q += 32) s_coef[warp][q] = coef5<T>(q);
    } else {
        for (int q = lane; q < 91; q += 32) s_coef[warp][q] = coef<T>(q);
    }

    TileArgs<T> A;
    if constexpr (sizeof(T) == 8) {
        A.alpha = p.alpha_in ? *p.alpha_in : __longlong_as_double((long long)ctl->amax[p.slot_in][0]);
        A.dtT = fixed ? p.dt_fixed : ctl->dt;
        if constexpr (PF) {
#pragma unroll
            for (int q = 0; q < 3; q++) A.alf[q] = __longlong_as_double((long long)ctl->amax[p.slot_in][q]);
        }
    } else {
        A.alpha = p.alpha_in ? (float)*p.alpha_in : ctl->alpha_f[p.slot_in][0];
        A.dtT = fixed ? p.f_dt_fixed : ctl->dt_f;
    }
    // slab mode: cell 0 follows the padding (the RHS output dU/dt is unpadded)
    const int off = p.halo ? HALO_CELLS : 0, offo = p.rhs_mode ? 0 : off;
    A.Us = static_cast<const T *>(p.Us) + off;
    A.U0 = p.U0 ? static_cast<const T *>(p.U0) + off : nullptr;
    A.out = static_cast<T *>(p.out) + offo;
    A.masks = p.masks;
    A.n = p.n;
    A.cs = (size_t)p.n + 2 * off;
    A.cso = (size_t)p.n + 2 * offo;
    A.halo = p.halo;
    A.bc_lo = p.bc_lo;
    A.bc_hi = p.bc_hi;
    A.dx = p.dx;
    A.f_dx = p.f_dx;
    A.gamma = pick<T>(p.gamma, p.f_gamma);
    A.gm1 = pick<T>(p.gamma - 1.0, p.f_gm1);
    A.a = pick<T>(p.a, p.f_a);
    A.eps = pick<T>(p.eps, p.f_eps);
    A.CT = pick<T>(p.CT, p.f_CT);
    A.rhs_mode = p.rhs_mode;
    A.stage = p.stage;
    A.ebase = 0;
    A.ctl = ctl;
    __syncwarp();
    constexpr int NA = PF ? 3 : 1;
    T ws[NA];
#pragma unroll
    for (int q = 0; q < NA; q++) ws[q] = T(0);
    const T w0 = tiles1d<T, SYS, SCH, PF>(A, s_U[warp], s_gp[warp], s_gm[warp], s_pr[warp], s_coef[warp],
                                          p.tile_lo + blockIdx.x * nw + warp, gridDim.x * nw,
                                          p.tile_hi > 0 ? p.tile_hi : 0x7fffffff, ws);
    if constexpr (!PF) ws[0] = w0;

    if (!p.rhs_mode) {
#pragma unroll
        for (int q = 0; q < NA; q++) {
            ws[q] = warp_max(ws[q]);
            if (lane == 0) s_red[q][warp] = ws[q];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int so = (p.stage + 1) % 3;
#pragma unroll
            for (int q = 0; q < NA; q++) {
                T v = s_red[q][0];
                for (int w = 1; w < nw; w++) v = fmax(v, s_red[q][w]);
                atomicMax(&ctl->amax[so][q], (unsigned long long)__double_as_longlong((double)v));
            }
            finish_launch(ctl, so, (p.stage + 2) % 3, p.stage == 2 && !fixed && !p.partial,
                          p.stage == 2 && !fixed && !p.partial, false, p.alpha_rec, NA);
        }
    }
}

// ==========================================================================
// FP32 stage kernel with paired splits.  The '+' split at cell j-3+t and the
// '-' split at cell j+4-t share one float2 lane pair, P[t] = (q+_{j-3+t},
// q-_{j+4-t}), t = 0..6.  With this mirror pairing the '-' window and the '-'
// polynomial are element-wise aligned with the '+' ones, so the projection,
// the smoothness measure and the polynomial run as packed f32x2 operations.
// Cutoff codes of the six (split, field) groups sit in 5-bit slots of one
// word (code bits 3..1 = d0, d1, d2; bits 4 and 0 receive the neighbours'
// bits), so all six Delta_i come out of three whole-word bit operations and
// index a Delta-addressed coefficient table directly.
// ==========================================================================
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// FP32 round-off floor of epsilon.  The characteristic values of a window
// carry rounding errors of a few ulps of their magnitude Q = max|w|, which
// reach 12 beta (3 a^2 + 13 b^2) and tau as noise up to ~1.3e4 (2^-24 Q)^2
// = 5e-11 Q^2.  With epsilon = dx^3 below that level (fine grids in FP32) the
// noise alone makes chi random in flat regions, switches stencils (including
// the downwind-biased candidates) and grows into grid-scale oscillations --
// the failure the choice of epsilon is meant to prevent.  In FP32 the epsilon
// of 12 beta is therefore max(12 dx^3, 2^-24 Q^2): the FP32 unit round-off
// times Q^2, three orders above that noise, so that tau/(beta + eps) stays
// below 1e-3 for pure noise, while jumps above ~1e-4 Q are measured as
// before.  (FP64 round-off is ~1e-32 Q^2, far below dx^3: FP64 keeps
// epsilon = dx^3.)
constexpr float RO_FLOOR12 = 5.9604644775390625e-08f;  // 2^-24 (epsilon of 12 beta)
constexpr float RO_FLOOR4 = RO_FLOOR12 / 3.f;           // the same floor for 4 beta

// Cutoff codes of a '+' window (.x) and a '-' window (.y), w0..w4 in upwind
// order.  beta is scaled by 4 (a^2 + 13/3 b^2) with eps4 = 4 eps, which
// leaves gamma unchanged; chi_k is evaluated as x_k^6 / sum x^6 with
// x = g / g_max in (0, 1] so that nothing overflows.  Returns the codes
// d0<<2 | d1<<1 | d2 of both splits.
// tau of both windows (Eq. tau5 on the 4-beta scale below), with the same
// operations as in cutoff2, for the keep-all test of all fields at once
__device__ __forceinline__ float2 tau_pair(float2 w0, float2 w1, float2 w2, float2 w3, float2 w4) {
    const float2 s0a = __ffma2_rn(f2(3.f), w2, __ffma2_rn(f2(-4.f), w1, w0));
    const float2 s0b = __fadd2_rn(__ffma2_rn(f2(-2.f), w1, w0), w2);
    const float2 s2a = __ffma2_rn(f2(3.f), w2, __ffma2_rn(f2(-4.f), w3, w4));
    const float2 s2b = __fadd2_rn(__ffma2_rn(f2(-2.f), w3, w2), w4);
    const float2 b0 = __ffma2_rn(s0b, __fmul2_rn(f2(13.f / 3.f), s0b), __fmul2_rn(s0a, s0a));
    const float2 b2 = __ffma2_rn(s2b, __fmul2_rn(f2(13.f / 3.f), s2b), __fmul2_rn(s2a, s2a));
    const float2 td = __ffma2_rn(f2(-1.f), b2, b0);
    return make_float2(fabsf(td.x), fabsf(td.y));
}

__device__ __forceinline__ void cutoff2(float2 w0, float2 w1, float2 w2, float2 w3, float2 w4, float eps4, float CT,
                                        float kt, unsigned &cp, unsigned &cm) {
    const float2 s0a = __ffma2_rn(f2(3.f), w2, __ffma2_rn(f2(-4.f), w1, w0));
    const float2 s0b = __fadd2_rn(__ffma2_rn(f2(-2.f), w1, w0), w2);
    const float2 s2a = __ffma2_rn(f2(3.f), w2, __ffma2_rn(f2(-4.f), w3, w4));
    const float2 s2b = __fadd2_rn(__ffma2_rn(f2(-2.f), w3, w2), w4);
    const float2 b0 = __ffma2_rn(s0b, __fmul2_rn(f2(13.f / 3.f), s0b), __fmul2_rn(s0a, s0a));
    const float2 b2 = __ffma2_rn(s2b, __fmul2_rn(f2(13.f / 3.f), s2b), __fmul2_rn(s2a, s2a));
    const float2 td = __ffma2_rn(f2(-1.f), b2, b0);
    const float2 tau = make_float2(fabsf(td.x), fabsf(td.y));
    // every stencil kept (see keep_all_factor): beta_min >= 0, so tau < kt eps
    // already suffices, before beta_1 is formed
    if (tau.x < kt * eps4 && tau.y < kt * eps4) {
        cp = 7u;
        cm = 7u;
        return;
    }
    const float2 s1a = __ffma2_rn(f2(-1.f), w3, w1);
    const float2 s1b = __fadd2_rn(__ffma2_rn(f2(-2.f), w2, w1), w3);
    const float2 b1 = __ffma2_rn(s1b, __fmul2_rn(f2(13.f / 3.f), s1b), __fmul2_rn(s1a, s1a));
    const float bmx = fminf(fminf(b0.x, b1.x), b2.x), bmy = fminf(fminf(b0.y, b1.y), b2.y);
    // every stencil of both windows kept (see keep_all_factor); tested first
    // with the unfloored epsilon, since the floor below only raises it
    if (tau.x < kt * (bmx + eps4) && tau.y < kt * (bmy + eps4)) {
        cp = 7u;
        cm = 7u;
        return;
    }
    // epsilon no smaller than the FP32 round-off level of the window (see
    // RO_FLOOR12), so that rounding noise cannot trigger the cutoff
    const float qx = fmaxf(fmaxf(fabsf(w0.x), fabsf(w2.x)), fabsf(w4.x));
    const float qy = fmaxf(fmaxf(fabsf(w0.y), fabsf(w2.y)), fabsf(w4.y));
    const float2 ro = __fmul2_rn(f2(RO_FLOOR4), __fmul2_rn(make_float2(qx, qy), make_float2(qx, qy)));
    const float2 ee = make_float2(fmaxf(eps4, ro.x), fmaxf(eps4, ro.y));
    if (tau.x < kt * (bmx + ee.x) && tau.y < kt * (bmy + ee.y)) {
        cp = 7u;
        cm = 7u;
        return;
    }
    const float2 d0 = __fadd2_rn(b0, ee), d1 = __fadd2_rn(b1, ee), d2 = __fadd2_rn(b2, ee);
    const float2 g0 = __ffma2_rn(tau, make_float2(rcp_approx(d0.x), rcp_approx(d0.y)), f2(1.f));
    const float2 g1 = __ffma2_rn(tau, make_float2(rcp_approx(d1.x), rcp_approx(d1.y)), f2(1.f));
    const float2 g2 = __ffma2_rn(tau, make_float2(rcp_approx(d2.x), rcp_approx(d2.y)), f2(1.f));
    const float2 rg = make_float2(rcp_approx(fmaxf(fmaxf(g0.x, g1.x), g2.x)), rcp_approx(fmaxf(fmaxf(g0.y, g1.y), g2.y)));
    float2 x0 = __fmul2_rn(g0, rg), x1 = __fmul2_rn(g1, rg), x2 = __fmul2_rn(g2, rg);
    x0 = __fmul2_rn(x0, x0);
    x1 = __fmul2_rn(x1, x1);
    x2 = __fmul2_rn(x2, x2);
    const float2 y0 = __fmul2_rn(__fmul2_rn(x0, x0), x0);
    const float2 y1 = __fmul2_rn(__fmul2_rn(x1, x1), x1);
    const float2 y2 = __fmul2_rn(__fmul2_rn(x2, x2), x2);
    const float2 thr = __fmul2_rn(f2(CT), __fadd2_rn(__fadd2_rn(y0, y1), y2));
    cp = ((y0.x < thr.x) ? 0u : 4u) | ((y1.x < thr.x) ? 0u : 2u) | ((y2.x < thr.x) ? 0u : 1u);
    cm = ((y0.y < thr.y) ? 0u : 4u) | ((y1.y < thr.y) ? 0u : 2u) | ((y2.y < thr.y) ? 0u : 1u);
}

// FP32 max characteristic speed with approximate reciprocal and square root
// (it only sets alpha and dt); flags as wavespeed1d.
template <int SYS>
__device__ __forceinline__ float wavespeed1d_fast(const float *Uc, float gm1, float gamma, float a, int *flag) {
    if (SYS == SYS_ADV) return fabsf(a);
    if (SYS == SYS_BURGERS) {
        if (!isfinite(Uc[0])) *flag |= ERR_NONFINITE;
        return fabsf(Uc[0]);
    }
    const float ri = rcp_approx(Uc[0]);
    const float u = Uc[1] * ri;
    const float p = gm1 * (Uc[2] - 0.5f * Uc[1] * u);
    const float c2 = gamma * p * ri;
    const float c = c2 * rsqrtf(c2);
    if (!isfinite(Uc[0]) || !isfinite(Uc[1]) || !isfinite(Uc[2]))
        *flag |= ERR_NONFINITE;
    else if (!(Uc[0] > 0.f) || !(p > 0.f))
        *flag |= ERR_NONPHYSICAL;
    return fabsf(u) + c;
}

// |u - c|, |u|, |u + c| of one FP32 1D Euler cell with wavespeed1d_fast's
// operations and flags (per-field alphas of a stage's output).
__device__ __forceinline__ void wavespeeds1d_fast(const float *Uc, float gm1, float gamma, float w[3], int *flag) {
    const float ri = rcp_approx(Uc[0]);
    const float u = Uc[1] * ri;
    const float p = gm1 * (Uc[2] - 0.5f * Uc[1] * u);
    const float c2 = gamma * p * ri;
    const float c = c2 * rsqrtf(c2);
    if (!isfinite(Uc[0]) || !isfinite(Uc[1]) || !isfinite(Uc[2]))
        *flag |= ERR_NONFINITE;
    else if (!(Uc[0] > 0.f) || !(p > 0.f))
        *flag |= ERR_NONPHYSICAL;
    w[0] = fabsf(u - c);
    w[1] = fabsf(u);
    w[2] = fabsf(u + c);
}

// Conversions between the FP64 state and the FP32 reconstruction of the
// mixed-precision form, by integer operations on the bit patterns, so that
// they use the integer pipe rather than the FP64 pipe (whose rate on GB300 is
// 1/64 of FP32).  to_f32: truncation toward zero (exact for every double
// that a float represents; |x| < 2^-126 flushes to a signed zero; overflow
// gives infinity, NaN stays NaN).  to_f64: exact for normal floats and zeros
// (subnormal floats flush to a signed zero).  Overloads on float are the
// identity, for the FP32 state.
__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned e = (hi >> 20) & 0x7ffu, sign = hi & 0x80000000u;
    unsigned f = sign | (((hi & 0x7fffffffu) - (896u << 20)) << 3) | (lo >> 29);
    if (e < 897u) f = sign;
    if (e > 1150u) f = sign | ((e == 2047u && ((hi & 0xfffffu) | lo)) ? 0x7fc00000u : 0x7f800000u);
    return __uint_as_float(f);
}
__device__ __forceinline__ double to_f64(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu, sign = u & 0x80000000u;
    unsigned hi = sign | (((u & 0x7fffffffu) >> 3) + (896u << 20)), lo = u << 29;
    if (e == 0u) {
        hi = sign;
        lo = 0u;
    }
    if (e == 255u) hi = sign | 0x7ff00000u | ((u & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)lo);
}

// Slot masks of the 6 x 5-bit word (see above).
constexpr unsigned SLOT_HI = 0x21084210u;   // bit 4 of every slot
constexpr unsigned SLOT_MID = 0x1CE739CEu;  // bits 3..1 of every slot
constexpr unsigned SLOT_LO = 0x02108421u;   // bit 0 of every slot
constexpr unsigned SLOT_PLUS = 0x00007FFFu; // slots 0..2 ('+' split)

// Delta-indexed coefficient table: row D holds Table co2's row for Table co3's
// choice at D ("no exist" rows get f11); filled by a 256-thread CTA.
__device__ __forceinline__ void fill_delta_table(float (*s_cf)[8]) {
    for (int q = threadIdx.x; q < 256; q += blockDim.x) {
        const int row = q >> 3, t = q & 7;
        int m = lut_select(row);
        if (m == 15) m = 11;
        s_cf[row][t] = t < 7 ? coef<float>(7 * m + t) : 0.f;
    }
}

// TENO5 counterpart: row D (only bits 3..1 = d0, d1, d2 are ever set) holds
// the Table co1 row of the code on taps 1..5 of the seven-tap layout.
__device__ __forceinline__ void fill_delta_table5(float (*s_cf)[8]) {
    for (int q = threadIdx.x; q < 256; q += blockDim.x) {
        const int row = q >> 3, t = q & 7;
        const unsigned code = ((row >> 3) & 1) | (((row >> 2) & 1) << 1) | (((row >> 1) & 1) << 2);
        int r = sel5(code);
        if (r == 7) r = 0;
        s_cf[row][t] = (t >= 1 && t <= 5) ? coef5<float>(5 * r + t - 1) : 0.f;
    }
}

// Five-bit code of a slot of the FP32 word (bits 3..1 = d0, d1, d2) in the
// oracle's d0 | d1<<1 | d2<<2 form (TENO5 masks).
__device__ __forceinline__ unsigned slot_code(unsigned s) {
    return ((s >> 3) & 1u) | (((s >> 2) & 1u) << 1) | (((s >> 1) & 1u) << 2);
}

// --------------------------------------------------------------------------
// FP32 Roe frame and back projection of one 1D Euler face (Remark 3), with
// every rounding written out: u~ = fma(s_l, u_l, s_r u_r) w, H~ likewise;
// the shared products b1 u~, u~^2 / 2 and b2 rounded on their own; u~/c~
// fused into L00 and L20; the back projection a f0 + b f1 + c f2 =
// fma(c, f2, fma(a, f0, b f1)) with H~ -+ u~ c~ fused.  (This is the order in
// which the compiler had contracted the same expressions written plainly;
// spelling it out keeps the FP32 results fixed whatever a compiler's
// contraction heuristics do.)  The FP32 1D stage kernels compute the frame
// with these roundings, so their results agree bit for bit.
// --------------------------------------------------------------------------
struct RoeF32 {
    float ut, cc, Ht;
    float L[3][3];  // rows: left eigenvectors of u-c, u, u+c
    int flag;       // ERR_NONPHYSICAL / ERR_NONFINITE when c^2 <= 0
};

__device__ __forceinline__ RoeF32 roe_frame_f32(float ul, float ur, float Hl, float Hr, float sl, float sr,
                                                float gm1) {
    RoeF32 F;
    const float w = rcp_approx(sl + sr);
    F.ut = __fmul_rn(__fmaf_rn(sl, ul, __fmul_rn(sr, ur)), w);
    F.Ht = __fmul_rn(__fmaf_rn(sl, Hl, __fmul_rn(sr, Hr)), w);
    const float q = __fmul_rn(__fmul_rn(0.5f, F.ut), F.ut);  // u~^2 / 2
    const float c2 = __fmul_rn(gm1, __fadd_rn(F.Ht, -q));
    const float rc = rsqrtf(c2);  // 1/c
    F.cc = __fmul_rn(c2, rc);
    const float b1 = __fmul_rn(gm1, __fmul_rn(rc, rc));
    const float b2 = __fmul_rn(q, b1);
    const float b1u = __fmul_rn(b1, F.ut);
    F.L[0][0] = __fmul_rn(0.5f, __fmaf_rn(F.ut, rc, b2));
    F.L[0][1] = __fmul_rn(-0.5f, __fadd_rn(b1u, rc));
    F.L[0][2] = __fmul_rn(0.5f, b1);
    F.L[1][0] = __fadd_rn(1.f, -b2);
    F.L[1][1] = b1u;
    F.L[1][2] = -b1;
    F.L[2][0] = __fmul_rn(0.5f, __fmaf_rn(-F.ut, rc, b2));
    F.L[2][1] = __fmul_rn(-0.5f, __fadd_rn(b1u, -rc));
    F.L[2][2] = F.L[0][2];
    F.flag = (c2 > 0.f) ? 0 : (isfinite(c2) ? ERR_NONPHYSICAL : ERR_NONFINITE);
    return F;
}

// R (columns: eigenvectors of u-c, u, u+c) times the characteristic fluxes f
__device__ __forceinline__ void back_project_f32(const RoeF32 &F, const float f[3], float fh[3]) {
    const float ut = F.ut, cc = F.cc, Ht = F.Ht;
    fh[0] = __fadd_rn(__fadd_rn(f[0], f[1]), f[2]);
    fh[1] = __fmaf_rn(__fadd_rn(ut, cc), f[2], __fmaf_rn(__fadd_rn(ut, -cc), f[0], __fmul_rn(ut, f[1])));
    fh[2] = __fmaf_rn(__fmaf_rn(ut, cc, Ht), f[2],
                      __fmaf_rn(__fmaf_rn(-ut, cc, Ht), f[0], __fmul_rn(__fmul_rn(__fmul_rn(0.5f, ut), ut), f[1])));
}

#ifndef T7_F32_MINB
#define T7_F32_MINB 2  // resident CTAs per SM the FP32 stage kernel is compiled for
#endif
// Waves of resident CTAs an FP32 launch's grid covers (see stage_grid): 1D
// Euler stages, scalar-law stages, 2D x sweeps
#ifndef T7_WAVES_EULER
#define T7_WAVES_EULER 2
#endif
#ifndef T7_WAVES_SCALAR
#define T7_WAVES_SCALAR 1
#endif
#ifndef T7_WAVES_X2D
#define T7_WAVES_X2D 2
#endif

// FP32 warp-tile sweep (paired splits); same contract as tiles1d.  s_cf is
// the Delta-indexed coefficient table [32][8].  S is the state type: float,
// or double for the mixed-precision form, where the state stays FP64, the
// reconstruction up to the face flux runs in FP32 and the flux difference and
// the RK combination run in FP64 -- each face flux enters both neighbouring
// cells as the same FP64 value, so domain sums are conserved to FP64 round-off.  The raw state of a warp
// tile's staged cells (lane and lane + 32) is loaded one tile ahead, and U^n
// of the tile's own cells at the start of the tile, so DRAM latency overlaps
// the face work.
template <int SYS, int SCH = SCH_TENO7EXT, typename S = float>
__device__ __forceinline__ float tiles1d_f32(const TileArgs<float> &A, float (*sU)[WC], float (*sgp)[WC],
                                             float (*sgm)[WC], float (*spr)[WC], const float (*s_cf)[8], int tile0,
                                             int tstride, int tile_end = 0x7fffffff) {
    constexpr bool MIXED = sizeof(S) == 8;
    constexpr int M = (SYS == SYS_EULER1D) ? 3 : 1;
    constexpr int NP = (SYS == SYS_EULER1D) ? 3 : 1;
    const int lane = threadIdx.x & 31;
    const float alpha = A.alpha, dtT = A.dtT, gamma = A.gamma, gm1 = A.gm1, a = A.a;
    // (TENO5's epsilon of 1e-40 is below FLT_MIN: raise it to FLT_MIN so that
    // beta + eps is never flushed to zero by the approximate reciprocal)
    const float eps4 = SCH == SCH_TENO5 ? fmaxf(4.f * A.eps, 1.17549435e-38f) : 4.f * A.eps, CT = A.CT;
    const float kt = keep_all_factor(CT);
    const float idx = 1.f / A.f_dx;
    const S *Us = reinterpret_cast<const S *>(A.Us);
    const S *U0 = reinterpret_cast<const S *>(A.U0);
    S *out = reinterpret_cast<S *>(A.out);
    const double idxD = 1.0 / A.dx, cD = A.dtD * idxD;
    const int n = A.n;
    const size_t cs = A.cs;
    const int ntiles = min((n + WT - 1) / WT, tile_end);  // tiles tile0, tile0 + tstride, ... below it
    DevCtl *ctl = A.ctl;
    float wsmax = 0.f;
    // Software pipelining: the raw state of a warp tile's staged cells (lane
    // and lane + 32) is loaded one tile ahead, and U^n of the tile's own cells
    // at the start of the tile, so DRAM latency overlaps the face work.
    // (held in the state type and rounded to float only when the tile is
    // used, so that a mixed-precision load is not waited for at once)
    S ua[M], ub[M];
    auto load_tile = [&](int tile) {
        const int c0 = tile * WT;
        int ga = c0 - 5 + lane, gb = c0 - 5 + 32 + lane;
        if (!(c0 >= 5 && c0 + WS - 5 <= n)) {
            // a staged cell outside the grid (first and last tiles; warp-uniform)
            if (ga < 0 || ga >= n) ga = ghost_or_halo(ga, n, A.bc_lo, A.bc_hi, A.halo);
            if (gb < 0 || gb >= n) gb = ghost_or_halo(gb, n, A.bc_lo, A.bc_hi, A.halo);
        }
#pragma unroll
        for (int k = 0; k < M; k++) {
            ua[k] = Us[(size_t)k * cs + chk(ctl, ga, A.halo ? -HALO_CELLS : 0, n + (A.halo ? HALO_CELLS : 0))];
            ub[k] = (lane < WS - 32) ? Us[(size_t)k * cs + chk(ctl, gb, A.halo ? -HALO_CELLS : 0,
                                                               n + (A.halo ? HALO_CELLS : 0))]
                                     : S(0);
        }
    };
    int tile = tile0;
    if (tile < ntiles) load_tile(tile);

    for (; tile < ntiles; tile += tstride) {
        const int c0 = tile * WT;
        const int jc = c0 - 2 + lane;  // this lane's cell (if it updates one)
        S u0r[M];
        if (!A.rhs_mode && A.stage > 0) {
            const int ic = jc < n ? jc : n - 1;
#pragma unroll
            for (int k = 0; k < M; k++) u0r[k] = U0[(size_t)k * cs + chk(ctl, ic < 0 ? 0 : ic, 0, n)];
        }
        // mixed: the FP64 stage input of the tile's own cells, which the RK
        // update needs unrounded, loaded here so that its latency overlaps the
        // face work (the staged copy is rounded to float)
        S usr[M];
        if (MIXED && !A.rhs_mode) {
            const int ic = jc < n ? jc : n - 1;
#pragma unroll
            for (int k = 0; k < M; k++) usr[k] = Us[(size_t)k * cs + chk(ctl, ic < 0 ? 0 : ic, 0, n)];
        }
        float Ucur[2][M];
#pragma unroll
        for (int k = 0; k < M; k++) {
            Ucur[0][k] = to_f32(ua[k]);
            Ucur[1][k] = to_f32(ub[k]);
        }
        if (tile + tstride < ntiles) load_tile(tile + tstride);
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const int c = lane + 32 * r;
            if (c >= WS) break;
            float U[M], F[M];
#pragma unroll
            for (int k = 0; k < M; k++) U[k] = Ucur[r][k];
            if (SYS == SYS_ADV) {
                F[0] = a * U[0];
            } else if (SYS == SYS_BURGERS) {
                F[0] = 0.5f * U[0] * U[0];
            } else {
                const float ri = rcp_approx(U[0]);
                const float u = U[1] * ri;
                const float pr = gm1 * (U[2] - 0.5f * U[1] * u);
                F[0] = U[1];
                F[1] = U[1] * u + pr;
                F[2] = u * (U[2] + pr);
                spr[0][c] = u;
                spr[NP > 1 ? 1 : 0][c] = (U[2] + pr) * ri;
                spr[NP > 2 ? 2 : 0][c] = U[0] * rsqrtf(U[0]);
            }
#pragma unroll
            for (int k = 0; k < M; k++) {
                sU[k][c] = U[k];
                if (SYS == SYS_ADV) {
                    // linear flux: (a +- alpha) / 2 is exactly 0 for the
                    // downwind split (alpha = |a|), so that split is exactly
                    // zero rather than FMA round-off noise
                    sgp[k][c] = (0.5f * (a + alpha)) * U[k];
                    sgm[k][c] = (0.5f * (a - alpha)) * U[k];
                } else {
                    sgp[k][c] = 0.5f * fmaf(alpha, U[k], F[k]);
                    sgm[k][c] = 0.5f * fmaf(-alpha, U[k], F[k]);
                }
            }
        }
        __syncwarp();

        const int j = c0 - 2 + lane;
        float2 L2[M][M];
        float ut = 0.f, cc = 0.f, Ht = 0.f;
        int flag = 0;
        if (SYS == SYS_EULER1D) {
            const RoeF32 F = roe_frame_f32(spr[0][lane + 3], spr[0][lane + 4], spr[NP > 1 ? 1 : 0][lane + 3],
                                           spr[NP > 1 ? 1 : 0][lane + 4], spr[NP > 2 ? 2 : 0][lane + 3],
                                           spr[NP > 2 ? 2 : 0][lane + 4], gm1);
            ut = F.ut;
            cc = F.cc;
            Ht = F.Ht;
#pragma unroll
            for (int k = 0; k < M; k++)
#pragma unroll
                for (int c = 0; c < M; c++) L2[k][c] = f2(F.L[k % 3][c % 3]);
            flag |= F.flag;
        }

        float2 P[M][7];
#pragma unroll
        for (int t = 0; t < 7; t++) {
            if (SCH == SCH_TENO5 && (t == 0 || t == 6)) {  // five-point stencils
#pragma unroll
                for (int k = 0; k < M; k++) P[k][t] = f2(0.f);
                continue;
            }
            float2 g[M];
#pragma unroll
            for (int c = 0; c < M; c++) g[c] = make_float2(sgp[c][lane + t], sgm[c][lane + 7 - t]);
#pragma unroll
            for (int k = 0; k < M; k++) {
                if (M == 1) {
                    P[k][t] = g[0];
                } else {
                    float2 q = __fmul2_rn(L2[k][0], g[0]);
#pragma unroll
                    for (int c = 1; c < M; c++) q = __ffma2_rn(L2[k][c], g[c], q);
                    P[k][t] = q;
                }
            }
        }
        unsigned word = 0;
#pragma unroll
        for (int k = 0; k < M; k++) {
            unsigned cp, cm;
            cutoff2(P[k][1], P[k][2], P[k][3], P[k][4], P[k][5], eps4, CT, kt, cp, cm);
            word |= (cp << (5 * k + 1)) | (cm << (5 * (3 + k) + 1));
        }
        unsigned D;
        if constexpr (SCH == SCH_TENO5) {
            D = word;  // TENO5: own bits only
        } else {
            const unsigned wl = __shfl_up_sync(0xffffffffu, word, 1);
            const unsigned wr = __shfl_down_sync(0xffffffffu, word, 1);
            const unsigned Dp = ((wl << 1) & SLOT_HI) | (word & SLOT_MID) | ((wr >> 1) & SLOT_LO);
            const unsigned Dm = ((wr << 1) & SLOT_HI) | (word & SLOT_MID) | ((wl >> 1) & SLOT_LO);
            D = (Dp & SLOT_PLUS) | (Dm & ~SLOT_PLUS);
        }
        const bool face_out = lane >= 1 && lane <= 30;

        float f[M];
        constexpr unsigned ALL_SMOOTH = SCH == SCH_TENO5 ? ((M == 3) ? SLOT_MID : ((14u) | (14u << 15)))
                                                         : ((M == 3) ? 0x3FFFFFFFu : ((31u) | (31u << 15)));
        if (SCH == SCH_TENO5 && (D & ALL_SMOOTH) == ALL_SMOOTH) {
            // every split of every field selects Table co1's fifth-order row
#pragma unroll
            for (int k = 0; k < M; k++) {
                float2 s = __fmul2_rn(f2(1.f / 30.f), P[k][1]);
                s = __ffma2_rn(f2(-13.f / 60.f), P[k][2], s);
                s = __ffma2_rn(f2(47.f / 60.f), P[k][3], s);
                s = __ffma2_rn(f2(9.f / 20.f), P[k][4], s);
                s = __ffma2_rn(f2(-1.f / 20.f), P[k][5], s);
                f[k] = s.x + s.y;
            }
        } else if (SCH == SCH_TENO5) {
#pragma unroll
            for (int k = 0; k < M; k++) {
                const float *cp = s_cf[(D >> (5 * k)) & 31u];
                const float *cm = s_cf[(D >> (5 * (3 + k))) & 31u];
                float2 s = __fmul2_rn(make_float2(cp[1], cm[1]), P[k][1]);
#pragma unroll
                for (int t = 2; t < 6; t++) s = __ffma2_rn(make_float2(cp[t], cm[t]), P[k][t], s);
                f[k] = s.x + s.y;
            }
        } else if ((D & ALL_SMOOTH) == ALL_SMOOTH) {
            // every split of every field selects f0 (the seventh-order polynomial)
#pragma unroll
            for (int k = 0; k < M; k++) {
                float2 s = __fmul2_rn(f2(-1.f / 140.f), P[k][0]);
                s = __ffma2_rn(f2(5.f / 84.f), P[k][1], s);
                s = __ffma2_rn(f2(-101.f / 420.f), P[k][2], s);
                s = __ffma2_rn(f2(319.f / 420.f), P[k][3], s);
                s = __ffma2_rn(f2(107.f / 210.f), P[k][4], s);
                s = __ffma2_rn(f2(-19.f / 210.f), P[k][5], s);
                s = __ffma2_rn(f2(1.f / 105.f), P[k][6], s);
                f[k] = s.x + s.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < M; k++) {
                const float *cp = s_cf[(D >> (5 * k)) & 31u];
                const float *cm = s_cf[(D >> (5 * (3 + k))) & 31u];
                float2 s = __fmul2_rn(make_float2(cp[0], cm[0]), P[k][0]);
#pragma unroll
                for (int t = 1; t < 7; t++) s = __ffma2_rn(make_float2(cp[t], cm[t]), P[k][t], s);
                f[k] = s.x + s.y;
            }
        }
        if (A.masks && face_out && j >= -1 && j <= n - 1) {
#pragma unroll
            for (int k = 0; k < M; k++) {
                const unsigned sp = (D >> (5 * k)) & 31u, sm = (D >> (5 * (3 + k))) & 31u;
                A.masks[(size_t)(0 * M + k) * (n + 1) + (j + 1)] = (uint8_t)(SCH == SCH_TENO5 ? slot_code(sp) : sp);
                A.masks[(size_t)(1 * M + k) * (n + 1) + (j + 1)] = (uint8_t)(SCH == SCH_TENO5 ? slot_code(sm) : sm);
            }
        }
        float fh[M];
        if (SYS == SYS_EULER1D) {
            RoeF32 F;
            F.ut = ut;
            F.cc = cc;
            F.Ht = Ht;
            float f3[3] = {f[0], f[1 % M], f[2 % M]}, fh3[3];
            back_project_f32(F, f3, fh3);
#pragma unroll
            for (int k = 0; k < M; k++) fh[k] = fh3[k % 3];
        } else {
            fh[0] = f[0];
        }
        if (flag && face_out && j >= -2 && j <= n) latch_error(ctl, flag, A.ebase + j);

        float fprev[M];
#pragma unroll
        for (int k = 0; k < M; k++) fprev[k] = __shfl_up_sync(0xffffffffu, fh[k], 1);
        const int i = j;
        if (MIXED && lane >= 2 && lane <= 30 && i < n) {
            // FP64 flux difference and RK combination (Shu-Osher form)
            double o[M];
            float of[M];
#pragma unroll
            for (int k = 0; k < M; k++) {
                const double d = to_f64(fprev[k]) - to_f64(fh[k]);
                if (A.rhs_mode) {
                    o[k] = d * idxD;
                } else {
                    const double v = fma(cD, d, (double)usr[k]);
                    if (A.stage == 0)
                        o[k] = v;
                    else if (A.stage == 1)
                        o[k] = fma(0.75, (double)u0r[k], 0.25 * v);
                    else
                        o[k] = fma(2.0 / 3.0, v, (1.0 / 3.0) * (double)u0r[k]);
                }
                out[(size_t)k * A.cso + chk(ctl, i, 0, n)] = (S)o[k];
                of[k] = to_f32(o[k]);
            }
            if (!A.rhs_mode) {
                int wflag = 0;
                wsmax = fmaxf(wsmax, wavespeed1d_fast<SYS>(of, gm1, gamma, a, &wflag));
                if (wflag) latch_error(ctl, wflag, A.ebase + i);
            }
        } else if (lane >= 2 && lane <= 30 && i < n) {
            float r[M];
#pragma unroll
            for (int k = 0; k < M; k++) r[k] = (fprev[k] - fh[k]) * idx;
            if (A.rhs_mode) {
#pragma unroll
                for (int k = 0; k < M; k++) out[(size_t)k * A.cso + chk(ctl, i, 0, n)] = r[k];
            } else {
                float o[M];
#pragma unroll
                for (int k = 0; k < M; k++) {
                    const float v = fmaf(dtT, r[k], sU[k][lane + 3]);
                    if (A.stage == 0) {
                        o[k] = v;
                    } else if (A.stage == 1) {
                        o[k] = fmaf(0.75f, (float)u0r[k], 0.25f * v);
                    } else {
                        // u0 + 2/3 (v - u0): float(1/3) + float(2/3) != 1 would
                        // grow the solution by 6e-8 every step
                        o[k] = fmaf(2.0f / 3.0f, v - (float)u0r[k], (float)u0r[k]);
                    }
                    out[(size_t)k * A.cso + chk(ctl, i, 0, n)] = (S)o[k];
                }
                int wflag = 0;
                wsmax = fmaxf(wsmax, wavespeed1d_fast<SYS>(o, gm1, gamma, a, &wflag));
                if (wflag) latch_error(ctl, wflag, A.ebase + i);
            }
        }
        __syncwarp();
    }

    return wsmax;
}

template <int SYS, int SCH, typename S = float>
__global__ void __launch_bounds__(WPB * 32, T7_F32_MINB) stage1d_f32_kernel(const Stage1D p) {
    constexpr int M = (SYS == SYS_EULER1D) ? 3 : 1;
    constexpr int NP = (SYS == SYS_EULER1D) ? 3 : 1;
    __shared__ float s_U[WPB][M][WC];
    __shared__ float s_gp[WPB][M][WC];
    __shared__ float s_gm[WPB][M][WC];
    __shared__ float s_pr[WPB][NP][WC];
    __shared__ __align__(16) float s_cf[32][8];  // row Delta: Table co2 row of Table co3's choice
    __shared__ float s_red[WPB];

    DevCtl *ctl = p.ctl;
    const bool fixed = p.dt_fixed > 0.0;
    if (!p.rhs_mode && !fixed && !ctl->active) return;  // uniform: the run has ended
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (SCH == SCH_TENO5)
        fill_delta_table5(s_cf);
    else
        fill_delta_table(s_cf);
    TileArgs<float> A;
    A.alpha = p.alpha_in ? (float)*p.alpha_in : ctl->alpha_f[p.slot_in][0];
    A.dtT = fixed ? p.f_dt_fixed : ctl->dt_f;
    A.dtD = fixed ? p.dt_fixed : ctl->dt;
    // (the pointers stay untyped here: the state type S may be double)
    // slab mode: cell 0 follows the padding (the RHS output dU/dt is unpadded)
    const int off = p.halo ? HALO_CELLS : 0, offo = p.rhs_mode ? 0 : off;
    A.Us = reinterpret_cast<const float *>(static_cast<const S *>(p.Us) + off);
    A.U0 = p.U0 ? reinterpret_cast<const float *>(static_cast<const S *>(p.U0) + off) : nullptr;
    A.out = reinterpret_cast<float *>(static_cast<S *>(p.out) + offo);
    A.masks = p.masks;
    A.n = p.n;
    A.cs = (size_t)p.n + 2 * off;
    A.cso = (size_t)p.n + 2 * offo;
    A.halo = p.halo;
    A.bc_lo = p.bc_lo;
    A.bc_hi = p.bc_hi;
    A.dx = p.dx;
    A.f_dx = p.f_dx;
    A.gamma = p.f_gamma;
    A.gm1 = p.f_gm1;
    A.a = p.f_a;
    A.eps = p.f_eps;
    A.CT = p.f_CT;
    A.rhs_mode = p.rhs_mode;
    A.stage = p.stage;
    A.ebase = 0;
    A.ctl = ctl;
    __syncthreads();
    float wsmax = tiles1d_f32<SYS, SCH, S>(A, s_U[warp], s_gp[warp], s_gm[warp], s_pr[warp], s_cf,
                                           p.tile_lo + blockIdx.x * nw + warp, gridDim.x * nw,
                                           p.tile_hi > 0 ? p.tile_hi : 0x7fffffff);

    if (!p.rhs_mode) {
        wsmax = warp_max(wsmax);
        if (lane == 0) s_red[warp] = wsmax;
        __syncthreads();
        if (threadIdx.x == 0) {
            float v = s_red[0];
#pragma unroll
            for (int w = 1; w < nw; w++) v = fmaxf(v, s_red[w]);
            const int so = (p.stage + 1) % 3;
            atomicMax(&ctl->amax[so][0], (unsigned long long)__double_as_longlong((double)v));
            finish_launch(ctl, so, (p.stage + 2) % 3, p.stage == 2 && !fixed && !p.partial,
                          p.stage == 2 && !fixed && !p.partial, false, p.alpha_rec);
        }
    }
}

// ==========================================================================
// FP32 stage kernel with paired FACES (grid-wide launches over the whole
// domain, FP32 state).  Lane l of a warp owns the two faces jA = c0-2+l and
// jB = c0+30+l of a WT2 = 61-cell warp tile (cells c0 .. c0+60), and every
// float2 holds (face A, face B).  The two splits run one after the other,
// each through the same projection, smoothness measure, neighbour exchange
// and polynomial as the paired-split kernel above, so every face sees the
// same per-element operations; the Roe frame, the back projection and the
// RK update of the two faces and cells run as packed f32x2 arithmetic, and a
// tile stages 71 cells for 61 updated (39 for 29 in the paired-split tiles).
// Neighbour faces: jA - 1 and jA + 1 are the A faces of lanes l-1 and l+1,
// except that face c0+30 (right of lane 31's A) is lane 0's B; jB - 1 and
// jB + 1 are the B faces of lanes l-1 and l+1, except that face c0+29 (left of
// lane 0's B) is lane 31's A.  Faces c0-2 (lane 0, A) and c0+61 (lane 31, B)
// lack a neighbour code and only serve their neighbours.
// Scalar advection with a = alpha > 0 (the host's dispatch guarantees it)
// reconstructs the '+' split only: the '-' split flux (a - alpha) u / 2 is
// identically zero, its windows are all zero, every stencil of them is kept
// and its polynomial is exactly zero.
// ==========================================================================
// 4-byte asynchronous global -> shared copies (cp.async, completion awaited
// by cp_async_wait_all)
static __device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
static __device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
static __device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

constexpr int WT2 = 61;  // cells updated per face-paired warp tile
constexpr int WS2 = 71;  // cells staged per face-paired warp tile (c0-5 .. c0+65)
// Staging rows of the face-paired kernel hold PAIRS (value of staged cell i,
// value of staged cell i + 32), i = 0 .. 38, so that one 64-bit shared load
// gives a tap of face A (lane l: cells from l) and of face B (cells from l + 32).
constexpr int WP2 = 40;

__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }

// PF (1D Euler, TENO7-ext): per-field alphas A.alf -- the staged rows hold the
// flux F (sgp) and the state (sU), and each field's split values are
// (L_k F +- alf[k] L_k U) / 2; ws3 receives the output's three characteristic
// speed maxima (the function then returns 0).
template <int SYS, int SCH, bool PF = false>
__device__ __forceinline__ float tiles1d_f32_fp(const TileArgs<float> &A, float2 (*sU)[WP2], float2 (*sgp)[WP2],
                                                float2 (*sgm)[WP2], float2 (*spr)[WP2], float2 (*su0)[32],
                                                const float (*s_cf)[8],
                                                int tile0, int tstride, float *ws3 = nullptr) {
    constexpr int M = (SYS == SYS_EULER1D) ? 3 : 1;
    constexpr int NP = (SYS == SYS_EULER1D) ? 3 : 1;
    constexpr bool PLUS_ONLY = SYS == SYS_ADV;
    constexpr int SH = 5 * M;                          // B slots sit SH bits above the A slots
    constexpr unsigned MASK_A = (1u << SH) - 1u;       // the A slots of a code word
    constexpr unsigned ALL_A = M == 3 ? 0x7FFFu : 31u; // every A slot all ones
    const int lane = threadIdx.x & 31;
    const float alpha = A.alpha, dtT = A.dtT, gamma = A.gamma, gm1 = A.gm1, a = A.a;
    const float eps4 = SCH == SCH_TENO5 ? fmaxf(4.f * A.eps, 1.17549435e-38f) : 4.f * A.eps, CT = A.CT;
    const float kt = keep_all_factor(CT);
    const float idx = 1.f / A.f_dx;
    const float *Us = A.Us;
    const float *U0 = A.U0;
    float *out = A.out;
    const int n = A.n;
    const size_t cs = A.cs, cso = A.cso;
    const int ntiles = (n + WT2 - 1) / WT2;
    DevCtl *ctl = A.ctl;
    float wsmax = 0.f;
    // raw state of the staged cells (rounds r = 0, 1, 2: cells c0-5+32r+lane),
    // loaded one tile ahead
    float ur[3][M];
    auto load_tile = [&](int tile) {
        const int c0 = tile * WT2;
        if (c0 >= 5 && c0 + WS2 - 5 <= n) {
            // every staged cell inside the grid (warp-uniform): no boundary map
#pragma unroll
            for (int r = 0; r < 3; r++) {
                const int g = c0 - 5 + 32 * r + lane;
#pragma unroll
                for (int k = 0; k < M; k++)
                    ur[r][k] = (r < 2 || lane < WS2 - 64) ? Us[(size_t)k * cs + chk(ctl, g, 0, n)] : 0.f;
            }
            return;
        }
#pragma unroll
        for (int r = 0; r < 3; r++) {
            int g = c0 - 5 + 32 * r + lane;
            if (g < 0 || g >= n) g = ghost_or_halo(g, n, A.bc_lo, A.bc_hi, A.halo);
            g = chk(ctl, g, A.halo ? -HALO_CELLS : 0, n + (A.halo ? HALO_CELLS : 0));
#pragma unroll
            for (int k = 0; k < M; k++) ur[r][k] = (r < 2 || lane < WS2 - 64) ? Us[(size_t)k * cs + g] : 0.f;
        }
    };
    int tile = tile0;
    if (tile < ntiles) load_tile(tile);

    for (; tile < ntiles; tile += tstride) {
        const int c0 = tile * WT2;
        const int jA = c0 - 2 + lane, jB = c0 + 30 + lane;  // faces, and the cells they update
        const bool updA = lane >= 2 && jA < n, updB = lane <= 30 && jB < n;
        // U^n of cells jA and jB (stages 1 and 2).  Euler: into su0 by
        // asynchronous copies, awaited only at the RK update, so that no
        // register holds them through the face computations (held in
        // registers, the loads were deferred to their use and waited for);
        // the scalar laws, with registers to spare, load them here
        constexpr bool U0_ASYNC = SYS == SYS_EULER1D;
        const bool use_u0 = !A.rhs_mode && A.stage > 0;
        float2 u0r[M];
        if (use_u0) {
            const int iA = jA < n ? jA : n - 1, iB = jB < n ? jB : n - 1;
            if constexpr (U0_ASYNC) {
#pragma unroll
                for (int k = 0; k < M; k++) {
                    cp_async4(&su0[k][lane].x, &U0[(size_t)k * cs + chk(ctl, iA < 0 ? 0 : iA, 0, n)]);
                    cp_async4(&su0[k][lane].y, &U0[(size_t)k * cs + chk(ctl, iB, 0, n)]);
                }
                cp_async_commit();
            } else {
#pragma unroll
                for (int k = 0; k < M; k++)
                    u0r[k] = make_float2(U0[(size_t)k * cs + chk(ctl, iA < 0 ? 0 : iA, 0, n)], U0[(size_t)k * cs + chk(ctl, iB, 0, n)]);
            }
        }
        float Ucur[3][M];
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int k = 0; k < M; k++) Ucur[r][k] = ur[r][k];
        if (tile + tstride < ntiles) load_tile(tile + tstride);
        // staged values (primitives, state, split fluxes) of the cells of rounds
        // r = 0, 1, 2 (staged cells lane, lane + 32, lane + 64).  Pair i =
        // (staged cell i, staged cell i + 32): after round 1 lane l writes pair l
        // (rounds 0, 1), after round 2 lanes l < 7 write pair l + 32 (rounds
        // 1, 2), one 64-bit store each
        float vpr[2][NP], vU[2][M], vgp[2][M], vgm[2][M];
#pragma unroll
        for (int r = 0; r < 3; r++) {
            const int c = lane + 32 * r;
            if (c >= WS2) break;
            const int h = r & 1;  // this round's slot; the previous round's is 1 - h
            float U[M], F[M];
#pragma unroll
            for (int k = 0; k < M; k++) U[k] = Ucur[r][k];
            if (SYS == SYS_ADV) {
                F[0] = a * U[0];
            } else if (SYS == SYS_BURGERS) {
                F[0] = 0.5f * U[0] * U[0];
            } else {
                const float ri = rcp_approx(U[0]);
                const float u = U[1] * ri;
                const float pr = gm1 * (U[2] - 0.5f * U[1] * u);
                F[0] = U[1];
                F[1] = U[1] * u + pr;
                F[2] = u * (U[2] + pr);
                vpr[h][0] = u;
                vpr[h][NP > 1 ? 1 : 0] = (U[2] + pr) * ri;
                vpr[h][NP > 2 ? 2 : 0] = U[0] * rsqrtf(U[0]);
            }
#pragma unroll
            for (int k = 0; k < M; k++) {
                vU[h][k] = U[k];
                if (SYS == SYS_ADV) {
                    vgp[h][k] = (0.5f * (a + alpha)) * U[k];
                } else {
                    if constexpr (PF) {
                        vgp[h][k] = F[k];
                        vgm[h][k] = F[k];  // (unused)
                    } else {
                        vgp[h][k] = 0.5f * fmaf(alpha, U[k], F[k]);
                        vgm[h][k] = 0.5f * fmaf(-alpha, U[k], F[k]);
                    }
                }
            }
            if (r == 0) continue;
            const int i = lane + 32 * (r - 1);  // the pair: (round r - 1, round r)
#pragma unroll
            for (int k = 0; k < M; k++) {
                sU[k][i] = make_float2(vU[1 - h][k], vU[h][k]);
                sgp[k][i] = make_float2(vgp[1 - h][k], vgp[h][k]);
                if (SYS != SYS_ADV) sgm[k][i] = make_float2(vgm[1 - h][k], vgm[h][k]);
            }
            if (SYS == SYS_EULER1D) {
#pragma unroll
                for (int q = 0; q < NP; q++) spr[q][i] = make_float2(vpr[1 - h][q], vpr[h][q]);
            }
        }
        __syncwarp();

        // ---- Roe frames of faces A and B (packed) --------------------------
        float2 L2[M][M];
        float2 ut = f2(0.f), cc = f2(0.f), Ht = f2(0.f);
        int flagA = 0, flagB = 0;
        if (SYS == SYS_EULER1D) {
            // the roundings of roe_frame_f32, for both faces at once
            const int P0 = NP > 1 ? 1 : 0, P1 = NP > 2 ? 2 : 0;
            const float2 ul = spr[0][lane + 3], ur_ = spr[0][lane + 4];
            const float2 Hl = spr[P0][lane + 3], Hr = spr[P0][lane + 4];
            const float2 sl = spr[P1][lane + 3], sr = spr[P1][lane + 4];
            const float2 ssum = __fadd2_rn(sl, sr);
            const float2 w = make_float2(rcp_approx(ssum.x), rcp_approx(ssum.y));
            ut = __fmul2_rn(__ffma2_rn(sl, ul, __fmul2_rn(sr, ur_)), w);
            Ht = __fmul2_rn(__ffma2_rn(sl, Hl, __fmul2_rn(sr, Hr)), w);
            const float2 q = __fmul2_rn(__fmul2_rn(f2(0.5f), ut), ut);  // u~^2 / 2
            const float2 c2 = __fmul2_rn(f2(gm1), __fadd2_rn(Ht, f2neg(q)));
            const float2 rc = make_float2(rsqrtf(c2.x), rsqrtf(c2.y));  // 1/c
            cc = __fmul2_rn(c2, rc);
            const float2 b1 = __fmul2_rn(f2(gm1), __fmul2_rn(rc, rc));
            const float2 b2 = __fmul2_rn(q, b1);
            const float2 b1u = __fmul2_rn(b1, ut);
            const float2 hb1 = __fmul2_rn(f2(0.5f), b1);
            L2[0][0] = __fmul2_rn(f2(0.5f), __ffma2_rn(ut, rc, b2));
            L2[0][1 % M] = __fmul2_rn(f2(-0.5f), __fadd2_rn(b1u, rc));
            L2[0][2 % M] = hb1;
            L2[1 % M][0] = __fadd2_rn(f2(1.f), f2neg(b2));
            L2[1 % M][1 % M] = b1u;
            L2[1 % M][2 % M] = f2neg(b1);
            L2[2 % M][0] = __fmul2_rn(f2(0.5f), __ffma2_rn(f2neg(ut), rc, b2));
            L2[2 % M][1 % M] = __fmul2_rn(f2(-0.5f), __fadd2_rn(b1u, f2neg(rc)));
            L2[2 % M][2 % M] = hb1;
            if (!(c2.x > 0.f)) flagA |= isfinite(c2.x) ? ERR_NONPHYSICAL : ERR_NONFINITE;
            if (!(c2.y > 0.f)) flagB |= isfinite(c2.y) ? ERR_NONPHYSICAL : ERR_NONFINITE;
        }

        // ---- the two splits: projection, cutoff, neighbour codes, polynomial
        float2 f[M];
        unsigned Dsave[2] = {0u, 0u};
#pragma unroll
        for (int s = 0; s < (PLUS_ONLY ? 1 : 2); s++) {
            float2 (*sg)[WP2] = (PF || s == 0) ? sgp : sgm;
            float2 P[M][7];
            if constexpr (PF) {
                // two passes over the taps, so that one tap's loads are live at a
                // time: P <- L_k U, then P <- (L_k F +- alf[k] P) / 2
#pragma unroll
                for (int t = 0; t < 7; t++) {
                    const int o = s == 0 ? lane + t : lane + 7 - t;
                    float2 gu[M];
#pragma unroll
                    for (int c = 0; c < M; c++) gu[c] = sU[c][o];
#pragma unroll
                    for (int k = 0; k < M; k++) {
                        float2 lu = __fmul2_rn(L2[k][0], gu[0]);
#pragma unroll
                        for (int c = 1; c < M; c++) lu = __ffma2_rn(L2[k][c], gu[c], lu);
                        P[k][t] = lu;
                    }
                }
#pragma unroll
                for (int t = 0; t < 7; t++) {
                    const int o = s == 0 ? lane + t : lane + 7 - t;
                    float2 g[M];
#pragma unroll
                    for (int c = 0; c < M; c++) g[c] = sgp[c][o];
#pragma unroll
                    for (int k = 0; k < M; k++) {
                        float2 lf = __fmul2_rn(L2[k][0], g[0]);
#pragma unroll
                        for (int c = 1; c < M; c++) lf = __ffma2_rn(L2[k][c], g[c], lf);
                        P[k][t] = __fmul2_rn(f2(0.5f), __ffma2_rn(f2(s == 0 ? A.alf[k] : -A.alf[k]), P[k][t], lf));
                    }
                }
            } else {
#pragma unroll
            for (int t = 0; t < 7; t++) {
                if (SCH == SCH_TENO5 && (t == 0 || t == 6)) {
#pragma unroll
                    for (int k = 0; k < M; k++) P[k][t] = f2(0.f);
                    continue;
                }
                // '+': cells j-3+t; '-': cells j+4-t (mirror image about j+1/2)
                const int o = s == 0 ? lane + t : lane + 7 - t;
                float2 g[M];
#pragma unroll
                for (int c = 0; c < M; c++) g[c] = sg[c][o];
#pragma unroll
                for (int k = 0; k < M; k++) {
                    if (M == 1) {
                        P[k][t] = g[0];
                    } else {
                        float2 q = __fmul2_rn(L2[k][0], g[0]);
#pragma unroll
                        for (int c = 1; c < M; c++) q = __ffma2_rn(L2[k][c], g[c], q);
                        P[k][t] = q;
                    }
                }
            }
            }
            // Every stencil of every window kept (tau < kt eps, see
            // keep_all_factor) is tested for all fields at once, without
            // branches in between, so that the fields' measures overlap; the
            // per-window test below gives the same bits whenever this holds.
            bool keep_all = true;
#pragma unroll
            for (int k = 0; k < M; k++) {
                const float2 tau = tau_pair(P[k][1], P[k][2], P[k][3], P[k][4], P[k][5]);
                keep_all = keep_all && tau.x < kt * eps4 && tau.y < kt * eps4;
            }
            unsigned word = 0;
            if (keep_all) {
#pragma unroll
                for (int k = 0; k < M; k++) word |= (7u << (5 * k + 1)) | (7u << (SH + 5 * k + 1));
            } else {
#pragma unroll
                for (int k = 0; k < M; k++) {
                    unsigned cA, cB;
                    cutoff2(P[k][1], P[k][2], P[k][3], P[k][4], P[k][5], eps4, CT, kt, cA, cB);
                    word |= (cA << (5 * k + 1)) | (cB << (SH + 5 * k + 1));
                }
            }
            unsigned D;
            if constexpr (SCH == SCH_TENO5) {
                D = word;
            } else {
                const unsigned wl = __shfl_sync(0xffffffffu, word, (lane + 31) & 31);
                const unsigned wr = __shfl_sync(0xffffffffu, word, (lane + 1) & 31);
                // codes of each face's left and right neighbour faces, in its own slots
                const unsigned LW = lane == 0 ? (wl & MASK_A) | (wl << SH) : wl;
                const unsigned RW = lane == 31 ? (wr >> SH) | (wr & ~MASK_A) : wr;
                D = s == 0 ? (((LW << 1) & SLOT_HI) | (word & SLOT_MID) | ((RW >> 1) & SLOT_LO))
                           : (((RW << 1) & SLOT_HI) | (word & SLOT_MID) | ((LW >> 1) & SLOT_LO));
            }
            Dsave[s] = D;
            constexpr unsigned ALL = SCH == SCH_TENO5 ? ((M == 3) ? SLOT_MID : (14u | (14u << 5)))
                                                      : (ALL_A | (ALL_A << SH));
            float2 fs[M];
            if (SCH == SCH_TENO5 && (D & ALL) == ALL) {
#pragma unroll
                for (int k = 0; k < M; k++) {
                    float2 v = __fmul2_rn(f2(1.f / 30.f), P[k][1]);
                    v = __ffma2_rn(f2(-13.f / 60.f), P[k][2], v);
                    v = __ffma2_rn(f2(47.f / 60.f), P[k][3], v);
                    v = __ffma2_rn(f2(9.f / 20.f), P[k][4], v);
                    v = __ffma2_rn(f2(-1.f / 20.f), P[k][5], v);
                    fs[k] = v;
                }
            } else if (SCH == SCH_TENO5) {
#pragma unroll
                for (int k = 0; k < M; k++) {
                    const float *cA = s_cf[(D >> (5 * k)) & 31u];
                    const float *cB = s_cf[(D >> (SH + 5 * k)) & 31u];
                    float2 v = __fmul2_rn(make_float2(cA[1], cB[1]), P[k][1]);
#pragma unroll
                    for (int t = 2; t < 6; t++) v = __ffma2_rn(make_float2(cA[t], cB[t]), P[k][t], v);
                    fs[k] = v;
                }
            } else if ((D & ALL) == ALL) {
#pragma unroll
                for (int k = 0; k < M; k++) {
                    float2 v = __fmul2_rn(f2(-1.f / 140.f), P[k][0]);
                    v = __ffma2_rn(f2(5.f / 84.f), P[k][1], v);
                    v = __ffma2_rn(f2(-101.f / 420.f), P[k][2], v);
                    v = __ffma2_rn(f2(319.f / 420.f), P[k][3], v);
                    v = __ffma2_rn(f2(107.f / 210.f), P[k][4], v);
                    v = __ffma2_rn(f2(-19.f / 210.f), P[k][5], v);
                    v = __ffma2_rn(f2(1.f / 105.f), P[k][6], v);
                    fs[k] = v;
                }
            } else {
#pragma unroll
                for (int k = 0; k < M; k++) {
                    const float *cA = s_cf[(D >> (5 * k)) & 31u];
                    const float *cB = s_cf[(D >> (SH + 5 * k)) & 31u];
                    float2 v = __fmul2_rn(make_float2(cA[0], cB[0]), P[k][0]);
#pragma unroll
                    for (int t = 1; t < 7; t++) v = __ffma2_rn(make_float2(cA[t], cB[t]), P[k][t], v);
                    fs[k] = v;
                }
            }
#pragma unroll
            for (int k = 0; k < M; k++) f[k] = s == 0 ? fs[k] : __fadd2_rn(f[k], fs[k]);
        }
        if (A.masks) {
            // '+' in index 0, '-' in index 1 (advection: every '-' code is all ones)
#pragma unroll
            for (int k = 0; k < M; k++) {
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int j = h == 0 ? jA : jB;
                    const bool ok = (h == 0 ? lane >= 1 : lane <= 30) && j >= -1 && j <= n - 1;
                    if (!ok) continue;
                    const int sh = h == 0 ? 5 * k : SH + 5 * k;
                    const unsigned sp = (Dsave[0] >> sh) & 31u;
                    const unsigned sm = PLUS_ONLY ? (SCH == SCH_TENO5 ? 14u : 31u) : (Dsave[1] >> sh) & 31u;
                    A.masks[(size_t)(0 * M + k) * (n + 1) + (j + 1)] =
                        (uint8_t)(SCH == SCH_TENO5 ? slot_code(sp) : sp);
                    A.masks[(size_t)(1 * M + k) * (n + 1) + (j + 1)] =
                        (uint8_t)(SCH == SCH_TENO5 ? slot_code(sm) : sm);
                }
            }
        }
        float2 fh[M];
        if (SYS == SYS_EULER1D) {
            // the roundings of back_project_f32, for both faces at once
            fh[0] = __fadd2_rn(__fadd2_rn(f[0], f[1 % M]), f[2 % M]);
            const float2 umc = __fadd2_rn(ut, f2neg(cc)), upc = __fadd2_rn(ut, cc);
            fh[1 % M] = __ffma2_rn(upc, f[2 % M], __ffma2_rn(umc, f[0], __fmul2_rn(ut, f[1 % M])));
            const float2 R20 = __ffma2_rn(f2neg(ut), cc, Ht), R22 = __ffma2_rn(ut, cc, Ht);
            const float2 R21 = __fmul2_rn(__fmul2_rn(f2(0.5f), ut), ut);
            fh[2 % M] = __ffma2_rn(R22, f[2 % M], __ffma2_rn(R20, f[0], __fmul2_rn(R21, f[1 % M])));
        } else {
            fh[0] = f[0];
        }
        if (flagA && lane >= 1 && jA >= -2 && jA <= n) latch_error(ctl, flagA, A.ebase + jA);
        if (flagB && lane <= 30 && jB <= n) latch_error(ctl, flagB, A.ebase + jB);

        // ---- flux difference and RK stage of cells jA and jB -------------
        float2 fprev[M];
#pragma unroll
        for (int k = 0; k < M; k++) {
            const float xr = __shfl_sync(0xffffffffu, fh[k].x, (lane + 31) & 31);
            const float yr = __shfl_sync(0xffffffffu, fh[k].y, (lane + 31) & 31);
            fprev[k] = make_float2(xr, lane == 0 ? xr : yr);
        }
        // every lane's copies have landed before it reads them, or before its
        // next tile issues new ones into the same slots
        if (U0_ASYNC && use_u0) cp_async_wait_all();
        if (updA || updB) {
            float2 r[M];
#pragma unroll
            for (int k = 0; k < M; k++) r[k] = __fmul2_rn(__fadd2_rn(fprev[k], f2neg(fh[k])), f2(idx));
            if (A.rhs_mode) {
#pragma unroll
                for (int k = 0; k < M; k++) {
                    if (updA) out[(size_t)k * cso + chk(ctl, jA, 0, n)] = r[k].x;
                    if (updB) out[(size_t)k * cso + chk(ctl, jB, 0, n)] = r[k].y;
                }
            } else {
                if (U0_ASYNC && use_u0) {
#pragma unroll
                    for (int k = 0; k < M; k++) u0r[k] = su0[k][lane];
                }
                float2 o[M];
#pragma unroll
                for (int k = 0; k < M; k++) {
                    const float2 v = __ffma2_rn(f2(dtT), r[k], sU[k][lane + 3]);
                    if (A.stage == 0) {
                        o[k] = v;
                    } else if (A.stage == 1) {
                        o[k] = __ffma2_rn(f2(0.75f), u0r[k], __fmul2_rn(f2(0.25f), v));
                    } else {
                        // u0 + 2/3 (v - u0): float(1/3) + float(2/3) != 1 would
                        // grow the solution by 6e-8 every step
                        o[k] = __ffma2_rn(f2(2.0f / 3.0f), __fadd2_rn(v, f2neg(u0r[k])), u0r[k]);
                    }
                    if (updA) out[(size_t)k * cso + chk(ctl, jA, 0, n)] = o[k].x;
                    if (updB) out[(size_t)k * cso + chk(ctl, jB, 0, n)] = o[k].y;
                }
                float oa[M], ob[M];
#pragma unroll
                for (int k = 0; k < M; k++) {
                    oa[k] = o[k].x;
                    ob[k] = o[k].y;
                }
                int wfA = 0, wfB = 0;
                if constexpr (PF) {
                    float w3a[3], w3b[3];
                    wavespeeds1d_fast(oa, gm1, gamma, w3a, &wfA);
                    wavespeeds1d_fast(ob, gm1, gamma, w3b, &wfB);
#pragma unroll
                    for (int q = 0; q < 3; q++) {
                        if (updA) ws3[q] = fmaxf(ws3[q], w3a[q]);
                        if (updB) ws3[q] = fmaxf(ws3[q], w3b[q]);
                    }
                    if (updA && wfA) latch_error(ctl, wfA, A.ebase + jA);
                    if (updB && wfB) latch_error(ctl, wfB, A.ebase + jB);
                } else {
                    const float wa = wavespeed1d_fast<SYS>(oa, gm1, gamma, a, &wfA);
                    const float wb = wavespeed1d_fast<SYS>(ob, gm1, gamma, a, &wfB);
                    if (updA) {
                        wsmax = fmaxf(wsmax, wa);
                        if (wfA) latch_error(ctl, wfA, A.ebase + jA);
                    }
                    if (updB) {
                        wsmax = fmaxf(wsmax, wb);
                        if (wfB) latch_error(ctl, wfB, A.ebase + jB);
                    }
                }
            }
        }
        __syncwarp();  // the next tile overwrites this warp's staging rows
    }
    return wsmax;
}

template <int SYS, int SCH, bool PF = false>
__global__ void __launch_bounds__(WPB * 32, T7_F32_MINB) stage1d_f32fp_kernel(const Stage1D p) {
    constexpr int M = (SYS == SYS_EULER1D) ? 3 : 1;
    constexpr int NP = (SYS == SYS_EULER1D) ? 3 : 1;
    constexpr int MG = (SYS == SYS_ADV) ? 1 : M;  // '-' staging rows (unused for advection)
    __shared__ float2 s_U[WPB][M][WP2];
    __shared__ float2 s_gp[WPB][M][WP2];
    __shared__ float2 s_gm[WPB][MG][WP2];
    __shared__ float2 s_pr[WPB][NP][WP2];
    __shared__ float2 s_u0[WPB][SYS == SYS_EULER1D ? M : 1][32];  // U^n of the cells a lane updates (cp.async)
    __shared__ __align__(16) float s_cf[32][8];
    __shared__ float s_red[PF ? 3 : 1][WPB];

    DevCtl *ctl = p.ctl;
    const bool fixed = p.dt_fixed > 0.0;
    if (!p.rhs_mode && !fixed && !ctl->active) return;  // uniform: the run has ended
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (SCH == SCH_TENO5)
        fill_delta_table5(s_cf);
    else
        fill_delta_table(s_cf);
    TileArgs<float> A;
    A.alpha = p.alpha_in ? (float)*p.alpha_in : ctl->alpha_f[p.slot_in][0];
    if constexpr (PF) {
#pragma unroll
        for (int q = 0; q < 3; q++) A.alf[q] = ctl->alpha_f[p.slot_in][q];
    }
    A.dtT = fixed ? p.f_dt_fixed : ctl->dt_f;
    A.dtD = fixed ? p.dt_fixed : ctl->dt;
    // slab mode: cell 0 follows the padding (the RHS output dU/dt is unpadded)
    const int off = p.halo ? HALO_CELLS : 0, offo = p.rhs_mode ? 0 : off;
    A.Us = static_cast<const float *>(p.Us) + off;
    A.U0 = p.U0 ? static_cast<const float *>(p.U0) + off : nullptr;
    A.out = static_cast<float *>(p.out) + offo;
    A.masks = p.masks;
    A.n = p.n;
    A.cs = (size_t)p.n + 2 * off;
    A.cso = (size_t)p.n + 2 * offo;
    A.bc_lo = p.bc_lo;
    A.bc_hi = p.bc_hi;
    A.dx = p.dx;
    A.f_dx = p.f_dx;
    A.gamma = p.f_gamma;
    A.gm1 = p.f_gm1;
    A.a = p.f_a;
    A.eps = p.f_eps;
    A.CT = p.f_CT;
    A.rhs_mode = p.rhs_mode;
    A.stage = p.stage;
    A.ebase = 0;
    A.halo = p.halo;
    A.ctl = ctl;
    __syncthreads();
    constexpr int NA = PF ? 3 : 1;
    float ws[NA];
#pragma unroll
    for (int q = 0; q < NA; q++) ws[q] = 0.f;
    const float w0 = tiles1d_f32_fp<SYS, SCH, PF>(A, s_U[warp], s_gp[warp], s_gm[warp], s_pr[warp], s_u0[warp], s_cf,
                                                  blockIdx.x * nw + warp, gridDim.x * nw, ws);
    if constexpr (!PF) ws[0] = w0;
    (void)lane;
    if (!p.rhs_mode) {
#pragma unroll
        for (int q = 0; q < NA; q++) {
            ws[q] = warp_max(ws[q]);
            if ((threadIdx.x & 31) == 0) s_red[q][warp] = ws[q];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int so = (p.stage + 1) % 3;
#pragma unroll
            for (int q = 0; q < NA; q++) {
                float v = s_red[q][0];
                for (int w = 1; w < nw; w++) v = fmaxf(v, s_red[q][w]);
                atomicMax(&ctl->amax[so][q], (unsigned long long)__double_as_longlong((double)v));
            }
            finish_launch(ctl, so, (p.stage + 2) % 3, p.stage == 2 && !fixed, p.stage == 2 && !fixed, false,
                          p.alpha_rec, NA);
        }
    }
}

// alpha of a 1D state into ctl->amax[slot][0] (PF: the three per-field
// alphas of 1D Euler into amax[slot][0..2]); grid-stride, one atomic per CTA
// and alpha; the last CTA converts them and plans the first RK step (see
// finish_launch).
template <typename T, int SYS, bool PF = false>
__global__ void __launch_bounds__(256) alpha1d_kernel(const Alpha1D p) {
    constexpr int NA = PF ? 3 : 1;
    __shared__ T s_red[NA][8];
    const T *U = static_cast<const T *>(p.U);
    const T gamma = T(p.gamma), gm1 = T(p.gamma - 1.0), a = T(p.a);
    constexpr int M = (SYS == SYS_EULER1D) ? 3 : 1;
    T m[NA];
#pragma unroll
    for (int q = 0; q < NA; q++) m[q] = T(0);
    int flag = 0, first = 0x7fffffff;
    const size_t cs = p.stride > 0 ? (size_t)p.stride : (size_t)p.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += gridDim.x * blockDim.x) {
        T Uc[M];
#pragma unroll
        for (int k = 0; k < M; k++) Uc[k] = U[(size_t)k * cs + chk(p.ctl, i, 0, p.n)];
        int f = 0;
        if constexpr (PF) {
            T w[3];
            wavespeeds1d<T>(Uc, gm1, gamma, w, &f);
#pragma unroll
            for (int q = 0; q < 3; q++) m[q] = fmax(m[q], w[q]);
        } else {
            m[0] = fmax(m[0], wavespeed1d<T, SYS>(Uc, gm1, gamma, a, &f));
        }
        if (f) {
            flag |= f;
            first = min(first, i);
        }
    }
    if (flag) latch_error(p.ctl, flag, first);
#pragma unroll
    for (int q = 0; q < NA; q++) {
        m[q] = warp_max(m[q]);
        if ((threadIdx.x & 31) == 0) s_red[q][threadIdx.x >> 5] = m[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NA; q++) {
            T v = s_red[q][0];
            for (int w = 1; w < 8; w++) v = fmax(v, s_red[q][w]);
            atomicMax(&p.ctl->amax[p.slot][q], (unsigned long long)__double_as_longlong((double)v));
        }
        finish_launch(p.ctl, p.slot, (p.slot + 1) % 3, false, true, false, p.alpha_rec, NA);
    }
}

// Scalar reconstruction of caller-padded values (t7_teno7_reconstruct).
// Tiles of NT faces per CTA with the cutoff words exchanged in shared memory.
template <typename T>
__global__ void __launch_bounds__(NT) recon_kernel(const Recon p) {
    __shared__ T s_v[NCP];
    __shared__ T s_coef[91];
    __shared__ unsigned s_bits[NT];
    const int tid = threadIdx.x, n = p.n;
    const int s = blockIdx.x * TILE;
    const T *v = static_cast<const T *>(p.v);
    const T eps = T(p.eps), CT = T(p.CT);
    const T kt = keep_all_factor(CT);
    for (int q = tid; q < 91; q += NT) s_coef[q] = coef<T>(q);
    for (int c = tid; c < NCELL; c += NT) {
        int l = s - HALO + c + 4;  // index into v (cell -4 is v[0])
        l = l < 0 ? 0 : (l > n + 7 ? n + 7 : l);
        s_v[c] = v[l];
    }
    __syncthreads();
    const int j = s - 2 + tid;
    unsigned bits;
    if (p.sign > 0)
        bits = cutoff_bits(s_v[tid + 1], s_v[tid + 2], s_v[tid + 3], s_v[tid + 4], s_v[tid + 5], eps, CT, kt);
    else
        bits = cutoff_bits(s_v[tid + 6], s_v[tid + 5], s_v[tid + 4], s_v[tid + 3], s_v[tid + 2], eps, CT, kt);
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
inline int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 152;
    }
    return sms;
}

// CTAs of a kernel resident on one SM at `threads` threads and `smem` bytes of
// dynamic shared memory (the CUDA occupancy calculator; at least 1), cached
// per (kernel, threads, smem), so that each launch configuration is queried
// once.
inline int resident_ctas(const void *kernel, int threads, size_t smem = 0) {
    struct Entry {
        const void *kernel;
        int threads;
        size_t smem;
        int ctas;
    };
    static Entry cache[64];
    static int used = 0;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < used; i++)
        if (cache[i].kernel == kernel && cache[i].threads == threads && cache[i].smem == smem) return cache[i].ctas;
    int ctas = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, kernel, threads, smem) != cudaSuccess) {
        (void)cudaGetLastError();  // not left for the launch's own error check
        ctas = 0;
    }
    if (ctas < 1) ctas = 1;
    if (used < 64) cache[used++] = {kernel, threads, smem, ctas};
    return ctas;
}

// Warps per CTA of the 1D stage and adjoint kernels: WPB, or -- for the
// FP64-pipe-bound kernels (spread = true) -- halved while that would leave SMs
// without a CTA, so small problems run one warp tile per SM instead of eight
// tiles on a few SMs (GB300's FP64 rate per SM is low; FP32 stage kernels at
// small sizes are launch-bound and keep WPB).  The kernels take it from
// blockDim.
inline int warps_per_cta(int ntiles, bool spread) {
    int nw = WPB;
    while (spread && nw > 1 && (ntiles + nw - 1) / nw < num_sms()) nw >>= 1;
    return nw;
}

// Warp tiles a stage launch covers: [tile_lo, tile_hi) of the domain's tiles
// (tile_hi <= 0: to the end); 0 if the range is empty or out of the domain.
inline int stage_tiles(const Stage1D &p) {
    const int all = (p.n + WT - 1) / WT;
    const int hi = p.tile_hi > 0 ? p.tile_hi : all;
    if (p.tile_lo < 0 || hi > all || hi <= p.tile_lo) return 0;
    return hi - p.tile_lo;
}

using Stage1DKernel = void (*)(const Stage1D);

// Grid of an FP32 stage launch: nctas CTAs of `threads` threads, capped at
// `waves` whole waves of the kernel's resident CTAs (the tiles are spread over
// the grid by a grid-stride loop, each warp loading its next tile while it
// computes the current one).  Measured on the 16.8M-cell workloads: the
// scalar laws run fastest as one wave (advection 70.6 -> 81.2, Burgers 42.3 ->
// 46.4 Gcell-steps/s against four waves: a warp's first tile load is not
// hidden, and one wave has the fewest), Euler as two (15.82 -> 15.90 against
// four, 15.76 as one: the shock tiles cost more, and the second wave evens
// out the SMs' loads).
inline int stage_grid(Stage1DKernel k, int nctas, int threads, int waves) {
    const int cap = num_sms() * resident_ctas(reinterpret_cast<const void *>(k), threads) * waves;
    return nctas < cap ? nctas : cap;
}

// FP32 paired-split stage kernels; S = float (FP32 state) or double (mixed).
template <typename S>
cudaError_t launch_stage1d_paired(const Stage1D &p, cudaStream_t st) {
    const int ntiles = stage_tiles(p);
    if (ntiles < 1) return cudaErrorInvalidValue;
    const int nw = warps_per_cta(ntiles, false);
    if (p.scheme != SCH_TENO7EXT && p.scheme != SCH_TENO5) return cudaErrorInvalidValue;
    const bool t5 = p.scheme == SCH_TENO5;
    const int nt2 = (p.n + WT2 - 1) / WT2;
    const int nw2 = warps_per_cta(nt2, false);
    Stage1DKernel k = nullptr;
    if (p.alpha_mode) {
        // per-field alphas: 1D Euler, TENO7-ext, FP32 state, whole-domain launches only
        if (sizeof(S) != 4 || p.sys != SYS_EULER1D || t5 || p.tile_lo != 0 || p.tile_hi > 0 || p.partial || p.halo)
            return cudaErrorInvalidValue;
        k = stage1d_f32fp_kernel<SYS_EULER1D, SCH_TENO7EXT, true>;
        k<<<stage_grid(k, (nt2 + nw2 - 1) / nw2, nw2 * 32, T7_WAVES_EULER), nw2 * 32, 0, st>>>(p);
        return cudaGetLastError();
    }
    // FP32 state over the whole domain or a slab: face-paired tiles
    // (advection when a > 0, where alpha = a makes the '-' split vanish).
    // Their results equal the paired-split kernel's bit for bit (the Roe
    // frame and back projection share the roundings of
    // roe_frame_f32/back_project_f32), so parted launches and batches, which
    // take the paired-split tiles, agree with them.
    if (sizeof(S) == 4 && p.tile_lo == 0 && p.tile_hi <= 0 && !p.partial &&
        ((p.sys == SYS_ADV && p.a > 0.0) || p.sys == SYS_BURGERS || p.sys == SYS_EULER1D)) {
        switch (p.sys) {
            case SYS_ADV:
                k = t5 ? stage1d_f32fp_kernel<SYS_ADV, SCH_TENO5> : stage1d_f32fp_kernel<SYS_ADV, SCH_TENO7EXT>;
                break;
            case SYS_BURGERS:
                k = t5 ? stage1d_f32fp_kernel<SYS_BURGERS, SCH_TENO5>
                       : stage1d_f32fp_kernel<SYS_BURGERS, SCH_TENO7EXT>;
                break;
            case SYS_EULER1D:
                k = t5 ? stage1d_f32fp_kernel<SYS_EULER1D, SCH_TENO5>
                       : stage1d_f32fp_kernel<SYS_EULER1D, SCH_TENO7EXT>;
                break;
            default: return cudaErrorInvalidValue;
        }
        const int waves = p.sys == SYS_EULER1D ? T7_WAVES_EULER : T7_WAVES_SCALAR;
        k<<<stage_grid(k, (nt2 + nw2 - 1) / nw2, nw2 * 32, waves), nw2 * 32, 0, st>>>(p);
        return cudaGetLastError();
    }
    switch (p.sys) {
        case SYS_ADV:
            k = t5 ? stage1d_f32_kernel<SYS_ADV, SCH_TENO5, S> : stage1d_f32_kernel<SYS_ADV, SCH_TENO7EXT, S>;
            break;
        case SYS_BURGERS:
            k = t5 ? stage1d_f32_kernel<SYS_BURGERS, SCH_TENO5, S> : stage1d_f32_kernel<SYS_BURGERS, SCH_TENO7EXT, S>;
            break;
        case SYS_EULER1D:
            k = t5 ? stage1d_f32_kernel<SYS_EULER1D, SCH_TENO5, S> : stage1d_f32_kernel<SYS_EULER1D, SCH_TENO7EXT, S>;
            break;
        default: return cudaErrorInvalidValue;
    }
    const int waves = p.sys == SYS_EULER1D ? T7_WAVES_EULER : T7_WAVES_SCALAR;
    k<<<stage_grid(k, (ntiles + nw - 1) / nw, nw * 32, waves), nw * 32, 0, st>>>(p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stage1d(const Stage1D &p, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        return launch_stage1d_paired<float>(p, st);
    } else {
        const int ntiles = stage_tiles(p);
        if (ntiles < 1) return cudaErrorInvalidValue;
        const int nw = warps_per_cta(ntiles, true);
        const int resident = num_sms() * 4 * (WPB / nw);  // a few waves of resident CTAs
        int grid = (ntiles + nw - 1) / nw;
        if (grid > resident) grid = resident;
        if (p.scheme != SCH_TENO7EXT && p.scheme != SCH_TENO5) return cudaErrorInvalidValue;
        const bool t5 = p.scheme == SCH_TENO5;
        if (p.alpha_mode) {  // per-field alphas: 1D Euler with TENO7-ext only
            if (p.sys != SYS_EULER1D || t5) return cudaErrorInvalidValue;
            stage1d_kernel<T, SYS_EULER1D, SCH_TENO7EXT, true><<<grid, nw * 32, 0, st>>>(p);
            return cudaGetLastError();
        }
        switch (p.sys) {
            case SYS_ADV:
                if (t5) stage1d_kernel<T, SYS_ADV, SCH_TENO5><<<grid, nw * 32, 0, st>>>(p);
                else stage1d_kernel<T, SYS_ADV, SCH_TENO7EXT><<<grid, nw * 32, 0, st>>>(p);
                break;
            case SYS_BURGERS:
                if (t5) stage1d_kernel<T, SYS_BURGERS, SCH_TENO5><<<grid, nw * 32, 0, st>>>(p);
                else stage1d_kernel<T, SYS_BURGERS, SCH_TENO7EXT><<<grid, nw * 32, 0, st>>>(p);
                break;
            case SYS_EULER1D:
                if (t5) stage1d_kernel<T, SYS_EULER1D, SCH_TENO5><<<grid, nw * 32, 0, st>>>(p);
                else stage1d_kernel<T, SYS_EULER1D, SCH_TENO7EXT><<<grid, nw * 32, 0, st>>>(p);
                break;
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
}

template <typename T>
cudaError_t launch_alpha1d(const Alpha1D &p, cudaStream_t st) {
    int grid = (p.n + 255) / 256;
    if (grid > num_sms() * 8) grid = num_sms() * 8;
    switch (p.sys) {
        case SYS_ADV: alpha1d_kernel<T, SYS_ADV><<<grid, 256, 0, st>>>(p); break;
        case SYS_BURGERS: alpha1d_kernel<T, SYS_BURGERS><<<grid, 256, 0, st>>>(p); break;
        case SYS_EULER1D:
            if (p.alpha_mode)
                alpha1d_kernel<T, SYS_EULER1D, true><<<grid, 256, 0, st>>>(p);
            else
                alpha1d_kernel<T, SYS_EULER1D><<<grid, 256, 0, st>>>(p);
            break;
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

// ==========================================================================
// Persistent ragged-batch kernel (1D Euler).  The CTA's warps form groups of
// G = p.group_warps warps; each group's leader takes the next tube from an
// atomic queue (the host orders tubes costliest first) and the group runs the
// tube's whole SSP-RK3 loop to t_end: alpha of U^n and the CFL step (the
// oracle's expressions), then three stages, each a warp-tile sweep over the
// tube followed by a group reduction of the new state's max(|u| + c), which is
// the next stage's alpha.  Group barriers are named barriers (id = group + 1).
// Tubes are independent, so groups never wait on each other.
// ==========================================================================
namespace t7 {

__device__ __forceinline__ void group_sync(int group, int G) {
    if (G == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(group + 1), "r"(G * 32) : "memory");
    }
}

template <typename T>
__global__ void __launch_bounds__(WPB * 32, (sizeof(T) == 4 ? 2 : 1)) batch1d_kernel(const Batch1D p) {
    __shared__ T s_U[WPB][3][WC];
    __shared__ T s_gp[WPB][3][WC];
    __shared__ T s_gm[WPB][3][WC];
    __shared__ T s_pr[WPB][3][WC];
    __shared__ T s_coef[WPB][92];
    __shared__ __align__(16) float s_cf[32][8];
    __shared__ T s_red[WPB];
    __shared__ int s_tube[WPB];
    constexpr bool F64 = sizeof(T) == 8;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = lane; q < 91; q += 32) s_coef[warp][q] = coef<T>(q);
    if constexpr (!F64) fill_delta_table(s_cf);
    __syncthreads();
    T *U = static_cast<T *>(p.U);
    T *W1 = static_cast<T *>(p.W1);
    T *W2 = static_cast<T *>(p.W2);
    const size_t cs = (size_t)p.Ntot;
    const T gamma = T(p.gamma), gm1 = T(p.gamma - 1.0);

    // The CTA's warps form groups of G warps (group = warp / G, rank wg within
    // it); the first nbig tubes of the order (the costliest) are run first with
    // the whole CTA as one group, so that no single tube outlasts the rest of
    // the batch on a small group.
    int G = WPB, group = 0, wg = warp;

    // group max over its G warps; every lane of the group gets the result
    auto group_max = [&](T v) -> T {
        v = warp_max(v);
        if (lane == 0) s_red[warp] = v;
        group_sync(group, G);
        T m = s_red[group * G];
        for (int w = 1; w < G; w++) m = fmax(m, s_red[group * G + w]);
        group_sync(group, G);
        return m;
    };

    auto run_tube = [&](int tube) {
        const long long off = p.offsets[tube];
        const int n = (int)(p.offsets[tube + 1] - off);
        const double dx = p.dx[tube];

        // alpha of U^n over the tube's cells
        T a0 = T(0);
        int flag = 0, first = 0x7fffffff;
        for (int i = wg * 32 + lane; i < n; i += G * 32) {
            T Uc[3] = {U[off + i], U[cs + off + i], U[2 * cs + off + i]};
            int f = 0;
            a0 = fmax(a0, wavespeed1d<T, SYS_EULER1D>(Uc, gm1, gamma, T(0), &f));
            if (f) {
                flag |= f;
                first = min(first, i);
            }
        }
        if (flag) latch_error(p.ctl, flag, (int)(off + first));
        T alpha = group_max(a0);

        TileArgs<T> A;
        A.masks = nullptr;
        A.n = n;
        A.cs = cs;
        A.cso = cs;
        A.bc_lo = p.bc_lo;
        A.bc_hi = p.bc_hi;
        A.dx = dx;
        A.f_dx = (float)dx;
        A.gamma = gamma;
        A.gm1 = gm1;
        A.a = T(0);
        A.eps = T((dx * dx) * dx);
        A.CT = T(p.CT);
        A.rhs_mode = 0;
        A.ebase = (int)off;
        A.halo = 0;
        A.ctl = p.ctl;
        A.U0 = U + off;
        T *ins[3] = {U + off, W1 + off, W2 + off};
        T *outs[3] = {W1 + off, W2 + off, U + off};

        double t = 0.0;
        int steps = 0;
        while (steps < p.max_steps && t < p.t_end) {
            double dt = (p.cfl * dx) / (double)alpha;
            if (t + dt > p.t_end) dt = p.t_end - t;
            A.dtT = T(dt);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                A.Us = ins[k];
                A.out = outs[k];
                A.stage = k;
                A.alpha = alpha;
                T ws;
                if constexpr (F64) {
                    ws = tiles1d<T, SYS_EULER1D>(A, s_U[warp], s_gp[warp], s_gm[warp], s_pr[warp], s_coef[warp], wg, G);
                } else {
                    ws = tiles1d_f32<SYS_EULER1D>(A, s_U[warp], s_gp[warp], s_gm[warp], s_pr[warp], s_cf, wg, G);
                }
                alpha = group_max(ws);  // also orders this stage's writes before the next stage's reads
            }
            t = t + dt;
            steps = steps + 1;
        }
        if (wg == 0 && lane == 0) {
            p.steps_out[tube] = steps;
            p.t_out[tube] = t;
        }
    };

    // phase 1: whole-CTA groups over order[0 .. nbig)
    for (;;) {
        if (warp == 0 && lane == 0) s_tube[0] = atomicAdd(p.queue + 1, 1);
        __syncthreads();
        const int q = s_tube[0];
        __syncthreads();
        if (q >= p.nbig) break;
        run_tube(p.order[q]);
    }
    // phase 2: groups of p.group_warps warps over order[nbig .. ntubes)
    G = p.group_warps;
    group = warp / G;
    wg = warp % G;
    for (;;) {
        if (wg == 0 && lane == 0) s_tube[group] = p.nbig + atomicAdd(p.queue, 1);
        group_sync(group, G);
        const int q = s_tube[group];
        group_sync(group, G);
        if (q >= p.ntubes) break;
        run_tube(p.order[q]);
    }
}

// Per-tube wave speed max(|u| + c) of the state, the alpha that sets the
// tube's first CFL step (Remark 3).  One CTA of 8 warps per tube; non-physical
// cells are skipped here (the batch kernel itself reports them).
template <typename T>
__global__ void __launch_bounds__(256) batch1d_alpha_kernel(const Batch1D p, double *alpha_out) {
    __shared__ T s_red[8];
    const T *U = static_cast<const T *>(p.U);
    const size_t cs = (size_t)p.Ntot;
    const T gamma = T(p.gamma), gm1 = T(p.gamma - 1.0);
    for (int tube = blockIdx.x; tube < p.ntubes; tube += gridDim.x) {
        const long long off = p.offsets[tube];
        const int n = (int)(p.offsets[tube + 1] - off);
        T a = T(0);
        for (int i = threadIdx.x; i < n; i += 256) {
            T Uc[3] = {U[off + i], U[cs + off + i], U[2 * cs + off + i]};
            int f = 0;
            const T w = wavespeed1d<T, SYS_EULER1D>(Uc, gm1, gamma, T(0), &f);
            if (!f) a = fmax(a, w);
        }
        a = warp_max(a);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = a;
        __syncthreads();
        if (threadIdx.x == 0) {
            T m = s_red[0];
            for (int w = 1; w < 8; w++) m = fmax(m, s_red[w]);
            alpha_out[tube] = (double)m;
        }
        __syncthreads();
    }
}

template <typename T>
cudaError_t launch_batch1d_alpha(const Batch1D &p, double *alpha_out, cudaStream_t st) {
    if (p.ntubes < 1) return cudaSuccess;
    const int grid = p.ntubes < num_sms() * 8 ? p.ntubes : num_sms() * 8;
    batch1d_alpha_kernel<T><<<grid, 256, 0, st>>>(p, alpha_out);
    return cudaGetLastError();
}

template <typename T>
int batch1d_groups(int group_warps) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch1d_kernel<T>, WPB * 32, 0) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    if (per_sm < 1) per_sm = 1;
    return num_sms() * per_sm * (WPB / (group_warps > 0 ? group_warps : WPB));
}

template <typename T>
cudaError_t launch_batch1d(const Batch1D &p, cudaStream_t st) {
    if (p.group_warps != 1 && p.group_warps != 2 && p.group_warps != 4 && p.group_warps != 8)
        return cudaErrorInvalidValue;
    if (p.nbig < 0 || p.nbig > p.ntubes) return cudaErrorInvalidValue;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch1d_kernel<T>, WPB * 32, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    batch1d_kernel<T><<<num_sms() * per_sm, WPB * 32, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace t7
