// teno7_adjoint.cuh -- discrete adjoint of the 1D Euler right-hand side
// L(U) = -(F_{i+1/2} - F_{i-1/2})/dx of the TENO7-ext scheme, with the stencil
// selection (every Delta_i) and the global Lax-Friedrichs alpha frozen at
// their values for the given state.  out = (dL/dU)^T v.
//
// Per face j+1/2 (one lane, warp tiles as the forward kernels) the kernel
// recomputes the forward face -- frame, projections, cutoff bits, Delta,
// polynomials, back-projection; the masks come out identical to the forward
// pass's because the arithmetic is the same -- and then propagates
//   lambda_F = (v_{j+1} - v_j)/dx                      (flux difference)
//   lambda_f = R^T lambda_F,  lambda_R = lambda_F f^T    (back-projection)
//   lambda_q = a_m lambda_f                              (frozen polynomial)
//   lambda_G = L^T lambda_q,  lambda_L += lambda_q G^T    (projection)
//   lambda_U += (A^T (lambda_G+ + lambda_G-) + alpha (lambda_G+ - lambda_G-))/2
//                                                        (G+- = (F +- alpha U)/2)
// and the frame's dependence on the two face cells through the Roe average:
// L and R as 2-direction dual numbers in (u~, H~), then the Roe average's
// derivatives by hand (roe_chain).  Contributions to the 8
// stencil cells are scattered with atomicAdd.
#pragma once
#include "teno7_adjoint_params.h"
#include "teno7_kernels.cuh"

namespace t7 {

// Forward-mode number with D directional derivatives.
template <typename T, int D>
struct Dual {
    T v;
    T d[D];
};

template <typename T, int D>
__device__ __forceinline__ Dual<T, D> dconst(T v) {
    Dual<T, D> r;
    r.v = v;
#pragma unroll
    for (int k = 0; k < D; k++) r.d[k] = T(0);
    return r;
}
template <typename T, int D>
__device__ __forceinline__ Dual<T, D> operator+(const Dual<T, D> &a, const Dual<T, D> &b) {
    Dual<T, D> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < D; k++) r.d[k] = a.d[k] + b.d[k];
    return r;
}
template <typename T, int D>
__device__ __forceinline__ Dual<T, D> operator-(const Dual<T, D> &a, const Dual<T, D> &b) {
    Dual<T, D> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < D; k++) r.d[k] = a.d[k] - b.d[k];
    return r;
}
template <typename T, int D>
__device__ __forceinline__ Dual<T, D> operator*(const Dual<T, D> &a, const Dual<T, D> &b) {
    Dual<T, D> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < D; k++) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
template <typename T, int D>
__device__ __forceinline__ Dual<T, D> operator*(T a, const Dual<T, D> &b) {
    Dual<T, D> r;
    r.v = a * b.v;
#pragma unroll
    for (int k = 0; k < D; k++) r.d[k] = a * b.d[k];
    return r;
}
// (one division for the derivatives: they need not round like the value)
template <typename T, int D>
__device__ __forceinline__ Dual<T, D> operator/(const Dual<T, D> &a, const Dual<T, D> &b) {
    Dual<T, D> r;
    r.v = a.v / b.v;
    const T ib = T(1) / b.v;
#pragma unroll
    for (int k = 0; k < D; k++) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
    return r;
}
template <typename T, int D>
__device__ __forceinline__ Dual<T, D> dsqrt(const Dual<T, D> &a) {
    Dual<T, D> r;
    r.v = sq_root(a.v);
    const T h = T(0.5) / r.v;
#pragma unroll
    for (int k = 0; k < D; k++) r.d[k] = a.d[k] * h;
    return r;
}

// Roe frame of 1D Euler at a face.  The frame depends on the two face cells
// only through the Roe-averaged velocity and enthalpy (u~, H~), so L and R are
// carried as dual numbers in those two directions; roe_chain then maps
// (lambda_u~, lambda_H~) back to the six cell variables through the Roe
// average.  Values are computed in the forward kernels' operation order.
template <typename T>
struct RoeFace {
    T ul, ur, Hl, Hr, sl, sr, rl, rr, ut, Ht;
};

template <typename T>
__device__ __forceinline__ void frame1d_dual(const T UL[3], const T UR[3], T gm1, Dual<T, 2> L[3][3],
                                             Dual<T, 2> R[3][3], RoeFace<T> &rf) {
    using D2 = Dual<T, 2>;
    rf.rl = UL[0];
    rf.rr = UR[0];
    rf.ul = UL[1] / UL[0];
    rf.ur = UR[1] / UR[0];
    const T pl = gm1 * (UL[2] - T(0.5) * UL[1] * rf.ul), pr = gm1 * (UR[2] - T(0.5) * UR[1] * rf.ur);
    rf.Hl = (UL[2] + pl) / UL[0];
    rf.Hr = (UR[2] + pr) / UR[0];
    rf.sl = sq_root(UL[0]);
    rf.sr = sq_root(UR[0]);
    rf.ut = (rf.sl * rf.ul + rf.sr * rf.ur) / (rf.sl + rf.sr);
    rf.Ht = (rf.sl * rf.Hl + rf.sr * rf.Hr) / (rf.sl + rf.sr);
    D2 ut = dconst<T, 2>(rf.ut), Ht = dconst<T, 2>(rf.Ht);
    ut.d[0] = T(1);
    Ht.d[1] = T(1);
    const D2 half = dconst<T, 2>(T(0.5)), g = dconst<T, 2>(gm1), one = dconst<T, 2>(T(1));
    const D2 c2 = g * (Ht - half * ut * ut);
    const D2 c = dsqrt(c2);
    const D2 b1 = g / c2;
    const D2 b2 = half * ut * ut * b1;
    const D2 mh = dconst<T, 2>(T(-0.5));
    R[0][0] = one;
    R[0][1] = one;
    R[0][2] = one;
    R[1][0] = ut - c;
    R[1][1] = ut;
    R[1][2] = ut + c;
    R[2][0] = Ht - ut * c;
    R[2][1] = half * ut * ut;
    R[2][2] = Ht + ut * c;
    L[0][0] = half * (b2 + ut / c);
    L[0][1] = mh * (b1 * ut + one / c);
    L[0][2] = half * b1;
    L[1][0] = one - b2;
    L[1][1] = b1 * ut;
    L[1][2] = dconst<T, 2>(T(0)) - b1;
    L[2][0] = half * (b2 - ut / c);
    L[2][1] = mh * (b1 * ut - one / c);
    L[2][2] = half * b1;
}

// (lambda_u~, lambda_H~) -> lambda of (rho, m, E) of the left (lx[0..2]) and
// right (lx[3..5]) cells: u~ = (sl ul + sr ur)/(sl + sr), H~ likewise, with
// s = sqrt(rho), u = m/rho, H = (E + p)/rho, p = (g-1)(E - m u/2).
template <typename T>
__device__ __forceinline__ void roe_chain(const RoeFace<T> &rf, T lut, T lHt, T gm1, T lx[6]) {
    const T iS = T(1) / (rf.sl + rf.sr);
#pragma unroll
    for (int side = 0; side < 2; side++) {
        const T s = side ? rf.sr : rf.sl, u = side ? rf.ur : rf.ul, H = side ? rf.Hr : rf.Hl;
        const T rho = side ? rf.rr : rf.rl;
        const T irho = T(1) / rho;
        const T lu = lut * s * iS, lH = lHt * s * iS;
        const T ls = (lut * (u - rf.ut) + lHt * (H - rf.Ht)) * iS;
        lx[3 * side + 0] = -lu * u * irho + lH * (T(0.5) * gm1 * u * u - H) * irho + ls * (T(0.5) / s);
        lx[3 * side + 1] = (lu - lH * gm1 * u) * irho;
        lx[3 * side + 2] = lH * (T(1) + gm1) * irho;
    }
}

template <typename T>
__device__ __forceinline__ void add_to(T *p, T v) {
    atomicAdd(p, v);
}

template <typename T>
__global__ void __launch_bounds__(WPB * 32, 1) rhs_adjoint1d_kernel(const Adjoint1D p) {
    __shared__ T s_U[WPB][3][WC];
    __shared__ T s_gp[WPB][3][WC];
    __shared__ T s_gm[WPB][3][WC];
    __shared__ T s_coef[WPB][92];
    __shared__ T s_uH[WPB][2][WC];  // velocity and total enthalpy of each staged cell
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = lane; q < 91; q += 32) s_coef[warp][q] = coef<T>(q);
    const T alpha = p.alpha_ptr ? T(*p.alpha_ptr) : T(__longlong_as_double((long long)p.ctl->amax[p.slot_in][0]));
    const T sc = T(p.scale);
    const T gm1 = T(p.gamma - 1.0), eps = T(p.eps), CT = T(p.CT), dxT = T(p.dx);
    const T kt = keep_all_factor(CT);
    const T *U = static_cast<const T *>(p.U);
    const T *V = static_cast<const T *>(p.v);
    T *out = static_cast<T *>(p.out);
    const int n = p.n;
    const int ntiles = (n + WT - 1) / WT;
    T (*sU)[WC] = s_U[warp];
    T (*sgp)[WC] = s_gp[warp];
    T (*sgm)[WC] = s_gm[warp];
    const T *scoef = s_coef[warp];
    __syncwarp();
    const int nw = blockDim.x >> 5;
    for (int tile = blockIdx.x * nw + warp; tile < ntiles; tile += gridDim.x * nw) {
        const int c0 = tile * WT;
        for (int c = lane; c < WS; c += 32) {
            int gi = c0 - 5 + c;
            if (gi < 0 || gi >= n) gi = ghost_map(gi, n, p.bc_lo, p.bc_hi);
            gi = chk(p.ctl, gi, 0, n);
            T Uc[3], F[3];
#pragma unroll
            for (int k = 0; k < 3; k++) Uc[k] = U[(size_t)k * n + gi];
            const T u = Uc[1] / Uc[0];
            const T pr = gm1 * (Uc[2] - T(0.5) * Uc[1] * u);
            F[0] = Uc[1];
            F[1] = Uc[1] * u + pr;
            F[2] = u * (Uc[2] + pr);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                sU[k][c] = Uc[k];
                sgp[k][c] = T(0.5) * (F[k] + alpha * Uc[k]);
                sgm[k][c] = T(0.5) * (F[k] - alpha * Uc[k]);
            }
            s_uH[warp][0][c] = u;
            s_uH[warp][1][c] = (Uc[2] + pr) / Uc[0];
        }
        __syncwarp();
        const int j = c0 - 2 + lane;  // face j+1/2
        // ---- forward face with the frame as dual numbers -------------------
        T UL[3], UR[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            UL[k] = sU[k][lane + 3];
            UR[k] = sU[k][lane + 4];
        }
        Dual<T, 2> Ld[3][3], Rd[3][3];
        RoeFace<T> rf;
        frame1d_dual<T>(UL, UR, gm1, Ld, Rd, rf);
        T qp[3][7], qm[3][7];
        unsigned word = 0;
#pragma unroll
        for (int k = 0; k < 3; k++) {
#pragma unroll
            for (int t = 0; t < 7; t++) {
                T sp = Ld[k][0].v * sgp[0][lane + t];
                T sm = Ld[k][0].v * sgm[0][lane + 1 + t];
#pragma unroll
                for (int c = 1; c < 3; c++) {
                    sp = sp + Ld[k][c].v * sgp[c][lane + t];
                    sm = sm + Ld[k][c].v * sgm[c][lane + 1 + t];
                }
                qp[k][t] = sp;
                qm[k][t] = sm;
            }
            if (!p.masks) {  // recorded masks make the cutoff unnecessary
                word |= cutoff_bits(qp[k][1], qp[k][2], qp[k][3], qp[k][4], qp[k][5], eps, CT, kt) << (3 * k);
                word |= cutoff_bits(qm[k][5], qm[k][4], qm[k][3], qm[k][2], qm[k][1], eps, CT, kt) << (3 * (3 + k));
            }
        }
        const unsigned wl = __shfl_up_sync(0xffffffffu, word, 1);
        const unsigned wr = __shfl_down_sync(0xffffffffu, word, 1);
        // each face once: tile w owns faces 29 w - 1 .. 29 w + 27 (lanes 1..29);
        // the last face n-1 falls on lane 30 when n is a multiple of 29
        const bool face_out = j >= -1 && j <= n - 1 && ((lane >= 1 && lane <= 29) || (lane == 30 && j == n - 1));
        if (face_out) {
            int mp[3], mm[3];
            T f[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (p.masks) {
                    mp[k] = lut_select(p.masks[(size_t)(0 * 3 + k) * (n + 1) + (j + 1)]);
                    mm[k] = lut_select(p.masks[(size_t)(1 * 3 + k) * (n + 1) + (j + 1)]);
                } else {
                    mp[k] = lut_select(pack_delta(wl >> (3 * k), word >> (3 * k), wr >> (3 * k)));
                    mm[k] = lut_select(pack_delta(wr >> (3 * (3 + k)), word >> (3 * (3 + k)), wl >> (3 * (3 + k))));
                }
                if (mp[k] == 15) mp[k] = 11;
                if (mm[k] == 15) mm[k] = 11;
                const T *cp = scoef + 7 * mp[k], *cm = scoef + 7 * mm[k];
                f[k] = poly7(cp, qp[k][0], qp[k][1], qp[k][2], qp[k][3], qp[k][4], qp[k][5], qp[k][6]) +
                       poly7(cm, qm[k][6], qm[k][5], qm[k][4], qm[k][3], qm[k][2], qm[k][1], qm[k][0]);
            }
            // ---- reverse --------------------------------------------------
            // lambda of the face flux: L_i = (F_{i-1/2} - F_{i+1/2})/dx
            T lF[3];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const T vr = (j + 1 <= n - 1) ? V[(size_t)c * n + chk(p.ctl, j + 1, 0, n)] : T(0);
                const T vl = (j >= 0) ? V[(size_t)c * n + chk(p.ctl, j, 0, n)] : T(0);
                lF[c] = sc * ((vr - vl) / dxT);
            }
            T lf[3], lR[3][3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                lf[k] = Rd[0][k].v * lF[0] + Rd[1][k].v * lF[1] + Rd[2][k].v * lF[2];
#pragma unroll
                for (int c = 0; c < 3; c++) lR[c][k] = lF[c] * f[k];
            }
            // projections: lambda_q -> lambda_G (per cell) and lambda_L
            T lL[3][3];
#pragma unroll
            for (int k = 0; k < 3; k++)
#pragma unroll
                for (int c = 0; c < 3; c++) lL[k][c] = T(0);
            for (int t = 0; t < 8; t++) {
                // local cell lane + t (cell j-3+t): '+' uses q+ index t (t <= 6),
                // '-' uses q- index t-1 (t >= 1), whose polynomial tap is 7-t
                T lgp[3] = {T(0), T(0), T(0)}, lgm[3] = {T(0), T(0), T(0)};
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const T lqp = (t <= 6) ? scoef[7 * mp[k] + t] * lf[k] : T(0);
                    const T lqm = (t >= 1) ? scoef[7 * mm[k] + (7 - t)] * lf[k] : T(0);
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        lgp[c] = lgp[c] + Ld[k][c].v * lqp;
                        lgm[c] = lgm[c] + Ld[k][c].v * lqm;
                        lL[k][c] = lL[k][c] + lqp * sgp[c][lane + t] + lqm * sgm[c][lane + t];
                    }
                }
                // G+- = (F +- alpha U)/2  ->  lambda_U = (A^T (lgp + lgm) + alpha (lgp - lgm))/2
                const T u = s_uH[warp][0][lane + t], H = s_uH[warp][1][lane + t];
                const T gam = gm1 + T(1);
                const T s0 = lgp[0] + lgm[0], s1 = lgp[1] + lgm[1], s2 = lgp[2] + lgm[2];
                // A = [[0,1,0],[(g-3)/2 u^2,(3-g)u,g-1],[u((g-1)/2 u^2 - H), H-(g-1)u^2, g u]]
                const T a10 = T(0.5) * (gam - T(3)) * u * u, a11 = (T(3) - gam) * u, a12 = gm1;
                const T a20 = u * (T(0.5) * gm1 * u * u - H), a21 = H - gm1 * u * u, a22 = gam * u;
                T lu[3];
                lu[0] = T(0.5) * (a10 * s1 + a20 * s2 + alpha * (lgp[0] - lgm[0]));
                lu[1] = T(0.5) * (s0 + a11 * s1 + a21 * s2 + alpha * (lgp[1] - lgm[1]));
                lu[2] = T(0.5) * (a12 * s1 + a22 * s2 + alpha * (lgp[2] - lgm[2]));
                const int cell = chk(p.ctl, ghost_map(j - 3 + t, n, p.bc_lo, p.bc_hi), 0, n);
#pragma unroll
                for (int c = 0; c < 3; c++) add_to(&out[(size_t)c * n + cell], lu[c]);
            }
            // frame: lambda_(u~, H~) = sum lambda_L dL/d. + lambda_R dR/d., then to the cells
            T lroe[2];
#pragma unroll
            for (int d = 0; d < 2; d++) {
                T acc = T(0);
#pragma unroll
                for (int a = 0; a < 3; a++)
#pragma unroll
                    for (int b = 0; b < 3; b++) acc = acc + lL[a][b] * Ld[a][b].d[d] + lR[a][b] * Rd[a][b].d[d];
                lroe[d] = acc;
            }
            T lx[6];
            roe_chain(rf, lroe[0], lroe[1], gm1, lx);
            const int cl = chk(p.ctl, ghost_map(j, n, p.bc_lo, p.bc_hi), 0, n),
                      cr = chk(p.ctl, ghost_map(j + 1, n, p.bc_lo, p.bc_hi), 0, n);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                add_to(&out[(size_t)c * n + cl], lx[c]);
                add_to(&out[(size_t)c * n + cr], lx[3 + c]);
            }
        }
        __syncwarp();
    }
}

// out = c1 x + c2 (y + c3 z); x may be null.
template <typename T>
__global__ void combine_kernel(T *out, const T *x, const T *y, const T *z, T c1, T c2, T c3, size_t N) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const T a = x ? c1 * x[i] : T(0);
        out[i] = a + c2 * (y[i] + c3 * z[i]);
    }
}

// out1 = a1 x + b1 y; out2 = a2 x + b2 y (if out2); x may be null.  out1 may
// alias x or y (each element is read before it is written).
template <typename T>
__global__ void combine2_kernel(T *out1, T *out2, const T *x, const T *y, T a1, T b1, T a2, T b2, size_t N) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const T xv = x ? x[i] : T(0), yv = y[i];
        out1[i] = a1 * xv + b1 * yv;
        if (out2) out2[i] = a2 * xv + b2 * yv;
    }
}

template <typename T>
cudaError_t launch_combine2(void *out1, void *out2, const void *x, const void *y, double a1, double b1, double a2,
                            double b2, size_t N, cudaStream_t st) {
    int grid = (int)((N + 255) / 256);
    if (grid > num_sms() * 8) grid = num_sms() * 8;
    combine2_kernel<T><<<grid, 256, 0, st>>>(static_cast<T *>(out1), static_cast<T *>(out2),
                                             static_cast<const T *>(x), static_cast<const T *>(y), T(a1), T(b1),
                                             T(a2), T(b2), N);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rhs_adjoint1d(const Adjoint1D &p, cudaStream_t st) {
    const int ntiles = (p.n + WT - 1) / WT;
    const int nw = warps_per_cta(ntiles, true);
    int grid = (ntiles + nw - 1) / nw;
    if (grid > num_sms() * 4 * (WPB / nw)) grid = num_sms() * 4 * (WPB / nw);
    rhs_adjoint1d_kernel<T><<<grid, nw * 32, 0, st>>>(p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_combine(void *out, const void *x, const void *y, const void *z, double c1, double c2, double c3,
                           size_t N, cudaStream_t st) {
    int grid = (int)((N + 255) / 256);
    if (grid > num_sms() * 8) grid = num_sms() * 8;
    combine_kernel<T><<<grid, 256, 0, st>>>(static_cast<T *>(out), static_cast<const T *>(x),
                                            static_cast<const T *>(y), static_cast<const T *>(z), T(c1), T(c2),
                                            T(c3), N);
    return cudaGetLastError();
}

}  // namespace t7
