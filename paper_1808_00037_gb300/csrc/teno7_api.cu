// teno7_api.cu -- the C ABI of libteno7 (declared in include/teno7.h): context
// and workspace management, argument validation, the SSP-RK3 stage sequence
// and the device-side CFL time stepping.  All compute is in the kernels of
// teno7_kernels.cuh; this file only validates, allocates and launches.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <numeric>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "teno7.h"
#include "teno7_internal.h"
#include "teno7_adjoint_params.h"

struct t7_ctx {
    t7_grid g;
    int m;                 // conserved variables
    size_t esize;          // bytes per element (8 or 4)
    size_t ncell;          // nx * ny
    cudaStream_t stream;
    int device;
    void *U1, *U2;         // RK stage buffers
    void *R;               // 2D: x part of L(U)
    void *Uhost;           // device state for the host-array entry point
    t7::DevCtl *ctl;       // device control block
    // ragged-batch metadata (device), grown on demand
    long long *b_off;
    double *b_dx, *b_t;
    int *b_order, *b_steps, *b_queue;
    int b_cap;
    int b_group;           // warps per tube chosen by t7_batch_autotune (0: not tuned)
    std::vector<double> b_cost;  // estimated cost (cells x estimated steps) of the tubes in processing order
    void *adj[3];          // adjoint work vectors (allocated on first use)
    uint8_t *adj_masks[3]; // FP32: forward masks of the three stage states
    t7::DevCtl *ctl_host;  // pinned mirror for status reads
    // CUDA graph of one chunk of RK3 steps of t7_run (small 1D problems, where
    // launch overhead dominates): captured on an internal stream for the
    // state pointer g_U, replayed behind events on the context's stream
    cudaStream_t gstream;
    cudaEvent_t g_in, g_out;
    cudaGraphExec_t gexec;
    void *g_U;
    // t7_run_host with a known step count: the last stage is launched in parts
    // and each finished part is copied to the host array on cstream
    cudaStream_t cstream;
    cudaEvent_t c_ev[8], c_done;
    cudaEvent_t sw_ev;     // t7_set_stream: orders the new stream after the old one
    char err[512];
};

namespace {

// NVTX range around an entry point (or a phase of one), for profiler
// timelines; costs a pointer test when no tool is attached.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

t7_status fail(t7_ctx *c, t7_status st, const char *fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

t7_status cuda_fail(t7_ctx *c, cudaError_t e, const char *what) {
    return fail(c, T7_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int nvars(int sys) { return sys == T7_EULER1D ? 3 : (sys == T7_EULER2D ? 4 : 1); }

bool is_1d(int sys) { return sys == T7_SCALAR_ADVECTION || sys == T7_EULER1D || sys == T7_BURGERS; }

// default epsilon: dx^3 for TENO7-ext, 1e-40 for the TENO5 baseline
double eps_of(double eps, double d, int scheme = T7_TENO7EXT) {
    return eps < 0.0 ? (scheme == T7_TENO5 ? 1e-40 : d * d * d) : eps;
}

__global__ void ctl_begin_kernel(t7::DevCtl *ctl, double t_end, double cfl, double dx, double dy, int max_steps) {
    for (int s = 0; s < 3; s++) ctl->amax[s][0] = ctl->amax[s][1] = ctl->amax[s][2] = 0ull;
    ctl->t = 0.0;
    ctl->dt = 0.0;
    ctl->t_end = t_end;
    ctl->cfl = cfl;
    ctl->dx = dx;
    ctl->dy = dy;
    ctl->steps = 0;
    ctl->max_steps = max_steps;
    ctl->active = 1;
    ctl->blocks_done = 0u;
}

t7::Stage1D stage_params(t7_ctx *c, const void *Us, const void *U0, void *out) {
    t7::Stage1D p;
    memset(&p, 0, sizeof(p));
    p.Us = Us;
    p.U0 = U0;
    p.out = out;
    p.n = c->g.nx;
    p.sys = c->g.sys;
    p.bc_lo = c->g.bc[0];
    p.bc_hi = c->g.bc[1];
    p.dx = c->g.dx;
    p.eps = eps_of(c->g.eps_x, c->g.dx, c->g.scheme);
    p.CT = c->g.CT;
    p.gamma = c->g.gamma;
    p.a = c->g.adv_speed;
    p.ctl = c->ctl;
    p.scheme = c->g.scheme;
    p.alpha_mode = c->g.alpha_mode;
    p.f_dx = (float)p.dx;
    p.f_eps = (float)p.eps;
    p.f_CT = (float)p.CT;
    p.f_gamma = (float)p.gamma;
    p.f_gm1 = (float)(p.gamma - 1.0);
    p.f_a = (float)p.a;
    return p;
}

cudaError_t stage(t7_ctx *c, const t7::Stage1D &p) {
    if (c->g.prec == T7_MIXED) return t7::launch_stage1d_mixed(p, c->stream);
    return c->g.prec == T7_F64 ? t7::launch_stage1d_f64(p, c->stream) : t7::launch_stage1d_f32(p, c->stream);
}

t7::Stage2D stage2d_params(t7_ctx *c, const void *Us, const void *U0, void *out, void *R) {
    t7::Stage2D p;
    memset(&p, 0, sizeof(p));
    p.Us = Us;
    p.U0 = U0;
    p.out = out;
    p.R = R;
    p.nx = c->g.nx;
    p.ny = c->g.ny;
    for (int b = 0; b < 4; b++) p.bc[b] = c->g.bc[b];
    p.dx = c->g.dx;
    p.dy = c->g.dy;
    p.eps_x = eps_of(c->g.eps_x, c->g.dx);
    p.eps_y = eps_of(c->g.eps_y, c->g.dy);
    p.CT = c->g.CT;
    p.gamma = c->g.gamma;
    p.ctl = c->ctl;
    p.f_dx = (float)p.dx;
    p.f_dy = (float)p.dy;
    p.f_eps_x = (float)p.eps_x;
    p.f_eps_y = (float)p.eps_y;
    p.f_CT = (float)p.CT;
    p.f_gamma = (float)p.gamma;
    p.f_gm1 = (float)(p.gamma - 1.0);
    return p;
}

cudaError_t stage2d(t7_ctx *c, const t7::Stage2D &p) {
    if (c->g.prec == T7_MIXED) return t7::launch_stage2d_mixed(p, c->stream);
    return c->g.prec == T7_F64 ? t7::launch_stage2d_f64(p, c->stream) : t7::launch_stage2d_f32(p, c->stream);
}

// alpha(U) (per direction in 2D) into slot 0, no slot cleared
cudaError_t alpha_launch(t7_ctx *c, const void *U) {
    if (c->g.sys == T7_EULER2D) {
        t7::Alpha2D a;
        memset(&a, 0, sizeof(a));
        a.U = U;
        a.nx = c->g.nx;
        a.ny = c->g.ny;
        a.gamma = c->g.gamma;
        a.ctl = c->ctl;
        a.slot = 0;
        return c->g.prec != T7_F32 ? t7::launch_alpha2d_f64(a, c->stream) : t7::launch_alpha2d_f32(a, c->stream);
    }
    t7::Alpha1D a;
    memset(&a, 0, sizeof(a));  // alpha_rec stays null
    a.U = U;
    a.n = c->g.nx;
    a.sys = c->g.sys;
    a.gamma = c->g.gamma;
    a.a = c->g.adv_speed;
    a.ctl = c->ctl;
    a.slot = 0;
    a.alpha_mode = c->g.alpha_mode;
    // (a mixed-precision state is FP64)
    return c->g.prec != T7_F32 ? t7::launch_alpha1d_f64(a, c->stream) : t7::launch_alpha1d_f32(a, c->stream);
}

// alpha(U) into slot 0 after clearing all slots
cudaError_t alpha_init(t7_ctx *c, const void *U) {
    cudaError_t e = cudaMemsetAsync(c->ctl->amax, 0, sizeof(c->ctl->amax), c->stream);
    if (e != cudaSuccess) return e;
    return alpha_launch(c, U);
}


// The last stage of a step (1D) in OUT_PARTS launches over consecutive
// ranges of warp tiles; each finished range of cells is copied from U to the
// host array host_out ([m][nx], pageable or page-locked) on the copy stream
// while the next range computes, so the result leaves the device at the
// CPU-GPU link's rate, overlapped with the stage's own compute.  All launches
// are queued before the copies, so that a copy to pageable memory that blocks
// the host does not hold back the compute.  The context's stream waits for the
// copies.
constexpr int OUT_PARTS = 8;
cudaError_t last_stage_to_host(t7_ctx *c, t7::Stage1D p, void *host_out) {
    TraceRange trace("last stage in parts, copied out");
    cudaError_t e = cudaSuccess;
    if (!c->cstream) {
        if ((e = cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking)) != cudaSuccess) return e;
        for (int k = 0; k < OUT_PARTS; k++)
            if ((e = cudaEventCreateWithFlags(&c->c_ev[k], cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&c->c_done, cudaEventDisableTiming)) != cudaSuccess) return e;
    }
    const int nx = c->g.nx;
    const int ntiles = (nx + t7::TILE_CELLS - 1) / t7::TILE_CELLS;
    const int parts = ntiles < OUT_PARTS ? ntiles : OUT_PARTS;
    int lo[OUT_PARTS], hi[OUT_PARTS];
    for (int k = 0; k < parts; k++) {
        lo[k] = (int)((long long)ntiles * k / parts);
        hi[k] = (int)((long long)ntiles * (k + 1) / parts);
        p.tile_lo = lo[k];
        p.tile_hi = hi[k];
        p.partial = k < parts - 1;
        if ((e = stage(c, p)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(c->c_ev[k], c->stream)) != cudaSuccess) return e;
    }
    const size_t es = c->esize, row = (size_t)nx * es;
    for (int k = 0; k < parts; k++) {
        const size_t c0 = (size_t)lo[k] * t7::TILE_CELLS;
        size_t c1 = (size_t)hi[k] * t7::TILE_CELLS;
        if (c1 > (size_t)nx) c1 = (size_t)nx;
        if ((e = cudaStreamWaitEvent(c->cstream, c->c_ev[k], 0)) != cudaSuccess) return e;
        if ((e = cudaMemcpy2DAsync(static_cast<char *>(host_out) + c0 * es, row,
                                   static_cast<const char *>(p.out) + c0 * es, row, (c1 - c0) * es, (size_t)c->m,
                                   cudaMemcpyDeviceToHost, c->cstream)) != cudaSuccess)
            return e;
    }
    if ((e = cudaEventRecord(c->c_done, c->cstream)) != cudaSuccess) return e;
    return cudaStreamWaitEvent(c->stream, c->c_done, 0);
}

// three stage launches; dt_fixed > 0 fixes the step, otherwise CFL on device.
// host_out (nullable, 1D): the step's result is also copied to this host array
// (see last_stage_to_host).
cudaError_t rk3(t7_ctx *c, void *U, double dt_fixed, void *host_out = nullptr) {
    void *bufs_in[3] = {U, c->U1, c->U2};
    void *bufs_out[3] = {c->U1, c->U2, U};
    if (c->g.sys == T7_EULER2D) {
        for (int k = 0; k < 3; k++) {
            t7::Stage2D p = stage2d_params(c, bufs_in[k], k == 0 ? nullptr : U, bufs_out[k], c->R);
            p.rhs_mode = 0;
            p.stage = k;
            p.dt_fixed = dt_fixed;
            p.f_dt_fixed = (float)dt_fixed;
            p.slot_in = k;
            cudaError_t e = stage2d(c, p);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    for (int k = 0; k < 3; k++) {
        t7::Stage1D p = stage_params(c, bufs_in[k], k == 0 ? nullptr : U, bufs_out[k]);
        p.rhs_mode = 0;
        p.stage = k;
        p.dt_fixed = dt_fixed;
        p.f_dt_fixed = (float)dt_fixed;
        p.slot_in = k;
        cudaError_t e = (k == 2 && host_out) ? last_stage_to_host(c, p, host_out) : stage(c, p);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// read and clear the latched device error; stream must be idle
t7_status collect(t7_ctx *c) {
    cudaError_t e = cudaMemcpy(c->ctl_host, c->ctl, sizeof(t7::DevCtl), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "reading the control block");
    int err = c->ctl_host->err, idx = c->ctl_host->err_index;
    if (err) {
        int zero = 0, big = 0x7fffffff;
        cudaMemcpy(&c->ctl->err, &zero, sizeof(int), cudaMemcpyHostToDevice);
        cudaMemcpy(&c->ctl->err_index, &big, sizeof(int), cudaMemcpyHostToDevice);
        if (err & t7::ERR_INDEX)
            return fail(c, T7_EINDEX, "index check failed (checked build): index %d", idx);
        if (err & t7::ERR_NONPHYSICAL)
            return fail(c, T7_ENONPHYSICAL, "non-physical state (rho <= 0, p <= 0 or c^2 <= 0) near index %d", idx);
        return fail(c, T7_ENONFINITE, "non-finite state or unreachable stencil pattern near index %d", idx);
    }
    return T7_OK;
}

t7_status check_sys(t7_ctx *c) {
    if (!c) return T7_EINVAL;
    return T7_OK;
}

}  // namespace

namespace t7 {
cudaError_t launch_ctl_begin(DevCtl *ctl, double t_end, double cfl, double dx, double dy, int max_steps,
                             cudaStream_t s) {
    ctl_begin_kernel<<<1, 1, 0, s>>>(ctl, t_end, cfl, dx, dy, max_steps);
    return cudaGetLastError();
}
}  // namespace t7

extern "C" {

t7_status t7_create(const t7_grid *g, void *stream, t7_ctx **out) {
    if (!g || !out) return T7_EINVAL;
    *out = nullptr;
    if (g->sys != T7_SCALAR_ADVECTION && g->sys != T7_EULER1D && g->sys != T7_BURGERS && g->sys != T7_EULER2D)
        return T7_EINVAL;
    if (g->prec != T7_F64 && g->prec != T7_F32 && g->prec != T7_MIXED) return T7_EINVAL;
    if (g->nx < 1 || g->ny < 1 || (is_1d(g->sys) && g->ny != 1)) return T7_EINVAL;
    if (!(g->dx > 0.0) || (g->sys == T7_EULER2D && !(g->dy > 0.0))) return T7_EINVAL;
    for (int b = 0; b < 4; b++)
        if (g->bc[b] != T7_BC_PERIODIC && g->bc[b] != T7_BC_ZERO_GRADIENT) return T7_EINVAL;
    if ((double)g->nx * (double)g->ny * nvars(g->sys) > 2147483647.0) return T7_EINVAL;
    if (!(g->CT > 0.0 && g->CT < 1.0)) return T7_EINVAL;
    if (g->scheme != T7_TENO7EXT && g->scheme != T7_TENO5) return T7_EINVAL;
    if (g->scheme == T7_TENO5 && !is_1d(g->sys)) return T7_EINVAL;  // the baseline runs the 1D systems
    if (g->alpha_mode != T7_ALPHA_GLOBAL && g->alpha_mode != T7_ALPHA_PER_FIELD) return T7_EINVAL;
    // per-field alphas: 1D Euler, TENO7-ext, FP64 or FP32
    if (g->alpha_mode == T7_ALPHA_PER_FIELD &&
        (g->sys != T7_EULER1D || g->scheme != T7_TENO7EXT || g->prec == T7_MIXED))
        return T7_EINVAL;
    t7_ctx *c = new (std::nothrow) t7_ctx();  // value-initialised: every pointer and count zero
    if (!c) return T7_ENOMEM;
    c->g = *g;
    c->m = nvars(g->sys);
    c->esize = g->prec == T7_F32 ? 4 : 8;
    c->ncell = (size_t)g->nx * g->ny;
    c->stream = (cudaStream_t)stream;
    cudaGetDevice(&c->device);
    size_t bytes = c->ncell * c->m * c->esize;
    if (cudaMalloc(&c->U1, bytes) != cudaSuccess || cudaMalloc(&c->U2, bytes) != cudaSuccess ||
        cudaMalloc(&c->Uhost, bytes) != cudaSuccess ||
        (g->sys == T7_EULER2D && cudaMalloc(&c->R, bytes) != cudaSuccess) ||
        cudaMalloc((void **)&c->ctl, sizeof(t7::DevCtl)) != cudaSuccess ||
        cudaMallocHost((void **)&c->ctl_host, sizeof(t7::DevCtl)) != cudaSuccess) {
        t7_destroy(c);
        cudaGetLastError();
        return T7_ENOMEM;
    }
    t7::DevCtl init;
    memset(&init, 0, sizeof(init));
    init.err_index = 0x7fffffff;
    init.max_steps = 0;
    if (cudaMemcpy(c->ctl, &init, sizeof(init), cudaMemcpyHostToDevice) != cudaSuccess) {
        t7_destroy(c);
        cudaGetLastError();
        return T7_ECUDA;
    }
    snprintf(c->err, sizeof(c->err), "no error");
    *out = c;
    return T7_OK;
}

t7_status t7_destroy(t7_ctx *c) {
    if (!c) return T7_EINVAL;
    if (c->U1) cudaFree(c->U1);
    if (c->U2) cudaFree(c->U2);
    if (c->Uhost) cudaFree(c->Uhost);
    if (c->R) cudaFree(c->R);
    if (c->b_off) cudaFree(c->b_off);
    if (c->b_dx) cudaFree(c->b_dx);
    if (c->b_t) cudaFree(c->b_t);
    if (c->b_order) cudaFree(c->b_order);
    if (c->b_steps) cudaFree(c->b_steps);
    if (c->b_queue) cudaFree(c->b_queue);
    for (int k = 0; k < 3; k++) {
        if (c->adj[k]) cudaFree(c->adj[k]);
        if (c->adj_masks[k]) cudaFree(c->adj_masks[k]);
    }
    if (c->ctl) cudaFree(c->ctl);
    if (c->ctl_host) cudaFreeHost(c->ctl_host);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->g_in) cudaEventDestroy(c->g_in);
    if (c->g_out) cudaEventDestroy(c->g_out);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    for (int k = 0; k < 8; k++)
        if (c->c_ev[k]) cudaEventDestroy(c->c_ev[k]);
    if (c->c_done) cudaEventDestroy(c->c_done);
    if (c->cstream) cudaStreamDestroy(c->cstream);
    if (c->sw_ev) cudaEventDestroy(c->sw_ev);
    delete c;
    return T7_OK;
}

t7_status t7_set_stream(t7_ctx *c, void *stream) {
    if (!c) return T7_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (s == c->stream) return T7_OK;
    // the context's buffers may still be in use by work queued on the old
    // stream: the new stream waits for it
    cudaError_t e = cudaSuccess;
    if (!c->sw_ev) e = cudaEventCreateWithFlags(&c->sw_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(c->sw_ev, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->sw_ev, 0);
    if (e != cudaSuccess) return cuda_fail(c, e, "t7_set_stream: ordering the new stream after the old one");
    c->stream = s;
    return T7_OK;
}

const char *t7_last_error(const t7_ctx *c) { return c ? c->err : "null context"; }

t7_status t7_sync(t7_ctx *c) {
    if (!c) return T7_EINVAL;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
    return collect(c);
}

t7_status t7_teno7_reconstruct(t7_ctx *c, const void *v, int n, int sign, double eps, void *fhat, uint8_t *d3,
                               uint8_t *D5) {
    TraceRange trace("t7_teno7_reconstruct");
    if (!c) return T7_EINVAL;
    if (!v || !fhat || n < 1 || (sign != 1 && sign != -1) || !(eps > 0.0))
        return fail(c, T7_EINVAL, "t7_teno7_reconstruct: bad argument");
    if (c->g.scheme != T7_TENO7EXT || c->g.prec == T7_MIXED)
        return fail(c, T7_EINVAL, "t7_teno7_reconstruct: a TENO7-ext FP64 or FP32 context only");
    t7::Recon p;
    memset(&p, 0, sizeof(p));
    p.v = v;
    p.fhat = fhat;
    p.d3 = d3;
    p.D5 = D5;
    p.n = n;
    p.sign = sign;
    p.eps = eps;
    p.CT = c->g.CT;
    p.ctl = c->ctl;
    cudaError_t e = c->g.prec == T7_F64 ? t7::launch_recon_f64(p, c->stream) : t7::launch_recon_f32(p, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "reconstruct launch");
    return T7_OK;
}

t7_status t7_euler_rhs(t7_ctx *c, const void *U, void *dUdt, uint8_t *masks) {
    TraceRange trace("t7_euler_rhs");
    t7_status st = check_sys(c);
    if (st) return st;
    if (!U || !dUdt) return fail(c, T7_EINVAL, "t7_euler_rhs: null array");
    cudaError_t e = alpha_init(c, U);
    if (e != cudaSuccess) return cuda_fail(c, e, "alpha");
    if (c->g.sys == T7_EULER2D) {
        t7::Stage2D p = stage2d_params(c, U, nullptr, dUdt, dUdt);
        p.rhs_mode = 1;
        p.masks = masks;
        p.slot_in = 0;
        e = stage2d(c, p);
        if (e != cudaSuccess) return cuda_fail(c, e, "rhs launch");
        return T7_OK;
    }
    t7::Stage1D p = stage_params(c, U, nullptr, dUdt);
    p.rhs_mode = 1;
    p.masks = masks;
    p.slot_in = 0;
    e = stage(c, p);
    if (e != cudaSuccess) return cuda_fail(c, e, "rhs launch");
    return T7_OK;
}

t7_status t7_cfl_dt(t7_ctx *c, const void *U, double cfl, double *dt_out) {
    TraceRange trace("t7_cfl_dt");
    t7_status st = check_sys(c);
    if (st) return st;
    if (!U || !dt_out || !(cfl > 0.0)) return fail(c, T7_EINVAL, "t7_cfl_dt: bad argument");
    cudaError_t e = alpha_init(c, U);
    if (e != cudaSuccess) return cuda_fail(c, e, "alpha");
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "sync");
    if ((st = collect(c))) return st;
    double alpha = 0.0, alpha_y = 0.0;
    unsigned long long bits = c->ctl_host->amax[0][0], bits_y = c->ctl_host->amax[0][1];
    memcpy(&alpha, &bits, sizeof(alpha));
    memcpy(&alpha_y, &bits_y, sizeof(alpha_y));
    if (c->g.alpha_mode == T7_ALPHA_PER_FIELD) {
        // the CFL step of the largest per-field alpha (equal to the global alpha)
        for (int k = 1; k < 3; k++) {
            double ak;
            unsigned long long bk = c->ctl_host->amax[0][k];
            memcpy(&ak, &bk, sizeof(ak));
            alpha = fmax(alpha, ak);
        }
        alpha_y = 0.0;
    }
    if (c->g.sys == T7_EULER2D)
        *dt_out = cfl / (alpha / c->g.dx + alpha_y / c->g.dy);
    else
        *dt_out = (cfl * c->g.dx) / alpha;
    return T7_OK;
}

t7_status t7_rk3_step(t7_ctx *c, void *U, double dt) {
    TraceRange trace("t7_rk3_step");
    t7_status st = check_sys(c);
    if (st) return st;
    if (!U || !(dt > 0.0)) return fail(c, T7_EINVAL, "t7_rk3_step: bad argument");
    cudaError_t e = alpha_init(c, U);
    if (e != cudaSuccess) return cuda_fail(c, e, "alpha");
    if ((e = rk3(c, U, dt)) != cudaSuccess) return cuda_fail(c, e, "stage launch");
    return T7_OK;
}

// ---------------------------------------------------------------- slabs ----
// One rank's (or one stream's) part of a 1D domain split into slabs: arrays
// padded by HALO_CELLS cells per side, halos filled by the caller, the global
// alpha passed in as a device value (see include/teno7.h).
static t7_status slab_check(t7_ctx *c, const char *what) {
    if (!c) return T7_EINVAL;
    if (c->g.alpha_mode != T7_ALPHA_GLOBAL) return fail(c, T7_EINVAL, "%s: slabs take the global alpha", what);
    if (!is_1d(c->g.sys) && c->g.sys != T7_EULER2D) return fail(c, T7_EINVAL, "%s: not a slab system", what);
    return T7_OK;
}

// 2D slab: offset (bytes) of row 0 of a padded array, and its variable stride
static size_t slab2d_row0(const t7_ctx *c) { return (size_t)t7::HALO_CELLS * c->g.nx * c->esize; }
static size_t slab2d_stride(const t7_ctx *c) { return (size_t)c->g.nx * (c->g.ny + 2 * t7::HALO_CELLS); }

static const void *off_c(const void *p, size_t bytes) {
    return p ? static_cast<const void *>(static_cast<const char *>(p) + bytes) : nullptr;
}

static cudaError_t stage2d_slab(t7_ctx *c, const t7::Stage2D &p) {
    if (c->g.prec == T7_MIXED) return t7::launch_stage2d_slab_mixed(p, c->stream);
    return c->g.prec == T7_F64 ? t7::launch_stage2d_slab_f64(p, c->stream) : t7::launch_stage2d_slab_f32(p, c->stream);
}

// one RHS (rhs_mode) or RK stage of a 2D slab; out is padded in RK mode
static t7::Stage2D slab2d_params(t7_ctx *c, const void *Us, const void *U0, void *out, int rhs_mode,
                                 const double *alpha_in) {
    const size_t row0 = slab2d_row0(c);
    void *o = rhs_mode ? out : static_cast<char *>(out) + row0;
    t7::Stage2D p = stage2d_params(c, off_c(Us, row0), off_c(U0, row0), o, rhs_mode ? out : c->R);
    p.halo = 1;
    p.sv = slab2d_stride(c);
    p.svo = rhs_mode ? (size_t)c->g.nx * c->g.ny : p.sv;
    p.alpha_in = alpha_in;
    p.rhs_mode = rhs_mode;
    return p;
}

static t7::Stage1D slab_params(t7_ctx *c, const void *Us, const void *U0, void *out, const double *alpha_in) {
    t7::Stage1D p = stage_params(c, Us, U0, out);
    p.halo = 1;
    p.alpha_in = alpha_in;
    return p;
}

// alpha of the slab's cells (the padded array's interior) into *alpha_out
static cudaError_t slab_alpha_launch(t7_ctx *c, const void *U, double *alpha_out) {
    cudaError_t e = cudaMemsetAsync(&c->ctl->amax[0][0], 0, 2 * sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return e;
    if (c->g.sys == T7_EULER2D) {
        t7::Alpha2D a;
        memset(&a, 0, sizeof(a));
        a.U = off_c(U, slab2d_row0(c));
        a.nx = c->g.nx;
        a.ny = c->g.ny;
        a.stride = slab2d_stride(c);
        a.gamma = c->g.gamma;
        a.ctl = c->ctl;
        a.slot = 0;
        a.alpha_rec = alpha_out;
        return c->g.prec != T7_F32 ? t7::launch_alpha2d_slab_f64(a, c->stream)
                                   : t7::launch_alpha2d_slab_f32(a, c->stream);
    }
    t7::Alpha1D a;
    memset(&a, 0, sizeof(a));
    a.U = static_cast<const char *>(U) + t7::HALO_CELLS * c->esize;
    a.n = c->g.nx;
    a.stride = c->g.nx + 2 * t7::HALO_CELLS;
    a.sys = c->g.sys;
    a.gamma = c->g.gamma;
    a.a = c->g.adv_speed;
    a.ctl = c->ctl;
    a.slot = 0;
    a.alpha_rec = alpha_out;
    return c->g.prec != T7_F32 ? t7::launch_alpha1d_f64(a, c->stream) : t7::launch_alpha1d_f32(a, c->stream);
}

extern "C" t7_status t7_slab_alpha(t7_ctx *c, const void *U, double *alpha_out) {
    TraceRange trace("t7_slab_alpha");
    t7_status st = slab_check(c, "t7_slab_alpha");
    if (st) return st;
    if (!U || !alpha_out) return fail(c, T7_EINVAL, "t7_slab_alpha: null pointer");
    cudaError_t e = slab_alpha_launch(c, U, alpha_out);
    if (e != cudaSuccess) return cuda_fail(c, e, "slab alpha launch");
    return T7_OK;
}

extern "C" t7_status t7_slab_rhs(t7_ctx *c, const void *U, const double *alpha, void *dUdt, uint8_t *masks) {
    TraceRange trace("t7_slab_rhs");
    t7_status st = slab_check(c, "t7_slab_rhs");
    if (st) return st;
    if (!U || !alpha || !dUdt) return fail(c, T7_EINVAL, "t7_slab_rhs: null pointer");
    if (c->g.sys == T7_EULER2D) {
        t7::Stage2D p = slab2d_params(c, U, nullptr, dUdt, 1, alpha);
        p.masks = masks;
        cudaError_t e = stage2d_slab(c, p);
        if (e != cudaSuccess) return cuda_fail(c, e, "slab rhs launch");
        return T7_OK;
    }
    t7::Stage1D p = slab_params(c, U, nullptr, dUdt, alpha);
    p.rhs_mode = 1;
    p.masks = masks;
    cudaError_t e = stage(c, p);
    if (e != cudaSuccess) return cuda_fail(c, e, "slab rhs launch");
    return T7_OK;
}

extern "C" t7_status t7_slab_stage(t7_ctx *c, int k, const void *Us, const void *U0, void *out, const double *alpha,
                                   double dt, double *alpha_out) {
    TraceRange trace("t7_slab_stage");
    t7_status st = slab_check(c, "t7_slab_stage");
    if (st) return st;
    if (k < 0 || k > 2 || !Us || !out || !alpha || !(dt > 0.0) || (k > 0 && !U0))
        return fail(c, T7_EINVAL, "t7_slab_stage: bad argument");
    if (Us == out) return fail(c, T7_EINVAL, "t7_slab_stage: the stage input may not alias the output");
    // the slot this launch reduces the output's alpha into starts at zero
    const int so = (k + 1) % 3;
    cudaError_t e = cudaMemsetAsync(&c->ctl->amax[so][0], 0, 2 * sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "slab stage slot");
    if (c->g.sys == T7_EULER2D) {
        t7::Stage2D p = slab2d_params(c, Us, k == 0 ? nullptr : U0, out, 0, alpha);
        p.stage = k;
        p.dt_fixed = dt;
        p.f_dt_fixed = (float)dt;
        p.slot_in = k;
        p.alpha_rec = alpha_out;
        e = stage2d_slab(c, p);
        if (e != cudaSuccess) return cuda_fail(c, e, "slab stage launch");
        return T7_OK;
    }
    t7::Stage1D p = slab_params(c, Us, k == 0 ? nullptr : U0, out, alpha);
    p.rhs_mode = 0;
    p.stage = k;
    p.dt_fixed = dt;
    p.f_dt_fixed = (float)dt;
    p.slot_in = k;
    p.alpha_rec = alpha_out;
    e = stage(c, p);
    if (e != cudaSuccess) return cuda_fail(c, e, "slab stage launch");
    return T7_OK;
}

// Steps per t7_run chunk, and the size up to which a chunk runs as one CUDA
// graph (below it a stage launch lasts a few microseconds and launch overhead
// dominates; above it the 3 launches per step cost nothing measurable).
constexpr int RUN_CHUNK = 64;
constexpr size_t GRAPH_MAX_VALUES = size_t(1) << 21;

// One chunk of RUN_CHUNK steps of U as a replayed graph (captured on first use
// for this U).  Returns 1 when the chunk was enqueued; 0, with no work
// enqueued, if the graph cannot be made or launched (the caller then launches
// the steps one by one); -1 if the chunk was launched but could not be ordered
// before later work on the context's stream.
static int run_chunk_graph(t7_ctx *c, void *U) {
    if (!c->gstream) {
        if (cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->g_in, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->g_out, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
    }
    if (!c->gexec || c->g_U != U) {
        if (c->gexec) cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
        cudaStream_t user = c->stream;
        c->stream = c->gstream;
        cudaError_t e = cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal);
        for (int q = 0; q < RUN_CHUNK && e == cudaSuccess; q++) e = rk3(c, U, -1.0);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(c->gstream, &g);
        c->stream = user;
        if (e != cudaSuccess || e2 != cudaSuccess || !g ||
            cudaGraphInstantiate(&c->gexec, g, 0) != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            c->gexec = nullptr;
            cudaGetLastError();
            return 0;
        }
        cudaGraphDestroy(g);
        c->g_U = U;
    }
    if (cudaEventRecord(c->g_in, c->stream) != cudaSuccess ||
        cudaStreamWaitEvent(c->gstream, c->g_in, 0) != cudaSuccess ||
        cudaGraphLaunch(c->gexec, c->gstream) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (cudaEventRecord(c->g_out, c->gstream) != cudaSuccess ||
        cudaStreamWaitEvent(c->stream, c->g_out, 0) != cudaSuccess)
        return -1;
    return 1;
}

// t7_run's loop; host_out (nullable, 1D, only with t_end = inf) receives a
// copy of the result of the last step, made while its last stage computes.
static t7_status run_core(t7_ctx *c, void *U, double cfl, double t_end, int max_steps, int *steps_out, double *t_out,
                          void *host_out) {
    t7_status st;
    cudaError_t e = t7::launch_ctl_begin(c->ctl, t_end, cfl, c->g.dx, c->g.dy, max_steps, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ctl");
    e = alpha_launch(c, U);
    if (e != cudaSuccess) return cuda_fail(c, e, "alpha");
    // Steps are launched in chunks; between chunks the host polls whether the
    // device-side clock has reached t_end (a step past it is a no-op anyway).
    const bool graphs = is_1d(c->g.sys) && c->ncell * c->m <= GRAPH_MAX_VALUES;
    int launched = 0;
    while (launched < max_steps) {
        int k = max_steps - launched < RUN_CHUNK ? max_steps - launched : RUN_CHUNK;
        const bool last_chunk = host_out && launched + k == max_steps;
        const int g = (graphs && k == RUN_CHUNK && !last_chunk) ? run_chunk_graph(c, U) : 0;
        if (g < 0) return cuda_fail(c, cudaGetLastError(), "ordering a graph chunk");
        if (g == 0) {
            for (int q = 0; q < k; q++) {
                void *last = (host_out && launched + q == max_steps - 1) ? host_out : nullptr;
                if ((e = rk3(c, U, -1.0, last)) != cudaSuccess) return cuda_fail(c, e, "stage launch");
            }
        }
        launched += k;
        if (isfinite(t_end)) {
            if ((e = cudaMemcpyAsync(c->ctl_host, c->ctl, sizeof(t7::DevCtl), cudaMemcpyDeviceToHost, c->stream)) !=
                cudaSuccess)
                return cuda_fail(c, e, "poll");
            if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "sync");
            if (!c->ctl_host->active || c->ctl_host->err || !(c->ctl_host->t < t_end)) break;
        }
    }
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "sync");
    st = collect(c);
    if (steps_out) *steps_out = c->ctl_host->steps;
    if (t_out) *t_out = c->ctl_host->t;
    return st;
}

t7_status t7_run(t7_ctx *c, void *U, double cfl, double t_end, int max_steps, int *steps_out, double *t_out) {
    TraceRange trace("t7_run");
    t7_status st = check_sys(c);
    if (st) return st;
    if (!U || !(cfl > 0.0) || max_steps < 0 || !(t_end >= 0.0)) return fail(c, T7_EINVAL, "t7_run: bad argument");
    return run_core(c, U, cfl, t_end, max_steps, steps_out, t_out, nullptr);
}

t7_status t7_run_host(t7_ctx *c, void *U_host, double cfl, double t_end, int max_steps, int *steps_out,
                      double *t_out) {
    TraceRange trace("t7_run_host");
    t7_status st = check_sys(c);
    if (st) return st;
    if (c->g.alpha_mode != T7_ALPHA_GLOBAL) return fail(c, T7_EINVAL, "t7_run_host takes the global alpha");
    if (!U_host || !(cfl > 0.0) || max_steps < 0 || !(t_end >= 0.0))
        return fail(c, T7_EINVAL, "t7_run_host: bad argument");
    size_t bytes = c->ncell * c->m * c->esize;
    cudaError_t e;
    {
        TraceRange phase("t7_run_host: copy in");
        e = cudaMemcpyAsync(c->Uhost, U_host, bytes, cudaMemcpyHostToDevice, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "H2D copy");
    // With a known number of steps (t_end = inf) in 1D, the last step's last
    // stage is launched in parts and each finished part is copied back while
    // the rest computes; otherwise the result is copied after the run.
    if (is_1d(c->g.sys) && isinf(t_end) && max_steps >= 1)
        return run_core(c, c->Uhost, cfl, t_end, max_steps, steps_out, t_out, U_host);
    st = run_core(c, c->Uhost, cfl, t_end, max_steps, steps_out, t_out, nullptr);
    if (st != T7_OK && st != T7_ENONPHYSICAL && st != T7_ENONFINITE) return st;
    e = cudaMemcpyAsync(U_host, c->Uhost, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "D2H copy");
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "sync");
    return st;
}

// -------------------------------------------------------------- adjoint ----
static t7_status adj_check(t7_ctx *c) {
    if (!c) return T7_EINVAL;
    if (c->g.alpha_mode != T7_ALPHA_GLOBAL) return fail(c, T7_EINVAL, "the adjoint takes the global alpha");
    if (c->g.sys != T7_EULER1D) return fail(c, T7_EINVAL, "the adjoint takes a 1D Euler context");
    if (c->g.scheme != T7_TENO7EXT || c->g.prec == T7_MIXED)
        return fail(c, T7_EINVAL, "the adjoint takes a TENO7-ext FP64 or FP32 context");
    const size_t bytes = c->ncell * c->m * c->esize;
    const size_t mbytes = (size_t)2 * 3 * (c->g.nx + 1);
    for (int k = 0; k < 3; k++) {
        if (!c->adj[k] && cudaMalloc(&c->adj[k], bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, T7_ENOMEM, "adjoint buffers");
        }
        if (c->g.prec == T7_F32 && !c->adj_masks[k] && cudaMalloc((void **)&c->adj_masks[k], mbytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, T7_ENOMEM, "adjoint mask buffers");
        }
    }
    return T7_OK;
}

// out = (dL/dU)^T v at U with alpha from `slot`, masks frozen (given or recomputed)
static cudaError_t adj_apply(t7_ctx *c, const void *U, int slot, const uint8_t *masks, const void *v, void *out) {
    cudaError_t e = cudaMemsetAsync(out, 0, c->ncell * c->m * c->esize, c->stream);
    if (e != cudaSuccess) return e;
    t7::Adjoint1D a;
    memset(&a, 0, sizeof(a));
    a.U = U;
    a.v = v;
    a.out = out;
    a.masks = masks;
    a.n = c->g.nx;
    a.bc_lo = c->g.bc[0];
    a.bc_hi = c->g.bc[1];
    a.dx = c->g.dx;
    a.eps = eps_of(c->g.eps_x, c->g.dx);
    a.CT = c->g.CT;
    a.gamma = c->g.gamma;
    a.ctl = c->ctl;
    a.slot_in = slot;
    a.scale = 1.0;
    return c->g.prec == T7_F64 ? t7::launch_rhs_adjoint1d_f64(a, c->stream) : t7::launch_rhs_adjoint1d_f32(a, c->stream);
}

// out += scale (dL/dU)^T v at U with recorded alpha and masks (no zeroing)
static cudaError_t adj_accumulate(t7_ctx *c, const void *U, const double *alpha, const uint8_t *masks, const void *v,
                                  void *out, double scale) {
    t7::Adjoint1D a;
    memset(&a, 0, sizeof(a));
    a.U = U;
    a.v = v;
    a.out = out;
    a.masks = masks;
    a.n = c->g.nx;
    a.bc_lo = c->g.bc[0];
    a.bc_hi = c->g.bc[1];
    a.dx = c->g.dx;
    a.eps = eps_of(c->g.eps_x, c->g.dx);
    a.CT = c->g.CT;
    a.gamma = c->g.gamma;
    a.ctl = c->ctl;
    a.alpha_ptr = alpha;
    a.scale = scale;
    return c->g.prec == T7_F64 ? t7::launch_rhs_adjoint1d_f64(a, c->stream) : t7::launch_rhs_adjoint1d_f32(a, c->stream);
}

static cudaError_t combine2(t7_ctx *c, void *out1, void *out2, const void *x, const void *y, double a1, double b1,
                            double a2, double b2) {
    const size_t N = c->ncell * c->m;
    return c->g.prec == T7_F64 ? t7::launch_combine2_f64(out1, out2, x, y, a1, b1, a2, b2, N, c->stream)
                               : t7::launch_combine2_f32(out1, out2, x, y, a1, b1, a2, b2, N, c->stream);
}

// Layout of one tape entry: U1, U2 (state-sized), the forward Delta codes of
// the three stage states ([2][3][n+1] bytes each) and their three alphas.
struct TapeLayout {
    size_t u1, u2, masks[3], alpha, total;
};
static TapeLayout tape_layout(const t7_ctx *c) {
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    TapeLayout L;
    const size_t sb = up(c->ncell * c->m * c->esize), mb = up((size_t)2 * c->m * (c->g.nx + 1));
    L.u1 = 0;
    L.u2 = sb;
    L.masks[0] = 2 * sb;
    L.masks[1] = 2 * sb + mb;
    L.masks[2] = 2 * sb + 2 * mb;
    L.alpha = 2 * sb + 3 * mb;
    L.total = L.alpha + 256;
    return L;
}

static cudaError_t combine(t7_ctx *c, void *out, const void *x, const void *y, const void *z, double c1, double c2,
                           double c3) {
    const size_t N = c->ncell * c->m;
    return c->g.prec == T7_F64 ? t7::launch_combine_f64(out, x, y, z, c1, c2, c3, N, c->stream)
                               : t7::launch_combine_f32(out, x, y, z, c1, c2, c3, N, c->stream);
}

// FP32: masks of the forward stage kernel at state U (alpha in `slot`), so the
// adjoint uses exactly the forward's selection
static cudaError_t forward_masks(t7_ctx *c, const void *U, int slot, uint8_t *masks, void *scratch) {
    t7::Stage1D p = stage_params(c, U, nullptr, scratch);
    p.rhs_mode = 1;
    p.masks = masks;
    p.slot_in = slot;
    return stage(c, p);
}

t7_status t7_euler_rhs_adjoint(t7_ctx *c, const void *U, const void *v, void *out) {
    TraceRange trace("t7_euler_rhs_adjoint");
    t7_status st = adj_check(c);
    if (st) return st;
    if (!U || !v || !out) return fail(c, T7_EINVAL, "t7_euler_rhs_adjoint: null array");
    cudaError_t e = alpha_init(c, U);
    const uint8_t *masks = nullptr;
    if (e == cudaSuccess && c->g.prec == T7_F32) {
        e = forward_masks(c, U, 0, c->adj_masks[0], c->adj[0]);
        masks = c->adj_masks[0];
    }
    if (e == cudaSuccess) e = adj_apply(c, U, 0, masks, v, out);
    if (e != cudaSuccess) return cuda_fail(c, e, "adjoint launch");
    return T7_OK;
}

t7_status t7_rk3_step_adjoint(t7_ctx *c, const void *U, double dt, void *lambda) {
    TraceRange trace("t7_rk3_step_adjoint");
    t7_status st = adj_check(c);
    if (st) return st;
    if (!U || !lambda || !(dt > 0.0)) return fail(c, T7_EINVAL, "t7_rk3_step_adjoint: bad argument");
    // Recompute the stage states U1, U2; slot k holds alpha of stage state k
    // while it is needed (the stage-1 launch clears slot 0, so alpha(U) is
    // taken again before the last adjoint application).  FP32 records each
    // state's forward masks as soon as its alpha is known.
    const void *Us[3] = {U, c->U1, c->U2};
    const uint8_t *mk[3] = {nullptr, nullptr, nullptr};
    cudaError_t e = alpha_init(c, U);
    for (int k = 0; k < 3 && e == cudaSuccess; k++) {
        if (c->g.prec == T7_F32) {
            e = forward_masks(c, Us[k], k, c->adj_masks[k], c->adj[0]);
            mk[k] = c->adj_masks[k];
        }
        if (k == 2 || e != cudaSuccess) break;
        t7::Stage1D p = stage_params(c, Us[k], k == 0 ? nullptr : U, k == 0 ? c->U1 : c->U2);
        p.rhs_mode = 0;
        p.stage = k;
        p.dt_fixed = dt;
        p.f_dt_fixed = (float)dt;
        p.slot_in = k;
        e = stage(c, p);
    }
    void *tmp = c->adj[0], *w = c->adj[1], *acc = c->adj[2];
    // U3 = U/3 + 2/3 (U2 + dt L(U2))
    if (e == cudaSuccess) e = adj_apply(c, Us[2], 2, mk[2], lambda, tmp);
    if (e == cudaSuccess) e = combine(c, w, nullptr, lambda, tmp, 0.0, 2.0 / 3.0, dt);
    if (e == cudaSuccess) e = combine(c, acc, nullptr, lambda, lambda, 0.0, 1.0 / 3.0, 0.0);
    // U2 = 3/4 U + 1/4 (U1 + dt L(U1))
    if (e == cudaSuccess) e = adj_apply(c, Us[1], 1, mk[1], w, tmp);
    if (e == cudaSuccess) e = combine(c, acc, acc, w, w, 1.0, 0.75, 0.0);
    if (e == cudaSuccess) e = combine(c, w, nullptr, w, tmp, 0.0, 0.25, dt);
    // U1 = U + dt L(U); alpha(U) into slot 0 again (cleared by the stage-1 launch)
    if (e == cudaSuccess) e = alpha_launch(c, U);
    if (e == cudaSuccess) e = adj_apply(c, Us[0], 0, mk[0], w, tmp);
    if (e == cudaSuccess) e = combine(c, lambda, acc, w, tmp, 1.0, 1.0, dt);
    if (e != cudaSuccess) return cuda_fail(c, e, "adjoint step");
    return T7_OK;
}

t7_status t7_tape_bytes(t7_ctx *c, size_t *bytes) {
    if (!c || !bytes) return T7_EINVAL;
    *bytes = tape_layout(c).total;
    return T7_OK;
}

t7_status t7_rk3_step_record(t7_ctx *c, const void *U_in, void *U_out, double dt, void *tape) {
    TraceRange trace("t7_rk3_step_record");
    t7_status st = adj_check(c);
    if (st) return st;
    if (!U_in || !U_out || !tape || !(dt > 0.0)) return fail(c, T7_EINVAL, "t7_rk3_step_record: bad argument");
    if ((reinterpret_cast<uintptr_t>(tape) & 255u) != 0)
        return fail(c, T7_EINVAL, "t7_rk3_step_record: tape must be 256-byte aligned");
    const TapeLayout L = tape_layout(c);
    unsigned char *t = static_cast<unsigned char *>(tape);
    double *alpha = reinterpret_cast<double *>(t + L.alpha);
    void *Ust[3] = {const_cast<void *>(U_in), t + L.u1, t + L.u2};
    void *Uo[3] = {t + L.u1, t + L.u2, U_out};
    cudaError_t e = cudaMemsetAsync(c->ctl->amax, 0, sizeof(c->ctl->amax), c->stream);
    if (e == cudaSuccess) {
        t7::Alpha1D a;
        memset(&a, 0, sizeof(a));
        a.U = U_in;
        a.n = c->g.nx;
        a.sys = c->g.sys;
        a.gamma = c->g.gamma;
        a.a = c->g.adv_speed;
        a.ctl = c->ctl;
        a.slot = 0;
        a.alpha_rec = alpha;
        e = c->g.prec == T7_F64 ? t7::launch_alpha1d_f64(a, c->stream) : t7::launch_alpha1d_f32(a, c->stream);
    }
    for (int k = 0; k < 3 && e == cudaSuccess; k++) {
        t7::Stage1D p = stage_params(c, Ust[k], k == 0 ? nullptr : U_in, Uo[k]);
        p.rhs_mode = 0;
        p.stage = k;
        p.dt_fixed = dt;
        p.f_dt_fixed = (float)dt;
        p.slot_in = k;
        p.masks = reinterpret_cast<uint8_t *>(t + L.masks[k]);
        p.alpha_rec = k < 2 ? alpha + k + 1 : nullptr;
        e = stage(c, p);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "recorded step");
    return T7_OK;
}

t7_status t7_rk3_step_adjoint_recorded(t7_ctx *c, const void *U_in, const void *tape, double dt, void *lambda) {
    TraceRange trace("t7_rk3_step_adjoint_recorded");
    t7_status st = adj_check(c);
    if (st) return st;
    if (!U_in || !tape || !lambda || !(dt > 0.0))
        return fail(c, T7_EINVAL, "t7_rk3_step_adjoint_recorded: bad argument");
    const TapeLayout L = tape_layout(c);
    const unsigned char *t = static_cast<const unsigned char *>(tape);
    const double *alpha = reinterpret_cast<const double *>(t + L.alpha);
    const void *Us[3] = {U_in, t + L.u1, t + L.u2};
    const uint8_t *mk[3];
    for (int k = 0; k < 3; k++) mk[k] = t + L.masks[k];
    void *A = c->adj[0], *W = c->adj[1], *T = c->adj[2];
    // U3 = U/3 + 2/3 (U2 + dt L(U2)):  W = 2/3 lam + 2/3 dt L2^T lam,  A = lam/3
    cudaError_t e = combine2(c, W, A, nullptr, lambda, 0.0, 2.0 / 3.0, 0.0, 1.0 / 3.0);
    if (e == cudaSuccess) e = adj_accumulate(c, Us[2], alpha + 2, mk[2], lambda, W, (2.0 / 3.0) * dt);
    // U2 = 3/4 U + 1/4 (U1 + dt L(U1)):  A += 3/4 W,  T = W/4 + dt/4 L1^T W
    if (e == cudaSuccess) e = combine2(c, A, T, A, W, 1.0, 0.75, 0.0, 0.25);
    if (e == cudaSuccess) e = adj_accumulate(c, Us[1], alpha + 1, mk[1], W, T, 0.25 * dt);
    // U1 = U + dt L(U):  lam = A + T + dt L0^T T
    if (e == cudaSuccess) e = combine2(c, lambda, nullptr, A, T, 1.0, 1.0, 0.0, 0.0);
    if (e == cudaSuccess) e = adj_accumulate(c, Us[0], alpha, mk[0], T, lambda, dt);
    if (e != cudaSuccess) return cuda_fail(c, e, "adjoint of a recorded step");
    return T7_OK;
}

// ---------------------------------------------------------------- batch ----
// Uploads the batch metadata and the processing order.  A tube's cost is
// estimated as cells x steps, its step count as min(max_steps,
// t_end alpha / (CFL dx)) with alpha the tube's wave speed in U (one pass of
// batch1d_alpha_kernel): both the cell count and the wave speed, which varies
// by more than an order of magnitude across random Riemann data, decide it.
// With t_end infinite (the autotuner's fixed-step trials) every tube takes
// max_steps steps and no pass is needed.
static t7_status batch_prepare(t7_ctx *c, const void *U, const int64_t *offsets, const double *dx, int ntubes,
                               double t_end, double cfl, int max_steps) {
    if (ntubes > c->b_cap) {
        cudaFree(c->b_off);
        cudaFree(c->b_dx);
        cudaFree(c->b_t);
        cudaFree(c->b_order);
        cudaFree(c->b_steps);
        cudaFree(c->b_queue);
        c->b_off = nullptr;
        c->b_dx = c->b_t = nullptr;
        c->b_order = c->b_steps = c->b_queue = nullptr;
        c->b_cap = 0;
        if (cudaMalloc((void **)&c->b_off, sizeof(long long) * (ntubes + 1)) != cudaSuccess ||
            cudaMalloc((void **)&c->b_dx, sizeof(double) * ntubes) != cudaSuccess ||
            cudaMalloc((void **)&c->b_t, sizeof(double) * ntubes) != cudaSuccess ||
            cudaMalloc((void **)&c->b_order, sizeof(int) * ntubes) != cudaSuccess ||
            cudaMalloc((void **)&c->b_steps, sizeof(int) * ntubes) != cudaSuccess ||
            cudaMalloc((void **)&c->b_queue, 2 * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, T7_ENOMEM, "batch metadata allocation failed");
        }
        c->b_cap = ntubes;
    }
    std::vector<long long> off(offsets, offsets + ntubes + 1);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(c->b_off, off.data(), sizeof(long long) * (ntubes + 1), cudaMemcpyHostToDevice,
                             c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c->b_dx, dx, sizeof(double) * ntubes, cudaMemcpyHostToDevice, c->stream)) !=
            cudaSuccess)
        return cuda_fail(c, e, "batch metadata copy");
    const bool timed = std::isfinite(t_end);
    std::vector<double> alpha(ntubes, 0.0);
    if (timed) {
        t7::Batch1D p;
        memset(&p, 0, sizeof(p));
        p.U = const_cast<void *>(U);
        p.offsets = c->b_off;
        p.ntubes = ntubes;
        p.Ntot = c->g.nx;
        p.gamma = c->g.gamma;
        // the per-tube alphas go to b_t, which the batch launch overwrites with final times
        e = c->g.prec == T7_F64 ? t7::launch_batch1d_alpha_f64(p, c->b_t, c->stream)
                                : t7::launch_batch1d_alpha_f32(p, c->b_t, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(alpha.data(), c->b_t, sizeof(double) * ntubes, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "batch wave speeds");
    }
    std::vector<double> cost(ntubes);
    for (int t = 0; t < ntubes; t++) {
        double steps = (double)max_steps;
        if (timed) {
            const double s = t_end * alpha[t] / (cfl * dx[t]);
            if (std::isfinite(s)) steps = std::min(steps, std::max(1.0, std::ceil(s)));
        }
        cost[t] = (double)(offsets[t + 1] - offsets[t]) * steps;
    }
    // costliest first
    std::vector<int> order(ntubes);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    c->b_cost.assign(ntubes, 0.0);
    for (int q = 0; q < ntubes; q++) c->b_cost[q] = cost[order[q]];  // in processing order
    if ((e = cudaMemcpyAsync(c->b_order, order.data(), sizeof(int) * ntubes, cudaMemcpyHostToDevice, c->stream)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "batch metadata copy");
    return T7_OK;
}

// Tubes whose estimated cost exceeds half of a group's fair share of the whole
// batch run on whole CTAs (the leading tubes of the costliest-first order), so
// that the longest tube does not set the run time on a small group.
static int batch_nbig(t7_ctx *c, int ntubes, int group) {
    if (group >= 8 || ntubes < 1) return 0;
    const int ngroups = c->g.prec == T7_F64 ? t7::batch1d_groups_f64(group) : t7::batch1d_groups_f32(group);
    double total = 0.0;
    for (int q = 0; q < ntubes; q++) total += c->b_cost[q];
    const double share = total / (ngroups > 0 ? ngroups : 1);
    int nbig = 0;
    while (nbig < ntubes && c->b_cost[nbig] > 0.5 * share) nbig++;
    return nbig;
}

static cudaError_t batch_launch(t7_ctx *c, void *U, int ntubes, double t_end, double cfl, int max_steps,
                                int group, bool whole_cta_phase) {
    cudaError_t e = cudaMemsetAsync(c->b_queue, 0, 2 * sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    t7::Batch1D p;
    memset(&p, 0, sizeof(p));
    p.U = U;
    p.W1 = c->U1;
    p.W2 = c->U2;
    p.offsets = c->b_off;
    p.dx = c->b_dx;
    p.order = c->b_order;
    p.ntubes = ntubes;
    p.Ntot = c->g.nx;
    p.bc_lo = c->g.bc[0];
    p.bc_hi = c->g.bc[1];
    p.t_end = t_end;
    p.cfl = cfl;
    p.gamma = c->g.gamma;
    p.CT = c->g.CT;
    p.max_steps = max_steps;
    p.group_warps = group;
    p.nbig = whole_cta_phase ? batch_nbig(c, ntubes, group) : 0;
    p.queue = c->b_queue;
    p.steps_out = c->b_steps;
    p.t_out = c->b_t;
    p.ctl = c->ctl;
    return c->g.prec == T7_F64 ? t7::launch_batch1d_f64(p, c->stream) : t7::launch_batch1d_f32(p, c->stream);
}

static t7_status batch_check(t7_ctx *c, void *U, const int64_t *offsets, const double *dx, int ntubes) {
    if (!c) return T7_EINVAL;
    if (c->g.alpha_mode != T7_ALPHA_GLOBAL) return fail(c, T7_EINVAL, "batches take the global alpha");
    if (c->g.sys != T7_EULER1D) return fail(c, T7_EINVAL, "batches take a 1D Euler context");
    if (c->g.scheme != T7_TENO7EXT || c->g.prec == T7_MIXED)
        return fail(c, T7_EINVAL, "batches take a TENO7-ext FP64 or FP32 context");
    if (!U || !offsets || !dx || ntubes < 1) return fail(c, T7_EINVAL, "batch: bad argument");
    if (offsets[0] != 0 || offsets[ntubes] != (int64_t)c->g.nx)
        return fail(c, T7_EINVAL, "batch: offsets must run from 0 to the context's nx (%d)", c->g.nx);
    for (int t = 0; t < ntubes; t++) {
        if (offsets[t + 1] - offsets[t] < 1) return fail(c, T7_EINVAL, "batch: tube %d is empty", t);
        if (!(dx[t] > 0.0)) return fail(c, T7_EINVAL, "batch: dx of tube %d is not positive", t);
    }
    return T7_OK;
}

t7_status t7_batch_run(t7_ctx *c, void *U, const int64_t *offsets, const double *dx, int ntubes, double t_end,
                       double cfl, int max_steps, int group_warps, int *steps_out, double *t_out) {
    TraceRange trace("t7_batch_run");
    t7_status st = batch_check(c, U, offsets, dx, ntubes);
    if (st) return st;
    if (!(cfl > 0.0) || !(t_end >= 0.0) || max_steps < 0) return fail(c, T7_EINVAL, "t7_batch_run: bad argument");
    const int gw = group_warps < 0 ? -group_warps : group_warps;
    int group = gw > 0 ? gw : (c->b_group > 0 ? c->b_group : 8);
    if (group != 1 && group != 2 && group != 4 && group != 8)
        return fail(c, T7_EINVAL, "t7_batch_run: group_warps must be 0, +-1, +-2, +-4 or +-8");
    if ((st = batch_prepare(c, U, offsets, dx, ntubes, t_end, cfl, max_steps))) return st;
    cudaError_t e = batch_launch(c, U, ntubes, t_end, cfl, max_steps, group, group_warps <= 0);
    if (e != cudaSuccess) return cuda_fail(c, e, "batch launch");
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "sync");
    if (steps_out && (e = cudaMemcpy(steps_out, c->b_steps, sizeof(int) * ntubes, cudaMemcpyDeviceToHost)) !=
                         cudaSuccess)
        return cuda_fail(c, e, "steps copy");
    if (t_out && (e = cudaMemcpy(t_out, c->b_t, sizeof(double) * ntubes, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(c, e, "t copy");
    return collect(c);
}

t7_status t7_batch_autotune(t7_ctx *c, const void *U, const int64_t *offsets, const double *dx, int ntubes,
                            double cfl, int trial_steps, int *group_out, float *ms_out) {
    TraceRange trace("t7_batch_autotune");
    t7_status st = batch_check(c, (void *)U, offsets, dx, ntubes);
    if (st) return st;
    if (!(cfl > 0.0) || trial_steps < 1) return fail(c, T7_EINVAL, "t7_batch_autotune: bad argument");
    if ((st = batch_prepare(c, U, offsets, dx, ntubes, INFINITY, cfl, trial_steps))) return st;
    const size_t bytes = c->ncell * c->m * c->esize;
    const int groups[4] = {1, 2, 4, 8};
    float best = 0.f;
    int best_g = 8;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int gi = 0; gi < 4; gi++) {
        // every candidate advances the same copy of the state by trial_steps steps
        cudaError_t e = cudaMemcpyAsync(c->Uhost, U, bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
        if (e == cudaSuccess) e = batch_launch(c, c->Uhost, ntubes, INFINITY, cfl, trial_steps, groups[gi], false);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(c, e, "autotune trial");
        }
        if (ms_out) ms_out[gi] = ms;
        if (gi == 0 || ms < best) {
            best = ms;
            best_g = groups[gi];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->b_group = best_g;
    if (group_out) *group_out = best_g;
    return collect(c);
}

}  // extern "C"
