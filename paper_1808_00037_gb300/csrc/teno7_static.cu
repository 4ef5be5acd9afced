// teno7_static.cu -- t7_rk3_step_static: one SSP-RK3 step of a 1D system that
// allocates no device memory, for callers that cannot call cudaMalloc (see
// include/teno7.h).  Its scratch -- the two RK stage buffers and the device
// control block the stage kernels reduce alpha into -- lives in the file-scope
// array below instead of a context's workspace.  The kernels are the same as
// t7_rk3_step's; only the origin of their scratch pointers differs.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "teno7.h"
#include "teno7_internal.h"

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char t7_static_scratch[T7_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
// Device address of t7_static_scratch per device ordinal, looked up once per
// device (std::call_once, so host threads making their first calls at the
// same time do not race on the slot).  The name t7_static_scratch in host
// code is only a host-side stand-in, never a device address.
struct ScratchSlot {
    std::once_flag once;
    void *ptr = nullptr;
    cudaError_t err = cudaSuccess;
};
ScratchSlot g_scratch[kMaxDevices];

constexpr size_t kCtlBytes = (sizeof(t7::DevCtl) + 255) / 256 * 256;

t7_status report(char *errbuf, size_t errlen, t7_status st, const char *fmt, ...) {
    if (errbuf && errlen) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(errbuf, errlen, fmt, ap);
        va_end(ap);
    }
    return st;
}

}  // namespace

extern "C" t7_status t7_rk3_step_static(const t7_grid *g, void *U, double dt, void *stream_ptr, char *errbuf,
                                        size_t errlen) {
    if (!g || !U || !(dt > 0.0)) return report(errbuf, errlen, T7_EINVAL, "t7_rk3_step_static: bad argument");
    if (g->sys != T7_SCALAR_ADVECTION && g->sys != T7_EULER1D && g->sys != T7_BURGERS)
        return report(errbuf, errlen, T7_EINVAL, "t7_rk3_step_static: only 1D systems are supported");
    if ((g->prec != T7_F64 && g->prec != T7_F32) || g->nx < 1 || g->ny != 1 || !(g->dx > 0.0) ||
        !(g->CT > 0.0 && g->CT < 1.0) || g->bc[0] < 0 || g->bc[0] > 1 || g->bc[1] < 0 || g->bc[1] > 1)
        return report(errbuf, errlen, T7_EINVAL, "t7_rk3_step_static: bad grid");
    if (g->scheme != T7_TENO7EXT || g->alpha_mode != T7_ALPHA_GLOBAL)
        return report(errbuf, errlen, T7_EINVAL, "t7_rk3_step_static: runs TENO7-ext with the global alpha only");
    const int m = g->sys == T7_EULER1D ? 3 : 1;
    const size_t esize = g->prec == T7_F64 ? 8 : 4;
    const size_t buf = ((size_t)m * g->nx * esize + 255) / 256 * 256;
    if (kCtlBytes + 2 * buf > (size_t)T7_STATIC_SCRATCH_BYTES)
        return report(errbuf, errlen, T7_EINVAL,
                      "t7_rk3_step_static: %d cells x %d variables x %zu bytes needs %zu scratch bytes, more than "
                      "the %u-byte static scratch; use t7_create/t7_rk3_step",
                      g->nx, m, esize, kCtlBytes + 2 * buf, (unsigned)T7_STATIC_SCRATCH_BYTES);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return report(errbuf, errlen, T7_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return report(errbuf, errlen, T7_EINVAL, "device ordinal %d too large", dev);
    ScratchSlot &slot = g_scratch[dev];
    std::call_once(slot.once, [&slot] {  // set-up, once per device, with that device current
        slot.err = cudaGetSymbolAddress(&slot.ptr, t7_static_scratch);
        if (slot.err == cudaSuccess && !slot.ptr) slot.err = cudaErrorInvalidSymbol;
    });
    if (slot.err != cudaSuccess)
        return report(errbuf, errlen, T7_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(slot.err));
    unsigned char *base = static_cast<unsigned char *>(slot.ptr);
    t7::DevCtl *ctl = reinterpret_cast<t7::DevCtl *>(base);
    void *U1 = base + kCtlBytes;
    void *U2 = base + kCtlBytes + buf;
    cudaStream_t stream = (cudaStream_t)stream_ptr;

    // The array keeps the previous call's contents: clear the control block
    // (alpha slots, error word, CTA counter); err_index starts large.
    if ((e = cudaMemsetAsync(ctl, 0, sizeof(t7::DevCtl), stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(&ctl->err_index, 0x7f, sizeof(int), stream)) != cudaSuccess)
        return report(errbuf, errlen, T7_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));

    t7::Alpha1D a;
    memset(&a, 0, sizeof(a));  // alpha_rec stays null
    a.U = U;
    a.n = g->nx;
    a.sys = g->sys;
    a.gamma = g->gamma;
    a.a = g->adv_speed;
    a.ctl = ctl;
    a.slot = 0;
    e = g->prec == T7_F64 ? t7::launch_alpha1d_f64(a, stream) : t7::launch_alpha1d_f32(a, stream);
    void *in[3] = {U, U1, U2};
    void *out[3] = {U1, U2, U};
    for (int k = 0; k < 3 && e == cudaSuccess; k++) {
        t7::Stage1D p;
        memset(&p, 0, sizeof(p));
        p.Us = in[k];
        p.U0 = k == 0 ? nullptr : U;
        p.out = out[k];
        p.n = g->nx;
        p.sys = g->sys;
        p.bc_lo = g->bc[0];
        p.bc_hi = g->bc[1];
        p.dx = g->dx;
        p.eps = g->eps_x < 0.0 ? g->dx * g->dx * g->dx : g->eps_x;
        p.CT = g->CT;
        p.gamma = g->gamma;
        p.a = g->adv_speed;
        p.stage = k;
        p.dt_fixed = dt;
        p.ctl = ctl;
        p.slot_in = k;
        p.f_dx = (float)p.dx;
        p.f_eps = (float)p.eps;
        p.f_CT = (float)p.CT;
        p.f_gamma = (float)p.gamma;
        p.f_gm1 = (float)(p.gamma - 1.0);
        p.f_a = (float)p.a;
        p.f_dt_fixed = (float)dt;
        e = g->prec == T7_F64 ? t7::launch_stage1d_f64(p, stream) : t7::launch_stage1d_f32(p, stream);
    }
    if (e != cudaSuccess) return report(errbuf, errlen, T7_ECUDA, "launch: %s", cudaGetErrorString(e));

    int err[2] = {0, 0};
    if ((e = cudaMemcpyAsync(err, &ctl->err, 2 * sizeof(int), cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(stream)) != cudaSuccess)
        return report(errbuf, errlen, T7_ECUDA, "status read: %s", cudaGetErrorString(e));
    if (err[0] & t7::ERR_INDEX)
        return report(errbuf, errlen, T7_EINDEX, "index check failed (checked build): index %d", err[1]);
    if (err[0] & t7::ERR_NONPHYSICAL)
        return report(errbuf, errlen, T7_ENONPHYSICAL, "non-physical state near index %d", err[1]);
    if (err[0]) return report(errbuf, errlen, T7_ENONFINITE, "non-finite state near index %d", err[1]);
    report(errbuf, errlen, T7_OK, "no error");
    return T7_OK;
}
