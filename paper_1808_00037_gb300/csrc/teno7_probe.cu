// teno7_probe.cu -- measured arithmetic peaks of the device (include/teno7_probe.h):
// long independent chains of fused multiply-adds, timed with CUDA events, give
// the FP32 (scalar and packed f32x2) and FP64 rates the stage kernels' ALU
// roofline is taken against.  Not part of the method.
#include <cuda_runtime.h>
#include <string.h>

#include "teno7_internal.h"
#include "teno7_probe.h"

namespace {

constexpr int kChains = 8;     // independent accumulators per thread
constexpr int kThreads = 256;  // threads per CTA

// Each thread runs kChains independent chains x <- x * a + b for `iters`
// iterations (2 flop per FMA); the results are written only if they reach an
// impossible value, so the chains are live but no memory traffic is timed.
__global__ void __launch_bounds__(kThreads) fma_f32_kernel(int iters, float a, float b, float *sink) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < 16; u++)
#pragma unroll
            for (int c = 0; c < kChains; c++) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    if (s == -1.2345f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) fma_f32x2_kernel(int iters, float a, float b, float *sink) {
    float2 x[kChains];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = make_float2((float)(threadIdx.x + c), (float)(threadIdx.x - c));
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < 16; u++)
#pragma unroll
            for (int c = 0; c < kChains; c++) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c].x + x[c].y;
    if (s == -1.2345f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) fma_f64_kernel(int iters, double a, double b, double *sink) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = (double)(threadIdx.x + c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < 16; u++)
#pragma unroll
            for (int c = 0; c < kChains; c++) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    if (s == -1.2345) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" t7_status t7_probe_fma(int kind, int iters, int repeats, void *stream_ptr, double *tflops, float *ms) {
    if (!tflops || (kind != T7_PROBE_F32 && kind != T7_PROBE_F32X2 && kind != T7_PROBE_F64) || iters < 1 ||
        repeats < 1)
        return T7_EINVAL;
    cudaStream_t st = (cudaStream_t)stream_ptr;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return T7_ECUDA;
    const void *fn = kind == T7_PROBE_F32 ? (const void *)fma_f32_kernel
                     : kind == T7_PROBE_F32X2 ? (const void *)fma_f32x2_kernel
                                              : (const void *)fma_f64_kernel;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0) != cudaSuccess || per_sm < 1)
        return T7_ECUDA;
    const int grid = sms * per_sm;
    void *sink = nullptr;
    if (cudaMalloc(&sink, (size_t)grid * sizeof(double)) != cudaSuccess) return T7_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    t7_status rc = T7_OK;
    float best = 0.f;
    auto launch = [&]() {
        if (kind == T7_PROBE_F32)
            fma_f32_kernel<<<grid, kThreads, 0, st>>>(iters, 0.999f, 1e-3f, (float *)sink);
        else if (kind == T7_PROBE_F32X2)
            fma_f32x2_kernel<<<grid, kThreads, 0, st>>>(iters, 0.999f, 1e-3f, (float *)sink);
        else
            fma_f64_kernel<<<grid, kThreads, 0, st>>>(iters, 0.999, 1e-3, (double *)sink);
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = T7_ECUDA;
    } else {
        launch();  // warm-up
        for (int r = 0; r < repeats && rc == T7_OK; r++) {
            float t = 0.f;
            if (cudaEventRecord(e0, st) != cudaSuccess) rc = T7_ECUDA;
            launch();
            if (rc == T7_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
                rc = T7_ECUDA;
            if (rc == T7_OK && (r == 0 || t < best)) best = t;
        }
        if (cudaGetLastError() != cudaSuccess) rc = T7_ECUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc != T7_OK) return rc;
    // 2 flop per FMA; f32x2 does two FMAs per instruction
    const double fmas = (double)grid * kThreads * kChains * 16.0 * iters * (kind == T7_PROBE_F32X2 ? 2.0 : 1.0);
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    if (ms) *ms = best;
    return T7_OK;
}

extern "C" t7_status t7_probe_index_check(int i, int lo, int hi, int *index_out, int *flagged_out,
                                          int *checked_build_out) {
    if (!index_out || !flagged_out || !checked_build_out || lo >= hi) return T7_EINVAL;
    void *buf = nullptr;
    if (cudaMalloc(&buf, sizeof(t7::DevCtl) + 2 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return T7_ENOMEM;
    }
    t7::DevCtl *ctl = static_cast<t7::DevCtl *>(buf);
    int *out = reinterpret_cast<int *>(static_cast<char *>(buf) + sizeof(t7::DevCtl));
    t7::DevCtl h;
    memset(&h, 0, sizeof(h));
    h.err_index = 0x7fffffff;
    int res[2] = {0, 0};
    t7_status rc = T7_OK;
    if (cudaMemcpy(ctl, &h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess ||
        t7::launch_index_check_probe(i, lo, hi, ctl, out, 0) != cudaSuccess ||
        cudaMemcpy(res, out, sizeof(res), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&h, ctl, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = T7_ECUDA;
    cudaFree(buf);
    if (rc != T7_OK) {
        cudaGetLastError();
        return rc;
    }
    *index_out = res[0];
    *flagged_out = (h.err & t7::ERR_INDEX) && h.err_index == i ? 1 : 0;
    *checked_build_out = res[1];
    return T7_OK;
}
