// lrb_fp64_peak_probe: the FP64 pipe's throughput on this device, measured.
//
// Every FP64 kernel of the library is bound by the FP64 pipe (GB300 runs
// binary64 FMAs on about two lanes per SM per clock), so its roofline
// denominator is that pipe's peak.  A figure derived from unit counts and the
// maximum clock assumes the clock the kernel actually ran at; this probe
// measures instead: every thread of a full-GPU grid runs eight independent
// FMA chains (enough independent work to keep the pipe busy on every
// sub-partition), and the rate is counted from the FMAs issued and the
// kernel's event-timed duration.
#include <algorithm>

#include "lrb_internal.h"

namespace lrb {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(kProbeThreads) k_dfma_probe(double* out, long long iters, double x, double y) {
    double a[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) a[c] = fma(a[c], x, y);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += a[c];
    // the store depends on every chain, so none of them is dead code; it
    // happens only for an impossible value, so the probe writes nothing
    if (s == -1.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace lrb

using namespace lrb;

extern "C" lrb_status lrb_fp64_peak_probe(int device, long long iters, double* tflops, double* ms) {
    if (!tflops || !ms || iters <= 0) {
        set_last_error("lrb_fp64_peak_probe: null output or iters <= 0");
        return LRB_ERR_INVALID;
    }
    cudaError_t e = cudaSetDevice(device);
    int sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfma_probe, kProbeThreads, 0);
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int grid = sms * std::max(1, std::min(per_sm, 4));
    if (e == cudaSuccess) {
        // a short warm-up launch, then the timed one
        k_dfma_probe<<<grid, kProbeThreads, 0, s>>>(nullptr, std::max(1LL, iters / 16), 0.9999999, 1e-9);
        e = cudaEventRecord(e0, s);
    }
    if (e == cudaSuccess) {
        k_dfma_probe<<<grid, kProbeThreads, 0, s>>>(nullptr, iters, 0.9999999, 1e-9);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return LRB_ERR_DEVICE;
    }
    const double flops = 2.0 * kProbeChains * (double)iters * grid * kProbeThreads;
    *ms = t;
    *tflops = flops / (t * 1e-3) / 1e12;
    return LRB_OK;
}
