// cr_probe.cu -- crsolve_peak_probe: the measured arithmetic rate of the GPU
// for the rooflines of the benchmark.
//
// The FP64 path is bound by the FP64 FMA pipe, whose rate no driver table
// lists for this GPU.  The probe runs independent FMA chains (eight per
// thread, enough threads for several warps per scheduler) with no memory
// traffic, times them with CUDA events on the caller's stream and returns
// the rate in GFLOP/s (2 flop per FMA).  The FP32 variant gives the rate of
// the FP32 levels of the mixed-precision form.
#include <cstdint>

#include "crsolve.h"
#include "cr_launch.h"
#include "cr_tc.cuh"

namespace {

__device__ double g_probe_sink_d;
__device__ float g_probe_sink_f;
__device__ unsigned long long g_probe_cycles;

template <class R>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, R b, R c) {
    const long long t0 = clock64();
    R a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = R(threadIdx.x) * R(1e-7) + R(i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
    }
    R s = R(0);
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    // never true for these inputs; keeps every chain live
    if (s == R(-1.25)) {
        if (sizeof(R) == 8) g_probe_sink_d = (double)s;
        else g_probe_sink_f = (float)s;
    }
    // the longest CTA in SM cycles: the CTAs of the single wave share their
    // SM's pipe, so the last one to finish spans the whole kernel
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(&g_probe_cycles, (unsigned long long)(clock64() - t0));
}

template <class R>
int run_probe(int iters, int blocks, int per_sm, cudaStream_t s, double *gflops, double *per_clk, double *mhz) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess) return CRSOLVE_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return CRSOLVE_ECUDA;
    }
    int rc = CRSOLVE_OK;
    const R b = R(0.999999), c = R(1e-6);
    k_fma_probe<R><<<blocks, 256, 0, s>>>(iters / 8, b, c);   // warm-up (clocks up, code loaded)
    float ms = 0.f;
    const unsigned long long zero = 0;
    if (cudaMemcpyToSymbolAsync(g_probe_cycles, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaEventRecord(e0, s) != cudaSuccess)
        rc = CRSOLVE_ECUDA;
    if (rc == CRSOLVE_OK) k_fma_probe<R><<<blocks, 256, 0, s>>>(iters, b, c);
    if (rc == CRSOLVE_OK && (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
                             cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = CRSOLVE_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    unsigned long long cycles = 0;
    if (rc == CRSOLVE_OK && cudaMemcpyFromSymbol(&cycles, g_probe_cycles, sizeof(cycles)) != cudaSuccess)
        rc = CRSOLVE_ECUDA;
    if (rc == CRSOLVE_OK) {
        const double flops = 2.0 * 8.0 * (double)iters * (double)blocks * 256.0;
        *gflops = ms > 0.f ? flops / ((double)ms * 1e-3) / 1e9 : 0.0;
        // FMA lanes per SM per clock: the clock-independent rate
        if (per_clk) *per_clk = cycles > 0 ? 8.0 * (double)iters * per_sm * 256.0 / (double)cycles : 0.0;
        if (mhz) *mhz = ms > 0.f ? (double)cycles / ((double)ms * 1e-3) / 1e6 : 0.0;
    }
    return rc;
}

}  // namespace

extern "C" int crsolve_peak_probe(int32_t kind, double *gflops, double *fma_per_clk_sm, double *sm_mhz,
                                  void *stream) {
    if (!gflops || (kind != CRSOLVE_PROBE_FP64_FMA && kind != CRSOLVE_PROBE_FP32_FMA)) return CRSOLVE_EINVAL;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CRSOLVE_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // exactly one full wave: as many CTAs of 256 threads as are resident on
    // every SM at once (up to 8: 64 warps, 16 per scheduler)
    int per_sm = 0;
    const cudaError_t e = kind == CRSOLVE_PROBE_FP64_FMA
                              ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<double>, 256, 0)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<float>, 256, 0);
    if (e != cudaSuccess || per_sm < 1) return CRSOLVE_ECUDA;
    if (per_sm > 8) per_sm = 8;
    const int blocks = per_sm * nsm;
    return kind == CRSOLVE_PROBE_FP64_FMA
               ? run_probe<double>(1 << 15, blocks, per_sm, s, gflops, fma_per_clk_sm, sm_mhz)
               : run_probe<float>(1 << 20, blocks, per_sm, s, gflops, fma_per_clk_sm, sm_mhz);
}

// ------------------------------------------------------- bounded-wait check
//
// The tensor-core kernels wait on mbarriers with mbar_wait, which gives up
// after a poll count (or two seconds) and lets the kernel report
// CRSOLVE_ETIMEOUT instead of hanging.  This kernel exercises that path on
// its own: it initialises an mbarrier that nothing ever arrives at (no MMA,
// no tensor memory, no other CTA), waits on it with the given poll limit, and
// records whether the wait gave up.
namespace {

__global__ void k_wait_check(int max_polls, int *gave_up) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t a = crs::smem_u32(&bar);
    if (threadIdx.x == 0) crs::mbar_init(a, 1);
    __syncthreads();
    const bool ok = crs::mbar_wait(a, 0, max_polls);
    if (threadIdx.x == 0) *gave_up = ok ? 0 : 1;
}

}  // namespace

extern "C" int crsolve_check_bounded_wait(int32_t max_polls, void *workspace, void *stream) {
    if (max_polls < 1 || !workspace || ((uintptr_t)workspace & 3u)) return CRSOLVE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int *flag = static_cast<int *>(workspace);
    int host = -1;
    if (cudaMemsetAsync(flag, 0xFF, sizeof(int), s) != cudaSuccess) return CRSOLVE_ECUDA;
    k_wait_check<<<1, 32, 0, s>>>(max_polls, flag);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&host, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CRSOLVE_ECUDA;
    return host == 1 ? CRSOLVE_ETIMEOUT : (host == 0 ? CRSOLVE_OK : CRSOLVE_ECUDA);
}
