// peak.cu -- lq_fp64_fma_rate: the FP64 fused multiply-add rate of the
// current device, measured.  The FP64 form of the step (section III.B's
// force and Algorithm 1's update in double precision) is bound by the FP64
// pipe on this GPU rather than by memory; its roofline needs the pipe's
// measured rate, not a figure derived from a data sheet.
//
// Every thread runs CHAINS independent dependent chains x <- x * a + b of
// `iters` fused multiply-adds each (a slightly below 1, b small, so the values
// stay normal and finite); CHAINS per thread hide the pipe latency.  Each
// thread writes the sum of its chains, so that nothing can be dropped.
#include <cuda_runtime.h>

#include <cstdint>

#include "lqmin.h"
#include "lq_kernels.h"

namespace lq {
namespace {

constexpr int CHAINS = 8;
constexpr int FMA_THREADS = 256;

__global__ void __launch_bounds__(FMA_THREADS) k_fp64_fma(long long iters, double a, double b, double *out) {
    double x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = __fma_rn(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    out[blockIdx.x * FMA_THREADS + threadIdx.x] = s;
}

}  // namespace
}  // namespace lq

extern "C" lq_status lq_fp64_fma_rate(int64_t iters, double *fma_per_s) {
    using namespace lq;
    if (!fma_per_s || iters <= 0) return LQ_EINVAL;
    int dev = 0, nsm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LQ_ECUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LQ_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_fma, FMA_THREADS, 0) != cudaSuccess)
        return LQ_ECUDA;
    const int blocks = nsm * (per_sm > 0 ? per_sm : 1);
    double *out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    lq_status ret = LQ_OK;
    if (cudaMalloc(&out, sizeof(double) * blocks * FMA_THREADS) != cudaSuccess) return LQ_ENOMEM;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        ret = LQ_ECUDA;
    } else {
        const double a = 0.999999, b = 1e-6;
        k_fp64_fma<<<blocks, FMA_THREADS, 0, s>>>(iters / 8 + 1, a, b, out);   // warm-up
        cudaEventRecord(e0, s);
        k_fp64_fma<<<blocks, FMA_THREADS, 0, s>>>(iters, a, b, out);
        cudaEventRecord(e1, s);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            ms <= 0.f) {
            ret = LQ_ECUDA;
        } else {
            const double fmas = (double)blocks * FMA_THREADS * CHAINS * (double)iters;
            *fma_per_s = fmas / (ms * 1e-3);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(out);
    return ret;
}
