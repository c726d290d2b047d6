// smcrt_microbench.cu -- measured ceilings for the packet kernel's roofline:
// FP32 FMA issue rate and int64 L2 atomic (RED) rates on this GPU.
#include <cmath>

#include "smcrt_internal.h"

namespace smcrt {

namespace {

constexpr int kFmaChains = 8;     // independent FMA chains per thread: hides the FMA latency
constexpr int kFmaIters = 16384;  // iterations per thread (8 FMAs each)
constexpr int kRedIters = 256;    // atomics per thread
constexpr unsigned kDistinctMask = (1u << 23) - 1u;   // 2^23 int64 = 64 MiB of distinct targets

__global__ void __launch_bounds__(256) fma_kernel(float *sink, float b, float c)
{
    float a[kFmaChains];
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) a[k] = (float)(threadIdx.x + k);
    for (int i = 0; i < kFmaIters; ++i) {
#pragma unroll
        for (int k = 0; k < kFmaChains; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) s += a[k];
    if (s == 12345.678f) sink[threadIdx.x] = s;   // keeps the chains live; never true for b < 1
}

__global__ void __launch_bounds__(256) red_kernel(unsigned long long *buf, unsigned mask, int hot)
{
    const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned h = tid * 2654435761u + 12345u;
    for (int i = 0; i < kRedIters; ++i) {
        h ^= h << 13; h ^= h >> 17; h ^= h << 5;   // xorshift32: scattered targets
        const unsigned idx = hot ? ((tid + (unsigned)i) & 31u) : (h & mask);
        atomicAdd(buf + idx, 1ull);
    }
}

double time_ms(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return (double)ms;
}

}  // namespace

}  // namespace smcrt

extern "C" int smcrt_microbench(int device, void *scratch_dev, size_t scratch_bytes, double *fp32_flops,
                                double *atomics_distinct, double *atomics_hot)
{
    using namespace smcrt;
    if (!scratch_dev || !fp32_flops || !atomics_distinct || !atomics_hot) return SMCRT_ERR_BAD_ARG;
    if (scratch_bytes < sizeof(unsigned long long) * ((size_t)kDistinctMask + 1)) return SMCRT_ERR_BAD_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return SMCRT_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return SMCRT_ERR_CUDA;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fma_kernel, 256, 0);
    const int blocks = sms * (occ > 0 ? occ : 1);
    unsigned long long *buf = (unsigned long long *)scratch_dev;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return SMCRT_ERR_CUDA;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = SMCRT_OK;
    // FP32: warm-up, then the best of three
    double best = 1e30;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, s);
        fma_kernel<<<blocks, 256, 0, s>>>((float *)scratch_dev, 0.999f, 1e-3f);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = SMCRT_ERR_CUDA; break; }
        if (rep > 0) best = fmin(best, time_ms(e0, e1));
    }
    if (rc == SMCRT_OK)
        *fp32_flops = (double)blocks * 256 * kFmaIters * kFmaChains * 2.0 / (best * 1e-3);
    // int64 RED to distinct and to 32 hot addresses
    int rocc = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rocc, red_kernel, 256, 0);
    const int rblocks = sms * (rocc > 0 ? rocc : 1);
    for (int hot = 0; hot < 2 && rc == SMCRT_OK; ++hot) {
        double bt = 1e30;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, s);
            red_kernel<<<rblocks, 256, 0, s>>>(buf, kDistinctMask, hot);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = SMCRT_ERR_CUDA; break; }
            if (rep > 0) bt = fmin(bt, time_ms(e0, e1));
        }
        const double rate = (double)rblocks * 256 * kRedIters / (bt * 1e-3);
        if (hot) *atomics_hot = rate; else *atomics_distinct = rate;
    }
    if (cudaGetLastError() != cudaSuccess) rc = SMCRT_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    return rc;
}
