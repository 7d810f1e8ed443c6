// Integer throughput microbenchmark: the denominator of the integer roofline of the key scans.
//
// Every thread runs eight independent accumulator chains of 32-bit operations; one step of a
// chain is an exclusive or with a value that changes every iteration, a population count and
// two additions -- the operations of the key scans.  The population count issues at a quarter of
// the rate of the other integer operations, so this mix (like the scans, which spend one per
// (key, candidate) on keys of at most 32 bits and two on wider keys) is bound by that pipe; the
// rate reported is population counts per second, measured over every SM at full occupancy.
//
// A second microbenchmark gives the denominator of the surrogate's fixed-order fp32 products:
// eight independent fused multiply-add chains per thread, every SM at full occupancy, reported
// as floating-point operations (two per fused multiply-add) per second.
//
// A third gives the denominator of the distance-table scan, whose limit is shared-memory load
// bandwidth: every warp reads 16-byte entries from shared memory, 32 consecutive entries per
// load instruction (512 bytes, four 128-byte wavefronts, no bank conflict), four independent
// loads per step at addresses that change every step; reported as wavefronts per second.
#include <cuda_runtime.h>

#include "internal.hpp"

namespace ct {

constexpr int IP_THREADS = 256, IP_ITERS = 4096, IP_CHAINS = 8;
constexpr int IP_POPC_PER_STEP = 1;

__global__ void __launch_bounds__(IP_THREADS) k_int_peak(uint32_t seed, uint32_t* __restrict__ sink) {
    uint32_t a[IP_CHAINS];
    const uint32_t w = seed * 0x9e3779b9u + blockIdx.x * IP_THREADS + threadIdx.x;
#pragma unroll
    for (int c = 0; c < IP_CHAINS; ++c) a[c] = w * (2u * c + 1u);
    for (int i = 0; i < IP_ITERS; ++i) {
#pragma unroll
        for (int c = 0; c < IP_CHAINS; ++c) {
            const uint32_t x = a[c] ^ (uint32_t)i;
            a[c] = x + (uint32_t)__popc(x) + (uint32_t)c;
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int c = 0; c < IP_CHAINS; ++c) r ^= a[c];
    if (r == 0x9e3779b9u) sink[0] = r;   // keeps the chains live; practically never written
}

constexpr int FP_ITERS = 4096, FP_CHAINS = 8;

__global__ void __launch_bounds__(IP_THREADS) k_fp32_peak(float seed, float* __restrict__ sink) {
    float a[FP_CHAINS];
    const float x = seed + 1e-7f * (float)(blockIdx.x * IP_THREADS + threadIdx.x);
#pragma unroll
    for (int c = 0; c < FP_CHAINS; ++c) a[c] = x + (float)c;
    for (int i = 0; i < FP_ITERS; ++i) {
#pragma unroll
        for (int c = 0; c < FP_CHAINS; ++c) a[c] = __fmaf_rn(a[c], 0.999999f, 1e-6f);
    }
    float r = 0.0f;
#pragma unroll
    for (int c = 0; c < FP_CHAINS; ++c) r += a[c];
    if (r == 12345.678f) sink[0] = r;   // keeps the chains live; practically never written
}

constexpr int SM_ITERS = 2048, SM_LOADS = 4, SM_ENTRIES = 2048;   // 32 KB of 16-byte entries

__global__ void __launch_bounds__(IP_THREADS) k_smem_peak(uint32_t seed, uint32_t* __restrict__ sink) {
    __shared__ uint4 tab[SM_ENTRIES];
    for (int e = threadIdx.x; e < SM_ENTRIES; e += IP_THREADS)
        tab[e] = make_uint4(seed + e, seed ^ e, seed * e, e);
    __syncthreads();
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(tab);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t acc[SM_LOADS] = {0u, 0u, 0u, 0u};
    for (int i = 0; i < SM_ITERS; ++i) {
#pragma unroll
        for (int k = 0; k < SM_LOADS; ++k) {
            // a row of 32 consecutive entries, a different row for every (step, load, warp)
            const int row = (i * 5 + k * 17 + warp * 3) & (SM_ENTRIES / 32 - 1);
            uint32_t x, y, z, w;
            asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(x), "=r"(y), "=r"(z), "=r"(w)
                         : "r"(base + (uint32_t)(row * 32 + lane) * 16u));
            acc[k] ^= x ^ y ^ z ^ w;
        }
    }
    const uint32_t r = acc[0] ^ acc[1] ^ acc[2] ^ acc[3];
    if (r == 0x9e3779b9u) sink[0] = r;   // keeps the loads live; practically never written
}

// Times one launch of `k` over every SM (grid: 8 resident CTAs of 256 per SM, four waves) after
// a warm-up launch; milliseconds into *ms.
template <class Launch>
static ct_status time_peak(Launch launch, cudaStream_t st, float* ms) {
    cudaEvent_t e0, e1;
    CT_TRY_CUDA(cudaEventCreate(&e0));
    CT_TRY_CUDA(cudaEventCreate(&e1));
    launch(1);   // warm-up
    cudaEventRecord(e0, st);
    launch(2);
    cudaEventRecord(e1, st);
    count_launch(2);
    cudaError_t err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) { set_error("%s", cudaGetErrorString(err)); return CT_ERR_CUDA; }
    return CT_OK;
}

}  // namespace ct

using namespace ct;

extern "C" ct_status ct_measure_fp32_peak(double* flop_per_s, ct_stream stream) {
    if (!flop_per_s) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    int dev = 0, sms = 148;
    CT_TRY_CUDA(cudaGetDevice(&dev));
    CT_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DevBuf<float> sink;
    CT_TRY(sink.ensure(1));
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned grid = (unsigned)sms * 8 * 4;
    float ms = 0.0f;
    const ct_status r = time_peak([&](int w) { k_fp32_peak<<<grid, IP_THREADS, 0, st>>>((float)w, sink.p); }, st, &ms);
    sink.release();
    CT_TRY(r);
    const double flop = 2.0 * (double)grid * IP_THREADS * FP_ITERS * FP_CHAINS;
    *flop_per_s = flop / (ms * 1e-3);
    return CT_OK;
}

extern "C" ct_status ct_measure_int_peak(double* popc_per_s, ct_stream stream) {
    if (!popc_per_s) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    int dev = 0, sms = 148;
    CT_TRY_CUDA(cudaGetDevice(&dev));
    CT_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DevBuf<uint32_t> sink;
    CT_TRY(sink.ensure(1));
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned grid = (unsigned)sms * 8 * 4;   // 8 resident CTAs of 256 per SM, four waves
    cudaEvent_t e0, e1;
    CT_TRY_CUDA(cudaEventCreate(&e0));
    CT_TRY_CUDA(cudaEventCreate(&e1));
    k_int_peak<<<grid, IP_THREADS, 0, st>>>(1u, sink.p);   // warm-up
    cudaEventRecord(e0, st);
    k_int_peak<<<grid, IP_THREADS, 0, st>>>(2u, sink.p);
    cudaEventRecord(e1, st);
    count_launch(2);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    sink.release();
    if (err != cudaSuccess) { set_error("%s", cudaGetErrorString(err)); return CT_ERR_CUDA; }
    const double popc = (double)grid * IP_THREADS * IP_ITERS * IP_CHAINS * IP_POPC_PER_STEP;
    *popc_per_s = popc / (ms * 1e-3);
    return CT_OK;
}

extern "C" ct_status ct_measure_smem_peak(double* wavefronts_per_s, ct_stream stream) {
    if (!wavefronts_per_s) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    int dev = 0, sms = 148;
    CT_TRY_CUDA(cudaGetDevice(&dev));
    CT_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DevBuf<uint32_t> sink;
    CT_TRY(sink.ensure(1));
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned grid = (unsigned)sms * 6 * 4;   // 6 resident CTAs of 256 (32 KB each) per SM, four waves
    float ms = 0.0f;
    const ct_status r = time_peak([&](int w) { k_smem_peak<<<grid, IP_THREADS, 0, st>>>((uint32_t)w, sink.p); }, st, &ms);
    sink.release();
    CT_TRY(r);
    const double wavefronts = 4.0 * (double)grid * (IP_THREADS / 32) * SM_ITERS * SM_LOADS;
    *wavefronts_per_s = wavefronts / (ms * 1e-3);
    return CT_OK;
}
