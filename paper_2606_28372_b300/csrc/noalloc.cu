// Repair without any device allocation.
//
// ct_repair sizes its scratch (pending-candidate lists and per-candidate
// argmin words) on demand with cudaMalloc and releases old scratch with
// cudaFree.  Some callers cannot allow that: host applications that reserve
// the device memory up front through their own pool allocator and forbid
// allocations from libraries, and latency-sensitive loops in which cudaFree's
// implicit device-wide synchronisation would stall work on other streams.
// ct_repair_noalloc gives them the same result with the scratch taken from a
// fixed array compiled into this library.
//
// The array below is a file-scope __device__ variable: every device that loads
// the library holds one copy (about 384 KB) until the process exits.  Host code
// cannot use the symbol itself as a device address, so the first call on each
// device looks the address up once with cudaGetSymbolAddress (with that device
// current) and caches it; make that first call before capturing any stream.
// All calls share the array and it keeps the previous call's contents, so the
// counters that must start at zero are cleared by every call, and calls whose
// execution overlaps on the GPU (different streams, or host threads without
// ordering) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.hpp"

namespace ct {

// kernels of the regular repair path (search.cu), launched here on the fixed scratch
__global__ void k_repair_init(const DevSpace* sp, const uint32_t* tables, const uint64_t* cand, int64_t n,
                              uint64_t* out, uint8_t* dist, int32_t* pend, uint32_t* count,
                              unsigned long long* best, uint32_t* status, uint64_t* fail);
__global__ void k_ball(const DevSpace* sp, const uint32_t* tables, const uint32_t* masks, const uint64_t* prefix,
                       int n_subsets, uint64_t points, const uint64_t* cand, const int32_t* pend,
                       const uint32_t* count, unsigned long long* best, const uint64_t* fail, const BallNext nx);
__global__ void k_ball_resolve(int d, const int32_t* pend_in, const uint32_t* count_in,
                               const unsigned long long* best_in, uint64_t* out, uint8_t* dist, int32_t* pend_out,
                               uint32_t* count_out, unsigned long long* best_out);
__global__ void k_scan(const uint64_t* keys, int64_t nv, uint64_t lowm, uint64_t highm, const uint64_t* cand,
                       const int32_t* pend, const uint32_t* count, unsigned long long* best);
__global__ void k_scan_resolve(const uint64_t* keys, const int32_t* pend, const uint32_t* count,
                               const unsigned long long* best, uint64_t* out, uint8_t* dist);

namespace {

constexpr int NA_SCAN_THREADS = 256;   // block size the scan kernel is compiled for
constexpr int NA_SCAN_CHUNK = 32;      // candidates per CTA of the scan kernel
constexpr int64_t NA_MAX = CT_REPAIR_NOALLOC_MAX;

// Layout: two pending lists, two argmin arrays, two counters.
struct NoallocScratch {
    int32_t pend[2][NA_MAX];
    unsigned long long best[2][NA_MAX];
    uint32_t count[2];
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
NoallocScratch* g_addr[MAX_DEVICES] = {};

ct_status scratch_address(NoallocScratch** out) {
    int dev = 0;
    CT_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) { set_error("device %d beyond the supported %d", dev, MAX_DEVICES); return CT_ERR_LIMIT; }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        CT_TRY_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_addr[dev] = static_cast<NoallocScratch*>(p);
    }
    *out = g_addr[dev];
    return CT_OK;
}

}  // namespace
}  // namespace ct

using namespace ct;

extern "C" ct_status ct_repair_noalloc(ct_space* s, const uint64_t* d_cand, int64_t n, uint64_t* d_out,
                                       uint8_t* d_dist, ct_stream stream) {
    if (!s || n < 0 || (n > 0 && (!d_cand || !d_out))) { set_error("bad argument"); return CT_ERR_INVALID_ARG; }
    if (n > NA_MAX) {
        set_error("ct_repair_noalloc takes at most %d candidates per call (got %lld); split the batch",
                  (int)NA_MAX, (long long)n);
        return CT_ERR_LIMIT;
    }
    if (!s->built) { set_error("space not built"); return CT_ERR_STATE; }
    if (s->n_valid == 0) { set_error("empty valid space"); return CT_ERR_EMPTY_SPACE; }
    if (n == 0) return CT_OK;
    NoallocScratch* sc = nullptr;
    CT_TRY(scratch_address(&sc));
    cudaStream_t st = (cudaStream_t)stream;
    int sms = 148, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int32_t* pend[2] = {sc->pend[0], sc->pend[1]};
    unsigned long long* best[2] = {sc->best[0], sc->best[1]};
    uint32_t* cnt[2] = {&sc->count[0], &sc->count[1]};
    const unsigned g1 = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
    const unsigned gw = (unsigned)std::min<int64_t>((n * 32 + 255) / 256, (int64_t)sms * 8);   // a warp per candidate
    CT_TRY_CUDA(cudaMemsetAsync(sc->count, 0, sizeof sc->count, st));   // the counters must start at zero
    k_repair_init<<<gw, 256, 0, st>>>(s->d, s->tables.p, d_cand, n, d_out, d_dist, pend[0], cnt[0], best[0],
                                      s->status.p, nullptr);   // no failing-constraint masks: full tests
    count_launch();
    // ball radii already enumerated (the build plans the ones the repair path uses); any
    // candidate left over goes to the exhaustive scan, so the result is exact either way
    const int dmax = std::min<int>(wanted_radius(s), (int)s->balls.size());
    int cur = 0;
    for (int d = 1; d <= dmax; ++d) {
        const BallRadius& br = s->balls[d - 1];
        const uint64_t work = (uint64_t)n * br.total;
        const unsigned gb = (unsigned)std::min<uint64_t>((work + 255) / 256, (uint64_t)sms * 16);
        k_ball<<<gb, 256, 0, st>>>(s->d, s->tables.p, br.d_masks.p, br.d_prefix.p, (int)br.masks.size(), br.total,
                                   d_cand, pend[cur], cnt[cur], best[cur], nullptr, BallNext{});   // resolved below
        CT_TRY_CUDA(cudaMemsetAsync(cnt[cur ^ 1], 0, sizeof(uint32_t), st));
        k_ball_resolve<<<g1, 256, 0, st>>>(d, pend[cur], cnt[cur], best[cur], d_out, d_dist, pend[cur ^ 1],
                                           cnt[cur ^ 1], best[cur ^ 1]);
        count_launch(2);
        cur ^= 1;
    }
    const unsigned chunks = (unsigned)((n + NA_SCAN_CHUNK - 1) / NA_SCAN_CHUNK);
    const unsigned gx = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>(((int64_t)s->n_valid + NA_SCAN_THREADS * 8 - 1) / (NA_SCAN_THREADS * 8), (int64_t)sms * 4));
    k_scan<<<dim3(gx, chunks), NA_SCAN_THREADS, 0, st>>>(s->keys.p, (int64_t)s->n_valid, s->h.swar_low,
                                                        s->h.swar_high, d_cand, pend[cur], cnt[cur], best[cur]);
    k_scan_resolve<<<g1, 256, 0, st>>>(s->keys.p, pend[cur], cnt[cur], best[cur], d_out, d_dist);
    count_launch(2);
    CT_TRY_CUDA(cudaGetLastError());
    return CT_OK;
}
