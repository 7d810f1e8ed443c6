// Repair without any device allocation.
//
// ct_repair sizes its scratch (pending-candidate lists, per-candidate argmin
// words and failing-constraint words) on demand from the library's block cache,
// which calls cudaMalloc when the cache has no block of the right size, and it
// may upload Hamming-ball tables the first time a radius is used.  Some callers
// cannot allow that: host applications that reserve the device memory up front
// through their own pool allocator and forbid allocations from libraries, and
// latency-sensitive loops in which an allocation or cudaFree's implicit
// device-wide synchronisation would stall work on other streams.
// ct_repair_noalloc gives them the same result, by the same kernels, with the
// scratch taken from a fixed array compiled into this library.
//
// The array below is a file-scope __device__ variable: every device that loads
// the library holds one copy (about 512 KB) until the process exits.  Host code
// cannot use the symbol itself as a device address, so the first call on each
// device looks the address up once with cudaGetSymbolAddress (with that device
// current) and caches it; make that first call before capturing any stream.  A
// cudaDeviceReset invalidates that address together with every other handle and
// buffer of this library.  All calls share the array and it keeps the previous
// call's contents, so the counters that must start at zero are cleared by every
// call, and calls whose execution overlaps on the GPU (different streams, or
// host threads without ordering) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.hpp"

namespace ct {
namespace {

constexpr int64_t NA_MAX = CT_REPAIR_NOALLOC_MAX;

// Layout: two pending lists and two argmin arrays (ping-pong between ball radii), the failing
// constraints of each candidate, the two list counters and the ball kernels' CTA ticket.
struct NoallocScratch {
    int32_t pend[2][NA_MAX];
    unsigned long long best[2][NA_MAX];
    uint64_t fail[NA_MAX];
    uint32_t count[2];
    uint32_t done;
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
NoallocScratch* g_addr[MAX_DEVICES] = {};

ct_status scratch_address(int dev, NoallocScratch** out) {
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
    int dev = 0;
    CT_TRY_CUDA(cudaGetDevice(&dev));
    NoallocScratch* sc = nullptr;
    CT_TRY(scratch_address(dev, &sc));
    cudaStream_t st = (cudaStream_t)stream;
    // the two counters and the ticket must start at zero (they are adjacent)
    CT_TRY_CUDA(cudaMemsetAsync(sc->count, 0, sizeof sc->count + sizeof sc->done, st));
    // only ball radii whose tables are already on the device (the build uploads the ones the
    // repair path uses); anything left over goes to the exhaustive scan, so the result is exact
    const int want = wanted_radius(s);
    int dmax = 0;
    while (dmax < want && dmax < (int)s->balls.size() && s->balls[dmax].d_masks.p && s->balls[dmax].d_prefix.p) ++dmax;
    const RepairPtrs p{{sc->pend[0], sc->pend[1]}, {&sc->count[0], &sc->count[1]}, {sc->best[0], sc->best[1]},
                       sc->fail, &sc->done};
    return repair_launch(s, p, dmax, d_cand, n, d_out, d_dist, st);
}
