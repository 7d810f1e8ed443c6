// Search-space definition and full resolution of the valid space (Section IV-A).
//
// Lowering (host): field layout of the packed keys, the scope and deepest
// parameter of every constraint, and a plan of enumeration blocks: consecutive
// parameters [s, e) whose Cartesian product has at most 4096 points.  Every
// constraint is attached to the block holding its deepest parameter; if its
// truth table over (its parameters before the block) x (the block's points) is
// small it becomes a bit-mask table, built on the GPU by interpreting the
// constraint over that sub-domain.
//
// Build (device): a prefix of the first blocks is expanded into the next one.
// For each parent prefix and each 32-point word of the next block the valid
// points are the AND of the constraint masks selected by the parent's fields;
// pass one counts per tile, a scan gives tile offsets, pass two recomputes the
// masks and writes the children, in increasing key order, through shared
// memory with coalesced stores.  The last block writes the final sorted keys.
// Work is proportional to the valid prefixes of every level, not to the
// Cartesian size; nothing spins on another block.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <map>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.hpp"

namespace ct {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}
const char* last_error() { return g_err.c_str(); }

static std::atomic<uint64_t> g_launches{0};
static std::atomic<uint64_t> g_allocs{0};

// ---- device block cache ----
namespace {
struct BlockCache {
    std::mutex mu;
    std::multimap<size_t, void*> free_blocks[64];   // per device: bytes -> block
    size_t held[64] = {};
};
BlockCache& cache() {
    static BlockCache* c = new BlockCache();   // lives until exit
    return *c;
}
constexpr size_t CACHE_MAX_BYTES = 64ull << 30;
int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d >= 0 && d < 64 ? d : 0;
}
void flush_device(BlockCache& c, int d) {
    for (auto& kv : c.free_blocks[d]) cudaFree(kv.second);
    c.free_blocks[d].clear();
    c.held[d] = 0;
}
}  // namespace

void* dev_alloc(size_t bytes, cudaError_t* err) {
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    BlockCache& c = cache();
    const int d = current_device();
    {
        std::lock_guard<std::mutex> lk(c.mu);
        auto it = c.free_blocks[d].lower_bound(bytes);
        if (it != c.free_blocks[d].end() && it->first <= 2 * bytes) {
            void* p = it->second;
            c.held[d] -= it->first;
            c.free_blocks[d].erase(it);
            return p;
        }
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        std::lock_guard<std::mutex> lk(c.mu);
        flush_device(c, d);
        e = cudaMalloc(&p, bytes);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (err) *err = e;
        return nullptr;
    }
    return p;
}

void dev_free(void* p, size_t bytes) {
    if (!p) return;
    BlockCache& c = cache();
    const int d = current_device();
    std::lock_guard<std::mutex> lk(c.mu);
    if (c.held[d] + bytes > CACHE_MAX_BYTES) { cudaFree(p); return; }
    c.free_blocks[d].emplace(bytes, p);
    c.held[d] += bytes;
}
void count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

constexpr int EXP_THREADS = 256;
constexpr int EXP_ROUNDS = 8;
constexpr int EXP_TILE = EXP_THREADS * EXP_ROUNDS;   // items (parent, word) per tile
constexpr uint64_t TABLE_WORDS_PER_CONS = 1ull << 22;   // 16 MB
constexpr uint64_t TABLE_WORDS_TOTAL = 1ull << 24;      // 64 MB

// ---------------------------------------------------------------------------
// table construction: one thread per (tabled constraint, row, point)
// ---------------------------------------------------------------------------
// value indices of keys, one (key, parameter) per thread
__global__ void k_unpack(const DevSpace* __restrict__ sp, const uint64_t* __restrict__ keys, int64_t n,
                         int32_t* __restrict__ idx) {
    const int np = sp->n;
    const int64_t total = n * np;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = g / np;
        const int k = (int)(g - i * np);
        idx[g] = field(sp, __ldg(keys + i), k);
    }
}

// Compact truth tables: bit (row, c) = the constraint at the outer values of `row` and the
// in-block scope values of combination c (one interpreted evaluation per combination).
__global__ void k_build_compact(const DevSpace* __restrict__ sp, const int32_t* __restrict__ cz_cons,
                                const uint64_t* __restrict__ cz_prefix, int n_cz, uint64_t total_words,
                                uint32_t* __restrict__ compact) {
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t gw = gid >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= total_words) return;   // whole warps share gw
    int lo = 0, hi = n_cz - 1;       // last i with cz_prefix[i] <= gw
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (cz_prefix[mid] <= gw) lo = mid; else hi = mid - 1;
    }
    const DevCons& cs = sp->cons[cz_cons[lo]];
    const uint64_t lw = gw - cz_prefix[lo];
    const uint32_t row = (uint32_t)(lw / cs.cz_W), wd = (uint32_t)(lw % cs.cz_W);
    const uint32_t c = wd * 32 + lane;
    bool bit = false;
    if (c < cs.cz_B) {
        int64_t pv[MAXP];            // only the scope's parameters are set: the program reads no other
        uint32_t o = row;
        for (int q = cs.n_outer - 1; q >= 0; --q) {
            const int k = cs.outer_k[q];
            const int32_t ik = (int32_t)(o % sp->r[k]);
            o /= sp->r[k];
            pv[k] = sp->values[sp->vstart[k] + ik];
        }
        uint32_t t = c;
        for (int q = 0; q < cs.n_in; ++q) {   // in_k runs from the last parameter backwards
            const int k = cs.in_k[q];
            const int32_t ik = (int32_t)(t % sp->r[k]);
            t /= sp->r[k];
            pv[k] = sp->values[sp->vstart[k] + ik];
        }
        bit = vm_eval(sp->prog, cs.pc, cs.len, pv);
    }
    const uint32_t word = __ballot_sync(0xffffffffu, bit);
    if (lane == 0) compact[gw] = word;
}

// Block truth tables: each CTA builds TB_WORDS_PER_CTA consecutive words of one tabled
// constraint's table (the constraints' words are split into such runs in order), a warp per
// 32-point word.  The CTA's thread 0 finds its constraint and run, and the constraint's and
// block's descriptors are copied to shared memory once.  A point's digits come from the block's
// point -> key-bits table (one coalesced load per word) instead of divisions.
constexpr int TB_WORDS_PER_CTA = 32;   // 8 warps x 4 words
__global__ void __launch_bounds__(256)
k_build_tables(const DevSpace* __restrict__ sp, const int32_t* __restrict__ tab_cons, int n_tab,
               const uint64_t* __restrict__ tab_prefix, const uint32_t* __restrict__ compact,
               const uint32_t* __restrict__ innerkey, uint32_t* __restrict__ tables) {
    __shared__ DevCons cs;
    __shared__ DevBlock bl;
    __shared__ int32_t rk[MAXP], offk[MAXP];
    __shared__ uint64_t run0_s, nw_s;
    __shared__ int ti_s;
    if (threadIdx.x < 32) {   // the constraint whose runs hold CTA blockIdx.x: warp 0, 32 constraints at a time
        const int lane = threadIdx.x;
        uint64_t first = 0;
        int found = -1;
        for (int c0 = 0; c0 < n_tab && found < 0; c0 += 32) {
            const int ti = c0 + lane;
            const uint64_t runs = ti < n_tab ? (tab_prefix[ti + 1] - tab_prefix[ti] + TB_WORDS_PER_CTA - 1) / TB_WORDS_PER_CTA : 0;
            uint64_t inc = runs;   // inclusive prefix of the runs over the lanes
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            const unsigned hit = __ballot_sync(0xffffffffu, ti < n_tab && blockIdx.x < first + inc);
            if (hit) {
                const int l = __ffs(hit) - 1;
                found = c0 + l;
                const uint64_t before = first + __shfl_sync(0xffffffffu, inc - runs, l);
                if (lane == 0) {
                    ti_s = found;
                    run0_s = (uint64_t)(blockIdx.x - before) * TB_WORDS_PER_CTA;
                    nw_s = tab_prefix[found + 1] - tab_prefix[found];
                }
            } else {
                first += __shfl_sync(0xffffffffu, inc, 31);
            }
        }
        if (found < 0 && lane == 0) ti_s = n_tab;
    }
    __syncthreads();
    const int ti = ti_s;
    if (ti >= n_tab) return;
    {
        const DevCons& gc = sp->cons[tab_cons[ti]];
        const int32_t* src = reinterpret_cast<const int32_t*>(&gc);
        int32_t* dst = reinterpret_cast<int32_t*>(&cs);
        for (int e = threadIdx.x; e < (int)(sizeof(DevCons) / 4); e += blockDim.x) dst[e] = src[e];
        const int32_t* srcb = reinterpret_cast<const int32_t*>(&sp->blocks[gc.block]);
        int32_t* dstb = reinterpret_cast<int32_t*>(&bl);
        for (int e = threadIdx.x; e < (int)(sizeof(DevBlock) / 4); e += blockDim.x) dstb[e] = srcb[e];
        for (int e = threadIdx.x; e < MAXP; e += blockDim.x) {
            rk[e] = e < sp->n ? sp->r[e] : 1;
            offk[e] = e < sp->n ? sp->off[e] : 0;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t nw = nw_s, run0 = run0_s;
    const uint32_t* ik = innerkey + bl.innerkey_off;
    for (uint64_t lw = run0 + warp; lw < nw && lw < run0 + TB_WORDS_PER_CTA; lw += 8) {
        const uint32_t row = (uint32_t)(lw / bl.W), wd = (uint32_t)(lw % bl.W);
        const int p = wd * 32 + lane;
        bool bit = false;
        if (p < bl.B && cs.cz_off != CZ_NONE) {   // gather from the compact table
            const uint64_t bits = (uint64_t)__ldg(ik + p) << bl.key_shift;   // the point's fields in place
            uint32_t c = 0;
            for (int q = 0; q < cs.n_in; ++q) {
                const int k = cs.in_k[q];
                c += (uint32_t)((bits & sp->fmask[k]) >> offk[k]) * (uint32_t)cs.in_stride[q];
            }
            bit = (__ldg(compact + cs.cz_off + (uint64_t)row * cs.cz_W + (c >> 5)) >> (c & 31)) & 1u;
        } else if (p < bl.B) {
            int64_t pv[MAXP];
            for (int k = 0; k < sp->n; ++k) pv[k] = 0;
            uint32_t o = row;
            for (int q = cs.n_outer - 1; q >= 0; --q) {
                const int k = cs.outer_k[q];
                const int32_t ikk = (int32_t)(o % rk[k]);
                o /= rk[k];
                pv[k] = sp->values[sp->vstart[k] + ikk];
            }
            int t = p;
            for (int k = bl.e - 1; k >= bl.s; --k) {
                const int32_t ikk = t % rk[k];
                t /= rk[k];
                pv[k] = sp->values[sp->vstart[k] + ikk];
            }
            bit = vm_eval(sp->prog, cs.pc, cs.len, pv);
        }
        const uint32_t word = __ballot_sync(0xffffffffu, bit);
        if (lane == 0) tables[cs.table_off + lw] = word;
    }
}

// ---------------------------------------------------------------------------
// expand: valid children of (parent, word)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t block_word(const DevSpace* __restrict__ sp, const uint32_t* __restrict__ tables,
                                               const DevBlock& bl, const uint32_t* __restrict__ ik,
                                               uint64_t parent, uint32_t wd) {
    uint32_t m = 0xffffffffu;
    const int rem = bl.B - (int)wd * 32;
    if (rem < 32) m = (1u << rem) - 1u;
    for (int c = bl.cons_begin; c < bl.cons_end && m; ++c) {
        const DevCons& cs = sp->cons[c];
        if (!cs.tabled) continue;
        uint32_t o = 0;
        for (int q = 0; q < cs.n_outer; ++q) o += (uint32_t)field(sp, parent, cs.outer_k[q]) * cs.outer_stride[q];
        m &= __ldg(tables + cs.table_off + (uint64_t)o * bl.W + wd);
    }
    if (m && bl.has_vm) {   // interpreted constraints, one point at a time
        uint32_t keep = m;
        for (uint32_t mm = m; mm; mm &= mm - 1) {
            const int b = __ffs(mm) - 1;
            const uint64_t key = parent | ((uint64_t)ik[wd * 32 + b] << bl.key_shift);
            int64_t pv[MAXP];
            for (int k = 0; k < bl.e; ++k) pv[k] = sp->values[sp->vstart[k] + field(sp, key, k)];
            for (int c = bl.cons_begin; c < bl.cons_end; ++c) {
                const DevCons& cs = sp->cons[c];
                if (!cs.tabled && !vm_eval(sp->prog, cs.pc, cs.len, pv)) { keep &= ~(1u << b); break; }
            }
        }
        m = keep;
    }
    return m;
}

__global__ void __launch_bounds__(EXP_THREADS)
k_expand_count(const DevSpace* __restrict__ sp, const uint32_t* __restrict__ tables,
               const uint32_t* __restrict__ innerkey, int j, const uint64_t* __restrict__ parents,
               uint64_t n_items, const unsigned long long* __restrict__ Fd, uint32_t* __restrict__ tile_counts) {
    const DevBlock& bl = sp->blocks[j];
    if (Fd) n_items = *Fd * (uint64_t)bl.W;   // launched for an upper bound: the level's own size
    const uint32_t* ik = innerkey + bl.innerkey_off;
    const uint64_t t0 = (uint64_t)blockIdx.x * EXP_TILE;
    uint32_t cnt = 0;
    for (int r = 0; r < EXP_ROUNDS; ++r) {
        const uint64_t it = t0 + (uint64_t)r * EXP_THREADS + threadIdx.x;
        if (it >= n_items) break;
        const uint64_t pi = it / (uint32_t)bl.W;
        const uint32_t wd = (uint32_t)(it - pi * (uint32_t)bl.W);
        const uint64_t parent = parents ? __ldg(parents + pi) : 0ull;
        cnt += __popc(block_word(sp, tables, bl, ik, parent, wd));
    }
    __shared__ uint32_t ws[EXP_THREADS / 32];
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int w = 0; w < EXP_THREADS / 32; ++w) s += ws[w];
        tile_counts[blockIdx.x] = s;
    }
}

// Exclusive scan of n tile counts into bases, and their sum into *total (one CTA of 1024
// threads).  Chunks of 8K counts are staged in shared memory with coalesced loads; each thread
// sums 8 contiguous counts, the thread sums are scanned with warp shuffles, and the bases go
// back through shared memory with coalesced stores; the running total carries between chunks.
constexpr int SCAN_T = 1024, SCAN_PER = 8, SCAN_CH = SCAN_T * SCAN_PER;
__global__ void __launch_bounds__(SCAN_T)
k_scan_tiles(const uint32_t* __restrict__ counts, uint64_t n, unsigned long long* __restrict__ base,
             unsigned long long* __restrict__ total) {
    __shared__ __align__(16) uint32_t cs[SCAN_CH + SCAN_CH / 32];   // padded: a thread's 8 counts in distinct banks
    __shared__ unsigned long long wsum[SCAN_T / 32];
    __shared__ unsigned long long carry_s;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    auto at = [](int i) { return i + (i >> 5); };
    unsigned long long carry = 0;
    for (uint64_t c0 = 0; c0 < n; c0 += SCAN_CH) {
        const int m = (int)min((uint64_t)SCAN_CH, n - c0);
        for (int i = t; i < SCAN_CH; i += SCAN_T) cs[at(i)] = i < m ? __ldg(counts + c0 + i) : 0u;
        __syncthreads();
        uint32_t v[SCAN_PER];
        unsigned long long sum = 0;
#pragma unroll
        for (int q = 0; q < SCAN_PER; ++q) { v[q] = cs[at(t * SCAN_PER + q)]; sum += v[q]; }
        unsigned long long inc = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = wsum[lane], wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long u = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += u;
            }
            wsum[lane] = wi - w;   // exclusive warp bases
            if (lane == 31) carry_s = wi;
        }
        __syncthreads();
        unsigned long long run = carry + wsum[warp] + inc - sum;
        // bases back into shared memory (as 64-bit, in two halves of the chunk), then out coalesced
        unsigned long long* bs = reinterpret_cast<unsigned long long*>(cs);
        __syncthreads();
        for (int h = 0; h < 2; ++h) {
            const int lo = h * (SCAN_CH / 2);
            if (t * SCAN_PER >= lo && t * SCAN_PER < lo + SCAN_CH / 2) {
#pragma unroll
                for (int q = 0; q < SCAN_PER; ++q) { bs[t * SCAN_PER + q - lo] = run; run += v[q]; }
            }
            __syncthreads();
            for (int i = t; i < SCAN_CH / 2; i += SCAN_T)
                if (lo + i < m) base[c0 + lo + i] = bs[i];
            __syncthreads();
        }
        carry += carry_s;
    }
    if (t == 0) *total = carry;
}

__global__ void __launch_bounds__(EXP_THREADS)
k_expand_emit(const DevSpace* __restrict__ sp, const uint32_t* __restrict__ tables,
              const uint32_t* __restrict__ innerkey, int j, const uint64_t* __restrict__ parents,
              uint64_t n_items, const unsigned long long* __restrict__ Fd,
              const unsigned long long* __restrict__ tile_base, const unsigned long long* __restrict__ total,
              unsigned long long expect, uint64_t* __restrict__ out) {
    extern __shared__ uint64_t stage[];                // EXP_THREADS * 32 keys
    __shared__ uint32_t wsum[EXP_THREADS / 32];
    if (expect != ~0ull && *total != expect) return;   // launched for another level size: write nothing
    const DevBlock& bl = sp->blocks[j];
    if (Fd) n_items = *Fd * (uint64_t)bl.W;             // launched for an upper bound: the level's own size
    const uint32_t* ik = innerkey + bl.innerkey_off;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t base = tile_base[blockIdx.x];
    const uint64_t t0 = (uint64_t)blockIdx.x * EXP_TILE;
    for (int r = 0; r < EXP_ROUNDS; ++r) {
        const uint64_t r0 = t0 + (uint64_t)r * EXP_THREADS;
        if (r0 >= n_items) break;                      // uniform across the CTA
        const uint64_t it = r0 + threadIdx.x;
        uint32_t m = 0;
        uint64_t parent = 0;
        uint32_t wd = 0;
        if (it < n_items) {
            const uint64_t pi = it / (uint32_t)bl.W;
            wd = (uint32_t)(it - pi * (uint32_t)bl.W);
            parent = parents ? __ldg(parents + pi) : 0ull;
            m = block_word(sp, tables, bl, ik, parent, wd);
        }
        // CTA exclusive scan of the popcounts
        const uint32_t c = __popc(m);
        uint32_t inc = c;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        uint32_t wbase = 0, tot = 0;
        for (int w = 0; w < EXP_THREADS / 32; ++w) {
            const uint32_t v = wsum[w];
            wbase += (w < warp) ? v : 0u;
            tot += v;
        }
        uint32_t pos = wbase + inc - c;
        for (uint32_t mm = m; mm; mm &= mm - 1) {
            const int b = __ffs(mm) - 1;
            stage[pos++] = parent | ((uint64_t)__ldg(ik + wd * 32 + b) << bl.key_shift);
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < tot; i += EXP_THREADS) out[base + i] = stage[i];
        base += tot;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// pattern mode: per-signature compacted inner-key lists, then broadcast-OR emission
// ---------------------------------------------------------------------------
constexpr int PAT_THREADS = 128;   // >= max words per block (4096 / 32)
constexpr int PE_THREADS = 256;    // threads of the pattern count/emit kernels (and most parents per tile)

// The pattern blocks of one launch: CTA b builds signature b - first[i] of block blk[i], for the
// last i with first[i] <= b.
struct PatBlocks {
    int32_t n;
    int32_t blk[MAXP];
    uint32_t first[MAXP];
};

__global__ void __launch_bounds__(PAT_THREADS)
k_build_patterns(const DevSpace* __restrict__ sp, const uint32_t* __restrict__ tables,
                 const uint32_t* __restrict__ innerkey, const __grid_constant__ PatBlocks pb,
                 uint32_t* __restrict__ pat_cnt, uint32_t* __restrict__ pat_list) {
    int i = 0;
    while (i + 1 < pb.n && pb.first[i + 1] <= blockIdx.x) ++i;
    const DevBlock& bl = sp->blocks[pb.blk[i]];
    const uint32_t sig = blockIdx.x - pb.first[i];
    __shared__ int32_t fidx[MAXP];
    __shared__ uint32_t wsum[PAT_THREADS / 32];
    if (threadIdx.x == 0) {
        uint32_t t = sig;
        for (int q = bl.n_u - 1; q >= 0; --q) {
            const int k = bl.u_k[q];
            fidx[k] = (int32_t)(t % (uint32_t)sp->r[k]);
            t /= (uint32_t)sp->r[k];
        }
    }
    __syncthreads();
    const uint32_t* ik = innerkey + bl.innerkey_off;
    const int t = threadIdx.x;
    uint32_t m = 0;
    if (t < bl.W) {
        m = 0xffffffffu;
        const int rem = bl.B - t * 32;
        if (rem < 32) m = (1u << rem) - 1u;
        for (int c = bl.cons_begin; c < bl.cons_end; ++c) {
            const DevCons& cs = sp->cons[c];
            uint32_t o = 0;
            for (int q = 0; q < cs.n_outer; ++q) o += (uint32_t)fidx[cs.outer_k[q]] * cs.outer_stride[q];
            m &= tables[cs.table_off + (uint64_t)o * bl.W + t];
        }
    }
    const int lane = t & 31, warp = t >> 5;
    const uint32_t c = __popc(m);
    uint32_t inc = c;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t base = 0, tot = 0;
    for (int w = 0; w < PAT_THREADS / 32; ++w) { base += (w < warp) ? wsum[w] : 0u; tot += wsum[w]; }
    uint32_t pos = base + inc - c;
    uint32_t* list = pat_list + bl.pat_list_off + (uint64_t)sig * bl.Bpad;
    for (uint32_t mm = m; mm; mm &= mm - 1) list[pos++] = ik[t * 32 + __ffs(mm) - 1];
    if (t == 0) pat_cnt[bl.pat_cnt_off + sig] = tot;
}

struct PatArgs {
    int32_t n_u;
    int32_t key_shift;
    uint32_t Bpad;
    int32_t pad_;
    uint64_t u_mask[MAXP];
    int32_t u_off[MAXP];
    int32_t u_stride[MAXP];
    const uint32_t* cnt;
    const uint32_t* list;
};

__device__ __forceinline__ uint32_t sig_of(const PatArgs& pa, uint64_t parent) {
    uint32_t sg = 0;
    for (int q = 0; q < pa.n_u; ++q) sg += (uint32_t)((parent & pa.u_mask[q]) >> pa.u_off[q]) * (uint32_t)pa.u_stride[q];
    return sg;
}

// Counts of the pattern emit's tiles: a CTA covers PE_THREADS consecutive parents, which are
// PE_THREADS / pt tiles of pt parents (pt a power of two from 8 to PE_THREADS).
__global__ void __launch_bounds__(PE_THREADS)
k_pcount(const __grid_constant__ PatArgs pa, const uint64_t* __restrict__ parents, uint64_t F,
         const unsigned long long* __restrict__ Fd, uint32_t pt, uint32_t* __restrict__ tile_counts) {
    if (Fd) F = *Fd;   // launched for an upper bound: the level's own size
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint64_t i = (uint64_t)blockIdx.x * PE_THREADS + t;
    uint32_t c = 0;
    if (i < F) c = __ldg(pa.cnt + sig_of(pa, parents ? __ldg(parents + i) : 0ull));
    const uint64_t tile0 = (uint64_t)blockIdx.x * (PE_THREADS / pt);
    if (pt <= 32) {   // a tile is pt aligned lanes of one warp
        for (uint32_t o = 1; o < pt; o <<= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if ((lane & (pt - 1)) == 0) tile_counts[tile0 + t / pt] = c;
        return;
    }
    __shared__ uint32_t ws[PE_THREADS / 32];
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) ws[warp] = c;
    __syncthreads();
    const int wpt = (int)(pt / 32);   // warps per tile
    if (t < PE_THREADS / (int)pt) {
        uint32_t sum = 0;
        for (int w = 0; w < wpt; ++w) sum += ws[t * wpt + w];
        tile_counts[tile0 + t] = sum;
    }
}

__global__ void __launch_bounds__(PE_THREADS)
k_pemit(const __grid_constant__ PatArgs pa, const uint64_t* __restrict__ parents, uint64_t F,
        const unsigned long long* __restrict__ Fd, uint32_t pt, uint32_t sub,
        const unsigned long long* __restrict__ tile_base, const unsigned long long* __restrict__ total,
        unsigned long long expect, uint64_t* __restrict__ out) {
    __shared__ uint32_t off_s[PE_THREADS], cnt_s[PE_THREADS], sig_s[PE_THREADS];
    __shared__ uint64_t par_s[PE_THREADS];
    __shared__ uint32_t wsum[PE_THREADS / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // the CTA's scan tile of pt parents and its part of sub parents in it
    const uint32_t parts = pt / sub;
    const uint64_t tile = blockIdx.x / parts;
    const uint32_t part = blockIdx.x - (uint32_t)(tile * parts);
    const uint64_t i0 = tile * pt;
    if (Fd) {   // launched for an upper bound: the level's own size
        F = *Fd;
        if (i0 >= F) return;
    }
    const uint64_t i = i0 + t;
    uint32_t c = 0, sg = 0;
    uint64_t parent = 0;
    if (t < (int)pt && i < F) {
        parent = parents ? __ldg(parents + i) : 0ull;
        sg = sig_of(pa, parent);
        c = __ldg(pa.cnt + sg);
    }
    uint32_t inc = c;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t base = 0;
    for (int w = 0; w < warp; ++w) base += wsum[w];
    off_s[t] = base + inc - c;
    cnt_s[t] = c;
    sig_s[t] = sg;
    par_s[t] = parent;
    __syncthreads();
    const uint64_t tb = tile_base[tile];
    if (expect != ~0ull && *total != expect) return;   // launched for another level size: write nothing
    const int np = (int)min((uint64_t)(part + 1) * sub, min((uint64_t)pt, F - i0));
    // wpp warps per parent (sub < 8) take its 32-key rows in turn
    constexpr int NW = PE_THREADS / 32;
    const int wpp = sub < NW ? NW / (int)sub : 1;
    const uint32_t S = 32u * (uint32_t)wpp;
    for (int p = (int)(part * sub) + warp / wpp; p < np; p += NW / wpp) {
        const uint32_t cp = cnt_s[p];
        const uint64_t par = par_s[p];
        const uint32_t* __restrict__ lst = pa.list + (uint64_t)sig_s[p] * pa.Bpad;
        uint64_t* __restrict__ o = out + tb + off_s[p];
        uint32_t jj = (uint32_t)(warp % wpp) * 32u + lane;
        for (; jj + 3 * S < cp; jj += 4 * S) {   // four independent 32-key rows per iteration
            const uint32_t a0 = __ldg(lst + jj), a1 = __ldg(lst + jj + S), a2 = __ldg(lst + jj + 2 * S),
                           a3 = __ldg(lst + jj + 3 * S);
            // streaming stores: the keys are written once per build, the pattern lists stay in L2
            __stcs(reinterpret_cast<unsigned long long*>(o + jj), par | ((uint64_t)a0 << pa.key_shift));
            __stcs(reinterpret_cast<unsigned long long*>(o + jj + S), par | ((uint64_t)a1 << pa.key_shift));
            __stcs(reinterpret_cast<unsigned long long*>(o + jj + 2 * S), par | ((uint64_t)a2 << pa.key_shift));
            __stcs(reinterpret_cast<unsigned long long*>(o + jj + 3 * S), par | ((uint64_t)a3 << pa.key_shift));
        }
        for (; jj < cp; jj += S)
            __stcs(reinterpret_cast<unsigned long long*>(o + jj), par | ((uint64_t)__ldg(lst + jj) << pa.key_shift));
    }
}

// Parents per scan tile of the pattern count and emit kernels: halved from 256 (down to 8) until
// the grid has about 64 tiles per SM, so that short parent lists still fill the SMs (with 256 per
// tile a level of 6,032 parents ran on 24 CTAs).
static uint64_t pattern_tile(uint64_t F) {
    int sms = 148, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t pt = PE_THREADS;
    while (pt > 8 && (F + pt - 1) / pt < (uint64_t)sms * 64) pt >>= 1;
    return pt;
}

// Parents per emit CTA: each emit CTA takes PE_SUB parents of its scan tile, one warp per parent,
// after scanning the whole tile's counts for their offsets.  Small CTAs keep the output the SMs
// write at one time short and even out the uneven child counts: the large space's last level
// (1.14M parents, scan tiles of 64) emits in 0.778 ms with 8 parents per CTA against 0.877 ms
// with 64 (8 per warp) and 0.810 ms with 16 (2 per warp); 4 and 2 parents per CTA, with 2 and 4
// warps sharing a parent's rows, took 1.03 and 1.73 ms.
constexpr uint64_t PE_SUB = 8;
static uint64_t emit_sub(uint64_t pt) { return pt < PE_SUB ? pt : PE_SUB; }

// ---------------------------------------------------------------------------
// host: lowering
// ---------------------------------------------------------------------------
static int ceil_log2(int64_t r) {
    int w = 0;
    while (((int64_t)1 << w) < r) ++w;
    return w;
}

static ct_status lower(ct_space* s, int32_t n, const int32_t* nv, const int64_t* vals, const ct_instr* prog,
                       int32_t n_instr) {
    DevSpace& h = s->h;
    if (n < 1 || n > MAXP) { set_error("n_params must be in [1, %d]", MAXP); return CT_ERR_LIMIT; }
    if (!nv || !vals || (n_instr > 0 && !prog) || n_instr < 0) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    h.n = n;
    int64_t total_vals = 0;
    for (int k = 0; k < n; ++k) {
        if (nv[k] < 1) { set_error("parameter %d has no values", k); return CT_ERR_INVALID_ARG; }
        if (nv[k] > BLOCK_BITS_MAX) { set_error("parameter %d has %d values (> %d)", k, nv[k], BLOCK_BITS_MAX); return CT_ERR_LIMIT; }
        h.r[k] = nv[k];
        h.vstart[k] = (int32_t)total_vals;
        total_vals += nv[k];
    }
    if (total_vals > MAXV) { set_error("%lld values in total (> %d)", (long long)total_vals, MAXV); return CT_ERR_LIMIT; }
    for (int64_t i = 0; i < total_vals; ++i) h.values[i] = vals[i];
    // key layout: param n-1 lowest
    int bits = 0;
    double cart_log2 = 0;
    for (int k = n - 1; k >= 0; --k) {
        h.w[k] = ceil_log2(h.r[k]);
        h.off[k] = bits;
        bits += h.w[k];
        cart_log2 += std::log2((double)h.r[k]);
    }
    if (bits > 64 || cart_log2 >= 62.99) { set_error("key needs %d bits (> 64) or Cartesian size >= 2^63", bits); return CT_ERR_KEY_OVERFLOW; }
    h.key_bits = bits;
    h.domain_bits = bits == 64 ? ~0ull : ((1ull << bits) - 1);
    h.swar_low = h.swar_high = 0;
    for (int k = 0; k < n; ++k) {
        h.fmask[k] = h.w[k] ? (((h.w[k] == 64) ? ~0ull : ((1ull << h.w[k]) - 1)) << h.off[k]) : 0ull;
        h.alt_rcp[k] = h.r[k] > 2 ? (uint32_t)((1ull << 32) / (uint64_t)(h.r[k] - 1) + 1) : 0u;
        if (h.w[k]) {
            h.swar_high |= 1ull << (h.off[k] + h.w[k] - 1);
            h.swar_low |= h.fmask[k] & ~(1ull << (h.off[k] + h.w[k] - 1));
        }
    }
    // constraints: split at END, validate stack discipline, collect scope
    if (n_instr > MAXI) { set_error("%d instructions (> %d)", n_instr, MAXI); return CT_ERR_LIMIT; }
    struct Raw { int pc, len; uint64_t scope; int level; };
    std::vector<Raw> raw;
    int start = 0, depth = 0;
    uint64_t scope = 0;
    for (int i = 0; i < n_instr; ++i) {
        const ct_instr& in = prog[i];
        switch (in.op) {
            case CT_OP_END:
                if (depth != 1) { set_error("constraint %zu leaves %d values on the stack", raw.size(), depth); return CT_ERR_INVALID_ARG; }
                {
                    int level = -1;
                    for (int k = 0; k < n; ++k) if (scope >> k & 1) level = k;
                    raw.push_back({start, i - start, scope, level});
                }
                start = i + 1; depth = 0; scope = 0;
                continue;
            case CT_OP_PARAM:
                if (in.arg < 0 || in.arg >= n) { set_error("instruction %d: parameter %d out of range", i, in.arg); return CT_ERR_INVALID_ARG; }
                scope |= 1ull << in.arg;
                ++depth; break;
            case CT_OP_CONST: ++depth; break;
            case CT_OP_NEG: case CT_OP_NOT:
                if (depth < 1) { set_error("instruction %d: stack underflow", i); return CT_ERR_INVALID_ARG; }
                break;
            default:
                if (in.op < CT_OP_ADD || in.op > CT_OP_OR) { set_error("instruction %d: bad opcode %d", i, in.op); return CT_ERR_INVALID_ARG; }
                if (depth < 2) { set_error("instruction %d: stack underflow", i); return CT_ERR_INVALID_ARG; }
                --depth; break;
        }
        if (depth > CT_MAX_STACK) { set_error("instruction %d: stack deeper than %d", i, CT_MAX_STACK); return CT_ERR_LIMIT; }
    }
    if (start != n_instr) { set_error("program does not end with CT_OP_END"); return CT_ERR_INVALID_ARG; }
    if ((int)raw.size() > MAXC) { set_error("%zu constraints (> %d)", raw.size(), MAXC); return CT_ERR_LIMIT; }
    for (int i = 0; i < n_instr; ++i) h.prog[i] = prog[i];

    // block plan: from the last parameter backwards, grow while the product fits
    std::vector<std::pair<int, int>> blocks;
    int e = n;
    while (e > 0) {
        int s0 = e - 1;
        int64_t prod = h.r[s0];
        while (s0 > 0 && prod * h.r[s0 - 1] <= BLOCK_BITS_MAX) { prod *= h.r[s0 - 1]; --s0; }
        blocks.push_back({s0, e});
        e = s0;
    }
    std::reverse(blocks.begin(), blocks.end());
    h.n_blocks = (int)blocks.size();
    std::vector<uint32_t> ik_all;
    for (int j = 0; j < h.n_blocks; ++j) {
        DevBlock& bl = h.blocks[j];
        bl.s = blocks[j].first;
        bl.e = blocks[j].second;
        int64_t B = 1;
        for (int k = bl.e - 1; k >= bl.s; --k) { bl.pstride[k - bl.s] = (int32_t)B; B *= h.r[k]; }
        bl.B = (int32_t)B;
        bl.W = (int32_t)((B + 31) / 32);
        bl.key_shift = h.off[bl.e - 1];
        bl.innerkey_off = (uint32_t)ik_all.size();
        ik_all.reserve(ik_all.size() + (size_t)B);
        int32_t dg[MAXP] = {};   // mixed-radix digits of point p, the last parameter fastest
        uint64_t key = 0;
        for (int64_t p = 0; p < B; ++p) {
            ik_all.push_back((uint32_t)(key >> bl.key_shift));
            for (int k = bl.e - 1; k >= bl.s; --k) {   // next point: an odometer step
                if (++dg[k] < h.r[k]) { key += 1ull << h.off[k]; break; }
                key -= (uint64_t)(h.r[k] - 1) << h.off[k];
                dg[k] = 0;
            }
        }
    }
    // attach constraints to blocks, sorted by block (stable)
    std::vector<int> order(raw.size());
    for (size_t i = 0; i < raw.size(); ++i) order[i] = (int)i;
    auto block_of = [&](int level) {
        if (level < 0) return 0;
        for (int j = 0; j < h.n_blocks; ++j) if (level >= h.blocks[j].s && level < h.blocks[j].e) return j;
        return 0;
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return block_of(raw[a].level) < block_of(raw[b].level); });
    h.n_cons = (int)raw.size();
    uint64_t words = 0;
    // table memory budget; CATUNE_TABLE_WORDS overrides it (0 interprets every constraint)
    uint64_t per_cons = TABLE_WORDS_PER_CONS, total_cap = TABLE_WORDS_TOTAL;
    if (const char* env = getenv("CATUNE_TABLE_WORDS")) per_cons = total_cap = strtoull(env, nullptr, 10);
    s->tab_cons.clear();
    s->tab_prefix.assign(1, 0);
    s->cz_cons.clear();
    s->cz_prefix.assign(1, 0);
    uint64_t cz_words = 0;
    for (int j = 0; j < h.n_blocks; ++j) { h.blocks[j].cons_begin = h.blocks[j].cons_end = 0; h.blocks[j].has_vm = 0; }
    for (int ci = 0; ci < h.n_cons; ++ci) {
        const Raw& rc = raw[order[ci]];
        DevCons& cs = h.cons[ci];
        memset(&cs, 0, sizeof cs);
        cs.pc = rc.pc; cs.len = rc.len; cs.level = rc.level; cs.block = block_of(rc.level);
        cs.scope = (uint32_t)rc.scope;
        const DevBlock& bl = h.blocks[cs.block];
        uint64_t rows = 1;
        cs.n_outer = 0;
        for (int k = 0; k < bl.s; ++k)
            if (rc.scope >> k & 1) { cs.outer_k[cs.n_outer++] = k; rows *= (uint64_t)h.r[k]; }
        uint64_t stride = 1;
        for (int q = cs.n_outer - 1; q >= 0; --q) { cs.outer_stride[q] = (int32_t)stride; stride *= h.r[cs.outer_k[q]]; }
        const uint64_t tw = rows * (uint64_t)bl.W;
        cs.cz_off = CZ_NONE;
        if (rows < (1ull << 31) && tw <= per_cons && words + tw <= total_cap) {
            cs.tabled = 1;
            cs.rows = (uint32_t)rows;
            cs.table_off = words;
            words += tw;
            s->tab_cons.push_back(ci);
            s->tab_prefix.push_back(words);
            // the table repeats each combination of the constraint's own parameters B / Bc
            // times: evaluate every combination once when that at least halves the work
            uint64_t bc = 1;
            cs.n_in = 0;
            for (int k = bl.e - 1; k >= bl.s; --k)
                if (rc.scope >> k & 1) { cs.in_k[cs.n_in] = k; cs.in_stride[cs.n_in++] = (int32_t)bc; bc *= (uint64_t)h.r[k]; }
            const uint64_t czw = rows * ((bc + 31) / 32);
            if (2 * bc <= (uint64_t)bl.B) {
                cs.cz_B = (uint32_t)bc;
                cs.cz_W = (uint32_t)((bc + 31) / 32);
                cs.cz_off = cz_words;
                cz_words += czw;
                s->cz_cons.push_back(ci);
                s->cz_prefix.push_back(cz_words);
            }
        } else {
            cs.tabled = 0;
        }
    }
    for (int ci = 0; ci < h.n_cons; ++ci) {
        DevBlock& bl = h.blocks[h.cons[ci].block];
        if (bl.cons_end == 0 && bl.cons_begin == 0) bl.cons_begin = ci;
        bl.cons_end = ci + 1;
        if (!h.cons[ci].tabled) bl.has_vm = 1;
    }
    for (int j = 0; j < h.n_blocks; ++j) if (h.blocks[j].cons_end == 0) h.blocks[j].cons_begin = 0;

    for (int k = 0; k < h.n; ++k) {
        h.pcons[k] = 0;
        for (int ci = 0; ci < h.n_cons; ++ci)
            if (h.cons[ci].scope >> k & 1) h.pcons[k] |= 1ull << ci;
    }


    // pattern plan: U = parameters before the block read by its constraints
    const uint64_t PAT_SIG_MAX = 1ull << 22, PAT_LIST_WORDS_MAX = 1ull << 26;   // 256 MB of lists
    s->pat_cnt_words = s->pat_list_words = 0;
    const bool no_patterns = getenv("CATUNE_NO_PATTERNS") != nullptr;   // forces the per-word path
    for (int j = 0; j < h.n_blocks; ++j) {
        DevBlock& bl = h.blocks[j];
        bl.pattern = 0;
        bl.n_u = 0;
        if (bl.has_vm || no_patterns) continue;
        uint64_t used = 0;
        for (int c = bl.cons_begin; c < bl.cons_end; ++c)
            for (int q = 0; q < h.cons[c].n_outer; ++q) used |= 1ull << h.cons[c].outer_k[q];
        uint64_t nsig = 1;
        for (int k = 0; k < bl.s; ++k)
            if (used >> k & 1) { bl.u_k[bl.n_u++] = k; nsig *= (uint64_t)h.r[k]; }
        const uint64_t bpad = ((uint64_t)bl.B + 3) / 4 * 4;
        if (nsig > PAT_SIG_MAX || s->pat_list_words + nsig * bpad > PAT_LIST_WORDS_MAX) continue;
        uint64_t st = 1;
        for (int q = bl.n_u - 1; q >= 0; --q) { bl.u_stride[q] = (int32_t)st; st *= (uint64_t)h.r[bl.u_k[q]]; }
        bl.pattern = 1;
        bl.n_sig = (uint32_t)nsig;
        bl.Bpad = (uint32_t)bpad;
        bl.pat_cnt_off = s->pat_cnt_words;
        bl.pat_list_off = s->pat_list_words;
        s->pat_cnt_words += nsig;
        s->pat_list_words += nsig * bpad;
    }

    s->frontier.resize(h.n_blocks);
    s->ik_host = std::move(ik_all);
    return CT_OK;
}

// Pinned host staging shared by the uploads of small host tables: one copy into it, one
// asynchronous copy per table, instead of a synchronous copy per table.  An event recorded after
// the copies guards the stage: the next upload waits for it before overwriting the stage.  With
// sync, the call also waits for its own copies (callers whose data other streams may read next).
namespace {
struct PinnedStage {
    std::mutex mu;
    char* p = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;   // the copies of the last upload
    int done_dev = -1;            // the device the event belongs to
    bool pending = false;
};
PinnedStage g_stage;

struct Upload {
    void* dst;
    const void* src;
    size_t bytes;
};

ct_status stage_uploads(const std::vector<Upload>& ups, cudaStream_t st, bool sync) {
    size_t bytes = 0;
    for (const Upload& u : ups) bytes += (u.bytes + 15) & ~size_t(15);
    if (!bytes) return CT_OK;
    std::lock_guard<std::mutex> lk(g_stage.mu);
    if (g_stage.pending) {   // the previous upload's copies may still read the stage
        CT_TRY_CUDA(cudaEventSynchronize(g_stage.done));
        g_stage.pending = false;
    }
    int dev = 0;
    CT_TRY_CUDA(cudaGetDevice(&dev));
    if (g_stage.done && g_stage.done_dev != dev) {   // an event is recorded on its own device's streams
        cudaEventDestroy(g_stage.done);
        g_stage.done = nullptr;
    }
    if (!g_stage.done) {
        CT_TRY_CUDA(cudaEventCreateWithFlags(&g_stage.done, cudaEventDisableTiming));
        g_stage.done_dev = dev;
    }
    if (g_stage.cap < bytes) {
        if (g_stage.p) cudaFreeHost(g_stage.p);
        g_stage.p = nullptr;
        g_stage.cap = 0;
        const size_t want = std::max<size_t>(bytes, 1 << 20);
        CT_TRY_CUDA(cudaMallocHost(reinterpret_cast<void**>(&g_stage.p), want));
        g_stage.cap = want;
    }
    size_t off = 0;
    for (const Upload& u : ups) {
        if (!u.bytes) continue;
        memcpy(g_stage.p + off, u.src, u.bytes);
        CT_TRY_CUDA(cudaMemcpyAsync(u.dst, g_stage.p + off, u.bytes, cudaMemcpyHostToDevice, st));
        off += (u.bytes + 15) & ~size_t(15);
    }
    if (sync) {
        CT_TRY_CUDA(cudaStreamSynchronize(st));
    } else {
        CT_TRY_CUDA(cudaEventRecord(g_stage.done, st));
        g_stage.pending = true;
    }
    return CT_OK;
}
}  // namespace

// first device use: descriptor, tables, ball plan and status word go to the current device
ct_status ensure_device(ct_space* s, cudaStream_t st, bool sync) {
    if (s->d) return CT_OK;
    const DevSpace& h = s->h;
    cudaGetDevice(&s->device);
    {
        cudaError_t e = cudaSuccess;
        s->d = static_cast<DevSpace*>(dev_alloc(sizeof(DevSpace), &e));
        if (!s->d) { set_error("device allocation failed: %s", cudaGetErrorString(e)); return CT_ERR_OOM; }
    }
    std::vector<Upload> ups;
    ups.push_back({s->d, &h, sizeof(DevSpace)});
    CT_TRY(s->innerkey.ensure(s->ik_host.size()));
    ups.push_back({s->innerkey.p, s->ik_host.data(), s->ik_host.size() * 4});
    CT_TRY(s->tables.ensure(s->tab_prefix.back()));
    if (!s->tab_cons.empty()) {
        CT_TRY(s->d_tab_cons.ensure(s->tab_cons.size()));
        CT_TRY(s->d_tab_prefix.ensure(s->tab_prefix.size()));
        ups.push_back({s->d_tab_cons.p, s->tab_cons.data(), s->tab_cons.size() * 4});
        ups.push_back({s->d_tab_prefix.p, s->tab_prefix.data(), s->tab_prefix.size() * 8});
    }
    if (!s->cz_cons.empty()) {
        CT_TRY(s->d_cz_cons.ensure(s->cz_cons.size()));
        CT_TRY(s->d_cz_prefix.ensure(s->cz_prefix.size()));
        ups.push_back({s->d_cz_cons.p, s->cz_cons.data(), s->cz_cons.size() * 4});
        ups.push_back({s->d_cz_prefix.p, s->cz_prefix.data(), s->cz_prefix.size() * 8});
    }
    CT_TRY(s->compact.ensure(s->cz_prefix.back()));
    s->h.compact = s->compact.p;   // before the descriptor's copy below is staged
    CT_TRY(s->status.ensure(1));
    CT_TRY_CUDA(cudaMemsetAsync(s->status.p, 0, 4, st));
    CT_TRY(s->pat_cnt.ensure(s->pat_cnt_words));
    CT_TRY(s->pat_list.ensure(s->pat_list_words));
    CT_TRY(stage_uploads(ups, st, sync));
    CT_TRY_CUDA(cudaFuncSetAttribute(k_expand_emit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     EXP_THREADS * 32 * (int)sizeof(uint64_t)));
    return CT_OK;
}

// Hamming-ball sizes: the number of points at distance exactly d is the d-th elementary
// symmetric polynomial of (r_k - 1) over the parameters with r_k > 1.  Radii stop where the
// subsets, the points or one subset's size outgrow the enumeration tables.
static void plan_ball_sizes(ct_space* s) {
    const DevSpace& h = s->h;
    std::vector<uint64_t> a;
    for (int k = 0; k < h.n; ++k) if (h.r[k] > 1) a.push_back((uint64_t)(h.r[k] - 1));
    const int m = (int)a.size();
    const uint64_t SUBSET_CAP = 1u << 20, POINT_CAP = 1ull << 40, BIG = POINT_CAP + 1;
    std::vector<uint64_t> e(MAX_RADIUS + 1, 0);
    e[0] = 1;
    for (uint64_t ak : a)
        for (int d = MAX_RADIUS; d >= 1; --d) {
            const unsigned __int128 v = (unsigned __int128)e[d] + (unsigned __int128)e[d - 1] * ak;
            e[d] = v > BIG ? BIG : (uint64_t)v;
        }
    std::vector<uint64_t> desc = a;
    std::sort(desc.rbegin(), desc.rend());
    s->ball_max = 0;
    unsigned __int128 subsets = 1, largest = 1;
    for (int d = 1; d <= std::min(m, MAX_RADIUS); ++d) {
        subsets = subsets * (unsigned)(m - d + 1) / (unsigned)d;   // C(m, d)
        largest *= desc[d - 1];
        if (subsets > SUBSET_CAP || e[d] > POINT_CAP || largest >= ((unsigned __int128)1 << 32)) break;
        s->ball_total[d] = e[d];
        s->ball_max = d;
    }
}

// Radius the repair path will use: the cost-model radius, or the one set by ct_set_repair_mode.
int wanted_radius(const ct_space* s) {
    if (s->repair_mode == 1) return 0;
    if (s->repair_mode == 2) return std::min(s->repair_max_radius, s->ball_max);
    return auto_radius(s);
}

// Host part of the ball tables: enumerates radii balls.size()+1 .. dmax (subsets of the
// parameters with r_k > 1, in lexicographic order, with prefix sums of their sizes).  No CUDA
// call, so the build runs it while its last level is still being emitted.
static void plan_balls(ct_space* s, int dmax) {
    dmax = std::min(dmax, s->ball_max);
    const DevSpace& h = s->h;
    std::vector<int> free_k;
    for (int k = 0; k < h.n; ++k) if (h.r[k] > 1) free_k.push_back(k);
    const int m = (int)free_k.size();
    for (int d = (int)s->balls.size() + 1; d <= dmax; ++d) {
        BallRadius br;
        br.d = d;
        br.prefix.reserve(s->ball_total[d] ? 1024 : 1);
        br.prefix.push_back(0);
        std::vector<int> idx(d);
        for (int i = 0; i < d; ++i) idx[i] = i;
        while (true) {
            uint32_t mask = 0;
            uint64_t sz = 1;
            for (int i = 0; i < d; ++i) { mask |= 1u << free_k[idx[i]]; sz *= (uint64_t)(h.r[free_k[idx[i]]] - 1); }
            br.masks.push_back(mask);
            br.total += sz;
            br.prefix.push_back(br.total);
            int i = d - 1;
            while (i >= 0 && idx[i] == m - d + i) --i;
            if (i < 0) break;
            ++idx[i];
            for (int t = i + 1; t < d; ++t) idx[t] = idx[t - 1] + 1;
        }
        s->balls.push_back(std::move(br));
    }
}


// Device part: uploads every planned radius that has no device tables yet.  sync = false only
// inside the build, whose final synchronisation then covers the copies.
static ct_status upload_balls(ct_space* s, cudaStream_t st, bool sync) {
    std::vector<Upload> ups;
    for (BallRadius& br : s->balls) {
        if (br.d_masks.p) continue;
        if (ups.empty()) CT_TRY(ensure_device(s, st, sync));
        CT_TRY(br.d_masks.ensure(br.masks.size()));
        CT_TRY(br.d_prefix.ensure(br.prefix.size()));
        ups.push_back({br.d_masks.p, br.masks.data(), br.masks.size() * 4});
        ups.push_back({br.d_prefix.p, br.prefix.data(), br.prefix.size() * 8});
    }
    return stage_uploads(ups, st, sync);
}

ct_status ensure_balls(ct_space* s, int dmax) {
    plan_balls(s, dmax);
    return upload_balls(s, nullptr, true);
}

static ct_status ensure_tables(ct_space* s, cudaStream_t st) {
    if (s->tables_ready) return CT_OK;
    const uint64_t words = s->tab_prefix.back();
    const uint64_t cz_words = s->cz_prefix.back();
    if (cz_words) {
        CT_TRY(s->compact.ensure(cz_words));
        const unsigned grid = (unsigned)((cz_words * 32 + 255) / 256);
        k_build_compact<<<grid, 256, 0, st>>>(s->d, s->d_cz_cons.p, s->d_cz_prefix.p, (int)s->cz_cons.size(), cz_words,
                                              s->compact.p);
        count_launch();
    }
    if (words) {
        uint64_t runs = 0;   // every constraint's words in runs of TB_WORDS_PER_CTA, one CTA each
        for (size_t i = 0; i + 1 < s->tab_prefix.size(); ++i)
            runs += (s->tab_prefix[i + 1] - s->tab_prefix[i] + TB_WORDS_PER_CTA - 1) / TB_WORDS_PER_CTA;
        if (runs > 0x7fffffffull) { set_error("%llu table runs", (unsigned long long)runs); return CT_ERR_LIMIT; }
        k_build_tables<<<(unsigned)runs, 256, 0, st>>>(s->d, s->d_tab_cons.p, (int)s->tab_cons.size(), s->d_tab_prefix.p,
                                                       s->compact.p, s->innerkey.p, s->tables.p);
        count_launch();
        CT_TRY_CUDA(cudaGetLastError());
    }
    PatBlocks pb;   // every pattern block in one launch: the blocks are independent
    memset(&pb, 0, sizeof pb);
    uint64_t ctas = 0;
    for (int j = 0; j < s->h.n_blocks; ++j) {
        const DevBlock& bl = s->h.blocks[j];
        if (!bl.pattern) continue;
        pb.blk[pb.n] = j;
        pb.first[pb.n] = (uint32_t)ctas;
        ++pb.n;
        ctas += bl.n_sig;
    }
    if (ctas > 0x7fffffffull) { set_error("%llu pattern signatures", (unsigned long long)ctas); return CT_ERR_LIMIT; }
    if (pb.n) {
        k_build_patterns<<<(unsigned)ctas, PAT_THREADS, 0, st>>>(s->d, s->tables.p, s->innerkey.p, pb, s->pat_cnt.p,
                                                                 s->pat_list.p);
        count_launch();
    }
    CT_TRY_CUDA(cudaGetLastError());
    s->tables_ready = true;
    return CT_OK;
}

static PatArgs pat_args(const ct_space* s, int j) {
    const DevSpace& h = s->h;
    const DevBlock& bl = h.blocks[j];
    PatArgs pa;
    memset(&pa, 0, sizeof pa);
    pa.n_u = bl.n_u;
    pa.key_shift = bl.key_shift;
    pa.Bpad = bl.Bpad;
    for (int q = 0; q < bl.n_u; ++q) {
        pa.u_mask[q] = h.fmask[bl.u_k[q]];
        pa.u_off[q] = h.off[bl.u_k[q]];
        pa.u_stride[q] = bl.u_stride[q];
    }
    pa.cnt = s->pat_cnt.p + bl.pat_cnt_off;
    pa.list = s->pat_list.p + bl.pat_list_off;
    return pa;
}

}  // namespace ct

using namespace ct;

ct_space::~ct_space() {
    for (auto& e : events) cudaEventDestroy(e);
    if (d) dev_free(d, sizeof(ct::DevSpace));
    pat_cnt.release(); pat_list.release();
    tables.release(); d_tab_cons.release(); d_tab_prefix.release(); innerkey.release();
    compact.release(); d_cz_cons.release(); d_cz_prefix.release();
    keys.release(); tile_counts.release(); tile_base.release(); d_total.release(); status.release();
    for (auto& f : frontier) f.release();
    for (auto& b : balls) { b.d_masks.release(); b.d_prefix.release(); }
    rs.release_all();
    rules.release_all();
    occ.release();
}

extern "C" {

const char* ct_last_error(void) { return ct::last_error(); }
const char* ct_version(void) { return "catune 0.1 (sm_103a)"; }

ct_status ct_define_space(int32_t n_params, const int32_t* n_values, const int64_t* values_flat,
                          const ct_instr* program, int32_t n_instr, ct_space** out) {
    if (!out) { set_error("out is NULL"); return CT_ERR_INVALID_ARG; }
    *out = nullptr;
    ct_space* s = new (std::nothrow) ct_space();
    if (!s) { set_error("host allocation failed"); return CT_ERR_OOM; }
    ct_status st = lower(s, n_params, n_values, values_flat, program, n_instr);
    if (st == CT_OK) plan_ball_sizes(s);
    if (st != CT_OK) { delete s; return st; }
    *out = s;
    return CT_OK;
}

void ct_space_destroy(ct_space* s) { delete s; }

ct_status ct_space_info_get(const ct_space* s, ct_space_info* info) {
    if (!s || !info) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    memset(info, 0, sizeof *info);
    info->n_params = s->h.n;
    info->n_constraints = s->h.n_cons;
    info->key_bits = s->h.key_bits;
    info->n_blocks = s->h.n_blocks;
    uint64_t cart = 1;
    for (int k = 0; k < s->h.n; ++k) {
        info->width[k] = s->h.w[k];
        info->offset[k] = s->h.off[k];
        info->n_values[k] = s->h.r[k];
        cart *= (uint64_t)s->h.r[k];
    }
    info->cartesian = cart;
    info->n_valid = s->n_valid;
    info->built = s->built;
    return CT_OK;
}

ct_status ct_pack_keys(const ct_space* s, const int32_t* idx, int64_t n, uint64_t* keys) {
    if (!s || (n > 0 && (!idx || !keys)) || n < 0) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    const int np = s->h.n;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t k = 0;
        for (int p = 0; p < np; ++p) {
            const int32_t v = idx[i * np + p];
            if (v < 0 || v >= s->h.r[p]) { set_error("row %lld: index %d of parameter %d out of range", (long long)i, v, p); return CT_ERR_INVALID_ARG; }
            k |= (uint64_t)v << s->h.off[p];
        }
        keys[i] = k;
    }
    return CT_OK;
}

ct_status ct_unpack_keys(const ct_space* s, const uint64_t* keys, int64_t n, int32_t* idx) {
    if (!s || (n > 0 && (!idx || !keys)) || n < 0) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    const int np = s->h.n;
    for (int64_t i = 0; i < n; ++i)
        for (int p = 0; p < np; ++p) idx[i * np + p] = (int32_t)((keys[i] & s->h.fmask[p]) >> s->h.off[p]);
    return CT_OK;
}

ct_status ct_unpack_keys_device(const ct_space* s, const uint64_t* d_keys, int64_t n, int32_t* d_idx,
                                ct_stream stream) {
    if (!s || (n > 0 && (!d_idx || !d_keys)) || n < 0) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    if (n == 0) return CT_OK;
    if (!s->d) { set_error("space not on the device yet (build it first)"); return CT_ERR_STATE; }
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t total = n * s->h.n;
    const unsigned g = (unsigned)std::min<int64_t>((total + 255) / 256, (int64_t)sms * 16);
    k_unpack<<<g, 256, 0, (cudaStream_t)stream>>>(s->d, d_keys, n, d_idx);
    count_launch();
    CT_TRY_CUDA(cudaGetLastError());
    return CT_OK;
}

// Largest upper bound of a level's size (in keys) for which a first build allocates the level's
// frontier by that bound and launches the level without reading its size back.
constexpr uint64_t FRONTIER_BOUND_MAX = 1ull << 25;   // 256 MB of keys

// One pass over the levels: per level the count kernel, the scan of the tile counts (the level's
// size into d_total[j]) and the emit.  The emit's grid and the next level's need the level's size
// on the host.
// - Hinted mode takes the sizes from the last build of this space (a space's definition never
//   changes, so its levels have the same sizes every time) and launches every level without
//   waiting; each emit compares the hint with its level's total on the device and writes nothing
//   if they differ, and the host checks all totals once at the end (*ok = false: a size
//   differed, the pass is void).
// - A first build reads a level's size back only where the host needs it: before the last level
//   (whose grids are sized by its exact parent count) and after it (|V|), or where a level's
//   Cartesian upper bound exceeds FRONTIER_BOUND_MAX.  Other levels run on that upper bound:
//   their frontier buffer and grids are sized by it and their kernels read the exact parent count
//   from the previous level's total on the device.
static ct_status build_levels(ct_space* s, cudaStream_t st, bool hinted, bool* ok) {
    const DevSpace& h = s->h;
    const uint64_t* parents = nullptr;
    uint64_t F = 1;          // parents of the level: exact when `known`, else an upper bound
    bool known = true;
    *ok = true;
    const float setup_ms = s->stats.host_setup_ms;
    memset(&s->stats, 0, sizeof s->stats);
    s->stats.timed = s->timing;
    s->stats.host_setup_ms = setup_ms;
    CT_TRY(s->d_total.ensure((size_t)h.n_blocks));
    s->h_totals.resize((size_t)h.n_blocks);
    const int n_hint = (int)s->hint.size();
    int L = h.n_blocks;      // levels launched
    for (int j = 0; j < h.n_blocks; ++j) {
        const DevBlock& bl = h.blocks[j];
        const bool last = j == h.n_blocks - 1;
        const uint64_t items = bl.pattern ? F : F * (uint64_t)bl.W;
        const uint64_t per_tile = bl.pattern ? pattern_tile(F) : EXP_TILE;
        const uint64_t tiles = (items + per_tile - 1) / per_tile;
        const uint64_t count_ctas = bl.pattern ? (F + PE_THREADS - 1) / PE_THREADS : tiles;
        const uint64_t emit_ctas = bl.pattern ? tiles * (per_tile / emit_sub(per_tile)) : tiles;
        if (emit_ctas > 0x7fffffffull || count_ctas > 0x7fffffffull) {
            set_error("level %d needs %llu tiles", j, (unsigned long long)tiles);
            return CT_ERR_LIMIT;
        }
        CT_TRY(s->tile_counts.ensure(bl.pattern ? count_ctas * (PE_THREADS / per_tile) : tiles));
        CT_TRY(s->tile_base.ensure(tiles));
        const unsigned long long* Fd = known ? nullptr : s->d_total.p + (j - 1);
        PatArgs pa;
        if (bl.pattern) pa = pat_args(s, j);
        if (s->timing) CT_TRY_CUDA(cudaEventRecord(s->events[4 * j], st));
        if (bl.pattern)
            k_pcount<<<(unsigned)count_ctas, PE_THREADS, 0, st>>>(pa, parents, F, Fd, (uint32_t)per_tile,
                                                                  s->tile_counts.p);
        else
            k_expand_count<<<(unsigned)tiles, EXP_THREADS, 0, st>>>(s->d, s->tables.p, s->innerkey.p, j, parents,
                                                                   items, Fd, s->tile_counts.p);
        if (s->timing) CT_TRY_CUDA(cudaEventRecord(s->events[4 * j + 1], st));
        unsigned long long* total = s->d_total.p + j;
        k_scan_tiles<<<1, SCAN_T, 0, st>>>(s->tile_counts.p, tiles, s->tile_base.p, total);
        count_launch(2);
        uint64_t Fn;
        bool known_next = true;
        const uint64_t bound = F * (uint64_t)bl.B;   // Cartesian bound of the level's size
        if (hinted) {
            Fn = j < n_hint ? s->hint[j] : 0;
        } else if (last || j + 1 == h.n_blocks - 1 || bound > FRONTIER_BOUND_MAX || bound / (uint64_t)bl.B != F) {
            // every total so far in one read (the unread levels' sizes for the statistics)
            CT_TRY_CUDA(cudaMemcpyAsync(s->h_totals.data(), s->d_total.p, (size_t)(j + 1) * 8, cudaMemcpyDeviceToHost, st));
            CT_TRY_CUDA(cudaStreamSynchronize(st));
            Fn = s->h_totals[j];
        } else {
            Fn = bound;
            known_next = false;
        }
        DevBuf<uint64_t>& dst = last ? s->keys : s->frontier[j];
        CT_TRY(dst.ensure(Fn));
        if (Fn) {
            const unsigned long long expect = hinted ? (unsigned long long)Fn : ~0ull;
            if (s->timing) CT_TRY_CUDA(cudaEventRecord(s->events[4 * j + 2], st));
            if (bl.pattern)
                k_pemit<<<(unsigned)emit_ctas, PE_THREADS, 0, st>>>(
                    pa, parents, F, Fd, (uint32_t)per_tile, (uint32_t)emit_sub(per_tile), s->tile_base.p, total, expect,
                    dst.p);
            else
                k_expand_emit<<<(unsigned)tiles, EXP_THREADS, EXP_THREADS * 32 * sizeof(uint64_t), st>>>(
                    s->d, s->tables.p, s->innerkey.p, j, parents, items, Fd, s->tile_base.p, total, expect, dst.p);
            if (s->timing) CT_TRY_CUDA(cudaEventRecord(s->events[4 * j + 3], st));
            count_launch();
            CT_TRY_CUDA(cudaGetLastError());
        }
        s->stats.parents[j] = F;
        s->stats.children[j] = Fn;
        parents = dst.p;
        F = Fn;
        known = known_next;
        if (known && F == 0) { L = j + 1; break; }
        if (last) {   // the host plans the ball tables while the last level is emitted
            s->n_valid = F;
            plan_balls(s, wanted_radius(s));
            CT_TRY(upload_balls(s, st, false));   // queued behind the emit
        }
    }
    if (hinted) {   // the levels ran on the hints: read every level's own size back and compare
        CT_TRY_CUDA(cudaMemcpyAsync(s->h_totals.data(), s->d_total.p, (size_t)L * 8, cudaMemcpyDeviceToHost, st));
        CT_TRY_CUDA(cudaStreamSynchronize(st));
        for (int j = 0; j < L; ++j)
            if (s->h_totals[j] != (unsigned long long)s->stats.children[j]) *ok = false;
    } else {
        // levels launched on bounds: their exact sizes came back with the last read.  A level that
        // came out empty ends the statistics there (the levels after it ran on no parents).
        for (int j = 0; j < L; ++j) {
            s->stats.children[j] = s->h_totals[j];
            s->stats.parents[j] = j ? s->h_totals[j - 1] : 1;
            if (s->h_totals[j] == 0) { L = j + 1; break; }
        }
    }
    s->stats.n_levels = L;
    // Level by level, every size was read back before it was needed: nothing is left to check, so
    // the call returns while the last level's emit (and the ball-table upload behind it) still
    // run; every later use of the keys is ordered after them on the stream.
    s->n_valid = s->stats.children[L - 1];
    return CT_OK;
}

// Whether every buffer a hinted pass writes already holds the hinted sizes: a hinted pass then
// allocates and releases nothing (no block goes back to the cache while earlier work that may
// read it is still queued).  Otherwise the build takes the level-by-level path, which grows
// buffers only after a synchronisation.
static bool hint_fits(const ct_space* s) {
    const DevSpace& h = s->h;
    const int L = (int)s->hint.size();
    if (L == 0 || L > h.n_blocks || s->d_total.cap < (size_t)h.n_blocks) return false;
    uint64_t F = 1;
    for (int j = 0; j < L; ++j) {
        const DevBlock& bl = h.blocks[j];
        const uint64_t items = bl.pattern ? F : F * (uint64_t)bl.W;
        const uint64_t per_tile = bl.pattern ? pattern_tile(F) : EXP_TILE;
        const uint64_t tiles = (items + per_tile - 1) / per_tile;
        const uint64_t counts = bl.pattern ? (F + PE_THREADS - 1) / PE_THREADS * (PE_THREADS / per_tile) : tiles;
        if (counts > s->tile_counts.cap || tiles > s->tile_base.cap) return false;
        const uint64_t Fn = s->hint[j];
        const DevBuf<uint64_t>& dst = (j == h.n_blocks - 1) ? s->keys : s->frontier[j];
        if (!dst.p || Fn > dst.cap) return false;
        F = Fn;
        if (F == 0) break;
    }
    return true;
}

// Hinted builds are on unless CATUNE_BUILD_PIPELINE=0.  CATUNE_BUILD_HINT_SKEW=k (nonzero) adds k
// to the hinted size of the last level, which makes the check fail: the emit writes nothing and
// the build is redone level by level (used to test that path).
static bool build_pipeline_enabled() {
    const char* e = getenv("CATUNE_BUILD_PIPELINE");
    return !(e && e[0] == '0');
}
static long long build_hint_skew() {
    const char* e = getenv("CATUNE_BUILD_HINT_SKEW");
    return e ? atoll(e) : 0;
}

ct_status ct_build_valid_space(ct_space* s, ct_stream stream, uint64_t* n_valid_out) {
    if (!s) { set_error("space is NULL"); return CT_ERR_INVALID_ARG; }
    using clk = std::chrono::steady_clock;
    const auto ms_since = [](clk::time_point a) { return std::chrono::duration<float, std::milli>(clk::now() - a).count(); };
    const auto t0 = clk::now();
    cudaStream_t st = (cudaStream_t)stream;
    CT_TRY(ensure_device(s, st, false));   // the build synchronises st before it returns
    CT_TRY(ensure_tables(s, st));
    s->stats.host_setup_ms = ms_since(t0);
    const auto t1 = clk::now();
    const DevSpace& h = s->h;
    s->built = false;
    s->occ_ready = false;
    if (s->timing && s->events.empty()) {
        s->events.resize(4 * (size_t)h.n_blocks);
        for (auto& e : s->events) CT_TRY_CUDA(cudaEventCreate(&e));
    }
    bool hinted = build_pipeline_enabled() && !s->hint.empty();
    if (hinted) {
        const long long skew = build_hint_skew();
        if (skew && (int)s->hint.size() == h.n_blocks) s->hint.back() = (uint64_t)((long long)s->hint.back() + skew);
        hinted = hint_fits(s);
    }
    bool ok = true;
    CT_TRY(build_levels(s, st, hinted, &ok));
    if (!ok) {   // a level size differed from the hint: redo the build reading each size back
        hinted = false;
        CT_TRY(build_levels(s, st, false, &ok));
    }
    s->hint.assign(s->stats.children, s->stats.children + s->stats.n_levels);
    s->stats.hinted = hinted ? 1 : 0;
    const uint64_t F = s->n_valid;
    s->built = true;
    if (n_valid_out) *n_valid_out = F;
    s->stats.host_levels_ms = ms_since(t1);
    const auto t2 = clk::now();
    if (F) CT_TRY(upload_balls(s, st, true));   // nothing left to upload, unless the last level was empty
    s->stats.host_balls_ms = ms_since(t2);
    s->stats.host_total_ms = ms_since(t0);
    if (F == 0) { set_error("no configuration satisfies the constraints"); return CT_ERR_EMPTY_SPACE; }
    return CT_OK;
}

ct_status ct_space_set_timing(ct_space* s, int32_t enable) {
    if (!s) { set_error("space is NULL"); return CT_ERR_INVALID_ARG; }
    s->timing = enable != 0;
    return CT_OK;
}

ct_status ct_space_build_stats(const ct_space* s, ct_build_stats* out) {
    if (!s || !out) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    *out = s->stats;
    if (s->stats.timed && s->built) {   // the kernel times, once the build's last event has completed
        const int L = s->stats.n_levels;
        CT_TRY_CUDA(cudaEventSynchronize(s->events[4 * (L - 1) + (s->stats.children[L - 1] ? 3 : 1)]));
        for (int j = 0; j < L; ++j) {
            CT_TRY_CUDA(cudaEventElapsedTime(&out->count_ms[j], s->events[4 * j], s->events[4 * j + 1]));
            if (s->stats.children[j])
                CT_TRY_CUDA(cudaEventElapsedTime(&out->emit_ms[j], s->events[4 * j + 2], s->events[4 * j + 3]));
        }
    }
    return CT_OK;
}

uint64_t ct_launch_count(void) { return g_launches.load(); }
uint64_t ct_alloc_count(void) { return g_allocs.load(); }

void ct_trim_cache(void) {
    BlockCache& c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    flush_device(c, current_device());
}

ct_status ct_space_keys(const ct_space* s, const uint64_t** d_keys, uint64_t* n) {
    if (!s || !d_keys) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    if (!s->built) { set_error("space not built"); return CT_ERR_STATE; }
    *d_keys = s->keys.p;
    if (n) *n = s->n_valid;
    return CT_OK;
}

ct_status ct_set_fitness(ct_space* s, const float* d_table, uint64_t n) {
    if (!s || !d_table) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    if (!s->built) { set_error("space not built"); return CT_ERR_STATE; }
    if (n != s->n_valid) { set_error("table has %llu entries, space has %llu valid", (unsigned long long)n, (unsigned long long)s->n_valid); return CT_ERR_INVALID_ARG; }
    s->fit = d_table;
    s->n_fit = n;
    return CT_OK;
}

ct_status ct_set_eval_cost(ct_space* s, const uint32_t* d_cost, uint64_t n) {
    if (!s) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    if (!d_cost) { s->cost = nullptr; return CT_OK; }
    if (!s->built) { set_error("space not built"); return CT_ERR_STATE; }
    if (n != s->n_valid) { set_error("cost table has %llu entries, space has %llu valid", (unsigned long long)n, (unsigned long long)s->n_valid); return CT_ERR_INVALID_ARG; }
    s->cost = d_cost;
    return CT_OK;
}

ct_status ct_space_status(ct_space* s, ct_stream stream) {
    if (!s) { set_error("space is NULL"); return CT_ERR_INVALID_ARG; }
    uint32_t v = 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (!s->d) return CT_OK;
    CT_TRY_CUDA(cudaMemcpyAsync(&v, s->status.p, 4, cudaMemcpyDeviceToHost, st));
    CT_TRY_CUDA(cudaMemsetAsync(s->status.p, 0, 4, st));
    CT_TRY_CUDA(cudaStreamSynchronize(st));
    if (v & ST_BAD_CANDIDATE) { set_error("a candidate key was outside the Cartesian domain"); return CT_ERR_INVALID_ARG; }
    return CT_OK;
}

}  // extern "C"
