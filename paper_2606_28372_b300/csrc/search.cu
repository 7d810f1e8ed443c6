// Validity lookup, nearest-valid repair and fitness lookup over the resolved space.
//
// Repair returns, for an invalid candidate u, the valid key v minimising
// (Hamming distance on value indices, key) — the exact nearest neighbour of
// Algorithm 1's Repair under the Hamming neighbour rule of Section IV-A.  Two
// exact strategies are combined:
//   ball search: for radius d = 1, 2, ... every point at distance exactly d is
//     generated (subsets of d parameters x alternative values) and tested with
//     the constraint truth masks; if any is valid, the smallest such key is the
//     answer because every point outside the ball is farther away;
//   streaming scan: for the candidates still pending, every valid key is read
//     once per chunk of 32 candidates; per (key, candidate) the distance is a
//     SWAR per-field non-zero test plus a population count, reduced as the packed
//     minimum of (distance << 57 | rank) by warp shuffles, shared memory and one
//     64-bit atomicMin per candidate and CTA.  On long key arrays, chunks of three or
//     more candidates use per-candidate distance tables instead (scan_lut.cu).
#include <cuda_runtime.h>

#include <climits>
#include <cstdlib>

#include "internal.hpp"

namespace ct {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_CHUNK = 32;        // candidates per CTA of the scan
constexpr unsigned long long NONE = ~0ull;
constexpr int64_t SCAN_FOLD_MAX = 4096;   // repairs of up to this many candidates resolve in the last scan CTA

// a warp per candidate (the warp's 32-ary rank search)
__global__ void k_lookup(const DevSpace* __restrict__ sp, const uint64_t* __restrict__ keys, int64_t nv,
                         const uint64_t* __restrict__ cand, int64_t n, int64_t* __restrict__ rank) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const uint64_t c = cand[i];
        const int64_t r = in_domain(sp, c) ? rank_of_warp(keys, nv, c, lane) : -1;
        if (lane == 0) rank[i] = r;
    }
}

// a warp per candidate: the warp's rank search, then lane 0 does the lookups and the memo
__global__ void k_evaluate(const DevSpace* __restrict__ sp, const uint64_t* __restrict__ keys, int64_t nv,
                           const float* __restrict__ table, const uint64_t* __restrict__ cand, int64_t n,
                           float* __restrict__ fit, int64_t* __restrict__ rank_out, uint32_t* __restrict__ memo,
                           unsigned long long* __restrict__ unique, const uint32_t* __restrict__ cost,
                           unsigned long long* __restrict__ cost_acc, float invalid_fit) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const uint64_t c = cand[i];
        const int64_t r = in_domain(sp, c) ? rank_of_warp(keys, nv, c, lane) : -1;
        if (lane) continue;
        if (fit) fit[i] = r >= 0 ? __ldg(table + r) : invalid_fit;
        if (rank_out) rank_out[i] = r;
        if (memo && r >= 0) {
            const uint32_t bit = 1u << (r & 31);
            const uint32_t old = atomicOr(memo + (r >> 5), bit);
            if (!(old & bit)) {   // first evaluation of this configuration
                atomicAdd(unique, 1ull);
                if (cost) atomicAdd(cost_acc, (unsigned long long)__ldg(cost + r));
            }
        }
    }
}

// a warp per candidate: lane c tests constraint c (and c + 32), a ballot gives the failing mask;
// lane 0 settles valid and out-of-domain candidates and queues the others
__global__ void k_repair_init(const DevSpace* __restrict__ sp, const uint32_t* __restrict__ tables,
                              const uint64_t* __restrict__ cand, int64_t n, uint64_t* __restrict__ out,
                              uint8_t* __restrict__ dist, int32_t* __restrict__ pend, uint32_t* __restrict__ count,
                              unsigned long long* __restrict__ best, uint32_t* __restrict__ status,
                              uint64_t* __restrict__ fail) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nc = sp->n_cons;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const uint64_t c = cand[i];
        if (!in_domain(sp, c)) {   // the same in every lane
            if (lane == 0) {
                out[i] = c;
                if (dist) dist[i] = 255;
                atomicOr(status, ST_BAD_CANDIDATE);
            }
            continue;
        }
        const bool f0 = lane < nc && !cons_at(sp, tables, c, lane);
        const bool f1 = lane + 32 < nc && !cons_at(sp, tables, c, lane + 32);
        const uint64_t f = (uint64_t)__ballot_sync(0xffffffffu, f0) | ((uint64_t)__ballot_sync(0xffffffffu, f1) << 32);
        if (lane) continue;
        if (!f) {
            out[i] = c;
            if (dist) dist[i] = 0;
            continue;
        }
        if (fail) fail[i] = f;   // the constraints the ball search has to fix
        const uint32_t slot = atomicAdd(count, 1u);
        pend[slot] = (int32_t)i;
        best[slot] = NONE;
    }
}

// The table test and the small radii in one launch: a CTA per candidate (in turn) tests its
// constraints (a lane per constraint), then, while it is invalid, every point at distance
// d = 1 .. nr of it, the CTA's threads taking the points in turn (the radii's subset tables and a
// point -> subset map in shared memory).  A candidate settled at some radius gets the smallest
// valid key of that radius; the others are queued, with their failing constraints, for the
// launches of the larger radii.  It replaces the table-test launch and the first nr radius
// launches when those balls are small (whose launches cost more than their points).
constexpr int NEAR_MAX_R = 3;          // radii in one launch
constexpr int NEAR_MAX_POINTS = 4096;  // points of those radii together
constexpr int NEAR_MAX_SUBSETS = 512;  // subsets of those radii together
struct NearArgs {
    int nr;                                // radii 1 .. nr
    uint32_t total[NEAR_MAX_R];            // points at each radius
    int nsub[NEAR_MAX_R];
    const uint32_t* masks[NEAR_MAX_R];
    const uint64_t* prefix[NEAR_MAX_R];
};

__global__ void __launch_bounds__(256, 4)
k_ball_near(const DevSpace* __restrict__ sp, const uint32_t* __restrict__ tables, const __grid_constant__ NearArgs na,
            const uint64_t* __restrict__ cand, int64_t n, uint64_t* __restrict__ out, uint8_t* __restrict__ dist,
            int32_t* __restrict__ pend, uint32_t* __restrict__ count, unsigned long long* __restrict__ best,
            uint32_t* __restrict__ status, uint64_t* __restrict__ fail) {
    __shared__ uint16_t sub_of[NEAR_MAX_POINTS];   // point (radius-major) -> subset within its radius
    __shared__ uint32_t start_of[NEAR_MAX_SUBSETS], mask_of[NEAR_MAX_SUBSETS];
    __shared__ unsigned long long best_s;
    __shared__ uint64_t fail_s;
    const int t = threadIdx.x, lane = t & 31, nt = blockDim.x;
    {   // the radii's subset tables: per radius, subsets after point offsets pbase, subset offsets sbase
        uint32_t pbase = 0;
        int sbase = 0;
        for (int r = 0; r < na.nr; ++r) {
            for (int e = t; e < na.nsub[r]; e += nt) {
                const uint32_t a = (uint32_t)__ldg(na.prefix[r] + e), b = (uint32_t)__ldg(na.prefix[r] + e + 1);
                start_of[sbase + e] = a;
                mask_of[sbase + e] = __ldg(na.masks[r] + e);
                for (uint32_t j = a; j < b; ++j) sub_of[pbase + j] = (uint16_t)e;
            }
            pbase += na.total[r];
            sbase += na.nsub[r];
        }
    }
    __syncthreads();
    const int nc = sp->n_cons;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const uint64_t c = cand[i];
        if (!in_domain(sp, c)) {   // the same for every thread
            if (t == 0) {
                out[i] = c;
                if (dist) dist[i] = 255;
                atomicOr(status, ST_BAD_CANDIDATE);
            }
            continue;
        }
        if (t < 32) {
            const bool f0 = lane < nc && !cons_at(sp, tables, c, lane);
            const bool f1 = lane + 32 < nc && !cons_at(sp, tables, c, lane + 32);
            const uint64_t f = (uint64_t)__ballot_sync(0xffffffffu, f0) | ((uint64_t)__ballot_sync(0xffffffffu, f1) << 32);
            if (lane == 0) {
                fail_s = f;
                best_s = NONE;
            }
        }
        __syncthreads();
        const uint64_t f = fail_s;
        int found = 0;
        if (!f) {
            found = 1;
            if (t == 0) {
                out[i] = c;
                if (dist) dist[i] = 0;
            }
        }
        uint32_t pbase = 0;
        int sbase = 0;
        for (int r = 0; r < na.nr && !found; ++r) {
            for (uint32_t j = t; j < na.total[r]; j += nt) {
                const int sl = sub_of[pbase + j];
                const uint32_t S = mask_of[sbase + sl];
                if (!fixes_possible(sp, f, S)) continue;
                uint32_t local = j - start_of[sbase + sl];
                uint32_t m = S;
                uint64_t key = c;
                while (m) {
                    const int k = 31 - __clz(m);
                    m &= ~(1u << k);
                    uint32_t a;
                    local = div_alt(sp, k, local, &a);
                    const uint32_t uk = (uint32_t)field(sp, c, k);
                    key = (key & ~sp->fmask[k]) | ((uint64_t)(a < uk ? a : a + 1u) << sp->off[k]);
                }
                if (key < *(volatile unsigned long long*)&best_s && valid_changed(sp, tables, key, S))
                    atomicMin(&best_s, (unsigned long long)key);
            }
            __syncthreads();
            const unsigned long long b = best_s;
            __syncthreads();   // read by every thread before the next radius can lower it
            if (b != NONE) {
                found = 1;
                if (t == 0) {
                    out[i] = b;
                    if (dist) dist[i] = (uint8_t)(r + 1);
                }
            }
            pbase += na.total[r];
            sbase += na.nsub[r];
        }
        if (!found && t == 0) {   // for the larger radii
            if (fail) fail[i] = f;
            const uint32_t slot = atomicAdd(count, 1u);
            pend[slot] = (int32_t)i;
            best[slot] = NONE;
        }
        __syncthreads();   // fail_s and best_s are rewritten for the next candidate
    }
}

// The resolve step of one radius, run by the last CTA of the ball kernel to finish (an atomic
// ticket after a fence; nothing waits): candidates whose ball held a valid point are settled, the
// others are queued for the next radius.
__device__ __forceinline__ void ball_resolve_last(const BallNext& nx, const int32_t* __restrict__ pend_in,
                                                  const uint32_t* __restrict__ count_in,
                                                  const unsigned long long* __restrict__ best_in) {
    if (!nx.done) return;
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();   // this CTA's atomics on best_in before its ticket
        last = atomicAdd(nx.done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) *nx.count_out = 0;
    __syncthreads();
    const uint32_t cnt = *count_in;
    for (uint32_t q = threadIdx.x; q < cnt; q += blockDim.x) {
        const unsigned long long b = __ldcg(best_in + q);
        const int32_t i = pend_in[q];
        if (b != NONE) {
            nx.out[i] = b;
            if (nx.dist) nx.dist[i] = (uint8_t)nx.d;
        } else {
            const uint32_t slot = atomicAdd(nx.count_out, 1u);
            nx.pend_out[slot] = i;
            nx.best_out[slot] = NONE;
        }
    }
    if (threadIdx.x == 0) *nx.done = 0;   // for the next launch
}

constexpr int BALL_SMEM_SUBSETS = 2048;   // subsets whose table k_ball stages in shared memory

// every point at Hamming distance exactly d of each pending candidate; with the candidates'
// failing-constraint masks, subsets that cannot fix them are skipped and only the constraints
// reading a changed parameter are tested
__global__ void __launch_bounds__(256)
k_ball(const DevSpace* __restrict__ sp, const uint32_t* __restrict__ tables, const uint32_t* __restrict__ masks,
       const uint64_t* __restrict__ prefix, int n_subsets, uint64_t points, const uint64_t* __restrict__ cand,
       const int32_t* __restrict__ pend, const uint32_t* __restrict__ count, unsigned long long* __restrict__ best,
       const uint64_t* __restrict__ fail, const BallNext nx, uint32_t cmax) {
    if (*count > cmax) return;   // this radius is k_ball_fs's (many pending candidates): no work, no resolve
    // the radius's subset table in shared memory when it fits: the per-point subset search then
    // waits for shared memory instead of a chain of L1/L2 reads
    __shared__ uint64_t pre_s[BALL_SMEM_SUBSETS];
    __shared__ uint32_t msk_s[BALL_SMEM_SUBSETS];
    const bool staged = n_subsets <= BALL_SMEM_SUBSETS;
    if (staged) {
        for (int e = threadIdx.x; e < n_subsets; e += blockDim.x) {
            pre_s[e] = __ldg(prefix + e);
            msk_s[e] = __ldg(masks + e);
        }
        __syncthreads();
    }
    const uint64_t* pre = staged ? pre_s : prefix;
    const uint32_t* msk = staged ? msk_s : masks;
    const uint64_t total = (uint64_t)(*count) * points;
    const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t g0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t dq = G / points, dj = G - dq * points;
    // Subsets of at least 16 points on average: a warp's 32 consecutive points span few subsets,
    // so lane 0 searches its subset and the other lanes step forward from it (the warp stays
    // together: its lanes run the loop while lane 0 has a point).
    const bool coop = points >= 16ull * (uint64_t)n_subsets;
    const int lane = threadIdx.x & 31;
    uint64_t q = g0 / points, j = g0 - q * points;   // (g / points, g % points), stepped with g
    for (uint64_t g = g0; coop ? g - lane < total : g < total; g += G, q += dq, j += dj) {
        if (j >= points) { j -= points; ++q; }
        const bool act = g < total;
        int lo = 0;
        if (coop) {
            int hi = n_subsets - 1;   // lane 0: last subset with prefix <= j
            if (lane == 0) {
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (pre[mid] <= j) lo = mid; else hi = mid - 1;
                }
            }
            const int lo0 = __shfl_sync(0xffffffffu, lo, 0);
            const uint64_t q0 = __shfl_sync(0xffffffffu, q, 0), j0 = __shfl_sync(0xffffffffu, j, 0);
            if (act && q == q0 && j >= j0) {
                lo = lo0;
                while (lo + 1 < n_subsets && pre[lo + 1] <= j) ++lo;
            } else if (act) {
                lo = 0;
                hi = n_subsets - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (pre[mid] <= j) lo = mid; else hi = mid - 1;
                }
            }
            if (!act) continue;
        } else {
            int hi = n_subsets - 1;   // last subset with prefix <= j
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (pre[mid] <= j) lo = mid; else hi = mid - 1;
            }
        }
        const uint64_t u = __ldg(cand + pend[q]);
        const uint32_t S = msk[lo];
        if (fail && !fixes_possible(sp, __ldg(fail + pend[q]), S)) continue;
        uint32_t local = (uint32_t)(j - pre[lo]);
        uint32_t m = S;
        uint64_t key = u;
        while (m) {
            const int k = 31 - __clz(m);
            m &= ~(1u << k);
            uint32_t a;
            local = div_alt(sp, k, local, &a);
            const uint32_t uk = (uint32_t)field(sp, u, k);
            const uint32_t v = a < uk ? a : a + 1u;
            key = (key & ~sp->fmask[k]) | ((uint64_t)v << sp->off[k]);
        }
        // the atomic only when the key beats the candidate's current best (read from L2): a
        // high-radius ball can hold 10^5 valid points of one candidate
        if (key < __ldcg(best + q) && (fail ? valid_changed(sp, tables, key, S) : valid_key(sp, tables, key)))
            atomicMin(best + q, (unsigned long long)key);
    }
    ball_resolve_last(nx, pend, count, best);
}

// Radii whose subsets hold at least this many points on average take the filtered search (a warp
// per (candidate, subset) pays for its plan only on large subsets; smaller ones keep a thread per
// point).  On the large space that is radius 5 and above.
constexpr uint64_t BALL_FS_MIN_AVG = 512;
// Radii whose subsets average between BALL_DUAL_MIN_AVG and BALL_FS_MIN_AVG points take the
// filtered search when at least BALL_DUAL_MIN_PENDING candidates are pending, the per-point search
// otherwise (radius 4 of the large space: 256 uniform candidates, 157 pending, 1.19 -> 0.99 ms per
// repair with the filtered search; 256 perturbed ones, 17 pending, 0.128 -> 0.156 ms).
constexpr uint64_t BALL_DUAL_MIN_AVG = 128;
constexpr uint32_t BALL_DUAL_MIN_PENDING = 64;

// The ball search with single-parameter filtering: a warp per (pending candidate, subset); the
// lanes take the subset's allowed points 32 at a time, test the constraints the masks do not
// settle, and the warp minimum goes to the candidate's best with at most one atomicMin.
__global__ void __launch_bounds__(256)
k_ball_fs(const DevSpace* __restrict__ sp, const uint32_t* __restrict__ tables, const uint32_t* __restrict__ masks,
          int n_subsets, const uint64_t* __restrict__ cand, const int32_t* __restrict__ pend,
          const uint32_t* __restrict__ count, unsigned long long* __restrict__ best, const uint64_t* __restrict__ fail,
          const BallNext nx, uint32_t cmin) {
    if (*count < cmin) return;   // this radius is k_ball's (few pending candidates): no work, no resolve
    const uint64_t total = (uint64_t)(*count) * (uint64_t)n_subsets;
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nwarps) {
        const uint64_t q = w / (uint64_t)n_subsets;
        const int si = (int)(w - q * (uint64_t)n_subsets);
        const int32_t i = pend[q];
        const uint32_t S = __ldg(masks + si);
        if (!fixes_possible(sp, __ldg(fail + i), S)) continue;   // the same in every lane
        const uint64_t u = __ldg(cand + i);
        BallPlan bp;
        const uint64_t size = ball_plan_warp(sp, tables, u, S, lane, bp);
        unsigned long long bl = ~0ull;
        for (uint64_t idx = (uint64_t)lane; idx < size; idx += 32) {
            const uint64_t key = ball_point(sp, u, bp, idx);
            if (key < bl && valid_rest(sp, tables, key, bp.rest)) bl = key;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, bl, o);
            bl = y < bl ? y : bl;
        }
        if (lane == 0 && bl != ~0ull && bl < __ldcg(best + q)) atomicMin(best + q, bl);
    }
    ball_resolve_last(nx, pend, count, best);
}

// Exhaustive streaming argmin of (distance, rank) for up to 32 candidates per CTA.
// Each thread reads two keys per 16-byte load and keeps, per candidate, the packed
// minimum (distance << 26 | iteration << 1 | which); keys ascend within a thread, so
// the smallest packed value is the smallest distance and, among equal distances, the
// smallest key.  The inner loop is instantiated for the number of pending candidates
// (1, 2, 4, 8, 16, 32), on 32-bit words when every field lies in the low 32 bits.
template <int Q, bool NARROW>
__device__ __forceinline__ void scan_run(const uint64_t* __restrict__ keys, int64_t nv, uint64_t lowm, uint64_t highm,
                                         const uint64_t* cq, int nq, unsigned long long* __restrict__ best,
                                         unsigned long long (*red)[SCAN_CHUNK]) {
    uint64_t c[Q];
    uint32_t b[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) { c[q] = cq[q < nq ? q : 0]; b[q] = 0xFFFFFFFFu; }
    const int64_t stride = (int64_t)gridDim.x * SCAN_THREADS * 2;
    const int64_t start = ((int64_t)blockIdx.x * SCAN_THREADS + threadIdx.x) * 2;
    const uint32_t lo32 = (uint32_t)lowm, hi32 = (uint32_t)highm;
    uint32_t it = 0;
    int64_t i = start;
    for (; i + 1 < nv; i += stride, ++it) {
        const ulonglong2 kk = __ldg(reinterpret_cast<const ulonglong2*>(keys + i));
        const uint32_t tag = it << 1;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            uint32_t d0, d1;
            if (NARROW) {
                const uint32_t x0 = (uint32_t)kk.x ^ (uint32_t)c[q], x1 = (uint32_t)kk.y ^ (uint32_t)c[q];
                d0 = __popc((((x0 & lo32) + lo32) | x0) & hi32);
                d1 = __popc((((x1 & lo32) + lo32) | x1) & hi32);
            } else {
                d0 = hamming_keys(kk.x, c[q], lowm, highm);
                d1 = hamming_keys(kk.y, c[q], lowm, highm);
            }
            const uint32_t p0 = (d0 << 26) | tag, p1 = (d1 << 26) | tag | 1u;
            b[q] = min(b[q], min(p0, p1));
        }
    }
    if (i < nv) {   // last key when nv is odd
        const uint64_t k = __ldg(keys + i);
#pragma unroll
        for (int q = 0; q < Q; ++q) b[q] = min(b[q], ((uint32_t)hamming_keys(k, c[q], lowm, highm) << 26) | (it << 1));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        unsigned long long v = ~0ull;
        if (b[q] != 0xFFFFFFFFu) {
            const uint32_t t = b[q] & ((1u << 26) - 1);
            const int64_t idx = start + (int64_t)(t >> 1) * stride + (t & 1u);
            v = ((unsigned long long)(b[q] >> 26) << 57) | (unsigned long long)idx;
        }
        for (int o = 16; o; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
            v = w < v ? w : v;
        }
        if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < nq) {
        unsigned long long v = ~0ull;
        for (int w = 0; w < SCAN_THREADS / 32; ++w) v = red[w][threadIdx.x] < v ? red[w][threadIdx.x] : v;
        atomicMin(best + threadIdx.x, v);
    }
}

// The resolve step of the exhaustive scan, run by the last CTA of the last scan kernel to finish
// (an atomic ticket after a fence; nothing waits): each pending candidate takes the key of its
// packed (distance << 57 | rank) minimum.  done = null: k_scan_resolve does it instead (many
// pending candidates, which one CTA would resolve slowly).
struct ScanNext {
    uint32_t* done;                 // CTAs finished (zero before the launch; the last CTA resets it)
    const uint64_t* keys;
    uint64_t* out;
    uint8_t* dist;
};

__device__ __forceinline__ void scan_resolve_last(const ScanNext& nx, const int32_t* __restrict__ pend,
                                                  const uint32_t* __restrict__ count,
                                                  const unsigned long long* __restrict__ best) {
    if (!nx.done) return;
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();   // this CTA's atomics on best before its ticket
        last = atomicAdd(nx.done, 1u) == gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const uint32_t cnt = *count;
    for (uint32_t q = threadIdx.x; q < cnt; q += blockDim.x) {
        const unsigned long long b = __ldcg(best + q);
        const int32_t i = pend[q];
        nx.out[i] = __ldg(nx.keys + (b & ((1ull << 57) - 1)));
        if (nx.dist) nx.dist[i] = (uint8_t)(b >> 57);
    }
    if (threadIdx.x == 0) *nx.done = 0;   // for the next launch
}

// Few pending candidates (<= few_max, at most 4): one candidate set per CTA, high
// occupancy, four independent 16-byte key loads in flight per thread.  A last chunk
// with more candidates is left to k_scan_wide or to the distance-table scan.
template <int Q, bool NARROW>
__device__ __forceinline__ void scan_run4(const uint64_t* __restrict__ keys, int64_t nv, uint64_t lowm,
                                          uint64_t highm, const uint64_t* cq, int nq,
                                          unsigned long long* __restrict__ best, unsigned long long (*red)[SCAN_CHUNK]) {
    constexpr int U = 4;
    uint64_t c[Q];
    uint32_t b[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) { c[q] = cq[q < nq ? q : 0]; b[q] = 0xFFFFFFFFu; }
    const int64_t stride = (int64_t)gridDim.x * SCAN_THREADS * 2;
    const int64_t start = ((int64_t)blockIdx.x * SCAN_THREADS + threadIdx.x) * 2;
    const uint32_t lo32 = (uint32_t)lowm, hi32 = (uint32_t)highm;
    uint32_t it = 0;
    int64_t i = start;
    for (; i + (U - 1) * stride + 1 < nv; i += U * stride, it += U) {
        ulonglong2 kk[U];
#pragma unroll
        for (int u = 0; u < U; ++u) kk[u] = __ldg(reinterpret_cast<const ulonglong2*>(keys + i + u * stride));
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t tag = (it + u) << 1;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                uint32_t d0, d1;
                if (NARROW) {
                    const uint32_t x0 = (uint32_t)kk[u].x ^ (uint32_t)c[q], x1 = (uint32_t)kk[u].y ^ (uint32_t)c[q];
                    d0 = __popc((((x0 & lo32) + lo32) | x0) & hi32);
                    d1 = __popc((((x1 & lo32) + lo32) | x1) & hi32);
                } else {
                    d0 = hamming_keys(kk[u].x, c[q], lowm, highm);
                    d1 = hamming_keys(kk[u].y, c[q], lowm, highm);
                }
                b[q] = min(b[q], min((d0 << 26) | tag, (d1 << 26) | tag | 1u));
            }
        }
    }
    for (; i < nv; i += stride, ++it) {   // remainder, one pair (or the odd last key) at a time
#pragma unroll
        for (int w = 0; w < 2; ++w) {
            if (i + w >= nv) break;
            const uint64_t k = __ldg(keys + i + w);
#pragma unroll
            for (int q = 0; q < Q; ++q)
                b[q] = min(b[q], ((uint32_t)hamming_keys(k, c[q], lowm, highm) << 26) | (it << 1) | (uint32_t)w);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        unsigned long long v = ~0ull;
        if (b[q] != 0xFFFFFFFFu) {
            const uint32_t t = b[q] & ((1u << 26) - 1);
            const int64_t idx = start + (int64_t)(t >> 1) * stride + (t & 1u);
            v = ((unsigned long long)(b[q] >> 26) << 57) | (unsigned long long)idx;
        }
        for (int o = 16; o; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
            v = w < v ? w : v;
        }
        if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < nq) {
        unsigned long long v = ~0ull;
        for (int w = 0; w < SCAN_THREADS / 32; ++w) v = red[w][threadIdx.x] < v ? red[w][threadIdx.x] : v;
        atomicMin(best + threadIdx.x, v);
    }
}

// The last chunk of pending candidates, when it holds at most four (every other
// chunk is full).  One wave of CTAs; each scans its slice of the keys.
__global__ void __launch_bounds__(SCAN_THREADS, 4)
k_scan_few(const uint64_t* __restrict__ keys, int64_t nv, uint64_t lowm, uint64_t highm,
           const uint64_t* __restrict__ cand, const int32_t* __restrict__ pend, const uint32_t* __restrict__ count,
           unsigned long long* __restrict__ best, int few_max, const ScanNext nx) {
    __shared__ uint64_t cq[SCAN_CHUNK];
    __shared__ unsigned long long red[SCAN_THREADS / 32][SCAN_CHUNK];
    const uint32_t cnt = *count;
    const uint32_t q0 = cnt ? (cnt - 1) / SCAN_CHUNK * SCAN_CHUNK : 0;
    const int nq = (int)(cnt - q0);
    if (cnt && nq <= few_max && nq <= 4) {
        if (threadIdx.x < SCAN_CHUNK) cq[threadIdx.x] = threadIdx.x < nq ? cand[pend[q0 + threadIdx.x]] : 0ull;
        __syncthreads();
        unsigned long long* bq = best + q0;
        if ((highm >> 32) == 0) {
            if (nq <= 1) scan_run4<1, true>(keys, nv, lowm, highm, cq, nq, bq, red);
            else if (nq <= 2) scan_run4<2, true>(keys, nv, lowm, highm, cq, nq, bq, red);
            else scan_run4<4, true>(keys, nv, lowm, highm, cq, nq, bq, red);
        } else {
            if (nq <= 1) scan_run4<1, false>(keys, nv, lowm, highm, cq, nq, bq, red);
            else if (nq <= 2) scan_run4<2, false>(keys, nv, lowm, highm, cq, nq, bq, red);
            else scan_run4<4, false>(keys, nv, lowm, highm, cq, nq, bq, red);
        }
    }
    scan_resolve_last(nx, pend, count, best);
}

// Every chunk with more than four pending candidates.  One wave of CTAs; each CTA
// scans its slice of the keys once per chunk.
__global__ void __launch_bounds__(SCAN_THREADS)
k_scan_wide(const uint64_t* __restrict__ keys, int64_t nv, uint64_t lowm, uint64_t highm,
            const uint64_t* __restrict__ cand, const int32_t* __restrict__ pend, const uint32_t* __restrict__ count,
            unsigned long long* __restrict__ best, const ScanNext nx) {
    __shared__ uint64_t cq[SCAN_CHUNK];
    __shared__ unsigned long long red[SCAN_THREADS / 32][SCAN_CHUNK];
    const uint32_t cnt = *count;
    for (uint32_t q0 = 0; q0 < cnt; q0 += SCAN_CHUNK) {
        const int nq = (int)min((uint32_t)SCAN_CHUNK, cnt - q0);
        if (nq <= 4) break;                       // only the last chunk can be that small
        __syncthreads();                          // previous chunk done with cq / red
        if (threadIdx.x < SCAN_CHUNK) cq[threadIdx.x] = threadIdx.x < nq ? cand[pend[q0 + threadIdx.x]] : 0ull;
        __syncthreads();
        unsigned long long* bq = best + q0;
        if ((highm >> 32) == 0) {
            if (nq <= 8) scan_run<8, true>(keys, nv, lowm, highm, cq, nq, bq, red);
            else if (nq <= 16) scan_run<16, true>(keys, nv, lowm, highm, cq, nq, bq, red);
            else scan_run<32, true>(keys, nv, lowm, highm, cq, nq, bq, red);
        } else {
            if (nq <= 8) scan_run<8, false>(keys, nv, lowm, highm, cq, nq, bq, red);
            else if (nq <= 16) scan_run<16, false>(keys, nv, lowm, highm, cq, nq, bq, red);
            else scan_run<32, false>(keys, nv, lowm, highm, cq, nq, bq, red);
        }
    }
    scan_resolve_last(nx, pend, count, best);
}

__global__ void k_scan_resolve(const uint64_t* __restrict__ keys, const int32_t* __restrict__ pend,
                               const uint32_t* __restrict__ count, const unsigned long long* __restrict__ best,
                               uint64_t* __restrict__ out, uint8_t* __restrict__ dist) {
    const uint32_t cnt = *count;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += gridDim.x * blockDim.x) {
        const unsigned long long b = best[q];
        const int32_t i = pend[q];
        out[i] = keys[b & ((1ull << 57) - 1)];
        if (dist) dist[i] = (uint8_t)(b >> 57);
    }
}

static int g_sm_count = 0;
static int sm_count() {
    if (!g_sm_count) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (g_sm_count <= 0) g_sm_count = 148;
    }
    return g_sm_count;
}

// Largest radius whose cumulative ball is cheaper than one scan pass per candidate:
// a ball point costs a table test (~8x a scanned key's SWAR distance).
int auto_radius(const ct_space* s, double div) {
    const double budget = (double)s->n_valid / div;
    double cum = 0;
    int d = 0;
    for (int r = 1; r <= s->ball_max; ++r) {
        cum += (double)s->ball_total[r];
        if (cum > budget) break;
        d = r;
    }
    return d;
}

ct_status repair_reserve(RepairScratch& rs, int64_t n) {
    if (!rs.done.p) {   // the ball kernels' ticket counter: zero between launches
        CT_TRY(rs.done.ensure(1));
        CT_TRY_CUDA(cudaMemset(rs.done.p, 0, sizeof(uint32_t)));
    }
    CT_TRY(rs.pend_a.ensure(n));
    CT_TRY(rs.pend_b.ensure(n));
    CT_TRY(rs.counts.ensure(2));
    CT_TRY(rs.best.ensure(2 * (size_t)n));
    CT_TRY(rs.fail.ensure(n));
    return CT_OK;
}

ct_status repair_launch(const ct_space* s, const RepairPtrs& p, int dmax, const uint64_t* d_cand, int64_t n,
                        uint64_t* d_out, uint8_t* d_dist, cudaStream_t st) {
    const int sms = sm_count();
    const unsigned g1 = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
    // the radii whose balls are small together go with the table test into one launch
    NearArgs na{};
    {
        uint64_t near_points = NEAR_MAX_POINTS;   // CATUNE_BALL_NEAR_POINTS lowers it (0: off; tests)
        if (const char* env = getenv("CATUNE_BALL_NEAR_POINTS"))
            near_points = std::min<uint64_t>(near_points, strtoull(env, nullptr, 10));
        uint64_t pts = 0;
        int subs = 0;
        for (int d = 1; d <= std::min(dmax, NEAR_MAX_R) && d <= (int)s->balls.size(); ++d) {
            const BallRadius& br = s->balls[d - 1];
            if (!br.d_masks.p || !br.d_prefix.p || pts + br.total > near_points ||
                subs + (int)br.masks.size() > NEAR_MAX_SUBSETS)
                break;
            na.total[na.nr] = (uint32_t)br.total;
            na.nsub[na.nr] = (int)br.masks.size();
            na.masks[na.nr] = br.d_masks.p;
            na.prefix[na.nr] = br.d_prefix.p;
            ++na.nr;
            pts += br.total;
            subs += (int)br.masks.size();
        }
    }
    if (na.nr > 0) {
        const unsigned gn = (unsigned)std::min<int64_t>(n, (int64_t)sms * 8);   // a CTA per candidate in turn
        k_ball_near<<<gn, 256, 0, st>>>(s->d, s->tables.p, na, d_cand, n, d_out, d_dist, p.pend[0], p.cnt[0],
                                        p.best[0], s->status.p, p.fail);
    } else {
        const unsigned gi = (unsigned)std::min<int64_t>((n * 32 + 255) / 256, (int64_t)sms * 8);   // a warp per candidate
        k_repair_init<<<gi, 256, 0, st>>>(s->d, s->tables.p, d_cand, n, d_out, d_dist, p.pend[0], p.cnt[0], p.best[0],
                                          s->status.p, p.fail);
    }
    count_launch();
    uint64_t fs_min_avg = BALL_FS_MIN_AVG;   // CATUNE_BALL_FS_MIN_AVG overrides it (tests)
    if (const char* env = getenv("CATUNE_BALL_FS_MIN_AVG")) fs_min_avg = strtoull(env, nullptr, 10);
    const uint64_t dual_min_avg = std::min<uint64_t>(fs_min_avg, BALL_DUAL_MIN_AVG);
    int cur = 0;
    for (int d = na.nr + 1; d <= dmax; ++d) {
        const BallRadius& br = s->balls[d - 1];
        // the kernel's last CTA resolves this radius: settles, and queues the rest for the next
        const BallNext nx{p.done, d, d_out, d_dist, p.pend[cur ^ 1], p.cnt[cur ^ 1], p.best[cur ^ 1]};
        const uint64_t fs_work = (uint64_t)n * br.masks.size() * 32;
        // one wave each: k_ball_fs holds 2 CTAs of 256 per SM (128 registers), k_ball 5 (48); on the
        // large space that took the repair of 256 perturbed candidates from 0.105 to 0.098 ms (the
        // empty launches of the dual radii are cheaper) and 256 uniform ones from 0.945 to 0.965
        const unsigned gfs = (unsigned)std::min<uint64_t>((fs_work + 255) / 256, (uint64_t)sms * 2);
        const uint64_t pt_work = (uint64_t)n * br.total;
        const unsigned gpt = (unsigned)std::min<uint64_t>((pt_work + 255) / 256, (uint64_t)sms * 5);
        if (br.total >= fs_min_avg * br.masks.size()) {
            // large subsets: a warp per (candidate, subset) over the filtered points
            k_ball_fs<<<gfs, 256, 0, st>>>(s->d, s->tables.p, br.d_masks.p, (int)br.masks.size(), d_cand, p.pend[cur],
                                           p.cnt[cur], p.best[cur], p.fail, nx, 0u);
        } else if (br.total >= dual_min_avg * br.masks.size()) {
            // mid-sized subsets: a thread per point while few candidates are pending, the filtered
            // search from BALL_DUAL_MIN_PENDING on; both are launched and the other one returns
            k_ball<<<gpt, 256, 0, st>>>(s->d, s->tables.p, br.d_masks.p, br.d_prefix.p, (int)br.masks.size(), br.total,
                                        d_cand, p.pend[cur], p.cnt[cur], p.best[cur], p.fail, nx,
                                        BALL_DUAL_MIN_PENDING - 1u);
            k_ball_fs<<<gfs, 256, 0, st>>>(s->d, s->tables.p, br.d_masks.p, (int)br.masks.size(), d_cand, p.pend[cur],
                                           p.cnt[cur], p.best[cur], p.fail, nx, BALL_DUAL_MIN_PENDING);
            count_launch();
        } else {
            // small subsets: a thread per point
            k_ball<<<gpt, 256, 0, st>>>(s->d, s->tables.p, br.d_masks.p, br.d_prefix.p, (int)br.masks.size(), br.total,
                                        d_cand, p.pend[cur], p.cnt[cur], p.best[cur], p.fail, nx, ~0u);
        }
        count_launch();
        cur ^= 1;
    }
    // whatever is left: exhaustive scan (a full ball search always ends here as well)
    // one wave each: 4 resident CTAs per SM for the few-candidate scan, 2 for the wide one
    const int64_t need = ((int64_t)s->n_valid + SCAN_THREADS * 8 - 1) / (SCAN_THREADS * 8);
    const unsigned gf = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * 4));
    const unsigned gw = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * 2));
    bool lut = false;   // long key arrays: per-candidate distance tables
    int lut_min = 0;
    CT_TRY(scan_lut(s, d_cand, p.pend[cur], p.cnt[cur], p.best[cur], st, &lut, &lut_min));
    // the last scan kernel's last CTA resolves, unless many candidates could be pending
    const bool fold = n <= SCAN_FOLD_MAX;
    const ScanNext nx = fold ? ScanNext{p.done, s->keys.p, d_out, d_dist} : ScanNext{};
    k_scan_few<<<gf, SCAN_THREADS, 0, st>>>(s->keys.p, (int64_t)s->n_valid, s->h.swar_low, s->h.swar_high, d_cand,
                                            p.pend[cur], p.cnt[cur], p.best[cur], lut ? lut_min - 1 : 4,
                                            lut ? nx : ScanNext{});
    count_launch();
    if (!lut) {
        k_scan_wide<<<gw, SCAN_THREADS, 0, st>>>(s->keys.p, (int64_t)s->n_valid, s->h.swar_low, s->h.swar_high,
                                                 d_cand, p.pend[cur], p.cnt[cur], p.best[cur], nx);
        count_launch();
    }
    if (!fold) {
        k_scan_resolve<<<g1, 256, 0, st>>>(s->keys.p, p.pend[cur], p.cnt[cur], p.best[cur], d_out, d_dist);
        count_launch();
    }
    CT_TRY_CUDA(cudaGetLastError());
    return CT_OK;
}

ct_status repair_impl(ct_space* s, RepairScratch& rs, const uint64_t* d_cand, int64_t n, uint64_t* d_out,
                      uint8_t* d_dist, cudaStream_t st) {
    if (n == 0) return CT_OK;
    if (n > 0x7fffffffLL) { set_error("n too large"); return CT_ERR_LIMIT; }
    CT_TRY(repair_reserve(rs, n));
    const int dmax = wanted_radius(s);
    CT_TRY(ensure_balls(s, dmax));   // normally planned already (after the build, at run creation)
    CT_TRY_CUDA(cudaMemsetAsync(rs.counts.p, 0, 8, st));
    const RepairPtrs p{{rs.pend_a.p, rs.pend_b.p}, {rs.counts.p, rs.counts.p + 1}, {rs.best.p, rs.best.p + n},
                       rs.fail.p, rs.done.p};
    return repair_launch(s, p, dmax, d_cand, n, d_out, d_dist, st);
}

}  // namespace ct

using namespace ct;

extern "C" {

ct_status ct_lookup(const ct_space* s, const uint64_t* d_cand, int64_t n, int64_t* d_rank, ct_stream stream) {
    if (!s || n < 0 || (n > 0 && (!d_cand || !d_rank))) { set_error("bad argument"); return CT_ERR_INVALID_ARG; }
    if (!s->built) { set_error("space not built"); return CT_ERR_STATE; }
    if (n == 0) return CT_OK;
    const unsigned g = (unsigned)std::min<int64_t>((n * 32 + 255) / 256, (int64_t)sm_count() * 8);   // a warp per key
    k_lookup<<<g, 256, 0, (cudaStream_t)stream>>>(s->d, s->keys.p, (int64_t)s->n_valid, d_cand, n, d_rank);
    count_launch();
    CT_TRY_CUDA(cudaGetLastError());
    return CT_OK;
}

ct_status ct_repair(ct_space* s, const uint64_t* d_cand, int64_t n, uint64_t* d_out, uint8_t* d_dist, ct_stream stream) {
    if (!s || n < 0 || (n > 0 && (!d_cand || !d_out))) { set_error("bad argument"); return CT_ERR_INVALID_ARG; }
    if (!s->built) { set_error("space not built"); return CT_ERR_STATE; }
    if (s->n_valid == 0) { set_error("empty valid space"); return CT_ERR_EMPTY_SPACE; }
    return repair_impl(s, s->rs, d_cand, n, d_out, d_dist, (cudaStream_t)stream);
}

ct_status ct_set_repair_mode(ct_space* s, int32_t mode, int32_t max_radius) {
    if (!s || mode < 0 || mode > 2 || max_radius < 0) { set_error("bad argument"); return CT_ERR_INVALID_ARG; }
    s->repair_mode = mode;
    s->repair_max_radius = max_radius;
    if (s->built && s->n_valid) return ensure_balls(s, wanted_radius(s));
    return CT_OK;
}

}  // extern "C"

namespace ct {
ct_status evaluate_impl(ct_space* s, uint32_t* memo, unsigned long long* unique, unsigned long long* cost_acc,
                        const uint64_t* d_keys, int64_t n, float* d_fit, int64_t* d_rank, cudaStream_t st,
                        float invalid_fit) {
    if (n == 0) return CT_OK;
    const unsigned g = (unsigned)std::min<int64_t>((n * 32 + 255) / 256, (int64_t)sm_count() * 8);   // a warp per key
    k_evaluate<<<g, 256, 0, st>>>(s->d, s->keys.p, (int64_t)s->n_valid, s->fit, d_keys, n, d_fit, d_rank, memo, unique,
                                  memo && cost_acc ? s->cost : nullptr, cost_acc, invalid_fit);
    count_launch();
    CT_TRY_CUDA(cudaGetLastError());
    return CT_OK;
}
}  // namespace ct
