// Exhaustive repair scan with per-candidate distance tables (long key arrays).
//
// The streaming pass of the exact Hamming repair (the nearest valid configuration under the
// Hamming neighbour rule of Section IV-A, ties to the smallest key) reads every valid key once per
// chunk of 32 pending candidates.  Instead of a SWAR distance per (key, candidate), the key's
// fields are split into groups of adjacent fields of at most 8 bits; for every group value the CTA
// tabulates, in shared memory, how many of the group's fields differ from each candidate.  Eight
// candidates share one 64-bit table entry (one 8-bit lane each), so the distances of a key to
// eight candidates are the lane-wise sum of one table entry per group.  A SWAR borrow test on the
// lanes finds the rare keys that improve some candidate; only those take the per-lane update.
//
// Per key: one extract per group (shared by all candidate sets) and one table read and add per
// group and set of eight candidates.  Ties: a thread visits its keys in increasing order and keeps
// strict improvements, and the packed (distance << 57 | rank) minimum across threads and CTAs
// keeps the smallest rank among the nearest keys, as the exact definition requires.
#include <cuda_runtime.h>

#include <cstdlib>
#include <mutex>

#include "internal.hpp"

namespace ct {

constexpr int SL_THREADS = 256;
constexpr int SL_CHUNK = 32;                    // candidates per pass: up to four sets of eight
constexpr int SL_MAX_GROUPS = 8;
constexpr int64_t SL_MIN_KEYS = 1ll << 22;      // shorter arrays keep the SWAR scan
constexpr int SL_LUT_MIN = 3;                   // a last chunk of 1 or 2 candidates keeps the SWAR scan
constexpr uint32_t SL_H32 = 0x80808080u;       // bit 7 of every lane
constexpr uint32_t SL_B32 = 0x7F7F7F7Fu;       // lane state = 127 + best distance

struct ScanLutPlan {
    int ng;                            // groups; group g owns table entries [256 g, 256 g + 256)
    int shift[SL_MAX_GROUPS];          // lowest key bit of the group
    uint32_t mask[SL_MAX_GROUPS];      // (1 << group width) - 1
    int k0[SL_MAX_GROUPS], k1[SL_MAX_GROUPS];   // parameters k0..k1 form the group
};

// Groups of adjacent parameters (lowest key bits first) with at most 8 key bits each; false when a
// parameter is wider than 8 bits, more than eight groups are needed, the key is wider than 59 bits
// (the table offsets are cut from the key shifted left by 5) or the key array is short.
static bool scan_lut_plan(const ct_space* s, ScanLutPlan& pl) {
    int64_t min_keys = SL_MIN_KEYS;   // CATUNE_SCAN_LUT_MIN_KEYS overrides it (tests)
    if (const char* env = getenv("CATUNE_SCAN_LUT_MIN_KEYS")) min_keys = strtoll(env, nullptr, 10);
    if ((int64_t)s->n_valid < min_keys) return false;
    const DevSpace& h = s->h;
    if (h.key_bits > 59) return false;
    pl.ng = 0;
    int k = h.n - 1;                   // the last parameter holds the lowest bits
    while (k >= 0 && h.w[k] == 0) --k;
    while (k >= 0) {
        if (pl.ng == SL_MAX_GROUPS || h.w[k] > 8) return false;
        const int g = pl.ng++;
        pl.k1[g] = k;
        pl.shift[g] = h.off[k];
        int width = h.w[k];
        --k;
        while (k >= 0 && width + h.w[k] <= 8) width += h.w[k--];
        pl.k0[g] = k + 1;
        pl.mask[g] = (1u << width) - 1u;
        while (k >= 0 && h.w[k] == 0) --k;
    }
    return pl.ng > 0;
}

// Tables of one chunk: entry 256 g + x, lane l of set s = number of group g's fields in which the
// group value x differs from candidate 8 s + l (0 for lanes past the chunk).  Stored as [entry][S].
__device__ void sl_tables(const DevSpace* __restrict__ sp, const ScanLutPlan& pl, const uint64_t* cq, int nq,
                          int S, unsigned long long* tab) {
    for (int e = threadIdx.x; e < 256 * pl.ng; e += SL_THREADS) {
        const int g = e >> 8;
        const uint32_t x = (uint32_t)e & 255u;
        if (x > pl.mask[g]) continue;   // never read
        const uint64_t local = (uint64_t)x << pl.shift[g];
        for (int s = 0; s < S; ++s) {
            unsigned long long word = 0;
            for (int l = 0; l < 8; ++l) {
                const int q = 8 * s + l;
                if (q >= nq) break;
                const uint64_t d = local ^ cq[q];
                uint32_t nd = 0;
                for (int k = pl.k0[g]; k <= pl.k1[g]; ++k) nd += (d & sp->fmask[k]) != 0;
                word |= (unsigned long long)nd << (8 * l);
            }
            tab[(size_t)e * S + s] = word;
        }
    }
}

// Lane states and best tags of one set of eight candidates, as two 32-bit halves: the lanes never
// carry or borrow into each other, so the halves are summed and tested independently.
template <int NG, int S>
__device__ __forceinline__ void sl_visit(uint64_t key, uint32_t tag, const uint32_t (&rs)[NG],
                                         const uint32_t (&mk)[NG], const char* __restrict__ tab, uint32_t (&vl)[S],
                                         uint32_t (&vh)[S], uint32_t* __restrict__ tg) {
    const uint64_t kx = key << 5;
    uint32_t a[NG];   // byte offset of the group's entry: (256 g + x) * 8 S
#pragma unroll
    for (int g = 0; g < NG; ++g) a[g] = ((uint32_t)(kx >> rs[g]) & mk[g]) | ((uint32_t)g << (11 + (S == 1 ? 0 : S == 2 ? 1 : 2)));
    uint32_t dl[S], dh[S];
#pragma unroll
    for (int s = 0; s < S; ++s) dl[s] = dh[s] = 0;
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        if (S == 1) {
            const uint2 w = *reinterpret_cast<const uint2*>(tab + a[g]);
            dl[0] += w.x;
            dh[0] += w.y;
        } else {
#pragma unroll
            for (int p = 0; p < S / 2; ++p) {
                const uint4 w = *reinterpret_cast<const uint4*>(tab + a[g] + 16 * p);
                dl[2 * p] += w.x;
                dh[2 * p] += w.y;
                dl[2 * p + 1] += w.z;
                dh[2 * p + 1] += w.w;
            }
        }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
        // lane l of v - D is 127 + best_l - D_l, in [63, 254]: no borrow between lanes, and its
        // bit 7 is set exactly when D_l < best_l
        const uint32_t ml = (vl[s] - dl[s]) & SL_H32, mh = (vh[s] - dh[s]) & SL_H32;
        if (ml | mh) {
            const uint32_t fl = (ml >> 7) * 0xFFu, fh = (mh >> 7) * 0xFFu;
            vl[s] = (vl[s] & ~fl) | ((dl[s] + SL_B32) & fl);
            vh[s] = (vh[s] & ~fh) | ((dh[s] + SL_B32) & fh);
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                if ((ml >> (8 * l + 7)) & 1u) tg[(8 * s + l) * SL_THREADS] = tag;
                if ((mh >> (8 * l + 7)) & 1u) tg[(8 * s + 4 + l) * SL_THREADS] = tag;
            }
        }
    }
}

// tags: [8 S candidates][SL_THREADS] key tags of each thread's best keys (shared memory; written
// only when a key improves a lane)
template <int NG, int S>
__device__ void sl_pass(const uint64_t* __restrict__ keys, int64_t nv, const ScanLutPlan& pl,
                        const char* __restrict__ tab, uint32_t* __restrict__ tags, int nq,
                        unsigned long long* __restrict__ best, unsigned long long (*red)[SL_CHUNK]) {
    constexpr int LGS = S == 1 ? 0 : S == 2 ? 1 : 2;
    constexpr int U = S == 1 ? 4 : 2;   // key pairs in flight per thread
    uint32_t rs[NG], mk[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        rs[g] = (uint32_t)(pl.shift[g] + 2 - LGS);
        mk[g] = pl.mask[g] << (3 + LGS);
    }
    uint32_t vl[S], vh[S];
    uint32_t* tg = tags + threadIdx.x;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        uint32_t il = 0, ih = 0;
#pragma unroll
        for (int l = 0; l < 4; ++l) {   // lanes past the chunk never improve
            il |= (8 * s + l < nq ? 254u : 127u) << (8 * l);
            ih |= (8 * s + 4 + l < nq ? 254u : 127u) << (8 * l);
        }
        vl[s] = il;
        vh[s] = ih;
    }
    const int64_t stride = (int64_t)gridDim.x * SL_THREADS * 2;
    const int64_t start = ((int64_t)blockIdx.x * SL_THREADS + threadIdx.x) * 2;
    uint32_t it = 0;
    int64_t i = start;
    if (S == 1) {   // one set: no prefetch, the registers keep 4 CTAs per SM
        for (; i + (U - 1) * stride + 1 < nv; i += U * stride, it += U) {
            ulonglong2 kk[U];
#pragma unroll
            for (int u = 0; u < U; ++u) kk[u] = __ldg(reinterpret_cast<const ulonglong2*>(keys + i + u * stride));
#pragma unroll
            for (int u = 0; u < U; ++u) {
                sl_visit<NG, S>(kk[u].x, (it + u) << 1, rs, mk, tab, vl, vh, tg);
                sl_visit<NG, S>(kk[u].y, ((it + u) << 1) | 1u, rs, mk, tab, vl, vh, tg);
            }
        }
    } else if (i + (U - 1) * stride + 1 < nv) {   // the next group of pairs is loaded while this one is visited
        ulonglong2 kk[U];
#pragma unroll
        for (int u = 0; u < U; ++u) kk[u] = __ldg(reinterpret_cast<const ulonglong2*>(keys + i + u * stride));
        for (;;) {
            const int64_t in = i + U * stride;
            const bool more = in + (U - 1) * stride + 1 < nv;
            ulonglong2 kn[U];
            if (more) {
#pragma unroll
                for (int u = 0; u < U; ++u) kn[u] = __ldg(reinterpret_cast<const ulonglong2*>(keys + in + u * stride));
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                sl_visit<NG, S>(kk[u].x, (it + u) << 1, rs, mk, tab, vl, vh, tg);
                sl_visit<NG, S>(kk[u].y, ((it + u) << 1) | 1u, rs, mk, tab, vl, vh, tg);
            }
            i = in;
            it += U;
            if (!more) break;
#pragma unroll
            for (int u = 0; u < U; ++u) kk[u] = kn[u];
        }
    }
    for (; i < nv; i += stride, ++it) {
        sl_visit<NG, S>(__ldg(keys + i), it << 1, rs, mk, tab, vl, vh, tg);
        if (i + 1 < nv) sl_visit<NG, S>(__ldg(keys + i + 1), (it << 1) | 1u, rs, mk, tab, vl, vh, tg);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < S; ++s) {
#pragma unroll
        for (int l = 0; l < 8; ++l) {
            unsigned long long x = ~0ull;
            const uint32_t lv = ((l < 4 ? vl[s] : vh[s]) >> (8 * (l & 3))) & 0xFFu;
            if (8 * s + l < nq && lv < 254u) {   // the lane improved at least once: its tag is set
                const uint64_t d = lv - 127u;
                const uint32_t t = tg[(8 * s + l) * SL_THREADS];
                const int64_t idx = start + (int64_t)(t >> 1) * stride + (t & 1u);
                x = (d << 57) | (unsigned long long)idx;
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
                x = y < x ? y : x;
            }
            if (lane == 0) red[warp][8 * s + l] = x;
        }
    }
    __syncthreads();
    if (threadIdx.x < nq) {
        unsigned long long x = ~0ull;
        for (int w = 0; w < SL_THREADS / 32; ++w) x = red[w][threadIdx.x] < x ? red[w][threadIdx.x] : x;
        atomicMin(best + threadIdx.x, x);
    }
}

// One kernel per set count S: S = 4 scans every chunk of more than 16 candidates (all full chunks),
// S = 2 and S = 1 the last chunk when it holds 9..16 or at most 8.  One wave of CTAs, each scanning
// its slice of the keys once per chunk; the per-S kernels keep the registers (and so the
// occupancy) of the short candidate sets low.
template <int S> struct SlBounds { static constexpr int ctas = 2; };
template <> struct SlBounds<1> { static constexpr int ctas = 4; };
template <> struct SlBounds<2> { static constexpr int ctas = 3; };

template <int NG, int S>
__global__ void __launch_bounds__(SL_THREADS, SlBounds<S>::ctas)
k_scan_lut(const DevSpace* __restrict__ sp, const uint64_t* __restrict__ keys, int64_t nv,
           const uint64_t* __restrict__ cand, const int32_t* __restrict__ pend, const uint32_t* __restrict__ count,
           unsigned long long* __restrict__ best, int lut_min, const __grid_constant__ ScanLutPlan pl) {
    extern __shared__ __align__(16) unsigned long long tab[];   // [256 groups][S], then the tags
    __shared__ uint64_t cq[SL_CHUNK];
    __shared__ unsigned long long red[SL_THREADS / 32][SL_CHUNK];
    const uint32_t cnt = *count;
    for (uint32_t q0 = 0; q0 < cnt; q0 += SL_CHUNK) {
        const int nq = (int)min((uint32_t)SL_CHUNK, cnt - q0);
        if ((nq <= 8 ? 1 : nq <= 16 ? 2 : 4) != S || nq < lut_min) continue;
        __syncthreads();   // the previous chunk is done with cq, tab and red
        if (threadIdx.x < SL_CHUNK) cq[threadIdx.x] = threadIdx.x < nq ? cand[pend[q0 + threadIdx.x]] : 0ull;
        __syncthreads();
        sl_tables(sp, pl, cq, nq, S, tab);
        __syncthreads();
        sl_pass<NG, S>(keys, nv, pl, reinterpret_cast<const char*>(tab),
                       reinterpret_cast<uint32_t*>(tab + (size_t)256 * pl.ng * S), nq, best + q0, red);
    }
}

template <int NG, int S>
static ct_status launch_one(const ct_space* s, const ScanLutPlan& pl, const uint64_t* d_cand, const int32_t* pend,
                            const uint32_t* count, unsigned long long* best, cudaStream_t st, int sms) {
    constexpr size_t TAGS = (size_t)8 * S * SL_THREADS * sizeof(uint32_t);
    const size_t smem = (size_t)256 * pl.ng * S * sizeof(unsigned long long) + TAGS;
    constexpr size_t SMEM_CAP = (size_t)SL_MAX_GROUPS * 256 * S * sizeof(unsigned long long) + TAGS;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(k_scan_lut<NG, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_CAP);
    });
    if (attr_err != cudaSuccess) { set_error("%s", cudaGetErrorString(attr_err)); return CT_ERR_CUDA; }
    int per_sm = 1;
    CT_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan_lut<NG, S>, SL_THREADS, smem));
    const int64_t need = ((int64_t)s->n_valid + SL_THREADS * 8 - 1) / (SL_THREADS * 8);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * std::max(1, per_sm)));
    k_scan_lut<NG, S><<<grid, SL_THREADS, smem, st>>>(s->d, s->keys.p, (int64_t)s->n_valid, d_cand, pend, count,
                                                      best, SL_LUT_MIN, pl);
    return CT_OK;
}

template <int NG>
static ct_status launch_ng(const ct_space* s, const ScanLutPlan& pl, const uint64_t* d_cand, const int32_t* pend,
                           const uint32_t* count, unsigned long long* best, cudaStream_t st) {
    int dev = 0, sms = 148;
    CT_TRY_CUDA(cudaGetDevice(&dev));
    CT_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CT_TRY((launch_one<NG, 4>(s, pl, d_cand, pend, count, best, st, sms)));
    CT_TRY((launch_one<NG, 2>(s, pl, d_cand, pend, count, best, st, sms)));
    CT_TRY((launch_one<NG, 1>(s, pl, d_cand, pend, count, best, st, sms)));
    count_launch(3);
    return CT_OK;
}

// The table scan for the pending candidates when the space suits it.  *launched tells whether it
// ran; when it did, a last chunk of fewer than *lut_min candidates is left to the SWAR scan.
ct_status scan_lut(const ct_space* s, const uint64_t* d_cand, const int32_t* pend, const uint32_t* count,
                   unsigned long long* best, cudaStream_t st, bool* launched, int* lut_min) {
    *launched = false;
    *lut_min = SL_LUT_MIN;
    ScanLutPlan pl;
    if (!scan_lut_plan(s, pl)) return CT_OK;
    ct_status r = CT_OK;
    switch (pl.ng) {
        case 1: r = launch_ng<1>(s, pl, d_cand, pend, count, best, st); break;
        case 2: r = launch_ng<2>(s, pl, d_cand, pend, count, best, st); break;
        case 3: r = launch_ng<3>(s, pl, d_cand, pend, count, best, st); break;
        case 4: r = launch_ng<4>(s, pl, d_cand, pend, count, best, st); break;
        case 5: r = launch_ng<5>(s, pl, d_cand, pend, count, best, st); break;
        case 6: r = launch_ng<6>(s, pl, d_cand, pend, count, best, st); break;
        case 7: r = launch_ng<7>(s, pl, d_cand, pend, count, best, st); break;
        default: r = launch_ng<8>(s, pl, d_cand, pend, count, best, st); break;
    }
    if (r == CT_OK) *launched = true;
    return r;
}

}  // namespace ct
