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
    int ng;                            // groups; group g owns table entries [goff[g], goff[g] + mask[g] + 1)
    int n_entries;                     // entries of all groups
    int goff[SL_MAX_GROUPS];
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
    pl.n_entries = 0;
    for (int g = 0; g < pl.ng; ++g) {
        pl.goff[g] = pl.n_entries;
        pl.n_entries += (int)pl.mask[g] + 1;
    }
    return pl.ng > 0;
}

// Tables of one chunk: entry goff[g] + x, lane l of set s = number of group g's fields in which
// the group value x differs from candidate 8 s + l (0 for lanes past the chunk); the groups'
// entries are packed (a group of w bits has 2^w of them).  One set: [entry].  Two or four sets:
// planes of 16-byte entries (sets 2p and 2p + 1 in plane p), so that the 16-byte reads of one
// plane by a warp spread over all eight 16-byte bank groups.
__device__ __forceinline__ size_t sl_index(int S, int ne, int e, int s) {
    return S == 1 ? (size_t)e : (size_t)(s >> 1) * 2 * ne + (size_t)e * 2 + (s & 1);
}
__device__ void sl_tables(const DevSpace* __restrict__ sp, const ScanLutPlan& pl, const uint64_t* cq, int nq,
                          int S, unsigned long long* tab) {
    for (int e = threadIdx.x; e < pl.n_entries; e += SL_THREADS) {
        int g = 0;
        while (g + 1 < pl.ng && e >= pl.goff[g + 1]) ++g;
        const uint32_t x = (uint32_t)(e - pl.goff[g]);
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
            tab[sl_index(S, pl.n_entries, e, s)] = word;
        }
    }
}

// Byte addressing of a key's table entries: entry of group g = ((key << 5) >> rs[g]) & mk[g],
// plus the group's first byte gb[g]; planes `plane` bytes apart.
template <int NG>
struct SlAddr {
    uint32_t rs[NG], mk[NG], gb[NG];
    uint32_t plane;
};

// Adds the table entries of groups [G0, G1) of one key (shifted left by 5) to the sums of each
// set of eight candidates, kept as two 32-bit halves: the lanes never carry or borrow into each
// other, so the halves are summed and tested independently.
template <int G0, int G1, int NG, int S>
__device__ __forceinline__ void sl_add(uint64_t kx, const SlAddr<NG>& ad, const char* __restrict__ tab,
                                       uint32_t (&dl)[S], uint32_t (&dh)[S]) {
    constexpr int LGE = S == 1 ? 3 : 4;
#pragma unroll
    for (int g = G0; g < G1; ++g) {
        // one or two sets: group g at entry 256 g (an OR, and constant plane strides); four sets:
        // the packed groups (an add)
        const uint32_t a = S == 4 ? ((uint32_t)(kx >> ad.rs[g]) & ad.mk[g]) + ad.gb[g]
                                  : ((uint32_t)(kx >> ad.rs[g]) & ad.mk[g]) | ((uint32_t)g << (8 + LGE));
        if (S == 1) {
            const uint2 w = *reinterpret_cast<const uint2*>(tab + a);
            dl[0] += w.x;
            dh[0] += w.y;
        } else {
#pragma unroll
            for (int p = 0; p < S / 2; ++p) {
                const uint4 w = *reinterpret_cast<const uint4*>(tab + a + p * (S == 4 ? ad.plane : 256u * NG << LGE));
                dl[2 * p] += w.x;
                dh[2 * p] += w.y;
                dl[2 * p + 1] += w.z;
                dh[2 * p + 1] += w.w;
            }
        }
    }
}

// The borrow test of one key against the chunk's sets: d = the key's distances (as 8-bit lanes
// in two 32-bit halves per set).  Lane l of v - d is 127 + best_l - d_l, in [63, 254]: no borrow
// between lanes, and its bit 7 is set exactly when d_l < best_l; only improved lanes are updated.
template <int S>
__device__ __forceinline__ void sl_test(uint32_t tag, const uint32_t (&dl)[S], const uint32_t (&dh)[S],
                                        uint32_t (&vl)[S], uint32_t (&vh)[S], uint32_t* __restrict__ tg) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
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

// The distances of a key: the sums of its upper groups (ul, uh, refreshed when the key's upper
// bits changed; sorted keys keep them for runs of hundreds to thousands of keys) plus its NL low
// groups' entries.
template <int NL, int NG, int S>
__device__ __forceinline__ void sl_dist(uint64_t key, int ushift, uint64_t& ucur, const SlAddr<NG>& ad,
                                        const char* __restrict__ tab, uint32_t (&ul)[S],
                                        uint32_t (&uh)[S], uint32_t (&dl)[S], uint32_t (&dh)[S]) {
    if (NL < NG) {
        const uint64_t u = key >> ushift;
        if (u != ucur) {
            ucur = u;
#pragma unroll
            for (int s = 0; s < S; ++s) ul[s] = uh[s] = 0;
            sl_add<NL, NG, NG, S>(key << 5, ad, tab, ul, uh);
        }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) { dl[s] = ul[s]; dh[s] = uh[s]; }
    sl_add<0, NL, NG, S>(key << 5, ad, tab, dl, dh);
}

// The pass over the keys for one chunk.  Each warp takes contiguous segments of SL_SEG keys
// (segment w, w + warps, ...) as rows of 32 keys, one key per lane: a warp's loads are
// contiguous 256-byte rows, each lane visits its keys in increasing order, and the lanes of a
// row share their upper fields.  Only the NL lowest groups are looked up per key; within a row
// group 1 mostly has one or two values, so its reads are mostly broadcasts.
// tags: [8 S candidates][SL_THREADS] key tags of each thread's best keys (shared memory; written
// only when a key improves a lane): tag = segment iteration * rows + row.
constexpr int SL_SEG = 2048;   // keys per warp segment (64 rows of 32)
constexpr int SL_NL = 2;       // groups looked up for every key
template <int NG, int S>
__device__ void sl_pass(const uint64_t* __restrict__ keys, int64_t nv, const ScanLutPlan& pl,
                        const char* __restrict__ tab, uint32_t* __restrict__ tags, int nq,
                        unsigned long long* __restrict__ best, unsigned long long (*red)[SL_CHUNK]) {
    constexpr int LGE = S == 1 ? 3 : 4;
    constexpr int NL = NG < SL_NL ? NG : SL_NL;
    constexpr int ROWS = SL_SEG / 32;
    constexpr int U = S == 4 ? 2 : 4;   // rows per step (their distances first, then their tests); the next
                                        // step's rows are loaded while this one is computed
    SlAddr<NG> ad;
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        ad.rs[g] = (uint32_t)(pl.shift[g] + 5 - LGE);
        ad.mk[g] = pl.mask[g] << LGE;
        ad.gb[g] = (uint32_t)pl.goff[g] << LGE;
    }
    ad.plane = (uint32_t)pl.n_entries << LGE;
    uint32_t vl[S], vh[S], ul[S], uh[S];
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
        ul[s] = uh[s] = 0;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nw = (int64_t)gridDim.x * (SL_THREADS / 32);
    const int64_t gw = (int64_t)blockIdx.x * (SL_THREADS / 32) + warp;
    const int ushift = NL < NG ? pl.shift[NL] : 0;
    uint64_t ucur = ~0ull;
    uint32_t m = 0;
    for (int64_t s0 = gw * SL_SEG; s0 < nv; s0 += nw * SL_SEG, ++m) {
        const int64_t base = s0 + lane;
        if (s0 + SL_SEG <= nv) {   // a whole segment (the same for every lane of the warp)
            uint64_t kn[U];
#pragma unroll
            for (int u = 0; u < U; ++u) kn[u] = __ldg(keys + base + (int64_t)u * 32);
#pragma unroll 1
            for (int j = 0; j < ROWS; j += U) {
                uint64_t kk[U];
#pragma unroll
                for (int u = 0; u < U; ++u) kk[u] = kn[u];
                if (j + U < ROWS) {
#pragma unroll
                    for (int u = 0; u < U; ++u) kn[u] = __ldg(keys + base + (int64_t)(j + U + u) * 32);
                }
                uint32_t dl[U][S], dh[U][S];
#pragma unroll
                for (int u = 0; u < U; ++u) sl_dist<NL, NG, S>(kk[u], ushift, ucur, ad, tab, ul, uh, dl[u], dh[u]);
#pragma unroll
                for (int u = 0; u < U; ++u) sl_test<S>(m * ROWS + (uint32_t)(j + u), dl[u], dh[u], vl, vh, tg);
            }
        } else {                   // the last, partial segment
            for (int j = 0; j < ROWS; ++j) {
                const int64_t i = base + (int64_t)j * 32;
                if (i < nv) {
                    uint32_t dl[S], dh[S];
                    sl_dist<NL, NG, S>(__ldg(keys + i), ushift, ucur, ad, tab, ul, uh, dl, dh);
                    sl_test<S>(m * ROWS + (uint32_t)j, dl, dh, vl, vh, tg);
                }
            }
        }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
#pragma unroll
        for (int l = 0; l < 8; ++l) {
            unsigned long long x = ~0ull;
            const uint32_t lv = ((l < 4 ? vl[s] : vh[s]) >> (8 * (l & 3))) & 0xFFu;
            if (8 * s + l < nq && lv < 254u) {   // the lane improved at least once: its tag is set
                const uint64_t d = lv - 127u;
                const uint32_t t = tg[(8 * s + l) * SL_THREADS];
                const int64_t idx = (gw + (int64_t)(t / ROWS) * nw) * SL_SEG + (int64_t)(t % ROWS) * 32 + lane;
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
template <int S> struct SlBounds { static constexpr int ctas = 3; };   // 32 candidates: 80 registers
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
                       reinterpret_cast<uint32_t*>(tab + (size_t)pl.n_entries * S), nq, best + q0, red);
    }
}

template <int NG, int S>
static ct_status launch_one(const ct_space* s, const ScanLutPlan& packed, const uint64_t* d_cand, const int32_t* pend,
                            const uint32_t* count, unsigned long long* best, cudaStream_t st, int sms) {
    // Four sets: the groups' entries packed (the large space: 704 entries instead of 1,536), so
    // that three CTAs fit an SM (2.38 -> 2.29 ms for 32 candidates).  One or two sets: each group
    // at a multiple of 256 entries, which measured faster there (0.90 / 1.27 ms for 4 / 16
    // candidates against 0.93 / 1.35 packed).
    ScanLutPlan pl = packed;
    if (S < 4) {
        for (int g = 0; g < pl.ng; ++g) pl.goff[g] = 256 * g;
        pl.n_entries = 256 * pl.ng;
    }
    constexpr size_t TAGS = (size_t)8 * S * SL_THREADS * sizeof(uint32_t);
    const size_t smem = (size_t)pl.n_entries * S * sizeof(unsigned long long) + TAGS;
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
