// The paper's own repair rules (Section IV-A neighbour definitions; Algorithm 1's
// index-distance repair for DE, Algorithm 2 for PSO/Firefly, Algorithm 3 for GA),
// as an exact streaming pass over the sorted valid keys.
//
// For every (valid key v, pending candidate u) one pass computes, field by field:
//   rule 1: the index distance sum_k |v_k - u_k|, kept as the packed minimum
//           (distance << 32 | rank): the nearest, smallest key among ties;
//   rule 2: membership of v in the strictly-adjacent, adjacent and Hamming sets of u
//           and the squared Euclidean distance between v's grid coordinates and the
//           particle position, summed in ascending parameter order in fp32; one packed
//           minimum (distance bits << 32 | rank) per set;
//   rule 3: the size of each set within each contiguous slice of keys.  A second
//           kernel picks a uniform member of the first non-empty set from one RNG word
//           and the slice holding it walks its keys in order to find it.
// "Adjacent" uses, per parameter, the nearest lower and higher value that occurs in
// some valid configuration.  Candidates whose three sets are all empty keep the
// Hamming nearest valid key.  Ranks are packed in 32 bits: |V| < 2^32.
#include <cuda_runtime.h>

#include <cstdlib>
#include <mutex>

#include "internal.hpp"

namespace ct {

constexpr int RT = 256;   // threads per CTA
constexpr int RQ = 8;     // candidates per CTA
constexpr int OCC_WORDS = BLOCK_BITS_MAX / 32;   // per parameter

struct RuleCand {
    uint64_t u;
    int32_t lo[MAXP], hi[MAXP];
};

// values of each parameter occurring in some valid key (bit v of occ[k * OCC_WORDS ...])
__global__ void __launch_bounds__(RT) k_occ(const DevSpace* __restrict__ sp, const uint64_t* __restrict__ keys,
                                            int64_t nv, uint32_t* __restrict__ occ) {
    __shared__ uint32_t s[MAXP * OCC_WORDS];
    const int n = sp->n;
    for (int e = threadIdx.x; e < n * OCC_WORDS; e += RT) s[e] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < nv; i += (int64_t)gridDim.x * RT) {
        const uint64_t key = keys[i];
        for (int k = 0; k < n; ++k) {
            const int v = field(sp, key, k);
            atomicOr(&s[k * OCC_WORDS + (v >> 5)], 1u << (v & 31));
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * OCC_WORDS; e += RT)
        if (s[e]) atomicOr(&occ[e], s[e]);
}

// valid candidates map to themselves; the others are queued with their adjacency bounds
__global__ void k_rule_prep(const DevSpace* __restrict__ sp, const uint32_t* __restrict__ tables,
                            const uint32_t* __restrict__ occ, const uint64_t* __restrict__ cand, int64_t n,
                            uint64_t* __restrict__ out, int32_t* __restrict__ pend, uint32_t* __restrict__ count,
                            RuleCand* __restrict__ rc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t c = cand[i];
        if (valid_key(sp, tables, c)) { out[i] = c; continue; }
        const uint32_t slot = atomicAdd(count, 1u);
        pend[slot] = (int32_t)i;
        RuleCand& r = rc[slot];
        r.u = c;
        for (int k = 0; k < sp->n; ++k) {
            const int uk = field(sp, c, k);
            int lo = -1, hi = -1;
            if (occ) {
                for (int t = uk - 1; t >= 0; --t) if ((occ[k * OCC_WORDS + (t >> 5)] >> (t & 31)) & 1u) { lo = t; break; }
                for (int t = uk + 1; t < sp->r[k]; ++t) if ((occ[k * OCC_WORDS + (t >> 5)] >> (t & 31)) & 1u) { hi = t; break; }
            }
            r.lo[k] = lo;
            r.hi[k] = hi;
        }
    }
}

// membership bits of v in the three sets of candidate r: bit0 strictly adjacent, bit1
// adjacent, bit2 Hamming; optionally the squared distance to the position x
__device__ __forceinline__ uint32_t rule_sets(const DevSpace* __restrict__ sp, uint64_t v, const RuleCand& r,
                                              const float* x, float eps, float* eu) {
    int nd = 0;
    bool sa = true, adj = true;
    float s = 0.0f;
    for (int k = 0; k < sp->n; ++k) {
        const int vk = field(sp, v, k), uk = field(sp, r.u, k);
        const int d = vk - uk;
        if (x) {
            const float dd = __fsub_rn(__fmul_rn((float)vk, eps), x[k]);
            s = __fadd_rn(s, __fmul_rn(dd, dd));
        }
        if (d == 0) continue;
        ++nd;
        if (d > 1 || d < -1) sa = false;
        if (vk != r.lo[k] && vk != r.hi[k]) adj = false;
    }
    if (eu) *eu = s;
    if (nd == 0) return 0u;
    return (sa ? 1u : 0u) | (adj ? 2u : 0u) | (nd == 1 ? 4u : 0u);
}

template <int RULE>
__global__ void __launch_bounds__(RT)
k_rule_scan(const DevSpace* __restrict__ sp, const uint64_t* __restrict__ keys, int64_t nv, int64_t slice,
            const RuleCand* __restrict__ rc, const int32_t* __restrict__ pend, const uint32_t* __restrict__ count,
            const float* __restrict__ pos, float eps, unsigned long long* __restrict__ best,
            uint32_t* __restrict__ cnt) {
    __shared__ RuleCand cs[RQ];
    __shared__ float xs[RQ][MAXP];
    __shared__ unsigned long long red[RT / 32][RQ][3];
    const uint32_t total = *count;
    const uint32_t q0 = blockIdx.y * RQ;
    if (q0 >= total) return;
    const int nq = min((uint32_t)RQ, total - q0);
    const int N = sp->n;
    for (int e = threadIdx.x; e < nq; e += RT) cs[e] = rc[q0 + e];
    if (RULE == 2)
        for (int e = threadIdx.x; e < nq * N; e += RT) xs[e / N][e % N] = pos[(size_t)pend[q0 + e / N] * N + e % N];
    __syncthreads();
    const int64_t lo = (int64_t)blockIdx.x * slice, hi = min(nv, lo + slice);
    unsigned long long b[RQ][3];
#pragma unroll
    for (int q = 0; q < RQ; ++q) b[q][0] = b[q][1] = b[q][2] = ~0ull;
    uint32_t c3[RQ][3];
#pragma unroll
    for (int q = 0; q < RQ; ++q) c3[q][0] = c3[q][1] = c3[q][2] = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += RT) {
        const uint64_t v = __ldg(keys + i);
#pragma unroll
        for (int q = 0; q < RQ; ++q) {
            if (q >= nq) break;
            if (RULE == 1) {
                int l1 = 0;
                for (int k = 0; k < N; ++k) l1 += abs(field(sp, v, k) - field(sp, cs[q].u, k));
                const unsigned long long p = ((unsigned long long)l1 << 32) | (unsigned long long)i;
                b[q][0] = p < b[q][0] ? p : b[q][0];
            } else if (RULE == 2) {
                float eu;
                const uint32_t m = rule_sets(sp, v, cs[q], xs[q], eps, &eu);
                const unsigned long long p = ((unsigned long long)__float_as_uint(eu) << 32) | (unsigned long long)i;
#pragma unroll
                for (int t = 0; t < 3; ++t)
                    if ((m >> t) & 1u) b[q][t] = p < b[q][t] ? p : b[q][t];
            } else {
                const uint32_t m = rule_sets(sp, v, cs[q], nullptr, 0.0f, nullptr);
#pragma unroll
                for (int t = 0; t < 3; ++t) c3[q][t] += (m >> t) & 1u;
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < RQ; ++q)
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            unsigned long long v = RULE == 3 ? (unsigned long long)c3[q][t] : b[q][t];
            for (int o = 16; o; o >>= 1) {
                const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
                v = RULE == 3 ? v + w : (w < v ? w : v);
            }
            if (lane == 0) red[warp][q][t] = v;
        }
    __syncthreads();
    if (threadIdx.x < nq * 3) {
        const int q = threadIdx.x / 3, t = threadIdx.x % 3;
        unsigned long long v = RULE == 3 ? 0ull : ~0ull;
        for (int w = 0; w < RT / 32; ++w) {
            const unsigned long long x = red[w][q][t];
            v = RULE == 3 ? v + x : (x < v ? x : v);
        }
        if (RULE == 3) cnt[((size_t)(q0 + q) * 3 + t) * gridDim.x + blockIdx.x] = (uint32_t)v;
        else if (RULE == 1 && t == 0) atomicMin(best + (size_t)(q0 + q) * 3, v);
        else if (RULE == 2) atomicMin(best + (size_t)(q0 + q) * 3 + t, v);
    }
}

// ------------------------------------------------------------------------------------
// Table form of the scan for long key slices.  The key's fields are cut into groups of
// adjacent fields (at most 8 bits, or one wider field of at most 12 bits; at most 8 groups;
// keys of at most 59 bits); for each pending candidate a CTA tabulates, per group and per bit
// pattern of the group, what the per-field loop above computes for those fields, and a
// (key, candidate) pair then costs one table read per group:
//   rule 1: the group's index distance, 16-bit lanes, eight candidates to a 16-byte entry (the
//           plan requires sum_k (r_k - 1) < 2^15 - 1, so lanes never carry and a borrow test
//           on 0x7fff + best - distance flags exactly the improving lanes);
//   rules 2, 3: a 16-byte entry of a flag byte per candidate (bit 0 "every field within +-1",
//           bit 1 "every field unchanged or at its lower / higher occurring value") and a count
//           byte per candidate (the number of changed fields); groups combine by AND of the flags
//           and a byte-wise sum of the counts, and only keys in some candidate's sets take the
//           per-candidate work.
// Groups are laid out widest first, so every group's first entry is a multiple of its size and
// a key's byte offset into the tables is one shift, AND and OR per group.  The minima, counts
// and (for set members) the fp32 Euclidean distance are those of the loop; a thread visits its
// keys in increasing order and keeps strict improvements, so the first key wins ties.
// ------------------------------------------------------------------------------------
constexpr int LUT_MAX_GROUPS = 8;
constexpr int LUT_MIN_SLICE = 32768;             // keys per CTA that amortise the tables
constexpr size_t LUT_MAX_BYTES = 64 * 1024;
constexpr size_t RULE2_MIN_BYTES = (size_t)3 * RQ * RT * sizeof(unsigned long long);

struct LutPlan {
    int ng, entries;                             // groups; entries of one table set
    int shift[LUT_MAX_GROUPS];                   // lowest key bit of the group
    uint32_t mask[LUT_MAX_GROUPS];               // (1 << width) - 1
    int base[LUT_MAX_GROUPS];                    // first entry of the group (a multiple of mask + 1)
    int k0[LUT_MAX_GROUPS], k1[LUT_MAX_GROUPS];  // parameters k0..k1 of the group
};

static bool lut_plan(const ct_space* s, int rule, int64_t slice, LutPlan& pl) {
    int64_t min_slice = LUT_MIN_SLICE;   // CATUNE_RULE_LUT_MIN_SLICE overrides it (tests)
    if (const char* env = getenv("CATUNE_RULE_LUT_MIN_SLICE")) min_slice = strtoll(env, nullptr, 10);
    if (slice < min_slice) return false;
    const DevSpace& h = s->h;
    if (h.key_bits > 59) return false;
    int64_t sum_r = 0;
    for (int k = 0; k < h.n; ++k) sum_r += h.r[k] - 1;
    if (rule == 1 && sum_r >= 32767) return false;   // 16-bit lanes with a borrow guard bit
    pl.ng = 0;
    int width[LUT_MAX_GROUPS];
    int k = h.n - 1;                             // the last parameter holds the lowest bits
    while (k >= 0) {
        if (pl.ng == LUT_MAX_GROUPS) return false;
        const int g = pl.ng++;
        pl.k1[g] = k;
        pl.shift[g] = h.off[k];
        int w = h.w[k];
        if (w > 12) return false;
        --k;
        while (k >= 0 && w <= 8 && w + h.w[k] <= 8) w += h.w[k--];
        pl.k0[g] = k + 1;
        pl.mask[g] = (1u << w) - 1u;
        width[g] = w;
    }
    pl.entries = 0;
    for (int w = 12; w >= 0; --w)                // widest first: bases stay aligned
        for (int g = 0; g < pl.ng; ++g)
            if (width[g] == w) { pl.base[g] = pl.entries; pl.entries += 1 << w; }
    const size_t bytes = (size_t)pl.entries * 16;
    return bytes <= LUT_MAX_BYTES;
}

// per-thread scan state of one chunk of RQ candidates
template <int RULE>
struct RuleScan {
    uint32_t v[4];                    // rule 1: 0x7fff + best distance, two 16-bit lanes per word
    int64_t bi[RQ];                   // rule 1: rank of the best key
    unsigned long long* b;            // rule 2: packed (distance bits, rank) of (candidate q, set t)
                                      // at b[(3 q + t) * RT] (shared memory: set members are rare)
    uint32_t c3[RQ][3];               // rule 3: set sizes
};

template <int RULE, int NG>
__device__ __forceinline__ void rule_visit(const DevSpace* __restrict__ sp, uint64_t v, int64_t i, int nq, int N,
                                           float eps, const float (*xs)[MAXP], const char* __restrict__ tab,
                                           const uint32_t (&rs)[NG], const uint32_t (&mk)[NG],
                                           const uint32_t (&bb)[NG], RuleScan<RULE>& S) {
    const uint64_t kx = v << 5;
    uint32_t a[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g) a[g] = ((uint32_t)(kx >> rs[g]) & mk[g]) | bb[g];
    if (RULE == 1) {
        uint32_t d[4] = {0, 0, 0, 0};
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            const uint4 w = *reinterpret_cast<const uint4*>(tab + a[g]);
            d[0] += w.x; d[1] += w.y; d[2] += w.z; d[3] += w.w;
        }
        uint32_t m[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) m[j] = (S.v[j] - d[j]) & 0x80008000u;
        if (m[0] | m[1] | m[2] | m[3]) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t f = (m[j] >> 15) * 0xffffu;
                S.v[j] = (S.v[j] & ~f) | ((d[j] + 0x7fff7fffu) & f);
                if (m[j] & 0x8000u) S.bi[2 * j] = i;
                if (m[j] & 0x80000000u) S.bi[2 * j + 1] = i;
            }
        }
    } else {
        uint32_t f0 = ~0u, f1 = ~0u, n0 = 0, n1 = 0;
#pragma unroll
        for (int g = 0; g < NG; ++g) {   // flag bytes AND, count bytes add
            const uint4 w = *reinterpret_cast<const uint4*>(tab + a[g]);
            f0 &= w.x; f1 &= w.y;
            n0 += w.z; n1 += w.w;
        }
        // the key matters to some candidate only if it is in one of its sets: an adjacency flag,
        // or exactly one changed parameter (a zero byte of n ^ 0x01..; the borrow test is exact
        // about whether any byte is zero)
        const uint32_t x0 = n0 ^ 0x01010101u, x1 = n1 ^ 0x01010101u;
        const uint32_t one = ((x0 - 0x01010101u) & ~x0) | ((x1 - 0x01010101u) & ~x1);
        if (!(((f0 | f1) & 0x03030303u) | (one & 0x80808080u))) return;
        const unsigned long long fl = ((unsigned long long)f1 << 32) | f0;
        const unsigned long long nd = ((unsigned long long)n1 << 32) | n0;
#pragma unroll
        for (int q = 0; q < RQ; ++q) {
            if (q >= nq) break;
            const uint32_t n = (uint32_t)((nd >> (8 * q)) & 0xffu);
            if (n == 0) continue;
            const uint32_t f = (uint32_t)((fl >> (8 * q)) & 3u);
            const uint32_t mm = f | (n == 1 ? 4u : 0u);
            if (RULE == 3) {
#pragma unroll
                for (int t = 0; t < 3; ++t) S.c3[q][t] += (mm >> t) & 1u;
            } else if (mm) {
                float sum = 0.0f;
                for (int k = 0; k < N; ++k) {
                    const float dd = __fsub_rn(__fmul_rn((float)field(sp, v, k), eps), xs[q][k]);
                    sum = __fadd_rn(sum, __fmul_rn(dd, dd));
                }
                const unsigned long long p = ((unsigned long long)__float_as_uint(sum) << 32) | (unsigned long long)i;
#pragma unroll
                for (int t = 0; t < 3; ++t)
                    if ((mm >> t) & 1u) {
                        unsigned long long& bt = S.b[(3 * q + t) * RT];
                        bt = p < bt ? p : bt;
                    }
            }
        }
    }
}

template <int RULE, int NG>
__global__ void __launch_bounds__(RT)
k_rule_scan_lut(const DevSpace* __restrict__ sp, const uint64_t* __restrict__ keys, int64_t nv, int64_t slice,
                const RuleCand* __restrict__ rc, const int32_t* __restrict__ pend, const uint32_t* __restrict__ count,
                const float* __restrict__ pos, float eps, unsigned long long* __restrict__ best,
                uint32_t* __restrict__ cnt, const __grid_constant__ LutPlan pl) {
    // [entries][2] (rule 1: two words of 16-bit distances; rules 2, 3: flag bytes, count bytes);
    // rule 2 then the per-thread minima [3 RQ][RT]
    extern __shared__ __align__(16) unsigned long long tab[];
    __shared__ RuleCand cs[RQ];
    __shared__ float xs[RQ][MAXP];
    __shared__ unsigned long long red[RT / 32][RQ][3];
    const uint32_t total = *count;
    const uint32_t q0 = blockIdx.y * RQ;
    if (q0 >= total) return;
    const int nq = min((uint32_t)RQ, total - q0);
    const int N = sp->n;
    for (int e = threadIdx.x; e < nq; e += RT) cs[e] = rc[q0 + e];
    if (RULE == 2)
        for (int e = threadIdx.x; e < nq * N; e += RT) xs[e / N][e % N] = pos[(size_t)pend[q0 + e / N] * N + e % N];
    __syncthreads();
    for (int e = threadIdx.x; e < pl.entries; e += RT) {
        int g = 0;
        while (g + 1 < pl.ng && !(e >= pl.base[g] && e <= pl.base[g] + (int)pl.mask[g])) ++g;
        const uint32_t local = (uint32_t)(e - pl.base[g]);
        unsigned long long t0 = 0, t1 = 0;
        for (int q = 0; q < nq; ++q) {
            int l1 = 0, nd = 0;
            bool sa = true, adj = true;
            for (int k = pl.k0[g]; k <= pl.k1[g]; ++k) {
                const int vk = (int)((local >> (sp->off[k] - pl.shift[g])) & ((1u << sp->w[k]) - 1u));
                const int uk = field(sp, cs[q].u, k);
                const int d = vk - uk;
                l1 += abs(d);
                if (d != 0) {
                    ++nd;
                    if (d > 1 || d < -1) sa = false;
                    if (vk != cs[q].lo[k] && vk != cs[q].hi[k]) adj = false;
                }
            }
            if (RULE == 1) {
                if (q < 4) t0 |= (unsigned long long)l1 << (16 * q);
                else t1 |= (unsigned long long)l1 << (16 * (q - 4));
            } else {   // a flag byte and a count byte per candidate
                t0 |= ((sa ? 1ull : 0ull) | (adj ? 2ull : 0ull)) << (8 * q);
                t1 |= (unsigned long long)nd << (8 * q);
            }
        }
        tab[2 * e] = t0;
        tab[2 * e + 1] = t1;
    }
    __syncthreads();
    constexpr int LGE = 4;                       // log2 of the entry size (16 bytes)
    uint32_t rs[NG], mk[NG], bb[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        rs[g] = (uint32_t)(pl.shift[g] + 5 - LGE);
        mk[g] = pl.mask[g] << LGE;
        bb[g] = (uint32_t)pl.base[g] << LGE;
    }
    RuleScan<RULE> S;
    S.b = tab + 2 * (size_t)pl.entries + threadIdx.x;   // rule 2 only (the region exists then)
    if (RULE == 2)
#pragma unroll
        for (int e = 0; e < 3 * RQ; ++e) S.b[e * RT] = ~0ull;
#pragma unroll
    for (int q = 0; q < RQ; ++q) {
        S.c3[q][0] = S.c3[q][1] = S.c3[q][2] = 0;
        S.bi[q] = 0;
    }
    unsigned long long b1[RQ];   // rule 1: packed (distance, rank) after the scan
#pragma unroll
    for (int q = 0; q < RQ; ++q) b1[q] = ~0ull;
#pragma unroll
    for (int j = 0; j < 4; ++j)   // lanes past the chunk start at 0x7fff and never improve
        S.v[j] = (2 * j < nq ? 0xfffeu : 0x7fffu) | ((2 * j + 1 < nq ? 0xfffeu : 0x7fffu) << 16);
    const char* tb = reinterpret_cast<const char*>(tab);
    const int64_t lo = (int64_t)blockIdx.x * slice, hi = min(nv, lo + slice);   // slice is even
    int64_t i = lo + 2 * threadIdx.x;
    for (; i + 2 * RT + 1 < hi; i += 4 * RT) {   // two key pairs in flight per thread
        const ulonglong2 k0 = __ldg(reinterpret_cast<const ulonglong2*>(keys + i));
        const ulonglong2 k1 = __ldg(reinterpret_cast<const ulonglong2*>(keys + i + 2 * RT));
        rule_visit<RULE, NG>(sp, k0.x, i, nq, N, eps, xs, tb, rs, mk, bb, S);
        rule_visit<RULE, NG>(sp, k0.y, i + 1, nq, N, eps, xs, tb, rs, mk, bb, S);
        rule_visit<RULE, NG>(sp, k1.x, i + 2 * RT, nq, N, eps, xs, tb, rs, mk, bb, S);
        rule_visit<RULE, NG>(sp, k1.y, i + 2 * RT + 1, nq, N, eps, xs, tb, rs, mk, bb, S);
    }
    for (; i < hi; i += 2 * RT) {
        rule_visit<RULE, NG>(sp, __ldg(keys + i), i, nq, N, eps, xs, tb, rs, mk, bb, S);
        if (i + 1 < hi) rule_visit<RULE, NG>(sp, __ldg(keys + i + 1), i + 1, nq, N, eps, xs, tb, rs, mk, bb, S);
    }
    if (RULE == 1) {
#pragma unroll
        for (int q = 0; q < RQ; ++q) {
            const uint32_t lv = (S.v[q >> 1] >> (16 * (q & 1))) & 0xffffu;
            if (q < nq && lv < 0xfffeu)   // the lane improved at least once
                b1[q] = ((unsigned long long)(lv - 0x7fffu) << 32) | (unsigned long long)S.bi[q];
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < RQ; ++q)
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            unsigned long long v = RULE == 3 ? (unsigned long long)S.c3[q][t]
                                   : RULE == 2 ? S.b[(3 * q + t) * RT] : (t == 0 ? b1[q] : ~0ull);
            for (int o = 16; o; o >>= 1) {
                const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
                v = RULE == 3 ? v + w : (w < v ? w : v);
            }
            if (lane == 0) red[warp][q][t] = v;
        }
    __syncthreads();
    if (threadIdx.x < nq * 3) {
        const int q = threadIdx.x / 3, t = threadIdx.x % 3;
        unsigned long long v = RULE == 3 ? 0ull : ~0ull;
        for (int w = 0; w < RT / 32; ++w) {
            const unsigned long long x = red[w][q][t];
            v = RULE == 3 ? v + x : (x < v ? x : v);
        }
        if (RULE == 3) cnt[((size_t)(q0 + q) * 3 + t) * gridDim.x + blockIdx.x] = (uint32_t)v;
        else if (RULE == 1 && t == 0) atomicMin(best + (size_t)(q0 + q) * 3, v);
        else if (RULE == 2) atomicMin(best + (size_t)(q0 + q) * 3 + t, v);
    }
}

template <int RULE, int NG>
static void launch_lut_ng(dim3 grid, size_t bytes, cudaStream_t st, const ct_space* s, int64_t slice,
                          const RuleCand* rc, const RuleScratch& r, const float* d_pos, float eps,
                          unsigned long long* best, uint32_t* cnt, const LutPlan& pl) {
    static std::once_flag once;   // allow the largest table set (and rule 2's minima) as dynamic shared memory
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_rule_scan_lut<RULE, NG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(LUT_MAX_BYTES + (RULE == 2 ? RULE2_MIN_BYTES : 0)));
    });
    k_rule_scan_lut<RULE, NG><<<grid, RT, bytes, st>>>(s->d, s->keys.p, (int64_t)s->n_valid, slice, rc, r.pend.p,
                                                      r.count.p, d_pos, eps, best, cnt, pl);
}

template <int RULE>
static void launch_lut(dim3 grid, size_t bytes, cudaStream_t st, const ct_space* s, int64_t slice, const RuleCand* rc,
                       const RuleScratch& r, const float* d_pos, float eps, unsigned long long* best, uint32_t* cnt,
                       const LutPlan& pl) {
    switch (pl.ng) {
        case 1: launch_lut_ng<RULE, 1>(grid, bytes, st, s, slice, rc, r, d_pos, eps, best, cnt, pl); break;
        case 2: launch_lut_ng<RULE, 2>(grid, bytes, st, s, slice, rc, r, d_pos, eps, best, cnt, pl); break;
        case 3: launch_lut_ng<RULE, 3>(grid, bytes, st, s, slice, rc, r, d_pos, eps, best, cnt, pl); break;
        case 4: launch_lut_ng<RULE, 4>(grid, bytes, st, s, slice, rc, r, d_pos, eps, best, cnt, pl); break;
        case 5: launch_lut_ng<RULE, 5>(grid, bytes, st, s, slice, rc, r, d_pos, eps, best, cnt, pl); break;
        case 6: launch_lut_ng<RULE, 6>(grid, bytes, st, s, slice, rc, r, d_pos, eps, best, cnt, pl); break;
        case 7: launch_lut_ng<RULE, 7>(grid, bytes, st, s, slice, rc, r, d_pos, eps, best, cnt, pl); break;
        default: launch_lut_ng<RULE, 8>(grid, bytes, st, s, slice, rc, r, d_pos, eps, best, cnt, pl); break;
    }
}

// rules 1 and 2: the winner of the first non-empty set (rule 1: the only one)
__global__ void k_rule_finish(const uint64_t* __restrict__ keys, const int32_t* __restrict__ pend,
                              const uint32_t* __restrict__ count, const unsigned long long* __restrict__ best,
                              uint64_t* __restrict__ out) {
    const uint32_t total = *count;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x)
        for (int t = 0; t < 3; ++t) {
            const unsigned long long b = best[(size_t)q * 3 + t];
            if (b != ~0ull) { out[pend[q]] = keys[b & 0xffffffffull]; break; }
        }
}

// rule 3: choose the set and the member's slice and index within the slice
__global__ void k_rule3_pick(const uint32_t* __restrict__ count, const int32_t* __restrict__ pend,
                             const uint32_t* __restrict__ cnt, int slices, const uint32_t* __restrict__ words,
                             int32_t* __restrict__ target) {
    const uint32_t total = *count;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        target[q * 3] = -1;
        for (int t = 0; t < 3; ++t) {
            const uint32_t* c = cnt + ((size_t)q * 3 + t) * slices;
            uint64_t sum = 0;
            for (int s = 0; s < slices; ++s) sum += c[s];
            if (!sum) continue;
            uint32_t pick = uint_below(words[pend[q]], (uint32_t)sum);
            int s = 0;
            while (pick >= c[s]) { pick -= c[s]; ++s; }
            target[q * 3] = s;
            target[q * 3 + 1] = t;
            target[q * 3 + 2] = (int32_t)pick;
            break;
        }
    }
}

// rule 3: the slice holding the chosen member walks its keys in order and writes it
__global__ void __launch_bounds__(RT)
k_rule3_select(const DevSpace* __restrict__ sp, const uint64_t* __restrict__ keys, int64_t nv, int64_t slice,
               const RuleCand* __restrict__ rc, const int32_t* __restrict__ pend, const uint32_t* __restrict__ count,
               const int32_t* __restrict__ target, uint64_t* __restrict__ out) {
    __shared__ uint32_t wsum[RT / 32];
    __shared__ int found;
    const uint32_t total = *count;
    const int64_t lo = (int64_t)blockIdx.x * slice, hi = min(nv, lo + slice);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t q = blockIdx.y; q < total; q += gridDim.y) {
        if (target[q * 3] != (int)blockIdx.x) continue;   // uniform across the CTA
        const int set = target[q * 3 + 1];
        uint32_t want = (uint32_t)target[q * 3 + 2];
        const RuleCand r = rc[q];
        if (threadIdx.x == 0) found = 0;
        __syncthreads();
        for (int64_t base = lo; base < hi; base += RT) {
            const int64_t i = base + threadIdx.x;
            bool m = false;
            if (i < hi) m = (rule_sets(sp, __ldg(keys + i), r, nullptr, 0.0f, nullptr) >> set) & 1u;
            const uint32_t bal = __ballot_sync(0xffffffffu, m);
            if (lane == 0) wsum[warp] = __popc(bal);
            __syncthreads();
            uint32_t before = 0, all = 0;
            for (int w = 0; w < RT / 32; ++w) { before += w < warp ? wsum[w] : 0u; all += wsum[w]; }
            if (want < all) {
                const uint32_t mine = before + __popc(bal & ((1u << lane) - 1u));
                if (m && mine == want) { out[pend[q]] = keys[i]; found = 1; }
            }
            __syncthreads();
            if (want < all || found) break;
            want -= all;
        }
        __syncthreads();
    }
}

__global__ void k_rule_words(uint64_t seed, uint32_t gen, int P, uint32_t* __restrict__ words) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P) words[i] = rng_word(seed, (uint32_t)i, gen, PU_GA_REPAIR, 0);
}

ct_status rule_reserve(RuleScratch& r, int64_t n, int slices) {
    CT_TRY(r.pend.ensure(n));
    CT_TRY(r.rc.ensure(n * sizeof(RuleCand)));
    CT_TRY(r.best.ensure(3 * (size_t)n));
    CT_TRY(r.count.ensure(1));
    CT_TRY(r.cnt.ensure(3 * (size_t)n * slices));
    CT_TRY(r.target.ensure(3 * (size_t)n));
    CT_TRY(r.words.ensure(n));
    return CT_OK;
}

static int rule_slices(const ct_space* s) {
    int sms = 148, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = ((int64_t)s->n_valid + 4095) / 4096;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 4));
}

ct_status ensure_occ(ct_space* s, cudaStream_t st) {
    if (s->occ_ready) return CT_OK;
    CT_TRY(s->occ.ensure((size_t)MAXP * OCC_WORDS));
    CT_TRY_CUDA(cudaMemsetAsync(s->occ.p, 0, (size_t)MAXP * OCC_WORDS * 4, st));
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(((int64_t)s->n_valid + RT - 1) / RT, 148 * 8));
    k_occ<<<g, RT, 0, st>>>(s->d, s->keys.p, (int64_t)s->n_valid, s->occ.p);
    count_launch();
    CT_TRY_CUDA(cudaGetLastError());
    s->occ_ready = true;
    return CT_OK;
}

int rule_slices_for(const ct_space* s) { return rule_slices(s); }

ct_status repair_rule_impl(ct_space* s, RuleScratch& r, int rule, const uint64_t* d_cand, int64_t n,
                           const float* d_pos, float eps, const uint32_t* d_words, uint64_t* d_out,
                           RepairScratch& rs, cudaStream_t st) {
    if (n == 0) return CT_OK;
    if (s->n_valid >= (1ull << 32)) { set_error("the paper's repair rules need |V| < 2^32"); return CT_ERR_LIMIT; }
    const int slices = rule_slices(s);
    CT_TRY(rule_reserve(r, n, slices));
    if (rule != 1) {
        CT_TRY(ensure_occ(s, st));
        CT_TRY(repair_impl(s, rs, d_cand, n, d_out, nullptr, st));   // fallback: Hamming nearest
    }
    CT_TRY_CUDA(cudaMemsetAsync(r.count.p, 0, 4, st));
    CT_TRY_CUDA(cudaMemsetAsync(r.best.p, 0xff, 3 * (size_t)n * 8, st));
    const unsigned g1 = (unsigned)std::min<int64_t>((n + 255) / 256, 148 * 8);
    k_rule_prep<<<g1, 256, 0, st>>>(s->d, s->tables.p, rule == 1 ? nullptr : s->occ.p, d_cand, n, d_out, r.pend.p,
                                    r.count.p, (RuleCand*)r.rc.p);
    int64_t slice = ((int64_t)s->n_valid + slices - 1) / slices;
    slice += slice & 1;   // even: the table scan reads key pairs
    const dim3 grid(slices, (unsigned)((n + RQ - 1) / RQ));
    RuleCand* rc = (RuleCand*)r.rc.p;
    LutPlan pl;
    const bool lut = lut_plan(s, rule, slice, pl);
    const size_t lut_bytes = lut ? (size_t)pl.entries * 16 + (rule == 2 ? RULE2_MIN_BYTES : 0) : 0;
    if (rule == 1) {
        if (lut)
            launch_lut<1>(grid, lut_bytes, st, s, slice, rc, r, nullptr, 0.0f, r.best.p, nullptr, pl);
        else
            k_rule_scan<1><<<grid, RT, 0, st>>>(s->d, s->keys.p, (int64_t)s->n_valid, slice, rc, r.pend.p, r.count.p,
                                                nullptr, 0.0f, r.best.p, nullptr);
        k_rule_finish<<<g1, 256, 0, st>>>(s->keys.p, r.pend.p, r.count.p, r.best.p, d_out);
    } else if (rule == 2) {
        if (lut)
            launch_lut<2>(grid, lut_bytes, st, s, slice, rc, r, d_pos, eps, r.best.p, nullptr, pl);
        else
            k_rule_scan<2><<<grid, RT, 0, st>>>(s->d, s->keys.p, (int64_t)s->n_valid, slice, rc, r.pend.p, r.count.p,
                                                d_pos, eps, r.best.p, nullptr);
        k_rule_finish<<<g1, 256, 0, st>>>(s->keys.p, r.pend.p, r.count.p, r.best.p, d_out);
    } else {
        if (lut)
            launch_lut<3>(grid, lut_bytes, st, s, slice, rc, r, nullptr, 0.0f, nullptr, r.cnt.p, pl);
        else
            k_rule_scan<3><<<grid, RT, 0, st>>>(s->d, s->keys.p, (int64_t)s->n_valid, slice, rc, r.pend.p, r.count.p,
                                                nullptr, 0.0f, nullptr, r.cnt.p);
        k_rule3_pick<<<g1, 256, 0, st>>>(r.count.p, r.pend.p, r.cnt.p, slices, d_words, r.target.p);
        k_rule3_select<<<dim3(slices, (unsigned)std::min<int64_t>(n, 64)), RT, 0, st>>>(
            s->d, s->keys.p, (int64_t)s->n_valid, slice, rc, r.pend.p, r.count.p, r.target.p, d_out);
    }
    count_launch(rule == 3 ? 4 : 3);
    CT_TRY_CUDA(cudaGetLastError());
    return CT_OK;
}

ct_status rule_words(uint64_t seed, uint32_t gen, int P, uint32_t* words, cudaStream_t st) {
    k_rule_words<<<(P + 255) / 256, 256, 0, st>>>(seed, gen, P, words);
    count_launch();
    CT_TRY_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace ct

using namespace ct;

extern "C" ct_status ct_repair_paper(ct_space* s, int32_t rule, const uint64_t* d_cand, int64_t n, const float* d_pos,
                                     float eps, const uint32_t* d_words, uint64_t* d_out, ct_stream stream) {
    if (!s || n < 0 || (n > 0 && (!d_cand || !d_out)) || rule < 1 || rule > 3 || (rule == 2 && n > 0 && !d_pos) ||
        (rule == 3 && n > 0 && !d_words)) {
        set_error("bad argument");
        return CT_ERR_INVALID_ARG;
    }
    if (!s->built) { set_error("space not built"); return CT_ERR_STATE; }
    if (s->n_valid == 0) { set_error("empty valid space"); return CT_ERR_EMPTY_SPACE; }
    return repair_rule_impl(s, s->rules, rule, d_cand, n, d_pos, eps, d_words, d_out, s->rs, (cudaStream_t)stream);
}
