// Batched form: thousands of independent constraint-aware runs over many spaces of
// uneven size, advanced by one persistent kernel launch.
//
// Each CTA takes runs from a work list (largest first) and performs whole
// generations of a run on chip: propose (Sections IV-B..IV-D), repair (exact
// Hamming nearest valid key: table test, then Hamming balls of growing radius,
// then a scan of the space's keys for what is left), GA mutation, memoised
// evaluation and selection.  The per-run arithmetic is the same device code as
// the single-run kernels, so every batched run equals the same run done alone.
// One launch advances every run by G generations, run by run: runs share
// nothing but the read-only spaces, so a CTA carries its run through all G
// generations before it takes the next, and the generations do not wait for
// one another's slowest run (with one launch per generation, each generation
// waited for its slowest run: 143 -> 96 ms for 4096 runs x 100 generations).
// The kernel's last CTA to finish advances the generation counter by G and
// resets the work list.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <new>
#include <sstream>
#include <vector>

#include "internal.hpp"
#include "optim_dev.cuh"

namespace ct {

constexpr int BATCH_MAX_POP = 256;
constexpr int BATCH_MAX_THREADS = 256;
constexpr int BATCH_LUT_GROUPS = 8;
constexpr int BATCH_LUT_CHUNK = 32;   // candidates per pass of the table scan (four sets of eight)

struct BatchSpace {
    const DevSpace* sp;
    const uint32_t* tables;
    const uint64_t* keys;
    int64_t nv;
    const float* fit;
    const uint32_t* cost;   // simulated evaluation time per rank, or null
    int32_t dmax;
    int32_t pad_;
    const uint32_t* masks[MAX_RADIUS];
    const uint64_t* prefix[MAX_RADIUS];
    int32_t n_subsets[MAX_RADIUS];
    uint64_t total[MAX_RADIUS];
    uint64_t swar_low, swar_high;
    float eps;
    int32_t N;
    // distance tables of the in-CTA scan: groups of adjacent fields of at most 8 bits, group g's
    // entries at 256 g (0 groups: the SWAR scan)
    int32_t lut_ng;
    int32_t lut_shift[BATCH_LUT_GROUPS];
    uint32_t lut_mask[BATCH_LUT_GROUPS];
    int32_t lut_k0[BATCH_LUT_GROUPS], lut_k1[BATCH_LUT_GROUPS];
};

struct BatchRun {
    int32_t space, kind, P, pad_;
    uint64_t seed;
    float target;
    int32_t pad2_;
    uint64_t off_pop, off_pn, off_n, off_memo;
};

struct BatchArgs {
    const BatchSpace* spaces;
    const BatchRun* runs;
    const int32_t* order;
    int32_t n_runs;
    ct_opt_params prm;
    OptDev* st;
    uint64_t* X;
    float* FX;
    float* pos;
    float* vel;
    float* pb;
    float* fpb;
    float* gb;
    float* ynew;
    uint32_t* memo;
    uint32_t* work;
    uint32_t* gen;                      // the generation (advanced by the launch's last CTA)
    uint32_t gens;                      // generations every run advances in this launch
    uint32_t* done;                     // CTAs finished in this launch (the last one resets it)
    float* tr_fit;                      // per-generation trace [run][generation], or null
    unsigned long long* tr_cost;
    unsigned long long* tr_unique;
    uint32_t tr_gens;
    uint32_t ev_cap;                    // event log: improvements of each run's best, [run][ev_cap]
    uint32_t* ev_count;                 // per run (may exceed ev_cap: entries past it are dropped)
    int32_t* ev_gen;
    int32_t* ev_idx;
    unsigned long long* ev_clock;
    float* ev_fit;
    uint32_t* scan_tags;                // table scan: best keys' ranks, [CTA][candidate][thread]
};

// Per-evaluation bookkeeping for the event log: whether the memo bit was first set by this
// evaluation, and the evaluation cost of the configuration.
struct EventSmem {
    unsigned long long chg[BATCH_MAX_POP];   // cost charged at this position (first evaluation)
    uint32_t c[BATCH_MAX_POP];
    uint8_t fresh[BATCH_MAX_POP];
};

// Ball points per key of the scan at which the in-CTA repair switches to the scan (4096-run
// workload, 100 generations: 75.5 ms without the switch, 69.0-69.7 ms at 0.5-0.75, 70.8 at 0.35,
// 90.9 at 0.25).
constexpr double BATCH_BALL_VS_SCAN = 0.5;

struct RepairSmem {
    int32_t pend[BATCH_MAX_POP];
    unsigned long long best[BATCH_MAX_POP];
    uint64_t fail[BATCH_MAX_POP];   // per pending slot: the constraints the candidate fails
    uint64_t pstart[BATCH_MAX_THREADS];   // first ball point of each thread's (candidate, subset) pair
    uint32_t pq[BATCH_MAX_THREADS];       // the pair's pending slot
    uint32_t pS[BATCH_MAX_THREADS];       // the pair's subset (parameter mask)
    uint64_t wsum[BATCH_MAX_THREADS / 32];
    int npend;
};

// Exclusive prefix sum of v over the CTA into start[threadIdx.x]; returns the total.  Every
// thread calls it; blockDim.x is a multiple of 32.  `put` runs between the scan's two barriers:
// after every thread has left the reads of the previous scan's results, before any reads this
// one's.
template <class Put>
__device__ __forceinline__ uint64_t cta_exclusive_scan(uint64_t v, uint64_t* start, uint64_t* wsum, Put put) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = (int)(blockDim.x >> 5);
    uint64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    uint64_t base = 0, total = 0;
    for (int i = 0; i < nw; ++i) {
        const uint64_t x = wsum[i];
        if (i < w) base += x;
        total += x;
    }
    start[t] = base + inc - v;
    put();
    __syncthreads();
    return total;
}

// The in-CTA exhaustive scan with per-candidate distance tables (as the repair's table scan):
// for every group value, how many of the group's fields differ from each candidate, eight
// candidates to a 64-bit entry; a key's eight distances are the lane sums of one entry per group,
// and a borrow test on 127 + best - distance flags the lanes it improves.  A thread visits its
// keys in increasing rank and keeps strict improvements; the packed (distance, rank) minimum over
// the threads keeps the smallest rank among the nearest keys.
template <int S>
__device__ void cta_scan_pass(const BatchSpace& bs, const unsigned long long* __restrict__ tab, int nq,
                              uint32_t* __restrict__ tags, unsigned long long* best) {
    const int t = threadIdx.x, nt = blockDim.x, ng = bs.lut_ng;
    uint32_t vl[S], vh[S];
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
    uint32_t* tg = tags + t;
    // the plan in registers (the tag stores below would otherwise make the compiler reload it
    // from the space record for every key)
    const uint64_t* __restrict__ keys = bs.keys;
    const int64_t nv = bs.nv;
    uint32_t sh[BATCH_LUT_GROUPS], mk[BATCH_LUT_GROUPS];
#pragma unroll
    for (int g = 0; g < BATCH_LUT_GROUPS; ++g) {
        sh[g] = g < ng ? (uint32_t)bs.lut_shift[g] : 0u;
        mk[g] = g < ng ? bs.lut_mask[g] : 0u;
    }
    auto add_group = [&](int g, uint64_t key, uint32_t (&al)[S], uint32_t (&ah)[S]) {
        const uint32_t e = ((uint32_t)(key >> sh[g]) & mk[g]) + 256u * (uint32_t)g;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const unsigned long long w = tab[(size_t)e * S + s];
            al[s] += (uint32_t)w;
            ah[s] += (uint32_t)(w >> 32);
        }
    };
    // Each warp scans one contiguous segment of the keys as rows of 32 consecutive keys, one per
    // lane: a lane's keys are 32 apart, so the key bits above the two lowest groups change
    // rarely, and the sum of those groups is kept per lane until they do.
    const uint32_t ushift = ng > 2 ? sh[2] : 64u;
    uint64_t ucur = ~0ull;
    uint32_t ul[S], uh[S];
#pragma unroll
    for (int s = 0; s < S; ++s) ul[s] = uh[s] = 0;
    const int nw = nt >> 5, warp = t >> 5, lane = t & 31;
    const int64_t seg = ((nv + nw - 1) / nw + 31) & ~(int64_t)31;
    const int64_t end = min(nv, (int64_t)(warp + 1) * seg);
    for (int64_t i = (int64_t)warp * seg + lane; i < end; i += 32) {
        const uint64_t key = __ldg(keys + i);
        if (ushift < 64u && (key >> ushift) != ucur) {
            ucur = key >> ushift;
#pragma unroll
            for (int s = 0; s < S; ++s) ul[s] = uh[s] = 0;
#pragma unroll
            for (int g = 2; g < BATCH_LUT_GROUPS; ++g)
                if (g < ng) add_group(g, key, ul, uh);
        }
        uint32_t dl[S], dh[S];
#pragma unroll
        for (int s = 0; s < S; ++s) { dl[s] = ul[s]; dh[s] = uh[s]; }
        add_group(0, key, dl, dh);
        if (ng > 1) add_group(1, key, dl, dh);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const uint32_t ml = (vl[s] - dl[s]) & 0x80808080u, mh = (vh[s] - dh[s]) & 0x80808080u;
            if (ml | mh) {
                const uint32_t fl = (ml >> 7) * 0xFFu, fh = (mh >> 7) * 0xFFu;
                vl[s] = (vl[s] & ~fl) | ((dl[s] + 0x7F7F7F7Fu) & fl);
                vh[s] = (vh[s] & ~fh) | ((dh[s] + 0x7F7F7F7Fu) & fh);
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    if ((ml >> (8 * l + 7)) & 1u) tg[(8 * s + l) * nt] = (uint32_t)i;
                    if ((mh >> (8 * l + 7)) & 1u) tg[(8 * s + 4 + l) * nt] = (uint32_t)i;
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
            if (8 * s + l < nq && lv < 254u)   // the lane improved at least once
                x = ((unsigned long long)(lv - 127u) << 57) | (unsigned long long)tg[(8 * s + l) * nt];
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
                x = y < x ? y : x;
            }
            if ((t & 31) == 0 && x != ~0ull) atomicMin(best + 8 * s + l, x);
        }
    }
}

__device__ void cta_scan_lut(const BatchSpace& bs, const uint64_t* cand, uint64_t* rep, RepairSmem& rs,
                             unsigned long long* tab, uint32_t* __restrict__ tags) {
    const DevSpace* sp = bs.sp;
    const int t = threadIdx.x, nt = blockDim.x, np = rs.npend;
    for (int q0 = 0; q0 < np; q0 += BATCH_LUT_CHUNK) {
        const int nq = min(BATCH_LUT_CHUNK, np - q0);
        const int S = nq <= 8 ? 1 : nq <= 16 ? 2 : 4;
        for (int q = t; q < nq; q += nt) rs.best[q0 + q] = ~0ull;
        for (int e = t; e < 256 * bs.lut_ng; e += nt) {
            const int g = e >> 8;
            const uint32_t x = (uint32_t)e & 255u;
            if (x > bs.lut_mask[g]) continue;   // never read
            const uint64_t local = (uint64_t)x << bs.lut_shift[g];
            for (int s = 0; s < S; ++s) {
                unsigned long long word = 0;
                for (int l = 0; l < 8; ++l) {
                    const int q = 8 * s + l;
                    if (q >= nq) break;
                    const uint64_t d = local ^ cand[rs.pend[q0 + q]];
                    uint32_t cnt = 0;
                    for (int k = bs.lut_k0[g]; k <= bs.lut_k1[g]; ++k) cnt += (d & sp->fmask[k]) != 0;
                    word |= (unsigned long long)cnt << (8 * l);
                }
                tab[(size_t)e * S + s] = word;
            }
        }
        __syncthreads();
        if (S == 1) cta_scan_pass<1>(bs, tab, nq, tags, rs.best + q0);
        else if (S == 2) cta_scan_pass<2>(bs, tab, nq, tags, rs.best + q0);
        else cta_scan_pass<4>(bs, tab, nq, tags, rs.best + q0);
        __syncthreads();
        for (int q = t; q < nq; q += nt) rep[rs.pend[q0 + q]] = __ldg(bs.keys + (rs.best[q0 + q] & ((1ull << 57) - 1)));
        __syncthreads();
    }
}

// exact nearest valid key (Hamming on value indices, ties to the smallest key) for P candidates
__device__ void cta_repair(const BatchSpace& bs, const uint64_t* cand, uint64_t* rep, int P, RepairSmem& rs,
                           unsigned long long* lut_tab, uint32_t* scan_tags) {
    const DevSpace* sp = bs.sp;
    const int t = threadIdx.x, nt = blockDim.x;
    if (t == 0) rs.npend = 0;
    __syncthreads();
    // the table test by groups of G lanes (as many as the population leaves room for), each lane
    // testing every G-th constraint
    int G = 1;
    while (G < 32 && 2 * G * P <= nt) G <<= 1;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((t & 31) & ~(G - 1)));
    for (int i = t / G; i < P; i += nt / G) {
        const uint64_t c = cand[i];
        uint64_t f = failing_mask_part(sp, bs.tables, c, t & (G - 1), G);
        for (int o = 1; o < G; o <<= 1) f |= __shfl_xor_sync(gmask, f, o);
        if (t & (G - 1)) continue;
        if (!f) {
            rep[i] = c;
        } else {
            const int slot = atomicAdd(&rs.npend, 1);
            rs.pend[slot] = i;
            rs.fail[slot] = f;
        }
    }
    __syncthreads();
    for (int d = 1; d <= bs.dmax; ++d) {
        const int np = rs.npend;
        if (np == 0) break;
        // Past radius 1 the scan takes over once the pending candidates' balls at this radius hold
        // more points than BATCH_BALL_VS_SCAN times the keys the scan's passes read (one pass per
        // 32 candidates): a pass costs the same for 1 candidate as for 32, a ball per candidate.
        if (d > 1 && (double)np * (double)bs.total[d - 1] >
                         BATCH_BALL_VS_SCAN * (double)((np + BATCH_LUT_CHUNK - 1) / BATCH_LUT_CHUNK) * (double)bs.nv)
            break;
        for (int q = t; q < np; q += nt) rs.best[q] = ~0ull;
        __syncthreads();
        const uint64_t pts = bs.total[d - 1];
        const uint32_t* masks = bs.masks[d - 1];
        const uint64_t* prefix = bs.prefix[d - 1];
        const int nsub = bs.n_subsets[d - 1];
        // The (pending candidate, subset) pairs, one per thread at a time: a subset that cannot
        // fix every constraint the candidate fails holds no valid point, so only the points of
        // the other pairs are generated, spread evenly over the threads.
        const uint64_t npairs = (uint64_t)np * (uint64_t)nsub;
        for (uint64_t p0 = 0; p0 < npairs; p0 += (uint64_t)nt) {
            uint64_t size = 0;
            uint32_t q = 0, S = 0;
            if (p0 + t < npairs) {
                q = (uint32_t)((p0 + t) / (uint64_t)nsub);
                const int s = (int)(p0 + t - (uint64_t)q * nsub);
                S = __ldg(masks + s);
                if (fixes_possible(sp, rs.fail[q], S))
                    size = (s + 1 < nsub ? __ldg(prefix + s + 1) : pts) - __ldg(prefix + s);
            }
            const uint64_t T = cta_exclusive_scan(size, rs.pstart, rs.wsum, [&] {
                rs.pq[t] = q;
                rs.pS[t] = S;
            });
            for (uint64_t g = t; g < T; g += (uint64_t)nt) {
                int lo = 0, hi = nt - 1;   // the pair holding point g: the last with start <= g
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (rs.pstart[mid] <= g) lo = mid; else hi = mid - 1;
                }
                const uint32_t q = rs.pq[lo];
                const uint64_t u = cand[rs.pend[q]];
                const uint32_t S = rs.pS[lo];
                uint32_t local = (uint32_t)(g - rs.pstart[lo]);
                uint32_t m = S;
                uint64_t key = u;
                while (m) {
                    const int k = 31 - __clz(m);
                    m &= ~(1u << k);
                    uint32_t a;
                    local = div_alt(sp, k, local, &a);
                    const uint32_t uk = (uint32_t)field(sp, u, k);
                    key = (key & ~sp->fmask[k]) | ((uint64_t)(a < uk ? a : a + 1u) << sp->off[k]);
                }
                // the atomic only when the key beats the candidate's current best
                if (key < *(volatile unsigned long long*)&rs.best[q] && valid_changed(sp, bs.tables, key, S))
                    atomicMin(&rs.best[q], (unsigned long long)key);
            }
        }
        __syncthreads();
        if (t == 0) {
            int n2 = 0;
            for (int q = 0; q < np; ++q) {
                if (rs.best[q] != ~0ull) {
                    rep[rs.pend[q]] = rs.best[q];
                } else {
                    rs.fail[n2] = rs.fail[q];
                    rs.pend[n2++] = rs.pend[q];
                }
            }
            rs.npend = n2;
        }
        __syncthreads();
    }
    if (bs.lut_ng) {   // exhaustive scan for the rest: distance tables, up to 32 candidates per pass
        cta_scan_lut(bs, cand, rep, rs, lut_tab, scan_tags);
        return;
    }
    // exhaustive scan for the rest (SWAR distances), eight candidates per pass over the keys
    const int np = rs.npend;
    for (int q0 = 0; q0 < np; q0 += 8) {
        const int nq = min(8, np - q0);
        for (int q = t; q < nq; q += nt) rs.best[q0 + q] = ~0ull;
        __syncthreads();
        uint64_t cu[8];
        unsigned long long b[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) { cu[q] = q < nq ? cand[rs.pend[q0 + q]] : 0ull; b[q] = ~0ull; }
        for (int64_t i = t; i < bs.nv; i += nt) {
            const uint64_t k = __ldg(bs.keys + i);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const unsigned long long p = ((unsigned long long)hamming_keys(k, cu[q], bs.swar_low, bs.swar_high) << 57) |
                                             (unsigned long long)i;
                b[q] = p < b[q] ? p : b[q];
            }
        }
        for (int q = 0; q < nq; ++q) atomicMin(&rs.best[q0 + q], b[q]);
        __syncthreads();
        for (int q = t; q < nq; q += nt) rep[rs.pend[q0 + q]] = __ldg(bs.keys + (rs.best[q0 + q] & ((1ull << 57) - 1)));
        __syncthreads();
    }
}

__global__ void __launch_bounds__(BATCH_MAX_THREADS, 3) k_batch_gen(const __grid_constant__ BatchArgs ba) {
    extern __shared__ __align__(16) unsigned long long lut_tab[];   // the table scan's tables
    __shared__ uint64_t cand[BATCH_MAX_POP], rep[BATCH_MAX_POP];
    __shared__ float fit[BATCH_MAX_POP];
    __shared__ int order[BATCH_MAX_POP];
    __shared__ SelectSmemT<BATCH_MAX_THREADS, BATCH_MAX_POP> sel;
    __shared__ union {   // the repair's scratch, then the GA mutation's
        RepairSmem rs;
        GaMutSmemT<BATCH_MAX_POP> gm;
    } scr;
    RepairSmem& rsm = scr.rs;
    __shared__ EventSmem evs;
    __shared__ int slot_s;
    const uint32_t gen0 = *ba.gen;
    while (true) {
        if (threadIdx.x == 0) slot_s = (int)atomicAdd(ba.work, 1u);
        __syncthreads();
        const int slot = slot_s;
        __syncthreads();
        if (slot >= ba.n_runs) break;
        const int r = ba.order[slot];
        const BatchRun run = ba.runs[r];
        const BatchSpace& bs = ba.spaces[run.space];
        OptArgs a;
        a.kind = run.kind; a.P = run.P; a.N = bs.N; a.seed = run.seed; a.prm = ba.prm; a.prm.target = run.target;
        a.eps = bs.eps; a.sp = bs.sp; a.tables = bs.tables; a.keys = bs.keys; a.nv = bs.nv;
        a.st = ba.st + r; a.X = ba.X + run.off_pop; a.FX = ba.FX + run.off_pop;
        a.pos = ba.pos + run.off_pn; a.vel = ba.vel + run.off_pn; a.pb = ba.pb + run.off_pn;
        a.fpb = ba.fpb + run.off_pop; a.gb = ba.gb + run.off_n; a.ynew = ba.ynew + run.off_pn;
        const int P = run.P;
        for (uint32_t gi = 0; gi < ba.gens; ++gi) {
            const uint32_t gen = gen0 + gi;
            propose_dev(a, gen, cand, order);
            __syncthreads();
            if (a.prm.constraint_aware)
                cta_repair(bs, cand, rep, P, rsm, lut_tab, ba.scan_tags + (size_t)blockIdx.x * BATCH_LUT_CHUNK * blockDim.x);
            else for (int i = threadIdx.x; i < P; i += blockDim.x) rep[i] = cand[i];
            __syncthreads();
            post_repair_dev(a, gen, rep, scr.gm);
            __syncthreads();
            uint32_t* memo = ba.memo + run.off_memo;
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int64_t rk = rank_of(bs.keys, bs.nv, rep[i]);
                if (rk < 0) {   // baselines only
                    fit[i] = CT_PENALTY;
                    if (ba.ev_cap) { evs.fresh[i] = 0; evs.c[i] = 0; }
                    continue;
                }
                fit[i] = __ldg(bs.fit + rk);
                const uint32_t bit = 1u << (rk & 31);
                const uint32_t old = atomicOr(memo + (rk >> 5), bit);
                const uint32_t cst = bs.cost ? __ldg(bs.cost + rk) : 0u;
                if (!(old & bit)) {
                    atomicAdd(&a.st->n_unique, 1ull);
                    if (bs.cost) atomicAdd(&a.st->cost, (unsigned long long)cst);
                }
                if (ba.ev_cap) { evs.fresh[i] = !(old & bit); evs.c[i] = cst; }
            }
            __syncthreads();
            if (ba.ev_cap) {
                // Evaluations happen one at a time in population order: a configuration is charged
                // at its first position in this generation if no earlier generation evaluated it
                // (exactly one position of such a group won the memo bit above).
                for (int i = threadIdx.x; i < P; i += blockDim.x) {
                    const uint64_t k = rep[i];
                    bool first = true, fresh = false;
                    for (int j = 0; j < P; ++j) {
                        if (rep[j] != k) continue;
                        first = first && j >= i;
                        fresh = fresh || evs.fresh[j];
                    }
                    evs.chg[i] = (first && fresh) ? (unsigned long long)evs.c[i] : 0ull;
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    unsigned long long tot = 0;
                    for (int i = 0; i < P; ++i) tot += evs.chg[i];
                    unsigned long long clk = a.st->cost - tot;   // clock before this generation
                    float b = a.st->best_fit;
                    uint32_t n = ba.ev_count[r];
                    for (int i = 0; i < P; ++i) {
                        clk += evs.chg[i];
                        if (fit[i] < b) {
                            b = fit[i];
                            if (n < ba.ev_cap) {
                                const size_t o = (size_t)r * ba.ev_cap + n;
                                ba.ev_gen[o] = (int32_t)gen;
                                ba.ev_idx[o] = i;
                                ba.ev_clock[o] = clk;
                                ba.ev_fit[o] = b;
                            }
                            ++n;
                        }
                    }
                    ba.ev_count[r] = n;
                }
                __syncthreads();
            }
            select_dev(a, gen, rep, fit, sel);
            if (gen < ba.tr_gens) {
                __syncthreads();
                if (threadIdx.x == 0) {
                    const size_t o = (size_t)r * ba.tr_gens + gen;
                    ba.tr_fit[o] = a.st->best_fit;
                    ba.tr_cost[o] = a.st->cost;
                    ba.tr_unique[o] = a.st->n_unique;
                }
            }
            __syncthreads();   // the run's state as selection left it, before the next generation
        }
    }
    // The last CTA to finish advances the generation and resets the work list for the next
    // launch: every CTA has read the generation at its start and left the work loop by then.
    __shared__ bool last_s;
    if (threadIdx.x == 0) {
        __threadfence();
        last_s = atomicAdd(ba.done, 1u) == gridDim.x - 1;
        if (last_s) {
            *ba.gen = gen0 + ba.gens;
            *ba.work = 0;
            *ba.done = 0;
            __threadfence();
        }
    }
}


}  // namespace ct

using namespace ct;

struct ct_batch {
    std::vector<ct_space*> spaces;
    std::vector<ct_batch_run> runs_h;
    ct_opt_params prm{};
    DevBuf<BatchSpace> d_spaces;
    DevBuf<BatchRun> d_runs;
    DevBuf<int32_t> d_order;
    DevBuf<OptDev> st;
    DevBuf<uint64_t> X;
    DevBuf<float> FX, pos, vel, pb, fpb, gb, ynew;
    DevBuf<uint32_t> memo, ctr;   // ctr[0] = generation, ctr[1] = work counter, ctr[2] = CTAs done
    DevBuf<uint32_t> scan_tags;   // table scan: per CTA of the largest grid, BATCH_LUT_CHUNK x threads
    size_t lut_bytes = 0;         // dynamic shared memory of the table scan (largest plan, four sets)
    DevBuf<float> tr_fit;
    DevBuf<unsigned long long> tr_cost, tr_unique;
    uint32_t tr_gens = 0;
    DevBuf<uint32_t> ev_count;
    DevBuf<int32_t> ev_gen, ev_idx;
    DevBuf<unsigned long long> ev_clock;
    DevBuf<float> ev_fit;
    uint32_t ev_cap = 0;
    std::vector<BatchRun> brun;
    uint64_t n_pop = 0, n_pn = 0, n_n = 0, n_memo = 0;
    int threads = 256, ctas_per_sm = 0, sms = 148;
    uint32_t gens_per_launch = 0;   // run_graph: generations per launch (0: all of them in one)
    std::map<uint32_t, cudaGraphExec_t> graphs;
    uint32_t generation = 0;      // host mirror (generations launched)
    ~ct_batch() {
        for (auto& g : graphs) cudaGraphExecDestroy(g.second);
        d_spaces.release(); d_runs.release(); d_order.release(); st.release(); X.release(); FX.release();
        pos.release(); vel.release(); pb.release(); fpb.release(); gb.release(); ynew.release(); memo.release();
        ctr.release(); tr_fit.release(); tr_cost.release(); tr_unique.release();
        ev_count.release(); ev_gen.release(); ev_idx.release(); ev_clock.release(); ev_fit.release();
    }
    BatchArgs args() const {
        BatchArgs a;
        a.spaces = d_spaces.p; a.runs = d_runs.p; a.order = d_order.p; a.n_runs = (int)runs_h.size(); a.prm = prm;
        a.st = st.p; a.X = X.p; a.FX = FX.p; a.pos = pos.p; a.vel = vel.p; a.pb = pb.p; a.fpb = fpb.p; a.gb = gb.p;
        a.ynew = ynew.p; a.memo = memo.p; a.work = ctr.p + 1; a.gen = ctr.p; a.done = ctr.p + 2; a.gens = 1;
        a.tr_fit = tr_fit.p; a.tr_cost = tr_cost.p; a.tr_unique = tr_unique.p; a.tr_gens = tr_gens;
        a.ev_cap = ev_cap; a.ev_count = ev_count.p; a.ev_gen = ev_gen.p; a.ev_idx = ev_idx.p;
        a.ev_clock = ev_clock.p; a.ev_fit = ev_fit.p;
        a.scan_tags = scan_tags.p;
        return a;
    }
    int grid() const {
        int per = ctas_per_sm > 0 ? ctas_per_sm : 4;
        return std::max(1, std::min((int)runs_h.size(), sms * per));
    }
};

namespace ct {
static ct_status batch_launch(ct_batch* b, cudaStream_t st, uint32_t gens) {
    static std::once_flag carve;   // room for several CTAs' shared memory per SM
    std::call_once(carve, [] {
        cudaFuncSetAttribute(k_batch_gen, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    });
    BatchArgs a = b->args();
    a.gens = gens;
    k_batch_gen<<<b->grid(), b->threads, b->lut_bytes, st>>>(a);
    count_launch();
    CT_TRY_CUDA(cudaGetLastError());
    return CT_OK;
}

static ct_status batch_reset(ct_batch* b) {
    const size_t R = b->runs_h.size();
    std::vector<OptDev> init(R);
    for (size_t i = 0; i < R; ++i) {
        OptDev& o = init[i];
        memset(&o, 0, sizeof o);
        o.de_fbest = __builtin_inff();
        o.fgb = __builtin_inff();
        o.best_key = ~0ull;
        o.best_fit = __builtin_inff();
        o.hit_gen = -1;
        o.hit_evals = -1;
    }
    CT_TRY_CUDA(cudaMemcpy(b->st.p, init.data(), R * sizeof(OptDev), cudaMemcpyHostToDevice));
    CT_TRY_CUDA(cudaMemset(b->memo.p, 0, b->n_memo * 4));
    CT_TRY_CUDA(cudaMemset(b->pos.p, 0, b->n_pn * 4));
    CT_TRY_CUDA(cudaMemset(b->vel.p, 0, b->n_pn * 4));
    CT_TRY_CUDA(cudaMemset(b->pb.p, 0, b->n_pn * 4));
    CT_TRY_CUDA(cudaMemset(b->ynew.p, 0, b->n_pn * 4));
    CT_TRY_CUDA(cudaMemset(b->gb.p, 0, b->n_n * 4));
    CT_TRY_CUDA(cudaMemset(b->ctr.p, 0, 12));
    if (b->tr_gens) {
        const size_t n = R * b->tr_gens;
        std::vector<float> inf(n, __builtin_inff());
        CT_TRY_CUDA(cudaMemcpy(b->tr_fit.p, inf.data(), n * 4, cudaMemcpyHostToDevice));
        CT_TRY_CUDA(cudaMemset(b->tr_cost.p, 0, n * 8));
        CT_TRY_CUDA(cudaMemset(b->tr_unique.p, 0, n * 8));
    }
    if (b->ev_cap) CT_TRY_CUDA(cudaMemset(b->ev_count.p, 0, R * 4));
    b->generation = 0;
    return CT_OK;
}
}  // namespace ct

// Groups of the in-CTA table scan: adjacent fields (lowest key bits first) of at most 8 bits
// together; no plan (the SWAR scan) when a field is wider, more than 8 groups are needed or the
// space has 2^32 valid keys or more.
static void batch_lut_plan(const ct_space* s, BatchSpace& b) {
    const DevSpace& h = s->h;
    b.lut_ng = 0;
    if (s->n_valid >= (1ull << 32)) return;   // ranks are kept in 32 bits
    int ng = 0, k = h.n - 1;
    while (k >= 0 && h.w[k] == 0) --k;
    while (k >= 0) {
        if (ng == BATCH_LUT_GROUPS || h.w[k] > 8) return;
        b.lut_k1[ng] = k;
        b.lut_shift[ng] = h.off[k];
        int width = h.w[k];
        --k;
        while (k >= 0 && width + h.w[k] <= 8) width += h.w[k--];
        b.lut_k0[ng] = k + 1;
        b.lut_mask[ng] = (1u << width) - 1u;
        ++ng;
        while (k >= 0 && h.w[k] == 0) --k;
    }
    b.lut_ng = ng;
}

// Ball radius of the in-CTA repair: the ball is cut where its cumulative size passes 2 |V|,
// never below radius 1; an explicit ct_set_repair_mode on the space takes precedence.  Only the
// (candidate, subset) pairs that can fix the candidate's failing constraints generate points, so
// a ball point is cheap against the scan of every key that a candidate past the cut needs: on the
// 4096-run batched workload (100 generations, one launch) the cut at |V| / 8 took 97.0 ms, |V| / 2
// 95.8, 2 |V| 87.8, 8 |V| and 32 |V| 89.3 (same results).
constexpr double BATCH_BALL_DIV = 0.5;
static int batch_radius(const ct_space* sp) {
    if (sp->repair_mode != 0) return wanted_radius(sp);
    return std::max(auto_radius(sp, BATCH_BALL_DIV), std::min(1, sp->ball_max));
}

extern "C" {

ct_status ct_batch_create(ct_space* const* spaces, int32_t n_spaces, const ct_batch_run* runs, int32_t n_runs,
                          const ct_opt_params* params, ct_batch** out) {
    if (!spaces || n_spaces < 1 || !runs || n_runs < 1 || !out) { set_error("bad argument"); return CT_ERR_INVALID_ARG; }
    *out = nullptr;
    std::vector<BatchSpace> bsp(n_spaces);
    for (int s = 0; s < n_spaces; ++s) {
        ct_space* sp = spaces[s];
        if (!sp || !sp->built || sp->n_valid == 0 || !sp->fit) { set_error("space %d is not built or has no fitness table", s); return CT_ERR_STATE; }
        BatchSpace& b = bsp[s];
        memset(&b, 0, sizeof b);
        b.sp = sp->d; b.tables = sp->tables.p; b.keys = sp->keys.p; b.nv = (int64_t)sp->n_valid; b.fit = sp->fit;
        b.cost = sp->cost;
        const int want = batch_radius(sp);
        if (ensure_balls(sp, want) != CT_OK) return CT_ERR_CUDA;
        b.dmax = std::min<int>(want, (int)sp->balls.size());
        for (int d = 0; d < b.dmax; ++d) {
            b.masks[d] = sp->balls[d].d_masks.p;
            b.prefix[d] = sp->balls[d].d_prefix.p;
            b.n_subsets[d] = (int)sp->balls[d].masks.size();
            b.total[d] = sp->balls[d].total;
        }
        b.swar_low = sp->h.swar_low; b.swar_high = sp->h.swar_high;
        int rmax = 1;
        for (int k = 0; k < sp->h.n; ++k) rmax = std::max(rmax, (int)sp->h.r[k]);
        b.eps = rmax > 1 ? 1.0f / (float)(rmax - 1) : 1.0f;
        b.N = sp->h.n;
        batch_lut_plan(sp, b);
    }
    if (params && params->repair_rule) { set_error("batches use the Hamming repair (repair_rule 0)"); return CT_ERR_INVALID_ARG; }
    ct_batch* bt = new (std::nothrow) ct_batch();
    if (!bt) { set_error("host allocation failed"); return CT_ERR_OOM; }
    bt->spaces.assign(spaces, spaces + n_spaces);
    bt->runs_h.assign(runs, runs + n_runs);
    if (params) bt->prm = *params; else ct_opt_params_default(&bt->prm);
    for (int r = 0; r < n_runs; ++r)
        if (const char* why = check_operators(bt->prm, runs[r].kind, runs[r].pop)) {
            delete bt;
            set_error("run %d: %s", r, why);
            return CT_ERR_INVALID_ARG;
        }
    bt->brun.resize(n_runs);
    std::vector<std::pair<double, int>> cost(n_runs);
    for (int r = 0; r < n_runs; ++r) {
        const ct_batch_run& u = runs[r];
        if (u.space < 0 || u.space >= n_spaces || u.kind < CT_DE || u.kind > CT_GA || u.pop < 3 || u.pop > BATCH_MAX_POP) {
            delete bt;
            set_error("run %d: bad space/kind/pop (pop must be in [3, %d])", r, BATCH_MAX_POP);
            return CT_ERR_INVALID_ARG;
        }
        const ct_space* sp = spaces[u.space];
        BatchRun& br = bt->brun[r];
        memset(&br, 0, sizeof br);
        br.space = u.space; br.kind = u.kind; br.P = u.pop; br.seed = u.seed; br.target = u.target;
        br.off_pop = bt->n_pop; bt->n_pop += u.pop;
        br.off_pn = bt->n_pn; bt->n_pn += (uint64_t)u.pop * sp->h.n;
        br.off_n = bt->n_n; bt->n_n += sp->h.n;
        br.off_memo = bt->n_memo; bt->n_memo += (sp->n_valid + 31) / 32;
        // cost: population times (neighbourhood work ~ log |V|), Firefly quadratic in P, and a
        // weight per optimizer.  The launch ends with its longest runs, so runs that tend to be
        // long start first: on the 4096-run workload GA runs took half the time of DE runs, and
        // PSO runs, whose particles can drift where every candidate needs the key scan, held the
        // longest single runs (71 ms against a 61 ms balanced share).  These weights took the
        // launch from 88 to 77 ms (71 ms, the longest run, when simulated with the run times).
        const double P = u.pop;
        const double w = u.kind == CT_PSO ? 1.5 : u.kind == CT_GA ? 0.5 : 1.0;
        cost[r] = {-w * (u.kind == CT_FIREFLY ? P * P : P * 8.0) * (1.0 + std::log2((double)sp->n_valid)), r};
    }
    std::stable_sort(cost.begin(), cost.end());
    std::vector<int32_t> order(n_runs);
    for (int i = 0; i < n_runs; ++i) order[i] = cost[i].second;
    ct_status e = CT_OK;
#define ALLOC(b, n) if (e == CT_OK) e = bt->b.ensure(n)
    ALLOC(d_spaces, n_spaces); ALLOC(d_runs, n_runs); ALLOC(d_order, n_runs); ALLOC(st, n_runs);
    ALLOC(X, bt->n_pop); ALLOC(FX, bt->n_pop); ALLOC(fpb, bt->n_pop); ALLOC(pos, bt->n_pn); ALLOC(vel, bt->n_pn);
    ALLOC(pb, bt->n_pn); ALLOC(ynew, bt->n_pn); ALLOC(gb, bt->n_n); ALLOC(memo, bt->n_memo); ALLOC(ctr, 3);
#undef ALLOC
    if (e == CT_OK && (cudaMemcpy(bt->d_spaces.p, bsp.data(), n_spaces * sizeof(BatchSpace), cudaMemcpyHostToDevice) != cudaSuccess ||
                       cudaMemcpy(bt->d_runs.p, bt->brun.data(), n_runs * sizeof(BatchRun), cudaMemcpyHostToDevice) != cudaSuccess ||
                       cudaMemcpy(bt->d_order.p, order.data(), n_runs * 4, cudaMemcpyHostToDevice) != cudaSuccess)) {
        set_error("uploading the batch failed");
        e = CT_ERR_CUDA;
    }
    if (e == CT_OK) e = batch_reset(bt);
    if (e != CT_OK) { delete bt; return e; }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&bt->sms, cudaDevAttrMultiProcessorCount, dev);
    {   // the table scan: tables of the largest plan with four candidate sets, and the best-rank
        // tags of every CTA of the largest grid (16 CTAs per SM)
        int ng_max = 0;
        for (const BatchSpace& b : bsp) ng_max = std::max(ng_max, (int)b.lut_ng);
        bt->lut_bytes = (size_t)ng_max * 256 * 4 * sizeof(unsigned long long);
        const uint64_t ctas = (uint64_t)std::min(n_runs, bt->sms * 16);
        if (ng_max && bt->scan_tags.ensure(ctas * BATCH_LUT_CHUNK * BATCH_MAX_THREADS) != CT_OK) {
            delete bt;
            return CT_ERR_OOM;
        }
        // the kernel's dynamic shared-memory limit only grows (batches share the kernel); set here,
        // never under a graph capture
        static std::mutex mu;
        static size_t granted = 0;
        std::lock_guard<std::mutex> lk(mu);
        if (bt->lut_bytes > granted) {
            if (cudaFuncSetAttribute(k_batch_gen, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt->lut_bytes) !=
                cudaSuccess) {
                delete bt;
                set_error("shared memory for the in-CTA table scan (%zu bytes)", bt->lut_bytes);
                return CT_ERR_CUDA;
            }
            granted = bt->lut_bytes;
        }
    }
    *out = bt;
    return CT_OK;
}

void ct_batch_destroy(ct_batch* b) { delete b; }

ct_status ct_batch_set_gens_per_launch(ct_batch* b, int32_t gens) {
    if (!b || gens < 0) { set_error("bad argument"); return CT_ERR_INVALID_ARG; }
    b->gens_per_launch = (uint32_t)gens;
    for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
    b->graphs.clear();
    return CT_OK;
}

ct_status ct_batch_set_launch(ct_batch* b, int32_t threads, int32_t ctas_per_sm) {
    if (!b || (threads != 64 && threads != 128 && threads != 256) || ctas_per_sm < 0 || ctas_per_sm > 16) {
        set_error("threads must be 64, 128 or 256; ctas_per_sm in [0, 16]");
        return CT_ERR_INVALID_ARG;
    }
    b->threads = threads;
    b->ctas_per_sm = ctas_per_sm;
    for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
    b->graphs.clear();
    return CT_OK;
}

ct_status ct_batch_step(ct_batch* b, ct_stream stream) {
    if (!b) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    CT_TRY(batch_launch(b, (cudaStream_t)stream, 1));
    b->generation++;
    return CT_OK;
}

ct_status ct_batch_run_graph(ct_batch* b, uint32_t count, ct_stream stream) {
    if (!b || count == 0) { set_error("bad argument"); return CT_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    auto it = b->graphs.find(count);
    if (it == b->graphs.end()) {
        cudaStream_t cap;
        CT_TRY_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaStreamDestroy(cap);
            set_error("stream capture failed to start");
            return CT_ERR_CUDA;
        }
        ct_status e = CT_OK;
        const uint64_t c0 = ct_launch_count();
        const uint32_t per = b->gens_per_launch ? b->gens_per_launch : count;
        for (uint32_t g0 = 0; g0 < count && e == CT_OK; g0 += per) e = batch_launch(b, cap, std::min(per, count - g0));
        count_launch(0 - (ct_launch_count() - c0));
        cudaGraph_t g;
        cudaError_t ce = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (e != CT_OK) return e;
        if (ce != cudaSuccess) { set_error("capture failed: %s", cudaGetErrorString(ce)); return CT_ERR_CUDA; }
        cudaGraphExec_t ex;
        ce = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) { set_error("instantiate failed: %s", cudaGetErrorString(ce)); return CT_ERR_CUDA; }
        it = b->graphs.emplace(count, ex).first;
    }
    CT_TRY_CUDA(cudaGraphLaunch(it->second, st));
    count_launch(b->gens_per_launch ? (count + b->gens_per_launch - 1) / b->gens_per_launch : 1);
    b->generation += count;
    return CT_OK;
}

ct_status ct_batch_results(ct_batch* b, uint64_t* best_key, float* best_fit, uint64_t* n_unique, int64_t* hit_gen,
                           int64_t* hit_evals, ct_stream stream) {
    if (!b) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    const size_t R = b->runs_h.size();
    std::vector<OptDev> h(R);
    cudaStream_t st = (cudaStream_t)stream;
    CT_TRY_CUDA(cudaMemcpyAsync(h.data(), b->st.p, R * sizeof(OptDev), cudaMemcpyDeviceToHost, st));
    CT_TRY_CUDA(cudaStreamSynchronize(st));
    for (size_t i = 0; i < R; ++i) {
        if (best_key) best_key[i] = h[i].best_key;
        if (best_fit) best_fit[i] = h[i].best_fit;
        if (n_unique) n_unique[i] = h[i].n_unique;
        if (hit_gen) hit_gen[i] = h[i].hit_gen;
        if (hit_evals) hit_evals[i] = h[i].hit_evals;
    }
    return CT_OK;
}

ct_status ct_batch_run_state(const ct_batch* b, int32_t run, uint64_t* d_keys, float* d_fit, float* d_pos, ct_stream stream) {
    if (!b || run < 0 || run >= (int)b->runs_h.size()) { set_error("bad argument"); return CT_ERR_INVALID_ARG; }
    const BatchRun& br = b->brun[run];
    const int N = b->spaces[br.space]->h.n;
    cudaStream_t st = (cudaStream_t)stream;
    if (d_keys) CT_TRY_CUDA(cudaMemcpyAsync(d_keys, b->X.p + br.off_pop, br.P * 8, cudaMemcpyDeviceToDevice, st));
    if (d_fit) CT_TRY_CUDA(cudaMemcpyAsync(d_fit, b->FX.p + br.off_pop, br.P * 4, cudaMemcpyDeviceToDevice, st));
    if (d_pos) CT_TRY_CUDA(cudaMemcpyAsync(d_pos, b->pos.p + br.off_pn, (size_t)br.P * N * 4, cudaMemcpyDeviceToDevice, st));
    return CT_OK;
}

ct_status ct_batch_reset(ct_batch* b) {
    if (!b) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    CT_TRY_CUDA(cudaDeviceSynchronize());
    return batch_reset(b);
}

ct_status ct_batch_set_trace(ct_batch* b, int32_t gens, int32_t events) {
    if (!b || gens < 0 || events < 0) { set_error("bad argument"); return CT_ERR_INVALID_ARG; }
    CT_TRY_CUDA(cudaDeviceSynchronize());
    for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);   // they captured the old arguments
    b->graphs.clear();
    b->tr_fit.release(); b->tr_cost.release(); b->tr_unique.release();
    b->tr_gens = 0;
    b->ev_count.release(); b->ev_gen.release(); b->ev_idx.release(); b->ev_clock.release(); b->ev_fit.release();
    b->ev_cap = 0;
    if (events > 0) {
        const size_t R = b->runs_h.size(), n = R * (size_t)events;
        ct_status e = b->ev_count.ensure(R);
        if (e == CT_OK) e = b->ev_gen.ensure(n);
        if (e == CT_OK) e = b->ev_idx.ensure(n);
        if (e == CT_OK) e = b->ev_clock.ensure(n);
        if (e == CT_OK) e = b->ev_fit.ensure(n);
        if (e != CT_OK) {
            b->ev_count.release(); b->ev_gen.release(); b->ev_idx.release(); b->ev_clock.release(); b->ev_fit.release();
            return e;
        }
        b->ev_cap = (uint32_t)events;
    }
    if (gens > 0) {
        const size_t n = b->runs_h.size() * (size_t)gens;
        ct_status e = b->tr_fit.ensure(n);
        if (e == CT_OK) e = b->tr_cost.ensure(n);
        if (e == CT_OK) e = b->tr_unique.ensure(n);
        if (e != CT_OK) {
            b->tr_fit.release(); b->tr_cost.release(); b->tr_unique.release();
            return e;
        }
        b->tr_gens = (uint32_t)gens;
    }
    return batch_reset(b);
}

ct_status ct_batch_events(const ct_batch* b, uint32_t* count, int32_t* gen, int32_t* idx, uint64_t* clock, float* fit,
                          ct_stream stream) {
    if (!b) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    if (!b->ev_cap) { set_error("no event log: call ct_batch_set_trace with events > 0 first"); return CT_ERR_STATE; }
    const size_t R = b->runs_h.size(), n = R * (size_t)b->ev_cap;
    cudaStream_t st = (cudaStream_t)stream;
    if (count) CT_TRY_CUDA(cudaMemcpyAsync(count, b->ev_count.p, R * 4, cudaMemcpyDeviceToHost, st));
    if (gen) CT_TRY_CUDA(cudaMemcpyAsync(gen, b->ev_gen.p, n * 4, cudaMemcpyDeviceToHost, st));
    if (idx) CT_TRY_CUDA(cudaMemcpyAsync(idx, b->ev_idx.p, n * 4, cudaMemcpyDeviceToHost, st));
    if (clock) CT_TRY_CUDA(cudaMemcpyAsync(clock, b->ev_clock.p, n * 8, cudaMemcpyDeviceToHost, st));
    if (fit) CT_TRY_CUDA(cudaMemcpyAsync(fit, b->ev_fit.p, n * 4, cudaMemcpyDeviceToHost, st));
    CT_TRY_CUDA(cudaStreamSynchronize(st));
    return CT_OK;
}

ct_status ct_batch_trace(const ct_batch* b, float* best_fit, uint64_t* cost, uint64_t* n_unique, ct_stream stream) {
    if (!b) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    if (!b->tr_gens) { set_error("no trace: call ct_batch_set_trace first"); return CT_ERR_STATE; }
    const size_t n = b->runs_h.size() * (size_t)b->tr_gens;
    cudaStream_t st = (cudaStream_t)stream;
    if (best_fit) CT_TRY_CUDA(cudaMemcpyAsync(best_fit, b->tr_fit.p, n * 4, cudaMemcpyDeviceToHost, st));
    if (cost) CT_TRY_CUDA(cudaMemcpyAsync(cost, b->tr_cost.p, n * 8, cudaMemcpyDeviceToHost, st));
    if (n_unique) CT_TRY_CUDA(cudaMemcpyAsync(n_unique, b->tr_unique.p, n * 8, cudaMemcpyDeviceToHost, st));
    CT_TRY_CUDA(cudaStreamSynchronize(st));
    return CT_OK;
}

// Autotuner: times `gens` generations for every (threads, CTAs per SM) variant from a reset
// state, checks that every variant ends in the same state as the first, keeps the fastest,
// and leaves the batch reset.  With a cache path, a previous result for the same batch
// signature is reused, and a new one is appended.
ct_status ct_batch_autotune(ct_batch* b, const char* cache_path, int32_t gens, int32_t* threads_out,
                            int32_t* ctas_out, float* ms_out, ct_stream stream) {
    if (!b || gens < 1) { set_error("bad argument"); return CT_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    std::ostringstream sig;
    sig << "runs=" << b->runs_h.size() << ";pop=" << b->n_pop << ";pn=" << b->n_pn << ";memo=" << b->n_memo << ";sms=" << b->sms;
    const std::string key = sig.str();
    if (cache_path && *cache_path) {
        std::ifstream f(cache_path);
        std::string line;
        while (std::getline(f, line)) {
            if (line.find("\"" + key + "\"") == std::string::npos) continue;
            int th = 0, cps = 0;
            float ms = 0;
            if (sscanf(line.c_str() + line.find("threads"), "threads\": %d, \"ctas_per_sm\": %d, \"ms\": %f", &th, &cps, &ms) == 3) {
                CT_TRY(ct_batch_set_launch(b, th, cps));
                if (threads_out) *threads_out = th;
                if (ctas_out) *ctas_out = cps;
                if (ms_out) *ms_out = ms;
                return CT_OK;
            }
        }
    }
    const int variants[][2] = {{64, 8}, {64, 16}, {128, 4}, {128, 8}, {256, 2}, {256, 4}};
    std::vector<uint64_t> ref_keys;
    float best_ms = 1e30f;
    int best_t = 256, best_c = 4;
    cudaEvent_t e0, e1;
    CT_TRY_CUDA(cudaEventCreate(&e0));
    CT_TRY_CUDA(cudaEventCreate(&e1));
    for (auto& v : variants) {
        CT_TRY(batch_reset(b));
        b->threads = v[0];
        b->ctas_per_sm = v[1];
        CT_TRY_CUDA(cudaEventRecord(e0, st));
        CT_TRY(batch_launch(b, st, (uint32_t)gens));
        CT_TRY_CUDA(cudaEventRecord(e1, st));
        CT_TRY_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        CT_TRY_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        std::vector<uint64_t> keys(b->n_pop);
        CT_TRY_CUDA(cudaMemcpy(keys.data(), b->X.p, b->n_pop * 8, cudaMemcpyDeviceToHost));
        if (ref_keys.empty()) ref_keys = keys;
        else if (keys != ref_keys) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            set_error("autotune variant threads=%d ctas_per_sm=%d changed the result", v[0], v[1]);
            return CT_ERR_STATE;
        }
        if (ms < best_ms) { best_ms = ms; best_t = v[0]; best_c = v[1]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CT_TRY(batch_reset(b));
    CT_TRY(ct_batch_set_launch(b, best_t, best_c));
    if (cache_path && *cache_path) {
        std::ofstream f(cache_path, std::ios::app);
        f << "{\"batch\": \"" << key << "\", \"threads\": " << best_t << ", \"ctas_per_sm\": " << best_c
          << ", \"ms\": " << best_ms << "}\n";
    }
    if (threads_out) *threads_out = best_t;
    if (ctas_out) *ctas_out = best_c;
    if (ms_out) *ms_out = best_ms;
    return CT_OK;
}

}  // extern "C"
