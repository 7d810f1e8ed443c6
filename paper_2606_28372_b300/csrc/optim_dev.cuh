// Per-run optimizer logic as CTA-level device functions (Sections IV-B..IV-D, Table IV),
// shared by the single-run kernels and the batched persistent kernel.
#pragma once
#include <map>

#include "internal.hpp"

namespace ct {

struct OptDev {
    uint64_t de_best;
    float de_fbest;
    int32_t stag;
    int32_t reinit_pending;
    float fgb;
    uint64_t best_key;
    float best_fit;
    uint32_t gen;              // next generation (advanced by select)
    unsigned long long n_unique;
    long long hit_gen, hit_evals;
    unsigned long long cost;   // simulated time of the configurations evaluated (each once)
};

struct OptArgs {
    int kind, P, N;
    uint64_t seed;
    ct_opt_params prm;
    float eps;
    const DevSpace* sp;
    const uint32_t* tables;
    const uint64_t* keys;
    int64_t nv;
    OptDev* st;
    uint64_t* X;
    float* FX;
    float* pos;
    float* vel;
    float* pb;
    float* fpb;
    float* gb;
    float* ynew;
};

constexpr int OPT_THREADS = 256;
constexpr int DE_MAX_PARTNERS = 5;

// random partners each DE mutation draws (-1: unknown mutation)
__host__ __device__ __forceinline__ int de_partners(int mutation) {
    switch (mutation) {
    case CT_DE_BEST1: case CT_DE_CURRENTTOBEST1: return 2;
    case CT_DE_RAND1: case CT_DE_RANDTOBEST1: return 3;
    case CT_DE_BEST2: return 4;
    case CT_DE_RAND2: return 5;
    default: return -1;
    }
}

// operator choices and population size: CT_OK or an error message
static inline const char* check_operators(const ct_opt_params& p, int kind, int pop) {
    if (de_partners(p.de_mutation) < 0) return "unknown DE mutation";
    if (p.de_crossover != CT_DE_BIN && p.de_crossover != CT_DE_EXP) return "unknown DE crossover";
    if (p.ga_crossover < CT_GA_SINGLE_POINT || p.ga_crossover > CT_GA_DISRUPTIVE_UNIFORM) return "unknown GA crossover";
    if (kind == CT_DE && pop < de_partners(p.de_mutation) + 1) return "DE population too small for its mutation";
    return nullptr;
}

__device__ __forceinline__ float clip01(float v) { return v < 0.0f ? 0.0f : (v > 1.0f ? 1.0f : v); }

__device__ __forceinline__ uint64_t stratified_key(const OptArgs& a, uint32_t k, uint32_t gen, uint32_t purpose) {
    const uint64_t nv = (uint64_t)a.nv;
    const uint64_t lo = (uint64_t)(((unsigned __int128)k * nv) / (uint32_t)a.P);
    const uint64_t hi = (uint64_t)(((unsigned __int128)(k + 1) * nv) / (uint32_t)a.P);
    uint64_t off = 0;
    if (hi > lo) {
        uint32_t w[4];
        rng_block(a.seed, k, gen, purpose, 0, w);
        off = uint64_below(w[1], w[0], hi - lo);
    }
    return __ldg(a.keys + lo + off);
}

__device__ __forceinline__ uint64_t snap_key(const OptArgs& a, const float* x) {
    uint64_t key = 0;
    for (int k = 0; k < a.N; ++k) {
        const float q = rintf(__fdiv_rn(x[k], a.eps));
        int v = (int)q;
        if (q < 0.0f) v = 0;
        if (v > a.sp->r[k] - 1) v = a.sp->r[k] - 1;
        key |= (uint64_t)v << a.sp->off[k];
    }
    return key;
}

// Cody-Waite reduction + degree-7 Taylor polynomial, binary32 ops rounded one by
// one; x <= 0, x < -80 gives 0.
__device__ __forceinline__ float exp_ct(float x) {
    if (!(x >= -80.0f)) return 0.0f;
    if (x > 0.0f) x = 0.0f;
    const float LOG2E = 1.44269504088896340736f;
    const float LN2_HI = 0.693145751953125f;
    const float LN2_LO = 1.42860682030941723212e-6f;
    const float nf = rintf(__fmul_rn(x, LOG2E));
    const float r = __fsub_rn(__fsub_rn(x, __fmul_rn(nf, LN2_HI)), __fmul_rn(nf, LN2_LO));
    float p = 1.0f / 5040.0f;
    p = __fadd_rn(__fmul_rn(p, r), 1.0f / 720.0f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f / 120.0f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f / 24.0f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f / 6.0f);
    p = __fadd_rn(__fmul_rn(p, r), 0.5f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f);
    const int n = (int)nf;
    return __fmul_rn(p, __int_as_float((n + 127) << 23));
}

// Beta(1,3)-shaped rank selection: smallest k with w*P^3 < 2^32*(P^3 - (P-k-1)^3).
__device__ __forceinline__ uint32_t beta_pick(uint32_t w, uint32_t P) {
    const uint64_t P3 = (uint64_t)P * P * P;
    const unsigned __int128 lhs = (unsigned __int128)w * P3;
    uint32_t lo = 0, hi = P - 1;   // predicate is monotone in k
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const uint64_t q = (uint64_t)(P - mid - 1);
        const unsigned __int128 rhs = ((unsigned __int128)(P3 - q * q * q)) << 32;
        if (lhs < rhs) hi = mid; else lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ uint32_t gen_of(const OptArgs& a, uint32_t gen_arg, int use_dev) {
    return use_dev ? a.st->gen : gen_arg;
}

// Proposals of one generation for one run; every thread of the CTA takes part.
// `order` is shared scratch of at least P ints.  `s` selects the RNG streams of
// proposal s of a screening pool (DE individual i + s*P, GA pair c + s*ceil(P/2));
// s = 0 is the plain method.
static __device__ void propose_dev(const OptArgs& a, uint32_t gen, uint64_t* __restrict__ cand, int* order, int s = 0) {
    const int P = a.P, N = a.N;
    const bool init = gen == 0 || (a.kind == CT_DE && a.st->reinit_pending);
    if (init && !a.prm.constraint_aware) {   // baselines: random start over the Cartesian product
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            uint32_t w[4];
            if (a.kind == CT_PSO || a.kind == CT_FIREFLY) {
                float* x = a.pos + (size_t)i * N;
                for (int j = 0; j < N; ++j) {
                    if ((j & 3) == 0) rng_block(a.seed, i, gen, PU_RAND_INIT, (uint32_t)j >> 2, w);
                    x[j] = u01(w[j & 3]);
                }
                cand[i] = snap_key(a, x);
            } else {
                uint64_t key = 0;
                for (int k = 0; k < N; ++k) {
                    if ((k & 3) == 0) rng_block(a.seed, i, gen, PU_RAND_INIT, (uint32_t)k >> 2, w);
                    key |= (uint64_t)uint_below(w[k & 3], (uint32_t)a.sp->r[k]) << a.sp->off[k];
                }
                cand[i] = key;
            }
        }
        return;
    }
    if (init) {
        for (int i = threadIdx.x; i < P; i += blockDim.x)
            cand[i] = stratified_key(a, (uint32_t)i, gen, gen == 0 ? PU_INIT : PU_REINIT);
        return;
    }
    const DevSpace* sp = a.sp;
    if (a.kind == CT_DE) {
        const uint64_t best = a.st->de_best;
        const int mut = a.prm.de_mutation;
        const int k = de_partners(mut);
        const float F = a.prm.de_F, CR = a.prm.de_CR;
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            const uint32_t si = (uint32_t)(i + s * P);
            // k distinct partners other than i: draw t is uniform below P-1-t and steps over
            // the excluded indices in ascending order
            uint32_t ex[DE_MAX_PARTNERS + 1], w[4];
            uint64_t xr[DE_MAX_PARTNERS];
            int ne = 1;
            ex[0] = (uint32_t)i;
            for (int t = 0; t < k; ++t) {
                if ((t & 3) == 0) rng_block(a.seed, si, gen, PU_MUT_PICK, (uint32_t)t >> 2, w);
                uint32_t v = uint_below(w[t & 3], (uint32_t)(P - 1 - t));
                for (int e = 0; e < ne; ++e)
                    if (v >= ex[e]) ++v;
                xr[t] = a.X[v];
                int p = ne++;
                while (p > 0 && ex[p - 1] > v) { ex[p] = ex[p - 1]; --p; }
                ex[p] = v;
            }
            const uint64_t xi = a.X[i];
            // crossover: which genes come from the mutant
            uint32_t cw[4];
            rng_block(a.seed, si, gen, PU_CROSS, 0, cw);
            const uint32_t j0 = uint_below(cw[0], (uint32_t)N);
            uint32_t take = 1u << j0;
            if (a.prm.de_crossover == 0) {          // binomial
                for (int j = 0; j < N; ++j) {
                    const uint32_t t = 1u + (uint32_t)j;
                    if ((t & 3u) == 0) rng_block(a.seed, si, gen, PU_CROSS, t >> 2, cw);
                    if (u01(cw[t & 3u]) < CR) take |= 1u << j;
                }
            } else {                                 // exponential: a cyclic run from j0
                for (int L = 1; L < N; ++L) {
                    if ((L & 3) == 0) rng_block(a.seed, si, gen, PU_CROSS, (uint32_t)L >> 2, cw);
                    if (!(u01(cw[L & 3]) < CR)) break;
                    take |= 1u << ((j0 + (uint32_t)L) % (uint32_t)N);
                }
            }
            uint64_t key = 0;
            for (int j = 0; j < N; ++j) {
                const int ii = field(sp, xi, j);
                int pick = ii;
                if (take >> j & 1u) {
                    const int ib = field(sp, best, j);
                    int x[DE_MAX_PARTNERS];
                    for (int t = 0; t < k; ++t) x[t] = field(sp, xr[t], j);
                    float m;
                    switch (mut) {   // fp32, one rounding per operation in this order
                    case CT_DE_BEST1:
                        m = __fadd_rn((float)ib, __fmul_rn(F, (float)(x[0] - x[1])));
                        break;
                    case CT_DE_RAND1:
                        m = __fadd_rn((float)x[0], __fmul_rn(F, (float)(x[1] - x[2])));
                        break;
                    case CT_DE_RAND2:
                        m = __fadd_rn(__fadd_rn((float)x[0], __fmul_rn(F, (float)(x[1] - x[2]))),
                                      __fmul_rn(F, (float)(x[3] - x[4])));
                        break;
                    case CT_DE_BEST2:
                        m = __fadd_rn(__fadd_rn((float)ib, __fmul_rn(F, (float)(x[0] - x[1]))),
                                      __fmul_rn(F, (float)(x[2] - x[3])));
                        break;
                    case CT_DE_CURRENTTOBEST1:
                        m = __fadd_rn(__fadd_rn((float)ii, __fmul_rn(F, (float)(ib - ii))),
                                      __fmul_rn(F, (float)(x[0] - x[1])));
                        break;
                    default:   // CT_DE_RANDTOBEST1
                        m = __fadd_rn(__fadd_rn((float)x[0], __fmul_rn(F, (float)(ib - x[0]))),
                                      __fmul_rn(F, (float)(x[1] - x[2])));
                        break;
                    }
                    const float q = rintf(m);
                    pick = (int)q;
                    if (q < 0.0f) pick = 0;
                    if (pick > sp->r[j] - 1) pick = sp->r[j] - 1;
                }
                key |= (uint64_t)pick << sp->off[j];
            }
            cand[i] = key;
        }
    } else if (a.kind == CT_PSO) {
        const ct_opt_params& pr = a.prm;
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            float* x = a.pos + (size_t)i * N;
            float* v = a.vel + (size_t)i * N;
            const float* p = a.pb + (size_t)i * N;
            uint32_t w[4];
            for (int j = 0; j < N; ++j) {
                const uint32_t t = 2u * j;
                if ((t & 3u) == 0) rng_block(a.seed, i, gen, PU_PSO_R, t >> 2, w);
                const float r1 = u01(w[t & 3u]), r2 = u01(w[(t + 1) & 3u]);
                const float t1 = __fmul_rn(pr.pso_w, v[j]);
                const float t2 = __fmul_rn(__fmul_rn(pr.pso_c1, r1), __fsub_rn(p[j], x[j]));
                const float t3 = __fmul_rn(__fmul_rn(pr.pso_c2, r2), __fsub_rn(a.gb[j], x[j]));
                const float nv = __fadd_rn(__fadd_rn(t1, t2), t3);
                v[j] = nv;
                x[j] = clip01(__fadd_rn(x[j], nv));
            }
            cand[i] = snap_key(a, x);
        }
    } else if (a.kind == CT_FIREFLY) {
        const ct_opt_params& pr = a.prm;
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            float y[MAXP];
            for (int d = 0; d < N; ++d) y[d] = a.pos[(size_t)i * N + d];
            const float fi = a.FX[i];
            for (int j = 0; j < P; ++j) {
                if (!(a.FX[j] < fi)) continue;
                const float* xj = a.pos + (size_t)j * N;
                float s = 0.0f;
                for (int d = 0; d < N; ++d) {
                    const float t = __fsub_rn(y[d], xj[d]);
                    s = __fadd_rn(s, __fmul_rn(t, t));
                }
                const float beta = __fmul_rn(pr.fa_beta0, exp_ct(__fmul_rn(-pr.fa_gamma, s)));
                uint32_t w[4];
                for (int d = 0; d < N; ++d) {
                    const uint32_t t = (uint32_t)(j * N + d);
                    if (d == 0 || (t & 3u) == 0) rng_block(a.seed, i, gen, PU_FA_ALPHA, t >> 2, w);
                    const float u = u01(w[t & 3u]);
                    const float nv = __fadd_rn(__fadd_rn(y[d], __fmul_rn(beta, __fsub_rn(xj[d], y[d]))),
                                               __fmul_rn(pr.fa_alpha, __fsub_rn(u, 0.5f)));
                    y[d] = clip01(nv);
                }
            }
            for (int d = 0; d < N; ++d) a.ynew[(size_t)i * N + d] = y[d];
            cand[i] = snap_key(a, y);
        }
    } else {  // GA
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            const float fi = a.FX[i];
            const uint64_t ki = a.X[i];
            int rk = 0;
            for (int j = 0; j < P; ++j) {
                const float fj = a.FX[j];
                const uint64_t kj = a.X[j];
                rk += (fj < fi) || (fj == fi && (kj < ki || (kj == ki && j < i)));
            }
            order[rk] = i;
        }
        __syncthreads();
        const uint32_t npairs = (uint32_t)(P + 1) / 2;
        for (int c = threadIdx.x; 2 * c < P; c += blockDim.x) {
            uint32_t w[4];
            const uint32_t sc = (uint32_t)c + (uint32_t)s * npairs;
            rng_block(a.seed, sc, gen, PU_GA_SEL, 0, w);
            const uint32_t pa = beta_pick(w[0], (uint32_t)P), pbk = beta_pick(w[1], (uint32_t)P);
            const uint64_t A = a.X[order[pa]], B = a.X[order[pbk]];
            int kind = a.prm.ga_crossover;
            if (kind == CT_GA_TWO_POINT && N < 3) kind = CT_GA_SINGLE_POINT;   // two cuts need three genes
            uint32_t cw[4];
            rng_block(a.seed, sc, gen, PU_GA_CUT, 0, cw);
            uint32_t fromb = 0;   // genes child 0 takes from the second parent
            if (kind == CT_GA_SINGLE_POINT) {
                const uint32_t cut = N >= 2 ? 1u + uint_below(cw[0], (uint32_t)N - 1) : 1u;
                for (int j = (int)cut; j < N; ++j) fromb |= 1u << j;
            } else if (kind == CT_GA_TWO_POINT) {
                const uint32_t c1 = 1u + uint_below(cw[0], (uint32_t)N - 1);
                uint32_t c2 = 1u + uint_below(cw[1], (uint32_t)N - 2);
                if (c2 >= c1) ++c2;
                const uint32_t lo = min(c1, c2), hi = max(c1, c2);
                for (uint32_t j = lo; j < hi; ++j) fromb |= 1u << j;
            } else if (kind == CT_GA_UNIFORM) {
                for (int j = 0; j < N; ++j) {
                    if (j > 0 && (j & 3) == 0) rng_block(a.seed, sc, gen, PU_GA_CUT, (uint32_t)j >> 2, cw);
                    if (!(u01(cw[j & 3]) < 0.5f)) fromb |= 1u << j;
                }
            } else {   // disruptive uniform: half (rounded down) of the differing genes, uniformly
                int D[MAXP], nd = 0;
                for (int j = 0; j < N; ++j)
                    if (field(sp, A, j) != field(sp, B, j)) D[nd++] = j;
                for (int t = 0; t < nd / 2; ++t) {   // partial Fisher-Yates
                    if (t > 0 && (t & 3) == 0) rng_block(a.seed, sc, gen, PU_GA_CUT, (uint32_t)t >> 2, cw);
                    const int s2 = t + (int)uint_below(cw[t & 3], (uint32_t)(nd - t));
                    const int tmp = D[t]; D[t] = D[s2]; D[s2] = tmp;
                    fromb |= 1u << D[t];
                }
            }
            uint64_t bmask = 0;
            for (int j = 0; j < N; ++j)
                if (fromb >> j & 1u) bmask |= sp->fmask[j];
            cand[2 * c] = (A & ~bmask) | (B & bmask);
            if (2 * c + 1 < P) cand[2 * c + 1] = (B & ~bmask) | (A & bmask);
        }
    }
}

// GA mutation: with probability p_mut, a random valid Hamming neighbour.  Aware runs: the child
// is valid (it was repaired), so a neighbour that changes parameter k is valid iff the constraints
// reading k hold at it.  A warp takes one child; its lanes test the neighbours in (parameter,
// value) order 32 at a time, a count pass and a pick pass over the same order.
__device__ __forceinline__ uint64_t ga_neighbour(const DevSpace* __restrict__ sp, uint64_t u, int N, uint32_t n,
                                                 int* kout) {
    int k = 0;
    uint32_t acc = 0;
    while (k < N - 1 && acc + (uint32_t)(sp->r[k] - 1) <= n) { acc += (uint32_t)(sp->r[k] - 1); ++k; }
    const uint32_t idx = n - acc, uk = (uint32_t)field(sp, u, k);
    const uint32_t v = idx < uk ? idx : idx + 1u;   // the other values of k, ascending
    *kout = k;
    return (u & ~sp->fmask[k]) | ((uint64_t)v << sp->off[k]);
}

// Shared scratch of the GA mutation's flat form (populations of at most MAX_POP).
constexpr int GA_MUT_WORDS = 4;   // at most 128 Hamming-1 neighbours per point
template <int MAX_POP>
struct GaMutSmemT {
    uint32_t ok[MAX_POP][GA_MUT_WORDS];   // bit n: neighbour n of the slot's candidate is valid
    int32_t idx[MAX_POP];                  // population index of each mutated candidate
    uint32_t draw[MAX_POP];                // its draw for the choice among the valid neighbours
    int n;
};
using GaMutSmem = GaMutSmemT<CT_MAX_POP>;

template <class GM>
static __device__ void post_repair_dev(const OptArgs& a, uint32_t gen, uint64_t* __restrict__ keys, GM& gm,
                                       int s = 0) {
    if (a.kind != CT_GA || gen == 0) return;
    const DevSpace* sp = a.sp;
    if (!a.prm.constraint_aware) {   // baseline: one random parameter takes another value
        for (int i = threadIdx.x; i < a.P; i += blockDim.x) {
            uint32_t w[4];
            rng_block(a.seed, (uint32_t)(i + s * a.P), gen, PU_GA_MUT, 0, w);
            if (!(u01(w[0]) < a.prm.ga_pmut)) continue;
            const uint64_t u = keys[i];
            const int k = (int)uint_below(w[1], (uint32_t)a.N);
            if (sp->r[k] < 2) continue;
            const uint32_t v = uint_below(w[2], (uint32_t)(sp->r[k] - 1)), uk = (uint32_t)field(sp, u, k);
            keys[i] = (u & ~sp->fmask[k]) | ((uint64_t)(v < uk ? v : v + 1u) << sp->off[k]);
        }
        return;
    }
    uint32_t total = 0;   // Hamming-1 neighbours of any point
    for (int k = 0; k < a.N; ++k) total += (uint32_t)(sp->r[k] - 1);
    if (total <= 32u * GA_MUT_WORDS) {
        // Flat form: the mutated candidates into a list, every (candidate, neighbour) pair tested
        // by one thread (a bit per valid neighbour), then per candidate the chosen valid
        // neighbour, counted in neighbour order as below.
        if (threadIdx.x == 0) gm.n = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < a.P; i += blockDim.x) {
            uint32_t w[4];
            rng_block(a.seed, (uint32_t)(i + s * a.P), gen, PU_GA_MUT, 0, w);
            if (!(u01(w[0]) < a.prm.ga_pmut)) continue;
            const int m = atomicAdd(&gm.n, 1);
            gm.idx[m] = i;
            gm.draw[m] = w[1];
#pragma unroll
            for (int q = 0; q < GA_MUT_WORDS; ++q) gm.ok[m][q] = 0u;
        }
        __syncthreads();
        const uint32_t nm = (uint32_t)gm.n;
        for (uint32_t f = threadIdx.x; f < nm * total; f += blockDim.x) {
            const uint32_t m = f / total, nb = f - m * total;
            int k;
            const uint64_t kk = ga_neighbour(sp, keys[gm.idx[m]], a.N, nb, &k);
            if (valid_changed(sp, a.tables, kk, 1u << k)) atomicOr(&gm.ok[m][nb >> 5], 1u << (nb & 31));
        }
        __syncthreads();
        for (uint32_t m = threadIdx.x; m < nm; m += blockDim.x) {
            uint32_t cnt = 0;
#pragma unroll
            for (int q = 0; q < GA_MUT_WORDS; ++q) cnt += (uint32_t)__popc(gm.ok[m][q]);
            if (!cnt) continue;
            uint32_t pick = uint_below(gm.draw[m], cnt);
            for (int q = 0; q < GA_MUT_WORDS; ++q) {
                uint32_t bal = gm.ok[m][q];
                const uint32_t c = (uint32_t)__popc(bal);
                if (pick < c) {   // the pick-th valid neighbour lies in this word
                    for (uint32_t t = 0; t < pick; ++t) bal &= bal - 1u;
                    int k;
                    const int i = gm.idx[m];
                    keys[i] = ga_neighbour(sp, keys[i], a.N, 32u * (uint32_t)q + (uint32_t)(__ffs(bal) - 1), &k);
                    break;
                }
                pick -= c;
            }
        }
        return;
    }
    const int lane = threadIdx.x & 31, nw = (int)(blockDim.x >> 5);
    for (int i = (int)(threadIdx.x >> 5); i < a.P; i += nw) {
        uint32_t w[4];
        rng_block(a.seed, (uint32_t)(i + s * a.P), gen, PU_GA_MUT, 0, w);
        if (!(u01(w[0]) < a.prm.ga_pmut)) continue;   // the same draw in every lane
        const uint64_t u = keys[i];
        uint32_t cnt = 0;
        for (uint32_t base = 0; base < total; base += 32) {
            bool ok = false;
            if (base + lane < total) {
                int k;
                const uint64_t kk = ga_neighbour(sp, u, a.N, base + lane, &k);
                ok = valid_changed(sp, a.tables, kk, 1u << k);
            }
            cnt += (uint32_t)__popc(__ballot_sync(0xffffffffu, ok));
        }
        if (!cnt) continue;
        const uint32_t pick = uint_below(w[1], cnt);
        uint32_t seen = 0;
        uint64_t res = u;
        for (uint32_t base = 0; base < total; base += 32) {
            bool ok = false;
            uint64_t kk = u;
            if (base + lane < total) {
                int k;
                kk = ga_neighbour(sp, u, a.N, base + lane, &k);
                ok = valid_changed(sp, a.tables, kk, 1u << k);
            }
            uint32_t bal = __ballot_sync(0xffffffffu, ok);
            const uint32_t c = (uint32_t)__popc(bal);
            if (pick < seen + c) {   // the (pick - seen)-th valid neighbour of this group
                for (uint32_t t = 0; t < pick - seen; ++t) bal &= bal - 1u;
                res = __shfl_sync(0xffffffffu, kk, __ffs(bal) - 1);
                break;
            }
            seen += c;
        }
        if (lane == 0) keys[i] = res;
    }
}

__device__ __forceinline__ bool lex_less(float fa, uint64_t ka, float fb, uint64_t kb) {
    return fa < fb || (fa == fb && ka < kb);
}

// Shared scratch of select_dev (block size <= MAX_THREADS, pop <= MAX_POP).
constexpr int SEL_MAX_THREADS = 512;
template <int MAX_THREADS, int MAX_POP>
struct SelectSmemT {
    float rf[MAX_THREADS];
    uint64_t rk[MAX_THREADS];
    int ri[MAX_THREADS];
    uint64_t xs[MAX_POP];      // population keys before selection
    uint64_t us[MAX_POP];      // evaluated keys
    uint8_t pass[MAX_POP];
    uint8_t acc[MAX_POP];
    int init_s;
};
using SelectSmem = SelectSmemT<SEL_MAX_THREADS, CT_MAX_POP>;

// Block-wide argmin of (f, index) over the entries each thread offers: smallest f;
// among equal f the largest index when last_tie, else the smallest.  Entries with
// idx < 0 are absent.  Returns the winning index (-1 if none) in every thread.
template <class SM>
__device__ __forceinline__ int block_argmin(float f, int idx, bool last_tie, SM& sm) {
    // (f, idx) pairs combine by a total order (absent entries lose), so any reduction order
    // gives the same winner: shuffles within each warp, then one warp over the warp winners
    auto better = [last_tie](float f2, int i2, float f1, int i1) {
        if (i2 < 0) return false;
        if (i1 < 0 || f2 < f1) return true;
        return f2 == f1 && (last_tie ? i2 > i1 : i2 < i1);
    };
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o; o >>= 1) {
        const float f2 = __shfl_xor_sync(0xffffffffu, f, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
        if (better(f2, i2, f, idx)) { f = f2; idx = i2; }
    }
    if (lane == 0) { sm.rf[warp] = f; sm.ri[warp] = idx; }
    __syncthreads();
    if (warp == 0) {
        float g = lane < nw ? sm.rf[lane] : 0.0f;
        int j = lane < nw ? sm.ri[lane] : -1;
        for (int o = 16; o; o >>= 1) {
            const float f2 = __shfl_xor_sync(0xffffffffu, g, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, j, o);
            if (better(f2, i2, g, j)) { g = f2; j = i2; }
        }
        if (lane == 0) sm.ri[0] = j;
    }
    __syncthreads();
    const int r = sm.ri[0];
    __syncthreads();
    return r;
}

// Selection / update after evaluation; every thread of the CTA takes part (block size a
// multiple of 32).  Sequential update rules are applied in closed form:
//   "best <- x_i if f_i <= f(best)" over ascending i ends at the last index with the
//   minimal f (if that minimum is <= the old best), "... if f_i < ..." at the first.
template <class SM>
static __device__ void select_dev(const OptArgs& a, uint32_t gen, const uint64_t* __restrict__ keys,
                                  const float* __restrict__ fit, SM& sm) {
    const int P = a.P, N = a.N;
    OptDev* st = a.st;
    const int t = threadIdx.x, nt = blockDim.x;
    if (t == 0) sm.init_s = gen == 0 || (a.kind == CT_DE && st->reinit_pending);
    for (int i = t; i < P; i += nt) { sm.us[i] = keys[i]; sm.xs[i] = a.X[i]; }
    // run best: min (fitness, key) over this generation's evaluations
    float bf = __int_as_float(0x7f800000);
    uint64_t bk = ~0ull;
    for (int i = t; i < P; i += nt)
        if (lex_less(fit[i], sm.us[i], bf, bk)) { bf = fit[i]; bk = sm.us[i]; }
    for (int o = 16; o; o >>= 1) {   // lexicographic minimum: a total order, any order of reduction
        const float f2 = __shfl_xor_sync(0xffffffffu, bf, o);
        const uint64_t k2 = __shfl_xor_sync(0xffffffffu, bk, o);
        if (lex_less(f2, k2, bf, bk)) { bf = f2; bk = k2; }
    }
    const int nw = (nt + 31) >> 5;
    if ((t & 31) == 0) { sm.rf[t >> 5] = bf; sm.rk[t >> 5] = bk; }
    __syncthreads();
    if (t == 0) {
        for (int w = 1; w < nw; ++w)
            if (lex_less(sm.rf[w], sm.rk[w], bf, bk)) { bf = sm.rf[w]; bk = sm.rk[w]; }
        if (lex_less(bf, bk, st->best_fit, st->best_key)) { st->best_fit = bf; st->best_key = bk; }
        if (st->hit_gen < 0 && st->best_fit <= a.prm.target) { st->hit_gen = gen; st->hit_evals = (long long)st->n_unique; }
    }
    __syncthreads();
    const bool init = sm.init_s;
    if (a.kind == CT_DE) {
        if (init) {
            int last = -1;
            float lf = 0.0f;
            for (int i = t; i < P; i += nt) {
                a.X[i] = sm.us[i];
                a.FX[i] = fit[i];
                if (last < 0 || fit[i] <= lf) { last = i; lf = fit[i]; }   // ascending i: ties keep the later
            }
            const int w = block_argmin(last >= 0 ? lf : 0.0f, last, true, sm);
            if (t == 0) {
                if (gen == 0 || fit[w] <= st->de_fbest) { st->de_best = sm.us[w]; st->de_fbest = fit[w]; }
                st->reinit_pending = 0;
                st->stag = 0;
            }
        } else {
            // duplicate tests: plain ORs over the population, unrolled so that eight shared loads
            // are in flight (no early exit; duplicates are rare)
            for (int i = t; i < P; i += nt) {
                const uint64_t u = sm.us[i];
                bool in_x = false;
#pragma unroll 8
                for (int k = 0; k < P; ++k) in_x |= sm.xs[k] == u;
                sm.pass[i] = fit[i] <= a.FX[i] && !in_x;
            }
            __syncthreads();
            int last = -1, n_acc = 0;
            float lf = 0.0f;
            for (int i = t; i < P; i += nt) {
                bool ok = sm.pass[i];
                const uint64_t u = sm.us[i];
                if (ok) {   // not an earlier passing trial with the same key
                    bool dup = false;
#pragma unroll 8
                    for (int k = 0; k < i; ++k) dup |= sm.us[k] == u && sm.pass[k];
                    ok = !dup;
                }
                sm.acc[i] = ok;
                if (ok) {
                    a.X[i] = u;
                    a.FX[i] = fit[i];
                    ++n_acc;
                    if (last < 0 || fit[i] <= lf) { last = i; lf = fit[i]; }
                }
            }
            const int w = block_argmin(last >= 0 ? lf : 0.0f, last, true, sm);
            n_acc = __reduce_add_sync(0xffffffffu, n_acc);
            if ((t & 31) == 0) sm.ri[t >> 5] = n_acc;
            __syncthreads();
            if (t == 0) {
                int total = 0;
                for (int k = 0; k < nw; ++k) total += sm.ri[k];
                if (w >= 0 && fit[w] <= st->de_fbest) { st->de_best = sm.us[w]; st->de_fbest = fit[w]; }
                st->stag = total ? 0 : st->stag + 1;
                if (st->stag >= 2) { st->reinit_pending = 1; st->stag = 0; }
            }
        }
    } else if (a.kind == CT_PSO || a.kind == CT_FIREFLY) {
        if (gen == 0) {
            for (int i = t; i < P; i += nt) {
                uint32_t w[4];
                for (int j = 0; j < N; ++j) {
                    const float x0 = a.prm.constraint_aware ? __fmul_rn((float)field(a.sp, sm.us[i], j), a.eps)
                                                            : a.pos[(size_t)i * N + j];
                    a.pos[(size_t)i * N + j] = x0;
                    a.pb[(size_t)i * N + j] = x0;
                    if (a.kind == CT_PSO) {
                        if ((j & 3) == 0) rng_block(a.seed, i, 0, PU_PSO_VEL, (uint32_t)j >> 2, w);
                        a.vel[(size_t)i * N + j] = __fmul_rn(__fsub_rn(__fmul_rn(2.0f, u01(w[j & 3])), 1.0f), a.eps);
                    }
                }
                a.fpb[i] = fit[i];
                a.FX[i] = fit[i];
            }
        } else if (a.kind == CT_PSO) {
            for (int i = t; i < P; i += nt)
                if (fit[i] < a.fpb[i]) {
                    a.fpb[i] = fit[i];
                    for (int j = 0; j < N; ++j) a.pb[(size_t)i * N + j] = a.pos[(size_t)i * N + j];
                }
        } else {
            for (int i = t; i < P; i += nt) {
                for (int j = 0; j < N; ++j) a.pos[(size_t)i * N + j] = a.ynew[(size_t)i * N + j];
                a.FX[i] = fit[i];
            }
        }
        __syncthreads();
        if (a.kind == CT_PSO) {
            int first = -1;
            float ff = 0.0f;
            for (int i = t; i < P; i += nt)
                if (first < 0 || a.fpb[i] < ff) { first = i; ff = a.fpb[i]; }   // ascending i: ties keep the earlier
            const int w = block_argmin(first >= 0 ? ff : 0.0f, first, false, sm);
            __shared__ int upd;
            if (t == 0) {
                upd = w >= 0 && a.fpb[w] < st->fgb;
                if (upd) st->fgb = a.fpb[w];
            }
            __syncthreads();
            if (upd)
                for (int j = t; j < N; j += nt) a.gb[j] = a.pb[(size_t)w * N + j];
        }
        for (int i = t; i < P; i += nt) {
            a.X[i] = sm.us[i];
            if (a.kind == CT_PSO) a.FX[i] = a.fpb[i];
        }
    } else {  // GA: generational replacement
        for (int i = t; i < P; i += nt) { a.X[i] = sm.us[i]; a.FX[i] = fit[i]; }
    }
    __syncthreads();
    if (t == 0) st->gen = gen + 1;
    __syncthreads();
}


struct SurrogateState;
void surrogate_free(SurrogateState* sg);

}  // namespace ct

using ct::DevBuf;
using ct::OptArgs;
using ct::OptDev;
using ct::RepairScratch;

struct ct_opt {
    ct_space* s = nullptr;
    int kind = 0, P = 0, N = 0;
    uint64_t seed = 0;
    ct_opt_params prm{};
    float eps = 1.0f;
    DevBuf<OptDev> st;
    DevBuf<uint64_t> X, cand, rep;
    DevBuf<float> FX, pos, vel, pb, fpb, gb, ynew, fit;
    DevBuf<uint32_t> memo;
    size_t memo_words = 0;
    std::map<uint32_t, cudaGraphExec_t> graphs;
    std::map<uint32_t, uint64_t> graph_kernels;   // kernels per replay of each graph
    // What the graphs captured from the space: key buffer, fitness and cost tables, |V| and the
    // repair strategy (its ball radii).  Any change drops them.
    struct GraphSig {
        const void* keys = nullptr;
        const void* fit = nullptr;
        const void* cost = nullptr;
        uint64_t nv = 0;
        int mode = -1, max_radius = -1, dmax = -1;
        bool operator==(const GraphSig& o) const {
            return keys == o.keys && fit == o.fit && cost == o.cost && nv == o.nv && mode == o.mode &&
                   max_radius == o.max_radius && dmax == o.dmax;
        }
    } graph_sig;
    uint32_t eager_steps = 0;                     // ct_opt_step calls that launched kernel by kernel
    uint32_t dev_gen = ~0u;                       // the generation the device state holds next (~0: unknown)
    RepairScratch rs;                             // run-owned repair scratch (fixed size: pop)
    ct::RuleScratch rules;                        // paper's repair rules (repair_rule = 1)
    ct::SurrogateState* sg = nullptr;             // MLP surrogate screening (DE, GA), or none
    // The device state is initialised asynchronously on the legacy default stream at creation;
    // `ready` is recorded after it, and the first use on another stream waits for it.
    cudaEvent_t ready = nullptr;
    mutable cudaStream_t ready_on = nullptr;      // the stream that last waited for `ready`
    mutable bool ready_seen = false;
    ~ct_opt() {
        if (ready) cudaEventDestroy(ready);
        ct::surrogate_free(sg);
        rules.release_all();
        for (auto& g : graphs) cudaGraphExecDestroy(g.second);
        st.release(); X.release(); cand.release(); rep.release(); FX.release(); pos.release(); vel.release();
        pb.release(); fpb.release(); gb.release(); ynew.release(); fit.release(); memo.release();
        rs.release_all();
    }
    // Orders stream st after the run's initialisation (a no-op once st has waited).
    ct_status wait_ready(cudaStream_t st) const {
        if (ready_seen && ready_on == st) return CT_OK;
        if (cudaStreamWaitEvent(st, ready, 0) != cudaSuccess) {
            ct::set_error("waiting for the run's initialisation failed");
            return CT_ERR_CUDA;
        }
        ready_seen = true;
        ready_on = st;
        return CT_OK;
    }
    OptArgs args() const {
        OptArgs a;
        a.kind = kind; a.P = P; a.N = N; a.seed = seed; a.prm = prm; a.eps = eps;
        a.sp = s->d; a.tables = s->tables.p; a.keys = s->keys.p; a.nv = (int64_t)s->n_valid;
        a.st = st.p; a.X = X.p; a.FX = FX.p; a.pos = pos.p; a.vel = vel.p; a.pb = pb.p; a.fpb = fpb.p; a.gb = gb.p;
        a.ynew = ynew.p;
        return a;
    }
};

