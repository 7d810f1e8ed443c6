/*
 * CPU ORACLE — TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct restatement of what the constraint-aware
 * auto-tuning hot path computes ("Constraint-aware Optimization in
 * Auto-Tuning", Sections IV-A..IV-D, Algorithms 1 and 3, Table IV).  Only the
 * test-suite, the package smoke check and the benchmark's CPU-baseline leg use
 * it.  It shares no code with the CUDA library: its own expression-tree
 * evaluator, its own key layout, its own Philox, its own exp.
 *
 * Conventions (double as the reading of the paper where it is silent):
 *   - a configuration is a tuple of value *indices* idx_k in [0, r_k);
 *   - key K = sum_k idx_k << off_k, param n-1 in the lowest bits, each field
 *     ceil(log2 r_k) bits wide (0 bits when r_k == 1);
 *   - the valid space V is every tuple whose constraints all hold (Section
 *     IV-A, CSP P=(X,D,C)), listed in increasing key order (= Cartesian order
 *     with the last parameter fastest);
 *   - constraint arithmetic is 64-bit two's complement, / and % truncate toward
 *     zero, a division or modulo by zero poisons the sub-expression;
 *   - fitness is a runtime: lower is better (Algorithm 1 accepts f(u) <= f(x)).
 *
 * Pins (tests/test_oracle_*.py): hand-counted tiny space, closed-form large
 * space, brute-force medium count, Philox known-answer vectors, exp error bound,
 * exhaustive repair invariants, optimizer reduction cases and rerun determinism.
 * The paper prints no optimizer trace, so each update rule is pinned on its own
 * (tests/test_oracle_moves.py): the PSO velocity carry and its cognitive and
 * social terms, the Firefly attraction and noise, each isolated at
 * hyper-parameters where the other terms vanish, and DE's acceptance and best
 * update replayed from the trace of whole runs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXP 64

/* ------------------------------------------------------------------------- */
/* constraint expression trees (the oracle's own format)                       */
/* ------------------------------------------------------------------------- */
enum {
    N_CONST = 0, N_PARAM, N_ADD, N_SUB, N_MUL, N_DIV, N_MOD, N_NEG, N_MIN, N_MAX,
    N_LT, N_LE, N_GT, N_GE, N_EQ, N_NE, N_AND, N_OR, N_NOT
};

typedef struct {
    int32_t op;
    int32_t a, b;   /* child node indices (-1 if unused); for N_PARAM, a = param index */
    int32_t pad;
    int64_t imm;
} or_node;

typedef struct {
    int64_t v;
    int poison;
} val_t;

static val_t eval_node(const or_node *nodes, int at, const int64_t *pv)
{
    const or_node *nd = &nodes[at];
    val_t r = {0, 0}, x, y;
    switch (nd->op) {
    case N_CONST: r.v = nd->imm; return r;
    case N_PARAM: r.v = pv[nd->a]; return r;
    case N_NEG:
        x = eval_node(nodes, nd->a, pv);
        r.v = (int64_t)(0ull - (uint64_t)x.v); r.poison = x.poison; return r;
    case N_NOT:
        x = eval_node(nodes, nd->a, pv);
        r.v = (x.poison || x.v == 0) ? 1 : 0; return r;
    default: break;
    }
    x = eval_node(nodes, nd->a, pv);
    y = eval_node(nodes, nd->b, pv);
    int p = x.poison | y.poison;
    int xt = !x.poison && x.v != 0, yt = !y.poison && y.v != 0;
    switch (nd->op) {
    case N_ADD: r.v = (int64_t)((uint64_t)x.v + (uint64_t)y.v); r.poison = p; break;
    case N_SUB: r.v = (int64_t)((uint64_t)x.v - (uint64_t)y.v); r.poison = p; break;
    case N_MUL: r.v = (int64_t)((uint64_t)x.v * (uint64_t)y.v); r.poison = p; break;
    case N_DIV:
    case N_MOD:
        if (p || y.v == 0) { r.poison = 1; break; }
        if (x.v == INT64_MIN && y.v == -1) { r.v = (nd->op == N_DIV) ? INT64_MIN : 0; break; }
        r.v = (nd->op == N_DIV) ? x.v / y.v : x.v % y.v;   /* C99: truncation */
        break;
    case N_MIN: r.v = x.v < y.v ? x.v : y.v; r.poison = p; break;
    case N_MAX: r.v = x.v > y.v ? x.v : y.v; r.poison = p; break;
    case N_LT: r.v = !p && x.v < y.v; break;
    case N_LE: r.v = !p && x.v <= y.v; break;
    case N_GT: r.v = !p && x.v > y.v; break;
    case N_GE: r.v = !p && x.v >= y.v; break;
    case N_EQ: r.v = !p && x.v == y.v; break;
    case N_NE: r.v = !p && x.v != y.v; break;
    case N_AND: r.v = xt && yt; break;
    case N_OR: r.v = xt || yt; break;
    default: r.poison = 1; break;
    }
    return r;
}

/* ------------------------------------------------------------------------- */
/* key layout                                                                 */
/* ------------------------------------------------------------------------- */
static int ceil_log2(int64_t r)
{
    int w = 0;
    while (((int64_t)1 << w) < r) w++;
    return w;
}

/* Writes widths/offsets; returns total key bits. */
int or_key_layout(int n, const int32_t *r, int32_t *width, int32_t *offset)
{
    int total = 0;
    for (int k = n - 1; k >= 0; k--) {
        width[k] = ceil_log2(r[k]);
        offset[k] = total;
        total += width[k];
    }
    return total;
}

typedef struct {
    int n;
    int32_t r[OR_MAXP], w[OR_MAXP], off[OR_MAXP];
    int bits;
} layout_t;

static void make_layout(layout_t *L, int n, const int32_t *r)
{
    L->n = n;
    memcpy(L->r, r, sizeof(int32_t) * n);
    L->bits = or_key_layout(n, r, L->w, L->off);
}

static uint64_t pack(const layout_t *L, const int32_t *idx)
{
    uint64_t k = 0;
    for (int i = 0; i < L->n; i++) k |= (uint64_t)idx[i] << L->off[i];
    return k;
}

static void unpack(const layout_t *L, uint64_t key, int32_t *idx)
{
    for (int i = 0; i < L->n; i++) {
        uint64_t m = L->w[i] ? ((L->w[i] == 64) ? ~0ull : ((1ull << L->w[i]) - 1)) : 0;
        idx[i] = (int32_t)((key >> L->off[i]) & m);
    }
}

/* 1 if every field is inside its domain and no bit above the key width is set */
static int key_in_domain(const layout_t *L, uint64_t key)
{
    if (L->bits < 64 && (key >> L->bits) != 0) return 0;
    int32_t idx[OR_MAXP];
    unpack(L, key, idx);
    for (int i = 0; i < L->n; i++)
        if (idx[i] >= L->r[i]) return 0;
    return 1;
}

/* ------------------------------------------------------------------------- */
/* brute-force enumeration (Section IV-A: resolve the whole space up front)   */
/* ------------------------------------------------------------------------- */
/* Visits Cartesian indices c in [c_lo, c_hi) in order; a point is valid iff all
 * m constraints (roots[j]) are true.  Writes the keys of valid points (if out is
 * non-NULL, at most cap) and returns how many valid points there are. */
int64_t or_enumerate(int n, const int32_t *r, const int64_t *values, const int32_t *vstart,
                     const or_node *nodes, const int32_t *roots, int m,
                     int64_t c_lo, int64_t c_hi, uint64_t *out, int64_t cap)
{
    layout_t L;
    make_layout(&L, n, r);
    int32_t idx[OR_MAXP];
    int64_t pv[OR_MAXP];
    int64_t count = 0;
    for (int64_t c = c_lo; c < c_hi; c++) {
        int64_t t = c;
        for (int k = n - 1; k >= 0; k--) {      /* mixed radix, last param fastest */
            idx[k] = (int32_t)(t % r[k]);
            t /= r[k];
        }
        for (int k = 0; k < n; k++) pv[k] = values[vstart[k] + idx[k]];
        int ok = 1;
        for (int j = 0; j < m && ok; j++) {
            val_t v = eval_node(nodes, roots[j], pv);
            ok = !v.poison && v.v != 0;
        }
        if (!ok) continue;
        if (out && count < cap) out[count] = pack(&L, idx);
        count++;
    }
    return count;
}

/* evaluate the constraints for explicit index tuples (rows of n), 1 = valid */
void or_check_tuples(int n, const int32_t *r, const int64_t *values, const int32_t *vstart,
                     const or_node *nodes, const int32_t *roots, int m,
                     const int32_t *tuples, int64_t count, uint8_t *valid_out)
{
    int64_t pv[OR_MAXP];
    for (int64_t i = 0; i < count; i++) {
        const int32_t *idx = tuples + i * n;
        int ok = 1;
        for (int k = 0; k < n; k++) {
            if (idx[k] < 0 || idx[k] >= r[k]) { ok = 0; break; }
            pv[k] = values[vstart[k] + idx[k]];
        }
        for (int j = 0; j < m && ok; j++) {
            val_t v = eval_node(nodes, roots[j], pv);
            ok = !v.poison && v.v != 0;
        }
        valid_out[i] = (uint8_t)ok;
    }
}

/* ------------------------------------------------------------------------- */
/* validity / rank lookup (Section IV-A: "query whether a solution is valid") */
/* ------------------------------------------------------------------------- */
static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

static int64_t rank_of(const uint64_t *keys, int64_t nv, uint64_t key)
{
    const uint64_t *p = (const uint64_t *)bsearch(&key, keys, (size_t)nv, sizeof(uint64_t), cmp_u64);
    return p ? (int64_t)(p - keys) : -1;
}

void or_lookup(const uint64_t *keys, int64_t nv, const uint64_t *cand, int64_t nc, int64_t *rank_out)
{
    for (int64_t i = 0; i < nc; i++) rank_out[i] = rank_of(keys, nv, cand[i]);
}

/* ------------------------------------------------------------------------- */
/* nearest-valid repair: argmin over V of (Hamming distance, key)             */
/* ------------------------------------------------------------------------- */
static int hamming(const layout_t *L, const int32_t *a, const int32_t *b)
{
    int d = 0;
    for (int i = 0; i < L->n; i++) d += a[i] != b[i];
    return d;
}

/* The plain definition: scan all of V.  `vt` holds V's index tuples row-wise. */
static uint64_t repair_one(const layout_t *L, const uint64_t *keys, const int32_t *vt, int64_t nv,
                           uint64_t cand, int *dist_out)
{
    int32_t u[OR_MAXP];
    unpack(L, cand, u);
    int best_d = L->n + 1;
    int64_t best_i = -1;
    for (int64_t i = 0; i < nv; i++) {
        const int32_t *v = vt + i * L->n;
        int d = 0;
        for (int k = 0; k < L->n && d < best_d; k++) d += u[k] != v[k];
        if (d < best_d) { best_d = d; best_i = i; }   /* keys ascend: first hit = smallest key */
    }
    *dist_out = best_d;
    return best_i >= 0 ? keys[best_i] : cand;
}

static int32_t *tuples_of(const layout_t *L, const uint64_t *keys, int64_t nv)
{
    int32_t *vt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1) * L->n);
    for (int64_t i = 0; i < nv; i++) unpack(L, keys[i], vt + i * L->n);
    return vt;
}

/* returns 0, or -1 if some candidate is outside the Cartesian domain */
int or_repair(int n, const int32_t *r, const uint64_t *keys, int64_t nv,
              const uint64_t *cand, int64_t nc, uint64_t *out, uint8_t *dist)
{
    layout_t L;
    make_layout(&L, n, r);
    for (int64_t i = 0; i < nc; i++)
        if (!key_in_domain(&L, cand[i])) return -1;
    if (nv == 0) return -2;
    int32_t *vt = tuples_of(&L, keys, nv);
    for (int64_t i = 0; i < nc; i++) {
        int d;
        out[i] = repair_one(&L, keys, vt, nv, cand[i], &d);
        dist[i] = (uint8_t)d;
    }
    free(vt);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)                           */
/* ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    /* round multipliers and Weyl key increments as published with the generator */
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

enum {
    P_INIT = 1, P_MUT_PICK = 2, P_CROSS = 3, P_PSO_R = 4, P_FA_ALPHA = 5, P_GA_SEL = 6,
    P_GA_CUT = 7, P_GA_MUT = 8, P_REINIT = 9, P_POOL = 10, P_MLP_INIT = 11, P_MLP_BATCH = 12,
    P_PSO_VEL = 13, P_GA_REPAIR = 14, P_RAND_INIT = 15
};

/* static penalty of an invalid configuration in the non-constraint-aware runs (the
 * magnitude of Kernel Tuner's default, positive because fitness is minimised) */
#define OR_PENALTY 1e20f

/* word t of the stream (individual, generation, purpose) under seed */
static uint32_t rng_word(uint64_t seed, uint32_t indiv, uint32_t gen, uint32_t purpose, uint32_t t)
{
    uint32_t ctr[4] = {t / 4u, indiv, gen, purpose};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    or_philox4x32_10(ctr, key, o);
    return o[t % 4u];
}

uint32_t or_rng_word(uint64_t seed, uint32_t indiv, uint32_t gen, uint32_t purpose, uint32_t t)
{
    return rng_word(seed, indiv, gen, purpose, t);
}

static float u01(uint32_t w) { return (float)(w >> 8) * (1.0f / 16777216.0f); }
static uint32_t uint_below(uint32_t w, uint32_t n) { return (uint32_t)(((uint64_t)w * n) >> 32); }
static uint64_t uint64_below(uint32_t whi, uint32_t wlo, uint64_t n)
{
    unsigned __int128 x = ((unsigned __int128)(((uint64_t)whi << 32) | wlo)) * n;
    return (uint64_t)(x >> 64);
}

/* ------------------------------------------------------------------------- */
/* exp for the Firefly attractiveness: Cody-Waite range reduction + Taylor    */
/* ------------------------------------------------------------------------- */
/* x <= 0.  n = rint(x*log2(e)); r = (x - n*LN2_HI) - n*LN2_LO; p = degree-7
 * Taylor polynomial of e^r by Horner; result p * 2^n.  Every float operation
 * is a separately rounded binary32 op.  x < -80 returns 0. */
float or_exp_ct(float x)
{
    if (!(x >= -80.0f)) return 0.0f;
    if (x > 0.0f) x = 0.0f;
    const float LOG2E = 1.44269504088896340736f;
    const float LN2_HI = 0.693145751953125f;            /* 11 significant bits: n*LN2_HI exact */
    const float LN2_LO = 1.42860682030941723212e-6f;    /* ln 2 - LN2_HI */
    float nf = rintf(x * LOG2E);
    float r = (x - nf * LN2_HI) - nf * LN2_LO;
    float p = 1.0f / 5040.0f;
    p = p * r + 1.0f / 720.0f;
    p = p * r + 1.0f / 120.0f;
    p = p * r + 1.0f / 24.0f;
    p = p * r + 1.0f / 6.0f;
    p = p * r + 0.5f;
    p = p * r + 1.0f;
    p = p * r + 1.0f;
    int n = (int)nf;
    union { uint32_t u; float f; } s;
    s.u = (uint32_t)(n + 127) << 23;   /* 2^n, n in [-116, 0] */
    return p * s.f;
}

/* ------------------------------------------------------------------------- */
/* the four constraint-aware optimizers                                       */
/* ------------------------------------------------------------------------- */
enum { K_DE = 0, K_PSO = 1, K_FIREFLY = 2, K_GA = 3 };

typedef struct {
    float de_F, de_CR;
    float pso_w, pso_c1, pso_c2;
    float fa_beta0, fa_gamma, fa_alpha;
    float ga_pmut;
    float target;        /* record unique evaluations when best <= target */
    int repair_rule;     /* 0: Hamming argmin for all; 1: the paper's rule per optimizer */
    int aware;           /* 1: constraint-aware; 0: random Cartesian start, no repair, penalty */
    int de_mutation;     /* 0 best1, 1 rand1, 2 rand2, 3 best2, 4 currenttobest1, 5 randtobest1 */
    int de_crossover;    /* 0 binomial, 1 exponential */
    int ga_crossover;    /* 0 single point, 1 two point, 2 uniform, 3 disruptive uniform */
    const uint32_t *cost; /* simulated time of evaluating each valid configuration (per rank), or NULL */
} or_params;

typedef struct {         /* per-generation trace, arrays of (G+1) x P unless noted */
    uint64_t *cand;      /* proposed (before repair) */
    uint64_t *rep;       /* after repair */
    uint64_t *evalk;     /* evaluated key (GA: after mutation; others = rep) */
    float *fit;          /* fitness of evalk */
    uint64_t *popk;      /* population keys after selection (DE, GA) */
    float *popf;         /* population fitness after selection */
    float *pos;          /* PSO / Firefly positions after the generation, (G+1) x P x n */
    uint64_t *best_key;  /* (G+1): run best over evaluations, min (f, key) */
    float *best_fit;     /* (G+1) */
    uint64_t *n_unique;  /* (G+1) */
    int64_t *hit;        /* [0] generation of first best<=target (-1), [1] n_unique then */
    uint64_t *cost;      /* (G+1): simulated time spent so far, the sum of the costs of the
                            configurations evaluated (each once) */
    /* every strict improvement of the run's best, in evaluation order (capacity P x (G+1)):
     * generation, population index, simulated time after that evaluation, new best */
    int32_t *ev_gen, *ev_idx;
    uint64_t *ev_clock;
    float *ev_fit;
    int64_t *ev_n;       /* [0]: number of events */
} or_trace;

typedef struct {
    layout_t L;
    const uint64_t *keys;
    int64_t nv;
    int32_t *vt;
    const float *table;
    uint8_t *memo;
    uint64_t n_unique;
    uint64_t best_key;
    float best_fit;
    const uint32_t *cost_tab;
    uint64_t cost;
    const or_trace *T;   /* event log */
    int g, i;            /* generation and population index being evaluated */
} ctx_t;

static float evaluate(ctx_t *C, uint64_t key)
{
    int64_t rk = rank_of(C->keys, C->nv, key);
    float f;
    if (rk < 0) {
        f = OR_PENALTY;                     /* only without constraint awareness: nothing is run */
    } else {
        if (!C->memo[rk]) {
            C->memo[rk] = 1;
            C->n_unique++;
            if (C->cost_tab) C->cost += C->cost_tab[rk];   /* a configuration is compiled and run once */
        }
        f = C->table[rk];
    }
    if (f < C->best_fit && C->T) {          /* the best value improves: log it */
        int64_t e = C->T->ev_n[0]++;
        C->T->ev_gen[e] = C->g;
        C->T->ev_idx[e] = C->i;
        C->T->ev_clock[e] = C->cost;
        C->T->ev_fit[e] = f;
    }
    if (f < C->best_fit || (f == C->best_fit && key < C->best_key)) {
        C->best_fit = f;
        C->best_key = key;
    }
    return f;
}

static uint64_t repair_key(ctx_t *C, uint64_t key);

/* ---- the paper's neighbour rules (Section IV-A) and repairs (Algorithms 1-3) ---- */

/* values of each parameter that occur in some valid configuration (bit v of occ[k]) */
static void occurring_values(ctx_t *C, uint8_t *occ /* n x 4096 */)
{
    memset(occ, 0, (size_t)C->L.n * 4096);
    for (int64_t i = 0; i < C->nv; i++)
        for (int k = 0; k < C->L.n; k++) occ[(size_t)k * 4096 + C->vt[i * C->L.n + k]] = 1;
}

/* 1: every parameter identical or the previous/next value index (strictly adjacent);
 * 2: every parameter identical or the nearest lower/higher value occurring in V (adjacent);
 * 3: exactly one parameter differs (Hamming).  u itself is never a neighbour. */
static int in_rule(const ctx_t *C, const uint8_t *occ, const int32_t *u, const int32_t *v, int rule)
{
    int ndiff = 0;
    for (int k = 0; k < C->L.n; k++) {
        int d = v[k] - u[k];
        if (d == 0) continue;
        ndiff++;
        if (rule == 1 && (d > 1 || d < -1)) return 0;
        if (rule == 2) {
            int lo = -1, hi = -1;
            for (int t = u[k] - 1; t >= 0; t--) if (occ[(size_t)k * 4096 + t]) { lo = t; break; }
            for (int t = u[k] + 1; t < C->L.r[k]; t++) if (occ[(size_t)k * 4096 + t]) { hi = t; break; }
            if (v[k] != lo && v[k] != hi) return 0;
        }
    }
    if (ndiff == 0) return 0;
    return rule == 3 ? ndiff == 1 : 1;
}

/* DE (Algorithm 1 Repair, Section IV-B): the valid configuration with the smallest sum of
 * absolute value-index differences; ties to the smallest key. */
static uint64_t repair_l1(ctx_t *C, uint64_t key)
{
    if (rank_of(C->keys, C->nv, key) >= 0) return key;
    int32_t u[OR_MAXP];
    unpack(&C->L, key, u);
    int64_t best = -1;
    int bd = 1 << 30;
    for (int64_t i = 0; i < C->nv; i++) {
        const int32_t *v = C->vt + i * C->L.n;
        int d = 0;
        for (int k = 0; k < C->L.n; k++) d += v[k] > u[k] ? v[k] - u[k] : u[k] - v[k];
        if (d < bd) { bd = d; best = i; }
    }
    return C->keys[best];
}

/* PSO / Firefly (Algorithm 2): the first non-empty neighbour set of the snapped point, the
 * member closest to the position x in continuous space (ties to the smallest key). */
static uint64_t repair_alg2(ctx_t *C, const uint8_t *occ, uint64_t key, const float *x, float eps)
{
    if (rank_of(C->keys, C->nv, key) >= 0) return key;
    int32_t u[OR_MAXP];
    unpack(&C->L, key, u);
    for (int rule = 1; rule <= 3; rule++) {
        int64_t best = -1;
        float bd = 0.0f;
        for (int64_t i = 0; i < C->nv; i++) {
            const int32_t *v = C->vt + i * C->L.n;
            if (!in_rule(C, occ, u, v, rule)) continue;
            float s = 0.0f;
            for (int k = 0; k < C->L.n; k++) {
                float d = (float)v[k] * eps - x[k];
                s = s + d * d;
            }
            if (best < 0 || s < bd) { bd = s; best = i; }
        }
        if (best >= 0) return C->keys[best];
    }
    return repair_key(C, key);   /* no neighbour in any set: the nearest valid (Hamming) */
}

/* GA (Algorithm 3): a uniformly random member (U[0, |n|) from word w, in key order) of the
 * first non-empty neighbour set. */
static uint64_t repair_alg3(ctx_t *C, const uint8_t *occ, uint64_t key, uint32_t w)
{
    if (rank_of(C->keys, C->nv, key) >= 0) return key;
    int32_t u[OR_MAXP];
    unpack(&C->L, key, u);
    for (int rule = 1; rule <= 3; rule++) {
        int64_t cnt = 0;
        for (int64_t i = 0; i < C->nv; i++) cnt += in_rule(C, occ, u, C->vt + i * C->L.n, rule);
        if (!cnt) continue;
        int64_t pick = (int64_t)uint_below(w, (uint32_t)cnt), seen = 0;
        for (int64_t i = 0; i < C->nv; i++)
            if (in_rule(C, occ, u, C->vt + i * C->L.n, rule) && seen++ == pick) return C->keys[i];
    }
    return repair_key(C, key);
}

static uint64_t repair_key(ctx_t *C, uint64_t key)
{
    if (rank_of(C->keys, C->nv, key) >= 0) return key;
    int d;
    return repair_one(&C->L, C->keys, C->vt, C->nv, key, &d);
}

/* valid-space sample: one rank per stratum [k|V|/P, (k+1)|V|/P) (reading of the LHS
 * initialisation of Section IV-B over the resolved valid list) */
static uint64_t stratified_key(ctx_t *C, uint64_t seed, uint32_t k, uint32_t P, uint32_t gen,
                               uint32_t purpose)
{
    uint64_t lo = (uint64_t)(((unsigned __int128)k * (uint64_t)C->nv) / P);
    uint64_t hi = (uint64_t)(((unsigned __int128)(k + 1) * (uint64_t)C->nv) / P);
    uint64_t off = 0;
    if (hi > lo) {
        uint32_t w0 = rng_word(seed, k, gen, purpose, 0), w1 = rng_word(seed, k, gen, purpose, 1);
        off = uint64_below(w1, w0, hi - lo);
    }
    return C->keys[lo + off];
}

/* Beta(1,3)-shaped rank selection: smallest k with w*P^3 < 2^32*(P^3-(P-k-1)^3) */
static uint32_t beta_pick(uint32_t w, uint32_t P)
{
    uint64_t P3 = (uint64_t)P * P * P;
    for (uint32_t k = 0; k < P; k++) {
        uint64_t q = (uint64_t)(P - k - 1);
        unsigned __int128 lhs = (unsigned __int128)w * P3;
        unsigned __int128 rhs = ((unsigned __int128)(P3 - q * q * q)) << 32;
        if (lhs < rhs) return k;
    }
    return P - 1;
}

static void record(ctx_t *C, const or_trace *T, int g, int P, const or_params *prm)
{
    (void)P;
    T->best_key[g] = C->best_key;
    T->best_fit[g] = C->best_fit;
    T->n_unique[g] = C->n_unique;
    T->cost[g] = C->cost;
    if (T->hit[0] < 0 && C->best_fit <= prm->target) {
        T->hit[0] = g;
        T->hit[1] = (int64_t)C->n_unique;
    }
}

static float coord_eps(const layout_t *L)
{
    int rmax = 1;
    for (int k = 0; k < L->n; k++) rmax = L->r[k] > rmax ? L->r[k] : rmax;
    return rmax > 1 ? 1.0f / (float)(rmax - 1) : 1.0f;
}

static uint64_t snap_key(const layout_t *L, const float *x, float eps)
{
    int32_t idx[OR_MAXP];
    for (int k = 0; k < L->n; k++) {
        float q = rintf(x[k] / eps);
        int v = (int)q;
        if (q < 0.0f) v = 0;
        if (v > L->r[k] - 1) v = L->r[k] - 1;
        idx[k] = v;
    }
    return pack(L, idx);
}

static float clip01(float v) { return v < 0.0f ? 0.0f : (v > 1.0f ? 1.0f : v); }


void or_mlp_forward(const float *params, int D, int H, int N, const int32_t *feats, int B, float *pred, float *acts);
void or_mlp_grad(const float *params, int D, int H, int N, const int32_t *feats, const float *y, int B, float *grad);
void or_mlp_sgd(float *params, float *mom, const float *grad, int64_t n, float lr, float mu);
void or_mlp_init(int D, int H, uint64_t seed, float *params);
int64_t or_mlp_param_count(int D, int H);

/* DE best1bin trial for target i, drawing from the RNG streams of individual si
 * (si = i for the plain method; i + s*P for proposal s of a surrogate pool). */
/* k distinct population indices other than i, each uniform over what is left: draw t takes
 * word t of MUT_PICK below P-1-t and steps over the excluded indices in ascending order */
static void de_picks(int P, int i, int k, uint64_t seed, uint32_t si, int g, uint32_t *r)
{
    uint32_t ex[8];
    int ne = 1;
    ex[0] = (uint32_t)i;
    for (int t = 0; t < k; t++) {
        uint32_t v = uint_below(rng_word(seed, si, g, P_MUT_PICK, (uint32_t)t), (uint32_t)(P - 1 - t));
        for (int e = 0; e < ne; e++)
            if (v >= ex[e]) v++;
        r[t] = v;
        int p = ne++;                              /* keep ex sorted */
        while (p > 0 && ex[p - 1] > v) { ex[p] = ex[p - 1]; p--; }
        ex[p] = v;
    }
}

/* random partners each DE mutation uses */
int or_de_partners(int mutation)
{
    static const int k[6] = {2, 3, 5, 4, 2, 3};   /* best1 rand1 rand2 best2 currenttobest1 randtobest1 */
    return mutation >= 0 && mutation < 6 ? k[mutation] : -1;
}

static uint64_t de_trial(ctx_t *C, const uint64_t *X, uint64_t de_best, int P, int i, uint32_t si, int g,
                         uint64_t seed, const or_params *prm)
{
    const int N = C->L.n;
    const float F = prm->de_F;
    int32_t best[OR_MAXP], xi[OR_MAXP], x[5][OR_MAXP], v[OR_MAXP], t[OR_MAXP];
    uint32_t r[5];
    const int k = or_de_partners(prm->de_mutation);
    de_picks(P, i, k, seed, si, g, r);
    unpack(&C->L, de_best, best);
    unpack(&C->L, X[i], xi);
    for (int q = 0; q < k; q++) unpack(&C->L, X[r[q]], x[q]);
    /* Mutate (Algorithm 1 and the variants of Section IV-B), on value indices in fp32, one
     * rounding per operation in the order written, then round half-even and clip */
    for (int j = 0; j < N; j++) {
        float m;
        switch (prm->de_mutation) {
        case 0:  /* best1: best + F (x0 - x1) */
            m = (float)best[j] + F * (float)(x[0][j] - x[1][j]);
            break;
        case 1:  /* rand1: x0 + F (x1 - x2) */
            m = (float)x[0][j] + F * (float)(x[1][j] - x[2][j]);
            break;
        case 2:  /* rand2: x0 + F (x1 - x2) + F (x3 - x4) */
            m = ((float)x[0][j] + F * (float)(x[1][j] - x[2][j])) + F * (float)(x[3][j] - x[4][j]);
            break;
        case 3:  /* best2: best + F (x0 - x1) + F (x2 - x3) */
            m = ((float)best[j] + F * (float)(x[0][j] - x[1][j])) + F * (float)(x[2][j] - x[3][j]);
            break;
        case 4:  /* currenttobest1: xi + F (best - xi) + F (x0 - x1) */
            m = ((float)xi[j] + F * (float)(best[j] - xi[j])) + F * (float)(x[0][j] - x[1][j]);
            break;
        default: /* randtobest1: x0 + F (best - x0) + F (x1 - x2) */
            m = ((float)x[0][j] + F * (float)(best[j] - x[0][j])) + F * (float)(x[1][j] - x[2][j]);
            break;
        }
        float q = rintf(m);
        int vv = (int)q;
        if (q < 0.0f) vv = 0;
        if (vv > C->L.r[j] - 1) vv = C->L.r[j] - 1;
        v[j] = vv;
    }
    uint32_t j0 = uint_below(rng_word(seed, si, g, P_CROSS, 0), (uint32_t)N);
    if (prm->de_crossover == 0) {
        /* binomial (Algorithm 1, Crossover): gene j from v with probability CR, gene j0 always */
        for (int j = 0; j < N; j++) {
            float rr = u01(rng_word(seed, si, g, P_CROSS, 1 + (uint32_t)j));
            t[j] = (rr < prm->de_CR || (uint32_t)j == j0) ? v[j] : xi[j];
        }
    } else {
        /* exponential: from gene j0 on (cyclically) genes come from v; after the first, each
         * further one only while the draws stay below CR */
        for (int j = 0; j < N; j++) t[j] = xi[j];
        t[j0] = v[j0];
        for (int L = 1; L < N; L++) {
            if (!(u01(rng_word(seed, si, g, P_CROSS, (uint32_t)L)) < prm->de_CR)) break;
            int j = (int)((j0 + (uint32_t)L) % (uint32_t)N);
            t[j] = v[j];
        }
    }
    return pack(&C->L, t);
}

/* GA pair c: two beta-selected parents of the ranked population, single-point
 * crossover; streams of pair sc. */
static void ga_pair(ctx_t *C, const uint64_t *X, const int *order, int P, uint32_t sc, int g, uint64_t seed,
                    const or_params *prm, uint64_t *child0, uint64_t *child1)
{
    const int N = C->L.n;
    int32_t ia[OR_MAXP], ib[OR_MAXP], ic[OR_MAXP], id[OR_MAXP];
    uint8_t from_b[OR_MAXP];                 /* child0 takes gene j from the second parent */
    uint32_t pa = beta_pick(rng_word(seed, sc, g, P_GA_SEL, 0), (uint32_t)P);
    uint32_t pbi = beta_pick(rng_word(seed, sc, g, P_GA_SEL, 1), (uint32_t)P);
    unpack(&C->L, X[order[pa]], ia);
    unpack(&C->L, X[order[pbi]], ib);
    for (int j = 0; j < N; j++) from_b[j] = 0;
    int kind = prm->ga_crossover;
    if (kind == 1 && N < 3) kind = 0;       /* two cut points need three genes */
    if (kind == 0) {                         /* single point: genes from the cut on */
        uint32_t cut = N >= 2 ? 1 + uint_below(rng_word(seed, sc, g, P_GA_CUT, 0), (uint32_t)N - 1) : 1;
        for (int j = 0; j < N; j++) from_b[j] = (uint32_t)j >= cut;
    } else if (kind == 1) {                  /* two points: genes in [lo, hi) */
        uint32_t c1 = 1 + uint_below(rng_word(seed, sc, g, P_GA_CUT, 0), (uint32_t)N - 1);
        uint32_t c2 = 1 + uint_below(rng_word(seed, sc, g, P_GA_CUT, 1), (uint32_t)N - 2);
        if (c2 >= c1) c2++;
        uint32_t lo = c1 < c2 ? c1 : c2, hi = c1 < c2 ? c2 : c1;
        for (int j = 0; j < N; j++) from_b[j] = (uint32_t)j >= lo && (uint32_t)j < hi;
    } else if (kind == 2) {                  /* uniform: each gene by a fair draw */
        for (int j = 0; j < N; j++) from_b[j] = !(u01(rng_word(seed, sc, g, P_GA_CUT, (uint32_t)j)) < 0.5f);
    } else {                                 /* disruptive uniform: exactly half (rounded down) of
                                                the genes where the parents differ, chosen uniformly */
        int D[OR_MAXP], nd = 0;
        for (int j = 0; j < N; j++)
            if (ia[j] != ib[j]) D[nd++] = j;
        for (int t = 0; t < nd / 2; t++) {   /* partial Fisher-Yates over D */
            int s2 = t + (int)uint_below(rng_word(seed, sc, g, P_GA_CUT, (uint32_t)t), (uint32_t)(nd - t));
            int tmp = D[t]; D[t] = D[s2]; D[s2] = tmp;
            from_b[D[t]] = 1;
        }
    }
    for (int j = 0; j < N; j++) {
        ic[j] = from_b[j] ? ib[j] : ia[j];
        id[j] = from_b[j] ? ia[j] : ib[j];
    }
    *child0 = pack(&C->L, ic);
    *child1 = pack(&C->L, id);
}

/* GA mutation of a repaired child: with probability p_mut, a random valid Hamming
 * neighbour enumerated by (parameter, value index); streams of individual si. */
static uint64_t ga_mutate(ctx_t *C, uint64_t key, uint32_t si, int g, uint64_t seed, const or_params *prm)
{
    const int N = C->L.n;
    if (!(u01(rng_word(seed, si, g, P_GA_MUT, 0)) < prm->ga_pmut)) return key;
    int32_t ia[OR_MAXP];
    unpack(&C->L, key, ia);
    int64_t cnt = 0;
    for (int k = 0; k < N; k++)
        for (int v = 0; v < C->L.r[k]; v++) {
            if (v == ia[k]) continue;
            int32_t save = ia[k];
            ia[k] = v;
            if (rank_of(C->keys, C->nv, pack(&C->L, ia)) >= 0) cnt++;
            ia[k] = save;
        }
    if (cnt == 0) return key;
    uint32_t pick = uint_below(rng_word(seed, si, g, P_GA_MUT, 1), (uint32_t)cnt);
    int64_t seen = 0;
    for (int k = 0; k < N; k++)
        for (int v = 0; v < C->L.r[k]; v++) {
            if (v == ia[k]) continue;
            int32_t save = ia[k];
            ia[k] = v;
            uint64_t kk = pack(&C->L, ia);
            ia[k] = save;
            if (rank_of(C->keys, C->nv, kk) >= 0) {
                if (seen == (int64_t)pick) return kk;
                seen++;
            }
        }
    return key;
}

/* non-constraint-aware start: a uniform Cartesian tuple (stream RAND_INIT, word k) */
static uint64_t random_tuple(ctx_t *C, uint64_t seed, uint32_t i, uint32_t g)
{
    int32_t t[OR_MAXP];
    for (int k = 0; k < C->L.n; k++) t[k] = (int32_t)uint_below(rng_word(seed, i, g, P_RAND_INIT, (uint32_t)k), (uint32_t)C->L.r[k]);
    return pack(&C->L, t);
}

/* non-constraint-aware GA mutation: one random parameter takes one of its other values */
static uint64_t ga_mutate_plain(ctx_t *C, uint64_t key, uint32_t si, int g, uint64_t seed, const or_params *prm)
{
    if (!(u01(rng_word(seed, si, g, P_GA_MUT, 0)) < prm->ga_pmut)) return key;
    int32_t u[OR_MAXP];
    unpack(&C->L, key, u);
    int k = (int)uint_below(rng_word(seed, si, g, P_GA_MUT, 1), (uint32_t)C->L.n);
    if (C->L.r[k] < 2) return key;
    int v = (int)uint_below(rng_word(seed, si, g, P_GA_MUT, 2), (uint32_t)(C->L.r[k] - 1));
    u[k] = v < u[k] ? v : v + 1;
    return pack(&C->L, u);
}

/* surrogate configuration and per-generation trace */
typedef struct {
    int pool, H, batch, steps, warm_mult;
    float lr, mu, mae_ratio;
    const float *logt;   /* log-fitness per valid rank */
} or_surr;

typedef struct {
    int8_t *used;        /* (G+1): proposals were screened this generation */
    float *mae, *tau;    /* (G+1): judge of this generation */
    int64_t *n_e;        /* (G+1): evaluated-set size after appending */
    float *params;       /* final fp32 master parameters */
} or_strace;

static void feats_of(const ctx_t *C, uint64_t key, int32_t *f)
{
    int32_t idx[OR_MAXP];
    unpack(&C->L, key, idx);
    int base = 0;
    for (int k = 0; k < C->L.n; k++) { f[k] = base + idx[k]; base += C->L.r[k]; }
}

static float predict1(const ctx_t *C, const float *params, int D, int H, uint64_t key)
{
    int32_t f[OR_MAXP];
    float y;
    feats_of(C, key, f);
    or_mlp_forward(params, D, H, C->L.n, f, 1, &y, NULL);
    return y;
}

/* Direct access to the paper's repairs for the pins: rule 1 = index distance (DE),
 * 2 = Algorithm 2 with positions pos (nc x n) and grid spacing eps, 3 = Algorithm 3 with
 * one RNG word per candidate. */
void or_repair_paper(int rule, int n, const int32_t *r, const uint64_t *keys, int64_t nv, const uint64_t *cand,
                     int64_t nc, const float *pos, float eps, const uint32_t *words, uint64_t *out)
{
    ctx_t C;
    make_layout(&C.L, n, r);
    C.keys = keys;
    C.nv = nv;
    C.vt = tuples_of(&C.L, keys, nv);
    uint8_t *occ = (uint8_t *)malloc((size_t)n * 4096);
    occurring_values(&C, occ);
    for (int64_t i = 0; i < nc; i++) {
        if (rule == 1) out[i] = repair_l1(&C, cand[i]);
        else if (rule == 2) out[i] = repair_alg2(&C, occ, cand[i], pos + (size_t)i * n, eps);
        else out[i] = repair_alg3(&C, occ, cand[i], words[i]);
    }
    free(occ);
    free(C.vt);
}

/* Runs G generations after the initial one; writes the trace.  Returns 0. */
int or_run(int kind, int n, const int32_t *r, const uint64_t *keys, int64_t nv, const float *table,
           int P, int G, uint64_t seed, const or_params *prm, or_trace *T, const or_surr *sg, or_strace *ST)
{
    if (or_de_partners(prm->de_mutation) < 0 || prm->de_crossover < 0 || prm->de_crossover > 1 ||
        prm->ga_crossover < 0 || prm->ga_crossover > 3)
        return -2;
    if (kind == K_DE && P < or_de_partners(prm->de_mutation) + 1) return -3;   /* too few partners */
    ctx_t C;
    make_layout(&C.L, n, r);
    C.keys = keys;
    C.nv = nv;
    C.table = table;
    C.vt = tuples_of(&C.L, keys, nv);
    C.memo = (uint8_t *)calloc((size_t)(nv > 0 ? nv : 1), 1);
    C.n_unique = 0;
    C.cost_tab = prm->cost;
    C.cost = 0;
    C.T = T;
    C.g = C.i = 0;
    T->ev_n[0] = 0;
    C.best_key = ~0ull;
    C.best_fit = INFINITY;
    T->hit[0] = -1;
    T->hit[1] = -1;

    const int N = n;
    uint64_t *X = (uint64_t *)malloc(sizeof(uint64_t) * P);
    float *FX = (float *)malloc(sizeof(float) * P);
    uint64_t *U = (uint64_t *)malloc(sizeof(uint64_t) * P);
    uint64_t *UR = (uint64_t *)malloc(sizeof(uint64_t) * P);
    uint64_t *UE = (uint64_t *)malloc(sizeof(uint64_t) * P);
    float *FU = (float *)malloc(sizeof(float) * P);
    float *pos = (float *)calloc((size_t)P * N, sizeof(float));
    float *vel = (float *)calloc((size_t)P * N, sizeof(float));
    float *pb = (float *)calloc((size_t)P * N, sizeof(float));
    float *fpb = (float *)malloc(sizeof(float) * P);
    float *gb = (float *)calloc((size_t)N, sizeof(float));
    float fgb = INFINITY;
    float *ynew = (float *)calloc((size_t)P * N, sizeof(float));
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * OR_MAXP * 4);
    int32_t *ia = tmp, *ib = tmp + OR_MAXP, *ic = tmp + 2 * OR_MAXP, *id = tmp + 3 * OR_MAXP;
    uint8_t *pass = (uint8_t *)malloc((size_t)P);
    int *order = (int *)malloc(sizeof(int) * P);
    const float eps = coord_eps(&C.L);

    uint64_t de_best = 0;
    float de_fbest = INFINITY;
    int stag = 0, reinit_pending = 0;

    /* surrogate state: network, momentum, evaluated set (keys and log-fitness) */
    int D = 0;
    for (int k = 0; k < N; k++) D += C.L.r[k];
    int64_t n_par = sg ? or_mlp_param_count(D, sg->H) : 0;
    float *mlp = sg ? (float *)malloc(sizeof(float) * (size_t)n_par) : NULL;
    float *mom = sg ? (float *)calloc((size_t)n_par, sizeof(float)) : NULL;
    float *grad = sg ? (float *)malloc(sizeof(float) * (size_t)n_par) : NULL;
    uint64_t *EK = sg ? (uint64_t *)malloc(sizeof(uint64_t) * (size_t)P * (G + 1)) : NULL;
    float *EY = sg ? (float *)malloc(sizeof(float) * (size_t)P * (G + 1)) : NULL;
    int32_t *bf = sg ? (int32_t *)malloc(sizeof(int32_t) * (size_t)sg->batch * N) : NULL;
    float *by = sg ? (float *)malloc(sizeof(float) * (size_t)sg->batch) : NULL;
    float *spred = (float *)malloc(sizeof(float) * P);
    int *newi = (int *)malloc(sizeof(int) * P);
    int64_t n_e = 0;
    int use_surr = 0;
    if (sg) or_mlp_init(D, sg->H, seed, mlp);
    uint8_t *occ = NULL;
    if (prm->repair_rule) {
        occ = (uint8_t *)malloc((size_t)N * 4096);
        occurring_values(&C, occ);
    }

    for (int g = 0; g <= G; g++) {
        int init_mode = (g == 0) || (kind == K_DE && reinit_pending);
        /* ---------------- propose ---------------- */
        if (init_mode && !prm->aware && (kind == K_PSO || kind == K_FIREFLY)) {
            /* random coordinates in [0,1]^N, snapped */
            for (int i = 0; i < P; i++) {
                float *x = pos + (size_t)i * N;
                for (int j = 0; j < N; j++) x[j] = u01(rng_word(seed, i, g, P_RAND_INIT, (uint32_t)j));
                U[i] = snap_key(&C.L, x, eps);
            }
        } else if (init_mode && !prm->aware) {
            for (int i = 0; i < P; i++) U[i] = random_tuple(&C, seed, (uint32_t)i, (uint32_t)g);
        } else if (init_mode) {
            uint32_t purpose = g == 0 ? P_INIT : P_REINIT;
            for (int i = 0; i < P; i++) U[i] = stratified_key(&C, seed, (uint32_t)i, (uint32_t)P, (uint32_t)g, purpose);
        } else if (kind == K_DE) {
            for (int i = 0; i < P; i++) U[i] = de_trial(&C, X, de_best, P, i, (uint32_t)i, g, seed, prm);
        } else if (kind == K_PSO) {
            for (int i = 0; i < P; i++) {
                float *x = pos + (size_t)i * N, *v = vel + (size_t)i * N, *p = pb + (size_t)i * N;
                for (int j = 0; j < N; j++) {
                    float r1 = u01(rng_word(seed, i, g, P_PSO_R, 2u * j));
                    float r2 = u01(rng_word(seed, i, g, P_PSO_R, 2u * j + 1));
                    float t1 = prm->pso_w * v[j];
                    float t2 = (prm->pso_c1 * r1) * (p[j] - x[j]);
                    float t3 = (prm->pso_c2 * r2) * (gb[j] - x[j]);
                    v[j] = (t1 + t2) + t3;
                    x[j] = clip01(x[j] + v[j]);
                }
                U[i] = snap_key(&C.L, x, eps);
            }
        } else if (kind == K_FIREFLY) {
            for (int i = 0; i < P; i++) {
                float *y = ynew + (size_t)i * N;
                memcpy(y, pos + (size_t)i * N, sizeof(float) * N);
                for (int j = 0; j < P; j++) {
                    if (!(FX[j] < FX[i])) continue;       /* move toward brighter (lower cost) */
                    const float *xj = pos + (size_t)j * N;
                    float s = 0.0f;
                    for (int d = 0; d < N; d++) { float t = y[d] - xj[d]; s = s + t * t; }
                    float beta = prm->fa_beta0 * or_exp_ct(-prm->fa_gamma * s);
                    for (int d = 0; d < N; d++) {
                        float a = u01(rng_word(seed, i, g, P_FA_ALPHA, (uint32_t)(j * N + d)));
                        float nv2 = (y[d] + beta * (xj[d] - y[d])) + prm->fa_alpha * (a - 0.5f);
                        y[d] = clip01(nv2);
                    }
                }
                U[i] = snap_key(&C.L, y, eps);
            }
        } else { /* GA: rank by (fitness, key), beta selection, single-point crossover */
            for (int i = 0; i < P; i++) order[i] = i;
            for (int a = 1; a < P; a++) {               /* insertion sort, stable */
                int v = order[a], b = a - 1;
                while (b >= 0 && (FX[order[b]] > FX[v] || (FX[order[b]] == FX[v] && X[order[b]] > X[v]))) {
                    order[b + 1] = order[b];
                    b--;
                }
                order[b + 1] = v;
            }
            for (int c = 0; 2 * c < P; c++) {
                uint64_t k0, k1;
                ga_pair(&C, X, order, P, (uint32_t)c, g, seed, prm, &k0, &k1);
                U[2 * c] = k0;
                if (2 * c + 1 < P) U[2 * c + 1] = k1;
            }
        }
        /* ---------------- repair (+ GA mutation), evaluate ---------------- */
        for (int i = 0; i < P; i++) {
            if (init_mode || !prm->aware) UR[i] = U[i];
            else if (!prm->repair_rule) UR[i] = repair_key(&C, U[i]);
            else if (kind == K_DE) UR[i] = repair_l1(&C, U[i]);
            else if (kind == K_GA) UR[i] = repair_alg3(&C, occ, U[i], rng_word(seed, i, g, P_GA_REPAIR, 0));
            else UR[i] = repair_alg2(&C, occ, U[i], (kind == K_PSO ? pos : ynew) + (size_t)i * N, eps);
            UE[i] = (kind == K_GA && !init_mode)
                        ? (prm->aware ? ga_mutate(&C, UR[i], (uint32_t)i, g, seed, prm)
                                      : ga_mutate_plain(&C, UR[i], (uint32_t)i, g, seed, prm))
                        : UR[i];
        }
        /* surrogate screening: proposals s = 1..pool-1 from streams offset by s, all
         * repaired (and mutated), the lowest prediction wins each slot */
        int screened = sg && use_surr && !init_mode && (kind == K_DE || kind == K_GA);
        if (screened) {
            const int npairs = (P + 1) / 2;
            for (int i = 0; i < P; i++) spred[i] = predict1(&C, mlp, D, sg->H, UE[i]);
            for (int s = 1; s < sg->pool; s++) {
                for (int i = 0; i < P; i++) {
                    uint64_t c0 = 0, c1 = 0;
                    if (kind == K_DE) c0 = de_trial(&C, X, de_best, P, i, (uint32_t)(i + s * P), g, seed, prm);
                    else {
                        ga_pair(&C, X, order, P, (uint32_t)(i / 2 + s * npairs), g, seed, prm, &c0, &c1);
                        if (i & 1) c0 = c1;
                    }
                    uint64_t cr = repair_key(&C, c0);
                    uint64_t ce = (kind == K_GA) ? ga_mutate(&C, cr, (uint32_t)(i + s * P), g, seed, prm) : cr;
                    float pr = predict1(&C, mlp, D, sg->H, ce);
                    if (pr < spred[i] || (pr == spred[i] && ce < UE[i])) {
                        spred[i] = pr;
                        U[i] = c0;
                        UR[i] = cr;
                        UE[i] = ce;
                    }
                }
            }
        }
        int64_t n_new = 0;
        for (int i = 0; i < P; i++) {
            int64_t rk = rank_of(C.keys, C.nv, UE[i]);
            if (sg && rk >= 0 && !C.memo[rk]) newi[n_new++] = i;
            C.g = g;
            C.i = i;
            FU[i] = evaluate(&C, UE[i]);
        }
        if (sg) {   /* judge on this generation's evaluations, then learn from them */
            float sa = 0.0f, sy = 0.0f, sd = 0.0f;
            for (int i = 0; i < P; i++) {
                float pr = predict1(&C, mlp, D, sg->H, UE[i]);
                float y = sg->logt[rank_of(C.keys, C.nv, UE[i])];
                sa = sa + fabsf(pr - y);
                sy = sy + y;
                spred[i] = y;
            }
            float mae = sa / (float)P, ybar = sy / (float)P;
            for (int i = 0; i < P; i++) sd = sd + fabsf(spred[i] - ybar);
            float tau = sg->mae_ratio * (sd / (float)P);
            for (int64_t q = 0; q < n_new; q++) {
                EK[n_e] = UE[newi[q]];
                EY[n_e] = sg->logt[rank_of(C.keys, C.nv, UE[newi[q]])];
                n_e++;
            }
            for (int t = 0; t < sg->steps && n_e > 0; t++) {
                for (int b = 0; b < sg->batch; b++) {
                    uint32_t pick = uint_below(rng_word(seed, (uint32_t)b, (uint32_t)g, P_MLP_BATCH, (uint32_t)t), (uint32_t)n_e);
                    feats_of(&C, EK[pick], bf + (size_t)b * N);
                    by[b] = EY[pick];
                }
                or_mlp_grad(mlp, D, sg->H, N, bf, by, sg->batch, grad);
                or_mlp_sgd(mlp, mom, grad, n_par, sg->lr, sg->mu);
            }
            if (ST) {
                ST->used[g] = (int8_t)screened;
                ST->mae[g] = mae;
                ST->tau[g] = tau;
                ST->n_e[g] = n_e;
            }
            use_surr = n_e >= (int64_t)sg->warm_mult * P && mae <= tau;
        }


        /* ---------------- select / update ---------------- */
        if (kind == K_DE) {
            if (init_mode) {
                for (int i = 0; i < P; i++) { X[i] = UE[i]; FX[i] = FU[i]; }
                if (g == 0) { de_best = X[0]; de_fbest = FX[0]; }
                for (int i = (g == 0 ? 1 : 0); i < P; i++)
                    if (FX[i] <= de_fbest) { de_best = X[i]; de_fbest = FX[i]; }
                reinit_pending = 0;
                stag = 0;
            } else {
                /* Algorithm 1 selection on the generation's snapshot: f(u) <= f(x) and u not in X */
                for (int i = 0; i < P; i++) {
                    int in_x = 0;
                    for (int k = 0; k < P && !in_x; k++) in_x = (X[k] == UE[i]);
                    pass[i] = (uint8_t)(FU[i] <= FX[i] && !in_x);
                }
                int accepted = 0;
                for (int i = 0; i < P; i++) {
                    int dup = 0;
                    for (int k = 0; k < i && !dup; k++) dup = pass[k] && UE[k] == UE[i];
                    if (!pass[i] || dup) continue;
                    X[i] = UE[i];
                    FX[i] = FU[i];
                    accepted++;
                    if (FU[i] <= de_fbest) { de_best = UE[i]; de_fbest = FU[i]; }
                }
                stag = accepted ? 0 : stag + 1;
                if (stag >= 2) { reinit_pending = 1; stag = 0; }
            }
        } else if (kind == K_PSO || kind == K_FIREFLY) {
            if (g == 0) {
                for (int i = 0; i < P; i++) {
                    unpack(&C.L, UE[i], ia);
                    for (int j = 0; j < N; j++) {
                        float x0 = prm->aware ? (float)ia[j] * eps : pos[(size_t)i * N + j];
                        pos[(size_t)i * N + j] = x0;
                        pb[(size_t)i * N + j] = x0;
                        if (kind == K_PSO) {
                            float a = u01(rng_word(seed, i, 0, P_PSO_VEL, (uint32_t)j));
                            vel[(size_t)i * N + j] = (2.0f * a - 1.0f) * eps;
                        }
                    }
                    fpb[i] = FU[i];
                    FX[i] = FU[i];
                }
            } else if (kind == K_PSO) {
                for (int i = 0; i < P; i++)
                    if (FU[i] < fpb[i]) {
                        fpb[i] = FU[i];
                        memcpy(pb + (size_t)i * N, pos + (size_t)i * N, sizeof(float) * N);
                    }
            } else {
                memcpy(pos, ynew, sizeof(float) * (size_t)P * N);
                for (int i = 0; i < P; i++) FX[i] = FU[i];
            }
            if (kind == K_PSO)
                for (int i = 0; i < P; i++)
                    if (fpb[i] < fgb) { fgb = fpb[i]; memcpy(gb, pb + (size_t)i * N, sizeof(float) * N); }
            if (T->pos) memcpy(T->pos + (size_t)g * P * N, pos, sizeof(float) * (size_t)P * N);
            for (int i = 0; i < P; i++) X[i] = UE[i];
        } else { /* GA: the children replace the population */
            for (int i = 0; i < P; i++) { X[i] = UE[i]; FX[i] = FU[i]; }
        }
        if (kind == K_PSO) for (int i = 0; i < P; i++) FX[i] = fpb[i];

        /* ---------------- trace ---------------- */
        size_t o = (size_t)g * P;
        memcpy(T->cand + o, U, sizeof(uint64_t) * P);
        memcpy(T->rep + o, UR, sizeof(uint64_t) * P);
        memcpy(T->evalk + o, UE, sizeof(uint64_t) * P);
        memcpy(T->fit + o, FU, sizeof(float) * P);
        memcpy(T->popk + o, X, sizeof(uint64_t) * P);
        memcpy(T->popf + o, FX, sizeof(float) * P);
        record(&C, T, g, P, prm);
    }
    free(X); free(FX); free(U); free(UR); free(UE); free(FU); free(pos); free(vel); free(pb);
    free(fpb); free(gb); free(ynew); free(tmp); free(pass); free(order); free(C.vt); free(C.memo);
    if (sg && ST && ST->params) memcpy(ST->params, mlp, sizeof(float) * (size_t)n_par);
    free(mlp); free(mom); free(grad); free(EK); free(EY); free(bf); free(by); free(spred); free(newi); free(occ);
    return 0;
}

/* exported helpers for the pins */
uint32_t or_beta_pick(uint32_t w, uint32_t P) { return beta_pick(w, P); }
float or_u01(uint32_t w) { return u01(w); }

/* ------------------------------------------------------------------------- */
/* MLP surrogate (a learned screen over proposals; not part of the paper)     */
/* ------------------------------------------------------------------------- */
/* Network: one-hot value indices (D = sum_k r_k features, N active) -> H -> H
 * -> H (ReLU) -> 1.  Parameters are fp32 masters, flat:
 *   W1[H][D], b1[H], W2[H][H], b2[H], W3[H][H], b3[H], W4[H], b4.
 * Forward uses bf16(W) (round to nearest even) with fp32 accumulation in
 * ascending input order: dense layers acc = fmaf(a_i, w_ji, acc) from 0, then
 * z = acc + b; the one-hot layer adds the active weights in ascending feature
 * order.  Loss: mean squared error against log-fitness. */

static float bf16r(float f)
{
    union { float f; uint32_t u; } v;
    v.f = f;
    uint32_t lsb = (v.u >> 16) & 1u;
    v.u += 0x7FFFu + lsb;
    v.u &= 0xFFFF0000u;
    return v.f;
}

float or_bf16_round(float f) { return bf16r(f); }

int64_t or_mlp_param_count(int D, int H) { return (int64_t)H * D + H + 2 * ((int64_t)H * H + H) + H + 1; }

typedef struct { float *W1, *b1, *W2, *b2, *W3, *b3, *W4, *b4; } mlp_view;

static mlp_view view_of(float *p, int D, int H)
{
    mlp_view v;
    v.W1 = p; p += (size_t)H * D;
    v.b1 = p; p += H;
    v.W2 = p; p += (size_t)H * H;
    v.b2 = p; p += H;
    v.W3 = p; p += (size_t)H * H;
    v.b3 = p; p += H;
    v.W4 = p; p += H;
    v.b4 = p;
    return v;
}

/* Glorot-uniform weights from the MLP_INIT stream (individual = tensor 1..4,
 * generation 0, word = element index), zero biases. */
void or_mlp_init(int D, int H, uint64_t seed, float *params)
{
    mlp_view v = view_of(params, D, H);
    memset(params, 0, sizeof(float) * (size_t)or_mlp_param_count(D, H));
    float *W[4] = {v.W1, v.W2, v.W3, v.W4};
    int64_t n[4] = {(int64_t)H * D, (int64_t)H * H, (int64_t)H * H, H};
    int fin[4] = {D, H, H, H}, fout[4] = {H, H, H, 1};
    for (int t = 0; t < 4; t++) {
        float a = sqrtf(6.0f / (float)(fin[t] + fout[t]));
        for (int64_t e = 0; e < n[t]; e++) {
            float u = u01(rng_word(seed, (uint32_t)(t + 1), 0, P_MLP_INIT, (uint32_t)e));
            W[t][e] = (2.0f * u - 1.0f) * a;
        }
    }
}

/* feats: B rows of N ascending feature indices.  acts (optional): per sample
 * z1,z2,z3 (3H) then h1,h2,h3 (3H), for the backward pass. */
void or_mlp_forward(const float *params, int D, int H, int N, const int32_t *feats, int B, float *pred, float *acts)
{
    mlp_view v = view_of((float *)params, D, H);
    float *z = (float *)malloc(sizeof(float) * 6 * (size_t)H);
    for (int b = 0; b < B; b++) {
        float *z1 = z, *z2 = z + H, *z3 = z + 2 * H, *h1 = z + 3 * H, *h2 = z + 4 * H, *h3 = z + 5 * H;
        const int32_t *f = feats + (size_t)b * N;
        for (int j = 0; j < H; j++) {
            float acc = 0.0f;
            for (int k = 0; k < N; k++) acc = acc + bf16r(v.W1[(size_t)j * D + f[k]]);
            z1[j] = acc + v.b1[j];
            h1[j] = z1[j] > 0.0f ? z1[j] : 0.0f;
        }
        for (int j = 0; j < H; j++) {
            float acc = 0.0f;
            for (int i = 0; i < H; i++) acc = fmaf(h1[i], bf16r(v.W2[(size_t)j * H + i]), acc);
            z2[j] = acc + v.b2[j];
            h2[j] = z2[j] > 0.0f ? z2[j] : 0.0f;
        }
        for (int j = 0; j < H; j++) {
            float acc = 0.0f;
            for (int i = 0; i < H; i++) acc = fmaf(h2[i], bf16r(v.W3[(size_t)j * H + i]), acc);
            z3[j] = acc + v.b3[j];
            h3[j] = z3[j] > 0.0f ? z3[j] : 0.0f;
        }
        float acc = 0.0f;
        for (int i = 0; i < H; i++) acc = fmaf(h3[i], bf16r(v.W4[i]), acc);
        pred[b] = acc + v.b4[0];
        if (acts) memcpy(acts + (size_t)b * 6 * H, z, sizeof(float) * 6 * (size_t)H);
    }
    free(z);
}

/* Gradient of the batch MSE (fp32, fixed order: every reduction over the batch
 * runs in ascending sample index, over neurons in ascending index). */
void or_mlp_grad(const float *params, int D, int H, int N, const int32_t *feats, const float *y, int B, float *grad)
{
    mlp_view v = view_of((float *)params, D, H);
    mlp_view g = view_of(grad, D, H);
    size_t np = (size_t)or_mlp_param_count(D, H);
    memset(grad, 0, sizeof(float) * np);
    float *acts = (float *)malloc(sizeof(float) * 6 * (size_t)H * B);
    float *pred = (float *)malloc(sizeof(float) * B);
    float *gout = (float *)malloc(sizeof(float) * B);
    float *d3 = (float *)malloc(sizeof(float) * (size_t)H * B);
    float *d2 = (float *)malloc(sizeof(float) * (size_t)H * B);
    float *d1 = (float *)malloc(sizeof(float) * (size_t)H * B);
    or_mlp_forward(params, D, H, N, feats, B, pred, acts);
    const float scale = 2.0f / (float)B;
#define Z(b, l, j) acts[(size_t)(b) * 6 * H + (size_t)(l) * H + (j)]
#define A(b, l, j) acts[(size_t)(b) * 6 * H + (size_t)(3 + (l)) * H + (j)]
    for (int b = 0; b < B; b++) gout[b] = scale * (pred[b] - y[b]);
    for (int b = 0; b < B; b++)
        for (int j = 0; j < H; j++) d3[(size_t)b * H + j] = Z(b, 2, j) > 0.0f ? gout[b] * bf16r(v.W4[j]) : 0.0f;
    for (int b = 0; b < B; b++)
        for (int i = 0; i < H; i++) {
            float acc = 0.0f;
            for (int j = 0; j < H; j++) acc = fmaf(d3[(size_t)b * H + j], bf16r(v.W3[(size_t)j * H + i]), acc);
            d2[(size_t)b * H + i] = Z(b, 1, i) > 0.0f ? acc : 0.0f;
        }
    for (int b = 0; b < B; b++)
        for (int i = 0; i < H; i++) {
            float acc = 0.0f;
            for (int j = 0; j < H; j++) acc = fmaf(d2[(size_t)b * H + j], bf16r(v.W2[(size_t)j * H + i]), acc);
            d1[(size_t)b * H + i] = Z(b, 0, i) > 0.0f ? acc : 0.0f;
        }
    /* weight and bias gradients, reductions over the batch in ascending b */
    for (int j = 0; j < H; j++) {
        float acc = 0.0f;
        for (int b = 0; b < B; b++) acc = fmaf(gout[b], A(b, 2, j), acc);
        g.W4[j] = acc;
    }
    { float acc = 0.0f; for (int b = 0; b < B; b++) acc = acc + gout[b]; g.b4[0] = acc; }
    for (int j = 0; j < H; j++) {
        for (int i = 0; i < H; i++) {
            float a3 = 0.0f, a2 = 0.0f;
            for (int b = 0; b < B; b++) {
                a3 = fmaf(d3[(size_t)b * H + j], A(b, 1, i), a3);
                a2 = fmaf(d2[(size_t)b * H + j], A(b, 0, i), a2);
            }
            g.W3[(size_t)j * H + i] = a3;
            g.W2[(size_t)j * H + i] = a2;
        }
        float s3 = 0.0f, s2 = 0.0f, s1 = 0.0f;
        for (int b = 0; b < B; b++) { s3 = s3 + d3[(size_t)b * H + j]; s2 = s2 + d2[(size_t)b * H + j]; s1 = s1 + d1[(size_t)b * H + j]; }
        g.b3[j] = s3;
        g.b2[j] = s2;
        g.b1[j] = s1;
        for (int b = 0; b < B; b++) {      /* one-hot layer: each active feature, samples in ascending order */
            const int32_t *f = feats + (size_t)b * N;
            for (int k = 0; k < N; k++) g.W1[(size_t)j * D + f[k]] = g.W1[(size_t)j * D + f[k]] + d1[(size_t)b * H + j];
        }
    }
#undef Z
#undef A
    free(acts); free(pred); free(gout); free(d3); free(d2); free(d1);
}

/* SGD with momentum on the fp32 masters: v = mu*v + g; p = p - lr*v. */
void or_mlp_sgd(float *params, float *mom, const float *grad, int64_t n, float lr, float mu)
{
    for (int64_t e = 0; e < n; e++) {
        mom[e] = mu * mom[e] + grad[e];
        params[e] = params[e] - lr * mom[e];
    }
}

/* fp64 forward/gradient on the given (unrounded) weights, for the finite-difference check */
double or_mlp_loss64(const double *params, int D, int H, int N, const int32_t *feats, const double *y, int B, double *grad)
{
    const double *W1 = params, *b1 = W1 + (size_t)H * D, *W2 = b1 + H, *b2 = W2 + (size_t)H * H, *W3 = b2 + H,
                 *b3 = W3 + (size_t)H * H, *W4 = b3 + H, *b4 = W4 + H;
    double *g = grad;
    size_t np = (size_t)or_mlp_param_count(D, H);
    if (g) memset(g, 0, sizeof(double) * np);
    double *gW1 = g, *gb1 = g ? gW1 + (size_t)H * D : 0, *gW2 = g ? gb1 + H : 0, *gb2 = g ? gW2 + (size_t)H * H : 0,
           *gW3 = g ? gb2 + H : 0, *gb3 = g ? gW3 + (size_t)H * H : 0, *gW4 = g ? gb3 + H : 0, *gb4 = g ? gW4 + H : 0;
    double *z = (double *)malloc(sizeof(double) * 9 * (size_t)H);
    double loss = 0;
    for (int b = 0; b < B; b++) {
        double *z1 = z, *z2 = z + H, *z3 = z + 2 * H, *h1 = z + 3 * H, *h2 = z + 4 * H, *h3 = z + 5 * H;
        double *d1 = z + 6 * H, *d2 = z + 7 * H, *d3 = z + 8 * H;
        const int32_t *f = feats + (size_t)b * N;
        for (int j = 0; j < H; j++) {
            double acc = b1[j];
            for (int k = 0; k < N; k++) acc += W1[(size_t)j * D + f[k]];
            z1[j] = acc; h1[j] = acc > 0 ? acc : 0;
        }
        for (int j = 0; j < H; j++) {
            double acc = b2[j];
            for (int i = 0; i < H; i++) acc += W2[(size_t)j * H + i] * h1[i];
            z2[j] = acc; h2[j] = acc > 0 ? acc : 0;
        }
        for (int j = 0; j < H; j++) {
            double acc = b3[j];
            for (int i = 0; i < H; i++) acc += W3[(size_t)j * H + i] * h2[i];
            z3[j] = acc; h3[j] = acc > 0 ? acc : 0;
        }
        double out = b4[0];
        for (int i = 0; i < H; i++) out += W4[i] * h3[i];
        double e = out - y[b];
        loss += e * e / B;
        if (!g) continue;
        double go = 2.0 * e / B;
        gb4[0] += go;
        for (int j = 0; j < H; j++) { gW4[j] += go * h3[j]; d3[j] = z3[j] > 0 ? go * W4[j] : 0; }
        for (int i = 0; i < H; i++) {
            double acc = 0;
            for (int j = 0; j < H; j++) acc += d3[j] * W3[(size_t)j * H + i];
            d2[i] = z2[i] > 0 ? acc : 0;
        }
        for (int i = 0; i < H; i++) {
            double acc = 0;
            for (int j = 0; j < H; j++) acc += d2[j] * W2[(size_t)j * H + i];
            d1[i] = z1[i] > 0 ? acc : 0;
        }
        for (int j = 0; j < H; j++) {
            gb3[j] += d3[j]; gb2[j] += d2[j]; gb1[j] += d1[j];
            for (int i = 0; i < H; i++) { gW3[(size_t)j * H + i] += d3[j] * h2[i]; gW2[(size_t)j * H + i] += d2[j] * h1[i]; }
            for (int k = 0; k < N; k++) gW1[(size_t)j * D + f[k]] += d1[j];
        }
    }
    free(z);
    return loss;
}
