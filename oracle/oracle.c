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
 * Optimizer trajectories themselves are "parity unpinned" by the paper (it
 * prints no trace); they are pinned by the reduction cases only.
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
    P_PSO_VEL = 13
};

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
} ctx_t;

static float evaluate(ctx_t *C, uint64_t key)
{
    int64_t rk = rank_of(C->keys, C->nv, key);
    if (rk < 0) return INFINITY;            /* unreachable after repair */
    if (!C->memo[rk]) { C->memo[rk] = 1; C->n_unique++; }
    float f = C->table[rk];
    if (f < C->best_fit || (f == C->best_fit && key < C->best_key)) {
        C->best_fit = f;
        C->best_key = key;
    }
    return f;
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

/* Runs G generations after the initial one; writes the trace.  Returns 0. */
int or_run(int kind, int n, const int32_t *r, const uint64_t *keys, int64_t nv, const float *table,
           int P, int G, uint64_t seed, const or_params *prm, or_trace *T)
{
    ctx_t C;
    make_layout(&C.L, n, r);
    C.keys = keys;
    C.nv = nv;
    C.table = table;
    C.vt = tuples_of(&C.L, keys, nv);
    C.memo = (uint8_t *)calloc((size_t)(nv > 0 ? nv : 1), 1);
    C.n_unique = 0;
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

    for (int g = 0; g <= G; g++) {
        int init_mode = (g == 0) || (kind == K_DE && reinit_pending);
        /* ---------------- propose ---------------- */
        if (init_mode) {
            uint32_t purpose = g == 0 ? P_INIT : P_REINIT;
            for (int i = 0; i < P; i++) U[i] = stratified_key(&C, seed, (uint32_t)i, (uint32_t)P, (uint32_t)g, purpose);
        } else if (kind == K_DE) {
            unpack(&C.L, de_best, ia);
            for (int i = 0; i < P; i++) {
                uint32_t w0 = rng_word(seed, i, g, P_MUT_PICK, 0), w1 = rng_word(seed, i, g, P_MUT_PICK, 1);
                uint32_t r2 = uint_below(w0, (uint32_t)P - 1);
                if (r2 >= (uint32_t)i) r2++;
                uint32_t r3 = uint_below(w1, (uint32_t)P - 2);
                uint32_t lo = (uint32_t)i < r2 ? (uint32_t)i : r2, hi = (uint32_t)i < r2 ? r2 : (uint32_t)i;
                if (r3 >= lo) r3++;
                if (r3 >= hi) r3++;
                unpack(&C.L, X[r2], ib);
                unpack(&C.L, X[r3], ic);
                unpack(&C.L, X[i], id);
                uint32_t jrand = uint_below(rng_word(seed, i, g, P_CROSS, 0), (uint32_t)N);
                int32_t t[OR_MAXP];
                for (int j = 0; j < N; j++) {
                    /* Algorithm 1, Mutate: m = i_r1 + F*(i_r2 - i_r3), round and clip */
                    float diff = (float)(ib[j] - ic[j]);
                    float m = (float)ia[j] + prm->de_F * diff;
                    float q = rintf(m);
                    int v = (int)q;
                    if (q < 0.0f) v = 0;
                    if (v > C.L.r[j] - 1) v = C.L.r[j] - 1;
                    /* Algorithm 1, Crossover (binomial) */
                    float rr = u01(rng_word(seed, i, g, P_CROSS, 1 + (uint32_t)j));
                    t[j] = (rr < prm->de_CR || (uint32_t)j == jrand) ? v : id[j];
                }
                U[i] = pack(&C.L, t);
            }
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
                uint32_t pa = beta_pick(rng_word(seed, c, g, P_GA_SEL, 0), (uint32_t)P);
                uint32_t pbi = beta_pick(rng_word(seed, c, g, P_GA_SEL, 1), (uint32_t)P);
                uint32_t cut = N >= 2 ? 1 + uint_below(rng_word(seed, c, g, P_GA_CUT, 0), (uint32_t)N - 1) : 1;
                unpack(&C.L, X[order[pa]], ia);
                unpack(&C.L, X[order[pbi]], ib);
                for (int j = 0; j < N; j++) {
                    ic[j] = (uint32_t)j < cut ? ia[j] : ib[j];
                    id[j] = (uint32_t)j < cut ? ib[j] : ia[j];
                }
                U[2 * c] = pack(&C.L, ic);
                if (2 * c + 1 < P) U[2 * c + 1] = pack(&C.L, id);
            }
        }
        /* ---------------- repair (+ GA mutation), evaluate ---------------- */
        for (int i = 0; i < P; i++) {
            UR[i] = init_mode ? U[i] : repair_key(&C, U[i]);
            UE[i] = UR[i];
            if (kind == K_GA && !init_mode) {
                if (u01(rng_word(seed, i, g, P_GA_MUT, 0)) < prm->ga_pmut) {
                    /* random valid Hamming neighbour, enumerated by (param, value index) */
                    unpack(&C.L, UR[i], ia);
                    int64_t cnt = 0;
                    for (int k = 0; k < N; k++)
                        for (int v = 0; v < C.L.r[k]; v++) {
                            if (v == ia[k]) continue;
                            int32_t save = ia[k];
                            ia[k] = v;
                            if (rank_of(C.keys, C.nv, pack(&C.L, ia)) >= 0) cnt++;
                            ia[k] = save;
                        }
                    if (cnt > 0) {
                        uint32_t pick = uint_below(rng_word(seed, i, g, P_GA_MUT, 1), (uint32_t)cnt);
                        int64_t seen = 0;
                        int done = 0;
                        for (int k = 0; k < N && !done; k++)
                            for (int v = 0; v < C.L.r[k] && !done; v++) {
                                if (v == ia[k]) continue;
                                int32_t save = ia[k];
                                ia[k] = v;
                                uint64_t kk = pack(&C.L, ia);
                                if (rank_of(C.keys, C.nv, kk) >= 0) {
                                    if (seen == (int64_t)pick) { UE[i] = kk; done = 1; }
                                    seen++;
                                }
                                ia[k] = save;
                            }
                    }
                }
            }
        }
        for (int i = 0; i < P; i++) FU[i] = evaluate(&C, UE[i]);

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
                        float x0 = (float)ia[j] * eps;
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
    return 0;
}

/* exported helpers for the pins */
uint32_t or_beta_pick(uint32_t w, uint32_t P) { return beta_pick(w, P); }
float or_u01(uint32_t w) { return u01(w); }
