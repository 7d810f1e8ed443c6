// Device-side data layout and helpers shared by the catune kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/catune.h"

namespace ct {

constexpr int MAXP = CT_MAX_PARAMS;
constexpr int MAXV = CT_MAX_VALUES;
constexpr int MAXC = CT_MAX_CONSTRAINTS;
constexpr int MAXI = CT_MAX_INSTR;
constexpr int BLOCK_BITS_MAX = 4096;   // points of one enumeration block (mask bits)
constexpr int MAX_RADIUS = 8;          // largest Hamming ball radius the ball search tables cover

// One constraint after lowering.  Constraints are stored sorted by block.
struct DevCons {
    int32_t pc, len;          // program slice in DevSpace::prog (END excluded)
    int32_t level;            // deepest parameter in the scope (-1: no parameter)
    int32_t block;            // enumeration block holding `level`
    int32_t tabled;           // 1: truth-mask table, 0: interpreted per point
    int32_t n_outer;          // parameters of the scope that lie before the block
    int32_t outer_k[MAXP];
    int32_t outer_stride[MAXP];
    uint64_t table_off;       // word offset of row 0 in the table arena
    uint32_t rows;            // prod of outer value counts
    uint32_t scope;           // parameters the constraint reads (bit k: parameter k)
    // compact truth table of a tabled constraint: one bit per combination of its own
    // parameters, [row][cz_W words] with the in-block scope parameters in_k mixed-radix
    // (stride in_stride, last fastest) inside a row; cz_off = CZ_NONE: the table bits
    // are interpreted one by one instead
    int32_t n_in;
    int32_t in_k[MAXP];
    int32_t in_stride[MAXP];
    uint32_t cz_B, cz_W;      // combinations and words per row
    uint64_t cz_off;          // word offset of row 0 in the compact arena
};
constexpr uint64_t CZ_NONE = ~0ull;

// One enumeration block: consecutive parameters [s, e) whose Cartesian product
// (B <= BLOCK_BITS_MAX points, W 32-bit words) is expanded per parent prefix.
struct DevBlock {
    int32_t s, e;
    int32_t B, W;
    int32_t pstride[MAXP];    // mixed-radix stride of parameter s + i inside the block
    uint32_t innerkey_off;    // offset of the block's point -> key-bits table
    int32_t key_shift;        // offset of the lowest field of the block (off[e-1])
    int32_t cons_begin, cons_end;
    int32_t has_vm;           // some constraint of the block is interpreted
    // pattern mode: the block's valid-point mask depends only on the parent's fields of the
    // parameters U (before the block) read by its constraints; one compacted inner-key list per
    // signature sig = mixed radix over U
    int32_t pattern;
    int32_t n_u;
    int32_t u_k[MAXP];
    int32_t u_stride[MAXP];
    uint32_t n_sig;
    uint32_t Bpad;            // list capacity per signature (B rounded up to 4)
    uint64_t pat_cnt_off;     // offset into the pattern count arena
    uint64_t pat_list_off;    // offset into the pattern list arena
};

struct DevSpace {
    int32_t n, key_bits, n_cons, n_blocks;
    int32_t r[MAXP], w[MAXP], off[MAXP], vstart[MAXP];
    uint64_t fmask[MAXP];     // field mask in place
    uint32_t alt_rcp[MAXP];   // floor(2^32 / (r_k - 1)) + 1: quotients by r_k - 1 (see div_alt)
    uint64_t swar_low;        // every bit of every field except the field's top bit
    uint64_t swar_high;       // the top bit of every field of width >= 1
    uint64_t domain_bits;     // bits used by the key
    const uint32_t* compact;  // compact truth tables of the tabled constraints (device arena)
    uint64_t pcons[MAXP];     // constraints reading parameter k (bit c: constraint c)
    int64_t values[MAXV];
    DevCons cons[MAXC];
    DevBlock blocks[MAXP];
    ct_instr prog[MAXI];
};

// ------------------------------------------------------------------------------
// Philox4x32-10 counter-based generator (Salmon et al., SC'11)
// ------------------------------------------------------------------------------
__host__ __device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
#ifdef __CUDA_ARCH__
        uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
#else
        uint64_t p0 = (uint64_t)0xD2511F53u * c[0], p1 = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
}

enum Purpose : uint32_t {
    PU_INIT = 1, PU_MUT_PICK = 2, PU_CROSS = 3, PU_PSO_R = 4, PU_FA_ALPHA = 5, PU_GA_SEL = 6,
    PU_GA_CUT = 7, PU_GA_MUT = 8, PU_REINIT = 9, PU_POOL = 10, PU_MLP_INIT = 11, PU_MLP_BATCH = 12,
    PU_PSO_VEL = 13, PU_GA_REPAIR = 14, PU_RAND_INIT = 15
};

// Word t of the stream (individual, generation, purpose) for `seed`:
// lane t % 4 of Philox(counter = (t / 4, individual, generation, purpose), key = seed).
__host__ __device__ __forceinline__ uint32_t rng_word(uint64_t seed, uint32_t indiv, uint32_t gen,
                                                      uint32_t purpose, uint32_t t) {
    uint32_t c[4] = {t >> 2, indiv, gen, purpose};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    return c[t & 3u];
}

// Block of 4 consecutive words starting at a multiple of 4.
__host__ __device__ __forceinline__ void rng_block(uint64_t seed, uint32_t indiv, uint32_t gen,
                                                   uint32_t purpose, uint32_t draw, uint32_t out[4]) {
    out[0] = draw; out[1] = indiv; out[2] = gen; out[3] = purpose;
    philox4x32_10(out, (uint32_t)seed, (uint32_t)(seed >> 32));
}

__host__ __device__ __forceinline__ float u01(uint32_t w) {
    return (float)(w >> 8) * (1.0f / 16777216.0f);
}
__host__ __device__ __forceinline__ uint32_t uint_below(uint32_t w, uint32_t n) {
    return (uint32_t)(((uint64_t)w * n) >> 32);
}
__device__ __forceinline__ uint64_t uint64_below(uint32_t whi, uint32_t wlo, uint64_t n) {
    return __umul64hi(((uint64_t)whi << 32) | wlo, n);
}

// ------------------------------------------------------------------------------
// key fields
// ------------------------------------------------------------------------------
__device__ __forceinline__ int32_t field(const DevSpace* sp, uint64_t key, int k) {
    return (int32_t)((key & sp->fmask[k]) >> sp->off[k]);
}

// t / (r_k - 1) and t % (r_k - 1) for any 32-bit t (r_k >= 2), by the reciprocal method of
// Granlund and Montgomery: with M = floor(2^32 / a) + 1, umulhi(t, M) is floor(t / a) or one
// more (M exceeds 2^32 / a by at most 1, so the error is below t / 2^32 < 1); one correction
// step fixes the overshoot.
__device__ __forceinline__ uint32_t div_alt(const DevSpace* __restrict__ sp, int k, uint32_t t, uint32_t* rem) {
    const uint32_t a = (uint32_t)sp->r[k] - 1u;
    if (a == 1u) { *rem = 0u; return t; }   // M = 2^32 + 1 does not fit
    uint32_t q = __umulhi(t, sp->alt_rcp[k]);
    int32_t r = (int32_t)(t - q * a);
    if (r < 0) { --q; r += (int32_t)a; }
    *rem = (uint32_t)r;
    return q;
}

// 1 when every field is < r_k and no bit above the key is set.
__device__ __forceinline__ bool in_domain(const DevSpace* sp, uint64_t key) {
    if (key & ~sp->domain_bits) return false;
    for (int k = 0; k < sp->n; ++k)
        if (field(sp, key, k) >= sp->r[k]) return false;
    return true;
}

// Number of fields in which a and b differ: per-field non-zero test on a^b by
// carrying every field's low bits into its top bit, then a population count.
__device__ __forceinline__ int hamming_keys(uint64_t a, uint64_t b, uint64_t lowm, uint64_t highm) {
    uint64_t x = a ^ b;
    uint64_t t = ((x & lowm) + lowm) | x;
    return __popcll(t & highm);
}

// ------------------------------------------------------------------------------
// constraint program interpreter (postfix, 64-bit, poison on division by zero)
// ------------------------------------------------------------------------------
__device__ __forceinline__ bool vm_eval(const ct_instr* __restrict__ prog, int pc, int len,
                                        const int64_t* pv) {
    int64_t st[CT_MAX_STACK];
    uint32_t poison = 0;  // bit i: slot i poisoned
    int sp = 0;
    for (int i = 0; i < len; ++i) {
        const ct_instr in = prog[pc + i];
        const int op = in.op;
        if (op == CT_OP_PARAM) { st[sp] = pv[in.arg]; poison &= ~(1u << sp); ++sp; continue; }
        if (op == CT_OP_CONST) { st[sp] = in.imm; poison &= ~(1u << sp); ++sp; continue; }
        if (op == CT_OP_NEG) {
            st[sp - 1] = (int64_t)(0ull - (uint64_t)st[sp - 1]);
            continue;
        }
        if (op == CT_OP_NOT) {
            bool t = !((poison >> (sp - 1)) & 1u) && st[sp - 1] != 0;
            st[sp - 1] = t ? 0 : 1;
            poison &= ~(1u << (sp - 1));
            continue;
        }
        const int64_t a = st[sp - 2], b = st[sp - 1];
        const bool pa = (poison >> (sp - 2)) & 1u, pb = (poison >> (sp - 1)) & 1u;
        const bool p = pa || pb;
        const bool at = !pa && a != 0, bt = !pb && b != 0;
        int64_t r = 0;
        bool rp = false;
        switch (op) {
            case CT_OP_ADD: r = (int64_t)((uint64_t)a + (uint64_t)b); rp = p; break;
            case CT_OP_SUB: r = (int64_t)((uint64_t)a - (uint64_t)b); rp = p; break;
            case CT_OP_MUL: r = (int64_t)((uint64_t)a * (uint64_t)b); rp = p; break;
            case CT_OP_DIV:
            case CT_OP_MOD:
                if (p || b == 0) { rp = true; break; }
                if (a == INT64_MIN && b == -1) { r = (op == CT_OP_DIV) ? INT64_MIN : 0; break; }
                if (a == (int32_t)a && b == (int32_t)b && !(a == INT32_MIN && b == -1)) {
                    // both operands fit in 32 bits: the same truncated quotient and remainder,
                    // with the much cheaper 32-bit division
                    const int32_t a32 = (int32_t)a, b32 = (int32_t)b;
                    r = (op == CT_OP_DIV) ? (int64_t)(a32 / b32) : (int64_t)(a32 % b32);
                    break;
                }
                r = (op == CT_OP_DIV) ? a / b : a % b;
                break;
            case CT_OP_MIN: r = a < b ? a : b; rp = p; break;
            case CT_OP_MAX: r = a > b ? a : b; rp = p; break;
            case CT_OP_LT: r = !p && a < b; break;
            case CT_OP_LE: r = !p && a <= b; break;
            case CT_OP_GT: r = !p && a > b; break;
            case CT_OP_GE: r = !p && a >= b; break;
            case CT_OP_EQ: r = !p && a == b; break;
            case CT_OP_NE: r = !p && a != b; break;
            case CT_OP_AND: r = at && bt; break;
            case CT_OP_OR: r = at || bt; break;
            default: rp = true; break;
        }
        --sp;
        st[sp - 1] = r;
        if (rp) poison |= 1u << (sp - 1); else poison &= ~(1u << (sp - 1));
    }
    return sp == 1 && !(poison & 1u) && st[0] != 0;
}

// One constraint at an in-domain key, given the key's point index p in the constraint's
// block: one bit of its truth-mask table, or the interpreted program.
__device__ __forceinline__ bool cons_holds(const DevSpace* __restrict__ sp, const uint32_t* __restrict__ tables,
                                          uint64_t key, const DevBlock& bl, int c, int32_t p) {
    const DevCons& cs = sp->cons[c];
    if (cs.tabled) {
        uint32_t o = 0;
        for (int q = 0; q < cs.n_outer; ++q) o += (uint32_t)field(sp, key, cs.outer_k[q]) * cs.outer_stride[q];
        const uint32_t wv = __ldg(tables + cs.table_off + (uint64_t)o * bl.W + (p >> 5));
        return (wv >> (p & 31)) & 1u;
    }
    int64_t pv[MAXP];
    for (int k = 0; k < sp->n; ++k) pv[k] = sp->values[sp->vstart[k] + field(sp, key, k)];
    return vm_eval(sp->prog, cs.pc, cs.len, pv);
}

// One constraint at an in-domain key from its compact truth table: only the constraint's own
// parameters are read (the block tables need the key's whole block).
__device__ __forceinline__ bool cons_holds_compact(const DevSpace* __restrict__ sp, const DevCons& cs, uint64_t key) {
    uint32_t row = 0, c = 0;
    for (int q = 0; q < cs.n_outer; ++q) row += (uint32_t)field(sp, key, cs.outer_k[q]) * (uint32_t)cs.outer_stride[q];
    for (int q = 0; q < cs.n_in; ++q) c += (uint32_t)field(sp, key, cs.in_k[q]) * (uint32_t)cs.in_stride[q];
    const uint32_t wv = __ldg(sp->compact + cs.cz_off + (uint64_t)row * cs.cz_W + (c >> 5));
    return (wv >> (c & 31)) & 1u;
}

// One constraint at an in-domain key, from its compact table when it has one.
__device__ __forceinline__ bool cons_at(const DevSpace* __restrict__ sp, const uint32_t* __restrict__ tables,
                                       uint64_t key, int c) {
    const DevCons& cs = sp->cons[c];
    if (cs.cz_off != CZ_NONE) return cons_holds_compact(sp, cs, key);
    const DevBlock& bl = sp->blocks[cs.block];
    int32_t p = 0;
    for (int k = bl.s; k < bl.e; ++k) p += field(sp, key, k) * bl.pstride[k - bl.s];
    return cons_holds(sp, tables, key, bl, c, p);
}

// Full-tuple constraint test of an in-domain key: AND over every constraint.
__device__ __forceinline__ bool valid_key(const DevSpace* __restrict__ sp,
                                          const uint32_t* __restrict__ tables, uint64_t key) {
    const int nb = sp->n_blocks;
    for (int j = 0; j < nb; ++j) {
        const DevBlock& bl = sp->blocks[j];
        int32_t p = 0;
        for (int k = bl.s; k < bl.e; ++k) p += field(sp, key, k) * bl.pstride[k - bl.s];
        for (int c = bl.cons_begin; c < bl.cons_end; ++c)
            if (!cons_holds(sp, tables, key, bl, c, p)) return false;
    }
    return true;
}

// The constraints an in-domain key fails (bit c: constraint c); 0 for a valid key.
__device__ __forceinline__ uint64_t failing_mask(const DevSpace* __restrict__ sp,
                                                 const uint32_t* __restrict__ tables, uint64_t key) {
    uint64_t f = 0;
    const int nb = sp->n_blocks;
    for (int j = 0; j < nb; ++j) {
        const DevBlock& bl = sp->blocks[j];
        int32_t p = 0;
        for (int k = bl.s; k < bl.e; ++k) p += field(sp, key, k) * bl.pstride[k - bl.s];
        for (int c = bl.cons_begin; c < bl.cons_end; ++c)
            if (!cons_holds(sp, tables, key, bl, c, p)) f |= 1ull << c;
    }
    return f;
}

// The constraints c = part (mod G) that an in-domain key fails (G a power of two): G lanes with
// parts 0 .. G - 1 together give failing_mask.
__device__ __forceinline__ uint64_t failing_mask_part(const DevSpace* __restrict__ sp,
                                                      const uint32_t* __restrict__ tables, uint64_t key, int part,
                                                      int G) {
    uint64_t f = 0;
    const int nb = sp->n_blocks;
    for (int j = 0; j < nb; ++j) {
        const DevBlock& bl = sp->blocks[j];
        int c = bl.cons_begin + ((part - bl.cons_begin) & (G - 1));
        if (c >= bl.cons_end) continue;
        int32_t p = 0;
        for (int k = bl.s; k < bl.e; ++k) p += field(sp, key, k) * bl.pstride[k - bl.s];
        for (; c < bl.cons_end; c += G)
            if (!cons_holds(sp, tables, key, bl, c, p)) f |= 1ull << c;
    }
    return f;
}

// Changing the parameters of S leaves every constraint that reads none of them as it was.  So
// a point that differs from a candidate exactly in S can be valid only if each constraint the
// candidate fails reads a parameter of S ...
__device__ __forceinline__ bool fixes_possible(const DevSpace* __restrict__ sp, uint64_t fail, uint32_t S) {
    while (fail) {
        const int c = __ffsll((long long)fail) - 1;
        fail &= fail - 1;
        if (!(sp->cons[c].scope & S)) return false;
    }
    return true;
}

// ... and then it is valid iff the constraints reading a parameter of S hold at it (the union of
// the parameters' constraint masks; only those constraints are visited).
__device__ __forceinline__ bool valid_changed(const DevSpace* __restrict__ sp, const uint32_t* __restrict__ tables,
                                              uint64_t key, uint32_t S) {
    uint64_t cm = 0;
    for (uint32_t m = S; m; m &= m - 1u) cm |= sp->pcons[__ffs((int)m) - 1];
    while (cm) {
        const int c = __ffsll((long long)cm) - 1;
        cm &= cm - 1;
        const DevCons& cs = sp->cons[c];
        if (cs.cz_off != CZ_NONE) {
            if (!cons_holds_compact(sp, cs, key)) return false;
            continue;
        }
        const DevBlock& bl = sp->blocks[cs.block];
        int32_t p = 0;
        for (int k = bl.s; k < bl.e; ++k) p += field(sp, key, k) * bl.pstride[k - bl.s];
        if (!cons_holds(sp, tables, key, bl, c, p)) return false;
    }
    return true;
}

// Single-parameter filtering of the Hamming balls.  A point that changes exactly the parameters S
// of a candidate u can be valid only if, for every k in S and every constraint c whose scope meets
// S in k alone, c holds at u with k set to the point's value of k: c reads no other changed
// parameter.  Parameters with more than 64 values are not filtered.

// position of the n-th (from 0) set bit of m; m has more than n set bits
__device__ __forceinline__ int nth_bit(uint64_t m, uint32_t n) {
    for (uint32_t t = 0; t < n; ++t) m &= m - 1;
    return __ffsll((long long)m) - 1;
}

// The constraints (bit c) a point must still be tested on.
__device__ __forceinline__ bool valid_rest(const DevSpace* __restrict__ sp, const uint32_t* __restrict__ tables,
                                           uint64_t key, uint64_t rest) {
    while (rest) {
        const int c = __ffsll((long long)rest) - 1;
        rest &= rest - 1;
        if (!cons_at(sp, tables, key, c)) return false;
    }
    return true;
}

// Enumeration plan of one (candidate, subset), built by a whole warp (every lane returns the same
// plan): per parameter of S (highest first, the fastest digit) its allowed values (mask; 0 for an
// unfiltered parameter, whose values are all but u_k) and their count, and the constraints still
// to test at each point (those reading a parameter of S that the masks do not settle).  The lanes
// test the values of a parameter in parallel and a ballot forms each constraint's mask.  Returns
// the number of points (0: none).
struct BallPlan {
    uint64_t al[MAX_RADIUS];
    uint32_t cnt[MAX_RADIUS], uk[MAX_RADIUS];
    int k[MAX_RADIUS];
    int d;
    uint64_t rest;
};

__device__ __forceinline__ uint64_t ball_plan_warp(const DevSpace* __restrict__ sp, const uint32_t* __restrict__ tables,
                                                   uint64_t u, uint32_t S, int lane, BallPlan& bp) {
    uint64_t size = 1, touched = 0, cov = 0;
    bp.d = 0;
    uint32_t m = S;
#pragma unroll
    for (int e = 0; e < MAX_RADIUS; ++e) {
        if (!m) break;
        const int k = 31 - __clz(m);
        m &= ~(1u << k);
        const int r = sp->r[k];
        const uint32_t uk = (uint32_t)field(sp, u, k);
        const uint64_t pc = sp->pcons[k];
        touched |= pc;
        uint64_t a = 0;
        uint32_t cnt = (uint32_t)r - 1u;
        if (r <= 64) {
            a = (r == 64 ? ~0ull : ((1ull << r) - 1ull)) & ~(1ull << uk);
            for (uint64_t cm = pc; cm && a; cm &= cm - 1) {
                const int c = __ffsll((long long)cm) - 1;
                if ((sp->cons[c].scope & S) != (1u << k)) continue;
                uint64_t mk = 0;
                for (int v0 = 0; v0 < r; v0 += 32) {
                    const int v = v0 + lane;
                    bool ok = false;
                    if (v < r && ((a >> v) & 1ull))
                        ok = cons_at(sp, tables, (u & ~sp->fmask[k]) | ((uint64_t)v << sp->off[k]), c);
                    mk |= (uint64_t)__ballot_sync(0xffffffffu, ok) << v0;
                }
                a &= mk;
                cov |= 1ull << c;
            }
            cnt = (uint32_t)__popcll(a);
        }
        bp.al[e] = a; bp.cnt[e] = cnt; bp.uk[e] = uk; bp.k[e] = k;
        bp.d = e + 1;
        size *= cnt;
    }
    bp.rest = touched & ~cov;
    return size;
}

// The idx-th point of a plan.
__device__ __forceinline__ uint64_t ball_point(const DevSpace* __restrict__ sp, uint64_t u, const BallPlan& bp,
                                               uint64_t idx) {
    uint64_t key = u;
#pragma unroll
    for (int e = 0; e < MAX_RADIUS; ++e) {
        if (e >= bp.d) break;
        const uint32_t dg = (uint32_t)(idx % bp.cnt[e]);
        idx /= bp.cnt[e];
        const uint32_t v = bp.al[e] ? (uint32_t)nth_bit(bp.al[e], dg) : (dg < bp.uk[e] ? dg : dg + 1u);
        key = (key & ~sp->fmask[bp.k[e]]) | ((uint64_t)v << sp->off[bp.k[e]]);
    }
    return key;
}

// lower_bound over the sorted keys: first position with keys[pos] >= x.
__device__ __forceinline__ int64_t lower_bound_keys(const uint64_t* __restrict__ keys, int64_t n, uint64_t x) {
    int64_t base = 0, len = n;
    while (len > 0) {
        int64_t half = len >> 1;
        uint64_t v = __ldg(keys + base + half);
        if (v < x) { base += half + 1; len -= half + 1; } else { len = half; }
    }
    return base;
}

__device__ __forceinline__ int64_t rank_of(const uint64_t* __restrict__ keys, int64_t n, uint64_t x) {
    int64_t p = lower_bound_keys(keys, n, x);
    return (p < n && __ldg(keys + p) == x) ? p : -1;
}

// rank_of by a whole warp (every lane returns the result): a 32-ary search, each round narrowing
// the range to one of 32 chunks with one probe per lane (the last key of each chunk), so about
// log32 |V| rounds of independent loads instead of log2 |V| dependent ones.
__device__ __forceinline__ int64_t rank_of_warp(const uint64_t* __restrict__ keys, int64_t n, uint64_t x, int lane) {
    int64_t lo = 0, len = n;   // the first key >= x lies in [lo, lo + len]
    while (len > 32) {
        const int64_t step = (len + 31) / 32;
        const int64_t pos = lo + (int64_t)(lane + 1) * step - 1;
        const bool below = pos < lo + len && __ldg(keys + pos) < x;
        const int c = __popc(__ballot_sync(0xffffffffu, below));   // chunks entirely below x
        const int64_t nlo = lo + (int64_t)c * step;
        len = min(step, lo + len - nlo);
        lo = nlo;
    }
    const bool below = lane < len && __ldg(keys + lo + lane) < x;
    const int64_t p = lo + __popc(__ballot_sync(0xffffffffu, below));
    return (p < n && __ldg(keys + p) == x) ? p : -1;
}

// Status bits recorded by kernels into the space's device status word.
constexpr uint32_t ST_BAD_CANDIDATE = 1u;

}  // namespace ct
