/*
 * catune — constraint-aware evolutionary auto-tuning hot path for B300 (sm_103a).
 *
 * C ABI of libcatune.so.  The calls follow the paper's statement of the problem
 * ("Constraint-aware Optimization in Auto-Tuning"):
 *   - a search space is a CSP P = (X, D, C): parameters X with finite value lists D
 *     and constraints C, each a predicate over a subset of the parameters
 *     (Section IV-A);
 *   - the whole valid space is resolved before tuning (Section IV-A), giving a
 *     sorted list of valid configurations that supports validity queries,
 *     random valid samples and neighbour lookups;
 *   - four optimizers (DE: Algorithm 1 and Section IV-B; PSO and Firefly:
 *     Section IV-C; GA: Section IV-D, Algorithm 3) propose candidates, repair
 *     invalid ones to a valid neighbour and evaluate only valid ones.
 *
 * Conventions
 *   - A configuration is a tuple of value *indices* idx_k in [0, r_k).  Its key is
 *     K = sum_k idx_k << off_k with field widths w_k = ceil(log2 r_k) (0 when
 *     r_k == 1) and parameter n-1 in the lowest bits, so increasing key order is
 *     Cartesian order with the last parameter varying fastest.  The total width
 *     must be <= 64 bits.
 *   - "d_" pointers are device pointers, owned by the caller unless stated.  Host
 *     pointers are plain host memory.  Handles (ct_space, ct_opt) are owned by the
 *     library; destroy them with the matching *_destroy call.
 *   - Calls that take a stream are stream-ordered and asynchronous.  Calls that
 *     return host values synchronise the stream and say so.
 *   - Every call returns a ct_status; no C++ exception crosses the ABI.
 *     ct_last_error() returns a thread-local message for the last failure.
 *   - Errors found by kernels (a candidate outside the Cartesian domain) are
 *     recorded in the space's device status word and returned by the next call
 *     that synchronises (ct_space_status, ct_opt_best, ct_build_valid_space).
 *   - Fitness is a cost (a runtime): lower is better, as in Algorithm 1
 *     (a trial replaces x_i when f(u_i) <= f(x_i)).
 */
#ifndef CATUNE_H
#define CATUNE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ct_space ct_space;
typedef struct ct_opt ct_opt;
typedef struct ct_batch ct_batch;
typedef void *ct_stream; /* a cudaStream_t; NULL is the legacy default stream */

typedef enum {
    CT_OK = 0,
    CT_ERR_INVALID_ARG = 1,  /* bad pointer/size/enum, or a candidate outside the domain */
    CT_ERR_KEY_OVERFLOW = 2, /* sum of field widths > 64, or Cartesian size >= 2^63 */
    CT_ERR_EMPTY_SPACE = 3,  /* no configuration satisfies the constraints */
    CT_ERR_OOM = 4,          /* device or host allocation failed */
    CT_ERR_CUDA = 5,         /* a CUDA runtime call failed (message in ct_last_error) */
    CT_ERR_TIMEOUT = 6,      /* reserved: a bounded device wait expired */
    CT_ERR_STATE = 7,        /* call out of order (e.g. repair before build) */
    CT_ERR_LIMIT = 8         /* a documented size limit was exceeded */
} ct_status;

/* Size limits of one space. */
#define CT_MAX_PARAMS 32
#define CT_MAX_VALUES 4096      /* total entries over all value lists */
#define CT_MAX_CONSTRAINTS 64
#define CT_MAX_INSTR 4096       /* total instructions over all constraint programs */
#define CT_MAX_STACK 16
#define CT_MAX_POP 1024

/* ------------------------------------------------------------------------- */
/* constraint programs                                                       */
/* ------------------------------------------------------------------------- */
/* Each constraint c_j (Section IV-A) is a postfix program over 64-bit signed
 * integers, terminated by CT_OP_END; the programs of all constraints are
 * concatenated.  A constraint holds iff its final value is non-zero and not
 * poisoned.  Arithmetic wraps (two's complement); DIV and MOD truncate toward
 * zero; DIV or MOD by zero poisons the result; arithmetic on a poisoned operand
 * stays poisoned; a comparison with a poisoned operand is 0; AND/OR/NOT treat a
 * poisoned operand as false. */
typedef enum {
    CT_OP_END = 0,
    CT_OP_PARAM = 1, /* push the *value* (not the index) of parameter `arg` */
    CT_OP_CONST = 2, /* push `imm` */
    CT_OP_ADD = 3, CT_OP_SUB = 4, CT_OP_MUL = 5, CT_OP_DIV = 6, CT_OP_MOD = 7,
    CT_OP_NEG = 8, CT_OP_MIN = 9, CT_OP_MAX = 10,
    CT_OP_LT = 11, CT_OP_LE = 12, CT_OP_GT = 13, CT_OP_GE = 14, CT_OP_EQ = 15, CT_OP_NE = 16,
    CT_OP_AND = 17, CT_OP_OR = 18, CT_OP_NOT = 19
} ct_opcode;

typedef struct {
    int32_t op;  /* ct_opcode */
    int32_t arg; /* parameter index for CT_OP_PARAM */
    int64_t imm; /* constant for CT_OP_CONST */
} ct_instr;

/* ------------------------------------------------------------------------- */
/* search space (Section IV-A)                                               */
/* ------------------------------------------------------------------------- */
/* Defines P = (X, D, C).  n_values[k] (>= 1) is the length of parameter k's
 * value list; values_flat holds all lists back to back (host memory, copied).
 * program holds n_instr instructions (copied).  Host-only: lowers the
 * constraints (scope, deepest parameter, block plan) and uploads the
 * description to the current device.
 * Errors: INVALID_ARG (malformed program, bad sizes), KEY_OVERFLOW, LIMIT, OOM, CUDA. */
ct_status ct_define_space(int32_t n_params, const int32_t *n_values, const int64_t *values_flat,
                          const ct_instr *program, int32_t n_instr, ct_space **out);
void ct_space_destroy(ct_space *space);

typedef struct {
    int32_t n_params;
    int32_t n_constraints;
    int32_t key_bits;
    int32_t n_blocks;          /* enumeration blocks chosen by the planner */
    int32_t width[CT_MAX_PARAMS];
    int32_t offset[CT_MAX_PARAMS];
    int32_t n_values[CT_MAX_PARAMS];
    uint64_t cartesian;        /* prod n_values */
    uint64_t n_valid;          /* 0 until ct_build_valid_space */
    int32_t built;
} ct_space_info;
ct_status ct_space_info_get(const ct_space *space, ct_space_info *info);

/* Host helpers: value-index tuples (n rows of n_params int32) <-> keys.  Pack
 * rejects indices outside [0, r_k) with INVALID_ARG. */
ct_status ct_pack_keys(const ct_space *space, const int32_t *idx, int64_t n, uint64_t *keys);
ct_status ct_unpack_keys(const ct_space *space, const uint64_t *keys, int64_t n, int32_t *idx);
/* Device form of ct_unpack_keys: d_idx[i * n_params + k] = value index of parameter k in
 * d_keys[i] (device buffers, caller-owned; asynchronous on `stream`). */
ct_status ct_unpack_keys_device(const ct_space *space, const uint64_t *d_keys, int64_t n, int32_t *d_idx,
                                ct_stream stream);

/* Resolves the whole valid space on the device (Section IV-A): decodes the
 * Cartesian points, evaluates the constraints and compacts the valid keys in
 * increasing key order into a library-owned device array.  Writes |V| to
 * *n_valid_out.  Rebuilding replaces the previous keys.  The first build reads
 * each level's size back (synchronising the stream) before launching the next
 * level, and returns as soon as the last level's size is known: the last level's
 * keys are still being written, and every later call on the stream (or any work
 * ordered after it) sees them complete.
 * A rebuild of the same space (whose definition cannot change), when its buffers
 * already hold the previous build's sizes, launches every level from those sizes:
 * each emit checks its size against this build's own count on the device and
 * writes nothing on a mismatch, and the host checks all sizes once at the end,
 * synchronising the stream (a mismatch redoes the build level by level).
 * CATUNE_BUILD_PIPELINE=0 in the environment turns rebuilds from the previous
 * sizes off.
 * Errors: EMPTY_SPACE (|V| = 0; the space stays usable for queries), OOM, CUDA. */
ct_status ct_build_valid_space(ct_space *space, ct_stream stream, uint64_t *n_valid_out);

/* Borrowed pointer to the sorted valid keys (valid until rebuild/destroy). */
ct_status ct_space_keys(const ct_space *space, const uint64_t **d_keys, uint64_t *n_valid);

/* Registers the fitness table: d_table[rank] is the cost of the rank-th valid
 * key (float32, caller-owned, borrowed until destroy or the next call). */
ct_status ct_set_fitness(ct_space *space, const float *d_table, uint64_t n);

/* Registers the simulated evaluation time of each valid configuration (Eq. 2's time axis):
 * d_cost[rank] in microseconds (uint32, caller-owned, borrowed like the fitness table; NULL
 * removes it).  Every run on the space then accumulates, exactly (integer sums), the cost of
 * each configuration the first time it evaluates it; invalid proposals cost nothing. */
ct_status ct_set_eval_cost(ct_space *space, const uint32_t *d_cost, uint64_t n);

/* Validity query (Section IV-A): d_rank[i] = position of d_cand[i] in the valid
 * keys, or -1 if it is not a valid configuration (including keys outside the
 * domain).  Binary search. */
ct_status ct_lookup(const ct_space *space, const uint64_t *d_cand, int64_t n, int64_t *d_rank,
                    ct_stream stream);

/* Nearest-valid repair (Algorithm 1 Repair; Hamming neighbours of Section IV-A):
 * d_out[i] = the valid key minimising (Hamming distance on value indices, key)
 * lexicographically; a valid candidate maps to itself with distance 0.
 * d_dist[i] = that distance (nullable).  A candidate outside the Cartesian domain
 * is copied through with d_dist = 255 and records INVALID_ARG in the space status.
 * Uses library-owned scratch sized for n (grown on demand).  Requires a built,
 * non-empty space (else STATE / EMPTY_SPACE). */
ct_status ct_repair(ct_space *space, const uint64_t *d_cand, int64_t n, uint64_t *d_out,
                    uint8_t *d_dist, ct_stream stream);

/* Repair that allocates nothing (the paper has no counterpart to this call).
 * Same arguments and result as ct_repair, by the same kernels, for callers that
 * must not allocate device memory: host applications that reserve device memory
 * through their own allocator and forbid allocations from libraries, and
 * latency-sensitive loops in which an allocation, or cudaFree's implicit
 * device-wide synchronisation, would stall other streams.  Scratch comes from a
 * fixed array compiled into the library (one ~512 KB copy on every device that
 * loads it, held until the process exits), so n may not exceed
 * CT_REPAIR_NOALLOC_MAX (larger n returns CT_ERR_LIMIT; split the batch).  It
 * searches only the Hamming-ball radii whose tables are already on the device
 * (the build uploads every radius ct_repair uses) and scans exhaustively for the
 * rest, so the result is always exact.  The first call on each device looks up
 * the array's device address once; make that call before capturing any stream.
 * A cudaDeviceReset invalidates that address, as it does every handle and
 * buffer of this library.  All calls share the array: calls whose execution
 * overlaps on the GPU race on it, so the caller must order them (one stream, or
 * explicit synchronisation).  The space must already be built. */
#define CT_REPAIR_NOALLOC_MAX 16384
ct_status ct_repair_noalloc(ct_space *space, const uint64_t *d_cand, int64_t n, uint64_t *d_out,
                            uint8_t *d_dist, ct_stream stream);

/* The paper's own repair rules.  Neighbours of u (Section IV-A): strictly adjacent
 * (every parameter equal or the previous/next value index), adjacent (every parameter
 * equal or the nearest lower/higher value occurring in some valid configuration),
 * Hamming (exactly one parameter differs).  Invalid candidates are repaired by
 *   rule 1 (DE, Algorithm 1 Repair): the valid configuration with the smallest sum of
 *          absolute value-index differences, ties to the smallest key;
 *   rule 2 (PSO/Firefly, Algorithm 2): the first non-empty neighbour set's member nearest,
 *          by squared Euclidean distance in fp32, to the position d_pos[i*n_params ...] in the
 *          continuous embedding with grid spacing eps (ties to the smallest key);
 *   rule 3 (GA, Algorithm 3): member U[0, size) of the first non-empty neighbour set, in key
 *          order, drawn from the 32-bit word d_words[i].
 * Candidates with no neighbour in any set get the Hamming nearest valid key.  Valid
 * candidates map to themselves.  Exact streaming pass over the valid keys (cost grows with
 * |V| x n); requires |V| < 2^32.  Library-owned scratch. */
ct_status ct_repair_paper(ct_space *space, int32_t rule, const uint64_t *d_cand, int64_t n, const float *d_pos,
                          float eps, const uint32_t *d_words, uint64_t *d_out, ct_stream stream);

/* Repair strategy knob (tests and the autotuner): mode 0 = automatic (Hamming
 * ball search up to a radius chosen from a cost model, then an exhaustive key
 * scan), 1 = exhaustive scan only, 2 = ball search up to max_radius then scan. */
ct_status ct_set_repair_mode(ct_space *space, int32_t mode, int32_t max_radius);

/* Fitness lookup (memoised evaluation, Section IV-B): d_fit[i] = table[rank],
 * +inf for an invalid key; d_rank (nullable) as in ct_lookup.  With a non-NULL
 * opt, marks each rank in the run's memo bitmap and counts first visits as
 * unique evaluations.  Requires ct_set_fitness. */
ct_status ct_evaluate(ct_space *space, ct_opt *opt, const uint64_t *d_keys, int64_t n, float *d_fit,
                      int64_t *d_rank, ct_stream stream);

/* Reads and clears the space's device status word (synchronises). */
ct_status ct_space_status(ct_space *space, ct_stream stream);

/* ------------------------------------------------------------------------- */
/* optimizers (Sections IV-B..IV-D, Table IV)                                */
/* ------------------------------------------------------------------------- */
typedef enum { CT_DE = 0, CT_PSO = 1, CT_FIREFLY = 2, CT_GA = 3 } ct_opt_kind;

/* DE mutation on value indices (Section IV-B; x0.. are distinct random members other than
 * the target xi, best the best so far):  best1 = best + F(x0 - x1);  rand1 = x0 + F(x1 - x2);
 * rand2 = x0 + F(x1 - x2) + F(x3 - x4);  best2 = best + F(x0 - x1) + F(x2 - x3);
 * currenttobest1 = xi + F(best - xi) + F(x0 - x1);  randtobest1 = x0 + F(best - x0) + F(x1 - x2);
 * fp32, left to right, then rounded half-even and clipped.  The population must exceed the
 * number of random members (2, 3, 5, 4, 2, 3). */
typedef enum {
    CT_DE_BEST1 = 0, CT_DE_RAND1 = 1, CT_DE_RAND2 = 2, CT_DE_BEST2 = 3, CT_DE_CURRENTTOBEST1 = 4,
    CT_DE_RANDTOBEST1 = 5
} ct_de_mutation;
/* DE crossover: binomial (each gene from the mutant with probability CR, one random gene
 * always) or exponential (a cyclic run of genes from a random start, extended while the draws
 * stay below CR). */
typedef enum { CT_DE_BIN = 0, CT_DE_EXP = 1 } ct_de_crossover;
/* GA crossover (Section IV-D): one cut point; two cut points (the middle segment swaps; with
 * fewer than three parameters, one cut); uniform (each gene by a fair draw); disruptive uniform
 * (exactly half, rounded down, of the genes where the parents differ, chosen uniformly). */
typedef enum {
    CT_GA_SINGLE_POINT = 0, CT_GA_TWO_POINT = 1, CT_GA_UNIFORM = 2, CT_GA_DISRUPTIVE_UNIFORM = 3
} ct_ga_crossover;

typedef struct {
    float de_F, de_CR;               /* Table IV: 0.7, 0.6 (best1bin) */
    float pso_w, pso_c1, pso_c2;     /* Table IV: 0.5, 3.0, 0.5 */
    float fa_beta0, fa_gamma, fa_alpha; /* Table IV: 1.0, 1.0, 0.2 */
    float ga_pmut;                   /* Table IV: mutation_chance 5 -> 0.2 */
    float target;                    /* record unique evaluations when best <= target */
    int32_t repair_rule;             /* 0: Hamming nearest valid for every optimizer (default);
                                        1: the paper's rule per optimizer (ct_repair_paper: DE
                                        rule 1, PSO/Firefly rule 2 on the particle position, GA
                                        rule 3).  Single runs only (not batches, not surrogates). */
    int32_t constraint_aware;        /* 1 (default): the constraint-aware methods above.  0: the
                                        non-constraint-aware baselines of Sections IV-B/IV-C:
                                        random start over the Cartesian product (PSO/Firefly:
                                        random coordinates), no repair, GA mutation to any other
                                        value of one random parameter, and a static penalty
                                        CT_PENALTY as the fitness of an invalid configuration
                                        (nothing is evaluated, nothing counted). */
    int32_t de_mutation;             /* ct_de_mutation (default CT_DE_BEST1, Table IV) */
    int32_t de_crossover;            /* ct_de_crossover (default CT_DE_BIN) */
    int32_t ga_crossover;            /* ct_ga_crossover (default CT_GA_SINGLE_POINT, Table IV) */
} ct_opt_params;

#define CT_PENALTY 1e20f

/* Fills *p with the Table IV values, target = -inf, the Hamming repair (repair_rule 0), the
 * constraint-aware methods, and best1bin / single-point operators. */
void ct_opt_params_default(ct_opt_params *p);

/* Creates one run: population `pop` (3..CT_MAX_POP; DE needs one more than the random
 * members its mutation draws), counter-based
 * RNG seed `seed`.  Allocates the run's device state (population, positions,
 * memo bitmap of |V| bits) on the space's device and initialises it
 * asynchronously on the legacy default stream, behind the work already queued
 * there (the space's build may still be writing its last keys); the run's first
 * use on any other stream waits for that initialisation.  Requires a built space
 * with a fitness table.  The space must outlive the run. */
ct_status ct_opt_create(ct_space *space, ct_opt_kind kind, const ct_opt_params *params, int32_t pop,
                        uint64_t seed, ct_opt **out);
void ct_opt_destroy(ct_opt *opt);

/* One generation is: propose -> repair -> post_repair -> evaluate -> select.
 * Generation 0 proposes the initial valid sample (one rank per stratum of the
 * valid list); later generations apply the optimizer's operators.  Generations
 * must be issued in order 0, 1, 2, ...; `generation` is also the RNG counter.
 *
 * propose: writes pop candidate keys (unrepaired) to d_cand (caller-owned). */
ct_status ct_propose_population(ct_opt *opt, uint32_t generation, uint64_t *d_cand, ct_stream stream);
/* post_repair: GA mutation (replace a repaired child by a random valid Hamming
 * neighbour with probability ga_pmut, Section IV-D); a no-op for the others. */
ct_status ct_opt_post_repair(ct_opt *opt, uint32_t generation, uint64_t *d_keys, ct_stream stream);
/* select: consumes the evaluated keys and their fitness (pop entries each):
 * DE greedy selection with the u-not-in-X rule and stagnation re-draw, PSO
 * personal/global best, Firefly brightness, GA generational replacement; updates
 * the run's best (minimum (fitness, key) over everything evaluated). */
ct_status ct_opt_select(ct_opt *opt, uint32_t generation, const uint64_t *d_keys, const float *d_fit,
                        ct_stream stream);
/* The whole generation with run-owned buffers.  The first two calls of a run
 * launch kernel by kernel; later ones (generation > 0, on a stream that is not
 * being captured) replay a cached one-generation CUDA graph, with the same
 * result and far fewer launches. */
ct_status ct_opt_step(ct_opt *opt, uint32_t generation, ct_stream stream);
/* Runs generations [first, first + count) as one CUDA graph (captured on the
 * first call for this count, replayed afterwards).  Generation 0, when included,
 * runs eagerly before the graph: its sample is valid by construction, so it
 * skips the repair launches.  A run's graphs are captured again when the space's
 * keys, fitness or cost table, or repair strategy change. */
ct_status ct_opt_run_graph(ct_opt *opt, uint32_t first, uint32_t count, ct_stream stream);

/* Run summary (synchronises): best key and fitness so far, unique evaluations,
 * and the generation / unique-evaluation count at which best first reached
 * params.target (-1 if never).  Any pointer may be NULL. */
ct_status ct_opt_best(ct_opt *opt, uint64_t *best_key, float *best_fit, uint64_t *n_unique,
                      int64_t *hit_generation, int64_t *hit_evals, ct_stream stream);

/* Simulated time spent by the run so far (synchronises): the sum, over the configurations
 * it has evaluated (each once), of the space's evaluation cost (ct_set_eval_cost; 0 without). */
ct_status ct_opt_cost(ct_opt *opt, uint64_t *cost, ct_stream stream);

/* Copies the run state to caller buffers (asynchronous; any pointer may be NULL):
 * population keys [pop], population fitness [pop] (PSO: personal-best
 * fitness), positions [pop x n_params] (PSO/Firefly). */
ct_status ct_opt_state(const ct_opt *opt, uint64_t *d_keys, float *d_fit, float *d_pos, ct_stream stream);

/* Checkpoint: serialises the whole run state (population, positions, bests,
 * counters, memo bitmap) into a host buffer.  With buf == NULL, *len receives
 * the size.  Load restores a run created with the same space, kind and pop.
 * Both synchronise. */
ct_status ct_opt_save(const ct_opt *opt, void *buf, size_t *len, ct_stream stream);
ct_status ct_opt_load(ct_opt *opt, const void *buf, size_t len, ct_stream stream);

/* Copies the last generation's chosen proposals (before repair), repaired keys,
 * evaluated keys (GA: after mutation) and their fitness, pop entries each. */
ct_status ct_opt_last_generation(const ct_opt *opt, uint64_t *d_cand, uint64_t *d_rep, uint64_t *d_eval, float *d_fit,
                                 ct_stream stream);

/* ------------------------------------------------------------------------- */
/* MLP surrogate screening (an addition to the paper's method)               */
/* ------------------------------------------------------------------------- */
/* A small network on one-hot value indices (D = sum_k n_values[k] inputs) ->
 * hidden -> hidden -> hidden (ReLU) -> 1 predicts log-fitness.  fp32 master
 * weights, bf16 (round to nearest even) weights in the forward and backward
 * passes, fp32 accumulation in ascending index order on CUDA cores.  Flat
 * parameter layout: W1[H][D], b1[H], W2[H][H], b2[H], W3[H][H], b3[H], W4[H], b4.
 * Trained by SGD with momentum on mean squared error. */
typedef struct {
    int32_t pool;        /* proposals per population slot (16) */
    int32_t hidden;      /* width H (256) */
    int32_t batch;       /* training batch (256) */
    int32_t steps;       /* SGD steps per generation (8) */
    int32_t warmup_mult; /* screening needs >= warmup_mult * pop evaluations (4) */
    float lr, momentum;  /* 1e-2, 0.9 */
    float mae_ratio;     /* screening needs MAE <= mae_ratio * mean |y - mean y| of the generation (1.0:
                            the surrogate must predict the new evaluations better than their mean) */
} ct_surrogate_params;
void ct_surrogate_params_default(ct_surrogate_params *p);

/* Turns on screening for a DE or GA run before its generation 0.  d_log_table:
 * log-fitness per valid rank (caller-owned, borrowed).  Each generation the
 * surrogate is judged on the configurations just evaluated and trained on
 * batches drawn from everything evaluated; while it is accurate enough, the run
 * proposes `pool` candidates per slot, repairs all of them and evaluates only the
 * lowest-predicted one per slot.  Such runs advance with ct_opt_step only (which
 * then synchronises once per generation); ct_opt_run_graph returns STATE. */
ct_status ct_opt_set_surrogate(ct_opt *opt, const ct_surrogate_params *params, const float *d_log_table);
/* Last generation: screened or not, screening next, MAE, threshold, evaluated-set
 * size; d_params (nullable) receives the fp32 master parameters.  Synchronises. */
ct_status ct_opt_surrogate_info(ct_opt *opt, int32_t *screened, int32_t *use_next, float *mae, float *tau,
                                uint64_t *n_evaluated, float *d_params, ct_stream stream);

/* The network on its own (caller-owned device buffers). */
int64_t ct_mlp_param_count(int32_t D, int32_t H);
/* Glorot-uniform weights from the counter-based RNG, zero biases. */
ct_status ct_mlp_init(int32_t D, int32_t H, uint64_t seed, float *d_params, ct_stream stream);
size_t ct_mlp_workspace_bytes(int32_t D, int32_t H, int32_t B);
/* d_feats: B rows of N ascending feature indices (one active input per parameter). */
ct_status ct_mlp_forward(int32_t D, int32_t H, int32_t N, const float *d_params, const int32_t *d_feats, int32_t B,
                         float *d_pred, void *d_work, ct_stream stream);
/* Gradient of the batch mean squared error.  d_param_of holds D entries: d_param_of[f] = the
 * parameter (0..N-1) owning feature f; an entry outside 0..N-1 marks a feature that no sample
 * activates (its weight gradient is 0). */
ct_status ct_mlp_grad(int32_t D, int32_t H, int32_t N, const float *d_params, const int32_t *d_feats,
                      const int32_t *d_param_of, const float *d_y, int32_t B, float *d_grad, void *d_work,
                      ct_stream stream);
/* v = momentum*v + g; p = p - lr*v, elementwise. */
ct_status ct_mlp_sgd(float *d_params, float *d_mom, const float *d_grad, int64_t n, float lr, float momentum,
                     ct_stream stream);

/* ------------------------------------------------------------------------- */
/* batched runs                                                              */
/* ------------------------------------------------------------------------- */
/* Many independent runs of the optimizers above (Sections IV-B..IV-D) over
 * several built spaces, advanced together by one persistent kernel launch in
 * which each CTA takes whole runs from a work list and carries each through the
 * launch's generations (propose, repair, GA mutation, memoised evaluation and
 * selection on chip) before it takes the next.
 * Every run gives exactly the trajectory ct_opt gives for the same space, kind,
 * population, seed and parameters.  Population per run: 3..256. */
typedef struct {
    int32_t space;  /* index into the spaces array given to ct_batch_create */
    int32_t kind;   /* ct_opt_kind */
    int32_t pop;
    int32_t pad;
    uint64_t seed;
    float target;   /* record unique evaluations when the run's best <= target */
    int32_t pad2;
} ct_batch_run;

/* spaces: n_spaces built spaces with fitness tables (borrowed; must outlive the
 * batch).  params: shared hyper-parameters (NULL = Table IV); each run's target
 * replaces params->target.  Allocates all run state on the device. */
ct_status ct_batch_create(ct_space *const *spaces, int32_t n_spaces, const ct_batch_run *runs, int32_t n_runs,
                          const ct_opt_params *params, ct_batch **out);
void ct_batch_destroy(ct_batch *batch);
/* One generation for every run (generation 0 first). Asynchronous. */
ct_status ct_batch_step(ct_batch *batch, ct_stream stream);
/* `count` generations of every run in one launch (captured once per count as a
 * one-node CUDA graph, replayed). Asynchronous. */
ct_status ct_batch_run_graph(ct_batch *batch, uint32_t count, ct_stream stream);
/* Per-run summaries into host arrays of n_runs entries (each may be NULL). Synchronises. */
ct_status ct_batch_results(ct_batch *batch, uint64_t *best_key, float *best_fit, uint64_t *n_unique,
                           int64_t *hit_generation, int64_t *hit_evals, ct_stream stream);
/* Copies run `run`'s population keys, fitness and positions to caller device buffers. */
ct_status ct_batch_run_state(const ct_batch *batch, int32_t run, uint64_t *d_keys, float *d_fit, float *d_pos,
                             ct_stream stream);
/* Returns every run to its state before generation 0 (synchronises the device). */
ct_status ct_batch_reset(ct_batch *batch);
/* Per-generation trace of the first `gens` generations (0 switches it off): after each
 * generation g < gens every run records its best fitness so far, its simulated time
 * (ct_opt_cost; evaluation costs are those registered on the spaces when the batch was
 * created) and its unique evaluations.  With events > 0 every run also logs, up to `events`
 * entries, each strict improvement of its best in evaluation order (a generation's proposals
 * are evaluated one at a time in population order): generation, population index, simulated
 * time after that evaluation, new best.  Resets the batch and drops captured graphs. */
ct_status ct_batch_set_trace(ct_batch *batch, int32_t gens, int32_t events);
/* Copies the event log into host arrays: count[n_runs] (events seen; entries past the capacity
 * are dropped), and n_runs x capacity entries, run-major, of generation, index, simulated time
 * and best (each may be NULL).  Synchronises. */
ct_status ct_batch_events(const ct_batch *batch, uint32_t *count, int32_t *gen, int32_t *idx, uint64_t *clock,
                          float *fit, ct_stream stream);
/* Copies the trace into host arrays of n_runs x gens entries, run-major (each may be NULL);
 * generations not yet run read +inf, 0, 0.  Synchronises. */
ct_status ct_batch_trace(const ct_batch *batch, float *best_fit, uint64_t *cost, uint64_t *n_unique,
                         ct_stream stream);
/* Launch shape of the persistent kernel: threads per CTA (64, 128 or 256) and
 * CTAs per SM (0 = 4). Results do not depend on it. */
ct_status ct_batch_set_launch(ct_batch *batch, int32_t threads, int32_t ctas_per_sm);
/* Generations per launch of ct_batch_run_graph: 0 (the default) advances every run through all
 * `count` generations in one launch; k > 0 captures launches of k generations each (k = 1: one
 * persistent launch per generation, `count` kernel nodes in the graph).  Results do not depend
 * on it; with one launch per generation, every generation waits for its slowest run.  Drops
 * captured graphs. */
ct_status ct_batch_set_gens_per_launch(ct_batch *batch, int32_t gens);
/* Autotuner: times `gens` generations for each launch shape from the reset state,
 * requires every shape to end in the same state, keeps the fastest and resets the
 * batch.  cache_path (nullable): a JSON-lines file; a stored result for the same
 * batch signature is reused, a new one appended.  Synchronises. */
ct_status ct_batch_autotune(ct_batch *batch, const char *cache_path, int32_t gens, int32_t *threads_out,
                            int32_t *ctas_per_sm_out, float *ms_out, ct_stream stream);

/* ------------------------------------------------------------------------- */
/* measurement                                                               */
/* ------------------------------------------------------------------------- */
/* Per-level statistics of the last ct_build_valid_space: parents expanded,
 * children written, and (when timing is enabled) the device time of the count
 * and emit kernels, measured with CUDA events recorded on the build's stream. */
typedef struct {
    int32_t n_levels;
    int32_t timed;
    uint64_t parents[CT_MAX_PARAMS];
    uint64_t children[CT_MAX_PARAMS];
    float count_ms[CT_MAX_PARAMS];
    float emit_ms[CT_MAX_PARAMS];
    /* host wall time of the call's phases (always recorded): device setup of the space
     * description and the one-off table kernels, the levels (launches and the per-level size
     * reads), the ball tables after the build, and the whole call */
    float host_setup_ms, host_levels_ms, host_balls_ms, host_total_ms;
    /* 1: the levels were launched from the previous build's sizes, without a read per level */
    int32_t hinted;
} ct_build_stats;
ct_status ct_space_set_timing(ct_space *space, int32_t enable);
/* With timing on, waits for the build's last timed kernel before it reads the times. */
ct_status ct_space_build_stats(const ct_space *space, ct_build_stats *stats);

/* Device memory released by the library (destroyed spaces and runs, shrunk
 * buffers) is kept in a process-wide cache, at most 64 GiB per device, and reused
 * by later allocations of a similar size; an allocation that fails empties the cache
 * and retries.  ct_trim_cache returns the current device's cached blocks to the
 * driver. */
void ct_trim_cache(void);

/* Integer denominator of the key scans' roofline: runs a microbenchmark of independent 32-bit
 * xor / population-count / add chains over every SM of the current device, bound like the scans
 * by the population-count pipe, and writes population counts per second (synchronises). */
ct_status ct_measure_int_peak(double *popc_per_s, ct_stream stream);

/* Denominator of the surrogate's fixed-order fp32 products (CUDA cores, no tensor cores): runs
 * independent fp32 fused multiply-add chains over every SM of the current device and writes
 * floating-point operations per second, two per fused multiply-add (synchronises). */
ct_status ct_measure_fp32_peak(double *flop_per_s, ct_stream stream);

/* Denominator of the distance-table scan (bound by shared-memory loads): runs a microbenchmark
 * in which every warp reads 32 consecutive 16-byte entries of shared memory per load (four
 * 128-byte wavefronts, no bank conflict), four independent loads per step, over every SM of the
 * current device, and writes shared-memory wavefronts per second (synchronises). */
ct_status ct_measure_smem_peak(double *wavefronts_per_s, ct_stream stream);

/* Number of kernels this library has launched in this process (all devices). */
uint64_t ct_launch_count(void);

/* Number of device blocks this library has taken in this process (all devices), whether
 * from its cache or from the driver: a call that leaves it unchanged allocated nothing. */
uint64_t ct_alloc_count(void);

/* ------------------------------------------------------------------------- */
/* misc                                                                      */
/* ------------------------------------------------------------------------- */
const char *ct_last_error(void);
const char *ct_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CATUNE_H */
