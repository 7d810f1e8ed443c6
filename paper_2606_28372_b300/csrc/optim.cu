// The four constraint-aware optimizers (Sections IV-B..IV-D, Table IV) on the GPU.
//
// One run = one CTA per kernel.  A generation is propose -> repair ->
// post_repair (GA mutation) -> evaluate -> select.  Every random number comes
// from the counter-based Philox stream (seed; counter = word/4, individual,
// generation, purpose), so every individual draws independently and the result
// does not depend on thread scheduling.  Floating-point steps use explicitly
// rounded single-precision operations (no contraction), in the order the
// paper's formulas are written, so trajectories are reproducible bit for bit.
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <new>

#include "internal.hpp"
#include "optim_dev.cuh"

namespace ct {
ct_status evaluate_impl(ct_space* s, uint32_t* memo, unsigned long long* unique, unsigned long long* cost_acc,
                        const uint64_t* d_keys, int64_t n, float* d_fit, int64_t* d_rank, cudaStream_t st,
                        float invalid_fit = __builtin_inff());
}

namespace ct {

__global__ void __launch_bounds__(OPT_THREADS) k_propose(OptArgs a, uint32_t gen_arg, int use_dev, uint64_t* __restrict__ cand) {
    __shared__ int order[CT_MAX_POP];
    propose_dev(a, gen_of(a, gen_arg, use_dev), cand, order);
}

__global__ void __launch_bounds__(OPT_THREADS) k_post_repair(OptArgs a, uint32_t gen_arg, int use_dev, uint64_t* __restrict__ keys) {
    __shared__ GaMutSmem gm;
    post_repair_dev(a, gen_of(a, gen_arg, use_dev), keys, gm);
}

__global__ void __launch_bounds__(OPT_THREADS) k_select(OptArgs a, uint32_t gen_arg, int use_dev, const uint64_t* __restrict__ keys,
                                                        const float* __restrict__ fit) {
    __shared__ SelectSmem sm;
    select_dev(a, gen_of(a, gen_arg, use_dev), keys, fit, sm);
}

__global__ void k_set_gen(OptDev* st, uint32_t g) { st->gen = g; }

// A new run's device state: the initial run record, and zeroed positions, velocities and bests.
__global__ void k_opt_init(OptDev* __restrict__ st, const OptDev init, float* __restrict__ pos,
                           float* __restrict__ vel, float* __restrict__ pb, float* __restrict__ ynew, size_t PN,
                           float* __restrict__ gb, int N) {
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (size_t)gridDim.x * blockDim.x;
    if (t0 == 0) *st = init;
    for (size_t i = t0; i < PN; i += nt) { pos[i] = 0.0f; vel[i] = 0.0f; pb[i] = 0.0f; ynew[i] = 0.0f; }
    for (size_t i = t0; i < (size_t)N; i += nt) gb[i] = 0.0f;
}

}  // namespace ct

using namespace ct;

namespace ct {
ct_status surrogate_step(ct_opt* o, uint32_t gen, cudaStream_t st);

__global__ void k_ga_repair_words(OptArgs a, uint32_t gen_arg, int use_dev, uint32_t* __restrict__ words) {
    const uint32_t gen = gen_of(a, gen_arg, use_dev);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.P; i += gridDim.x * blockDim.x)
        words[i] = rng_word(a.seed, (uint32_t)i, gen, PU_GA_REPAIR, 0);
}

static ct_status repair_step(ct_opt* o, const OptArgs& a, uint32_t gen, int use_dev, cudaStream_t st) {
    if (!o->prm.constraint_aware) {   // baselines: candidates are evaluated as proposed
        CT_TRY_CUDA(cudaMemcpyAsync(o->rep.p, o->cand.p, (size_t)o->P * 8, cudaMemcpyDeviceToDevice, st));
        return CT_OK;
    }
    if (!o->prm.repair_rule) return repair_impl(o->s, o->rs, o->cand.p, o->P, o->rep.p, nullptr, st);
    if (o->kind == CT_DE)
        return repair_rule_impl(o->s, o->rules, 1, o->cand.p, o->P, nullptr, 0.0f, nullptr, o->rep.p, o->rs, st);
    if (o->kind == CT_GA) {
        k_ga_repair_words<<<(o->P + 255) / 256, 256, 0, st>>>(a, gen, use_dev, o->rules.words.p);
        count_launch();
        return repair_rule_impl(o->s, o->rules, 3, o->cand.p, o->P, nullptr, 0.0f, o->rules.words.p, o->rep.p, o->rs, st);
    }
    return repair_rule_impl(o->s, o->rules, 2, o->cand.p, o->P, o->kind == CT_PSO ? a.pos : a.ynew, a.eps, nullptr,
                            o->rep.p, o->rs, st);
}

static ct_status step_impl(ct_opt* o, uint32_t gen, int use_dev, cudaStream_t st) {
    const OptArgs a = o->args();
    k_propose<<<1, OPT_THREADS, 0, st>>>(a, gen, use_dev, o->cand.p);
    count_launch();
    if (!use_dev && gen == 0 && o->prm.constraint_aware) {
        // the initial sample draws valid ranks, so repair is the identity: skip its launches
        CT_TRY_CUDA(cudaMemcpyAsync(o->rep.p, o->cand.p, (size_t)o->P * 8, cudaMemcpyDeviceToDevice, st));
    } else {
        CT_TRY(repair_step(o, a, gen, use_dev, st));
    }
    if (o->kind == CT_GA && (use_dev || gen > 0)) {   // GA mutation; a no-op for the other kinds
        k_post_repair<<<1, OPT_THREADS, 0, st>>>(a, gen, use_dev, o->rep.p);
        count_launch();
    }
    CT_TRY(evaluate_impl(o->s, o->memo.p, &o->st.p->n_unique, &o->st.p->cost, o->rep.p, o->P, o->fit.p, nullptr, st,
                         CT_PENALTY));
    k_select<<<1, OPT_THREADS, 0, st>>>(a, gen, use_dev, o->rep.p, o->fit.p);
    count_launch();
    CT_TRY_CUDA(cudaGetLastError());
    if (!use_dev) o->dev_gen = gen + 1;   // select advances the device's generation
    return CT_OK;
}
}  // namespace ct

extern "C" {

void ct_opt_params_default(ct_opt_params* p) {
    if (!p) return;
    p->de_F = 0.7f; p->de_CR = 0.6f;
    p->pso_w = 0.5f; p->pso_c1 = 3.0f; p->pso_c2 = 0.5f;
    p->fa_beta0 = 1.0f; p->fa_gamma = 1.0f; p->fa_alpha = 0.2f;
    p->ga_pmut = 0.2f;
    p->target = -__builtin_inff();
    p->repair_rule = 0;
    p->constraint_aware = 1;
    p->de_mutation = CT_DE_BEST1;
    p->de_crossover = CT_DE_BIN;
    p->ga_crossover = CT_GA_SINGLE_POINT;
}

ct_status ct_opt_create(ct_space* s, ct_opt_kind kind, const ct_opt_params* params, int32_t pop, uint64_t seed, ct_opt** out) {
    if (!s || !out) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    *out = nullptr;
    if (kind < CT_DE || kind > CT_GA) { set_error("bad optimizer kind %d", (int)kind); return CT_ERR_INVALID_ARG; }
    if (pop < 3 || pop > CT_MAX_POP) { set_error("pop must be in [3, %d]", CT_MAX_POP); return CT_ERR_INVALID_ARG; }
    if (!s->built || s->n_valid == 0) { set_error("space not built or empty"); return CT_ERR_STATE; }
    if (!s->fit) { set_error("no fitness table"); return CT_ERR_STATE; }
    {
        ct_opt_params chk;
        if (params) chk = *params; else ct_opt_params_default(&chk);
        if (const char* why = check_operators(chk, kind, pop)) { set_error("%s", why); return CT_ERR_INVALID_ARG; }
    }
    ct_opt* o = new (std::nothrow) ct_opt();
    if (!o) { set_error("host allocation failed"); return CT_ERR_OOM; }
    o->s = s; o->kind = kind; o->P = pop; o->N = s->h.n; o->seed = seed;
    if (params) o->prm = *params; else ct_opt_params_default(&o->prm);
    int rmax = 1;
    for (int k = 0; k < s->h.n; ++k) rmax = s->h.r[k] > rmax ? s->h.r[k] : rmax;
    o->eps = rmax > 1 ? 1.0f / (float)(rmax - 1) : 1.0f;
    const size_t PN = (size_t)pop * o->N;
    o->memo_words = (s->n_valid + 31) / 32;
    ct_status e = CT_OK;
#define ALLOC(b, n) if (e == CT_OK) e = o->b.ensure(n)
    ALLOC(st, 1); ALLOC(X, pop); ALLOC(cand, pop); ALLOC(rep, pop); ALLOC(FX, pop); ALLOC(fit, pop);
    ALLOC(pos, PN); ALLOC(vel, PN); ALLOC(pb, PN); ALLOC(fpb, pop); ALLOC(gb, o->N); ALLOC(ynew, PN);
    ALLOC(memo, o->memo_words);
#undef ALLOC
    if (e == CT_OK) e = repair_reserve(o->rs, pop);
    if (e == CT_OK && o->prm.repair_rule) {   // everything the rule path needs, before any capture
        if (s->n_valid >= (1ull << 32)) { set_error("the paper's repair rules need |V| < 2^32"); e = CT_ERR_LIMIT; }
        if (e == CT_OK) e = rule_reserve(o->rules, pop, rule_slices_for(s));
        if (e == CT_OK) e = ensure_occ(s, nullptr);
        if (e == CT_OK && cudaDeviceSynchronize() != cudaSuccess) { set_error("occurrence table failed"); e = CT_ERR_CUDA; }
    }
    if (e != CT_OK) { delete o; return e; }
    OptDev init{};
    init.de_fbest = __builtin_inff();
    init.fgb = __builtin_inff();
    init.best_key = ~0ull;
    init.best_fit = __builtin_inff();
    init.hit_gen = -1;
    init.hit_evals = -1;
    // Asynchronous on the legacy default stream, after everything queued before (a space's build
    // may still be writing its last keys); the run's first use on another stream waits for the
    // event recorded behind it.
    const unsigned gi = (unsigned)std::min<size_t>((PN + 255) / 256 + 1, 1024);
    k_opt_init<<<gi, 256, 0, cudaStreamLegacy>>>(o->st.p, init, o->pos.p, o->vel.p, o->pb.p, o->ynew.p, PN, o->gb.p, o->N);
    count_launch();
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemsetAsync(o->memo.p, 0, o->memo_words * 4, cudaStreamLegacy) != cudaSuccess ||
        cudaEventCreateWithFlags(&o->ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(o->ready, cudaStreamLegacy) != cudaSuccess) {
        set_error("initialising run state failed");
        delete o;
        return CT_ERR_CUDA;
    }
    *out = o;
    return CT_OK;
}

void ct_opt_destroy(ct_opt* o) { delete o; }

ct_status ct_propose_population(ct_opt* o, uint32_t gen, uint64_t* d_cand, ct_stream stream) {
    if (!o || !d_cand) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    CT_TRY(o->wait_ready((cudaStream_t)stream));
    k_propose<<<1, OPT_THREADS, 0, (cudaStream_t)stream>>>(o->args(), gen, 0, d_cand);
    count_launch();
    CT_TRY_CUDA(cudaGetLastError());
    return CT_OK;
}

ct_status ct_opt_post_repair(ct_opt* o, uint32_t gen, uint64_t* d_keys, ct_stream stream) {
    if (!o || !d_keys) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    CT_TRY(o->wait_ready((cudaStream_t)stream));
    k_post_repair<<<1, OPT_THREADS, 0, (cudaStream_t)stream>>>(o->args(), gen, 0, d_keys);
    count_launch();
    CT_TRY_CUDA(cudaGetLastError());
    return CT_OK;
}

ct_status ct_opt_select(ct_opt* o, uint32_t gen, const uint64_t* d_keys, const float* d_fit, ct_stream stream) {
    if (!o || !d_keys || !d_fit) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    CT_TRY(o->wait_ready((cudaStream_t)stream));
    k_select<<<1, OPT_THREADS, 0, (cudaStream_t)stream>>>(o->args(), gen, 0, d_keys, d_fit);
    count_launch();
    CT_TRY_CUDA(cudaGetLastError());
    o->dev_gen = gen + 1;
    return CT_OK;
}

ct_status ct_evaluate(ct_space* s, ct_opt* o, const uint64_t* d_keys, int64_t n, float* d_fit, int64_t* d_rank,
                      ct_stream stream) {
    if (!s || n < 0 || (n > 0 && !d_keys)) { set_error("bad argument"); return CT_ERR_INVALID_ARG; }
    if (!s->built) { set_error("space not built"); return CT_ERR_STATE; }
    if (!s->fit && d_fit) { set_error("no fitness table"); return CT_ERR_STATE; }
    if (o && o->s != s) { set_error("run belongs to another space"); return CT_ERR_INVALID_ARG; }
    if (o) CT_TRY(o->wait_ready((cudaStream_t)stream));
    return evaluate_impl(s, o ? o->memo.p : nullptr, o ? &o->st.p->n_unique : nullptr, o ? &o->st.p->cost : nullptr,
                         d_keys, n, d_fit, d_rank, (cudaStream_t)stream);
}

// Generations [first, first + count) as one cached CUDA graph (generation read on the device).
static ct_status run_graph_impl(ct_opt* o, uint32_t first, uint32_t count, cudaStream_t st) {
    if (first == 0) {   // the initial generation runs eagerly (it skips the repair launches)
        CT_TRY(step_impl(o, 0, 0, st));
        if (--count == 0) return CT_OK;
        first = 1;
    }
    const ct_space* s = o->s;
    ct_opt::GraphSig sig;
    sig.keys = s->keys.p; sig.fit = s->fit; sig.cost = s->cost; sig.nv = s->n_valid;
    sig.mode = s->repair_mode; sig.max_radius = s->repair_max_radius; sig.dmax = wanted_radius(s);
    if (!(o->graph_sig == sig)) {   // the space changed under the graphs: capture again
        for (auto& gx : o->graphs) cudaGraphExecDestroy(gx.second);
        o->graphs.clear();
        o->graph_kernels.clear();
        o->graph_sig = sig;
    }
    auto it = o->graphs.find(count);
    if (it == o->graphs.end()) {
        CT_TRY(ensure_balls(o->s, sig.dmax));   // the ball tables the captured repair reads
        cudaStream_t cap;
        CT_TRY_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t g;
        ct_status e = CT_OK;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaStreamDestroy(cap);
            set_error("stream capture failed to start");
            return CT_ERR_CUDA;
        }
        const uint64_t c0 = ct_launch_count();
        for (uint32_t i = 0; i < count && e == CT_OK; ++i) e = step_impl(o, 0, 1, cap);
        const uint64_t captured = ct_launch_count() - c0;
        count_launch(0 - captured);   // captured launches have not run yet
        o->graph_kernels[count] = captured;
        cudaError_t ce = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (e != CT_OK) return e;
        if (ce != cudaSuccess) { set_error("capture failed: %s", cudaGetErrorString(ce)); return CT_ERR_CUDA; }
        cudaGraphExec_t ex;
        ce = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) { set_error("instantiate failed: %s", cudaGetErrorString(ce)); return CT_ERR_CUDA; }
        it = o->graphs.emplace(count, ex).first;
    }
    if (o->dev_gen != first) {   // the graph reads the generation on the device
        k_set_gen<<<1, 1, 0, st>>>(o->st.p, first);
        count_launch();
    }
    CT_TRY_CUDA(cudaGraphLaunch(it->second, st));
    count_launch(o->graph_kernels[count]);
    o->dev_gen = first + count;
    return CT_OK;
}

// Eager steps after which ct_opt_step replays a cached one-generation graph instead of launching
// kernel by kernel (a run that is stepped repeatedly; a short session captures nothing).
constexpr uint32_t STEP_GRAPH_AFTER = 2;

ct_status ct_opt_step(ct_opt* o, uint32_t gen, ct_stream stream) {
    if (!o) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    CT_TRY(o->wait_ready(st));
    if (o->sg) return surrogate_step(o, gen, st);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CT_TRY_CUDA(cudaStreamIsCapturing(st, &cs));
    if (gen > 0 && o->eager_steps >= STEP_GRAPH_AFTER && cs == cudaStreamCaptureStatusNone)
        return run_graph_impl(o, gen, 1, st);
    ++o->eager_steps;
    return step_impl(o, gen, 0, st);
}

ct_status ct_opt_run_graph(ct_opt* o, uint32_t first, uint32_t count, ct_stream stream) {
    if (!o || count == 0) { set_error("bad argument"); return CT_ERR_INVALID_ARG; }
    if (o->sg) { set_error("runs with a surrogate advance with ct_opt_step"); return CT_ERR_STATE; }
    cudaStream_t st = (cudaStream_t)stream;
    CT_TRY(o->wait_ready(st));
    return run_graph_impl(o, first, count, st);
}

ct_status ct_opt_best(ct_opt* o, uint64_t* best_key, float* best_fit, uint64_t* n_unique, int64_t* hit_generation,
                      int64_t* hit_evals, ct_stream stream) {
    if (!o) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    OptDev h;
    cudaStream_t st = (cudaStream_t)stream;
    CT_TRY(o->wait_ready(st));
    CT_TRY_CUDA(cudaMemcpyAsync(&h, o->st.p, sizeof h, cudaMemcpyDeviceToHost, st));
    CT_TRY_CUDA(cudaStreamSynchronize(st));
    if (best_key) *best_key = h.best_key;
    if (best_fit) *best_fit = h.best_fit;
    if (n_unique) *n_unique = h.n_unique;
    if (hit_generation) *hit_generation = h.hit_gen;
    if (hit_evals) *hit_evals = h.hit_evals;
    return ct_space_status(o->s, stream);
}

ct_status ct_opt_cost(ct_opt* o, uint64_t* cost, ct_stream stream) {
    if (!o || !cost) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long h = 0;
    CT_TRY(o->wait_ready(st));
    CT_TRY_CUDA(cudaMemcpyAsync(&h, &o->st.p->cost, sizeof h, cudaMemcpyDeviceToHost, st));
    CT_TRY_CUDA(cudaStreamSynchronize(st));
    *cost = h;
    return CT_OK;
}

ct_status ct_opt_state(const ct_opt* o, uint64_t* d_keys, float* d_fit, float* d_pos, ct_stream stream) {
    if (!o) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    CT_TRY(o->wait_ready(st));
    if (d_keys) CT_TRY_CUDA(cudaMemcpyAsync(d_keys, o->X.p, o->P * 8, cudaMemcpyDeviceToDevice, st));
    if (d_fit) CT_TRY_CUDA(cudaMemcpyAsync(d_fit, o->FX.p, o->P * 4, cudaMemcpyDeviceToDevice, st));
    if (d_pos) CT_TRY_CUDA(cudaMemcpyAsync(d_pos, o->pos.p, (size_t)o->P * o->N * 4, cudaMemcpyDeviceToDevice, st));
    return CT_OK;
}

// checkpoint layout: header, OptDev, then the device arrays in a fixed order
struct CkptHeader { uint32_t magic, version; int32_t kind, P, N; uint32_t pad; uint64_t seed, memo_words; };

ct_status ct_opt_save(const ct_opt* o, void* buf, size_t* len, ct_stream stream) {
    if (!o || !len) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    const size_t PN = (size_t)o->P * o->N;
    const size_t need = sizeof(CkptHeader) + sizeof(OptDev) + o->P * (8 + 4 + 4) + PN * 4 * 4 + o->N * 4 + o->memo_words * 4;
    if (!buf) { *len = need; return CT_OK; }
    if (*len < need) { set_error("buffer too small (%zu < %zu)", *len, need); return CT_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    CT_TRY(o->wait_ready(st));
    char* p = (char*)buf;
    CkptHeader hd{0x43545054u, 1u, o->kind, o->P, o->N, 0u, o->seed, o->memo_words};
    memcpy(p, &hd, sizeof hd); p += sizeof hd;
    struct { const void* src; size_t bytes; } parts[] = {
        {o->st.p, sizeof(OptDev)}, {o->X.p, (size_t)o->P * 8}, {o->FX.p, (size_t)o->P * 4}, {o->fpb.p, (size_t)o->P * 4},
        {o->pos.p, PN * 4}, {o->vel.p, PN * 4}, {o->pb.p, PN * 4}, {o->ynew.p, PN * 4}, {o->gb.p, (size_t)o->N * 4},
        {o->memo.p, o->memo_words * 4}};
    for (auto& pt : parts) { CT_TRY_CUDA(cudaMemcpyAsync(p, pt.src, pt.bytes, cudaMemcpyDeviceToHost, st)); p += pt.bytes; }
    CT_TRY_CUDA(cudaStreamSynchronize(st));
    *len = need;
    return CT_OK;
}

ct_status ct_opt_load(ct_opt* o, const void* buf, size_t len, ct_stream stream) {
    if (!o || !buf) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    const size_t PN = (size_t)o->P * o->N;
    const size_t need = sizeof(CkptHeader) + sizeof(OptDev) + o->P * (8 + 4 + 4) + PN * 4 * 4 + o->N * 4 + o->memo_words * 4;
    if (len < need) { set_error("checkpoint too short"); return CT_ERR_INVALID_ARG; }
    CkptHeader hd;
    memcpy(&hd, buf, sizeof hd);
    if (hd.magic != 0x43545054u || hd.kind != o->kind || hd.P != o->P || hd.N != o->N || hd.memo_words != o->memo_words) {
        set_error("checkpoint does not match this run (kind/pop/space)");
        return CT_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    CT_TRY(o->wait_ready(st));
    const char* p = (const char*)buf + sizeof hd;
    struct { void* dst; size_t bytes; } parts[] = {
        {o->st.p, sizeof(OptDev)}, {o->X.p, (size_t)o->P * 8}, {o->FX.p, (size_t)o->P * 4}, {o->fpb.p, (size_t)o->P * 4},
        {o->pos.p, PN * 4}, {o->vel.p, PN * 4}, {o->pb.p, PN * 4}, {o->ynew.p, PN * 4}, {o->gb.p, (size_t)o->N * 4},
        {o->memo.p, o->memo_words * 4}};
    for (auto& pt : parts) { CT_TRY_CUDA(cudaMemcpyAsync(pt.dst, p, pt.bytes, cudaMemcpyHostToDevice, st)); p += pt.bytes; }
    CT_TRY_CUDA(cudaStreamSynchronize(st));
    o->seed = hd.seed;
    o->dev_gen = ~0u;   // the loaded state carries its own generation
    return CT_OK;
}

}  // extern "C"
