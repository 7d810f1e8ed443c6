// Host-side internals of libcatune: handle layouts, error plumbing, shared launch helpers.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace ct {

void set_error(const char* fmt, ...);
void count_launch(uint64_t n = 1);

#define CT_TRY_CUDA(call)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            ::ct::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                            __LINE__);                                                      \
            return CT_ERR_CUDA;                                                             \
        }                                                                                   \
    } while (0)

#define CT_TRY(st)                     \
    do {                               \
        ct_status s_ = (st);           \
        if (s_ != CT_OK) return s_;    \
    } while (0)

// Process-wide cache of device blocks: a released block is kept for reuse by a later
// request of at most its size and at least half of it; on an allocation failure the
// cache is emptied and the allocation retried.  ct_trim_cache() returns it to the driver.
void* dev_alloc(size_t bytes, cudaError_t* err);
void dev_free(void* p, size_t bytes);

// Device buffer with grow-only capacity (blocks come from the cache above).
template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t cap = 0;
    ct_status ensure(size_t n) {
        if (n <= cap && p) return CT_OK;
        release();
        const size_t want = n ? n : 1;
        cudaError_t e = cudaSuccess;
        p = static_cast<T*>(dev_alloc(want * sizeof(T), &e));
        if (!p) {
            set_error("device allocation of %zu bytes failed: %s", want * sizeof(T), cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? CT_ERR_OOM : CT_ERR_CUDA;
        }
        cap = want;
        return CT_OK;
    }
    void release() {
        if (p) dev_free(p, cap * sizeof(T));
        p = nullptr;
        cap = 0;
    }
};

// Hamming-ball enumeration tables for one radius: the d-subsets of parameters (as
// bit masks over parameters with r_k > 1) and the prefix sums of their sizes
// prod_{k in S} (r_k - 1).
struct BallRadius {
    int d = 0;
    uint64_t total = 0;                // points at exactly distance d
    std::vector<uint32_t> masks;
    std::vector<uint64_t> prefix;      // size masks.size() + 1
    DevBuf<uint32_t> d_masks;
    DevBuf<uint64_t> d_prefix;
};

struct RepairScratch {
    DevBuf<int32_t> pend_a, pend_b;    // pending candidate indices
    DevBuf<uint32_t> counts;           // [0]: pending a, [1]: pending b
    DevBuf<unsigned long long> best;   // per pending slot: best key / packed (dist, rank)
    DevBuf<uint64_t> fail;             // per candidate: the constraints it fails
    DevBuf<uint32_t> done;             // ball kernels: CTAs finished (the last one resolves the radius)
    void release_all() {
        pend_a.release(); pend_b.release(); counts.release(); best.release(); fail.release(); done.release();
    }
};

// The resolve step of one ball radius, done by the ball kernel's last CTA (see search.cu).
struct BallNext {
    uint32_t* done;                 // CTAs finished (zero before the launch; the last CTA resets it)
    int d;                          // the radius
    uint64_t* out;                  // settled candidates: the repaired key
    uint8_t* dist;                  // ... and its distance (may be null)
    int32_t* pend_out;              // the rest, for the next radius
    uint32_t* count_out;
    unsigned long long* best_out;
};

// Scratch of the paper's repair rules (candidates, adjacency bounds, per-set minima,
// per-slice counts, chosen members, RNG words).
struct RuleScratch {
    DevBuf<int32_t> pend;
    DevBuf<uint8_t> rc;
    DevBuf<unsigned long long> best;
    DevBuf<uint32_t> count, cnt, words;
    DevBuf<int32_t> target;
    void release_all() {
        pend.release(); rc.release(); best.release(); count.release(); cnt.release(); words.release();
        target.release();
    }
};

}  // namespace ct

struct ct_space {
    int device = 0;
    ct::DevSpace h{};                      // host copy of the descriptor
    ct::DevSpace* d = nullptr;             // device copy
    std::vector<int> tab_cons;             // tabled constraints (indices into h.cons)
    std::vector<uint64_t> tab_prefix;      // cumulative table words, size tab_cons.size() + 1
    ct::DevBuf<uint32_t> tables;           // truth-mask arena
    ct::DevBuf<int32_t> d_tab_cons;
    ct::DevBuf<uint64_t> d_tab_prefix;
    std::vector<int> cz_cons;              // tabled constraints with a compact truth table
    std::vector<uint64_t> cz_prefix;       // cumulative compact words, size cz_cons.size() + 1
    ct::DevBuf<uint32_t> compact;          // compact truth tables (input of the table build)
    ct::DevBuf<int32_t> d_cz_cons;
    ct::DevBuf<uint64_t> d_cz_prefix;
    ct::DevBuf<uint32_t> innerkey;         // per block: point -> key bits (shifted)
    bool tables_ready = false;
    std::vector<uint32_t> ik_host;         // innerkey tables before upload
    ct::DevBuf<uint32_t> pat_cnt, pat_list;  // pattern-mode arenas
    uint64_t pat_cnt_words = 0, pat_list_words = 0;

    // build
    ct::DevBuf<uint64_t> keys;
    uint64_t n_valid = 0;
    bool built = false;
    std::vector<ct::DevBuf<uint64_t>> frontier;
    ct::DevBuf<uint32_t> tile_counts;
    ct::DevBuf<unsigned long long> tile_base;
    ct::DevBuf<unsigned long long> d_total;   // per level: the level's size (written by its scan)
    unsigned long long h_total = 0;
    std::vector<unsigned long long> h_totals;
    std::vector<uint64_t> hint;            // level sizes of the last build (empty before the first)

    // repair
    std::vector<ct::BallRadius> balls;     // enumerated radii 1..balls.size() (planned on demand)
    uint64_t ball_total[ct::MAX_RADIUS + 1] = {};   // points at distance d (sizes only)
    int ball_max = 0;                      // largest radius the ball tables may cover
    int repair_mode = 0, repair_max_radius = 0;
    ct::RepairScratch rs;
    ct::RuleScratch rules;                 // the paper's repair rules (public entry point)
    ct::DevBuf<uint32_t> occ;              // values of each parameter occurring in V
    bool occ_ready = false;

    // evaluate
    const float* fit = nullptr;
    uint64_t n_fit = 0;
    const uint32_t* cost = nullptr;        // simulated evaluation time per rank (borrowed), or null

    ct::DevBuf<uint32_t> status;           // device status word

    // measurement
    bool timing = false;
    ct_build_stats stats{};
    std::vector<cudaEvent_t> events;
    ~ct_space();
};

namespace ct {
ct_status ensure_device(ct_space* s, cudaStream_t st = nullptr, bool sync = true);   // sync: wait for the uploads
ct_status ensure_balls(ct_space* s, int dmax);
int wanted_radius(const ct_space* s);
ct_status repair_impl(ct_space* s, RepairScratch& rs, const uint64_t* d_cand, int64_t n, uint64_t* d_out,
                      uint8_t* d_dist, cudaStream_t st);
// Device scratch of one repair call: pending lists, their counters and argmin words (ping-pong
// between radii), the failing-constraint word of each candidate, and the ball kernels' CTA
// ticket.  The counters must be zero when the call starts, and so must the ticket (the ball
// kernels leave it at zero).
struct RepairPtrs {
    int32_t* pend[2];
    uint32_t* cnt[2];
    unsigned long long* best[2];
    uint64_t* fail;
    uint32_t* done;
};
// The launches of one repair (table test, Hamming balls of radii 1..dmax whose tables are on
// the device, exhaustive scan of whatever is left, resolve), on caller-provided scratch for n
// candidates; allocates nothing.
ct_status repair_launch(const ct_space* s, const RepairPtrs& p, int dmax, const uint64_t* d_cand, int64_t n,
                        uint64_t* d_out, uint8_t* d_dist, cudaStream_t st);
int auto_radius(const ct_space* s, double div = 8.0);   // div: the scan pass's cost, in ball points
ct_status scan_lut(const ct_space* s, const uint64_t* d_cand, const int32_t* pend, const uint32_t* count,
                   unsigned long long* best, cudaStream_t st, bool* launched, int* lut_min);
ct_status repair_reserve(RepairScratch& rs, int64_t n);
ct_status rule_reserve(RuleScratch& r, int64_t n, int slices);
int rule_slices_for(const ct_space* s);
ct_status ensure_occ(ct_space* s, cudaStream_t st);
ct_status repair_rule_impl(ct_space* s, RuleScratch& r, int rule, const uint64_t* d_cand, int64_t n,
                           const float* d_pos, float eps, const uint32_t* d_words, uint64_t* d_out,
                           RepairScratch& rs, cudaStream_t st);
}  // namespace ct
