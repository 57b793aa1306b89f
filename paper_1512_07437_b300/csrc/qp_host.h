// Host-side internals of libqp: device context, plans, buffers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/qp.h"
#include "qp_internal.h"

namespace qph {

constexpr int kMaxK = 46340;            // k(k-1)/2 stays below 2^30
constexpr int64_t kMaxLen = 1 << 20;    // per-sequence length limit

struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf();
    void release();
    cudaError_t ensure(size_t need);    // grow-only; contents are not kept
};

struct HostBuf {                        // pinned host memory
    void* ptr = nullptr;
    size_t bytes = 0;
    HostBuf() = default;
    HostBuf(const HostBuf&) = delete;
    HostBuf& operator=(const HostBuf&) = delete;
    ~HostBuf();
    cudaError_t ensure(size_t need);
};

// Work plan of one family shape (the vector of sequence lengths).
struct Plan {
    int k = 0;
    int64_t p0 = 0, p1 = 0;              // the pairs p0 <= p < p1 of the family's linear order
    std::vector<int64_t> lens;
    int max_len = 0;
    int64_t n_pairs = 0, n_rows = 0, n_strips = 0;
    int64_t bst_stride = 0, bex_stride = 0, bnd_stride = 0;   // per-warp FP32 scratch
    std::vector<int2> pairs;
    std::vector<int64_t> row_off, strip_off;
    std::vector<int32_t> order;          // pair ids, longest first
    std::vector<int64_t> work;           // swept lane-steps per pair
    double work_sum = 0;
    DevBuf d_pairs, d_row_off, d_strip_off, d_items;
};

struct LaunchOverride {                  // benchmark knobs (0 / -1: automatic)
    int warps_per_block = 0;
    int blocks_per_sm = 0;
    int variant = -1;
    int ckpt = -1;                       // 0 stored form, 1 checkpointed form
    int wpp = 0;                         // warps per pair (1, 2)
    bool graph = true;                   // run each call as one captured CUDA graph
    int64_t scratch_bytes = 0;           // budget of the FP32 / FP64 scratch
    int tree_form = -1;                  // guide tree: 0 one CTA, state in global memory; 1 one CTA,
                                         // state in shared memory; 2 cluster form; -1 automatic
    int tree_ctas = 0;                   // guide tree cluster form: CTAs (1, 2, 4, 8, 16; 0 automatic)
    int64_t pool_entries = 0;            // initial entry pool of a call (0: estimated)
    int cons_form = -1;                  // consistency: 0 row form, 1 staged form, -1 automatic
    int cons_chunk_rows = 0;             // consistency staged form: at most this many rows per CTA (0: by shared memory)
    int cons_min_unit = 0;               // consistency staged form: coarsest unit 2^-u accepted (0: 21)
    int cons_ctas_per_sm = 0;            // consistency staged form: CTAs per SM (1 or 2; 0: 2)
    int cons_wait_polls = 0;             // consistency staged form: waits on a stage buffer (0: default)
    int cons_stall_test = 0;             // testing: withhold the first batch's arrival (the wait runs out)
    int spin_limit = 0;                  // testing: polls of the FP32 kernel's strip waits (0: default)
    int tab_copies = -1;                 // emission table copies (1 or kTabCopies; -1: automatic)
    int host_chunks = 0;                 // host output: pair ranges whose copies overlap the next range's
                                         // compute (0 automatic, 1 never, n >= 2 forced)
};

// Device bytes the kernels' scratch may take: the override, else 45% of the
// free device memory, at most 48 GiB.
int64_t scratch_budget(const LaunchOverride& t);

// Launch configurations of the FP32 kernel the autotuner chooses from:
// config = variant + kF32Variants * (w + 2 * layout), with w indexing kWpp
// (warps per pair) and layout 0 = blocks of 2 warps with one emission table,
// 1 = blocks of 8 warps with the bank-sliced table (kTabCopies copies).
constexpr int kWpp[2] = {1, 2};
constexpr int kTuneConfigs = qpk::kF32Variants * 2 * 2;
inline int config_variant(int cfg) { return cfg % qpk::kF32Variants; }
inline int config_wpp(int cfg) { return kWpp[(cfg / qpk::kF32Variants) % 2]; }
inline int config_layout(int cfg) { return cfg / (qpk::kF32Variants * 2); }

// Online choice among the allowed launch configurations, per shape bucket
// (pair count, longest sequence, mean work): each is timed on kTuneSamples
// real calls (the first of a configuration can pay for cold caches and fresh
// scratch), then the fastest (best sample) is kept.
constexpr int kTuneSamples = 2;
struct TuneEntry {
    double ms[kTuneConfigs];
    int n[kTuneConfigs];
    TuneEntry() { for (int v = 0; v < kTuneConfigs; ++v) { ms[v] = -1.0; n[v] = 0; } }
    int choose(unsigned allowed) const {
        for (int v = 0; v < kTuneConfigs; ++v)
            if ((allowed >> v & 1u) && n[v] < kTuneSamples) return v;
        int best = -1;
        for (int v = 0; v < kTuneConfigs; ++v)
            if ((allowed >> v & 1u) && (best < 0 || ms[v] < ms[best])) best = v;
        return best < 0 ? 0 : best;
    }
    void record(int v, double t) {
        ms[v] = ms[v] < 0 ? t : (t < ms[v] ? t : ms[v]);
        ++n[v];
    }
};

// Configurations worth trying for a launch of n_pairs pairs whose longest
// sequence spans max_strips strips, on warps_full resident warps: several
// warps per pair only when pairs are too few to balance the grid and pairs
// have strips to share; wpp must divide warps_per_block.  Layout 1 (8-warp
// blocks, bank-sliced table) only when wide_layout: the launch fills the grid
// and two such blocks fit an SM; warps_per_block is layout 0's.
unsigned allowed_configs(int64_t n_pairs, int max_strips, int64_t warps_full, int warps_per_block,
                         const LaunchOverride& t, bool wide_layout = false);

// Grid of the persistent FP32 kernel for blocks_needed blocks of work: at most
// blocks_per_sm per SM, and a multiple of the SM count once it exceeds it.
int64_t balanced_grid(int sm_count, int blocks_per_sm, int64_t blocks_needed);

// Identity of a captured call sequence (see launch_graph).
struct GraphKey {
    const void* p[24];
    int64_t v[16];
    qpk::Problem pb;
};

struct Context {
    int device = 0;
    int sm_count = 0;
    int cc_major = 0, cc_minor = 0;
    int smem_optin = 0;                  // shared memory a block may opt in to (bytes)
    int smem_per_sm = 0;                 // shared memory of an SM (bytes)
    int f32_blocks_per_sm = 3;
    int f64_blocks_per_sm = 2;
    cudaStream_t stream = nullptr;
    cudaStream_t copy_stream = nullptr;  // host output in ranges: the copies of a finished range
    int64_t tune_alias = 0;              // when set, calls take this shape's tuned launch (and do not time)
    cudaEvent_t ev_join = nullptr;       // orders the library stream after the legacy default stream
    cudaEvent_t ev[6] = {};
    cudaGraphExec_t gexec = nullptr;     // the last captured call sequence
    GraphKey gkey;                       // what it was captured with
    bool gkey_valid = false;
    int64_t graph_captures = 0, graph_relaunches = 0, plain_calls = 0, pool_retries = 0;
    // result blocks freed by the caller, kept for the next call of the same
    // shape (same addresses: the captured graph is relaunched as it is)
    std::mutex spare_mu;
    std::list<std::pair<size_t, void*>> spare;   // least recently freed first
    size_t spare_bytes = 0;
    cudaError_t take_block(void** p, size_t bytes, cudaStream_t st);
    void give_block(void* p, size_t bytes);
    std::mutex mu;
    std::vector<std::shared_ptr<Plan>> plans;
    // workspace (grow-only)
    DevBuf ascii, codes, off, seqlogq, cst, d_raw, status, fam;
    qpk::RawParams last_raw;             // parameters the tables in cst were derived from
    bool raw_valid = false;
    DevBuf row_cnt, chunk_off, pair_nnz, fallback, pool, pool64;
    // selective consistency: workspace, entry pool, pinned status, events
    std::mutex cons_mu;
    DevBuf cons_ws, cons_pool;
    HostBuf cons_h;
    int64_t cons_pool_hint = 0;
    int64_t cons_fma = 0;                // multiply-adds of the last relaxation
    int cons_last_form = -1;             // form of the last relaxation (0 row form, 1 staged form)
    int last_variant = -1, last_wpp = -1, last_wpb = -1, last_copies = -1;   // last FP32 launch
    cudaEvent_t cons_ev[2] = {};
    // guide tree: working memory kept between calls, pinned staging
    std::mutex tree_mu;
    DevBuf tree_ws;
    HostBuf tree_h;
    int tree_optin = 0;                  // shared memory a CTA may opt in to
    DevBuf bst, bex, bnd, bck, stg;
    DevBuf d_b, d_diag, d_cnt, d_stg, d_stg64;
    // entry budget: the full CSR before the filter, per-pair counts after it,
    // the select's state and histogram
    DevBuf bud_rp, bud_off, bud_col, bud_val, bud_val64, bud_nnz, bud_state, bud_hist;
    HostBuf h_status, h_off, h_fam;
    int64_t pool_cap = 0;
    int64_t pool_hint = 0;
    LaunchOverride tune;
    std::map<int64_t, TuneEntry> tuner;
    static int64_t tune_key(int64_t n_pairs, int max_len, double work);
    std::shared_ptr<Plan> plan_for(int k, const int64_t* off, int* status, int64_t p0 = 0, int64_t p1 = -1);
};

// Device layout of a result's fixed-size part (one allocation): per-pair and
// per-row arrays and the k x k distance matrices.  col / val live in a second
// allocation sized by the entry count.
inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
struct ResultLayout {
    size_t o_pro = 0, o_rp = 0, o_pno = 0, o_dist = 0, o_d64 = 0, o_mea = 0, o_lh = 0, o_lp = 0, o_fl = 0;
    size_t bytes = 0;
    ResultLayout() = default;
    ResultLayout(int64_t n_pairs, int64_t n_rows, int k) {
        size_t sz = 0;
        o_pro = sz;  sz += align256(sizeof(int64_t) * (n_pairs + 1));
        o_rp = sz;   sz += align256(sizeof(int32_t) * n_rows);
        o_pno = sz;  sz += align256(sizeof(int64_t) * (n_pairs + 1));
        o_dist = sz; sz += align256(sizeof(float) * (size_t)k * k);
        o_d64 = sz;  sz += align256(sizeof(double) * (size_t)k * k);
        o_mea = sz;  sz += align256(sizeof(double) * n_pairs);
        o_lh = sz;   sz += align256(sizeof(double) * n_pairs);
        o_lp = sz;   sz += align256(sizeof(double) * n_pairs);
        o_fl = sz;   sz += align256(sizeof(int32_t) * n_pairs);
        bytes = sz;
    }
    // bytes of the col / val part for nnz entries
    static size_t entry_bytes(int64_t nnz, bool f64) {
        return align256(sizeof(int32_t) * nnz) + align256(sizeof(float) * nnz) +
               (f64 ? align256(sizeof(double) * nnz) : 0);
    }
};

// Owner of a result's memory (qp_result::owner_).
struct ResultOwner {
    int device = 0;
    bool on_device = true;
    void* dev_a = nullptr;   // fixed-size part (ResultLayout)
    void* dev_b = nullptr;   // col / val part
    size_t bytes_a = 0, bytes_b = 0;   // sizes when the blocks may be kept for reuse (else 0)
    void* host = nullptr;     // host copy (one block: take_host_block)
    size_t host_bytes = 0;
    bool host_pinned = false;
};

// Host blocks of results copied to host memory: pinned (so the copies run at
// full link speed) and kept after qp_result_free for the next result of the
// same size, since pinning memory is slow and cudaFreeHost waits for the
// device.  Plain malloc memory when pinning fails.
void* take_host_block(size_t bytes, bool* pinned);
void give_host_block(void* p, size_t bytes, bool pinned);

// Fills the public result from the two device parts (B may be null when nnz = 0
// is known in advance).  The caller sets nnz, n_fallback, guard_info, kernel_ms.
void fill_result(qp_result* r, ResultOwner* own, const ResultLayout& L, int k, int64_t n_pairs,
                 int64_t n_rows, int64_t nnz_bound, bool f64, int precision, int device);

// Letters of an alphabet (QP_PROTEIN: 20, QP_NUCLEOTIDE: 4) and the error
// message for a residue outside it.
inline int alphabet_size(int alphabet) { return alphabet == QP_NUCLEOTIDE ? 4 : 20; }
inline const char* alphabet_error(int alphabet) {
    return alphabet == QP_NUCLEOTIDE ? "a residue is outside the nucleotide alphabet ACGT (U read as T)"
                                     : "a residue is outside the 20-letter alphabet ACDEFGHIKLMNPQRSTVWY";
}
// Host check of one residue byte (the encode kernel checks again on the device).
inline bool valid_residue(uint8_t c, int alphabet) {
    const char* letters = alphabet == QP_NUCLEOTIDE ? "ACGTUacgtu" : "ACDEFGHIKLMNPQRSTVWYacdefghiklmnpqrstvwy";
    for (const char* l = letters; *l; ++l)
        if ((uint8_t)*l == c) return true;
    return false;
}

int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
const char* last_error();
int validate_family(const qp_family* f);
int validate_params(const qp_params* p);
void make_raw(const qp_params* p, qpk::RawParams* r);
void make_coef(const qp_params* p, qpk::Coef* c);
int row_capacity(const qp_params* p, int max_len);
std::shared_ptr<Plan> build_plan(int k, const int64_t* off, int64_t p0 = 0, int64_t p1 = -1);
Context* get_context(int device, int* status);
// The stream a call runs on: the caller's, or when it is NULL the library's
// stream, made to wait first for all work issued so far to the legacy
// default stream (so inputs written there are complete).
cudaError_t call_stream(Context* C, void* user, cudaStream_t* st);

// Longest sequence the FP32 form takes on the context's device with blocks of
// warps_per_block warps: every warp stages its pair's column residues in
// shared memory, so such a block must fit the per-block opt-in shared memory
// (0 when not even a one-residue block fits).
int f32_max_len(const Context* C, int warps_per_block);
int run_family(Context* C, const qp_family* f, const qp_params* prm, int32_t out_on_device,
               qp_result** out, int64_t p0 = 0, int64_t p1 = -1);
int to_host(qp_result* r, cudaStream_t st);
cudaError_t launch_graph(Context* C, cudaStream_t st, const GraphKey& key,
                         const std::function<cudaError_t()>& enqueue);
constexpr int kF64FollowGrid = 16;      // CTAs of the FP64 follow-up of an FP32 call
void free_result(qp_result* r);

}  // namespace qph
