// Serving loop with continuous batching: many families processed in one run
// under a device memory limit (the paper's bulk mode and memory limit,
// Methods, "Other algorithmic improvements").
//
//   submit (caller's thread): checks and copies the family, builds its pair
//     plan and the device bytes it will hold while resident; queues it.
//   worker thread: admits queued families while a family slot is free and
//     the memory budget holds their bytes (arrival order; later families
//     that fit pass one that does not, until it has waited past the aging
//     bound).  An admitted
//     family's sequences, work arrays, entry pool and per-pair results stay
//     in device memory until it completes.  The worker keeps two persistent
//     launches of the FP32 posterior kernel queued back to back on its
//     stream; each launch draws pairs from every admitted family (least
//     remaining work first; families admitted longer ago than the aging
//     bound get up to half of every launch), so a family admitted while
//     others run joins the next launch and shares it with them.  Pairs whose range guards fired go to
//     an FP64 follow-up launch.  When all pairs of a family are done its CSR
//     is assembled on the device and the family moves to the finisher.
//   finisher thread: reads the entry count, copies the result to the host
//     (unless results stay on the device), frees the family's working memory
//     and returns its bytes to the budget.
#include "../../include/qp.h"
#include "qp_host.h"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <vector>

using namespace qph;

namespace {

constexpr int kSlots = 64;                 // families resident at once
constexpr int kRecs = 4;                   // launch records (FP32 launches and FP64 follow-ups)
constexpr int kInflight = 2;               // FP32 launches queued on the device
constexpr int64_t kMaxItems = 1 << 20;     // pairs per launch
constexpr int kF64Grid = 16;               // CTAs of an FP64 follow-up launch
constexpr int kWpb = 4;                    // warps per block of the FP32 kernel

enum { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3, kCancelled = 4 };

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Job {
    uint64_t ticket = 0;
    std::vector<uint8_t> residues;
    std::vector<int64_t> offsets;
    std::shared_ptr<Plan> plan;
    double cells = 0;               // sum of m*n over the pairs
    int64_t pool_cap = 0;           // entries of the initial pool
    size_t blk_bytes = 0, res_bytes = 0;
    size_t reserve = 0;             // bytes held while resident (grows if the pool does)
    int state = kQueued;
    bool cancel = false;
    int rc = QP_OK;
    std::string err;
    qp_result* result = nullptr;
    double t_submit = 0, t_admit = 0, t_work_done = 0, t_done = 0;
};

// Offsets inside a family's resident block.
struct BlkLayout {
    size_t o_ascii, o_codes, o_off, o_logq, o_pairs, o_strip, o_rowcnt, o_chunk, o_pnnz, o_used, bytes;
    BlkLayout(int k, int64_t total, int64_t P, int64_t n_rows, int64_t n_strips) {
        size_t s = 0;
        o_ascii = s;  s += align256(total);
        o_codes = s;  s += align256(total);
        o_off = s;    s += align256(sizeof(int64_t) * (k + 1));
        o_logq = s;   s += align256(sizeof(double) * k);
        o_pairs = s;  s += align256(sizeof(int2) * P);
        o_strip = s;  s += align256(sizeof(int64_t) * (P + 1));
        o_rowcnt = s; s += align256(sizeof(int32_t) * n_rows);
        o_chunk = s;  s += align256(sizeof(int64_t) * n_strips);
        o_pnnz = s;   s += align256(sizeof(int64_t) * P);
        o_used = s;   s += align256(sizeof(unsigned long long));
        bytes = s;
    }
};

// An admitted family (worker-owned until it moves to the finisher).
struct Fam {
    std::shared_ptr<Job> job;
    int slot = -1;
    char* blk = nullptr;
    int2* pool = nullptr;
    int64_t pool_cap = 0;
    ResultOwner* own = nullptr;      // dev_a = fixed result part
    ResultLayout lay;
    qpk::FamDesc fd;
    int64_t next = 0;                // entries of plan->order already launched
    int64_t outstanding = 0;         // launched and not complete
    double remaining = 0;            // work not yet launched
    int attempts = 0;
    int64_t n_fallback = 0;
    int32_t guard[12] = {};
    bool have_guard = false;
    bool failed = false;
    int rc = QP_OK;
    std::string err;
    cudaEvent_t ev_done = nullptr;
    qp_result* result = nullptr;
};

struct Rec {
    int phase = 0;                   // 0 free, 1 FP32 queued, 2 FP64 follow-up queued
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int2* d_items = nullptr;
    int2* d_fallback = nullptr;
    qpk::Status* d_status = nullptr;
    std::vector<int2> items;
    std::vector<std::pair<int, int64_t>> per_fam, per_fam_f64;
    double work = 0, cells = 0;
    int variant = 0;
    int cfg = 0;
    int64_t tkey = 0;
};

}  // namespace

struct qp_server {
    qp_params params;
    qpk::Coef cf;
    size_t budget = 0;
    int device = 0;
    int out_on_device = 0;
    Context* ctx = nullptr;
    cudaStream_t cs = nullptr, up = nullptr, down = nullptr;
    double target_ms = 30.0, aging_s = 5.0;
    // device state
    qpk::Consts* d_cst = nullptr;
    qpk::RawParams* d_raw = nullptr;
    qpk::FamDesc* d_fams = nullptr;
    qpk::Status* d_enc_status = nullptr;
    void* d_rec_mem = nullptr;
    HostBuf h_status, h_fb, h_used;
    // kernel scratch, sized for sequences up to scratch_len (stream-ordered on cs)
    int scratch_len = 0;
    int cap = 0;
    int64_t scratch_warps = 0;
    int bps[qpk::kF32Variants] = {};
    int f64_grid = 0;            // CTAs of the FP64 follow-up (its scratch holds that many pairs)
    size_t scratch_bytes = 0;
    bool ckpt = false;               // checkpointed form of the FP32 kernel
    void *bst = nullptr, *bex = nullptr, *bnd = nullptr, *bck = nullptr, *stg = nullptr;
    void *d_b = nullptr, *d_diag = nullptr, *d_cnt = nullptr, *d_stg = nullptr, *d_stg64 = nullptr;
    // shared with the callers (mu)
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_fin;
    std::deque<std::shared_ptr<Job>> queue;
    std::map<uint64_t, std::shared_ptr<Job>> jobs;
    std::deque<std::unique_ptr<Fam>> fin_queue;
    uint64_t next_ticket = 1;
    bool stop = false, worker_done = false;
    size_t reserved = 0;
    int fatal_rc = QP_OK;
    std::string fatal_err;
    qp_server_stats stats;
    // worker only
    std::unique_ptr<Fam> fams[kSlots];
    Rec recs[kRecs];
    std::deque<int> issued;
    std::map<int64_t, TuneEntry> tuner;
    double rate = 4.0e6;             // work units (swept lane-steps) per ms, running estimate
    std::thread worker, finisher;
};

namespace {

// CTAs of the FP64 follow-up for sequences up to L: kF64Grid, fewer when
// their scratch would pass kF64Scratch (each CTA holds a whole pair's
// stored backward values, (L + 1)^2 of them), at least one
constexpr int64_t kF64Scratch = (int64_t)2 << 30;
int64_t f64_cta_bytes(int L, int cap) {
    const int64_t L1 = L + 1;
    return (int64_t)(sizeof(double2) * L1 * L1 + sizeof(double) * 3 * qpk::kNS * L1 + sizeof(int32_t) * (5 * L1 + 8) +
                     (sizeof(int2) + sizeof(double)) * (int64_t)L * cap);
}
int f64_grid_for(int L, int cap) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(kF64Grid, kF64Scratch / f64_cta_bytes(L, cap)));
}

// Device bytes of the kernels' scratch for sequences up to L.  The stored
// form is used while its scratch takes at most a third of the budget, else
// the checkpointed form.
size_t scratch_bytes_for(const qp_server* S, int L, int64_t* warps_out, int* bps_out, int* cap_out,
                         bool* ckpt_out) {
    if (L <= 0) return 0;
    const int cap = row_capacity(&S->params, L);
    bool ckpt = false;
    int64_t warps = 0;
    size_t b = 0;
    for (int pass = 0; pass < 2; ++pass) {
        int bmax = 1;
        for (int v = 0; v < qpk::kF32Variants; ++v) {
            int bb = 0;
            qpk::posterior_f32_occupancy(kWpb, L, &bb, v, ckpt);
            bb = std::max(1, std::min(bb, 8));
            if (bps_out) bps_out[v] = bb;
            bmax = std::max(bmax, bb);
        }
        warps = (int64_t)S->ctx->sm_count * bmax * kWpb;
        // room for one or two warps per pair
        b = std::max(qpk::F32Scratch(L, cap, ckpt, 1).bytes(warps), qpk::F32Scratch(L, cap, ckpt, 2).bytes(warps));
        if (ckpt || S->ctx->tune.ckpt == 0 || (S->ctx->tune.ckpt < 0 && b <= S->budget / 3)) break;
        ckpt = true;
    }
    b += (size_t)f64_grid_for(L, cap) * (size_t)f64_cta_bytes(L, cap);
    if (warps_out) *warps_out = warps;
    if (cap_out) *cap_out = cap;
    if (ckpt_out) *ckpt_out = ckpt;
    return b;
}

void free_scratch(qp_server* S) {
    for (void** p : {&S->bst, &S->bex, &S->bnd, &S->bck, &S->stg, &S->d_b, &S->d_diag, &S->d_cnt, &S->d_stg,
                     &S->d_stg64}) {
        if (*p) cudaFreeAsync(*p, S->cs);
        *p = nullptr;
    }
    S->scratch_len = 0;
    S->scratch_bytes = 0;
}

// (Re)size the scratch for sequences up to L; stream-ordered on cs, so launches
// already queued keep the old buffers until they finish.
int set_scratch(qp_server* S, int L) {
    if (L == S->scratch_len) return QP_OK;
    free_scratch(S);
    int64_t warps = 0;
    int cap = 0;
    bool ckpt = false;
    const size_t bytes = scratch_bytes_for(S, L, &warps, S->bps, &cap, &ckpt);
    // room for one warp per pair and for two (every buffer per warp)
    const qpk::F32Scratch s1(L, cap, ckpt, 1), s2(L, cap, ckpt, 2);
    const int64_t L1 = L + 1;
    const size_t f64g = (size_t)f64_grid_for(L, cap);
    struct A { void** p; size_t b; } al[] = {
        {&S->bst, sizeof(float2) * (size_t)std::max(s1.bst, s2.bst) * (size_t)warps},
        {&S->bex, sizeof(int2) * (size_t)std::max(s1.bex, s2.bex) * (size_t)warps},
        {&S->bnd, sizeof(float4) * (size_t)std::max(s1.bnd, s2.bnd) * (size_t)warps},
        {&S->bck, sizeof(float4) * (size_t)std::max(s1.bck, s2.bck) * (size_t)warps},
        {&S->stg, sizeof(int2) * (size_t)s1.stg * warps},
        {&S->d_b, sizeof(double2) * (size_t)(L1 * L1) * f64g},
        {&S->d_diag, sizeof(double) * (size_t)(3 * qpk::kNS * L1) * f64g},
        {&S->d_cnt, sizeof(int32_t) * (size_t)(5 * L1 + 8) * f64g},
        {&S->d_stg, sizeof(int2) * (size_t)L * cap * f64g},
        {&S->d_stg64, sizeof(double) * (size_t)L * cap * f64g},
    };
    for (auto& a : al) {
        cudaError_t e = cudaMallocAsync(a.p, std::max<size_t>(a.b, 256), S->cs);
        if (e != cudaSuccess) {
            *a.p = nullptr;
            cudaGetLastError();
            free_scratch(S);
            return fail(QP_ENOMEM, "server scratch for length %d (%zu bytes) failed", L, bytes);
        }
    }
    S->scratch_len = L;
    S->scratch_warps = warps;
    S->f64_grid = (int)f64g;
    S->cap = cap;
    S->ckpt = ckpt;
    S->scratch_bytes = bytes;
    return QP_OK;
}

qpk::Problem base_problem(qp_server* S, const Rec& R, int n_items, int wpp = 1, int64_t n_big = 0) {
    qpk::Problem Pb;
    memset(&Pb, 0, sizeof Pb);
    Pb.cf = S->cf;
    Pb.cf.spin_limit = S->ctx->tune.spin_limit;   // testing knob of the two-warp form (0: default)
    Pb.cst = S->d_cst;
    Pb.fams = S->d_fams;
    Pb.items = R.d_items;
    Pb.n_work = n_items;
    Pb.cap = S->cap;
    Pb.pool = nullptr;          // every family brings its own pool
    Pb.pool64 = nullptr;
    Pb.status = R.d_status;
    Pb.fallback = R.d_fallback;
    const int L = S->scratch_len;
    const int64_t L1 = L + 1;
    const qpk::F32Scratch sz(L, S->cap, S->ckpt, wpp);
    Pb.bst = (float2*)S->bst; Pb.bst_stride = sz.bst;
    Pb.bex = (int2*)S->bex;   Pb.bex_stride = sz.bex;
    Pb.bnd = (float4*)S->bnd; Pb.bnd_stride = sz.bnd;
    Pb.bck = (float4*)S->bck; Pb.bck_stride = sz.bck;
    Pb.ckpt = S->ckpt ? 1 : 0;
    Pb.wpp = wpp;
    Pb.n_big = (int32_t)n_big;
    Pb.stg = (int2*)S->stg;   Pb.stg_stride = sz.stg;
    Pb.d_b = (double2*)S->d_b; Pb.d_b_stride = L1 * L1;
    Pb.d_diag = (double*)S->d_diag; Pb.d_diag_stride = 3 * qpk::kNS * L1;
    Pb.f64_smem_diag = qpk::posterior_f64_smem_diag(L) ? 1 : 0;
    Pb.d_cnt = (int32_t*)S->d_cnt; Pb.d_cnt_stride = 5 * L1 + 8;
    Pb.d_stg = (int2*)S->d_stg; Pb.d_stg64 = (double*)S->d_stg64;
    Pb.d_stg_stride = (int64_t)L * S->cap;
    Pb.f64_all = 0;
    Pb.max_len = L;
    return Pb;
}

// Moves a job to a final state (caller holds mu).
void finish_job(qp_server* S, Job& J, int state, int rc, const std::string& err, qp_result* r) {
    J.state = state;
    J.rc = rc;
    J.err = err;
    J.t_done = now_s();
    if (state == kDone && J.cancel) {          // cancelled while it was being finished
        if (r) qp_result_free(r);
        r = nullptr;
        J.state = kCancelled;
    }
    J.result = r;
    if (J.state == kDone) S->stats.completed++;
    else if (J.state == kCancelled) S->stats.cancelled++;
    else S->stats.failed++;
    S->cv_done.notify_all();
}

// Frees an admitted family that will not produce a result (worker).
void drop_family(qp_server* S, std::unique_ptr<Fam>& F, int state, int rc, const std::string& err) {
    if (F->blk) cudaFreeAsync(F->blk, S->cs);
    if (F->pool) cudaFreeAsync(F->pool, S->cs);
    if (F->own) {
        if (F->own->dev_a) cudaFreeAsync(F->own->dev_a, S->cs);
        if (F->own->dev_b) cudaFreeAsync(F->own->dev_b, S->cs);
        delete F->own;
    }
    if (F->ev_done) cudaEventDestroy(F->ev_done);
    cudaStreamSynchronize(S->cs);
    std::lock_guard<std::mutex> g(S->mu);
    S->reserved -= F->job->reserve;
    S->stats.resident--;
    finish_job(S, *F->job, state, rc, err, nullptr);
    S->cv_work.notify_all();
    F.reset();
}

void fail_all(qp_server* S, int rc, const std::string& err) {
    std::lock_guard<std::mutex> g(S->mu);
    if (S->fatal_rc == QP_OK) { S->fatal_rc = rc; S->fatal_err = err; }
}

// Items of a launch that will not complete normally (its launch or a read of
// its status failed): the families stop waiting for them.
void release_items(qp_server* S, const std::vector<std::pair<int, int64_t>>& per_fam) {
    for (auto& pf : per_fam)
        if (S->fams[pf.first]) S->fams[pf.first]->outstanding -= pf.second;
}

// ------------------------------------------------------------------ admission
int admit_one(qp_server* S, const std::shared_ptr<Job>& J, int slot) {
    const Plan& pl = *J->plan;
    const int k = pl.k;
    const int64_t P = pl.n_pairs;
    const int64_t total = J->offsets[k];
    std::unique_ptr<Fam> F(new Fam());
    F->job = J;
    F->slot = slot;
    F->pool_cap = J->pool_cap;
    F->lay = ResultLayout(P, pl.n_rows, k);
    F->own = new ResultOwner();
    F->own->device = S->device;
    const BlkLayout B(k, total, P, pl.n_rows, pl.n_strips);
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stats.resident++;
        S->stats.max_resident = std::max(S->stats.max_resident, S->stats.resident);
    }
    S->fams[slot] = std::move(F);
    Fam* Fp = S->fams[slot].get();
    cudaError_t e;
    auto oom = [&](const char* what) {
        cudaGetLastError();
        std::string msg = std::string("server: device allocation of ") + what + " failed";
        cudaStreamSynchronize(S->up);
        drop_family(S, S->fams[slot], kFailed, QP_ENOMEM, msg);
        return QP_ENOMEM;
    };
    if ((e = cudaMallocAsync((void**)&Fp->blk, B.bytes, S->up)) != cudaSuccess) { Fp->blk = nullptr; return oom("the family block"); }
    if ((e = cudaMallocAsync((void**)&Fp->pool, sizeof(int2) * Fp->pool_cap, S->up)) != cudaSuccess) { Fp->pool = nullptr; return oom("the entry pool"); }
    if ((e = cudaMallocAsync(&Fp->own->dev_a, Fp->lay.bytes, S->up)) != cudaSuccess) { Fp->own->dev_a = nullptr; return oom("the result"); }
    if ((e = cudaEventCreateWithFlags(&Fp->ev_done, cudaEventDisableTiming)) != cudaSuccess) { Fp->ev_done = nullptr; return oom("an event"); }
    char* blk = Fp->blk;
    char* A = (char*)Fp->own->dev_a;
    qpk::FamDesc& fd = Fp->fd;
    memset(&fd, 0, sizeof fd);
    fd.codes = (const uint8_t*)(blk + B.o_codes);
    fd.seq_off = (const int64_t*)(blk + B.o_off);
    fd.seq_logq = (const double*)(blk + B.o_logq);
    fd.pairs = (const int2*)(blk + B.o_pairs);
    fd.pair_row_off = (const int64_t*)(A + Fp->lay.o_pro);
    fd.pair_strip_off = (const int64_t*)(blk + B.o_strip);
    fd.k = k;
    fd.row_cnt = (int32_t*)(blk + B.o_rowcnt);
    fd.chunk_off = (int64_t*)(blk + B.o_chunk);
    fd.pair_nnz = (int64_t*)(blk + B.o_pnnz);
    fd.mea = (double*)(A + Fp->lay.o_mea);
    fd.logz_h = (double*)(A + Fp->lay.o_lh);
    fd.logz_p = (double*)(A + Fp->lay.o_lp);
    fd.dist = (float*)(A + Fp->lay.o_dist);
    fd.dist64 = (double*)(A + Fp->lay.o_d64);
    fd.pair_flags = (int32_t*)(A + Fp->lay.o_fl);
    fd.pool = Fp->pool;
    fd.pool64 = nullptr;
    fd.pool_used = (unsigned long long*)(blk + B.o_used);
    fd.pool_base = 0;
    fd.pool_cap = Fp->pool_cap;
    fd.n_done = nullptr;
    // inputs and plan arrays (pageable sources are staged by the copy call)
    const cudaStream_t up = S->up;
    if ((e = cudaMemcpyAsync(blk + B.o_ascii, J->residues.data(), total, cudaMemcpyHostToDevice, up)) != cudaSuccess ||
        (e = cudaMemcpyAsync(blk + B.o_off, J->offsets.data(), sizeof(int64_t) * (k + 1), cudaMemcpyHostToDevice, up)) != cudaSuccess ||
        (e = cudaMemcpyAsync(blk + B.o_pairs, pl.pairs.data(), sizeof(int2) * P, cudaMemcpyHostToDevice, up)) != cudaSuccess ||
        (e = cudaMemcpyAsync(blk + B.o_strip, pl.strip_off.data(), sizeof(int64_t) * (P + 1), cudaMemcpyHostToDevice, up)) != cudaSuccess ||
        (e = cudaMemcpyAsync(A + Fp->lay.o_pro, pl.row_off.data(), sizeof(int64_t) * (P + 1), cudaMemcpyHostToDevice, up)) != cudaSuccess ||
        (e = cudaMemsetAsync(blk + B.o_used, 0, sizeof(unsigned long long), up)) != cudaSuccess ||
        (e = cudaMemsetAsync(A + Fp->lay.o_dist, 0, sizeof(float) * (size_t)k * k, up)) != cudaSuccess ||
        (e = cudaMemsetAsync(A + Fp->lay.o_d64, 0, sizeof(double) * (size_t)k * k, up)) != cudaSuccess ||
        (e = cudaMemsetAsync(A + Fp->lay.o_fl, 0, sizeof(int32_t) * P, up)) != cudaSuccess ||
        (e = cudaMemcpyAsync(S->d_fams + slot, &fd, sizeof fd, cudaMemcpyHostToDevice, up)) != cudaSuccess ||
        (e = cudaStreamSynchronize(up)) != cudaSuccess) {
        const int rc = cuda_fail(e, "server: family upload");
        fail_all(S, rc, last_error());
        Fp->failed = true;               // dropped by the worker's stop path
        return rc;
    }
    if ((e = qpk::launch_encode((const uint8_t*)(blk + B.o_ascii), (uint8_t*)(blk + B.o_codes), total,
                                (const int64_t*)(blk + B.o_off), k, (double*)(blk + B.o_logq), S->d_cst,
                                S->d_enc_status, S->cs)) != cudaSuccess) {
        const int rc = cuda_fail(e, "k_encode");
        fail_all(S, rc, last_error());
        Fp->failed = true;
        return rc;
    }
    Fp->remaining = pl.work_sum;
    J->residues.clear();
    J->residues.shrink_to_fit();
    return QP_OK;
}

// Admission: families are taken in arrival order; one that does not fit the
// budget is passed over by later ones that do (backfill) until it has waited
// longer than the aging bound, after which nothing passes it.
void admit(qp_server* S) {
    for (;;) {
        int slot = -1;
        for (int s = 0; s < kSlots; ++s)
            if (!S->fams[s]) { slot = s; break; }
        if (slot < 0) return;
        int L = 0;
        bool any_resident = false;
        for (int s = 0; s < kSlots; ++s)
            if (S->fams[s]) { any_resident = true; L = std::max(L, S->fams[s]->job->plan->max_len); }
        std::shared_ptr<Job> J;
        int Ls = 0;
        {
            std::lock_guard<std::mutex> g(S->mu);
            const double t = now_s();
            for (auto it = S->queue.begin(); it != S->queue.end();) {
                if ((*it)->state != kQueued) { it = S->queue.erase(it); continue; }
                const Job& C = **it;
                // scratch is grow-only while families are resident; with none
                // resident it is kept when it covers the newcomer and fits,
                // else resized to the newcomer
                int ls;
                if (any_resident) {
                    ls = std::max(std::max(L, C.plan->max_len), S->scratch_len);
                } else {
                    ls = C.plan->max_len;
                    if (S->scratch_len >= ls && S->reserved + C.reserve + S->scratch_bytes <= S->budget)
                        ls = S->scratch_len;
                }
                const size_t scratch = ls == S->scratch_len ? S->scratch_bytes
                                                            : scratch_bytes_for(S, ls, nullptr, nullptr, nullptr, nullptr);
                if (S->reserved + C.reserve + scratch <= S->budget) {
                    J = *it;
                    Ls = ls;
                    S->queue.erase(it);
                    break;
                }
                if (t - C.t_submit > S->aging_s) break;     // hold the memory for this one
                ++it;
            }
            if (!J) return;                                 // wait for memory
            S->reserved += J->reserve;
            J->state = kRunning;
            J->t_admit = now_s();
        }
        int rc = set_scratch(S, Ls);
        if (rc != QP_OK) {
            std::lock_guard<std::mutex> g(S->mu);
            S->reserved -= J->reserve;
            finish_job(S, *J, kFailed, rc, last_error(), nullptr);
            continue;
        }
        admit_one(S, J, slot);
        if (S->fatal_rc != QP_OK) return;
    }
}

// ------------------------------------------------------------------ launches
bool issue(qp_server* S) {
    int ri = -1;
    int inflight = 0;
    for (int i = 0; i < kRecs; ++i) {
        if (S->recs[i].phase == 1) ++inflight;
        if (S->recs[i].phase == 0 && ri < 0) ri = i;
    }
    if (inflight >= kInflight || ri < 0) return false;
    // families with pairs to launch.  Those admitted longer ago than the
    // aging bound get up to half of the launch, oldest first; the rest of the
    // launch goes to the family with the least remaining work first.
    const double t = now_s();
    std::vector<Fam*> cand, aged;
    for (int s = 0; s < kSlots; ++s) {
        Fam* F = S->fams[s].get();
        if (F && !F->failed && !F->job->cancel && F->next < F->job->plan->n_pairs) {
            cand.push_back(F);
            if (t - F->job->t_admit > S->aging_s) aged.push_back(F);
        }
    }
    if (cand.empty()) return false;
    std::stable_sort(aged.begin(), aged.end(),
                     [](const Fam* a, const Fam* b) { return a->job->t_admit < b->job->t_admit; });
    std::stable_sort(cand.begin(), cand.end(), [](const Fam* a, const Fam* b) { return a->remaining < b->remaining; });
    Rec& R = S->recs[ri];
    R.items.clear();
    R.per_fam.clear();
    R.per_fam_f64.clear();
    R.work = 0;
    R.cells = 0;
    const double budget = std::max(1.0, S->target_ms * S->rate);
    std::vector<std::pair<int64_t, int2>> take;
    std::map<int, int64_t> per;
    auto fill = [&](const std::vector<Fam*>& order, double limit) {
        for (Fam* F : order) {
            if (R.work >= limit || (int64_t)take.size() >= kMaxItems) break;
            const Plan& pl = *F->job->plan;
            int64_t n = 0;
            while (F->next < pl.n_pairs && (R.work < limit || take.empty()) && (int64_t)take.size() < kMaxItems) {
                const int32_t q = pl.order[F->next++];
                const int64_t w = pl.work[q];
                take.push_back(std::make_pair(w, make_int2(F->slot, q)));
                R.work += (double)w;
                F->remaining -= (double)w;
                const int2 ab = pl.pairs[q];
                R.cells += (double)pl.lens[ab.x] * (double)pl.lens[ab.y];
                ++n;
            }
            if (n) {
                per[F->slot] += n;
                F->outstanding += n;
            }
        }
    };
    fill(aged, 0.5 * budget);
    fill(cand, budget);
    R.per_fam.assign(per.begin(), per.end());
    // one longest-first order over the whole launch
    std::stable_sort(take.begin(), take.end(),
                     [](const std::pair<int64_t, int2>& a, const std::pair<int64_t, int2>& b) { return a.first > b.first; });
    R.items.resize(take.size());
    for (size_t i = 0; i < take.size(); ++i) R.items[i] = take[i].second;
    const int n_items = (int)R.items.size();
    cudaError_t e;
    if ((e = cudaMemcpyAsync(R.d_items, R.items.data(), sizeof(int2) * n_items, cudaMemcpyHostToDevice, S->up)) != cudaSuccess ||
        (e = cudaMemsetAsync(R.d_status, 0, sizeof(qpk::Status), S->up)) != cudaSuccess ||
        (e = cudaStreamSynchronize(S->up)) != cudaSuccess) {
        fail_all(S, cuda_fail(e, "server: launch upload"), last_error());
        release_items(S, R.per_fam);
        return false;
    }
    R.tkey = Context::tune_key(n_items, S->scratch_len, R.work) ^ ((int64_t)S->ckpt << 62);
    const int max_strips = (S->scratch_len + 1 + qpk::kStripRows - 1) / qpk::kStripRows;
    const unsigned allowed = allowed_configs(n_items, max_strips, S->scratch_warps, kWpb, S->ctx->tune);
    R.cfg = S->tuner[R.tkey].choose(allowed);
    R.variant = config_variant(R.cfg);
    const int W = config_wpp(R.cfg);
    int bps = 0;
    qpk::posterior_f32_occupancy(kWpb, S->scratch_len, &bps, R.variant, S->ckpt, W);
    bps = std::max(1, std::min(bps, S->bps[R.variant]));
    // two warps per pair: the spare warps double up on the longest items
    // (items come longest first), the rest run on one warp each
    const int64_t full_w = std::min<int64_t>((int64_t)S->ctx->sm_count * bps * kWpb, S->scratch_warps);
    const int64_t n_big = W > 1 ? std::max<int64_t>(0, std::min<int64_t>(n_items, full_w - n_items)) : 0;
    int64_t grid = balanced_grid(S->ctx->sm_count, bps, ((int64_t)n_items + n_big + kWpb - 1) / kWpb);
    grid = std::min<int64_t>(grid, S->scratch_warps / kWpb);
    const qpk::Problem Pb = base_problem(S, R, n_items, W, n_big);
    cudaEventRecord(R.ev0, S->cs);
    if ((e = qpk::launch_posterior_f32(Pb, (int)grid, kWpb, S->cs, R.variant)) != cudaSuccess) {
        fail_all(S, cuda_fail(e, "k_posterior_f32 launch"), last_error());
        release_items(S, R.per_fam);
        return false;
    }
    cudaEventRecord(R.ev1, S->cs);
    R.phase = 1;
    S->issued.push_back(ri);
    std::lock_guard<std::mutex> g(S->mu);
    S->stats.launches_f32++;
    S->stats.max_families_per_launch = std::max<int32_t>(S->stats.max_families_per_launch, (int32_t)R.per_fam.size());
    return true;
}

void retire(qp_server* S, int ri) {
    Rec& R = S->recs[ri];
    float ms = 0.f;
    cudaEventElapsedTime(&ms, R.ev0, R.ev1);
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stats.kernel_ms += ms;
    }
    if (R.phase == 2) {
        for (auto& pf : R.per_fam_f64)
            if (S->fams[pf.first]) S->fams[pf.first]->outstanding -= pf.second;
        std::lock_guard<std::mutex> g(S->mu);
        S->stats.launches_f64++;
        R.phase = 0;
        return;
    }
    // FP32 launch
    if (ms > 1.0f) S->rate = 0.7 * S->rate + 0.3 * (R.work / ms);
    if (S->ctx->tune.variant < 0) {
        TuneEntry& te = S->tuner[R.tkey];
        te.record(R.cfg, ms);
    }
    qpk::Status hs;
    cudaError_t e = cudaMemcpyAsync(S->h_status.ptr, R.d_status, sizeof hs, cudaMemcpyDeviceToHost, S->up);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->up);
    if (e != cudaSuccess) {
        fail_all(S, cuda_fail(e, "server: status read"), last_error());
        release_items(S, R.per_fam);
        R.phase = 0;
        return;
    }
    memcpy(&hs, S->h_status.ptr, sizeof hs);
    std::map<int, int64_t> fb;
    if (hs.n_fallback > 0) {
        const int nf = hs.n_fallback;
        e = S->h_fb.ensure(sizeof(int2) * nf);
        if (e == cudaSuccess) e = cudaMemcpyAsync(S->h_fb.ptr, R.d_fallback, sizeof(int2) * nf, cudaMemcpyDeviceToHost, S->up);
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->up);
        if (e != cudaSuccess) {
            fail_all(S, cuda_fail(e, "server: fallback read"), last_error());
            release_items(S, R.per_fam);
            R.phase = 0;
            return;
        }
        const int2* it = (const int2*)S->h_fb.ptr;
        for (int i = 0; i < nf; ++i) fb[it[i].x]++;
    }
    for (auto& pf : R.per_fam) {
        Fam* F = S->fams[pf.first].get();
        if (!F) continue;
        const int64_t nfb = fb.count(pf.first) ? fb[pf.first] : 0;
        F->outstanding -= pf.second - nfb;
        F->n_fallback += nfb;
        if (nfb && !F->have_guard) {
            for (int i = 0; i < 10; ++i) F->guard[i] = hs.diag[i];
            F->have_guard = true;
        }
        if (hs.stage_overflow && !F->failed) {
            F->failed = true;
            F->rc = QP_ECUDA;
            F->err = "internal: a row exceeded its entry capacity";
        }
    }
    if (hs.n_fallback > 0) {
        R.per_fam_f64.assign(fb.begin(), fb.end());
        const qpk::Problem Pb = base_problem(S, R, (int)R.items.size());
        cudaEventRecord(R.ev0, S->cs);
        e = qpk::launch_posterior_f64(Pb, std::min(hs.n_fallback, S->f64_grid), S->cs);
        if (e != cudaSuccess) {
            fail_all(S, cuda_fail(e, "k_posterior_f64 launch"), last_error());
            release_items(S, R.per_fam_f64);
            R.phase = 0;
            return;
        }
        cudaEventRecord(R.ev1, S->cs);
        R.phase = 2;
        S->issued.push_back(ri);
        return;
    }
    R.phase = 0;
}

// All pairs of F are done: rerun on a full pool, else assemble and hand over.
void finalize(qp_server* S, int slot) {
    std::unique_ptr<Fam>& F = S->fams[slot];
    const Plan& pl = *F->job->plan;
    const int64_t P = pl.n_pairs;
    cudaError_t e = cudaMemcpyAsync(S->h_used.ptr, F->fd.pool_used, sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, S->up);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->up);
    if (e != cudaSuccess) { fail_all(S, cuda_fail(e, "server: pool counter read"), last_error()); return; }
    unsigned long long used = 0;
    memcpy(&used, S->h_used.ptr, sizeof used);
    if ((int64_t)used > F->pool_cap) {
        if (++F->attempts >= 3) {
            drop_family(S, F, kFailed, QP_ENOMEM, "the entry pool kept overflowing");
            return;
        }
        const int64_t cap = (int64_t)(used * 5 / 4) + 4096;
        const size_t extra = (sizeof(int2) + sizeof(int32_t) + sizeof(float)) * (size_t)(cap - F->pool_cap);
        cudaFreeAsync(F->pool, S->cs);
        F->pool = nullptr;
        if ((e = cudaMallocAsync((void**)&F->pool, sizeof(int2) * cap, S->cs)) != cudaSuccess) {
            F->pool = nullptr;
            cudaGetLastError();
            drop_family(S, F, kFailed, QP_ENOMEM, "server: entry pool growth failed");
            return;
        }
        {
            std::lock_guard<std::mutex> g(S->mu);
            S->reserved += extra;
            F->job->reserve += extra;
        }
        F->pool_cap = cap;
        F->fd.pool = F->pool;
        F->fd.pool_cap = cap;
        cudaMemsetAsync(F->fd.pool_used, 0, sizeof(unsigned long long), S->cs);
        cudaMemsetAsync(F->fd.pair_flags, 0, sizeof(int32_t) * P, S->cs);
        cudaMemcpyAsync(S->d_fams + slot, &F->fd, sizeof F->fd, cudaMemcpyHostToDevice, S->cs);
        F->next = 0;
        F->remaining = pl.work_sum;
        F->n_fallback = 0;
        return;
    }
    // CSR assembly on the device
    ResultOwner* own = F->own;
    const size_t szb = ResultLayout::entry_bytes((int64_t)used, false);
    if ((e = cudaMallocAsync(&own->dev_b, std::max<size_t>(szb, 256), S->cs)) != cudaSuccess) {
        own->dev_b = nullptr;
        cudaGetLastError();
        drop_family(S, F, kFailed, QP_ENOMEM, "server: result allocation failed");
        return;
    }
    qp_result* r = (qp_result*)calloc(1, sizeof(qp_result));
    if (!r) { drop_family(S, F, kFailed, QP_ENOMEM, "host allocation failed"); return; }
    fill_result(r, own, F->lay, pl.k, P, pl.n_rows, (int64_t)used, false, QP_F32_SCALED, S->device);
    const qpk::FamDesc& fd = F->fd;
    if ((e = qpk::launch_scan_nnz(fd.pair_nnz, P, r->pair_nnz_off, S->cs)) != cudaSuccess ||
        (e = qpk::launch_compact(fd.pairs, fd.seq_off, fd.pair_row_off, fd.pair_strip_off, fd.row_cnt,
                                 fd.chunk_off, F->pool, nullptr, P, r->pair_nnz_off, r->row_ptr, r->col,
                                 r->val, nullptr, S->cs)) != cudaSuccess ||
        (e = cudaEventRecord(F->ev_done, S->cs)) != cudaSuccess) {
        free(r);
        fail_all(S, cuda_fail(e, "server: CSR assembly"), last_error());
        return;
    }
    r->n_fallback = F->n_fallback;
    for (int i = 0; i < 12; ++i) r->guard_info[i] = F->guard[i];
    F->result = r;
    F->own = nullptr;                    // now owned by the result
    F->job->t_work_done = now_s();
    std::lock_guard<std::mutex> g(S->mu);
    S->fin_queue.push_back(std::move(F));
    S->cv_fin.notify_all();
}

void worker_main(qp_server* S) {
    cudaSetDevice(S->device);
    for (;;) {
        bool progressed = false;
        while (!S->issued.empty()) {
            const int ri = S->issued.front();
            const cudaError_t q = cudaEventQuery(S->recs[ri].ev1);
            if (q == cudaErrorNotReady) break;
            S->issued.pop_front();
            if (q != cudaSuccess) {
                fail_all(S, cuda_fail(q, "server: posterior launch"), last_error());
                Rec& R = S->recs[ri];
                release_items(S, R.phase == 2 ? R.per_fam_f64 : R.per_fam);
                R.phase = 0;
                continue;
            }
            retire(S, ri);
            progressed = true;
        }
        bool stopping;
        {
            std::lock_guard<std::mutex> g(S->mu);
            stopping = S->stop || S->fatal_rc != QP_OK;
        }
        // families that are done, failed or cancelled
        for (int s = 0; s < kSlots; ++s) {
            std::unique_ptr<Fam>& F = S->fams[s];
            if (!F || F->outstanding > 0) continue;
            bool cancel;
            {
                std::lock_guard<std::mutex> g(S->mu);
                cancel = F->job->cancel;
            }
            if (stopping) {
                if (!S->issued.empty()) continue;      // let queued launches drain first
                const int rc = S->fatal_rc != QP_OK ? S->fatal_rc : QP_ECANCELLED;
                const std::string err = S->fatal_rc != QP_OK ? S->fatal_err : "the server shut down";
                drop_family(S, F, rc == QP_ECANCELLED ? kCancelled : kFailed, rc, err);
            } else if (cancel) {
                drop_family(S, F, kCancelled, QP_ECANCELLED, "cancelled");
            } else if (F->failed) {
                drop_family(S, F, kFailed, F->rc, F->err);
            } else if (F->next >= F->job->plan->n_pairs) {
                finalize(S, s);
            } else {
                continue;
            }
            progressed = true;
        }
        if (stopping) {
            bool any = !S->issued.empty();
            for (int s = 0; s < kSlots; ++s) any = any || (bool)S->fams[s];
            if (!any) {
                std::lock_guard<std::mutex> g(S->mu);
                const int rc = S->fatal_rc != QP_OK ? S->fatal_rc : QP_ECANCELLED;
                const std::string err = S->fatal_rc != QP_OK ? S->fatal_err : "the server shut down";
                for (auto& J : S->queue)
                    if (J->state == kQueued) finish_job(S, *J, rc == QP_ECANCELLED ? kCancelled : kFailed, rc, err, nullptr);
                S->queue.clear();
                if (S->stop) break;
            }
        } else {
            admit(S);
            while (issue(S)) progressed = true;
        }
        std::unique_lock<std::mutex> g(S->mu);
        if (S->stop && !stopping) continue;
        if (progressed) continue;
        if (!S->issued.empty())
            S->cv_work.wait_for(g, std::chrono::microseconds(200));
        else
            S->cv_work.wait_for(g, std::chrono::milliseconds(50));
    }
    cudaStreamSynchronize(S->cs);
    free_scratch(S);
    cudaStreamSynchronize(S->cs);
    std::lock_guard<std::mutex> g(S->mu);
    S->worker_done = true;
    S->cv_fin.notify_all();
}

void finisher_main(qp_server* S) {
    cudaSetDevice(S->device);
    for (;;) {
        std::unique_ptr<Fam> F;
        {
            std::unique_lock<std::mutex> g(S->mu);
            S->cv_fin.wait(g, [&] { return !S->fin_queue.empty() || S->worker_done; });
            if (S->fin_queue.empty()) return;
            F = std::move(S->fin_queue.front());
            S->fin_queue.pop_front();
        }
        qp_result* r = F->result;
        const int64_t P = r->n_pairs;
        int rc = QP_OK;
        std::string err;
        cudaError_t e = cudaStreamWaitEvent(S->down, F->ev_done, 0);
        int64_t nnz = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&nnz, r->pair_nnz_off + P, sizeof nnz, cudaMemcpyDeviceToHost, S->down);
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->down);
        if (e != cudaSuccess) { rc = cuda_fail(e, "server: result read"); err = last_error(); }
        r->nnz = nnz;
        if (rc == QP_OK && !S->out_on_device) {
            rc = to_host(r, S->down);
            if (rc != QP_OK) err = last_error();
        }
        cudaFreeAsync(F->blk, S->down);
        cudaFreeAsync(F->pool, S->down);
        cudaStreamSynchronize(S->down);
        cudaEventDestroy(F->ev_done);
        std::lock_guard<std::mutex> g(S->mu);
        Job& J = *F->job;
        const double t = now_s();
        r->kernel_ms[0] = 1e3 * (J.t_admit - J.t_submit);
        r->kernel_ms[1] = 1e3 * (J.t_work_done - J.t_admit);
        r->kernel_ms[2] = 1e3 * (t - J.t_work_done);
        r->kernel_ms[3] = 1e3 * (t - J.t_submit);
        S->reserved -= J.reserve;
        S->stats.resident--;
        if (rc == QP_OK) {
            S->stats.pairs_done += P;
            S->stats.cells_done += J.cells;
            finish_job(S, J, kDone, QP_OK, "", r);
        } else {
            qp_result_free(r);
            finish_job(S, J, kFailed, rc, err, nullptr);
        }
        S->cv_work.notify_all();
    }
}

}  // namespace

extern "C" {

int qp_server_create(const qp_params* params, size_t mem_budget, int32_t out_on_device, qp_server** out) {
    if (!out) return fail(QP_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate_params(params);
    if (rc == QP_OK && params->entry_budget != 0)
        rc = fail(QP_EINVAL, "entry_budget is not supported by a server (its memory budget admits families)");
    if (rc != QP_OK) return rc;
    if (params->precision != QP_F32_SCALED) return fail(QP_EINVAL, "the server runs the FP32 form only");
    if (mem_budget == 0) return fail(QP_EINVAL, "mem_budget must be > 0");
    cudaError_t e = cudaSetDevice(params->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    Context* C = get_context(params->device, &rc);
    if (!C) return rc;
    std::unique_ptr<qp_server> S(new qp_server());
    memset(&S->stats, 0, sizeof S->stats);
    S->params = *params;
    S->params.stream = nullptr;
    make_coef(params, &S->cf);
    S->budget = mem_budget;
    S->device = params->device;
    S->out_on_device = out_on_device ? 1 : 0;
    S->ctx = C;
    if (const char* v = getenv("QP_SERVER_LAUNCH_MS")) S->target_ms = std::max(0.1, atof(v));
    if (const char* v = getenv("QP_SERVER_AGING_MS")) S->aging_s = std::max(0.0, atof(v)) * 1e-3;
    // the server's own memory pool keeps freed blocks for reuse
    cudaMemPool_t mp;
    if (cudaDeviceGetDefaultMemPool(&mp, S->device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    if ((e = cudaStreamCreateWithFlags(&S->cs, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&S->up, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&S->down, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreate");
    const size_t rec_bytes = align256(sizeof(int2) * kMaxItems) * 2 + align256(sizeof(qpk::Status));
    if ((e = cudaMalloc((void**)&S->d_cst, sizeof(qpk::Consts))) != cudaSuccess ||
        (e = cudaMalloc((void**)&S->d_raw, sizeof(qpk::RawParams))) != cudaSuccess ||
        (e = cudaMalloc((void**)&S->d_fams, sizeof(qpk::FamDesc) * kSlots)) != cudaSuccess ||
        (e = cudaMalloc((void**)&S->d_enc_status, sizeof(qpk::Status))) != cudaSuccess ||
        (e = cudaMalloc(&S->d_rec_mem, rec_bytes * kRecs)) != cudaSuccess) {
        cudaGetLastError();
        return fail(QP_ENOMEM, "server allocation failed");
    }
    if ((e = S->h_status.ensure(sizeof(qpk::Status))) != cudaSuccess ||
        (e = S->h_used.ensure(sizeof(unsigned long long))) != cudaSuccess ||
        (e = S->h_fb.ensure(4096)) != cudaSuccess)
        return fail(QP_ENOMEM, "server host allocation failed");
    for (int i = 0; i < kRecs; ++i) {
        char* m = (char*)S->d_rec_mem + rec_bytes * i;
        S->recs[i].d_items = (int2*)m;
        S->recs[i].d_fallback = (int2*)(m + align256(sizeof(int2) * kMaxItems));
        S->recs[i].d_status = (qpk::Status*)(m + 2 * align256(sizeof(int2) * kMaxItems));
        if ((e = cudaEventCreate(&S->recs[i].ev0)) != cudaSuccess || (e = cudaEventCreate(&S->recs[i].ev1)) != cudaSuccess)
            return cuda_fail(e, "cudaEventCreate");
    }
    qpk::RawParams raw;
    make_raw(params, &raw);
    if ((e = cudaMemsetAsync(S->d_enc_status, 0, sizeof(qpk::Status), S->cs)) != cudaSuccess ||
        (e = qpk::launch_setup(&raw, S->d_raw, S->d_cst, S->cs)) != cudaSuccess ||
        (e = cudaStreamSynchronize(S->cs)) != cudaSuccess)
        return cuda_fail(e, "server set-up");
    qp_server* raw_s = S.release();
    raw_s->worker = std::thread(worker_main, raw_s);
    raw_s->finisher = std::thread(finisher_main, raw_s);
    *out = raw_s;
    return QP_OK;
}

int qp_server_submit(qp_server* S, const qp_family* family, uint64_t* ticket) {
    if (!S || !ticket) return fail(QP_EINVAL, "server or ticket is NULL");
    *ticket = 0;
    int rc = validate_family(family);
    if (rc != QP_OK) return rc;
    if (family->residues_on_device) return fail(QP_EINVAL, "the server takes host-resident families");
    {
        // the server's FP32 launches use blocks of kWpb warps
        const int lim = f32_max_len(S->ctx, kWpb);
        for (int a = 0; a < family->k; ++a) {
            const int64_t L = family->offsets[a + 1] - family->offsets[a];
            if (L > lim)
                return fail(QP_EINVAL, "sequence %d has %lld residues; the server takes at most %d on this device",
                            a, (long long)L, lim);
        }
    }
    const double t_submit = now_s();
    const int k = family->k;
    const int64_t total = family->offsets[k];
    for (int64_t i = 0; i < total; ++i)
        if (!valid_residue(family->residues[i], S->params.alphabet))
            return fail(QP_EINVAL, "%s", alphabet_error(S->params.alphabet));
    auto J = std::make_shared<Job>();
    J->residues.assign(family->residues, family->residues + total);
    J->offsets.assign(family->offsets, family->offsets + k + 1);
    J->plan = build_plan(k, family->offsets);
    const Plan& pl = *J->plan;
    for (int64_t q = 0; q < pl.n_pairs; ++q)
        J->cells += (double)pl.lens[pl.pairs[q].x] * (double)pl.lens[pl.pairs[q].y];
    // entry pool estimate (grown and rerun if a family needs more)
    const double per_row = std::min<double>(pl.max_len + 1.0, 4.0 + 0.04 / S->params.threshold);
    J->pool_cap = (int64_t)(per_row * (double)pl.n_rows) + 4096;
    J->blk_bytes = BlkLayout(k, total, pl.n_pairs, pl.n_rows, pl.n_strips).bytes;
    J->res_bytes = ResultLayout(pl.n_pairs, pl.n_rows, k).bytes;
    J->reserve = J->blk_bytes + J->res_bytes + sizeof(int2) * (size_t)J->pool_cap +
                 ResultLayout::entry_bytes(J->pool_cap, false);
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(S->device);
    const size_t scratch = scratch_bytes_for(S, pl.max_len, nullptr, nullptr, nullptr, nullptr);
    cudaSetDevice(cur);
    if (J->reserve + scratch > S->budget)
        return fail(QP_EINVAL, "the family needs %zu bytes (%zu resident + %zu kernel scratch), more than the budget %zu",
                    J->reserve + scratch, J->reserve, scratch, S->budget);
    std::lock_guard<std::mutex> g(S->mu);
    if (S->fatal_rc != QP_OK) return fail(S->fatal_rc, "%s", S->fatal_err.c_str());
    if (S->stop) return fail(QP_ECANCELLED, "the server is shutting down");
    J->ticket = S->next_ticket++;
    J->t_submit = t_submit;
    S->jobs[J->ticket] = J;
    S->queue.push_back(J);
    S->stats.submitted++;
    S->cv_work.notify_all();
    *ticket = J->ticket;
    return QP_OK;
}

int qp_server_poll(qp_server* S, uint64_t ticket, int32_t timeout_ms, qp_result** out) {
    if (!S || !out) return fail(QP_EINVAL, "server or out is NULL");
    *out = nullptr;
    std::unique_lock<std::mutex> g(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return fail(QP_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    auto J = it->second;
    auto done = [&] { return J->state >= kDone; };
    if (!done()) {
        if (timeout_ms == 0) return fail(QP_ENOTREADY, "ticket %llu is not finished", (unsigned long long)ticket);
        if (timeout_ms < 0) S->cv_done.wait(g, done);
        else if (!S->cv_done.wait_for(g, std::chrono::milliseconds(timeout_ms), done))
            return fail(QP_ETIMEOUT, "ticket %llu did not finish within %d ms", (unsigned long long)ticket, timeout_ms);
    }
    S->jobs.erase(it);
    if (J->state == kCancelled) return fail(QP_ECANCELLED, "ticket %llu was cancelled", (unsigned long long)ticket);
    if (J->state == kFailed) return fail(J->rc, "%s", J->err.c_str());
    *out = J->result;
    J->result = nullptr;
    return QP_OK;
}

int qp_server_cancel(qp_server* S, uint64_t ticket) {
    if (!S) return fail(QP_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return fail(QP_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    Job& J = *it->second;
    J.cancel = true;
    if (J.state == kQueued) finish_job(S, J, kCancelled, QP_ECANCELLED, "cancelled", nullptr);
    S->cv_work.notify_all();
    return QP_OK;
}

int qp_server_get_stats(qp_server* S, qp_server_stats* out) {
    if (!S || !out) return fail(QP_EINVAL, "server or out is NULL");
    std::lock_guard<std::mutex> g(S->mu);
    *out = S->stats;
    out->queued = 0;
    for (auto& J : S->queue) out->queued += J->state == kQueued;
    out->reserved_bytes = (int64_t)S->reserved;
    out->scratch_bytes = (int64_t)S->scratch_bytes;
    return QP_OK;
}

void qp_server_destroy(qp_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        for (auto& kv : S->jobs) kv.second->cancel = true;
        S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    if (S->finisher.joinable()) S->finisher.join();
    for (auto& kv : S->jobs)
        if (kv.second->result) qp_result_free(kv.second->result);
    cudaSetDevice(S->device);
    for (auto& R : S->recs) {
        if (R.ev0) cudaEventDestroy(R.ev0);
        if (R.ev1) cudaEventDestroy(R.ev1);
    }
    cudaFree(S->d_cst);
    cudaFree(S->d_raw);
    cudaFree(S->d_fams);
    cudaFree(S->d_enc_status);
    cudaFree(S->d_rec_mem);
    if (S->cs) cudaStreamDestroy(S->cs);
    if (S->up) cudaStreamDestroy(S->up);
    if (S->down) cudaStreamDestroy(S->down);
    // hand the blocks the pool kept for reuse back to the device
    cudaMemPool_t mp;
    if (cudaDeviceGetDefaultMemPool(&mp, S->device) == cudaSuccess) {
        cudaDeviceSynchronize();
        cudaMemPoolTrimTo(mp, 0);
    }
    cudaGetLastError();
    delete S;
}

}  // extern "C"
