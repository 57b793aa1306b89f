// Serving loop: families are submitted, admitted by device memory, processed,
// and polled.  (Sequential worker; see qp.h for the contract.)
#include "../../include/qp.h"
#include "qp_host.h"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <string>
#include <thread>
#include <vector>

using namespace qph;

struct QpJob {
    uint64_t ticket = 0;
    std::vector<uint8_t> residues;
    std::vector<int64_t> offsets;
    size_t reserve = 0;
    int state = 0;            // 0 queued, 1 running, 2 done, 3 failed, 4 cancelled
    int rc = QP_OK;
    std::string err;
    qp_result* result = nullptr;
    double t_submit = 0, t_done = 0;
};

struct qp_server {
    qp_params params;
    size_t budget = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<QpJob>> queue;
    std::map<uint64_t, std::shared_ptr<QpJob>> jobs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    Context* ctx = nullptr;
    cudaStream_t stream = nullptr;
};

static double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// worst-case device bytes a family needs while it is processed
static size_t family_reserve(const qp_family* f, const qp_params* p) {
    const int64_t k = f->k;
    int64_t maxL = 0, tot = f->offsets[k];
    for (int64_t a = 0; a < k; ++a) maxL = std::max<int64_t>(maxL, f->offsets[a + 1] - f->offsets[a]);
    const int64_t P = k * (k - 1) / 2;
    const int64_t rows = (k - 1) * tot;               // sum over pairs of (m+1), bounded
    const double per_row = std::min<double>(maxL + 1.0, 4.0 + 0.04 / p->threshold);
    size_t b = 0;
    b += (size_t)tot * 2 + sizeof(int64_t) * (k + 1) + sizeof(double) * k;
    b += sizeof(int32_t) * (size_t)rows * 2;          // row counts + row pointers
    b += sizeof(int64_t) * (size_t)P * 6;             // per-pair arrays
    b += (sizeof(float) + sizeof(double)) * (size_t)k * k;
    b += (size_t)(per_row * (double)rows) * (sizeof(int2) + sizeof(int32_t) + sizeof(float));
    return b;
}

static void worker_main(qp_server* S) {
    cudaSetDevice(S->device);
    for (;;) {
        std::shared_ptr<QpJob> job;
        {
            std::unique_lock<std::mutex> g(S->mu);
            S->cv.wait(g, [&] { return S->stop || !S->queue.empty(); });
            if (S->stop) return;
            job = S->queue.front();
            S->queue.pop_front();
            if (job->state == 4) continue;
            job->state = 1;
        }
        qp_family f;
        f.k = (int32_t)(job->offsets.size() - 1);
        f.residues_on_device = 0;
        f.residues = job->residues.data();
        f.offsets = job->offsets.data();
        qp_params p = S->params;
        p.stream = S->stream;
        qp_result* r = nullptr;
        int rc;
        {
            std::lock_guard<std::mutex> g(S->ctx->mu);
            rc = run_family(S->ctx, &f, &p, 0, &r);
        }
        std::string err = rc == QP_OK ? "" : last_error();
        {
            std::lock_guard<std::mutex> g(S->mu);
            job->rc = rc;
            job->err = err;
            job->result = r;
            job->t_done = now_s();
            if (job->state == 4) { if (r) qp_result_free(r); job->result = nullptr; }
            else job->state = rc == QP_OK ? 2 : 3;
        }
        S->cv.notify_all();
    }
}

extern "C" {

int qp_server_create(const qp_params* params, size_t mem_budget, qp_server** out) {
    if (!out) return fail(QP_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate_params(params);
    if (rc != QP_OK) return rc;
    if (params->precision != QP_F32_SCALED) return fail(QP_EINVAL, "the server runs the FP32 form only");
    if (mem_budget == 0) return fail(QP_EINVAL, "mem_budget must be > 0");
    cudaError_t e = cudaSetDevice(params->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    Context* C = get_context(params->device, &rc);
    if (!C) return rc;
    qp_server* S = new qp_server();
    S->params = *params;
    S->budget = mem_budget;
    S->device = params->device;
    S->ctx = C;
    e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete S; return cuda_fail(e, "cudaStreamCreate"); }
    S->worker = std::thread(worker_main, S);
    *out = S;
    return QP_OK;
}

int qp_server_submit(qp_server* S, const qp_family* family, uint64_t* ticket) {
    if (!S || !ticket) return fail(QP_EINVAL, "server or ticket is NULL");
    int rc = validate_family(family);
    if (rc != QP_OK) return rc;
    if (family->residues_on_device) return fail(QP_EINVAL, "the server takes host-resident families");
    const size_t need = family_reserve(family, &S->params);
    if (need > S->budget) return fail(QP_EINVAL, "family needs %zu bytes, more than the budget %zu", need, S->budget);
    auto job = std::make_shared<QpJob>();
    job->residues.assign(family->residues, family->residues + family->offsets[family->k]);
    job->offsets.assign(family->offsets, family->offsets + family->k + 1);
    job->reserve = need;
    job->t_submit = now_s();
    {
        std::lock_guard<std::mutex> g(S->mu);
        job->ticket = S->next_ticket++;
        S->jobs[job->ticket] = job;
        S->queue.push_back(job);
    }
    S->cv.notify_all();
    *ticket = job->ticket;
    return QP_OK;
}

int qp_server_poll(qp_server* S, uint64_t ticket, int32_t timeout_ms, qp_result** out) {
    if (!S || !out) return fail(QP_EINVAL, "server or out is NULL");
    *out = nullptr;
    std::unique_lock<std::mutex> g(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return fail(QP_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    auto job = it->second;
    auto done = [&] { return job->state >= 2; };
    if (!done()) {
        if (timeout_ms == 0) return fail(QP_ENOTREADY, "ticket %llu is not finished", (unsigned long long)ticket);
        if (timeout_ms < 0) S->cv.wait(g, done);
        else if (!S->cv.wait_for(g, std::chrono::milliseconds(timeout_ms), done))
            return fail(QP_ETIMEOUT, "ticket %llu did not finish within %d ms", (unsigned long long)ticket, timeout_ms);
    }
    S->jobs.erase(it);
    if (job->state == 4) return fail(QP_ECANCELLED, "ticket %llu was cancelled", (unsigned long long)ticket);
    if (job->state == 3) return fail(job->rc, "%s", job->err.c_str());
    *out = job->result;
    job->result = nullptr;
    return QP_OK;
}

int qp_server_cancel(qp_server* S, uint64_t ticket) {
    if (!S) return fail(QP_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return fail(QP_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    if (it->second->state < 2) it->second->state = 4;
    S->cv.notify_all();
    return QP_OK;
}

void qp_server_destroy(qp_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        for (auto& kv : S->jobs)
            if (kv.second->state < 2) kv.second->state = 4;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto& kv : S->jobs)
        if (kv.second->result) qp_result_free(kv.second->result);
    if (S->stream) cudaStreamDestroy(S->stream);
    delete S;
}

}  // extern "C"
