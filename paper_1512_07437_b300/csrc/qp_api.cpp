// C ABI of the all-pairs posterior stage: validation, per-device context,
// planning of the persistent launch, result assembly.
#include "../../include/qp.h"
#include "qp_internal.h"
#include "qp_host.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

namespace qph {

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(QP_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

const char* last_error() { return g_err.c_str(); }

// ------------------------------------------------------------------ buffers
DevBuf::~DevBuf() { release(); }
void DevBuf::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}
cudaError_t DevBuf::ensure(size_t need) {
    if (need <= bytes && ptr) return cudaSuccess;
    release();
    size_t want = std::max<size_t>(need, 256);
    cudaError_t e = cudaMalloc(&ptr, want);
    if (e != cudaSuccess) { ptr = nullptr; cudaGetLastError(); return e; }
    bytes = want;
    return cudaSuccess;
}

HostBuf::~HostBuf() { if (ptr) cudaFreeHost(ptr); }
cudaError_t HostBuf::ensure(size_t need) {
    if (need <= bytes && ptr) return cudaSuccess;
    if (ptr) cudaFreeHost(ptr);
    ptr = nullptr;
    bytes = 0;
    cudaError_t e = cudaMallocHost(&ptr, std::max<size_t>(need, 256));
    if (e != cudaSuccess) { ptr = nullptr; cudaGetLastError(); return e; }
    bytes = std::max<size_t>(need, 256);
    return cudaSuccess;
}

// ------------------------------------------------------------------ validation
int validate_family(const qp_family* f) {
    if (!f) return fail(QP_EINVAL, "family is NULL");
    if (f->k < 2) return fail(QP_EINVAL, "family needs k >= 2 sequences (k = %d)", f->k);
    if (f->k > kMaxK) return fail(QP_EINVAL, "k = %d exceeds the limit %d", f->k, kMaxK);
    if (!f->offsets) return fail(QP_EINVAL, "offsets is NULL");
    if (!f->residues) return fail(QP_EINVAL, "residues is NULL");
    if (f->offsets[0] != 0) return fail(QP_EINVAL, "offsets[0] must be 0");
    for (int a = 0; a < f->k; ++a) {
        const int64_t L = f->offsets[a + 1] - f->offsets[a];
        if (L < 1) return fail(QP_EINVAL, "sequence %d is empty", a);
        if (L > kMaxLen) return fail(QP_EINVAL, "sequence %d is longer than %lld", a, (long long)kMaxLen);
    }
    return QP_OK;
}

static bool near1(double s) { return std::fabs(s - 1.0) <= 1e-9; }

int validate_params(const qp_params* p) {
    if (!p) return fail(QP_EINVAL, "params is NULL");
    double s = 0;
    for (int i = 0; i < 5; ++i) {
        if (!(p->pi[i] >= 0.0)) return fail(QP_EINVAL, "pi[%d] must be >= 0", i);
        s += p->pi[i];
    }
    if (!near1(s)) return fail(QP_EINVAL, "pi must sum to 1 (sum %.12g)", s);
    if (!(p->delta1 >= 0 && p->delta2 >= 0 && 2 * p->delta1 + 2 * p->delta2 <= 1.0))
        return fail(QP_EINVAL, "need delta1, delta2 >= 0 and 2 delta1 + 2 delta2 <= 1");
    if (!(p->eps1 >= 0 && p->eps1 < 1 && p->eps2 >= 0 && p->eps2 < 1))
        return fail(QP_EINVAL, "eps1, eps2 must be in [0, 1)");
    if (p->alphabet != QP_PROTEIN && p->alphabet != QP_NUCLEOTIDE)
        return fail(QP_EINVAL, "alphabet must be QP_PROTEIN or QP_NUCLEOTIDE");
    if (p->reserved_ != 0) return fail(QP_EINVAL, "reserved_ must be 0");
    const int na = alphabet_size(p->alphabet);
    s = 0;
    for (int a = 0; a < na; ++a)
        for (int b = 0; b < na; ++b) {
            const int i = a * 20 + b;
            if (!(p->emit_pair[i] >= 0.0)) return fail(QP_EINVAL, "emit_pair[%d] must be >= 0", i);
            s += p->emit_pair[i];
        }
    if (!near1(s)) return fail(QP_EINVAL, "emit_pair must sum to 1 over the alphabet (sum %.12g)", s);
    s = 0;
    for (int i = 0; i < na; ++i) {
        if (!(p->emit_bg[i] > 0.0)) return fail(QP_EINVAL, "emit_bg[%d] must be > 0", i);
        s += p->emit_bg[i];
    }
    if (!near1(s)) return fail(QP_EINVAL, "emit_bg must sum to 1 over the alphabet (sum %.12g)", s);
    double te = 0;
    for (int i = 0; i < 5; ++i) {
        if (!(p->end_w[i] >= 0.0 && std::isfinite(p->end_w[i])))
            return fail(QP_EINVAL, "end_w[%d] must be finite and >= 0", i);
        te += p->end_w[i];
    }
    if (!(te > 0)) return fail(QP_EINVAL, "end_w must not be all zero");
    for (int a = 0; a < na; ++a)
        for (int b = 0; b < na; ++b)
            if (!std::isfinite(p->score[a * 20 + b])) return fail(QP_EINVAL, "score[%d] is not finite", a * 20 + b);
    if (!(p->temperature > 0 && std::isfinite(p->temperature))) return fail(QP_EINVAL, "temperature must be > 0");
    if (!std::isfinite(p->gap_open) || !std::isfinite(p->gap_ext)) return fail(QP_EINVAL, "gap penalties must be finite");
    if (p->end_gap_mode != 0) return fail(QP_EINVAL, "only end_gap_mode 0 is supported");
    if (p->combine < 0 || p->combine > 3) return fail(QP_EINVAL, "combine must be one of QP_COMBINE_*");
    if (!(p->threshold > 0.0 && p->threshold <= 1.0)) return fail(QP_EINVAL, "threshold must be in (0, 1]");
    if (p->precision != QP_F32_SCALED && p->precision != QP_F64_PLAIN)
        return fail(QP_EINVAL, "precision must be QP_F32_SCALED or QP_F64_PLAIN");
    if (p->entry_budget < 0) return fail(QP_EINVAL, "entry_budget must be >= 0");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) { cudaGetLastError(); return cuda_fail(e, "cudaGetDeviceCount"); }
    if (p->device < 0 || p->device >= ndev) return fail(QP_EINVAL, "device %d does not exist (%d devices)", p->device, ndev);
    return QP_OK;
}

// ------------------------------------------------------------------ derived constants
void make_raw(const qp_params* p, qpk::RawParams* r) {
    memcpy(r->pi, p->pi, sizeof r->pi);
    r->delta1 = p->delta1; r->eps1 = p->eps1; r->delta2 = p->delta2; r->eps2 = p->eps2;
    memcpy(r->emit_pair, p->emit_pair, sizeof r->emit_pair);
    memcpy(r->emit_bg, p->emit_bg, sizeof r->emit_bg);
    memcpy(r->end_w, p->end_w, sizeof r->end_w);
    memcpy(r->score, p->score, sizeof r->score);
    r->gap_open = p->gap_open; r->gap_ext = p->gap_ext; r->temperature = p->temperature;
    r->threshold = p->threshold;
    r->combine = p->combine;
    r->n_alpha = alphabet_size(p->alphabet);
}

void make_coef(const qp_params* p, qpk::Coef* c) {
    c->tMM = (float)(1.0 - 2.0 * p->delta1 - 2.0 * p->delta2);
    c->d1 = (float)p->delta1; c->d2 = (float)p->delta2;
    c->e1 = (float)p->eps1; c->e2 = (float)p->eps2;
    c->c1 = (float)(1.0 - p->eps1); c->c2 = (float)(1.0 - p->eps2);
    c->Wo = (float)std::exp(p->gap_open / p->temperature);
    c->We = (float)std::exp(p->gap_ext / p->temperature);
    for (int s = 0; s < 5; ++s) { c->pi[s] = (float)p->pi[s]; c->tau[s] = (float)p->end_w[s]; }
    c->theta = (float)p->threshold;
    c->k_open = make_float2(c->d1, c->Wo);
    c->k_ext = make_float2(c->e1, c->We);
    c->k_mm = make_float2(c->tMM, 1.f);
    c->k_close = make_float2(c->c1, 1.f);
    c->tab_x = 8;                     // one table copy (see set_tab_copies)
    c->tab_y = 8 * qpk::kTab;
    c->spin_limit = 0;
    switch (p->combine) {
        case QP_COMBINE_RMS: c->combine = 0; c->wh = 0.5f; c->wp = 0.5f; break;
        case QP_COMBINE_MEAN: c->combine = 1; c->wh = 0.5f; c->wp = 0.5f; break;
        case QP_COMBINE_HMM: c->combine = 1; c->wh = 1.f; c->wp = 0.f; break;
        default: c->combine = 1; c->wh = 0.f; c->wp = 1.f; break;
    }
}

int row_capacity(const qp_params* p, int max_len) {
    // a row's combined posteriors sum to at most sqrt(2) (rms) or 1, so at most
    // that many / theta entries reach the threshold
    const double bound = (p->combine == QP_COMBINE_RMS) ? std::sqrt(2.0) : 1.0;
    const double c = std::floor(bound / p->threshold) + 2.0;
    const double lim = (double)max_len + 1.0;
    return (int)std::min(c, lim);
}

// ------------------------------------------------------------------ planning
std::shared_ptr<Plan> build_plan(int k, const int64_t* off, int64_t p0, int64_t p1) {
    auto pl = std::make_shared<Plan>();
    pl->k = k;
    const int64_t P_all = (int64_t)k * (k - 1) / 2;
    if (p1 < 0) p1 = P_all;
    pl->p0 = p0;
    pl->p1 = p1;
    pl->lens.resize(k);
    int maxL = 0;
    for (int a = 0; a < k; ++a) {
        pl->lens[a] = off[a + 1] - off[a];
        maxL = std::max<int>(maxL, (int)pl->lens[a]);
    }
    pl->max_len = maxL;
    // the plan covers the pairs p0 <= p < p1 of the linear order (all of them
    // by default), numbered from 0 within the plan
    const int64_t P = p1 - p0;
    pl->n_pairs = P;
    pl->pairs.resize(P);
    pl->row_off.resize(P + 1);
    pl->strip_off.resize(P + 1);
    pl->work.resize(P);
    int64_t ro = 0, so = 0, q = 0, g = 0;
    int64_t bst = 0, bex = 0;
    double work_sum = 0;
    for (int a = 0; a < k && g < p1; ++a) {
        const int64_t row_pairs = k - 1 - a;
        if (g + row_pairs <= p0) { g += row_pairs; continue; }    // the whole row of pairs precedes the range
        // what depends on x = sequence a alone: its strips, and the rows per
        // lane summed over them
        const int m = (int)pl->lens[a];
        const int ns = (m + 1 + qpk::kStripRows - 1) / qpk::kStripRows;
        const int last = (m + 1 - (ns - 1) * qpk::kStripRows + 31) / 32;
        const int64_t rows_per_lane = (int64_t)(ns - 1) * qpk::kRmax + (last <= 1 ? 1 : last <= 2 ? 2 : last <= 4 ? 4 : 8);
        const int b0 = std::max<int64_t>(a + 1, a + 1 + (p0 - g));
        const int b1 = (int)std::min<int64_t>(k, a + 1 + (p1 - g));
        int64_t n_max = 0, n_sum = 0;      // columns + skew of the row's pairs
        for (int b = b0; b < b1; ++b, ++q) {
            const int64_t nn = pl->lens[b] + 32;
            pl->pairs[q] = make_int2(a, b);
            pl->row_off[q] = ro;
            pl->strip_off[q] = so;
            ro += m + 1;
            so += ns;
            // swept lane-steps of the pair: rows per lane over the strips x (columns + skew)
            pl->work[q] = rows_per_lane * nn;
            n_max = std::max(n_max, nn);
            n_sum += nn;
        }
        g += row_pairs;
        bst = std::max<int64_t>(bst, (int64_t)ns * qpk::kStripRows * n_max);
        bex = std::max<int64_t>(bex, (int64_t)ns * ((n_max + qpk::kC - 1) / qpk::kC) * 32);
        work_sum += (double)(rows_per_lane * n_sum);    // exact per row
    }
    pl->row_off[P] = ro;
    pl->strip_off[P] = so;
    pl->n_rows = ro;
    pl->n_strips = so;
    // (the FP32 kernel's ring reads up to kD_ring - 1 blocks past a strip)
    pl->bst_stride = bst + (int64_t)qpk::kD_ring * qpk::kWarp * qpk::kRmax;
    pl->bex_stride = bex;
    pl->bnd_stride = 2 * (int64_t)(maxL + 1);
    pl->work_sum = work_sum;
    // longest first keeps the persistent workers balanced (greedy LPT): a
    // stable LSD radix sort by decreasing work, ties in pair order, linear in
    // the pair count (a comparison sort took 0.6 s for 4.5 million pairs)
    {
        int64_t maxw = 0;
        for (int64_t i = 0; i < P; ++i) maxw = std::max(maxw, pl->work[i]);
        std::vector<uint64_t> key(P), key2(P);
        std::vector<int32_t> idx(P), idx2(P);
        for (int64_t i = 0; i < P; ++i) {
            key[i] = (uint64_t)(maxw - pl->work[i]);
            idx[i] = (int32_t)i;
        }
        int bits = 0;
        while (bits < 63 && (maxw >> bits) != 0) ++bits;
        constexpr int kDigit = 11;
        constexpr uint64_t kMask = (1u << kDigit) - 1;
        std::vector<int64_t> cnt((size_t)1 << kDigit);
        for (int shift = 0; shift < bits; shift += kDigit) {
            std::fill(cnt.begin(), cnt.end(), 0);
            for (int64_t i = 0; i < P; ++i) ++cnt[(key[i] >> shift) & kMask];
            int64_t run = 0;
            for (auto& c : cnt) { const int64_t t = c; c = run; run += t; }
            for (int64_t i = 0; i < P; ++i) {
                const int64_t d = cnt[(key[i] >> shift) & kMask]++;
                key2[d] = key[i];
                idx2[d] = idx[i];
            }
            key.swap(key2);
            idx.swap(idx2);
        }
        pl->order.swap(idx);
    }
    return pl;
}

int64_t balanced_grid(int sm_count, int blocks_per_sm, int64_t blocks_needed) {
    const int64_t full = (int64_t)sm_count * blocks_per_sm;
    int64_t g = std::max<int64_t>(1, std::min<int64_t>(full, blocks_needed));
    // more blocks than SMs: the same number on every SM (the blocks beyond
    // the work find none and end), else SMs with one block more than others
    // finish last
    if (g > sm_count) g = std::min<int64_t>(full, (g + sm_count - 1) / sm_count * sm_count);
    return g;
}

unsigned allowed_configs(int64_t n_pairs, int max_strips, int64_t warps_full, int warps_per_block,
                         const LaunchOverride& t, bool wide_layout) {
    unsigned mask = 0;
    for (int cfg = 0; cfg < kTuneConfigs; ++cfg) {
        const int v = config_variant(cfg), W = config_wpp(cfg), lay = config_layout(cfg);
        if (t.variant >= 0 && v != t.variant) continue;
        if (t.wpp > 0 && W != t.wpp) continue;
        if (lay == 1 && (!wide_layout || W > 1)) continue;
        // W must divide the block; groups of several warps use named barriers 1-4
        if (warps_per_block % W || (W > 1 && warps_per_block / W > 4)) continue;
        // two warps per pair only while the pairs leave warps idle (the spare
        // warps then double up on the longest pairs)
        if (t.wpp <= 0 && W > 1 && (max_strips < W || n_pairs >= warps_full)) continue;
        mask |= 1u << cfg;
    }
    return mask ? mask : 1u;
}

int64_t scratch_budget(const LaunchOverride& t) {
    if (t.scratch_bytes > 0) return t.scratch_bytes;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaGetLastError(); fr = 0; }
    const int64_t cap = (int64_t)48 << 30;
    return std::max<int64_t>((int64_t)1 << 30, std::min<int64_t>(cap, (int64_t)(0.45 * (double)fr)));
}

// ------------------------------------------------------------------ result blocks
// Freed result blocks are kept for the next call of the same shape, so that
// repeated calls see the same addresses and relaunch their captured graph.
// The most recently freed blocks are kept; the oldest go first when the cache
// exceeds its bounds.
constexpr size_t kSpareCap = (size_t)8 << 30;   // bytes of result blocks kept for reuse
constexpr size_t kSpareCount = 32;

cudaError_t Context::take_block(void** p, size_t bytes, cudaStream_t st) {
    {
        std::lock_guard<std::mutex> g(spare_mu);
        for (auto it = spare.rbegin(); it != spare.rend(); ++it) {
            if (it->first == bytes) {
                *p = it->second;
                spare.erase(std::next(it).base());
                spare_bytes -= bytes;
                return cudaSuccess;
            }
        }
    }
    cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e != cudaSuccess) { *p = nullptr; cudaGetLastError(); }
    return e;
}

void Context::give_block(void* p, size_t bytes) {
    if (!p) return;
    if (bytes == 0 || bytes > kSpareCap) { cudaFreeAsync(p, stream); return; }
    std::lock_guard<std::mutex> g(spare_mu);
    spare.emplace_back(bytes, p);
    spare_bytes += bytes;
    while (spare_bytes > kSpareCap || spare.size() > kSpareCount) {
        cudaFreeAsync(spare.front().second, stream);
        spare_bytes -= spare.front().first;
        spare.pop_front();
    }
}

// ------------------------------------------------------------------ autotuner key
int64_t Context::tune_key(int64_t n_pairs, int max_len, double work) {
    // buckets: pair count (half powers of two), longest sequence (64s), mean
    // work per pair (powers of two)
    const int pb = n_pairs > 0 ? (int)std::floor(2.0 * std::log2((double)n_pairs)) : 0;
    const int lb = max_len / 64;
    const int wb = n_pairs > 0 ? (int)std::floor(std::log2(1.0 + work / (double)n_pairs)) : 0;
    return ((int64_t)pb << 40) | ((int64_t)lb << 16) | (int64_t)wb;
}

// ------------------------------------------------------------------ device context
static std::mutex g_ctx_mu;
static std::map<int, std::unique_ptr<Context>> g_ctx;

Context* get_context(int device, int* status) {
    std::lock_guard<std::mutex> g(g_ctx_mu);
    auto it = g_ctx.find(device);
    if (it != g_ctx.end()) return it->second.get();
    std::unique_ptr<Context> c(new Context());
    c->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) { *status = cuda_fail(e, "cudaSetDevice"); return nullptr; }
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) { *status = cuda_fail(e, "cudaGetDeviceProperties"); return nullptr; }
    c->sm_count = prop.multiProcessorCount;
    c->cc_major = prop.major; c->cc_minor = prop.minor;
    c->smem_optin = (int)prop.sharedMemPerBlockOptin;
    c->smem_per_sm = (int)prop.sharedMemPerMultiprocessor;
    if (prop.major < 10) {
        *status = fail(QP_ECUDA, "device %d is sm_%d%d; this library is built for sm_103a", device, prop.major, prop.minor);
        return nullptr;
    }
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { *status = cuda_fail(e, "cudaStreamCreate"); return nullptr; }
    for (auto& ev : c->ev) {
        e = cudaEventCreate(&ev);
        if (e != cudaSuccess) { *status = cuda_fail(e, "cudaEventCreate"); return nullptr; }
    }
    e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) { *status = cuda_fail(e, "cudaEventCreate"); return nullptr; }
    int bps64 = 0;
    qpk::posterior_f64_occupancy(&bps64);
    c->f64_blocks_per_sm = std::max(1, std::min(bps64, 4));
    if (const char* v = getenv("QP_F32_VARIANT")) c->tune.variant = atoi(v);
    if (const char* v = getenv("QP_F32_CKPT")) c->tune.ckpt = atoi(v);
    if (const char* v = getenv("QP_F32_BLOCKS")) c->tune.blocks_per_sm = atoi(v);
    if (const char* v = getenv("QP_F32_WPP")) c->tune.wpp = atoi(v);
    if (const char* v = getenv("QP_GRAPH")) c->tune.graph = atoi(v) != 0;
    if (const char* v = getenv("QP_HOST_CHUNKS")) c->tune.host_chunks = std::max(0, std::min(atoi(v), 16));
    if (const char* v = getenv("QP_SCRATCH_BYTES")) c->tune.scratch_bytes = atoll(v);
    Context* raw = c.get();
    g_ctx[device] = std::move(c);
    return raw;
}

int f32_max_len(const Context* C, int warps_per_block) {
    const size_t cap = (size_t)C->smem_optin;
    if (qpk::posterior_f32_smem(warps_per_block, 1, 1) > cap) return 0;
    int lo = 1, hi = (int)kMaxLen;
    while (lo < hi) {
        const int mid = lo + (hi - lo + 1) / 2;
        if (qpk::posterior_f32_smem(warps_per_block, mid, 1) <= cap) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// the FP32 form's length limit for a family (blocks of two warps, the
// smallest the autotuner launches)
static int check_f32_lengths(const Context* C, const qp_family* f, const qp_params* prm) {
    if (prm->precision != QP_F32_SCALED) return QP_OK;
    const int lim = f32_max_len(C, 2);
    for (int a = 0; a < f->k; ++a) {
        const int64_t L = f->offsets[a + 1] - f->offsets[a];
        if (L > lim)
            return fail(QP_EINVAL, "sequence %d has %lld residues; the FP32 form takes at most %d on this device",
                        a, (long long)L, lim);
    }
    return QP_OK;
}

cudaError_t call_stream(Context* C, void* user, cudaStream_t* st) {
    if (user) {
        *st = (cudaStream_t)user;
        return cudaSuccess;
    }
    *st = C->stream;
    cudaError_t e = cudaEventRecord(C->ev_join, cudaStreamLegacy);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(C->stream, C->ev_join, 0);
    return e;
}

std::shared_ptr<Plan> Context::plan_for(int k, const int64_t* off, int* status, int64_t p0, int64_t p1) {
    // cache keyed by the length vector and the pair range
    std::vector<int64_t> lens(k);
    for (int a = 0; a < k; ++a) lens[a] = off[a + 1] - off[a];
    if (p1 < 0) p1 = (int64_t)k * (k - 1) / 2;
    for (auto& pl : plans)
        if (pl->k == k && pl->p0 == p0 && pl->p1 == p1 && pl->lens == lens) return pl;
    auto pl = build_plan(k, off, p0, p1);
    const int64_t P = pl->n_pairs;
    std::vector<int2> items(P);
    for (int64_t i = 0; i < P; ++i) items[i] = make_int2(0, pl->order[i]);
    cudaError_t e;
    if ((e = pl->d_pairs.ensure(sizeof(int2) * P)) != cudaSuccess ||
        (e = pl->d_row_off.ensure(sizeof(int64_t) * (P + 1))) != cudaSuccess ||
        (e = pl->d_strip_off.ensure(sizeof(int64_t) * (P + 1))) != cudaSuccess ||
        (e = pl->d_items.ensure(sizeof(int2) * P)) != cudaSuccess) {
        *status = fail(QP_ENOMEM, "plan allocation failed: %s", cudaGetErrorString(e));
        return nullptr;
    }
    cudaMemcpy(pl->d_pairs.ptr, pl->pairs.data(), sizeof(int2) * P, cudaMemcpyHostToDevice);
    cudaMemcpy(pl->d_row_off.ptr, pl->row_off.data(), sizeof(int64_t) * (P + 1), cudaMemcpyHostToDevice);
    cudaMemcpy(pl->d_strip_off.ptr, pl->strip_off.data(), sizeof(int64_t) * (P + 1), cudaMemcpyHostToDevice);
    e = cudaMemcpy(pl->d_items.ptr, items.data(), sizeof(int2) * P, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { *status = cuda_fail(e, "plan upload"); return nullptr; }
    plans.push_back(pl);
    if (plans.size() > 16) plans.erase(plans.begin());   // (a family and its ranges fit)
    return pl;
}

// ------------------------------------------------------------------ one family
void fill_result(qp_result* r, ResultOwner* own, const ResultLayout& L, int k, int64_t n_pairs,
                 int64_t n_rows, int64_t nnz_bound, bool f64, int precision, int device) {
    char* A = (char*)own->dev_a;
    char* B = (char*)own->dev_b;
    r->k = k;
    r->on_device = 1;
    r->precision = precision;
    r->device = device;
    r->n_pairs = n_pairs;
    r->n_rows = n_rows;
    r->pair_row_off = (int64_t*)(A + L.o_pro);
    r->row_ptr = (int32_t*)(A + L.o_rp);
    r->pair_nnz_off = (int64_t*)(A + L.o_pno);
    r->col = (int32_t*)B;
    r->val = B ? (float*)(B + align256(sizeof(int32_t) * nnz_bound)) : nullptr;
    r->val64 = (B && f64) ? (double*)(B + align256(sizeof(int32_t) * nnz_bound) +
                                      align256(sizeof(float) * nnz_bound)) : nullptr;
    r->dist = (float*)(A + L.o_dist);
    r->dist64 = (double*)(A + L.o_d64);
    r->mea = (double*)(A + L.o_mea);
    r->log_z_hmm = (double*)(A + L.o_lh);
    r->log_z_pf = (double*)(A + L.o_lp);
    r->pair_flags = (int32_t*)(A + L.o_fl);
    r->owner_ = own;
}

int run_family(Context* C, const qp_family* f, const qp_params* prm, int32_t out_on_device,
               qp_result** out, int64_t p0, int64_t p1) {
    cudaError_t e;
    const int k = f->k;
    cudaStream_t st;
    if ((e = call_stream(C, prm->stream, &st)) != cudaSuccess) return cuda_fail(e, "stream order");
    int status = QP_OK;
    auto pl = C->plan_for(k, f->offsets, &status, p0, p1);
    if (!pl) return status;
    const int64_t P = pl->n_pairs;
    const int64_t total_res = f->offsets[k];
    const bool f64 = prm->precision == QP_F64_PLAIN;
    const int cap = row_capacity(prm, pl->max_len);
    const int64_t budget = scratch_budget(C->tune);

    // ---- inputs and fixed workspace
    if ((e = C->codes.ensure(total_res)) != cudaSuccess ||
        (!f->residues_on_device && (e = C->ascii.ensure(total_res)) != cudaSuccess) ||
        (e = C->off.ensure(sizeof(int64_t) * (k + 1))) != cudaSuccess ||
        (e = C->seqlogq.ensure(sizeof(double) * k)) != cudaSuccess ||
        (e = C->cst.ensure(sizeof(qpk::Consts))) != cudaSuccess ||
        (e = C->status.ensure(sizeof(qpk::Status))) != cudaSuccess ||
        (e = C->fam.ensure(sizeof(qpk::FamDesc))) != cudaSuccess ||
        (e = C->h_status.ensure(sizeof(qpk::Status) + 64)) != cudaSuccess ||
        (e = C->h_fam.ensure(sizeof(qpk::FamDesc))) != cudaSuccess ||
        (e = C->h_off.ensure(sizeof(int64_t) * (k + 1))) != cudaSuccess ||
        (e = C->row_cnt.ensure(sizeof(int32_t) * pl->n_rows)) != cudaSuccess ||
        (e = C->chunk_off.ensure(sizeof(int64_t) * pl->n_strips)) != cudaSuccess ||
        (e = C->pair_nnz.ensure(sizeof(int64_t) * P)) != cudaSuccess ||
        (e = C->fallback.ensure(sizeof(int2) * P)) != cudaSuccess)
        return fail(QP_ENOMEM, "workspace allocation failed: %s", cudaGetErrorString(e));
    memcpy(C->h_off.ptr, f->offsets, sizeof(int64_t) * (k + 1));
    const uint8_t* d_ascii = f->residues;
    if (!f->residues_on_device) {
        // pageable user memory: copied before (outside) the captured sequence
        e = cudaMemcpyAsync(C->ascii.ptr, f->residues, total_res, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "copy residues");
        d_ascii = (const uint8_t*)C->ascii.ptr;
    }
    // derived tables: recomputed only when the parameters change
    qpk::RawParams raw;
    memset(&raw, 0, sizeof raw);
    make_raw(prm, &raw);
    if (!C->raw_valid || memcmp(&raw, &C->last_raw, sizeof raw) != 0) {
        if ((e = C->d_raw.ensure(sizeof(qpk::RawParams))) != cudaSuccess)
            return fail(QP_ENOMEM, "workspace allocation failed");
        if ((e = qpk::launch_setup(&raw, (qpk::RawParams*)C->d_raw.ptr, (qpk::Consts*)C->cst.ptr, st)) != cudaSuccess)
            return cuda_fail(e, "k_setup");
        C->last_raw = raw;
        C->raw_valid = true;
    }

    // ---- launch configuration of the FP32 kernel
    // The autotuner picks the register variant, the warps per pair and the
    // block layout: blocks of 2 warps with one emission table (finer
    // placement over the SMs), or, for launches that fill the grid when two
    // such blocks fit an SM, blocks of 8 warps holding the bank-sliced table
    // (kTabCopies copies: conflict-free lookups).  The launch knobs
    // warps_per_block and tab_copies fix the layout instead.
    const bool layout_forced = C->tune.warps_per_block > 0 || C->tune.tab_copies >= 0;
    int wpb = 2;
    int copies = 1;
    auto set_layout = [&](int lay) {
        if (layout_forced) {
            wpb = C->tune.warps_per_block > 0 ? C->tune.warps_per_block : 2;
            copies = C->tune.tab_copies >= 0 ? C->tune.tab_copies : 1;
        } else {
            wpb = lay == 1 ? 8 : 2;
            copies = lay == 1 ? qpk::kTabCopies : 1;
        }
    };
    set_layout(0);
    int variant = 0, cfg = 0, W = 1;
    bool ckpt = false;
    int64_t grid = 1, tkey = 0;
    qpk::Problem Pb;
    memset(&Pb, 0, sizeof Pb);
    make_coef(prm, &Pb.cf);
    Pb.cst = (const qpk::Consts*)C->cst.ptr;
    Pb.fams = (const qpk::FamDesc*)C->fam.ptr;
    Pb.items = (const int2*)pl->d_items.ptr;
    Pb.n_work = (int32_t)P;
    Pb.cap = cap;
    Pb.status = (qpk::Status*)C->status.ptr;
    Pb.fallback = (int2*)C->fallback.ptr;
    Pb.max_len = pl->max_len;
    Pb.cf.spin_limit = C->tune.spin_limit;
    auto set_tables = [&]() {
        Pb.tab_copies = copies > 1 ? qpk::kTabCopies : 1;
        Pb.cf.tab_x = 8u * (uint32_t)Pb.tab_copies;
        Pb.cf.tab_y = 8u * (uint32_t)(qpk::kTab * Pb.tab_copies);
    };
    set_tables();
    if (!f64) {
        auto occupancy = [&](int v, bool ck, int w = 1) {
            int b = C->tune.blocks_per_sm;
            if (b <= 0) {
                qpk::posterior_f32_occupancy(wpb, pl->max_len, &b, v, ck, w, Pb.tab_copies);
                b = std::max(1, std::min(b, 8));
            }
            return b;
        };
        // bytes of a grid of `warps` warps, w warps per pair (every buffer is
        // per warp; the stored form keeps the plan's tighter per-pair sizes)
        auto scratch_of = [&](bool ck, int w, int64_t warps) -> int64_t {
            const qpk::F32Scratch sz(pl->max_len, cap, ck, w);
            if (ck) return (int64_t)sz.bytes(warps);
            return warps * (int64_t)(sizeof(float2) * pl->bst_stride + sizeof(int2) * pl->bex_stride +
                                     sizeof(float4) * (sz.bnd + sz.bck) + sizeof(int2) * sz.stg);
        };
        // stored form unless its scratch for a full grid exceeds the budget;
        // then the checkpointed form, on a grid cut to the budget if need be
        ckpt = C->tune.ckpt >= 0 ? C->tune.ckpt != 0 : false;
        const int64_t warps_full = (int64_t)C->sm_count * occupancy(0, false) * wpb;
        if (C->tune.ckpt < 0)
            ckpt = scratch_of(false, 1, std::min<int64_t>(warps_full, ((P + wpb - 1) / wpb) * wpb)) > budget;
        const int max_strips = (pl->max_len + 1 + qpk::kStripRows - 1) / qpk::kStripRows;
        const bool wide = !layout_forced && P >= warps_full &&
                          qpk::posterior_f32_tab_copies(8, pl->max_len, C->smem_per_sm) > 1;
        const unsigned allowed = allowed_configs(P, max_strips, warps_full, wpb, C->tune, wide);
        tkey = (C->tune_alias ? C->tune_alias : Context::tune_key(P, pl->max_len, pl->work_sum)) ^
               ((int64_t)ckpt << 62);
        cfg = C->tuner[tkey].choose(allowed);
        variant = config_variant(cfg);
        W = config_wpp(cfg);
        set_layout(config_layout(cfg));
        set_tables();
        // with two warps per pair, the spare warps of a launch whose pairs do
        // not fill the grid double up on the longest pairs (items come longest
        // first): n_big items run on two warps, the rest on one
        int64_t n_big = 0;
        if (W > 1) {
            const int64_t full_w = (int64_t)C->sm_count * occupancy(variant, ckpt, W) * wpb;
            n_big = std::max<int64_t>(0, std::min<int64_t>(P, full_w - P));
        }
        Pb.n_big = (int32_t)n_big;
        grid = balanced_grid(C->sm_count, occupancy(variant, ckpt, W), (P + n_big + wpb - 1) / wpb);
        grid = std::min<int64_t>(grid, std::max<int64_t>(1, budget / std::max<int64_t>(1, scratch_of(ckpt, W, wpb))));
        grid = std::max<int64_t>(grid, 1);
        const int64_t warps = grid * wpb;
        const qpk::F32Scratch sz(pl->max_len, cap, ckpt, W);
        const int64_t bst_stride = ckpt ? sz.bst : pl->bst_stride;
        const int64_t bex_stride = ckpt ? sz.bex : pl->bex_stride;
        if ((e = C->bst.ensure(sizeof(float2) * bst_stride * warps)) != cudaSuccess ||
            (e = C->bex.ensure(sizeof(int2) * bex_stride * warps)) != cudaSuccess ||
            (e = C->bnd.ensure(sizeof(float4) * sz.bnd * warps)) != cudaSuccess ||
            (e = C->bck.ensure(sizeof(float4) * sz.bck * warps)) != cudaSuccess ||
            (e = C->stg.ensure(sizeof(int2) * sz.stg * warps)) != cudaSuccess)
            return fail(QP_ENOMEM, "FP32 scratch allocation failed");
        Pb.bst = (float2*)C->bst.ptr; Pb.bst_stride = bst_stride;
        Pb.bex = (int2*)C->bex.ptr; Pb.bex_stride = bex_stride;
        Pb.bnd = (float4*)C->bnd.ptr; Pb.bnd_stride = sz.bnd;
        Pb.bck = (float4*)C->bck.ptr; Pb.bck_stride = sz.bck;
        Pb.ckpt = ckpt ? 1 : 0;
        Pb.wpp = W;
        Pb.stg = (int2*)C->stg.ptr; Pb.stg_stride = sz.stg;
        C->last_variant = variant; C->last_wpp = W; C->last_wpb = wpb; C->last_copies = Pb.tab_copies;
    }
    // FP64 form: over every pair (plain form), or as the follow-up of the FP32
    // kernel on a small fixed grid that finds its pairs in the fallback list
    // (it ends at once when the list is empty, so no host decision is needed)
    int f64_grid;
    {
        const int64_t L = pl->max_len + 1;
        // the stored backward values of a pair take (m + 1)(n + 1) cells: at
        // most the product of the two longest lengths (+1 each), which for a
        // family with one very long sequence is far below L * L
        int64_t l1 = 0, l2 = 0;
        for (int a = 0; a < k; ++a) {
            const int64_t la = f->offsets[a + 1] - f->offsets[a];
            if (la > l1) { l2 = l1; l1 = la; } else if (la > l2) l2 = la;
        }
        const int64_t db = (l1 + 1) * (l2 + 1);
        const int64_t per_cta = (int64_t)(sizeof(double2) * db + sizeof(double) * 3 * qpk::kNS * L +
                                          sizeof(int32_t) * (5 * L + 8) +
                                          (sizeof(int2) + sizeof(double)) * (int64_t)pl->max_len * cap);
        // (the follow-up grid keeps at most ~1 GiB of FP64 scratch)
        const int64_t want = f64 ? std::min<int64_t>(P, (int64_t)C->sm_count * C->f64_blocks_per_sm)
                                 : std::min<int64_t>(std::min<int64_t>(P, kF64FollowGrid),
                                                     std::max<int64_t>(2, ((int64_t)1 << 30) / per_cta));
        // sequences so long that one CTA's FP64 scratch exceeds the budget get
        // no follow-up (a pair that would need it makes the call fail below)
        f64_grid = (int)std::min<int64_t>(want, budget / per_cta);
        if (f64 && f64_grid < 1)
            return fail(QP_ENOMEM, "the FP64 form needs %lld bytes per pair at length %d, more than the scratch "
                        "budget %lld", (long long)per_cta, pl->max_len, (long long)budget);
        if (f64_grid > 0 && ((e = C->d_b.ensure(sizeof(double2) * db * f64_grid)) != cudaSuccess ||
            (e = C->d_diag.ensure(sizeof(double) * 3 * qpk::kNS * L * f64_grid)) != cudaSuccess ||
            (e = C->d_cnt.ensure(sizeof(int32_t) * (5 * L + 8) * f64_grid)) != cudaSuccess ||
            (e = C->d_stg.ensure(sizeof(int2) * (int64_t)pl->max_len * cap * f64_grid)) != cudaSuccess ||
            (e = C->d_stg64.ensure(sizeof(double) * (int64_t)pl->max_len * cap * f64_grid)) != cudaSuccess))
            return fail(QP_ENOMEM, "FP64 scratch allocation failed");
        Pb.d_b = (double2*)C->d_b.ptr; Pb.d_b_stride = db;
        Pb.d_diag = (double*)C->d_diag.ptr; Pb.d_diag_stride = 3 * qpk::kNS * L;
        Pb.f64_smem_diag = qpk::posterior_f64_smem_diag(pl->max_len) ? 1 : 0;
        Pb.d_cnt = (int32_t*)C->d_cnt.ptr; Pb.d_cnt_stride = 5 * L + 8;
        Pb.d_stg = (int2*)C->d_stg.ptr; Pb.d_stg64 = (double*)C->d_stg64.ptr;
        Pb.d_stg_stride = (int64_t)pl->max_len * cap;
        Pb.f64_all = f64 ? 1 : 0;
    }

    // ---- result: fixed part, and col / val at the pool's capacity (the
    // entry count is known only at the end; no host decision in between)
    ResultOwner* own = new ResultOwner();
    own->device = C->device;
    auto bail = [&](int code) {
        if (own->dev_a) cudaFreeAsync(own->dev_a, st);
        if (own->dev_b) cudaFreeAsync(own->dev_b, st);
        cudaStreamSynchronize(st);
        delete own;
        return code;
    };
    const ResultLayout lay(P, pl->n_rows, k);
    int64_t call_cap = 0;    // entries this call's pool and result may hold
    e = C->take_block(&own->dev_a, lay.bytes, st);
    if (e != cudaSuccess) return bail(fail(QP_ENOMEM, "result allocation (%zu bytes) failed", lay.bytes));
    own->bytes_a = lay.bytes;
    char* A = (char*)own->dev_a;
    {
        const double per_row = std::min<double>(pl->max_len + 1.0, 4.0 + 0.04 / prm->threshold);
        int64_t est = (int64_t)(per_row * (double)pl->n_rows) + 4096;
        est = std::max<int64_t>(est, C->pool_hint);
        if (C->tune.pool_entries > 0) est = std::min<int64_t>(est, C->tune.pool_entries);
        if ((e = C->pool.ensure(sizeof(int2) * est)) != cudaSuccess ||
            (f64 && (e = C->pool64.ensure(sizeof(double) * est)) != cudaSuccess))
            return bail(fail(QP_ENOMEM, "pool allocation failed"));
        C->pool_cap = (int64_t)(C->pool.bytes / sizeof(int2));
        if (f64) C->pool_cap = std::min<int64_t>(C->pool_cap, (int64_t)(C->pool64.bytes / sizeof(double)));
        // this call's capacity: its own estimate, not the largest pool an
        // earlier (larger) call left (the result's entry block is sized by it)
        call_cap = std::min<int64_t>(C->pool_cap, est);
    }

    qpk::FamDesc fd;
    memset(&fd, 0, sizeof fd);
    fd.codes = (const uint8_t*)C->codes.ptr;
    fd.seq_off = (const int64_t*)C->off.ptr;
    fd.seq_logq = (const double*)C->seqlogq.ptr;
    fd.pairs = (const int2*)pl->d_pairs.ptr;
    fd.pair_row_off = (const int64_t*)pl->d_row_off.ptr;
    fd.pair_strip_off = (const int64_t*)pl->d_strip_off.ptr;
    fd.k = k;
    fd.row_cnt = (int32_t*)C->row_cnt.ptr;
    fd.chunk_off = (int64_t*)C->chunk_off.ptr;
    fd.pair_nnz = (int64_t*)C->pair_nnz.ptr;
    fd.mea = (double*)(A + lay.o_mea);
    fd.logz_h = (double*)(A + lay.o_lh);
    fd.logz_p = (double*)(A + lay.o_lp);
    fd.dist = (float*)(A + lay.o_dist);
    fd.dist64 = (double*)(A + lay.o_d64);
    fd.pair_flags = (int32_t*)(A + lay.o_fl);
    qpk::Status* d_status = (qpk::Status*)C->status.ptr;
    fd.pool_used = &d_status->pool_used;
    fd.pool_base = 0;

    qpk::Status hs;
    memset(&hs, 0, sizeof hs);
    int64_t nnz = 0;
    bool timed_call = false;
    // entry budget: the full CSR goes to scratch, a select finds the raised
    // threshold and a filter writes the result (at most n_keep entries)
    const bool ebudget = prm->entry_budget > 0;
    const int64_t n_keep = ebudget ? prm->entry_budget / (f64 ? 16 : 8) : 0;
    auto nnz_cap_of = [&]() { return ebudget ? std::min<int64_t>(call_cap, n_keep) : call_cap; };
    if (ebudget &&
        ((e = C->bud_rp.ensure(sizeof(int32_t) * pl->n_rows)) != cudaSuccess ||
         (e = C->bud_off.ensure(sizeof(int64_t) * (P + 1))) != cudaSuccess ||
         (e = C->bud_nnz.ensure(sizeof(int64_t) * P)) != cudaSuccess ||
         (e = C->bud_state.ensure(sizeof(qpk::SelectState))) != cudaSuccess ||
         (e = C->bud_hist.ensure(sizeof(unsigned) * qpk::kBudgetBins + 16)) != cudaSuccess ||
         (e = qpk::prepare_budget_kernels()) != cudaSuccess))
        return bail(fail(QP_ENOMEM, "entry budget scratch allocation failed"));
    for (int attempt = 0;; ++attempt) {
        if (own->dev_b) { C->give_block(own->dev_b, own->bytes_b); own->dev_b = nullptr; }
        if (ebudget &&
            ((e = C->bud_col.ensure(sizeof(int32_t) * call_cap)) != cudaSuccess ||
             (e = C->bud_val.ensure(sizeof(float) * call_cap)) != cudaSuccess ||
             (f64 && (e = C->bud_val64.ensure(sizeof(double) * call_cap)) != cudaSuccess)))
            return bail(fail(QP_ENOMEM, "entry budget scratch allocation failed"));
        const int64_t nnz_cap = nnz_cap_of();
        own->bytes_b = std::max<size_t>(ResultLayout::entry_bytes(nnz_cap, f64), 256);
        e = C->take_block(&own->dev_b, own->bytes_b, st);
        if (e != cudaSuccess) return bail(fail(QP_ENOMEM, "result allocation failed"));
        qp_result probe;
        memset(&probe, 0, sizeof probe);
        fill_result(&probe, own, lay, k, P, pl->n_rows, nnz_cap, f64, prm->precision, C->device);
        fd.pool_cap = call_cap;
        memcpy(C->h_fam.ptr, &fd, sizeof fd);
        Pb.pool = (int2*)C->pool.ptr;
        Pb.pool64 = f64 ? (double*)C->pool64.ptr : nullptr;
        // the whole call, one host synchronisation at the end
        // timed: CUDA events around the posterior kernels (plain launches only:
        // a captured sequence carries none)
        bool timed = false;
        bool start_in_enqueue = false;   // plain launches: the start event follows the input copies
        auto enqueue = [&]() -> cudaError_t {
            cudaError_t x;
            if ((x = cudaMemcpyAsync(C->off.ptr, C->h_off.ptr, sizeof(int64_t) * (k + 1), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
                (x = cudaMemcpyAsync(C->fam.ptr, C->h_fam.ptr, sizeof fd, cudaMemcpyHostToDevice, st)) != cudaSuccess)
                return x;
            if (start_in_enqueue) cudaEventRecord(C->ev[0], st);
            if ((x = cudaMemsetAsync(C->status.ptr, 0, sizeof(qpk::Status), st)) != cudaSuccess ||
                (x = cudaMemcpyAsync(A + lay.o_pro, pl->d_row_off.ptr, sizeof(int64_t) * (P + 1), cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
                (x = cudaMemsetAsync(A + lay.o_dist, 0, sizeof(float) * (size_t)k * k, st)) != cudaSuccess ||
                (x = cudaMemsetAsync(A + lay.o_d64, 0, sizeof(double) * (size_t)k * k, st)) != cudaSuccess ||
                (x = cudaMemsetAsync(A + lay.o_fl, 0, sizeof(int32_t) * P, st)) != cudaSuccess)
                return x;
            if ((x = qpk::launch_encode(d_ascii, (uint8_t*)C->codes.ptr, total_res, (const int64_t*)C->off.ptr, k,
                                        (double*)C->seqlogq.ptr, (const qpk::Consts*)C->cst.ptr, d_status, st)) != cudaSuccess)
                return x;
            if (timed) cudaEventRecord(C->ev[1], st);
            if (!f64 && (x = qpk::launch_posterior_f32(Pb, (int)grid, wpb, st, variant)) != cudaSuccess) return x;
            if (timed) cudaEventRecord(C->ev[2], st);
            if (f64_grid > 0 && (x = qpk::launch_posterior_f64(Pb, f64_grid, st)) != cudaSuccess) return x;
            if (timed) cudaEventRecord(C->ev[3], st);
            if (!ebudget) {
                if ((x = qpk::launch_scan_nnz(fd.pair_nnz, P, probe.pair_nnz_off, st)) != cudaSuccess ||
                    (x = qpk::launch_compact(fd.pairs, fd.seq_off, fd.pair_row_off, fd.pair_strip_off, fd.row_cnt,
                                             fd.chunk_off, Pb.pool, Pb.pool64, P, probe.pair_nnz_off, probe.row_ptr,
                                             probe.col, probe.val, probe.val64, st, nullptr,
                                             &d_status->pool_overflow)) != cudaSuccess)
                    return x;
            } else {
                int64_t* b_off = (int64_t*)C->bud_off.ptr;
                int32_t* b_rp = (int32_t*)C->bud_rp.ptr;
                int32_t* b_col = (int32_t*)C->bud_col.ptr;
                float* b_val = (float*)C->bud_val.ptr;
                double* b_val64 = f64 ? (double*)C->bud_val64.ptr : nullptr;
                qpk::SelectState* sel = (qpk::SelectState*)C->bud_state.ptr;
                unsigned* hist = (unsigned*)C->bud_hist.ptr;
                // smallest and largest key, after the histogram
                unsigned long long* minmax = (unsigned long long*)(hist + qpk::kBudgetBins);
                if ((x = cudaMemsetAsync(minmax, 0xff, sizeof(unsigned long long), st)) != cudaSuccess ||
                    (x = cudaMemsetAsync(minmax + 1, 0, sizeof(unsigned long long), st)) != cudaSuccess ||
                    (x = qpk::launch_scan_nnz(fd.pair_nnz, P, b_off, st)) != cudaSuccess ||
                    (x = qpk::launch_compact(fd.pairs, fd.seq_off, fd.pair_row_off, fd.pair_strip_off, fd.row_cnt,
                                             fd.chunk_off, Pb.pool, Pb.pool64, P, b_off, b_rp, b_col, b_val,
                                             b_val64, st, minmax, &d_status->pool_overflow)) != cudaSuccess ||
                    (x = qpk::launch_budget_select(b_off + P, n_keep, prm->threshold, f64, b_val, b_val64, minmax,
                                                   sel, hist, d_status, 4 * C->sm_count, st)) != cudaSuccess ||
                    (x = qpk::launch_budget_count(fd.pairs, fd.seq_off, fd.pair_row_off, b_off, b_rp, b_val,
                                                  b_val64, sel, P, probe.row_ptr, (int64_t*)C->bud_nnz.ptr,
                                                  d_status, st)) != cudaSuccess ||
                    (x = qpk::launch_scan_nnz((const int64_t*)C->bud_nnz.ptr, P, probe.pair_nnz_off, st)) !=
                        cudaSuccess ||
                    (x = qpk::launch_budget_copy(fd.pairs, fd.seq_off, fd.pair_row_off, b_off, b_rp, b_col, b_val,
                                                 b_val64, sel, P, probe.pair_nnz_off, probe.row_ptr, probe.col,
                                                 probe.val, probe.val64, nnz_cap, d_status, st)) != cudaSuccess)
                    return x;
            }
            char* hs_p = (char*)C->h_status.ptr;
            if ((x = cudaMemcpyAsync(hs_p, C->status.ptr, sizeof(qpk::Status), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                (x = cudaMemcpyAsync(hs_p + sizeof(qpk::Status), probe.pair_nnz_off + P, sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                return x;
            return cudaSuccess;
        };
        // events only outside the captured sequence: the whole call; the
        // kernels time themselves (Status time stamps).  Plain launches record
        // the start after their first input copies.  Measured on B300: when the
        // event record was the first command on the stream after the previous
        // range's synchronisation, while the copy stream still held that
        // range's device-to-host copies, the stream waited for those copies
        // (each range of a host-output call with device-resident residues
        // took about 13 ms longer: 105 against 68 ms for the 500-sequence
        // family); with a copy first it did not.
        if (C->tune.graph && !C->tune_alias) cudaEventRecord(C->ev[0], st);
        else start_in_enqueue = true;
        // (the ranges of a host-output call run as plain launches: their shapes
        // alternate, so a captured graph would be rebuilt on every call)
        if (C->tune.graph && !C->tune_alias) {
            // everything the sequence's nodes hold (pointers, sizes, launch
            // shapes, kernel parameters): equal keys relaunch the cached graph
            GraphKey key;
            memset(&key, 0, sizeof key);
            const void* ptrs[] = {C->off.ptr, C->h_off.ptr, C->fam.ptr, C->h_fam.ptr, C->status.ptr,
                                  C->h_status.ptr, A, own->dev_b, pl->d_row_off.ptr, d_ascii, C->codes.ptr,
                                  C->seqlogq.ptr, C->cst.ptr, (const void*)st, C->bud_rp.ptr, C->bud_off.ptr,
                                  C->bud_col.ptr, C->bud_val.ptr, C->bud_val64.ptr, C->bud_nnz.ptr,
                                  C->bud_state.ptr, C->bud_hist.ptr};
            static_assert(sizeof ptrs / sizeof ptrs[0] <= sizeof key.p / sizeof key.p[0], "graph key");
            memcpy(key.p, ptrs, sizeof ptrs);
            const int64_t vals[] = {k, P, pl->n_rows, total_res, nnz_cap, grid, wpb, variant, f64_grid, f64 ? 1 : 0,
                                    ebudget ? n_keep : -1};
            memcpy(key.v, vals, sizeof vals);
            key.pb = Pb;
            e = launch_graph(C, st, key, enqueue);
            if (e != cudaSuccess && cudaPeekAtLastError() == cudaSuccess) {
                // the graph could not be built or launched (nothing ran): keep
                // to plain launches on this device from now on
                fprintf(stderr, "libqp: CUDA graph launch failed (%s); using plain launches\n",
                        cudaGetErrorName(e));
                C->tune.graph = false;
                timed = true;
                e = enqueue();
            }
        } else {
            timed = true;
            ++C->plain_calls;
            e = enqueue();
        }
        cudaEventRecord(C->ev[4], st);
        timed_call = timed;
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return bail(cuda_fail(e, "posterior stage"));
        memcpy(&hs, C->h_status.ptr, sizeof hs);
        memcpy(&nnz, (char*)C->h_status.ptr + sizeof(qpk::Status), sizeof nnz);
        if (hs.bad_residue)
            return bail(fail(QP_EINVAL, "%s", alphabet_error(prm->alphabet)));
        if (hs.stage_overflow) return bail(fail(QP_ECUDA, "internal: a row exceeded its entry capacity"));
        if (hs.select_error) return bail(fail(QP_ECUDA, "internal: the entry budget's selection failed"));
        if (!f64 && f64_grid == 0 && hs.n_fallback > 0)
            return bail(fail(QP_ENOMEM, "%d pair(s) tripped an FP32 range guard and need the FP64 form, whose "
                             "scratch at length %d exceeds the budget", hs.n_fallback, pl->max_len));
        if (!f64 && hs.t_f32[1] > hs.t_f32[0] && hs.t_f32[0] > 0)
            if (!C->tune_alias) C->tuner[tkey].record(cfg, 1e-6 * (double)(hs.t_f32[1] - hs.t_f32[0]));
        if (!hs.pool_overflow) break;
        if (attempt >= 2) return bail(fail(QP_ENOMEM, "the entry pool kept overflowing"));
        // grow the pool (and the result's entry part) to what was asked for, and run again
        ++C->pool_retries;
        const int64_t need = (int64_t)(hs.pool_used * 5 / 4) + 4096;
        C->pool_hint = need;
        if ((e = C->pool.ensure(sizeof(int2) * need)) != cudaSuccess ||
            (f64 && (e = C->pool64.ensure(sizeof(double) * need)) != cudaSuccess))
            return bail(fail(QP_ENOMEM, "pool allocation (%lld entries) failed", (long long)need));
        C->pool_cap = (int64_t)(C->pool.bytes / sizeof(int2));
        if (f64) C->pool_cap = std::min<int64_t>(C->pool_cap, (int64_t)(C->pool64.bytes / sizeof(double)));
        call_cap = std::min<int64_t>(C->pool_cap, need);
    }

    qp_result* r = (qp_result*)calloc(1, sizeof(qp_result));
    if (!r) return bail(fail(QP_ENOMEM, "host allocation failed"));
    fill_result(r, own, lay, k, P, pl->n_rows, nnz_cap_of(), f64, prm->precision, C->device);
    r->nnz = nnz;
    r->threshold_used = ebudget ? hs.theta_used : (f64 ? prm->threshold : (double)(float)prm->threshold);
    r->n_fallback = f64 ? 0 : hs.n_fallback;
    for (int i = 0; i < 10; ++i) r->guard_info[i] = hs.diag[i];
    // device time of the FP32 and FP64 kernels (their own time stamps), of
    // everything else, and of the whole call (events around it)
    auto span = [](const unsigned long long* t) {
        return (t[0] > 0 && t[1] > t[0]) ? 1e-6 * (double)(t[1] - t[0]) : 0.0;
    };
    float ms = 0, k32 = 0, k64 = 0;
    cudaEventElapsedTime(&ms, C->ev[0], C->ev[4]);
    r->kernel_ms[0] = span(hs.t_f32);
    r->kernel_ms[1] = span(hs.t_f64);
    if (timed_call && cudaEventElapsedTime(&k32, C->ev[1], C->ev[2]) == cudaSuccess &&
        cudaEventElapsedTime(&k64, C->ev[2], C->ev[3]) == cudaSuccess) {
        r->kernel_ms[0] = k32;
        r->kernel_ms[1] = k64;
    }
    r->kernel_ms[3] = ms;
    r->kernel_ms[2] = std::max(0.0, (double)ms - r->kernel_ms[0] - r->kernel_ms[1]);
    if (!out_on_device) {
        int rc = to_host(r, st);
        if (rc != QP_OK) { qp_result_free(r); return rc; }
    }
    *out = r;
    return QP_OK;
}

// Runs the enqueue function as one CUDA graph on stream st.  When the key
// (every pointer, size and launch shape the sequence uses) equals the one of
// the context's executable graph, that graph is relaunched as it is.  Else the
// sequence is captured, the executable graph is updated in place when the
// topology is unchanged, or instantiated anew, and launched.  A stream that is
// already capturing gets the plain sequence.
cudaError_t launch_graph(Context* C, cudaStream_t st, const GraphKey& key,
                         const std::function<cudaError_t()>& enqueue) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return enqueue();
    }
    if (C->gexec && C->gkey_valid && memcmp(&key, &C->gkey, sizeof key) == 0) {
        ++C->graph_relaunches;
        return cudaGraphLaunch(C->gexec, st);
    }
    C->gkey_valid = false;
    ++C->graph_captures;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t ee = enqueue();
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(st, &g);
    if (ee != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return ee != cudaSuccess ? ee : e;
    }
    if (C->gexec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(C->gexec, g, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(C->gexec);
            C->gexec = nullptr;
        }
    }
    if (!C->gexec) {
        e = cudaGraphInstantiate(&C->gexec, g, 0);
        if (e != cudaSuccess) {
            C->gexec = nullptr;
            cudaGraphDestroy(g);
            return e;
        }
    }
    cudaGraphDestroy(g);
    C->gkey = key;
    C->gkey_valid = true;
    return cudaGraphLaunch(C->gexec, st);
}

namespace {
std::mutex g_host_mu;
std::multimap<size_t, void*> g_host_spare;    // pinned blocks by size
size_t g_host_spare_bytes = 0;
constexpr size_t kHostSpareCap = (size_t)8 << 30;
constexpr size_t kHostSpareCount = 16;
}  // namespace

void* take_host_block(size_t bytes, bool* pinned) {
    {
        std::lock_guard<std::mutex> g(g_host_mu);
        auto it = g_host_spare.find(bytes);
        if (it != g_host_spare.end()) {
            void* p = it->second;
            g_host_spare.erase(it);
            g_host_spare_bytes -= bytes;
            *pinned = true;
            return p;
        }
    }
    void* p = nullptr;
    if (cudaMallocHost(&p, bytes) == cudaSuccess && p) {
        *pinned = true;
        return p;
    }
    cudaGetLastError();
    *pinned = false;
    return malloc(bytes);
}

void give_host_block(void* p, size_t bytes, bool pinned) {
    if (!p) return;
    if (!pinned) { free(p); return; }
    {
        std::lock_guard<std::mutex> g(g_host_mu);
        if (g_host_spare_bytes + bytes <= kHostSpareCap && g_host_spare.size() < kHostSpareCount) {
            g_host_spare.emplace(bytes, p);
            g_host_spare_bytes += bytes;
            return;
        }
    }
    cudaFreeHost(p);
}

int to_host(qp_result* r, cudaStream_t st) {
    ResultOwner* own = (ResultOwner*)r->owner_;
    const int64_t P = r->n_pairs;
    const size_t k2 = (size_t)r->k * r->k;
    struct Part { void** field; size_t bytes; };
    Part parts[] = {
        {(void**)&r->pair_row_off, sizeof(int64_t) * (P + 1)},
        {(void**)&r->row_ptr, sizeof(int32_t) * r->n_rows},
        {(void**)&r->pair_nnz_off, sizeof(int64_t) * (P + 1)},
        {(void**)&r->col, sizeof(int32_t) * r->nnz},
        {(void**)&r->val, sizeof(float) * r->nnz},
        {(void**)&r->val64, r->val64 ? sizeof(double) * r->nnz : 0},
        {(void**)&r->dist, sizeof(float) * k2},
        {(void**)&r->dist64, sizeof(double) * k2},
        {(void**)&r->mea, sizeof(double) * P},
        {(void**)&r->log_z_hmm, sizeof(double) * P},
        {(void**)&r->log_z_pf, sizeof(double) * P},
        {(void**)&r->pair_flags, sizeof(int32_t) * P},
    };
    size_t tot = 0;
    for (auto& p : parts) tot += align256(p.bytes);
    const size_t hbytes = std::max<size_t>(tot, 64);
    bool pinned = false;
    char* h = (char*)take_host_block(hbytes, &pinned);
    if (!h) return fail(QP_ENOMEM, "host result allocation (%zu bytes) failed", tot);
    size_t o = 0;
    cudaError_t e = cudaSuccess;
    for (auto& p : parts) {
        if (*p.field) {
            if (p.bytes) {
                e = cudaMemcpyAsync(h + o, *p.field, p.bytes, cudaMemcpyDeviceToHost, st);
                if (e != cudaSuccess) break;
            }
            *p.field = h + o;
        }
        o += align256(p.bytes);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { give_host_block(h, hbytes, pinned); return cuda_fail(e, "copy result to host"); }
    if (own->dev_a || own->dev_b) {
        int rc = QP_OK;
        Context* C = get_context(own->device, &rc);
        if (C) {
            C->give_block(own->dev_a, own->bytes_a);
            C->give_block(own->dev_b, own->bytes_b);
        } else {
            if (own->dev_a) cudaFreeAsync(own->dev_a, st);
            if (own->dev_b) cudaFreeAsync(own->dev_b, st);
        }
    }
    own->dev_a = own->dev_b = nullptr;
    own->host = h;
    own->host_bytes = hbytes;
    own->host_pinned = pinned;
    own->on_device = false;
    r->on_device = 0;
    return QP_OK;
}

void free_result(qp_result* r) {
    if (!r) return;
    ResultOwner* own = (ResultOwner*)r->owner_;
    if (own) {
        if (own->dev_a || own->dev_b) {
            int cur = 0, rc = 0;
            cudaGetDevice(&cur);
            cudaSetDevice(own->device);
            Context* C = get_context(own->device, &rc);
            if (C) {
                C->give_block(own->dev_a, own->bytes_a);
                C->give_block(own->dev_b, own->bytes_b);
            } else {
                if (own->dev_a) cudaFreeAsync(own->dev_a, nullptr);
                if (own->dev_b) cudaFreeAsync(own->dev_b, nullptr);
            }
            cudaSetDevice(cur);
        }
        give_host_block(own->host, own->host_bytes, own->host_pinned);
        delete own;
    }
    free(r);
}


// ------------------------------------------------------------------ host output in ranges
// A large family asked for in host memory: its pairs are cut into G ranges of
// about equal work (the linear pair order, as qp_split_pairs), each computed
// on the device in turn; the arrays of a finished range are copied to the
// host result on a second stream while the next range computes, so that the
// copy of the sparse matrices (8 bytes an entry over the host link) overlaps
// the computation instead of following it.  The result is the one
// qp_posteriors returns in a single piece, bit for bit: a range's row
// pointers are pair-local, its pair offsets are shifted by the entries and
// rows of the ranges before it, and its distances fill its own pairs only.
constexpr double kPipeCells = 2e9;       // smallest family (cells) computed in ranges for host output
constexpr double kRangeRatio = 0.7;      // work of a range over the one before it

int host_chunks_for(const Context* C, const qp_family* f, const qp_params* prm) {
    if (prm->precision != QP_F32_SCALED || prm->entry_budget != 0 || C->tune.host_chunks == 1) return 1;
    double cells = 0.0, len_sum = 0.0, len_sq = 0.0;
    for (int a = 0; a < f->k; ++a) {
        const double L = (double)(f->offsets[a + 1] - f->offsets[a]);
        len_sum += L;
        len_sq += L * L;
    }
    cells = 0.5 * (len_sum * len_sum - len_sq);
    const int64_t P = (int64_t)f->k * (f->k - 1) / 2;
    int G = C->tune.host_chunks >= 2 ? C->tune.host_chunks
          : (cells < kPipeCells ? 1 : (int)std::min(8.0, std::max(2.0, cells / 1.5e9)));
    return (int)std::min<int64_t>(G, P);
}

int run_family_ranges(Context* C, const qp_family* f, const qp_params* prm, int G, qp_result** out) {
    const int k = f->k;
    const int64_t P = (int64_t)k * (k - 1) / 2;
    // ranges shrinking by kRangeRatio along the pair order: a range's copy
    // (about 0.7 of its compute time at C3's density) then fits under the
    // next range's compute, and the last copy, which nothing hides, is short
    std::vector<int64_t> bounds(G + 1);
    {
        std::vector<double> cum(P + 1);
        cum[0] = 0.0;
        int64_t q = 0;
        for (int a = 0; a < k; ++a)
            for (int b = a + 1; b < k; ++b, ++q)
                cum[q + 1] = cum[q] + (double)(f->offsets[a + 1] - f->offsets[a]) * (double)(f->offsets[b + 1] - f->offsets[b]);
        const double total = cum[P];
        const double norm = (1.0 - std::pow(kRangeRatio, G)) / (1.0 - kRangeRatio);
        bounds[0] = 0;
        bounds[G] = P;
        double acc = 0.0, w = 1.0;
        for (int c = 1; c < G; ++c) {
            acc += w / norm;
            w *= kRangeRatio;
            // the first boundary whose prefix work reaches the target, every range non-empty
            int64_t b = std::lower_bound(cum.begin(), cum.end(), acc * total) - cum.begin();
            b = std::max<int64_t>(b, bounds[c - 1] + 1);
            b = std::min<int64_t>(b, P - (G - c));
            bounds[c] = b;
        }
    }
    int rc = QP_OK;
    cudaError_t e;
    if (!C->copy_stream && (e = cudaStreamCreateWithFlags(&C->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "copy stream");
    // the ranges take the launch the autotuner chose for the whole family's shape
    {
        auto full = C->plan_for(k, f->offsets, &rc);
        if (!full) return rc;
        C->tune_alias = Context::tune_key(full->n_pairs, full->max_len, full->work_sum);
    }
    struct Span { int64_t rows, nnz; };
    std::vector<qp_result*> parts(G, nullptr);
    std::vector<Span> off(G + 1, Span{0, 0});
    // host result: fixed arrays exact, col / val at a capacity grown on demand
    const size_t k2 = (size_t)k * k;
    int64_t n_rows = 0;
    for (int a = 0; a < k; ++a) n_rows += (int64_t)(f->offsets[a + 1] - f->offsets[a] + 1) * (k - 1 - a);
    size_t o_pro = 0, o_rp, o_pno, o_mea, o_lh, o_lp, o_fl, o_d32, o_d64, o_col, fixed;
    {
        size_t o = 0;
        o_pro = o; o += align256(sizeof(int64_t) * (P + 1));
        o_rp = o; o += align256(sizeof(int32_t) * n_rows);
        o_pno = o; o += align256(sizeof(int64_t) * (P + 1));
        o_mea = o; o += align256(sizeof(double) * P);
        o_lh = o; o += align256(sizeof(double) * P);
        o_lp = o; o += align256(sizeof(double) * P);
        o_fl = o; o += align256(sizeof(int32_t) * P);
        o_d32 = o; o += align256(sizeof(float) * k2);
        o_d64 = o; o += align256(sizeof(double) * k2);
        o_col = o;
        fixed = o;
    }
    char* h = nullptr;
    size_t hbytes = 0;
    bool pinned = false;
    int64_t cap = 0;   // entries col / val can hold
    auto layout_bytes = [&](int64_t c) { return fixed + 2 * align256(sizeof(int32_t) * (size_t)c); };
    auto val_at = [&](char* base, int64_t c) { return base + o_col + align256(sizeof(int32_t) * (size_t)c); };
    auto cleanup = [&](int code) {
        cudaStreamSynchronize(C->copy_stream);
        for (auto* r : parts) if (r) free_result(r);
        if (h) give_host_block(h, hbytes, pinned);
        C->tune_alias = 0;
        return code;
    };
    for (int c = 0; c < G; ++c) {
        rc = run_family(C, f, prm, 1, &parts[c], bounds[c], bounds[c + 1]);
        if (rc != QP_OK) return cleanup(rc);
        qp_result* r = parts[c];
        const int64_t need = off[c].nnz + r->nnz;
        if (need > cap) {
            // first range: the entries of the whole family estimated from its
            // density per pair-cell (+12.5%); later ranges grow the block
            int64_t want = need;
            if (c == 0) {
                const double frac = (double)(bounds[1] - bounds[0]) / (double)P;
                want = (int64_t)((double)r->nnz / std::max(frac, 1e-9) * 1.125) + (1 << 20);
            } else {
                want = std::max<int64_t>(need + need / 8, (int64_t)((double)cap * 1.25));
            }
            want = ((want + (1 << 22) - 1) >> 22) << 22;   // whole 4M-entry steps: repeated calls reuse the block
            bool pin2 = false;
            const size_t nb = layout_bytes(want);
            char* h2 = (char*)take_host_block(nb, &pin2);
            if (!h2) return cleanup(fail(QP_ENOMEM, "host result allocation (%zu bytes) failed", nb));
            if (h) {
                cudaStreamSynchronize(C->copy_stream);
                memcpy(h2, h, fixed + sizeof(int32_t) * (size_t)off[c].nnz);
                memcpy(val_at(h2, want), val_at(h, cap), sizeof(float) * (size_t)off[c].nnz);
                give_host_block(h, hbytes, pinned);
            }
            h = h2; hbytes = nb; pinned = pin2; cap = want;
        }
        const int64_t Pc = r->n_pairs, p0 = bounds[c];
        cudaStream_t cs = C->copy_stream;
        struct Copy { void* dst; const void* src; size_t bytes; };
        const Copy copies[] = {
            {h + o_pro + sizeof(int64_t) * p0, r->pair_row_off, sizeof(int64_t) * (Pc + 1)},
            {h + o_rp + sizeof(int32_t) * off[c].rows, r->row_ptr, sizeof(int32_t) * r->n_rows},
            {h + o_pno + sizeof(int64_t) * p0, r->pair_nnz_off, sizeof(int64_t) * (Pc + 1)},
            {h + o_col + sizeof(int32_t) * off[c].nnz, r->col, sizeof(int32_t) * r->nnz},
            {val_at(h, cap) + sizeof(float) * off[c].nnz, r->val, sizeof(float) * r->nnz},
            {h + o_mea + sizeof(double) * p0, r->mea, sizeof(double) * Pc},
            {h + o_lh + sizeof(double) * p0, r->log_z_hmm, sizeof(double) * Pc},
            {h + o_lp + sizeof(double) * p0, r->log_z_pf, sizeof(double) * Pc},
            {h + o_fl + sizeof(int32_t) * p0, r->pair_flags, sizeof(int32_t) * Pc},
        };
        for (const Copy& x : copies)
            if (x.bytes && (e = cudaMemcpyAsync(x.dst, x.src, x.bytes, cudaMemcpyDeviceToHost, cs)) != cudaSuccess)
                return cleanup(cuda_fail(e, "copy a range of the result to host"));
        off[c + 1] = Span{off[c].rows + r->n_rows, off[c].nnz + r->nnz};
    }
    if ((e = cudaStreamSynchronize(C->copy_stream)) != cudaSuccess) return cleanup(cuda_fail(e, "copy stream"));
    C->tune_alias = 0;
    // offsets: each range's local offsets shifted by the ranges before it
    int64_t* pro = (int64_t*)(h + o_pro);
    int64_t* pno = (int64_t*)(h + o_pno);
    for (int c = 0; c < G; ++c)
        for (int64_t p = bounds[c]; p < bounds[c + 1]; ++p) { pro[p] += off[c].rows; pno[p] += off[c].nnz; }
    pro[P] = off[G].rows;
    pno[P] = off[G].nnz;
    // distances from the MEA scores: d = 1 - A / min(m, n), the kernels'
    // expression in the same FP64 operations, so the values are the same bits
    float* d32 = (float*)(h + o_d32);
    double* d64 = (double*)(h + o_d64);
    memset(d32, 0, sizeof(float) * k2);
    memset(d64, 0, sizeof(double) * k2);
    {
        const double* mea = (const double*)(h + o_mea);
        int64_t q = 0;
        for (int a = 0; a < k; ++a)
            for (int b = a + 1; b < k; ++b, ++q) {
                const int64_t la = f->offsets[a + 1] - f->offsets[a], lb = f->offsets[b + 1] - f->offsets[b];
                const double d = 1.0 - mea[q] / (double)std::min(la, lb);
                d64[(size_t)a * k + b] = d64[(size_t)b * k + a] = d;
                d32[(size_t)a * k + b] = d32[(size_t)b * k + a] = (float)d;
            }
    }
    qp_result* res = (qp_result*)calloc(1, sizeof(qp_result));
    ResultOwner* own = new ResultOwner();
    if (!res || !own) { free(res); delete own; return cleanup(fail(QP_ENOMEM, "result allocation failed")); }
    *res = *parts[0];
    res->on_device = 0;
    res->n_pairs = P;
    res->n_rows = off[G].rows;
    res->nnz = off[G].nnz;
    res->pair_row_off = pro;
    res->row_ptr = (int32_t*)(h + o_rp);
    res->pair_nnz_off = pno;
    res->col = (int32_t*)(h + o_col);
    res->val = (float*)val_at(h, cap);
    res->val64 = nullptr;
    res->dist = d32;
    res->dist64 = d64;
    res->mea = (double*)(h + o_mea);
    res->log_z_hmm = (double*)(h + o_lh);
    res->log_z_pf = (double*)(h + o_lp);
    res->pair_flags = (int32_t*)(h + o_fl);
    res->n_fallback = 0;
    for (int i = 0; i < 4; ++i) res->kernel_ms[i] = 0.0;
    bool guard = false;
    for (auto* r : parts) {
        res->n_fallback += r->n_fallback;
        for (int i = 0; i < 4; ++i) res->kernel_ms[i] += r->kernel_ms[i];
        if (!guard && r->guard_info[0]) {
            for (int i = 0; i < 12; ++i) res->guard_info[i] = r->guard_info[i];
            guard = true;
        }
    }
    own->device = C->device;
    own->on_device = false;
    own->host = h;
    own->host_bytes = hbytes;
    own->host_pinned = pinned;
    res->owner_ = own;
    h = nullptr;
    for (auto*& r : parts) { free_result(r); r = nullptr; }
    *out = res;
    return QP_OK;
}

}  // namespace qph

// ================================================================== C ABI
extern "C" {

int qp_posteriors(const qp_family* family, const qp_params* params, int32_t out_on_device,
                  qp_result** out) {
    using namespace qph;
    if (!out) return fail(QP_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate_family(family);
    if (rc != QP_OK) return rc;
    rc = validate_params(params);
    if (rc != QP_OK) return rc;
    cudaError_t e = cudaSetDevice(params->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    Context* C = get_context(params->device, &rc);
    if (!C) return rc;
    if ((rc = check_f32_lengths(C, family, params)) != QP_OK) return rc;
    std::lock_guard<std::mutex> g(C->mu);
    if (!out_on_device) {
        const int G = host_chunks_for(C, family, params);
        if (G > 1) return run_family_ranges(C, family, params, G, out);
    }
    return run_family(C, family, params, out_on_device, out);
}

int qp_posteriors_range(const qp_family* family, const qp_params* params, int64_t p_begin, int64_t p_end,
                        int32_t out_on_device, qp_result** out) {
    using namespace qph;
    if (!out) return fail(QP_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate_family(family);
    if (rc != QP_OK) return rc;
    rc = validate_params(params);
    if (rc != QP_OK) return rc;
    const int64_t P = (int64_t)family->k * (family->k - 1) / 2;
    if (!(p_begin >= 0 && p_begin < p_end && p_end <= P))
        return fail(QP_EINVAL, "pair range [%lld, %lld) is empty or outside [0, %lld)", (long long)p_begin,
                    (long long)p_end, (long long)P);
    cudaError_t e = cudaSetDevice(params->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    Context* C = get_context(params->device, &rc);
    if (!C) return rc;
    if ((rc = check_f32_lengths(C, family, params)) != QP_OK) return rc;
    std::lock_guard<std::mutex> g(C->mu);
    return run_family(C, family, params, out_on_device, out, p_begin, p_end);
}

void qp_result_free(qp_result* result) { qph::free_result(result); }

int qp_get_counter(int32_t device, const char* name, int64_t* value) {
    using namespace qph;
    if (!name || !value) return fail(QP_EINVAL, "name or value is NULL");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) { cudaGetLastError(); return fail(QP_ECUDA, "no CUDA device"); }
    if (device < 0 || device >= ndev) return fail(QP_EINVAL, "device %d does not exist", device);
    int rc = QP_OK;
    Context* C = get_context(device, &rc);
    if (!C) return rc;
    std::lock_guard<std::mutex> g(C->mu);
    const std::string n(name);
    if (n == "graph_captures") *value = C->graph_captures;
    else if (n == "graph_relaunches") *value = C->graph_relaunches;
    else if (n == "plain_calls") *value = C->plain_calls;
    else if (n == "pool_retries") *value = C->pool_retries;
    else if (n == "consistency_fma") *value = C->cons_fma;
    else if (n == "consistency_form") *value = C->cons_last_form;
    else if (n == "f32_variant") *value = C->last_variant;
    else if (n == "f32_wpp") *value = C->last_wpp;
    else if (n == "f32_warps_per_block") *value = C->last_wpb;
    else if (n == "f32_tab_copies") *value = C->last_copies;
    else if (n == "f32_max_len") *value = f32_max_len(C, 2);
    else return fail(QP_EINVAL, "unknown counter '%s'", name);
    return QP_OK;
}

int qp_set_option(int32_t device, const char* name, int64_t value) {
    using namespace qph;
    if (!name) return fail(QP_EINVAL, "name is NULL");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) { cudaGetLastError(); return fail(QP_ECUDA, "no CUDA device"); }
    if (device < 0 || device >= ndev) return fail(QP_EINVAL, "device %d does not exist", device);
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    int rc = QP_OK;
    Context* C = get_context(device, &rc);
    if (!C) return rc;
    std::lock_guard<std::mutex> g(C->mu);
    const std::string n(name);
    if (n == "variant") {
        if (value >= qpk::kF32Variants) return fail(QP_EINVAL, "variant must be < %d", qpk::kF32Variants);
        C->tune.variant = value < 0 ? -1 : (int)value;
    } else if (n == "ckpt") {
        C->tune.ckpt = value < 0 ? -1 : (value ? 1 : 0);
    } else if (n == "wpp") {
        if (value > 0 && value != 1 && value != 2) return fail(QP_EINVAL, "wpp must be 1 or 2");
        C->tune.wpp = value > 0 ? (int)value : 0;
    } else if (n == "tab_copies") {
        // emission table copies in shared memory: 1, 16 (bank-sliced), or -1 automatic
        if (value > 1 && value != qpk::kTabCopies) return fail(QP_EINVAL, "tab_copies must be 1, %d or -1", qpk::kTabCopies);
        C->tune.tab_copies = value < 0 ? -1 : (value == 0 ? -1 : (int)value);
    } else if (n == "host_chunks") {
        // host output: pair ranges (0 automatic, 1 never, n >= 2 forced, at most 16)
        C->tune.host_chunks = value > 0 ? (int)std::min<int64_t>(value, 16) : 0;
    } else if (n == "spin_limit") {
        // testing: polls of a wait for another warp's strip before the pair
        // is handed to the FP64 form (0 / -1: the default, about 4M)
        C->tune.spin_limit = value > 0 ? (int)std::min<int64_t>(value, 1 << 30) : 0;
    } else if (n == "graph") {
        C->tune.graph = value != 0;
    } else if (n == "blocks_per_sm") {
        C->tune.blocks_per_sm = value > 0 ? (int)std::min<int64_t>(value, 32) : 0;
    } else if (n == "warps_per_block") {
        if (value > 8) return fail(QP_EINVAL, "warps_per_block must be <= 8");
        C->tune.warps_per_block = value > 0 ? (int)value : 0;
    } else if (n == "scratch_bytes") {
        C->tune.scratch_bytes = value > 0 ? value : 0;
    } else if (n == "pool_entries") {
        // start the next calls from a pool of at most this many entries (the
        // pool grows when a call overflows it); 0 / -1: estimated
        C->tune.pool_entries = value > 0 ? value : 0;
        C->pool.release();
        C->pool64.release();
        C->pool_cap = 0;
        C->pool_hint = 0;
    } else if (n == "tree_form") {
        if (value > 2) return fail(QP_EINVAL, "tree_form must be 0, 1, 2 or -1");
        C->tune.tree_form = value < 0 ? -1 : (int)value;
    } else if (n == "tree_ctas") {
        if (value > 0 && (value > 16 || (value & (value - 1))))
            return fail(QP_EINVAL, "tree_ctas must be 1, 2, 4, 8 or 16");
        C->tune.tree_ctas = value > 0 ? (int)value : 0;
    } else if (n == "cons_form") {
        if (value > 1) return fail(QP_EINVAL, "cons_form must be 0, 1 or -1");
        C->tune.cons_form = value < 0 ? -1 : (int)value;
    } else if (n == "cons_wait_polls") {
        C->tune.cons_wait_polls = value > 0 ? (int)std::min<int64_t>(value, 1 << 20) : 0;
    } else if (n == "cons_stall_test") {
        C->tune.cons_stall_test = value > 0 ? 1 : 0;
    } else if (n == "cons_ctas_per_sm") {
        if (value > 2) return fail(QP_EINVAL, "cons_ctas_per_sm must be 1, 2 or 0");
        C->tune.cons_ctas_per_sm = value > 0 ? (int)value : 0;
    } else if (n == "cons_min_unit") {
        if (value > 31) return fail(QP_EINVAL, "cons_min_unit must be <= 31");
        C->tune.cons_min_unit = value > 0 ? (int)value : 0;
    } else if (n == "cons_chunk_rows") {
        C->tune.cons_chunk_rows = value > 0 ? (int)std::min<int64_t>(value, 1 << 20) : 0;
    } else {
        return fail(QP_EINVAL, "unknown option '%s'", name);
    }
    return QP_OK;
}

const char* qp_last_error(void) { return qph::last_error(); }

const char* qp_version(void) { return "qp-b300 0.1 (sm_103a)"; }

}  // extern "C"
