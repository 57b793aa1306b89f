// Allocation-free entry point: one pair through the FP32 posterior kernel with
// all scratch memory taken from a fixed array that lives in this library's
// device image.  No cudaMalloc, cudaFree or allocating library call is made.
#include "../../include/qp.h"
#include "qp_host.h"
#include "qp_internal.h"

#include <cstring>
#include <mutex>

namespace {

using namespace qpk;

constexpr int kSMaxLen = QP_STATIC_MAX_LEN;
constexpr int kSCap = kSMaxLen + 1;                               // staging capacity per row, worst case
constexpr int kSStrips = (kSMaxLen + 1 + kStripRows - 1) / kStripRows;
constexpr int kSChunks = (kSMaxLen + 32 + kC - 1) / kC;

constexpr size_t al(size_t v) { return (v + 255) & ~(size_t)255; }

// Fixed layout of the scratch array (worst-case sizes for m, n <= kSMaxLen).
constexpr size_t oConsts = 0;
constexpr size_t oRaw = oConsts + al(sizeof(Consts));
constexpr size_t oStatus = oRaw + al(sizeof(RawParams));
constexpr size_t oFam = oStatus + al(sizeof(Status));
constexpr size_t oSmall = oFam + al(sizeof(FamDesc));
constexpr size_t oCodes = oSmall + al(1024);
constexpr size_t oRowCnt = oCodes + al(2 * kSMaxLen);
constexpr size_t oBst = oRowCnt + al(sizeof(int32_t) * (kSMaxLen + 1));
constexpr size_t oBex = oBst + al(sizeof(float2) * ((size_t)kSStrips * kStripRows * (kSMaxLen + 32) +
                                                    (size_t)kD_ring * kWarp * kRmax));
constexpr size_t oBnd = oBex + al(sizeof(int2) * (size_t)kSStrips * kSChunks * 32);
constexpr size_t oBck = oBnd + al(sizeof(float4) * 2 * (size_t)(kSMaxLen + 1));
constexpr size_t oStg = oBck + al(sizeof(float4) * 2 * (size_t)(kSMaxLen + 1));
constexpr size_t oPool = oStg + al(sizeof(int2) * (size_t)kWarp * 4 * group_capacity(kSMaxLen, kSCap));
constexpr size_t kSBytes = oPool + al(sizeof(int2) * (size_t)kSMaxLen * kSCap);

// Small per-call tables, copied from the host in one piece (offset oSmall).
struct SmallTables {
    int2 items[1];
    int2 pairs[1];
    int2 fallback[1];
    int32_t pair_flags[1];
    int64_t seq_off[3];
    int64_t row_off[2];
    int64_t strip_off[2];
    int64_t chunk_off[kSStrips];
    int64_t pair_nnz[1];
    int64_t pair_nnz_off[2];
    double seq_logq[2];
    double mea[1];
    double logz_h[1];
    double logz_p[1];
    float dist[4];
    double dist64[4];
};
static_assert(sizeof(SmallTables) <= 1024, "small tables overflow their slot");

// The scratch itself: one copy per device that loads the library.
static __device__ __align__(256) unsigned char g_static_scratch[kSBytes];

std::mutex g_setup_mu;
void* g_scratch_addr[128] = {};

// Device address of the scratch array on the current device (set up once per
// device; the host-side symbol is only a stand-in for it).
int scratch_address(int device, unsigned char** out) {
    if (device < 0 || device >= 128) return qph::fail(QP_EINVAL, "device %d out of range", device);
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return qph::cuda_fail(e, "cudaGetSymbolAddress of the static scratch array");
        }
        g_scratch_addr[device] = p;
    }
    *out = (unsigned char*)g_scratch_addr[device];
    return QP_OK;
}

// Puts the caller's current device back when the call returns.
struct DeviceRestore {
    int dev = -1;
    DeviceRestore() {
        if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); dev = -1; }
    }
    ~DeviceRestore() {
        if (dev >= 0) cudaSetDevice(dev);
    }
};

}  // namespace

extern "C" int qp_pair_posteriors_static(const uint8_t* residues, int32_t m, int32_t n,
                                         const qp_params* params, int32_t* row_ptr, int32_t* col,
                                         float* val, int64_t nnz_capacity, double* pair_out,
                                         int64_t* nnz_out) {
    using namespace qph;
    if (nnz_out) *nnz_out = 0;
    DeviceRestore restore;
    int rc = validate_params(params);
    if (rc != QP_OK) return rc;
    if (params->precision != QP_F32_SCALED)
        return fail(QP_EINVAL, "qp_pair_posteriors_static runs the FP32 form only");
    if (m < 1 || n < 1 || m > kSMaxLen || n > kSMaxLen)
        return fail(QP_EINVAL, "qp_pair_posteriors_static takes 1 <= m, n <= %d (got m = %d, n = %d); "
                    "use qp_posteriors for longer sequences", kSMaxLen, m, n);
    if (!residues || !row_ptr || !pair_out || !nnz_out || nnz_capacity < 0 ||
        (nnz_capacity > 0 && (!col || !val)))
        return fail(QP_EINVAL, "qp_pair_posteriors_static: a required pointer is NULL");
    cudaError_t e = cudaSetDevice(params->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    unsigned char* S = nullptr;
    rc = scratch_address(params->device, &S);
    if (rc != QP_OK) return rc;
    cudaStream_t st = (cudaStream_t)params->stream;

    Consts* cst = (Consts*)(S + oConsts);
    Status* status = (Status*)(S + oStatus);
    FamDesc* fam = (FamDesc*)(S + oFam);
    SmallTables* sm = (SmallTables*)(S + oSmall);
    uint8_t* codes = (uint8_t*)(S + oCodes);
    const int ns = (m + 1 + kStripRows - 1) / kStripRows;
    const int cap = row_capacity(params, m > n ? m : n);

    // host images of the small tables and of the family descriptor
    SmallTables h;
    memset(&h, 0, sizeof h);
    h.items[0] = make_int2(0, 0);
    h.pairs[0] = make_int2(0, 1);
    h.seq_off[0] = 0; h.seq_off[1] = m; h.seq_off[2] = (int64_t)m + n;
    h.row_off[0] = 0; h.row_off[1] = m + 1;
    h.strip_off[0] = 0; h.strip_off[1] = ns;
    FamDesc fd;
    memset(&fd, 0, sizeof fd);
    fd.codes = codes;
    fd.seq_off = sm->seq_off;
    fd.seq_logq = sm->seq_logq;
    fd.pairs = sm->pairs;
    fd.pair_row_off = sm->row_off;
    fd.pair_strip_off = sm->strip_off;
    fd.k = 2;
    fd.row_cnt = (int32_t*)(S + oRowCnt);
    fd.chunk_off = sm->chunk_off;
    fd.pair_nnz = sm->pair_nnz;
    fd.mea = sm->mea;
    fd.logz_h = sm->logz_h;
    fd.logz_p = sm->logz_p;
    fd.dist = sm->dist;
    fd.dist64 = sm->dist64;
    fd.pair_flags = sm->pair_flags;
    fd.pool_used = &status->pool_used;
    fd.pool_base = 0;
    fd.pool_cap = (int64_t)kSMaxLen * kSCap;
    fd.n_done = nullptr;

    // the array keeps the previous call's contents: every table that is read
    // before it is written, and every counter, is rewritten here
    if ((e = cudaMemcpyAsync(sm, &h, sizeof h, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(fam, &fd, sizeof fd, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(status, 0, sizeof(Status), st)) != cudaSuccess)
        return cuda_fail(e, "qp_pair_posteriors_static: set-up copies");

    RawParams raw;
    make_raw(params, &raw);
    if ((e = launch_setup(&raw, (RawParams*)(S + oRaw), cst, st)) != cudaSuccess) return cuda_fail(e, "k_setup");
    if ((e = launch_encode(residues, codes, (int64_t)m + n, sm->seq_off, 2, sm->seq_logq, cst, status,
                           st)) != cudaSuccess)
        return cuda_fail(e, "k_encode");

    Problem Pb;
    memset(&Pb, 0, sizeof Pb);
    make_coef(params, &Pb.cf);
    Pb.cst = cst;
    Pb.fams = fam;
    Pb.items = sm->items;
    Pb.n_work = 1;
    Pb.cap = cap;
    Pb.pool = (int2*)(S + oPool);
    Pb.pool64 = nullptr;
    Pb.status = status;
    Pb.fallback = sm->fallback;
    Pb.bst = (float2*)(S + oBst); Pb.bst_stride = 0;
    Pb.bex = (int2*)(S + oBex); Pb.bex_stride = 0;
    Pb.bnd = (float4*)(S + oBnd); Pb.bnd_stride = 0;
    Pb.bck = (float4*)(S + oBck); Pb.bck_stride = 0;
    Pb.wpp = 1;
    Pb.stg = (int2*)(S + oStg); Pb.stg_stride = 0;
    Pb.f64_all = 0;
    Pb.max_len = m > n ? m : n;
    if ((e = launch_posterior_f32(Pb, 1, 1, st)) != cudaSuccess) return cuda_fail(e, "k_posterior_f32");

    Status hs;
    if ((e = cudaMemcpyAsync(&hs, status, sizeof hs, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "k_posterior_f32");
    if (hs.bad_residue)
        return fail(QP_EINVAL, "%s", qph::alphabet_error(params->alphabet));
    if (hs.stage_overflow || hs.pool_overflow)
        return fail(QP_ECUDA, "internal: static scratch entry capacity exceeded");
    if (hs.n_fallback > 0)
        return fail(QP_ENOMEM, "the pair tripped an FP32 range guard; its FP64 recomputation needs more "
                    "scratch than this entry point holds (use qp_posteriors)");
    const int64_t nnz = (int64_t)hs.pool_used;
    *nnz_out = nnz;
    if (nnz > nnz_capacity)
        return fail(QP_EINVAL, "output capacity %lld is too small: the pair has %lld entries",
                    (long long)nnz_capacity, (long long)nnz);
    if ((e = launch_scan_nnz(sm->pair_nnz, 1, sm->pair_nnz_off, st)) != cudaSuccess ||
        (e = launch_compact(sm->pairs, sm->seq_off, sm->row_off, sm->strip_off, fd.row_cnt, sm->chunk_off,
                            Pb.pool, nullptr, 1, sm->pair_nnz_off, row_ptr, col, val, nullptr, st)) != cudaSuccess)
        return cuda_fail(e, "CSR assembly");
    // pair_out = (MEA score, distance, log Z_hmm, log Z_pf)
    if ((e = cudaMemcpyAsync(pair_out + 0, sm->mea, sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(pair_out + 1, sm->dist64 + 1, sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(pair_out + 2, sm->logz_h, sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(pair_out + 3, sm->logz_p, sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "qp_pair_posteriors_static: outputs");
    return QP_OK;
}
