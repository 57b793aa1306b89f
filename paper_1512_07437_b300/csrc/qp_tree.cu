// Guide tree by weighted UPGMA (paper, Methods, stage II: the distances of
// stage I feed weighted UPGMA, after Sneath and Sokal).
//
// Weighted UPGMA (WPGMA): join the two clusters at the smallest distance; the
// distance from the joined cluster to any other is the mean of the distances
// from its two parts, whatever their sizes.  Clusters live in slots 0..k-1
// (slot i starts as leaf i); joining slots i < j puts the new cluster in
// slot i and empties slot j.  Ties: the smallest distance, then the smallest
// i, then the smallest j.  All arithmetic is FP64 and each new distance is
// one rounded operation pair ((d_ix + d_jx) * 0.5), so the tree is
// bit-identical to any FP64 implementation of the same rule.
//
// Device layout: a working copy D of the k x k matrix, kept symmetric and
// made from the caller's upper triangle (k_tree_mirror, 32 x 32 tiles), and
// per slot the minimum of its row over the live columns to its right with
// the column where it is reached (smallest column on ties).  k_tree_rows
// sets those (a warp per row); k_tree_join runs all k - 1 joins in one
// block: an argmin over the row minima; the averaging of row i with row j,
// which also yields row i's new minimum; and a re-scan of only the rows whose
// minimum pointed at i or j -- every other row can only improve, through
// column i.  The per-slot state sits in shared memory when it fits.
#include "../../include/qp.h"
#include "qp_host.h"

#include <cfloat>
#include <vector>

namespace {

constexpr int kMaxThreads = 1024;
constexpr int kRowWarps = 8;              // warps per block of k_tree_rows
constexpr int kSmemSlots = 8192;          // per-slot state in shared memory up to this k
constexpr int kSlotBytes = 8 + 4 + 4 + 4 + 1;

struct TreeWork {
    const double* in;   // caller's k x k matrix (upper triangle read)
    double* D;          // [k * k] symmetric working copy
    double* rmin;       // [k] row minimum over live columns to the right (DBL_MAX: none)
    int* ridx;          // [k] its column (-1: none, or slot empty)
    int* cid;           // [k] id of the cluster in the slot
    int* list;          // [k] rows to re-scan
    unsigned char* alive;
    int32_t* merges;    // [k - 1][2]
    double* heights;    // [k - 1]
    int* status;        // 0: ok
    int k;
    int smem_state;     // per-slot state in shared memory (k <= kSmemSlots)
};

__device__ __forceinline__ bool less_pair(double v, int i, double bv, int bi) {
    return v < bv || (v == bv && i < bi);
}

// (value, index) minimum over a warp; (DBL_MAX, -1) is the empty element.
__device__ __forceinline__ void warp_argmin(double& v, int& i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, v, o);
        const int oi = __shfl_down_sync(0xffffffffu, i, o);
        if (oi >= 0 && (i < 0 || less_pair(ov, oi, v, i))) { v = ov; i = oi; }
    }
}

// Minimum of row r over live columns c > r (smallest c on ties), by one warp;
// loads are issued four at a time.  D is written by the same kernel, so it is
// read through the coherent path (no __restrict__, no read-only cache).
__device__ void scan_row(const double* D, const unsigned char* alive, int k, int r, int lane,
                         double* rmin, int* ridx) {
    const double* row = D + (size_t)r * k;
    double bv = DBL_MAX;
    int bc = -1;
    for (int c0 = r + 1 + lane; c0 < k; c0 += 128) {
        double v[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = c0 + 32 * u;
            ok[u] = c < k && alive[c];
            v[u] = ok[u] ? row[c] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (ok[u] && (bc < 0 || less_pair(v[u], c0 + 32 * u, bv, bc))) { bv = v[u]; bc = c0 + 32 * u; }
    }
    warp_argmin(bv, bc);
    if (lane == 0) {
        rmin[r] = bc < 0 ? DBL_MAX : bv;
        ridx[r] = bc;
    }
}

// D[i][j] = D[j][i] = in[min(i,j)][max(i,j)], D[i][i] = 0; a 32 x 32 tile per
// block of 32 x 8 threads, read through shared memory so both halves stay
// coalesced.
__global__ void k_tree_mirror(TreeWork w) {
    __shared__ double S[32][33];
    const int ty = blockIdx.y, tx = blockIdx.x;
    const int sy = min(ty, tx), sx = max(ty, tx);
    const int k = w.k;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int i = sy * 32 + r, j = sx * 32 + threadIdx.x;
        S[r][threadIdx.x] = (i < k && j < k) ? w.in[(size_t)i * k + j] : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int c = threadIdx.x;
        const int i = ty * 32 + r, j = tx * 32 + c;
        if (i >= k || j >= k) continue;
        double v;
        if (ty < tx || (ty == tx && r < c)) v = S[r][c];
        else if (ty > tx || r > c) v = S[c][r];
        else v = 0.0;
        w.D[(size_t)i * k + j] = v;
    }
}

__global__ void k_tree_rows(TreeWork w) {
    const int r = blockIdx.x * kRowWarps + (threadIdx.x >> 5);
    if (r < w.k) {
        // every slot is live before the first join
        const double* row = w.D + (size_t)r * w.k;
        const int lane = threadIdx.x & 31;
        double bv = DBL_MAX;
        int bc = -1;
        for (int c = r + 1 + lane; c < w.k; c += 32) {
            const double v = row[c];
            if (bc < 0 || less_pair(v, c, bv, bc)) { bv = v; bc = c; }
        }
        warp_argmin(bv, bc);
        if (lane == 0) {
            w.rmin[r] = bc < 0 ? DBL_MAX : bv;
            w.ridx[r] = bc;
        }
    }
}

__global__ void __launch_bounds__(kMaxThreads) k_tree_join(TreeWork w) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_v[32];
    __shared__ int s_i[32];
    __shared__ int s_a, s_b, s_n;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nt = blockDim.x, nw = nt >> 5;
    const int k = w.k;
    double* D = w.D;
    double* rmin = w.rmin;
    int* ridx = w.ridx;
    int* cid = w.cid;
    int* list = w.list;
    unsigned char* alive = w.alive;
    if (w.smem_state) {
        rmin = (double*)smem;
        ridx = (int*)(rmin + k);
        cid = ridx + k;
        list = cid + k;
        alive = (unsigned char*)(list + k);
        for (int r = tid; r < k; r += nt) {
            rmin[r] = w.rmin[r];
            ridx[r] = w.ridx[r];
        }
    }
    for (int r = tid; r < k; r += nt) {
        cid[r] = r;
        alive[r] = 1;
    }
    __syncthreads();
    for (int s = 0; s < k - 1; ++s) {
        // 1. the pair to join: the smallest row minimum, smallest slot on ties
        double bv = DBL_MAX;
        int br = -1;
        for (int r = tid; r < k; r += nt) {
            const int c = ridx[r];
            if (c >= 0 && (br < 0 || less_pair(rmin[r], r, bv, br))) { bv = rmin[r]; br = r; }
        }
        warp_argmin(bv, br);
        if (lane == 0) { s_v[wid] = bv; s_i[wid] = br; }
        __syncthreads();
        if (wid == 0) {
            bv = lane < nw ? s_v[lane] : DBL_MAX;
            br = lane < nw ? s_i[lane] : -1;
            warp_argmin(bv, br);
            if (lane == 0) {
                // at least two slots are live, so the smallest live slot has a
                // live column to its right; a = -1 would be an internal error
                const int a = br;
                if (a < 0) {
                    *w.status = 1;
                } else {
                    const int b = ridx[a];
                    w.merges[2 * s] = cid[a];
                    w.merges[2 * s + 1] = cid[b];
                    w.heights[s] = bv * 0.5;
                    cid[a] = k + s;
                    alive[b] = 0;
                    ridx[b] = -1;
                    rmin[b] = DBL_MAX;
                    s_b = b;
                }
                s_a = a;
                s_n = 0;
            }
        }
        __syncthreads();
        const int a = s_a, b = s_b;
        if (a < 0) break;
        // 2. distances of the joined cluster (the mean of its two parts), the
        // new minimum of row a, and the row minima that column a or b moves
        const double* Ra = D + (size_t)a * k;
        const double* Rb = D + (size_t)b * k;
        double mv = DBL_MAX;
        int mc = -1;
        for (int x = tid; x < k; x += nt) {
            if (!alive[x] || x == a) continue;
            const double v = (Ra[x] + Rb[x]) * 0.5;
            D[(size_t)a * k + x] = v;
            D[(size_t)x * k + a] = v;
            if (x > a) {
                if (mc < 0 || less_pair(v, x, mv, mc)) { mv = v; mc = x; }
                if (x < b && ridx[x] == b) list[atomicAdd(&s_n, 1)] = x;
            } else {
                const int c = ridx[x];
                if (c == a || c == b) {
                    list[atomicAdd(&s_n, 1)] = x;
                } else if (less_pair(v, a, rmin[x], c)) {
                    rmin[x] = v;
                    ridx[x] = a;
                }
            }
        }
        warp_argmin(mv, mc);
        if (lane == 0) { s_v[wid] = mv; s_i[wid] = mc; }
        __syncthreads();
        if (wid == 0) {
            mv = lane < nw ? s_v[lane] : DBL_MAX;
            mc = lane < nw ? s_i[lane] : -1;
            warp_argmin(mv, mc);
            if (lane == 0) {
                rmin[a] = mc < 0 ? DBL_MAX : mv;
                ridx[a] = mc;
            }
        }
        // 3. re-scan the rows whose minimum was in column a or b
        const int n = s_n;
        for (int q = wid; q < n; q += nw) scan_row(D, alive, k, list[q], lane, rmin, ridx);
        __syncthreads();
    }
}

int join_threads(int k) {
    const int t = (k + 31) / 32 * 32;
    return t < 64 ? 64 : (t > kMaxThreads ? kMaxThreads : t);
}

}  // namespace

extern "C" int qp_guide_tree(const double* dist, int32_t k, int32_t on_device, int32_t device, void* stream,
                             int32_t* merges, double* heights) {
    using namespace qph;
    if (k < 2 || k > kMaxK) return fail(QP_EINVAL, "guide tree: k must be in [2, %d] (got %d)", kMaxK, k);
    if (!dist || !merges || !heights) return fail(QP_EINVAL, "guide tree: a pointer is NULL");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) { cudaGetLastError(); return fail(QP_ECUDA, "no CUDA device"); }
    if (device < 0 || device >= ndev) return fail(QP_EINVAL, "device %d does not exist", device);
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    int rc = QP_OK;
    Context* C = get_context(device, &rc);
    if (!C) return rc;
    cudaStream_t st;
    if ((e = call_stream(C, stream, &st)) != cudaSuccess) return cuda_fail(e, "guide tree: stream order");
    const size_t kk = (size_t)k * k;
    int tree_smem;
    {
        std::lock_guard<std::mutex> g(C->mu);
        tree_smem = C->tune.tree_smem;
    }
    const bool small = k <= kSmemSlots && tree_smem != 0;
    const size_t smem = small ? (size_t)k * kSlotBytes : 0;
    e = cudaFuncSetAttribute(k_tree_join, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemSlots * kSlotBytes);
    if (e != cudaSuccess) return cuda_fail(e, "guide tree: shared memory size");
    size_t sz = 0;
    const size_t o_D = sz;   sz += align256(sizeof(double) * kk);
    const size_t o_in = sz;  sz += on_device ? 0 : align256(sizeof(double) * kk);
    const size_t o_mn = sz;  sz += align256(sizeof(double) * k);
    const size_t o_ix = sz;  sz += align256(sizeof(int) * k);
    const size_t o_ci = sz;  sz += small ? 0 : align256(sizeof(int) * k);
    const size_t o_li = sz;  sz += small ? 0 : align256(sizeof(int) * k);
    const size_t o_al = sz;  sz += small ? 0 : align256(k);
    const size_t o_mg = sz;  sz += on_device ? 0 : align256(sizeof(int32_t) * 2 * (k - 1));
    const size_t o_h = sz;   sz += on_device ? 0 : align256(sizeof(double) * (k - 1));
    const size_t o_st = sz;  sz += align256(sizeof(int));
    char* m = nullptr;
    if ((e = cudaMallocAsync((void**)&m, sz, st)) != cudaSuccess) {
        cudaGetLastError();
        return fail(QP_ENOMEM, "guide tree: %zu bytes of workspace", sz);
    }
    TreeWork w;
    w.k = k;
    w.smem_state = small ? 1 : 0;
    w.D = (double*)(m + o_D);
    w.in = on_device ? dist : (const double*)(m + o_in);
    w.rmin = (double*)(m + o_mn);
    w.ridx = (int*)(m + o_ix);
    w.cid = small ? nullptr : (int*)(m + o_ci);
    w.list = small ? nullptr : (int*)(m + o_li);
    w.alive = small ? nullptr : (unsigned char*)(m + o_al);
    w.merges = on_device ? merges : (int32_t*)(m + o_mg);
    w.heights = on_device ? heights : (double*)(m + o_h);
    w.status = (int*)(m + o_st);
    int h_status = 0;
    e = cudaMemsetAsync(w.status, 0, sizeof(int), st);
    if (e == cudaSuccess && !on_device)
        e = cudaMemcpyAsync((void*)w.in, dist, sizeof(double) * kk, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        const int tiles = (k + 31) / 32;
        k_tree_mirror<<<dim3(tiles, tiles), dim3(32, 8), 0, st>>>(w);
        k_tree_rows<<<(k + kRowWarps - 1) / kRowWarps, kRowWarps * 32, 0, st>>>(w);
        k_tree_join<<<1, join_threads(k), smem, st>>>(w);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !on_device) {
        e = cudaMemcpyAsync(merges, w.merges, sizeof(int32_t) * 2 * (k - 1), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(heights, w.heights, sizeof(double) * (k - 1), cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, w.status, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(m, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "guide tree");
    if (h_status != 0) return fail(QP_ECUDA, "guide tree: internal error (no pair to join)");
    return QP_OK;
}
