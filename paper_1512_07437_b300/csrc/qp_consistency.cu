// Selective consistency (paper, Methods, stage III and "Selective
// consistency"): every sparse posterior matrix S_xy is relaxed through the
// third sequences z whose tree distances to x and y both stay within T, and
// its own signal is amplified:
//     S'_xy = (2 h_xy S_xy + sum_{z in Z_xy} S_xz S_zy) / (2 + |Z_xy|),
//     Z_xy  = {z not in {x, y} : max(d_xz, d_zy) <= T},
//     h_xy  = 1 + (h - 1) min(|Z_xy|, n_max) / n_max,
// where d_xy is the number of sequences in the smallest guide-tree subtree
// holding x and y, S_yx = S_xy transposed, and the 2 counts x and y
// themselves (S_xx = I, the relaxation of ProbCons restricted to Z).  The
// result is kept sparse at the threshold.
//
// Selection without a distance matrix: with the leaves in DFS order every
// subtree is a contiguous range, and {z : d_xz <= T} is the range R_x of the
// highest ancestor of x with at most T leaves.  Two such ranges are nested
// or disjoint, so Z_xy = (R_x intersect R_y) minus {x, y} is one contiguous
// range of the DFS order.
//
// Kernels:
//   k_cons_tree       parent / size / DFS order / R_x from the guide tree's
//                     joins (one thread: O(k));
//   k_cons_tcount,    the transposed CSR of every pair (rows of b), built
//   k_cons_tscan,     row by row so each transposed row lists its entries in
//   k_cons_tfill      ascending order (deterministic);
//   k_cons_relax      a CTA per pair, warps over the rows of x: a dense
//                     accumulator row in shared memory, a Gustavson product
//                     per z with lanes over (outer entry, inner entry) pairs,
//                     then the amplified S_xy row, the scale, the threshold,
//                     and the kept entries into a pool chunk per row.  Each
//                     product (at most 1) is rounded to 32-bit fixed point
//                     (units of 2^-30) and added into a 64-bit accumulator:
//                     integer addition is associative, so the sum does not
//                     depend on the order the lanes' atomics land in
//                     (bit-reproducible results) and is exact apart from one
//                     rounding per product.  No 64-bit conversion per
//                     product: those run on B300's narrow FP64 pipe;
//   k_cons_compact    CSR of every pair from the row chunks.
#include "../../include/qp.h"
#include "qp_host.h"

#include <cmath>
#include <cstring>
#include <vector>

namespace {

constexpr unsigned FULLM = 0xffffffffu;
constexpr int kConsWarps = 8;                 // warps per CTA (fewer for very long sequences)
constexpr int kConsMaxLen = 25600;            // accumulator row of one warp: 200 KB of shared memory
constexpr float kFix = 1073741824.0f;         // 2^30: fixed-point unit of a product (products are <= 1)
constexpr float kUnfix = 1.0f / 1073741824.0f;

// 64-bit fixed-point sum (>= 0) to float: two 32-bit conversions in a fixed
// order (deterministic), then the unit
__device__ __forceinline__ float unfix(unsigned long long a) {
    if (a == 0ull) return 0.0f;
    return (__uint2float_rn((unsigned)(a >> 32)) * 4294967296.0f + __uint2float_rn((unsigned)a)) * kUnfix;
}
constexpr size_t kConsSmem = 200 * 1024;

struct ConsIn {
    // input CSR (rows of a for pair (a, b))
    const int64_t* pro;     // [P + 1] first row pointer of pair p
    const int32_t* rp;      // [n_rows]
    const int64_t* pno;     // [P + 1] first entry of pair p
    const int32_t* col;
    const float* val;
    // transposed CSR (rows of b for pair (a, b)), same entry offsets pno
    const int64_t* tpro;    // [P + 1]
    const int32_t* trp;     // [n_rows_t]
    // (column, value bits) of every entry, interleaved for single 8-byte
    // loads: the posteriors (fcv) and their transposes (tcv)
    const int2* fcv;
    const int2* tcv;
    const int32_t* len;     // [k]
    const int32_t* leaf_at; // [k] leaf at each DFS position
    const int32_t* pos;     // [k] DFS position of each leaf
    const int32_t* rlo;     // [k] R_x = [rlo, rhi) in DFS positions
    const int32_t* rhi;
    int k;
    int64_t P;
};

struct ConsOut {
    int2* pool;                     // (column, value bits)
    int64_t pool_cap;
    unsigned long long* pool_used;
    int32_t* overflow;
    int32_t* row_cnt;               // [n_rows] kept entries of each row
    int64_t* row_off;               // [n_rows] its chunk in the pool
    int32_t* nz;                    // [P] |Z_xy| (diagnostic)
    unsigned long long* fma;        // multiply-adds of the relaxation (all pairs)
};

__device__ __forceinline__ int64_t pidx(int a, int b, int k) {
    return (int64_t)a * k - (int64_t)a * (a + 1) / 2 + (b - a - 1);
}

// (a, b) of linear pair index p (a < b)
__device__ __forceinline__ int2 pair_of(int64_t p, int k) {
    // a = the largest a with start(a) <= p, start(a) = a k - a (a + 1) / 2
    const double kk = 2.0 * k - 1.0;
    int a = (int)floor((kk - sqrt(kk * kk - 8.0 * (double)p)) * 0.5);
    if (a < 0) a = 0;
    while (a > 0 && pidx(a, a + 1, k) > p) --a;
    while (a + 1 < k - 1 && pidx(a + 1, a + 2, k) <= p) ++a;
    const int b = (int)(p - pidx(a, a + 1, k)) + a + 1;
    return make_int2(a, b);
}

// ---------------------------------------------------------------- guide tree ranges

__global__ void k_cons_tree(const int32_t* merges, int k, int32_t* parent, int32_t* size, int32_t* left,
                            int32_t* right, int32_t* stack, int32_t* leaf_at, int32_t* pos, int32_t* first,
                            int32_t* status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int nn = 2 * k - 1;
    for (int v = 0; v < nn; ++v) { parent[v] = -1; size[v] = v < k ? 1 : 0; left[v] = right[v] = -1; }
    for (int s = 0; s < k - 1; ++s) {
        const int a = merges[2 * s], b = merges[2 * s + 1], v = k + s;
        if (a < 0 || a >= v || b < 0 || b >= v || a == b || parent[a] >= 0 || parent[b] >= 0) {
            *status = 1;                // not a valid join sequence
            return;
        }
        parent[a] = parent[b] = v;
        left[v] = a;
        right[v] = b;
        size[v] = size[a] + size[b];
    }
    // DFS from the root, left subtree first: the leaf order, and the first
    // DFS position of every node (a node's leaves follow it at once)
    int top = 0, np = 0;
    stack[top++] = nn - 1;
    while (top > 0) {
        const int v = stack[--top];
        first[v] = np;
        if (v < k) {
            leaf_at[np] = v;
            pos[v] = np++;
        } else {
            stack[top++] = right[v];
            stack[top++] = left[v];
        }
    }
    if (np != k) *status = 1;
}

// R_x = the leaf range of the highest ancestor of x with at most T leaves
// (thread per leaf; at most T steps up once T < k)
__global__ void k_cons_ranges(int k, int T, const int32_t* parent, const int32_t* size, const int32_t* first,
                              int32_t* rlo, int32_t* rhi, const int32_t* status) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= k) return;
    if (*status) { rlo[x] = rhi[x] = 0; return; }
    int a = x;
    while (parent[a] >= 0 && size[parent[a]] <= T) a = parent[a];
    rlo[x] = first[a];
    rhi[x] = first[a] + size[a];
}

// ---------------------------------------------------------------- transposed CSR

// row lengths of the transposed matrices (warp per pair)
__global__ void k_cons_tcount(ConsIn in, int32_t* tcnt) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= in.P) return;
    const int2 ab = pair_of(p, in.k);
    const int m = in.len[ab.x], n = in.len[ab.y];
    int32_t* c = tcnt + in.tpro[p];
    for (int j = lane; j <= n; j += 32) c[j] = 0;
    __syncwarp();
    const int32_t* rp = in.rp + in.pro[p];
    const int32_t* col = in.col + in.pno[p];
    // one row at a time: within a row the columns are distinct
    for (int i = 0; i < m; ++i) {
        for (int e = rp[i] + lane; e < rp[i + 1]; e += 32) c[col[e]] += 1;
        __syncwarp();
    }
}

// exclusive scan of each pair's transposed row lengths into row pointers
__global__ void k_cons_tscan(ConsIn in, int32_t* tcnt, int32_t* trp) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= in.P) return;
    const int2 ab = pair_of(p, in.k);
    const int n = in.len[ab.y];
    const int64_t o = in.tpro[p];
    int carry = 0;
    for (int j0 = 0; j0 <= n; j0 += 32) {
        const int j = j0 + lane;
        const int v = j < n ? tcnt[o + j] : 0;
        int incl = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int u = __shfl_up_sync(FULLM, incl, d);
            if (lane >= d) incl += u;
        }
        if (j <= n) {
            trp[o + j] = carry + incl - v;
            tcnt[o + j] = carry + incl - v;     // becomes the fill cursor
        }
        carry += __shfl_sync(FULLM, incl, 31);
    }
}

// entries in transposed order: rows of a visited in order, so each
// transposed row lists its entries by ascending row of a
__global__ void k_cons_tfill(ConsIn in, int32_t* cursor, int2* tcv) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= in.P) return;
    const int2 ab = pair_of(p, in.k);
    const int m = in.len[ab.x];
    int32_t* cur = cursor + in.tpro[p];
    const int32_t* rp = in.rp + in.pro[p];
    const int64_t base = in.pno[p];
    for (int i = 0; i < m; ++i) {
        for (int e = rp[i] + lane; e < rp[i + 1]; e += 32) {
            const int j = in.col[base + e];
            const int q = cur[j]++;
            tcv[base + q] = make_int2(i, __float_as_int(in.val[base + e]));
        }
        __syncwarp();
    }
}

// the posteriors' (column, value) pairs interleaved
__global__ void k_cons_interleave(const int32_t* col, const float* val, int64_t nnz, int2* cv) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        cv[e] = make_int2(col[e], __float_as_int(val[e]));
}

// ---------------------------------------------------------------- relaxation

// rows of S_ab (a != b): the stored pair when a < b, else the transposed one
struct MatRef {
    const int32_t* rp;
    const int2* cv;     // (column, value bits)
};

__device__ __forceinline__ MatRef mat_of(const ConsIn& in, int a, int b) {
    MatRef M;
    if (a < b) {
        const int64_t p = pidx(a, b, in.k);
        M.rp = in.rp + in.pro[p];
        M.cv = in.fcv + in.pno[p];
    } else {
        const int64_t p = pidx(b, a, in.k);
        M.rp = in.trp + in.tpro[p];
        M.cv = in.tcv + in.pno[p];
    }
    return M;
}

// the products of one outer entry (t, vk) with row t of B added into acc:
// the row's entries are loaded eight at a time before their atomics
__device__ __forceinline__ unsigned long long add_products(unsigned long long* acc, const MatRef& B, int t,
                                                           float vk) {
    const int b0 = B.rp[t], nb = B.rp[t + 1] - b0;
    for (int f0 = 0; f0 < nb; f0 += 8) {
        int2 cv[8];
#pragma unroll
        for (int f = 0; f < 8; ++f) cv[f] = f0 + f < nb ? B.cv[b0 + f0 + f] : make_int2(-1, 0);
#pragma unroll
        for (int f = 0; f < 8; ++f)
            if (cv[f].x >= 0)
                atomicAdd(&acc[cv[f].x], (unsigned long long)(unsigned)__float2int_rn(vk * __int_as_float(cv[f].y)));
    }
    return (unsigned long long)nb;
}

// the selected z of a pair and the bases of its two matrices (S_xz rows of
// x, S_zy rows of z), built once per pair in shared memory
struct ZRef {
    MatRef A;
    MatRef B;
};
constexpr int kZTab = 256;                  // table entries (T = 200 selects at most 198 z)

__global__ void __launch_bounds__(kConsWarps * 32, 4) k_cons_relax(ConsIn in, ConsOut out, int nwarps, int acc_len,
                                                                    float h, int n_max, float theta,
                                                                    const int32_t* tree_status) {
    extern __shared__ unsigned long long acc_all[];
    __shared__ ZRef ztab[kZTab];
    const int64_t p = blockIdx.x;
    if (*tree_status) return;                       // not a tree: the call fails
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int2 xy = pair_of(p, in.k);
    const int x = xy.x, y = xy.y;
    const int m = in.len[x], n = in.len[y];
    unsigned long long* acc = acc_all + (size_t)wid * acc_len;
    // Z_xy: the intersection of the two ranges, x and y left out
    const int lo = max(in.rlo[x], in.rlo[y]), hi = min(in.rhi[x], in.rhi[y]);
    int nz = max(0, hi - lo);
    const int px = in.pos[x], py = in.pos[y];
    if (nz > 0 && px >= lo && px < hi) --nz;
    if (nz > 0 && py >= lo && py < hi) --nz;
    const float hxy = 1.0f + (h - 1.0f) * (float)min(nz, n_max) / (float)n_max;
    const float self = 2.0f * hxy;
    const float scale = 1.0f / (2.0f + (float)nz);
    if (threadIdx.x == 0) out.nz[p] = nz;
    // the table of selected z (in DFS order), when they fit
    const bool tab = nz <= kZTab;
    if (tab) {
        // position of DFS slot u in the table: u - lo, less one once past x or y
        for (int u = lo + threadIdx.x; u < hi; u += blockDim.x) {
            const int z = in.leaf_at[u];
            if (z == x || z == y) continue;
            const int slot = u - lo - (px >= lo && px < u ? 1 : 0) - (py >= lo && py < u ? 1 : 0);
            ztab[slot].A = mat_of(in, x, z);
            ztab[slot].B = mat_of(in, z, y);
        }
    }
    __syncthreads();
    if (wid >= nwarps) return;
    const int64_t row_base = in.pro[p];
    const MatRef own = mat_of(in, x, y);
    const int g = lane >> 2, q = lane & 3;          // 8 groups (one z each) of 4 lanes (outer entries)
    unsigned long long fmas = 0;
    for (int i = wid; i < m; i += nwarps) {
        for (int j = lane; j < n; j += 32) acc[j] = 0ull;
        __syncwarp();
        if (tab) {
            for (int z0 = 0; z0 < nz; z0 += 8) {
                const int zi = z0 + g;
                if (zi < nz) {
                    const ZRef Z = ztab[zi];
                    const int a0 = Z.A.rp[i], na = Z.A.rp[i + 1] - a0;
                    for (int e = q; e < na; e += 4) {
                        const int2 tv = Z.A.cv[a0 + e];
                        fmas += add_products(acc, Z.B, tv.x, __int_as_float(tv.y) * kFix);
                    }
                }
            }
        } else {
            // many z (T well above 200): the same sums, z walked in DFS order
            for (int u0 = lo; u0 < hi; u0 += 8) {
                const int u = u0 + g;
                if (u < hi) {
                    const int z = in.leaf_at[u];
                    if (z != x && z != y) {
                        const MatRef A = mat_of(in, x, z);
                        const MatRef B = mat_of(in, z, y);
                        const int a0 = A.rp[i], na = A.rp[i + 1] - a0;
                        for (int e = q; e < na; e += 4) {
                            const int2 tv = A.cv[a0 + e];
                            fmas += add_products(acc, B, tv.x, __int_as_float(tv.y) * kFix);
                        }
                    }
                }
            }
        }
        __syncwarp();
        // every lane turns its own slots into float bits (in place), then the
        // amplified own signal, then the scale and the threshold
        for (int j = lane; j < n; j += 32) acc[j] = (unsigned long long)__float_as_uint(unfix(acc[j]));
        __syncwarp();
        const int s0 = own.rp[i], sn = own.rp[i + 1] - s0;
        for (int f = lane; f < sn; f += 32) {       // the own row's columns are distinct
            const int2 cv = own.cv[s0 + f];
            acc[cv.x] = (unsigned long long)__float_as_uint(__uint_as_float((unsigned)acc[cv.x]) +
                                                             self * __int_as_float(cv.y));
        }
        __syncwarp();
        int kept = 0;
        for (int j0 = 0; j0 < n; j0 += 32) {
            const int j = j0 + lane;
            const bool keep = j < n && __uint_as_float((unsigned)acc[j]) * scale >= theta;
            kept += __popc(__ballot_sync(FULLM, keep));
        }
        unsigned long long off = 0;
        if (lane == 0 && kept > 0) off = atomicAdd(out.pool_used, (unsigned long long)kept);
        off = __shfl_sync(FULLM, off, 0);
        const bool fits = (int64_t)off + kept <= out.pool_cap;
        if (!fits && lane == 0) atomicExch(out.overflow, 1);
        if (lane == 0) {
            out.row_cnt[row_base + i] = kept;
            out.row_off[row_base + i] = (int64_t)off;
        }
        if (fits) {
            int w = 0;
            const unsigned below = (1u << lane) - 1u;
            for (int j0 = 0; j0 < n; j0 += 32) {
                const int j = j0 + lane;
                const float v = j < n ? __uint_as_float((unsigned)acc[j]) * scale : 0.0f;
                const bool keep = j < n && v >= theta;
                const unsigned mk = __ballot_sync(FULLM, keep);
                if (keep) out.pool[off + w + __popc(mk & below)] = make_int2(j, __float_as_int(v));
                w += __popc(mk);
            }
        }
        __syncwarp();
    }
    for (int d = 16; d > 0; d >>= 1) fmas += __shfl_xor_sync(FULLM, fmas, d);
    if (lane == 0 && fmas) atomicAdd(out.fma, fmas);
}

// CSR of every pair from the row chunks (warp per pair): row pointers from
// the row counts, then the chunks in row order
__global__ void k_cons_compact(ConsIn in, ConsOut out, const int64_t* pair_nnz_off, int32_t* row_ptr,
                               int32_t* col, float* val) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= in.P || *out.overflow) return;
    const int2 ab = pair_of(p, in.k);
    const int m = in.len[ab.x];
    const int64_t ro = in.pro[p], base = pair_nnz_off[p];
    int carry = 0;
    for (int r0 = 0; r0 <= m; r0 += 32) {
        const int r = r0 + lane;
        const int v = r < m ? out.row_cnt[ro + r] : 0;
        int incl = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int u = __shfl_up_sync(FULLM, incl, d);
            if (lane >= d) incl += u;
        }
        if (r <= m) row_ptr[ro + r] = carry + incl - v;
        carry += __shfl_sync(FULLM, incl, 31);
    }
    __syncwarp();
    for (int r = 0; r < m; ++r) {
        const int beg = row_ptr[ro + r], cnt = out.row_cnt[ro + r];
        const int64_t src = out.row_off[ro + r];
        for (int e = lane; e < cnt; e += 32) {
            const int2 t = out.pool[src + e];
            col[base + beg + e] = t.x;
            val[base + beg + e] = __int_as_float(t.y);
        }
    }
}

// per-pair entry counts (for the scan of the pair offsets)
__global__ void k_cons_pair_nnz(ConsIn in, ConsOut out, int64_t* pair_nnz) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= in.P) return;
    const int2 ab = pair_of(p, in.k);
    const int m = in.len[ab.x];
    const int64_t ro = in.pro[p];
    long long s = 0;
    for (int r = lane; r < m; r += 32) s += out.row_cnt[ro + r];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(FULLM, s, d);
    if (lane == 0) pair_nnz[p] = s;
}

}  // namespace

extern "C" int qp_consistency(const qp_result* post, const int64_t* offsets, const int32_t* merges,
                              int32_t merges_on_device, const qp_consistency_params* cp, int32_t out_on_device,
                              qp_result** out) {
    using namespace qph;
    if (!out) return fail(QP_EINVAL, "consistency: out is NULL");
    *out = nullptr;
    if (!post || !offsets || !merges || !cp) return fail(QP_EINVAL, "consistency: a pointer is NULL");
    const int k = post->k;
    if (k < 2 || k > 16384) return fail(QP_EINVAL, "consistency: k must be in [2, 16384] (got %d)", k);
    if (!(cp->T >= 0 && cp->n_max >= 1 && cp->h >= 1.0 && std::isfinite(cp->h) && cp->threshold > 0.0 &&
          cp->threshold <= 1.0))
        return fail(QP_EINVAL, "consistency: need T >= 0, n_max >= 1, finite h >= 1 and 0 < threshold <= 1");
    if (offsets[0] != 0) return fail(QP_EINVAL, "consistency: offsets[0] must be 0");
    std::vector<int32_t> lens(k);
    int64_t rows = 0, rows_t = 0;
    int maxlen = 0;
    for (int a = 0; a < k; ++a) {
        const int64_t L = offsets[a + 1] - offsets[a];
        if (L < 1 || L > kConsMaxLen)
            return fail(QP_EINVAL, "consistency: sequence %d has length %lld (1 .. %d)", a, (long long)L,
                        kConsMaxLen);
        lens[a] = (int32_t)L;
        maxlen = std::max(maxlen, (int)L);
    }
    const int64_t P = (int64_t)k * (k - 1) / 2;
    std::vector<int64_t> tpro(P + 1);
    {
        int64_t p = 0;
        for (int a = 0; a < k; ++a)
            for (int b = a + 1; b < k; ++b) {
                rows += lens[a] + 1;
                tpro[p++] = rows_t;
                rows_t += lens[b] + 1;
            }
        tpro[P] = rows_t;
    }
    if (post->n_pairs != P || post->n_rows != rows)
        return fail(QP_EINVAL, "consistency: the posteriors do not match the offsets (pairs or rows differ)");
    const int device = post->device;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    int rc = QP_OK;
    Context* C = get_context(device, &rc);
    if (!C) return rc;
    std::lock_guard<std::mutex> lock(C->cons_mu);
    cudaStream_t st;
    if ((e = call_stream(C, nullptr, &st)) != cudaSuccess) return cuda_fail(e, "consistency: stream order");
    const int64_t nnz_in = post->nnz;

    // ---- device workspace
    size_t sz = 0;
    auto take = [&](size_t bytes) { const size_t o = sz; sz += align256(std::max<size_t>(bytes, 16)); return o; };
    const bool host_in = !post->on_device;
    const size_t o_pro = host_in ? take(sizeof(int64_t) * (P + 1)) : 0;
    const size_t o_rp = host_in ? take(sizeof(int32_t) * rows) : 0;
    const size_t o_pno = host_in ? take(sizeof(int64_t) * (P + 1)) : 0;
    const size_t o_col = host_in ? take(sizeof(int32_t) * nnz_in) : 0;
    const size_t o_val = host_in ? take(sizeof(float) * nnz_in) : 0;
    const size_t o_tpro = take(sizeof(int64_t) * (P + 1));
    const size_t o_trp = take(sizeof(int32_t) * rows_t);
    const size_t o_tcur = take(sizeof(int32_t) * rows_t);
    const size_t o_tcv = take(sizeof(int2) * nnz_in);
    const size_t o_fcv = take(sizeof(int2) * nnz_in);
    const size_t o_len = take(sizeof(int32_t) * k);
    const size_t o_mg = take(sizeof(int32_t) * 2 * (k - 1));
    const size_t o_tree = take(sizeof(int32_t) * (size_t)(2 * k - 1) * 6 + sizeof(int32_t) * k * 4);
    const size_t o_cnt = take(sizeof(int32_t) * rows);
    const size_t o_off = take(sizeof(int64_t) * rows);
    const size_t o_nz = take(sizeof(int32_t) * P);
    const size_t o_pn = take(sizeof(int64_t) * P);
    const size_t o_st = take(64);
    if ((e = C->cons_ws.ensure(sz)) != cudaSuccess) return fail(QP_ENOMEM, "consistency: %zu bytes of workspace", sz);
    char* W = (char*)C->cons_ws.ptr;
    ConsIn in;
    in.k = k;
    in.P = P;
    in.pro = host_in ? (const int64_t*)(W + o_pro) : post->pair_row_off;
    in.rp = host_in ? (const int32_t*)(W + o_rp) : post->row_ptr;
    in.pno = host_in ? (const int64_t*)(W + o_pno) : post->pair_nnz_off;
    in.col = host_in ? (const int32_t*)(W + o_col) : post->col;
    in.val = host_in ? (const float*)(W + o_val) : post->val;
    in.tpro = (const int64_t*)(W + o_tpro);
    in.trp = (const int32_t*)(W + o_trp);
    in.tcv = (const int2*)(W + o_tcv);
    in.fcv = (const int2*)(W + o_fcv);
    in.len = (const int32_t*)(W + o_len);
    int32_t* tr = (int32_t*)(W + o_tree);
    const int nn = 2 * k - 1;
    int32_t *parent = tr, *size = tr + nn, *left = tr + 2 * nn, *right = tr + 3 * nn, *stack = tr + 4 * nn,
            *first = tr + 5 * nn, *leaf_at = tr + 6 * nn, *pos = leaf_at + k, *rlo = pos + k, *rhi = rlo + k;
    in.leaf_at = leaf_at;
    in.pos = pos;
    in.rlo = rlo;
    in.rhi = rhi;
    int32_t* d_status = (int32_t*)(W + o_st);
    if ((e = C->cons_h.ensure(64)) != cudaSuccess) return fail(QP_ENOMEM, "consistency: pinned staging");
    int32_t* h_status = (int32_t*)C->cons_h.ptr;

    auto up = [&](size_t o, const void* src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(W + o, src, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
    };
    if ((e = cudaMemsetAsync(d_status, 0, 64, st)) != cudaSuccess ||
        (e = up(o_tpro, tpro.data(), sizeof(int64_t) * (P + 1))) != cudaSuccess ||
        (e = up(o_len, lens.data(), sizeof(int32_t) * k)) != cudaSuccess ||
        (e = cudaMemcpyAsync(W + o_mg, merges, sizeof(int32_t) * 2 * (k - 1),
                             merges_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
        return cuda_fail(e, "consistency: inputs");
    if (host_in &&
        ((e = up(o_pro, post->pair_row_off, sizeof(int64_t) * (P + 1))) != cudaSuccess ||
         (e = up(o_rp, post->row_ptr, sizeof(int32_t) * rows)) != cudaSuccess ||
         (e = up(o_pno, post->pair_nnz_off, sizeof(int64_t) * (P + 1))) != cudaSuccess ||
         (e = up(o_col, post->col, sizeof(int32_t) * nnz_in)) != cudaSuccess ||
         (e = up(o_val, post->val, sizeof(float) * nnz_in)) != cudaSuccess))
        return cuda_fail(e, "consistency: posterior upload");

    if (!C->cons_ev[0] && ((e = cudaEventCreate(&C->cons_ev[0])) != cudaSuccess ||
                           (e = cudaEventCreate(&C->cons_ev[1])) != cudaSuccess))
        return cuda_fail(e, "consistency: events");
    cudaEvent_t ev0 = C->cons_ev[0], ev1 = C->cons_ev[1];
    cudaEventRecord(ev0, st);
    const int warp_blocks = (int)((P * 32 + 255) / 256);
    k_cons_tree<<<1, 32, 0, st>>>((const int32_t*)(W + o_mg), k, parent, size, left, right, stack, leaf_at,
                                  pos, first, d_status);
    k_cons_ranges<<<(k + 127) / 128, 128, 0, st>>>(k, cp->T, parent, size, first, rlo, rhi, d_status);
    k_cons_tcount<<<warp_blocks, 256, 0, st>>>(in, (int32_t*)(W + o_tcur));
    k_cons_tscan<<<warp_blocks, 256, 0, st>>>(in, (int32_t*)(W + o_tcur), (int32_t*)(W + o_trp));
    k_cons_tfill<<<warp_blocks, 256, 0, st>>>(in, (int32_t*)(W + o_tcur), (int2*)(W + o_tcv));
    k_cons_interleave<<<(int)std::min<int64_t>(8 * C->sm_count, (nnz_in + 255) / 256 + 1), 256, 0, st>>>(
        in.col, in.val, nnz_in, (int2*)(W + o_fcv));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "consistency: set-up kernels");

    // ---- relaxation into the pool (grown and run again when it overflows)
    const int nwarps =
        (int)std::max<size_t>(1, std::min<size_t>(kConsWarps, kConsSmem / (sizeof(unsigned long long) * maxlen)));
    const int acc_len = maxlen;
    const size_t smem = sizeof(unsigned long long) * (size_t)nwarps * acc_len;
    if ((e = cudaFuncSetAttribute(k_cons_relax, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kConsSmem)) !=
        cudaSuccess)
        return cuda_fail(e, "consistency: shared memory size");
    ConsOut o;
    o.overflow = d_status + 1;
    o.pool_used = (unsigned long long*)(d_status + 2);
    o.row_cnt = (int32_t*)(W + o_cnt);
    o.row_off = (int64_t*)(W + o_off);
    o.nz = (int32_t*)(W + o_nz);
    o.fma = (unsigned long long*)(d_status + 4);
    int64_t cap = std::max<int64_t>(C->cons_pool_hint, 2 * nnz_in + 4096);
    int64_t used = 0;
    for (int attempt = 0;; ++attempt) {
        if ((e = C->cons_pool.ensure(sizeof(int2) * cap)) != cudaSuccess)
            return fail(QP_ENOMEM, "consistency: entry pool of %lld entries", (long long)cap);
        o.pool = (int2*)C->cons_pool.ptr;
        o.pool_cap = (int64_t)(C->cons_pool.bytes / sizeof(int2));
        if ((e = cudaMemsetAsync(d_status + 1, 0, 20, st)) != cudaSuccess) return cuda_fail(e, "consistency");
        k_cons_relax<<<(unsigned)P, nwarps * 32, smem, st>>>(in, o, nwarps, acc_len, (float)cp->h, cp->n_max,
                                                             (float)cp->threshold, d_status);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "consistency: k_cons_relax");
        if ((e = cudaMemcpyAsync(h_status, d_status, 24, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_fail(e, "consistency");
        if (h_status[0]) return fail(QP_EINVAL, "consistency: merges are not a valid join sequence of k leaves");
        memcpy(&used, h_status + 2, sizeof used);
        if (!h_status[1]) {
            unsigned long long f = 0;
            memcpy(&f, h_status + 4, sizeof f);
            std::lock_guard<std::mutex> g(C->mu);
            C->cons_fma = (int64_t)f;
            break;
        }
        if (attempt >= 2) return fail(QP_ENOMEM, "consistency: the entry pool kept overflowing");
        cap = used + used / 4 + 4096;
        C->cons_pool_hint = cap;
    }

    // ---- the result: pair layout of the posteriors, entries of the relaxation
    ResultOwner* own = new ResultOwner();
    own->device = device;
    const ResultLayout lay(P, rows, k);
    if ((e = C->take_block(&own->dev_a, lay.bytes, st)) != cudaSuccess) {
        delete own;
        return fail(QP_ENOMEM, "consistency: result allocation");
    }
    own->bytes_a = lay.bytes;
    own->bytes_b = std::max<size_t>(ResultLayout::entry_bytes(used, false), 256);
    if ((e = C->take_block(&own->dev_b, own->bytes_b, st)) != cudaSuccess) {
        C->give_block(own->dev_a, own->bytes_a);
        delete own;
        return fail(QP_ENOMEM, "consistency: result allocation");
    }
    qp_result* r = (qp_result*)calloc(1, sizeof(qp_result));
    if (!r) return fail(QP_ENOMEM, "host allocation failed");
    fill_result(r, own, lay, k, P, rows, used, false, QP_F32_SCALED, device);
    const cudaMemcpyKind kind = post->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t k2 = (size_t)k * k;
    int64_t* pn = (int64_t*)(W + o_pn);
    if ((e = cudaMemcpyAsync(r->pair_row_off, in.pro, sizeof(int64_t) * (P + 1), cudaMemcpyDeviceToDevice, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(r->dist, post->dist, sizeof(float) * k2, kind, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(r->dist64, post->dist64, sizeof(double) * k2, kind, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(r->mea, post->mea, sizeof(double) * P, kind, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(r->log_z_hmm, post->log_z_hmm, sizeof(double) * P, kind, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(r->log_z_pf, post->log_z_pf, sizeof(double) * P, kind, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(r->pair_flags, post->pair_flags, sizeof(int32_t) * P, kind, st)) != cudaSuccess) {
        qp_result_free(r);
        return cuda_fail(e, "consistency: result copies");
    }
    k_cons_pair_nnz<<<warp_blocks, 256, 0, st>>>(in, o, pn);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = qpk::launch_scan_nnz(pn, P, r->pair_nnz_off, st)) != cudaSuccess) {
        qp_result_free(r);
        return cuda_fail(e, "consistency: pair offsets");
    }
    k_cons_compact<<<warp_blocks, 256, 0, st>>>(in, o, r->pair_nnz_off, r->row_ptr, r->col, r->val);
    cudaEventRecord(ev1, st);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess) {
        qp_result_free(r);
        return cuda_fail(e, "consistency");
    }
    r->nnz = used;
    r->threshold_used = (double)(float)cp->threshold;
    float ms = 0;
    cudaEventElapsedTime(&ms, ev0, ev1);
    r->kernel_ms[0] = ms;          // transpose, relaxation and assembly (the last attempt's relaxation)
    r->kernel_ms[3] = ms;
    if (!out_on_device) {
        rc = to_host(r, st);
        if (rc != QP_OK) { qp_result_free(r); return rc; }
    }
    *out = r;
    return QP_OK;
}
