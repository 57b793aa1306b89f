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
//   k_cons_tree,      parent / size / DFS order / R_x from the guide tree's
//   k_cons_ranges     joins (one thread: O(k)), then R_x per leaf;
//   k_cons_tcount,    the transposed CSR of every pair (rows of b); the fill
//   k_cons_tscan,     walks the rows in order, so each transposed row lists
//   k_cons_tfill      its entries in ascending order (deterministic);
//   k_cons_interleave the entries as (row << 16 | column, value) pairs;
//   staged form (default, T <= 256):
//   k_cons_stats      the largest value and row sum (the fixed-point unit);
//   k_cons_bands      per row, the column band of the rows up to / from it;
//   k_cons_relax_staged  a CTA per row chunk of a pair: a producer warp
//                     stages the selected z (A's chunk entries, the band of
//                     B's rows they reach) by TMA bulk copies into two
//                     buffers, each refilled as soon as every warp is done
//                     with it; the products go into a dense 32-bit
//                     fixed-point accumulator in shared memory (see the
//                     kernel);
//   row form (T > 256, or values too large for the staged unit):
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
//   k_cons_pair_nnz,  CSR of every pair from the row chunks.
//   k_cons_compact
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
    // (row << 16 | column, value bits) of every entry, interleaved for single
    // 8-byte loads: the posteriors (fcv) and their transposes (tcv)
    const int2* fcv;
    const int2* tcv;
    // column bands of the rows (staged form): for row r of a matrix,
    // (largest column of rows 0..r) << 16 | (smallest column of rows r..end),
    // indexed like rp / trp
    const int32_t* fband;
    const int32_t* tband;
    const int32_t* len;     // [k]
    const int2* pairs;      // [P] (a, b) of pair p
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


// an entry's row and column in one word (both below 2^16)
__device__ __forceinline__ int pack_key(int row, int col) { return (row << 16) | col; }
__device__ __forceinline__ int key_col(int key) { return key & 0xffff; }
__device__ __forceinline__ int key_row(int key) { return (int)((unsigned)key >> 16); }

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
    const int2 ab = in.pairs[p];
    const int m = in.len[ab.x], n = in.len[ab.y];
    int32_t* c = tcnt + in.tpro[p];
    for (int j = lane; j <= n; j += 32) c[j] = 0;
    __syncwarp();
    const int32_t* rp = in.rp + in.pro[p];
    const int32_t* col = in.col + in.pno[p];
    // every entry at once: integer counts do not depend on the order
    const int nnz = rp[m];
    for (int e = lane; e < nnz; e += 32) atomicAdd(&c[col[e]], 1);
}

// exclusive scan of each pair's transposed row lengths into row pointers
__global__ void k_cons_tscan(ConsIn in, int32_t* tcnt, int32_t* trp) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= in.P) return;
    const int2 ab = in.pairs[p];
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
    const int2 ab = in.pairs[p];
    const int m = in.len[ab.x];
    int32_t* cur = cursor + in.tpro[p];
    const int32_t* rp = in.rp + in.pro[p];
    const int64_t base = in.pno[p];
    for (int i = 0; i < m; ++i) {
        for (int e = rp[i] + lane; e < rp[i + 1]; e += 32) {
            const int j = in.col[base + e];
            const int q = cur[j]++;
            tcv[base + q] = make_int2(pack_key(j, i), __float_as_int(in.val[base + e]));
        }
        __syncwarp();
    }
}

// the posteriors' entries as (key, value bits) pairs, key = row << 16 |
// column (lengths are below 2^16), for single 8-byte loads that carry
// both indices (warp per pair)
__global__ void k_cons_interleave(ConsIn in, int2* cv) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= in.P) return;
    const int2 ab = in.pairs[p];
    const int m = in.len[ab.x];
    const int32_t* rp = in.rp + in.pro[p];
    const int64_t base = in.pno[p];
    // a lane per row, 32 rows at a time (rows are short)
    for (int i = lane; i < m; i += 32)
        for (int e = rp[i]; e < rp[i + 1]; ++e)
            cv[base + e] = make_int2(pack_key(i, in.col[base + e]), __float_as_int(in.val[base + e]));
}

// ---------------------------------------------------------------- relaxation

// rows of S_ab (a != b): the stored pair when a < b, else the transposed one
struct MatRef {
    const int32_t* rp;
    const int2* cv;     // (row << 16 | column, value bits)
    const int32_t* band;
};

__device__ __forceinline__ MatRef mat_of(const ConsIn& in, int a, int b) {
    MatRef M;
    if (a < b) {
        const int64_t p = pidx(a, b, in.k);
        M.rp = in.rp + in.pro[p];
        M.cv = in.fcv + in.pno[p];
        M.band = in.fband ? in.fband + in.pro[p] : nullptr;
    } else {
        const int64_t p = pidx(b, a, in.k);
        M.rp = in.trp + in.tpro[p];
        M.cv = in.tcv + in.pno[p];
        M.band = in.tband ? in.tband + in.tpro[p] : nullptr;
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
                atomicAdd(&acc[key_col(cv[f].x)],
                          (unsigned long long)(unsigned)__float2int_rn(vk * __int_as_float(cv[f].y)));
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
    const int2 xy = in.pairs[p];
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
                        fmas += add_products(acc, Z.B, key_col(tv.x), __int_as_float(tv.y) * kFix);
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
                            fmas += add_products(acc, B, key_col(tv.x), __int_as_float(tv.y) * kFix);
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
            acc[key_col(cv.x)] = (unsigned long long)__float_as_uint(__uint_as_float((unsigned)acc[key_col(cv.x)]) +
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

// ---------------------------------------------------------------- staged form

// largest value and largest row sum of every matrix and of its transpose
// (lane per row, entries summed in order: deterministic), for the staged
// form's fixed-point unit; stats[0] / stats[1] hold float bits (values >= 0)
__global__ void k_cons_stats(ConsIn in, unsigned* stats) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= in.P) return;
    const int2 ab = in.pairs[p];
    float vmax = 0.f, smax = 0.f;
    for (int side = 0; side < 2; ++side) {
        const int rows = in.len[side ? ab.y : ab.x];
        const int32_t* rp = side ? in.trp + in.tpro[p] : in.rp + in.pro[p];
        const int2* cv = (side ? in.tcv : in.fcv) + in.pno[p];
        for (int r = lane; r < rows; r += 32) {
            float s = 0.f;
            for (int f = rp[r]; f < rp[r + 1]; ++f) {
                const float v = __int_as_float(cv[f].y);
                s += v;
                vmax = fmaxf(vmax, v);
            }
            smax = fmaxf(smax, s);
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        vmax = fmaxf(vmax, __shfl_xor_sync(FULLM, vmax, d));
        smax = fmaxf(smax, __shfl_xor_sync(FULLM, smax, d));
    }
    if (lane == 0) {
        atomicMax(&stats[0], __float_as_uint(vmax));
        atomicMax(&stats[1], __float_as_uint(smax));
    }
}

// one selected z of a (pair, row chunk): A = S_xz (rows i0 .. i1 - 1 of x)
// and the band of rows of B = S_zy those entries reach (rows bt0 .. bt1 - 1
// of z), in global memory
struct ZEnt {
    const int2* acv;        // A's entries of the chunk (keys carry their rows)
    const int32_t* brp;     // B's row pointers from row bt0
    const int2* bcv;        // B's entries from entry b0
    int na;                 // A's entries of the chunk
    int bt0, nbr;           // first row of the band, rows in it
    int b0, nb;             // first entry of the band, entries in it
};

// where the products read one z from: its staged copy in shared memory, or
// global memory for a z larger than a stage buffer; B's row pointers are
// indexed by t - bt0 and give entry numbers, its entries by number - b0
struct SView {
    const int2* acv;        // global memory (a batch of one z larger than a buffer)
    const int32_t* brp;
    const int2* bcv;
    int aoff, broff, bvoff; // byte offsets in the stage buffer (a staged batch)
    int bt0, b0;
};

struct StageCfg {
    int ztab;               // z table entries (>= the selected z of any pair)
    int slot_bytes;         // one of the two stage buffers (a multiple of 16)
    int acc_cells;          // accumulator cells (rows of the chunk x n)
    int wait_polls;         // waits on a stage buffer's barrier before the CTA gives up
    int stall_first;        // testing: the first batch's arrival is withheld (its wait runs out)
};

constexpr int kStThreads = 512;             // 16 warps: one CTA per SM (its shared memory)
constexpr int kStBatch = 32;                // z per stage buffer at most (a lane of the producer warp each)
constexpr int kMinUnit = 21;                // coarsest fixed-point unit (2^-21) the staged form accepts by default
constexpr int kStGroup = 1;                 // threads per A entry along a row of B
constexpr int kStMaxRows = 1024;            // rows of a chunk at most
constexpr int kStMinRows = 32;              // rows of the longest sequence a chunk should hold (CTAs per SM)
constexpr int kStLongRows = 16;             // below this many rows per chunk, smaller stage buffers
constexpr int kStSpin = 1 << 16;            // waits on a stage buffer's barrier before the call is failed
constexpr unsigned kStSuspendNs = 20000;    // longest suspension of one wait (ns)

// column bands of every matrix and of its transpose (warp per pair, 32
// rows at a time): band[r] = (max over rows 0..r of the last column) << 16 |
// (min over rows r..end of the first column); empty rows count as 0 / 0xffff.
// The entries of rows i0 .. i1 - 1 then lie in columns
// [band[i0] & 0xffff, band[i1 - 1] >> 16].
__global__ void k_cons_bands(ConsIn in, int32_t* fband, int32_t* tband) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= in.P) return;
    const int2 ab = in.pairs[p];
    for (int side = 0; side < 2; ++side) {
        const int rows = in.len[side ? ab.y : ab.x];
        const int32_t* rp = side ? in.trp + in.tpro[p] : in.rp + in.pro[p];
        const int2* cv = (side ? in.tcv : in.fcv) + in.pno[p];
        int32_t* band = side ? tband + in.tpro[p] : fband + in.pro[p];
        // prefix maxima of the last columns, forward
        int carry = 0;
        for (int r0 = 0; r0 < rows; r0 += 32) {
            const int r = r0 + lane;
            int v = 0;
            if (r < rows) {
                const int e0 = rp[r], e1 = rp[r + 1];
                if (e1 > e0) v = key_col(cv[e1 - 1].x);
            }
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int t = __shfl_up_sync(FULLM, v, d);
                if (lane >= d) v = max(v, t);
            }
            v = max(v, carry);
            if (r < rows) band[r] = v << 16;
            carry = __shfl_sync(FULLM, v, 31);
        }
        __syncwarp();
        // suffix minima of the first columns, backward
        carry = 0xffff;
        for (int r1 = rows; r1 > 0; r1 -= 32) {
            const int r = r1 - 1 - lane;
            int v = 0xffff;
            if (r >= 0) {
                const int e0 = rp[r], e1 = rp[r + 1];
                if (e1 > e0) v = key_col(cv[e0].x);
            }
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int t = __shfl_up_sync(FULLM, v, d);
                if (lane >= d) v = min(v, t);
            }
            v = min(v, carry);
            if (r >= 0) band[r] |= v;
            carry = __shfl_sync(FULLM, v, 31);
        }
    }
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// waits for the phase with the given parity: the thread is suspended until
// the phase completes or about kStSuspendNs pass (no busy polling)
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kStSuspendNs)
        : "memory");
    return ok != 0;
}
// TMA bulk copy global -> shared (16-byte aligned addresses, a multiple of
// 16 bytes), completing on the barrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__host__ __device__ constexpr int r16(int b) { return (b + 15) & ~15; }

// the bulk copy of [g, g + bytes): from the 16-byte boundary at or below g
// (those bytes share g's 16-byte block, so they lie in the same allocation)
// to the next one at or above g + bytes (every array read here ends at least
// 16 bytes before the end of its allocation: allocations are padded to 256
// bytes); returns the copy's size, *head = the offset of g in it
__device__ __forceinline__ int bulk_span(const void* g, int bytes, int* head) {
    const uintptr_t a = (uintptr_t)g;
    *head = (int)(a & 15);
    return bytes > 0 ? r16(*head + bytes) : 0;
}

// Relaxation of rows i0 .. i1 - 1 of one pair (a work item) with the
// selected z staged in shared memory.  A producer warp's lanes take one z
// each of the next batch, a warp scan packs as many as fit into a stage
// buffer, and each lane issues the TMA bulk copies of its z (A's entries of
// the chunk, B's row pointers and entries), completing on the buffer's
// barrier; a z larger than a buffer is read from global memory.  Two
// buffers: the next batch lands while this one is multiplied.  Warp 0
// issues the first two batches; after that the last warp to finish a batch
// issues the batch after next into its buffer, so no warp waits at a
// CTA-wide barrier between batches (a warp waits only for a batch to land).
// The batch's
// A entries (t, v) are numbered through, G threads per entry (the key of an
// entry holds its row, so no search is needed); the threads of an entry run
// along row t of B and add v * S_zy(t, j) into the chunk's dense
// accumulator as 32-bit fixed point in units of 2^-u: u is the largest unit
// with (selected z bound) x (largest value) x (largest row sum) x 2^u <=
// 2^31, so no sum can overflow, and integer atomics keep the result
// independent of their order (bit-reproducible).  Then, per row, the
// amplified own signal, the scale and the threshold; one pool reservation
// for the chunk's kept entries.
template <int G, int MINB>
__global__ void __launch_bounds__(kStThreads, MINB) k_cons_relax_staged(ConsIn in, ConsOut out, const int4* __restrict__ work,
                                                                    StageCfg sc, float h, int n_max, float theta, int nzb,
                                                                    const unsigned* __restrict__ stats, int min_unit,
                                                                    int32_t* wide, int32_t* stage_err,
                                                                    const int32_t* tree_status) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned long long red[kStThreads / 32];
    __shared__ unsigned long long s_base;
    __shared__ __align__(8) unsigned long long bars[2];
    __shared__ int bcount[2];
    __shared__ int bglob[2];                        // the batch is one z read from global memory
    __shared__ int bnext[2];                        // next A entry of the batch a warp takes
    __shared__ int bps[2][kStBatch + 1];            // first A entry of each z of a batch
    __shared__ int s_nissued;                       // batches issued so far
    __shared__ int bdone[2];                        // warps done with the buffer's current batch
    __shared__ int s_zq;                            // first z not yet issued
    __shared__ int s_bail;                          // a stage wait ran out: every warp leaves
    __shared__ int s_clo, s_chi;                    // columns the chunk's sums can reach
    if (*tree_status) return;
    // a CTA whose stage wait ran out has failed the call: the rest leave at once
    if (*(volatile int32_t*)stage_err) return;
    if (smem_u32(smem) & 15) {                       // bulk copies need 16-byte aligned buffers
        if (threadIdx.x == 0) atomicExch(stage_err, 1);
        return;
    }
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nwarps = nthr >> 5;
    // the fixed-point unit (the same in every CTA)
    // a cell's sum: at most nzb selected z, each adding at most (largest
    // value) x (largest row sum), plus the amplified own value (<= 2 h V)
    const float V = __uint_as_float(stats[0]);
    const float bound = (float)nzb * V * __uint_as_float(stats[1]) + 2.0f * h * V;
    int u = 30;
    if (bound > 0.f) {
        if (!(bound <= 1e30f)) u = -1;
        else { int ex; frexpf(bound, &ex); u = min(30, 31 - ex); }
    }
    if (u < min_unit) {
        if (tid == 0) atomicExch(wide, 1);
        return;
    }
    const float unit = ldexpf(1.f, u), inv_unit = ldexpf(1.f, -u);

    const int4 w = work[blockIdx.x];
    const int p = w.x, i0 = w.y, i1 = w.z, rc = i1 - i0;
    const int2 xy = in.pairs[p];
    const int x = xy.x, y = xy.y;
    const int n = in.len[y];
    const int lo = max(in.rlo[x], in.rlo[y]), hi = min(in.rhi[x], in.rhi[y]);
    int nz = max(0, hi - lo);
    const int px = in.pos[x], py = in.pos[y];
    if (nz > 0 && px >= lo && px < hi) --nz;
    if (nz > 0 && py >= lo && py < hi) --nz;
    const float hxy = 1.0f + (h - 1.0f) * (float)min(nz, n_max) / (float)n_max;
    const float self = 2.0f * hxy;
    const float scale = 1.0f / (2.0f + (float)nz);
    if (tid == 0 && i0 == 0) out.nz[p] = nz;

    ZEnt* zt = (ZEnt*)smem;
    SView* views = (SView*)(smem + sizeof(ZEnt) * sc.ztab);
    unsigned char* slots = (unsigned char*)(views + 2 * kStBatch);
    unsigned* acc = (unsigned*)(slots + 2 * sc.slot_bytes);
    int* rcnt = (int*)(acc + sc.acc_cells);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        bnext[0] = bnext[1] = 0;
        bdone[0] = bdone[1] = 0;
        s_nissued = 0;
        s_bail = 0;
        const MatRef own = mat_of(in, x, y);
        s_clo = own.band[i0] & 0xffff;
        s_chi = own.band[i1 - 1] >> 16;
    }
    int cmn = 0x7fffffff, cmx = -1;                  // columns of this thread's staged bands
    for (int v = lo + tid; v < hi; v += nthr) {
        const int z = in.leaf_at[v];
        if (z == x || z == y) continue;
        const int slot = v - lo - (px >= lo && px < v ? 1 : 0) - (py >= lo && py < v ? 1 : 0);
        const MatRef A = mat_of(in, x, z), B = mat_of(in, z, y);
        const int a0 = A.rp[i0], na = A.rp[i1] - a0;
        ZEnt e;
        e.acv = A.cv + a0;
        e.na = na;
        e.bt0 = 0; e.nbr = 0; e.b0 = 0; e.nb = 0;
        if (na > 0) {
            const int t0 = A.band[i0] & 0xffff, t1 = (A.band[i1 - 1] >> 16) + 1;
            e.bt0 = t0; e.nbr = t1 - t0;
            e.b0 = B.rp[t0]; e.nb = B.rp[t1] - e.b0;
            cmn = min(cmn, B.band[t0] & 0xffff);
            cmx = max(cmx, B.band[t1 - 1] >> 16);
        }
        e.brp = B.rp + e.bt0;
        e.bcv = B.cv + e.b0;
        zt[slot] = e;
    }
    __syncthreads();
    // the columns the chunk's sums can reach: those of its own rows and of
    // every staged band of B (nothing outside them is zeroed or scanned)
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        cmn = min(cmn, __shfl_xor_sync(FULLM, cmn, d));
        cmx = max(cmx, __shfl_xor_sync(FULLM, cmx, d));
    }
    if (lane == 0 && cmx >= 0) {
        atomicMin(&s_clo, cmn);
        atomicMax(&s_chi, cmx);
    }

    // producer (warp 0): the batch of z starting at zs into buffer s;
    // returns its size (the same in every lane).  A z larger than a buffer
    // forms a batch of its own, read from global memory.
    auto issue = [&](int zs, int s) {
        const int zi = zs + lane;
        int need = 0, na = 0, h2 = 0, h3 = 0, h4 = 0, c2 = 0, c3 = 0, c4 = 0;
        ZEnt Z = {};
        if (zi < nz) {
            Z = zt[zi];
            na = Z.na;
            c2 = bulk_span(Z.acv, Z.na * 8, &h2);
            c3 = bulk_span(Z.brp, Z.nbr > 0 ? (Z.nbr + 1) * 4 : 0, &h3);
            c4 = bulk_span(Z.bcv, Z.nb * 8, &h4);
            need = c2 + c3 + c4;
        }
        const bool glob0 = __shfl_sync(FULLM, need, 0) > sc.slot_bytes;
        int incl = need, nincl = na;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(FULLM, incl, d), tn = __shfl_up_sync(FULLM, nincl, d);
            if (lane >= d) { incl += t; nincl += tn; }
        }
        const bool fits = zi < nz && incl <= sc.slot_bytes;
        const unsigned stop = __ballot_sync(FULLM, !fits);
        const int cnt = glob0 ? 1 : (stop ? __ffs(stop) - 1 : 32);   // lanes [0, cnt) form the batch
        const int total = glob0 ? 0 : __shfl_sync(FULLM, incl, cnt - 1);
        const int off = s * sc.slot_bytes + (incl - need);
        if (lane < cnt) {
            SView v;
            v.bt0 = Z.bt0;
            v.b0 = Z.b0;
            v.acv = Z.acv; v.brp = Z.brp; v.bcv = Z.bcv;
            v.aoff = off + h2;
            v.broff = off + c2 + h3;
            v.bvoff = off + c2 + c3 + h4;
            views[s * kStBatch + lane] = v;
            bps[s][lane] = nincl - na;
            if (lane == cnt - 1) bps[s][cnt] = nincl;
        }
        if (lane == 0) { bcount[s] = cnt; bglob[s] = glob0 ? 1 : 0; ++s_nissued; }
        __syncwarp();
        const bool withhold = sc.stall_first && zs == 0;   // testing only
        if (lane == 0 && !withhold) mbar_arrive_expect_tx(&bars[s], (unsigned)total);
        __syncwarp();
        if (lane < cnt && !glob0 && !withhold) {
            unsigned char* b = slots + off;
            if (c2) bulk_g2s(b, (const unsigned char*)Z.acv - h2, c2, &bars[s]);
            if (c3) bulk_g2s(b + c2, (const unsigned char*)Z.brp - h3, c3, &bars[s]);
            if (c4) bulk_g2s(b + c2 + c3, (const unsigned char*)Z.bcv - h4, c4, &bars[s]);
        }
        return cnt;
    };

    if (wid == 0 && nz > 0) {
        int zq = issue(0, 0);
        if (zq < nz) zq += issue(zq, 1);
        if (lane == 0) s_zq = zq;
    }
    __syncthreads();
    // (a threshold that rounds to 0 in FP32 keeps every cell)
    const int clo = theta > 0.f ? max(s_clo, 0) : 0, chi = theta > 0.f ? min(s_chi, n - 1) : n - 1;
    for (int r = wid; r < rc; r += nwarps)
        for (int j = clo + lane; j <= chi; j += 32) acc[r * n + j] = 0u;
    __syncthreads();

    unsigned long long fmas = 0;
    const int lg = lane % G;
    constexpr int kGrab = 32 / G;                    // A entries a warp takes at a time
    int bail = -1;
    for (int zs = 0, b = 0; zs < nz; ++b) {
        const int s = b & 1;
        bool ok = false;
        for (int it = 0; it < sc.wait_polls && !ok; ++it) {
            ok = mbar_try_wait(&bars[s], (unsigned)((b >> 1) & 1));
            if (!ok && *(volatile int*)&s_bail) break;   // another warp gave up
        }
        ok = __all_sync(FULLM, ok);                  // one decision for the warp
        if (!ok) {
            if (lane == 0) atomicExch(&s_bail, 1);
            bail = b;
            break;
        }
        const int cnt = bcount[s];
        const bool glob = bglob[s] != 0;
        const int* ps = bps[s];
        const SView* vt = views + s * kStBatch;
        const int na_all = ps[cnt];
        // the batch's A entries, numbered through its z, taken kGrab at a
        // time by whichever warp is free
        for (;;) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&bnext[s], kGrab);
            base = __shfl_sync(FULLM, base, 0);
            if (base >= na_all) break;
            // the z holding entry `base` (ps ascending, ps[0] = 0), then this lane's
            int k = 0, hi = cnt;
            while (hi - k > 1) {
                const int mid = (k + hi) >> 1;
                if (ps[mid] <= base) k = mid; else hi = mid;
            }
            const int q = base + lane / G;
            if (q < na_all) {
                while (q >= ps[k + 1]) ++k;
                const SView v = vt[k];
                const int e = q - ps[k];
                if (glob) {
                    const int2 tv = v.acv[e];
                    const int t = key_col(tv.x) - v.bt0;
                    unsigned* accr = acc + (key_row(tv.x) - i0) * n;
                    const int b0 = v.brp[t] - v.b0, b1 = v.brp[t + 1] - v.b0;
                    const float vs = __int_as_float(tv.y) * unit;
                    if (lg == 0) fmas += (unsigned long long)(b1 - b0);
                    for (int f = b0 + lg; f < b1; f += G) {
                        const int2 jw = v.bcv[f];
                        atomicAdd(accr + key_col(jw.x), __float2uint_rn(vs * __int_as_float(jw.y)));
                    }
                } else {
                    // shared-memory loads from the stage buffer
                    const int2 tv = *(const int2*)(slots + v.aoff + 8 * e);
                    const int t = key_col(tv.x) - v.bt0;
                    unsigned* accr = acc + (key_row(tv.x) - i0) * n;
                    const int32_t* brp = (const int32_t*)(slots + v.broff);
                    const int b0 = brp[t] - v.b0, b1 = brp[t + 1] - v.b0;
                    const int2* bcv = (const int2*)(slots + v.bvoff);
                    const float vs = __int_as_float(tv.y) * unit;
                    if (lg == 0) fmas += (unsigned long long)(b1 - b0);
                    int f = b0 + lg;
                    for (; f + G < b1; f += 2 * G) {        // two loads in flight
                        const int2 jw0 = bcv[f], jw1 = bcv[f + G];
                        atomicAdd(accr + key_col(jw0.x), __float2uint_rn(vs * __int_as_float(jw0.y)));
                        atomicAdd(accr + key_col(jw1.x), __float2uint_rn(vs * __int_as_float(jw1.y)));
                    }
                    if (f < b1) {
                        const int2 jw = bcv[f];
                        atomicAdd(accr + key_col(jw.x), __float2uint_rn(vs * __int_as_float(jw.y)));
                    }
                }
            }
        }
        zs += cnt;
        // this warp is done with buffer s; the last warp to finish the batch
        // refills it with the batch after next while the others go on with
        // the next one (no CTA-wide barrier per batch).  Fences order the
        // warps' reads of the buffer before the refill's copies.
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            __threadfence_block();
            last = atomicAdd(&bdone[s], 1) == nwarps - 1;
        }
        if (__shfl_sync(FULLM, last, 0)) {
            __threadfence_block();
            const int zq = *(volatile int*)&s_zq;
            if (lane == 0) { bdone[s] = 0; bnext[s] = 0; }
            if (zq < nz) {
                __syncwarp();
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                const int c = issue(zq, s);
                if (lane == 0) s_zq = zq + c;
            }
            __syncwarp();
        }
    }
    if (__syncthreads_or(bail >= 0)) {
        // the call fails; copies still in flight land in this CTA's buffers:
        // wait (again bounded) for the last batch issued into each buffer
        // (a later batch is only issued once the earlier one has landed),
        // then leave
        if (tid == 0) {
            atomicExch(stage_err, 1);
            for (int bb = s_nissued - 1; bb >= 0 && bb >= s_nissued - 2; --bb) {
                bool done = false;
                for (int it = 0; it < sc.wait_polls && !done; ++it)
                    done = mbar_try_wait(&bars[bb & 1], (unsigned)((bb >> 1) & 1));
            }
        }
        __syncthreads();
        return;
    }

    // the amplified own signal, in the same units
    const int64_t row_base = in.pro[p];
    {
        const MatRef own = mat_of(in, x, y);
        const int oa0 = own.rp[i0], ona = own.rp[i1] - oa0;
        const float su = self * unit;
        for (int q = tid; q < ona; q += nthr) {
            const int2 tv = own.cv[oa0 + q];
            atomicAdd(acc + (key_row(tv.x) - i0) * n + key_col(tv.x), __float2uint_rn(su * __int_as_float(tv.y)));
        }
    }
    __syncthreads();
    // rows of the chunk (a warp per row): the kept entries counted
    for (int r = wid; r < rc; r += nwarps) {
        const unsigned* ar = acc + r * n;
        int kept = 0;
        for (int j0 = clo; j0 <= chi; j0 += 32) {
            const int j = j0 + lane;
            const bool keep = j <= chi && (__uint2float_rn(ar[j]) * inv_unit) * scale >= theta;
            kept += __popc(__ballot_sync(FULLM, keep));
        }
        if (lane == 0) rcnt[r] = kept;
    }
    __syncthreads();
    // one reservation in the pool for the chunk: row offsets by a scan (warp 0)
    if (wid == 0) {
        int carry = 0;
        for (int r0 = 0; r0 < rc; r0 += 32) {
            const int r = r0 + lane;
            const int c = r < rc ? rcnt[r] : 0;
            int incl = c;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int t = __shfl_up_sync(FULLM, incl, d);
                if (lane >= d) incl += t;
            }
            if (r < rc) rcnt[r] = carry + incl - c;
            carry += __shfl_sync(FULLM, incl, 31);
        }
        if (lane == 0) {
            const unsigned long long off = carry > 0 ? atomicAdd(out.pool_used, (unsigned long long)carry) : 0ull;
            const bool fits = (int64_t)off + carry <= out.pool_cap;
            if (!fits) atomicExch(out.overflow, 1);
            s_base = fits ? off : ~0ull;
        }
    }
    __syncthreads();
    const unsigned long long base = s_base;
    for (int r = wid; r < rc; r += nwarps) {
        const int i = i0 + r;
        const unsigned* ar = acc + r * n;
        const int64_t off = (int64_t)base + rcnt[r];
        int wpos = 0;
        const unsigned below = (1u << lane) - 1u;
        for (int j0 = clo; j0 <= chi; j0 += 32) {
            const int j = j0 + lane;
            const float v = j <= chi ? (__uint2float_rn(ar[j]) * inv_unit) * scale : 0.0f;
            const bool keep = j <= chi && v >= theta;
            const unsigned mk = __ballot_sync(FULLM, keep);
            if (keep && base != ~0ull) out.pool[off + wpos + __popc(mk & below)] = make_int2(j, __float_as_int(v));
            wpos += __popc(mk);
        }
        if (lane == 0) {
            out.row_cnt[row_base + i] = wpos;
            out.row_off[row_base + i] = off;
        }
    }
    // multiply-adds: one global atomic per CTA
    for (int d = 16; d > 0; d >>= 1) fmas += __shfl_xor_sync(FULLM, fmas, d);
    if (lane == 0) red[wid] = fmas;
    __syncthreads();
    if (tid == 0) {
        unsigned long long sum = 0;
        for (int q = 0; q < nwarps; ++q) sum += red[q];
        if (sum) atomicAdd(out.fma, sum);
    }
}

// CSR of every pair from the row chunks (warp per pair): row pointers from
// the row counts, then the chunks in row order
__global__ void k_cons_compact(ConsIn in, ConsOut out, const int64_t* pair_nnz_off, int32_t* row_ptr,
                               int32_t* col, float* val) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= in.P || *out.overflow) return;
    const int2 ab = in.pairs[p];
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
    // a lane per row, 32 rows at a time (rows are short)
    for (int r = lane; r < m; r += 32) {
        const int beg = row_ptr[ro + r], cnt = out.row_cnt[ro + r];
        const int64_t src = out.row_off[ro + r];
        for (int e = 0; e < cnt; ++e) {
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
    const int2 ab = in.pairs[p];
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
    std::vector<int2> pairs(P);
    {
        int64_t p = 0;
        for (int a = 0; a < k; ++a)
            for (int b = a + 1; b < k; ++b) {
                pairs[p] = make_int2(a, b);
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
    // row pointers: always a padded copy in the workspace (the staged form's
    // bulk copies read up to 15 bytes past an array's end)
    const size_t o_rp = take(sizeof(int32_t) * rows);
    const size_t o_pno = host_in ? take(sizeof(int64_t) * (P + 1)) : 0;
    const size_t o_col = host_in ? take(sizeof(int32_t) * nnz_in) : 0;
    const size_t o_val = host_in ? take(sizeof(float) * nnz_in) : 0;
    const size_t o_tpro = take(sizeof(int64_t) * (P + 1));
    const size_t o_trp = take(sizeof(int32_t) * rows_t);
    const size_t o_tcur = take(sizeof(int32_t) * rows_t);
    const size_t o_tcv = take(sizeof(int2) * nnz_in);
    const size_t o_fcv = take(sizeof(int2) * nnz_in);
    const size_t o_len = take(sizeof(int32_t) * k);
    const size_t o_pairs = take(sizeof(int2) * P);
    const size_t o_mg = take(sizeof(int32_t) * 2 * (k - 1));
    const size_t o_tree = take(sizeof(int32_t) * (size_t)(2 * k - 1) * 6 + sizeof(int32_t) * k * 4);
    const size_t o_cnt = take(sizeof(int32_t) * rows);
    const size_t o_off = take(sizeof(int64_t) * rows);
    const size_t o_nz = take(sizeof(int32_t) * P);
    const size_t o_pn = take(sizeof(int64_t) * P);
    const size_t o_st = take(64);
    // ---- the staged form: stage buffers, accumulator rows, work items
    // (row chunks of every pair, in pair order)
    StageCfg sc{};
    int max_rc = 0;
    std::vector<int4> work;
    bool staged = C->tune.cons_form != 0 && cp->T <= kZTab;
    // shared memory of a CTA of the staged form with `ctas` CTAs per SM: z
    // table, views, two stage buffers, accumulator rows, row counts (at most
    // kStMaxRows rows per chunk); less the static shared memory and a margin
    auto stage_cfg = [&](int ctas, int slot_div) {
        StageCfg c{};
        const int per_cta = std::min(C->smem_optin, C->smem_per_sm / ctas - 1024) - 1024;
        c.ztab = std::max(1, std::min(cp->T, k));
        c.slot_bytes = (per_cta / slot_div) & ~15;
        const int fixed = (int)(sizeof(ZEnt) * c.ztab + sizeof(SView) * 2 * kStBatch) + 2 * c.slot_bytes +
                          4 * kStMaxRows;
        c.acc_cells = (per_cta - fixed) / 4;
        return c;
    };
    // two CTAs per SM, unless their accumulators would hold fewer than
    // kStMinRows rows of the longest sequence: shorter chunks re-stage more of
    // every z's band and repeat the per-chunk work more often.  Measured: 64
    // sequences of 200-400 (36 rows with two CTAs) run faster with two; 500
    // of 150-500 (26 rows) and 100 of 2000-4000 (3) with one CTA and chunks
    // twice as long
    int st_ctas = C->tune.cons_ctas_per_sm;
    if (st_ctas <= 0) st_ctas = stage_cfg(2, 5).acc_cells / maxlen >= kStMinRows ? 2 : 1;
    // each stage buffer a fifth of the CTA's shared memory, or an eighth when
    // the accumulator would otherwise hold fewer than kStLongRows rows of the
    // longest sequence: longer chunks then gain more than smaller batches
    // cost.  Measured: 100 sequences of 2000-4000 (7.6 rows) 253 -> 232 ms;
    // 500 of 150-500 (94 rows) keep a fifth (277 ms with an eighth, 198 with
    // a fifth)
    const int slot_div = stage_cfg(st_ctas, 5).acc_cells / maxlen >= kStLongRows ? 5 : 8;
    if (staged) {
        sc = stage_cfg(st_ctas, slot_div);
        sc.wait_polls = C->tune.cons_wait_polls > 0 ? C->tune.cons_wait_polls : kStSpin;
        sc.stall_first = C->tune.cons_stall_test ? 1 : 0;
        if (sc.acc_cells < maxlen) staged = false;
    }
    if (staged) {
        for (int a = 0, p = 0; a < k && staged; ++a)
            for (int b = a + 1; b < k; ++b, ++p) {
                int rcn = std::min(std::min(lens[a], sc.acc_cells / lens[b]), kStMaxRows);
                if (C->tune.cons_chunk_rows > 0) rcn = std::min(rcn, C->tune.cons_chunk_rows);
                rcn = std::max(rcn, 1);
                max_rc = std::max(max_rc, rcn);
                for (int i0 = 0; i0 < lens[a]; i0 += rcn) work.push_back(make_int4(p, i0, std::min(lens[a], i0 + rcn), 0));
                if (work.size() > ((size_t)1 << 26)) { staged = false; break; }
            }
        if (!staged) std::vector<int4>().swap(work);
    }
    const size_t o_work = take(sizeof(int4) * std::max<size_t>(work.size(), 1));
    const size_t o_fband = staged ? take(sizeof(int32_t) * rows) : 0;
    const size_t o_tband = staged ? take(sizeof(int32_t) * rows_t) : 0;
    if ((e = C->cons_ws.ensure(sz)) != cudaSuccess) return fail(QP_ENOMEM, "consistency: %zu bytes of workspace", sz);
    char* W = (char*)C->cons_ws.ptr;
    ConsIn in;
    in.k = k;
    in.P = P;
    in.pro = host_in ? (const int64_t*)(W + o_pro) : post->pair_row_off;
    in.rp = (const int32_t*)(W + o_rp);
    in.pno = host_in ? (const int64_t*)(W + o_pno) : post->pair_nnz_off;
    in.col = host_in ? (const int32_t*)(W + o_col) : post->col;
    in.val = host_in ? (const float*)(W + o_val) : post->val;
    in.tpro = (const int64_t*)(W + o_tpro);
    in.trp = (const int32_t*)(W + o_trp);
    in.tcv = (const int2*)(W + o_tcv);
    in.fcv = (const int2*)(W + o_fcv);
    in.fband = staged ? (const int32_t*)(W + o_fband) : nullptr;
    in.tband = staged ? (const int32_t*)(W + o_tband) : nullptr;
    in.len = (const int32_t*)(W + o_len);
    in.pairs = (const int2*)(W + o_pairs);
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
        (e = up(o_pairs, pairs.data(), sizeof(int2) * P)) != cudaSuccess ||
        (e = cudaMemcpyAsync(W + o_mg, merges, sizeof(int32_t) * 2 * (k - 1),
                             merges_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
        return cuda_fail(e, "consistency: inputs");
    if ((e = cudaMemcpyAsync(W + o_rp, post->row_ptr, sizeof(int32_t) * rows,
                             host_in ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "consistency: row pointers");
    if (!work.empty() && (e = up(o_work, work.data(), sizeof(int4) * work.size())) != cudaSuccess)
        return cuda_fail(e, "consistency: work items");
    if (host_in &&
        ((e = up(o_pro, post->pair_row_off, sizeof(int64_t) * (P + 1))) != cudaSuccess ||
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
    k_cons_interleave<<<warp_blocks, 256, 0, st>>>(in, (int2*)(W + o_fcv));
    unsigned* d_stats = (unsigned*)(d_status + 6);     // largest value, largest row sum (float bits)
    int32_t* d_wide = d_status + 8;                    // the staged form's unit would be too coarse
    if (staged) {
        k_cons_stats<<<warp_blocks, 256, 0, st>>>(in, d_stats);
        k_cons_bands<<<warp_blocks, 256, 0, st>>>(in, (int32_t*)(W + o_fband), (int32_t*)(W + o_tband));
    }
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
        if ((e = cudaMemsetAsync(d_status + 1, 0, 20, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(d_wide, 0, 4, st)) != cudaSuccess)
            return cuda_fail(e, "consistency");
        if (staged) {
            const int nzb = std::max(1, std::min(cp->T, k - 2));
            const size_t dyn = sizeof(ZEnt) * sc.ztab + sizeof(SView) * 2 * kStBatch + 2 * (size_t)sc.slot_bytes +
                               4 * (size_t)sc.acc_cells + 4 * (size_t)kStMaxRows;
            auto kern = st_ctas == 1 ? k_cons_relax_staged<kStGroup, 1> : k_cons_relax_staged<kStGroup, 2>;
            if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn)) != cudaSuccess)
                return cuda_fail(e, "consistency: shared memory size");
            kern<<<(unsigned)work.size(), kStThreads, dyn, st>>>(
                in, o, (const int4*)(W + o_work), sc, (float)cp->h, cp->n_max, (float)cp->threshold, nzb, d_stats,
                C->tune.cons_min_unit > 0 ? C->tune.cons_min_unit : kMinUnit, d_wide, d_status + 9, d_status);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "consistency: k_cons_relax_staged");
        } else {
            k_cons_relax<<<(unsigned)P, nwarps * 32, smem, st>>>(in, o, nwarps, acc_len, (float)cp->h, cp->n_max,
                                                                 (float)cp->threshold, d_status);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "consistency: k_cons_relax");
        }
        if ((e = cudaMemcpyAsync(h_status, d_status, 40, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_fail(e, "consistency");
        if (h_status[0]) return fail(QP_EINVAL, "consistency: merges are not a valid join sequence of k leaves");
        if (h_status[9]) return fail(QP_ECUDA, "consistency: a stage buffer's copies did not complete in time");
        if (staged && h_status[8]) {
            // values or row sums too large for a fine enough 32-bit unit: the
            // row form (64-bit sums) from the start
            staged = false;
            C->cons_last_form = 0;
            --attempt;
            continue;
        }
        C->cons_last_form = staged ? 1 : 0;
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
