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
// Bookkeeping shared by all forms: per slot x, the minimum of row x over the
// live columns to its right and the column where it is reached (smallest
// column on ties).  After a join of (a, b) only three kinds of rows change:
// row a (its new minimum comes out of the averaging itself), rows whose
// minimum sat in column a or b (re-scanned), and rows left of a, which can
// only improve through column a.  A join is one argmin over the row minima,
// one averaging pass, and a few row scans.
//
// The joins are a serial chain, so each form is built for latency:
//   cluster form (k up to about 660): the symmetric matrix lives in the
//     shared memory of a thread-block cluster of 1-16 CTAs, each owning a
//     slab of full rows.  Every CTA publishes the best row minimum of its
//     slab (and its share of row a's new minimum) into every CTA's shared
//     memory; after one cluster barrier each CTA reduces those to the same
//     pair.  The averaging touches only the CTA's own rows (column a and b)
//     plus remote stores of row a into its owner, so a join costs one
//     cluster barrier and a few shared-memory passes;
//   single-CTA forms (larger k): the matrix stays in global memory (L2 for
//     all but the largest k); one CTA runs the joins with the per-slot state
//     in shared memory up to k = 8192, else in global memory.
// The working matrix is a symmetric copy of the caller's upper triangle
// (k_tree_mirror), with an even row stride so every row starts 16-byte
// aligned.  Distances are compared through order-preserving 64-bit integer
// keys of their bit patterns (dkey): FP64 compares run on B300's narrow FP64
// path and would sit on the serial chain of every reduction; the only FP64
// arithmetic left is the averaging itself.
#include "../../include/qp.h"
#include "qp_host.h"

#include <cooperative_groups.h>

#include <climits>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

namespace {

namespace cg = cooperative_groups;

constexpr int kMaxThreads = 1024;
constexpr int kRowWarps = 8;              // warps per block of k_tree_rows
constexpr int kSmemSlots = 8192;          // single-CTA form: slot state in shared memory up to this k
constexpr int kSlotBytes = 8 + 4 + 4 + 4 + 1;
constexpr int kClusterThreads = 128;      // threads per CTA of the cluster form
constexpr int kMaxCluster = 16;           // CTAs per cluster (16 needs the non-portable size)
constexpr int kRowsPerLane = 6;           // cluster form: at most this many rows of a CTA's slab per lane
constexpr int kSpinLimit = 1 << 24;       // bounded waits of the cluster form's exchange

struct TreeWork {
    const double* in;   // caller's k x k matrix (upper triangle read), row stride k
    double* D;          // [k][ld] symmetric working copy
    long long* rmin;    // [k] key of the row minimum over live columns to the right (kNone: none)
    int* ridx;          // [k] its column (-1: none, or slot empty)
    int* cid;           // [k] id of the cluster in the slot
    int* list;          // [k] rows to re-scan
    unsigned char* alive;
    int32_t* merges;    // [k - 1][2]
    double* heights;    // [k - 1]
    int* status;        // 0: ok
    int k;
    int ld;             // row stride of D (k rounded up to even)
    int smem_state;     // single-CTA form: per-slot state in shared memory
};

constexpr long long kNone = LLONG_MAX;     // key of "no entry"

// One entry of the argmin exchange of the cluster form: key, row, column
// (16 bytes, sent as one vector store).
struct __align__(16) Part {
    long long v;
    int r;
    int c;
};

// Shared-memory layout of one CTA of the cluster form holding R rows: the
// rows at an odd stride ls (column-wise writes of the prologue stay free of
// bank conflicts), the row minima of the prologue, the exchange buffers, and
// the cluster ids (CTA 0).
struct ClusterSmem {
    size_t o_rmin, o_part, o_bar, o_ridx, o_cid, bytes;
    __host__ __device__ ClusterSmem(int R, int ls, int k) {
        size_t o = (size_t)R * ls * sizeof(double);
        o_rmin = o;  o += (size_t)R * sizeof(long long);
        o = (o + 15) & ~(size_t)15;
        o_part = o;  o += 4 * kMaxCluster * sizeof(Part);
        o_bar = o;   o += 2 * sizeof(unsigned long long);   // one mbarrier per exchange buffer
        o_ridx = o;  o += (size_t)R * sizeof(int);
        o_cid = o;   o += (size_t)k * sizeof(int);
        bytes = (o + 15) & ~(size_t)15;
    }
};

// Integer key with the order of the doubles (for every value but NaN): the
// bit pattern, magnitude bits flipped for negatives, both zeros mapped to 0.
__device__ __forceinline__ long long dkey(double d) {
    const long long b = __double_as_longlong(d);
    if ((b & LLONG_MAX) == 0) return 0;
    return b >= 0 ? b : (b ^ LLONG_MAX);
}

__device__ __forceinline__ bool less_pair(long long v, int i, long long bv, int bi) {
    return v < bv || (v == bv && i < bi);
}

// (key, index) minimum over a warp into lane 0; (kNone, -1) is empty.
__device__ __forceinline__ void warp_argmin(long long& v, int& i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long ov = __shfl_down_sync(0xffffffffu, v, o);
        const int oi = __shfl_down_sync(0xffffffffu, i, o);
        if (oi >= 0 && (i < 0 || less_pair(ov, oi, v, i))) { v = ov; i = oi; }
    }
}

// (key, row) minimum over a warp, in every lane, by redux.sync steps (high
// key half, low half, row) and, when asked for, the column of the winner by
// one more (rows are distinct, so the winner is unique); an empty entry is
// (kNone, INT_MAX).
template <bool WITH_COL>
__device__ __forceinline__ void warp_min_key(long long& key, int& r, int& c) {
    const int hi = (int)(key >> 32);
    const unsigned lo = (unsigned)((unsigned long long)key & 0xffffffffull);
    const int mhi = __reduce_min_sync(0xffffffffu, hi);
    const unsigned mlo = __reduce_min_sync(0xffffffffu, hi == mhi ? lo : 0xffffffffu);
    const bool eq = hi == mhi && lo == mlo;
    const unsigned mr = __reduce_min_sync(0xffffffffu, eq ? (unsigned)r : 0xffffffffu);
    if (WITH_COL) c = (int)__reduce_max_sync(0xffffffffu, eq && (unsigned)r == mr ? (unsigned)c : 0u);
    key = (long long)(((unsigned long long)(unsigned)mhi << 32) | mlo);
    r = (int)mr;
}

// Minimum of row r (values `row`) over live columns c > r (smallest c on
// ties), by one warp; loads are issued eight at a time.  D is written by the
// same kernel, so it is read through the coherent path (no __restrict__).
__device__ void scan_row(const double* row, const unsigned char* alive, int k, int r, int lane, long long* rmin,
                         int* ridx) {
    long long bv = kNone;
    int bc = -1;
    for (int c0 = r + 1 + lane; c0 < k; c0 += 256) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = c0 + 32 * u;
            v[u] = c < k ? row[c] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = c0 + 32 * u;
            const long long kv = dkey(v[u]);
            if (c < k && alive[c] && (bc < 0 || less_pair(kv, c, bv, bc))) { bv = kv; bc = c; }
        }
    }
    warp_argmin(bv, bc);
    if (lane == 0) {
        *rmin = bc < 0 ? kNone : bv;
        *ridx = bc;
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
        if (i >= k || j >= w.ld) continue;
        double v;
        if (j >= k) v = 0.0;                       // padding column
        else if (ty < tx || (ty == tx && r < c)) v = S[r][c];
        else if (ty > tx || r > c) v = S[c][r];
        else v = 0.0;
        w.D[(size_t)i * w.ld + j] = v;
    }
}

// ---------------------------------------------------------------- cluster form

// Marker stored in a dead column: its key is the largest (kNone), so scans
// never pick it.
__device__ __forceinline__ double dead_value() { return __longlong_as_double(LLONG_MAX); }

// Minimum over live columns c > x of a row held in shared memory, by one
// warp: (key, column) in every lane, (kNone, INT_MAX) when there is none.
// Each lane keeps four independent minima (columns lane + 32 u mod 128) so
// the loads and compares of consecutive columns overlap.
__device__ __forceinline__ void scan_row_keys(const double* row, int x, int k, int lane, long long& key, int& col) {
    long long bv[4] = {kNone, kNone, kNone, kNone};
    int bc[4] = {INT_MAX, INT_MAX, INT_MAX, INT_MAX};
    int c = x + 1 + lane;
    for (; c + 96 < k; c += 128) {
        long long kv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) kv[u] = dkey(row[c + 32 * u]);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (kv[u] < bv[u]) { bv[u] = kv[u]; bc[u] = c + 32 * u; }   // ascending: equal keys keep the first
    }
#pragma unroll
    for (int u = 0; u < 3; ++u) {
        const int cu = c + 32 * u;
        if (cu < k) {
            const long long kv = dkey(row[cu]);
            if (kv < bv[u]) { bv[u] = kv; bc[u] = cu; }
        }
    }
#pragma unroll
    for (int u = 1; u < 4; ++u)
        if (bv[u] < bv[0] || (bv[u] == bv[0] && bc[u] < bc[0])) { bv[0] = bv[u]; bc[0] = bc[u]; }
    int dummy = 0;
    warp_min_key<false>(bv[0], bc[0], dummy);           // columns are distinct across lanes
    key = bv[0];
    col = bc[0];
}

// ---- exchange between the CTAs of a cluster: stores into another CTA's
// shared memory that count their bytes on that CTA's mbarrier

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t map_rank(uint32_t addr, int rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ void st_async_b64(uint32_t raddr, unsigned long long v, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];"
                 :: "r"(raddr), "l"(v), "r"(rbar) : "memory");
}

__device__ __forceinline__ void st_async_v2b64(uint32_t raddr, unsigned long long v0, unsigned long long v1,
                                               uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.b64 [%0], {%1, %2}, [%3];"
                 :: "r"(raddr), "l"(v0), "l"(v1), "r"(rbar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count) : "memory");
}

// the local arrival of a phase, announcing the bytes it waits for
__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 st, [%0], %1; }"
                 :: "r"(bar), "r"(bytes) : "memory");
}

// waits (bounded) for the phase of the given parity; false when it ran out
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < kSpinLimit; ++it) {
        uint32_t done;
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2; "
                     "selp.u32 %0, 1, 0, p; }"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// The cluster form.  Prologue (all warps): the CTA's slab of rows from the
// caller's upper triangle, and their row minima.  Joins (warp 0 alone; the
// other warps wait at the final cluster barrier): each lane owns rows lane,
// lane + 32, ... (J of them) of the slab and keeps their minima in
// registers.  Exchange e (e = 0 before the first join, e = s + 1 after join
// s) uses buffer and mbarrier e & 1: every CTA sends its two entries to every
// CTA, and during join s the CTAs write row a_s into its owner, whose
// mbarrier e = s + 1 also counts those bytes.  A CTA sends for exchange e
// only after it has received exchange e - 1, which needs every CTA's
// entries of e - 1, so no buffer is overwritten while it is read.
template <int J>
__global__ void __launch_bounds__(kClusterThreads, 1) k_tree_cluster(TreeWork w, int R, int ls) {
    constexpr int NT = kClusterThreads, NW = NT / 32;
    cg::cluster_group cl = cg::this_cluster();
    const int nc = (int)cl.num_blocks();
    const int me = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int k = w.k;
    const int r0 = me * R;
    const int nr = max(0, min(k, r0 + R) - r0);
    extern __shared__ __align__(16) unsigned char smem[];
    const ClusterSmem L(R, ls, k);
    double* Dl = (double*)smem;                            // row r0 + i at Dl + i * ls
    long long* rmin_s = (long long*)(smem + L.o_rmin);
    Part* part = (Part*)(smem + L.o_part);                 // [2 buffers][row, candidate][kMaxCluster]
    unsigned long long* bar = (unsigned long long*)(smem + L.o_bar);
    int* ridx_s = (int*)(smem + L.o_ridx);
    int* cid = (int*)(smem + L.o_cid);
    const bool multi = nc > 1;

    // slab: D(r, c) = in[r][c] right of the diagonal (row segments), in[c][r]
    // left of it (column segments, contiguous along the slab's rows)
    for (int i = wid; i < nr; i += NW) {
        const int r = r0 + i;
        const double* src = w.in + (size_t)r * k;
        double* dst = Dl + (size_t)i * ls;
#pragma unroll 4
        for (int c = r + 1 + lane; c < k; c += 32) dst[c] = src[c];
        if (lane == 0) dst[r] = 0.0;
    }
    for (int c = wid; c < r0 + nr - 1; c += NW) {
        const double* src = w.in + (size_t)c * k + r0;
#pragma unroll 4
        for (int i = max(0, c - r0 + 1) + lane; i < nr; i += 32) Dl[(size_t)i * ls + c] = src[i];
    }
    if (me == 0)
        for (int c = tid; c < k; c += NT) cid[c] = c;
    if (tid == 0 && multi) {
        mbar_init(smem_addr(&bar[0]), 1);
        mbar_init(smem_addr(&bar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    for (int i = wid; i < nr; i += NW) {
        long long key;
        int col;
        scan_row_keys(Dl + (size_t)i * ls, r0 + i, k, lane, key, col);
        if (lane == 0) { rmin_s[i] = key; ridx_s[i] = col; }
    }
    __syncthreads();
    if (multi) cl.sync();                                  // every CTA runs and has its mbarriers ready
    if (wid != 0) {
        if (multi) cl.sync();                              // the final barrier
        return;
    }

    long long rm[J];                                       // row minimum keys of the lane's rows
    int rx[J];                                             // their columns (INT_MAX: none)
    unsigned live = 0;
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int i = j * 32 + lane;
        rm[j] = kNone;
        rx[j] = INT_MAX;
        if (i < nr) {
            rm[j] = rmin_s[i];
            rx[j] = ridx_s[i];
            live |= 1u << j;
        }
    }
    const uint32_t part_a = smem_addr(part), bar_a = smem_addr(bar);
    bool ok = true;
    // the exchanged entries: this CTA's best row minimum (rows other than the
    // last a) and its share of row a's new minimum (qv, qx); with one CTA
    // they stay in registers
    long long pv, qv = kNone;
    int pr, pc, qx = INT_MAX;
    auto row_partial = [&](int skip) {
        pv = kNone;
        pr = INT_MAX;
        pc = 0;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int x = r0 + j * 32 + lane;
            if (((live >> j) & 1) && x != skip && rx[j] != INT_MAX && (rm[j] < pv || (rm[j] == pv && x < pr))) {
                pv = rm[j];
                pr = x;
                pc = rx[j];
            }
        }
        warp_min_key<true>(pv, pr, pc);
    };
    auto send = [&](int buf) {
        if (lane < nc) {
            const uint32_t slot = part_a + (uint32_t)((buf * 2 * kMaxCluster + me) * sizeof(Part));
            const uint32_t rbar = map_rank(bar_a + buf * 8, lane);
            st_async_v2b64(map_rank(slot, lane), (unsigned long long)pv,
                           (unsigned long long)(unsigned)pr | ((unsigned long long)(unsigned)pc << 32), rbar);
            st_async_v2b64(map_rank(slot + kMaxCluster * sizeof(Part), lane), (unsigned long long)qv,
                           (unsigned long long)(unsigned)qx, rbar);
        }
    };
    const uint32_t xbytes = (uint32_t)(nc * 2 * sizeof(Part));   // entries a CTA receives per exchange
    row_partial(-1);
    if (multi) {
        if (lane == 0) mbar_expect(bar_a, xbytes);
        send(0);
    }

    int a_prev = -1;
    for (int s = 0; s < k - 1; ++s) {
        const int buf = s & 1;
        // 1. the pair, from the exchanged entries
        long long v = pv, cv = qv;
        int a = pr, b = pc, cx = qx;
        if (multi) {
            ok &= mbar_wait(bar_a + buf * 8, (s >> 1) & 1);
            v = kNone;
            cv = kNone;
            a = INT_MAX;
            cx = INT_MAX;
            if (lane < nc) {
                const Part p = part[buf * 2 * kMaxCluster + lane];
                const Part q = part[(buf * 2 + 1) * kMaxCluster + lane];
                v = p.v; a = p.r; b = p.c;
                cv = q.v; cx = q.r;
            }
            int cd = 0;
            warp_min_key<true>(v, a, b);
            warp_min_key<false>(cv, cx, cd);
        }
        // row a_prev's new minimum competes with the published rows
        if (a_prev >= 0 && cx != INT_MAX && (cv < v || (cv == v && a_prev < a))) {
            v = cv;
            a = a_prev;
            b = cx;
        }
        if (a == INT_MAX) {
            // at least two slots are live, so some live row has a live column
            // to its right: this cannot happen.  Control stays uniform.
            ok = false;
            a = 0;
            b = k - 1;
        }
        if (me == 0 && lane == 0) {
            w.merges[2 * s] = cid[a];
            w.merges[2 * s + 1] = cid[b];
            cid[a] = k + s;
        }
        // 2. averaging of column a with column b in the own rows (loads and
        // FP64 arithmetic of all the lane's rows first, so they overlap); row a
        // gets the same values in its owner's shared memory
        const int oa = a / R;
        const bool own_a = oa == me;
        double* rowA = Dl + (size_t)(a - r0) * ls;                 // valid when own_a
        const uint32_t rrow = multi && !own_a ? map_rank(smem_addr(Dl) + (uint32_t)((a - oa * R) * ls * 8), oa) : 0;
        const uint32_t rbar = multi && !own_a ? map_rank(bar_a + (buf ^ 1) * 8, oa) : 0;
        double nv[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int i = j * 32 + lane;
            nv[j] = 0.0;
            if ((live >> j) & 1) {
                const double* row = Dl + (size_t)i * ls;
                nv[j] = (row[a] + row[b]) * 0.5;
            }
        }
        unsigned need = 0;
        int written = 0;
        qv = kNone;
        qx = INT_MAX;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            if (!((live >> j) & 1)) continue;
            const int i = j * 32 + lane, x = r0 + i;
            double* row = Dl + (size_t)i * ls;
            if (x == a_prev) {
                rm[j] = cx != INT_MAX ? cv : kNone;
                rx[j] = cx;
            }
            if (x == b) {
                w.heights[s] = row[a];                      // d(a, b); halved after the last join
                live &= ~(1u << j);
                continue;
            }
            row[b] = dead_value();
            if (x == a) continue;
            row[a] = nv[j];
            if (own_a) {
                rowA[x] = nv[j];
                ++written;
            } else {
                st_async_b64(rrow + (uint32_t)x * 8, (unsigned long long)__double_as_longlong(nv[j]), rbar);
            }
            const long long kv = dkey(nv[j]);
            if (x < a) {
                const int c = rx[j];
                if (c == a || c == b) {
                    need |= 1u << j;
                } else if (kv < rm[j] || (kv == rm[j] && a < c)) {
                    rm[j] = kv;
                    rx[j] = a;
                }
            } else {
                if (kv < qv) { qv = kv; qx = x; }          // row a's new minimum (ascending x)
                if (x < b && rx[j] == b) need |= 1u << j;
            }
        }
        int qd = 0;
        warp_min_key<false>(qv, qx, qd);
        __syncwarp();
        // 3. re-scan the own rows whose minimum was in column a or b
#pragma unroll
        for (int j = 0; j < J; ++j) {
            unsigned m = __ballot_sync(0xffffffffu, (need >> j) & 1);
            while (m) {
                const int l = __ffs(m) - 1;
                m &= m - 1;
                const int i = j * 32 + l;
                long long key;
                int col;
                scan_row_keys(Dl + (size_t)i * ls, r0 + i, k, lane, key, col);
                if (lane == l) {
                    rm[j] = key;
                    rx[j] = col;
                }
            }
        }
        // 4. exchange for the next join: the owner of row a also waits for the
        // k - s - 2 values of row a that the other CTAs write
        const bool last = s == k - 2;
        if (!last) row_partial(a);
        if (multi) {
            int own = written;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) own += __shfl_xor_sync(0xffffffffu, own, o);
            const uint32_t rows_in = own_a ? (uint32_t)(k - s - 2 - own) * 8u : 0u;
            if (lane == 0) mbar_expect(bar_a + (buf ^ 1) * 8, (last ? 0u : xbytes) + rows_in);
            if (!last) send(buf ^ 1);
        }
        __syncwarp();
        a_prev = a;
    }
    if (multi) {
        // the values of the last row a reach its owner before any CTA leaves,
        // and every CTA's heights are written before CTA 0 scales them
        if (a_prev / R == me) ok &= mbar_wait(bar_a + ((k - 1) & 1) * 8, ((k - 1) >> 1) & 1);
        cl.sync();
    }
    if (me == 0)
        for (int t = lane; t < k - 1; t += 32) w.heights[t] *= 0.5;
    if (!ok && lane == 0) atomicExch(w.status, 1);
}

// ---------------------------------------------------------------- single-CTA forms

__global__ void k_tree_rows(TreeWork w) {
    const int r = blockIdx.x * kRowWarps + (threadIdx.x >> 5);
    if (r < w.k) {
        // every slot is live before the first join
        const double* row = w.D + (size_t)r * w.ld;
        const int lane = threadIdx.x & 31;
        long long bv = kNone;
        int bc = -1;
        for (int c = r + 1 + lane; c < w.k; c += 32) {
            const long long v = dkey(row[c]);
            if (bc < 0 || less_pair(v, c, bv, bc)) { bv = v; bc = c; }
        }
        warp_argmin(bv, bc);
        if (lane == 0) {
            w.rmin[r] = bc < 0 ? kNone : bv;
            w.ridx[r] = bc;
        }
    }
}

__global__ void __launch_bounds__(kMaxThreads) k_tree_join(TreeWork w) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_v[32];
    __shared__ int s_i[32];
    __shared__ int s_a, s_b, s_n;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nt = blockDim.x, nw = nt >> 5;
    const int k = w.k, ld = w.ld;
    double* D = w.D;
    long long* rmin = w.rmin;
    int* ridx = w.ridx;
    int* cid = w.cid;
    int* list = w.list;
    unsigned char* alive = w.alive;
    if (w.smem_state) {
        rmin = (long long*)smem;
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
        long long bv = kNone;
        int br = -1;
        for (int r = tid; r < k; r += nt) {
            const int c = ridx[r];
            if (c >= 0 && (br < 0 || less_pair(rmin[r], r, bv, br))) { bv = rmin[r]; br = r; }
        }
        warp_argmin(bv, br);
        if (lane == 0) { s_v[wid] = bv; s_i[wid] = br; }
        __syncthreads();
        if (wid == 0) {
            bv = lane < nw ? s_v[lane] : kNone;
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
                    cid[a] = k + s;
                    alive[b] = 0;
                    ridx[b] = -1;
                    rmin[b] = kNone;
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
        const double* Ra = D + (size_t)a * ld;
        const double* Rb = D + (size_t)b * ld;
        long long mv = kNone;
        int mc = -1;
        for (int x = tid; x < k; x += nt) {
            if (x == b) {
                w.heights[s] = Ra[b] * 0.5;      // the joining distance d(a, b) itself
                continue;
            }
            if (!alive[x] || x == a) continue;
            const double v = (Ra[x] + Rb[x]) * 0.5;
            const long long kv = dkey(v);
            D[(size_t)a * ld + x] = v;
            D[(size_t)x * ld + a] = v;
            if (x > a) {
                if (mc < 0 || less_pair(kv, x, mv, mc)) { mv = kv; mc = x; }
                if (x < b && ridx[x] == b) list[atomicAdd(&s_n, 1)] = x;
            } else {
                const int c = ridx[x];
                if (c == a || c == b) {
                    list[atomicAdd(&s_n, 1)] = x;
                } else if (less_pair(kv, a, rmin[x], c)) {
                    rmin[x] = kv;
                    ridx[x] = a;
                }
            }
        }
        warp_argmin(mv, mc);
        if (lane == 0) { s_v[wid] = mv; s_i[wid] = mc; }
        __syncthreads();
        if (wid == 0) {
            mv = lane < nw ? s_v[lane] : kNone;
            mc = lane < nw ? s_i[lane] : -1;
            warp_argmin(mv, mc);
            if (lane == 0) {
                rmin[a] = mc < 0 ? kNone : mv;
                ridx[a] = mc;
            }
        }
        // 3. re-scan the rows whose minimum was in column a or b
        const int n = s_n;
        for (int q = wid; q < n; q += nw) {
            const int r = list[q];
            scan_row(D + (size_t)r * ld, alive, k, r, lane, &rmin[r], &ridx[r]);
        }
        __syncthreads();
    }
}

int join_threads(int k) {
    const int t = (k + 31) / 32 * 32;
    return t < 64 ? 64 : (t > kMaxThreads ? kMaxThreads : t);
}

// CTAs of the cluster form for k slots (forced: exactly `want`): about 8
// rows per CTA -- the smallest power of two >= k / 8, at most 16 -- or more
// when the slab does not fit one CTA's shared memory, and a cluster the
// device can place (checked once per device and count, at the largest
// shared-memory size); 0 when none does.  A join costs a few passes of one
// warp over its rows plus one exchange, so more CTAs with fewer rows each
// are faster (measured on B300 for k from 32 to 660).
template <int J>
void* cluster_kernel() { return (void*)k_tree_cluster<J>; }

// the instance for R rows per CTA (J = rows per lane)
void* cluster_kernel_for(int R) {
    const int j = (R + 31) / 32;
    return j <= 1 ? cluster_kernel<1>() : j == 2 ? cluster_kernel<2>() : j == 3 ? cluster_kernel<3>()
         : j == 4 ? cluster_kernel<4>() : cluster_kernel<6>();
}

int cluster_ctas(int device, int k, int want, int optin, size_t* bytes, int* R, int* ls) {
    static std::mutex mu;
    static std::map<std::pair<int, void*>, bool> placeable;
    const int stride = k | 1;
    int first = 1;
    while (first < kMaxCluster && first * 8 < k) first *= 2;
    for (int c = want > 0 ? want : first; c <= kMaxCluster; c *= 2) {
        if (want > 0 && c != want) break;
        const int r = (k + c - 1) / c;
        const ClusterSmem L(r, stride, k);
        if (r > 32 * kRowsPerLane || L.bytes + 1024 > (size_t)optin) continue;
        bool ok;
        const void* kern = cluster_kernel_for(r);
        {
            std::lock_guard<std::mutex> g(mu);
            auto it = placeable.find({device * 64 + c, (void*)kern});
            if (it != placeable.end()) {
                ok = it->second;
            } else {
                // the largest size any call may ask for, so concurrent calls agree
                ok = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024) ==
                         cudaSuccess &&
                     cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
                if (ok) {
                    cudaLaunchConfig_t cfg = {};
                    cudaLaunchAttribute at[1];
                    at[0].id = cudaLaunchAttributeClusterDimension;
                    at[0].val.clusterDim.x = c;
                    at[0].val.clusterDim.y = 1;
                    at[0].val.clusterDim.z = 1;
                    cfg.gridDim = dim3(c);
                    cfg.blockDim = dim3(kClusterThreads);
                    cfg.dynamicSmemBytes = optin - 1024;
                    cfg.attrs = at;
                    cfg.numAttrs = 1;
                    int n = 0;
                    ok = cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n >= 1;
                }
                cudaGetLastError();
                placeable[{device * 64 + c, (void*)kern}] = ok;
            }
        }
        if (!ok) continue;
        *bytes = L.bytes;
        *R = r;
        *ls = stride;
        return c;
    }
    return 0;
}

// Working memory kept for the next call up to this size (larger matrices
// are allocated and released within the call).
constexpr size_t kKeepBytes = size_t(256) << 20;

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
    std::lock_guard<std::mutex> tree_lock(C->tree_mu);    // one call at a time uses the kept memory
    cudaStream_t st;
    if ((e = call_stream(C, stream, &st)) != cudaSuccess) return cuda_fail(e, "guide tree: stream order");
    int form, want_ctas;
    {
        std::lock_guard<std::mutex> g(C->mu);
        form = C->tune.tree_form;
        want_ctas = C->tune.tree_ctas;
    }
    const int ld = k + (k & 1);
    if (C->tree_optin == 0) cudaDeviceGetAttribute(&C->tree_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    size_t cl_bytes = 0;
    int R = 0, ls = 0, ncta = 0;
    if (form < 0 || form == 2) ncta = cluster_ctas(device, k, want_ctas, C->tree_optin, &cl_bytes, &R, &ls);
    if (form == 2 && ncta == 0)
        return fail(QP_EINVAL, "guide tree: the cluster form does not fit k = %d (CTAs %d)", k, want_ctas);
    const bool single = ncta == 0;
    const bool small = single && k <= kSmemSlots && form != 0;
    if (single) {
        e = cudaFuncSetAttribute(k_tree_join, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemSlots * kSlotBytes);
        if (e != cudaSuccess) return cuda_fail(e, "guide tree: shared memory size");
    }
    // device working memory: the symmetric copy (single-CTA forms), the
    // input (host input), slot state, outputs (host output), status
    const size_t kk = (size_t)k * k;
    size_t sz = 0;
    const size_t o_D = sz;   sz += single ? align256(sizeof(double) * k * (size_t)ld) : 0;
    const size_t o_in = sz;  sz += on_device ? 0 : align256(sizeof(double) * kk);
    const size_t o_mn = sz;  sz += single ? align256(sizeof(long long) * k) : 0;
    const size_t o_ix = sz;  sz += single ? align256(sizeof(int) * k) : 0;
    const size_t o_ci = sz;  sz += single && !small ? align256(sizeof(int) * k) : 0;
    const size_t o_li = sz;  sz += single && !small ? align256(sizeof(int) * k) : 0;
    const size_t o_al = sz;  sz += single && !small ? align256(k) : 0;
    const size_t o_mg = sz;  sz += on_device ? 0 : align256(sizeof(int32_t) * 2 * (k - 1));
    const size_t o_h = sz;   sz += on_device ? 0 : align256(sizeof(double) * (k - 1));
    const size_t o_st = sz;  sz += align256(sizeof(int));
    char* m = nullptr;
    const bool keep = sz <= kKeepBytes;
    if (keep) {
        if ((e = C->tree_ws.ensure(sz)) != cudaSuccess) return fail(QP_ENOMEM, "guide tree: %zu bytes of workspace", sz);
        m = (char*)C->tree_ws.ptr;
    } else if ((e = cudaMallocAsync((void**)&m, sz, st)) != cudaSuccess) {
        cudaGetLastError();
        return fail(QP_ENOMEM, "guide tree: %zu bytes of workspace", sz);
    }
    // pinned staging of the status word and of host outputs
    const size_t h_out = on_device ? 0 : sizeof(int32_t) * 2 * (k - 1) + sizeof(double) * (k - 1);
    if ((e = C->tree_h.ensure(16 + h_out)) != cudaSuccess) {
        if (!keep) cudaFreeAsync(m, st);
        return fail(QP_ENOMEM, "guide tree: pinned staging");
    }
    int* h_status = (int*)C->tree_h.ptr;
    char* h_stage = (char*)C->tree_h.ptr + 16;
    TreeWork w;
    w.k = k;
    w.ld = ld;
    w.smem_state = small ? 1 : 0;
    w.D = single ? (double*)(m + o_D) : nullptr;
    w.in = on_device ? dist : (const double*)(m + o_in);
    w.rmin = single ? (long long*)(m + o_mn) : nullptr;
    w.ridx = single ? (int*)(m + o_ix) : nullptr;
    w.cid = single && !small ? (int*)(m + o_ci) : nullptr;
    w.list = single && !small ? (int*)(m + o_li) : nullptr;
    w.alive = single && !small ? (unsigned char*)(m + o_al) : nullptr;
    w.merges = on_device ? merges : (int32_t*)(m + o_mg);
    w.heights = on_device ? heights : (double*)(m + o_h);
    w.status = (int*)(m + o_st);
    e = cudaMemsetAsync(w.status, 0, sizeof(int), st);
    if (e == cudaSuccess && !on_device)
        e = cudaMemcpyAsync((void*)w.in, dist, sizeof(double) * kk, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        if (single) {
            const int tx = (ld + 31) / 32, ty = (k + 31) / 32;
            k_tree_mirror<<<dim3(tx, ty), dim3(32, 8), 0, st>>>(w);
            k_tree_rows<<<(k + kRowWarps - 1) / kRowWarps, kRowWarps * 32, 0, st>>>(w);
            k_tree_join<<<1, join_threads(k), small ? (size_t)k * kSlotBytes : 0, st>>>(w);
            e = cudaGetLastError();
        } else {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = ncta;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(ncta);
            cfg.blockDim = dim3(kClusterThreads);
            cfg.dynamicSmemBytes = cl_bytes;
            cfg.stream = st;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            void* args[] = {&w, &R, &ls};
            e = cudaLaunchKernelExC(&cfg, cluster_kernel_for(R), args);
        }
    }
    if (e == cudaSuccess && !on_device)
        e = cudaMemcpyAsync(h_stage, w.merges, sizeof(int32_t) * 2 * (k - 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && !on_device)
        e = cudaMemcpyAsync(h_stage + sizeof(int32_t) * 2 * (k - 1), w.heights, sizeof(double) * (k - 1),
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_status, w.status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (!keep) cudaFreeAsync(m, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "guide tree");
    if (*h_status != 0) return fail(QP_ECUDA, "guide tree: internal error (no pair to join)");
    if (!on_device) {
        memcpy(merges, h_stage, sizeof(int32_t) * 2 * (k - 1));
        memcpy(heights, h_stage + sizeof(int32_t) * 2 * (k - 1), sizeof(double) * (k - 1));
    }
    return QP_OK;
}
