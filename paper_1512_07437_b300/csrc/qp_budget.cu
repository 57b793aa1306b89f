// Memory-budgeted sparsity (paper, Methods, "Other algorithmic improvements":
// the posterior matrices of all pairs are fitted into a user-given amount of
// memory by lowering the sparsity coefficient, i.e. by keeping fewer entries).
//
// Given the CSR at threshold theta (T entries in all) and room for N entries,
// theta' is the smallest threshold whose kept entries number at most N:
// theta when T <= N, else the next representable value above the (N+1)-th
// largest entry, in the precision the entries are compared in (float for the
// FP32 form, double for the FP64 form).  Entries equal to that (N+1)-th value
// are all dropped, so fewer than N may remain.
//
// The values are positive, so their bit patterns order like the values; the
// (N+1)-th largest is found by a radix select on the bit patterns.  The
// compaction records the smallest and largest key; their common leading bits
// are known before the first pass (for values in [theta, 1] that is the sign
// and most of the exponent), and each pass resolves 14 more bits with a
// histogram of the keys that share the bits found so far (2 passes for float
// entries in practice, at most 3; at most 5 for double).  Every kernel reads its counts from
// device memory, so the sequence needs no host decision (it runs inside the
// captured call).  The filtered CSR is then written from the full one.
#include "qp_internal.h"

namespace qpk {

namespace {

constexpr unsigned FULLM = 0xffffffffu;
constexpr int kDigitBits = 14;
constexpr int kBins = 1 << kDigitBits;
static_assert(kBins == kBudgetBins, "histogram size");

template <typename K>
__device__ __forceinline__ K key_at(const void* vals, int64_t i);
template <>
__device__ __forceinline__ uint32_t key_at<uint32_t>(const void* vals, int64_t i) {
    return __float_as_uint(((const float*)vals)[i]);
}
template <>
__device__ __forceinline__ unsigned long long key_at<unsigned long long>(const void* vals, int64_t i) {
    return (unsigned long long)__double_as_longlong(((const double*)vals)[i]);
}

__global__ void k_sel_init(const int64_t* total, int64_t n_keep, double theta, int f64,
                           const unsigned long long* minmax, SelectState* s, unsigned* hist, Status* st) {
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) hist[i] = 0;
    if (threadIdx.x == 0) {
        s->total = *total;
        // bits shared by every key: the smallest and the largest agree on them
        const int KB = f64 ? 64 : 32;
        const unsigned long long lo = minmax[0], hi = minmax[1];
        int common = KB;
        if (s->total > 0 && lo != hi) common = __clzll((long long)(lo ^ hi)) - (64 - KB);
        s->prefix = (s->total > 0 && common > 0) ? (lo >> (KB - common)) : 0ull;
        s->bits_done = s->total > 0 ? common : 0;
        s->rank = n_keep;                 // 0-based rank, from the top, of the (N+1)-th largest
        // nothing to select when the pool overflowed (the call runs again)
        s->active = (s->total > n_keep && !st->pool_overflow) ? 1 : 0;
        s->theta_f = (float)theta;
        s->theta_d = theta;
        s->f64 = f64;
        st->theta_used = f64 ? theta : (double)(float)theta;
    }
}

// histogram of the next digit of the keys that carry the prefix found so far
template <typename K>
__global__ void k_sel_hist(const void* vals, const SelectState* s, unsigned* hist) {
    extern __shared__ unsigned h[];                   // kBins counters (dynamic: 64 KB)
    constexpr int KB = (int)sizeof(K) * 8;
    if (!s->active || s->bits_done >= KB) return;   // the same for every thread of the grid
    const int done = s->bits_done;
    const int dig = min(kDigitBits, KB - done);
    const int shift = KB - done - dig;
    const K prefix = (K)s->prefix;
    const K mask = (K)((1u << dig) - 1u);
    const int64_t n = s->total;
    for (int b = threadIdx.x; b < kBins; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const K key = key_at<K>(vals, i);
        if (done == 0 || (key >> (KB - done)) == prefix) atomicAdd(&h[(int)((key >> shift) & mask)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < (1 << dig); b += blockDim.x)
        if (h[b]) atomicAdd(&hist[b], h[b]);
}

// writes the cut one unit above the found key
template <typename K>
__device__ __forceinline__ void write_cut(SelectState* s, Status* st, unsigned long long key) {
    if (sizeof(K) == 4) {
        const float t = __uint_as_float((uint32_t)key + 1u);
        s->theta_f = t;
        st->theta_used = (double)t;
    } else {
        const double t = __longlong_as_double((long long)(key + 1ull));
        s->theta_d = t;
        st->theta_used = t;
    }
}

// the digit whose bucket holds the wanted rank (one block of 1024 threads,
// 16 bins each, counted from the top bin); after the last digit, the
// threshold one unit above the found key
template <typename K>
__global__ void __launch_bounds__(1024) k_sel_pick(SelectState* s, unsigned* hist, Status* st) {
    constexpr int KB = (int)sizeof(K) * 8;
    __shared__ unsigned long long wsum[32];
    __shared__ int found;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (!s->active) return;                       // the same for every thread
    const int done = s->bits_done;
    if (done >= KB) {
        // every bit is known (all keys of the bucket are equal): the cut, once
        if (done == KB && tid == 0) {
            s->bits_done = KB + 1;
            write_cut<K>(s, st, s->prefix);
        }
        return;
    }
    const int dig = min(kDigitBits, KB - done);
    const int nb = 1 << dig;
    const int per = (nb + 1023) / 1024;
    unsigned long long sum = 0;
    for (int q = 0; q < per; ++q) {
        const int j = tid * per + q;
        if (j < nb) sum += hist[nb - 1 - j];
    }
    unsigned long long incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(FULLM, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[wid] = incl;
    if (tid == 0) found = 0;
    __syncthreads();
    if (wid == 0) {
        unsigned long long w = wsum[lane], wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(FULLM, wi, o);
            if (lane >= o) wi += u;
        }
        wsum[lane] = wi - w;                     // exclusive prefix of each warp
    }
    __syncthreads();
    const unsigned long long excl = wsum[wid] + incl - sum;
    const unsigned long long rank = (unsigned long long)s->rank;
    if (excl <= rank && rank < excl + sum) {
        // this thread's bins hold the rank (exactly one thread: the ranges tile)
        unsigned long long acc = excl;
        for (int q = 0; q < per; ++q) {
            const int j = tid * per + q;
            const unsigned c = hist[nb - 1 - j];
            if (rank < acc + c) {
                const unsigned long long prefix = (s->prefix << dig) | (unsigned long long)(nb - 1 - j);
                s->prefix = prefix;
                s->rank = (long long)(rank - acc);
                if (done + dig == KB) {
                    // prefix is the (N+1)-th largest key: keep entries strictly above it
                    s->bits_done = KB + 1;
                    write_cut<K>(s, st, prefix);
                } else {
                    s->bits_done = done + dig;
                }
                found = 1;
                break;
            }
            acc += c;
        }
    }
    __syncthreads();
    for (int b = tid; b < kBins; b += 1024) hist[b] = 0;   // ready for the next pass
    if (tid == 0 && !found) {
        // the counts do not hold the rank: a logic error, reported to the host
        st->select_error = 1;
        s->active = 0;
    }
}

// thresholds read once per thread (the output stores could alias the state)
struct Cut {
    float f;
    double d;
    __device__ explicit Cut(const SelectState* s) : f(s->theta_f), d(s->theta_d) {}
};

__device__ __forceinline__ bool kept(const float* val, const double* val64, int64_t i, const Cut& t) {
    return val64 ? val64[i] >= t.d : val[i] >= t.f;
}

// row pointers and entry count of every pair after the filter (warp per pair)
__global__ void k_budget_count(const int2* __restrict__ pairs, const int64_t* __restrict__ seq_off,
                               const int64_t* __restrict__ pair_row_off, const int64_t* __restrict__ in_off,
                               const int32_t* __restrict__ in_rowptr, const float* in_val, const double* in_val64,
                               const SelectState* s, int64_t n_pairs, int32_t* __restrict__ out_rowptr,
                               int64_t* __restrict__ out_nnz, const Status* st) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= n_pairs || st->pool_overflow) return;   // the call runs again
    const int2 ab = pairs[p];
    const int m = (int)(seq_off[ab.x + 1] - seq_off[ab.x]);
    const int64_t ro = pair_row_off[p], base = in_off[p];
    const Cut cut(s);
    // a lane per row (32 rows in flight), then a scan of the counts
    int carry = 0;
    for (int r0 = 0; r0 <= m; r0 += 32) {
        const int r = r0 + lane;
        int cnt = 0;
        if (r < m) {
            const int beg = in_rowptr[ro + r], end = in_rowptr[ro + r + 1];
            for (int e = beg; e < end; ++e) cnt += kept(in_val, in_val64, base + e, cut) ? 1 : 0;
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(FULLM, incl, o);
            if (lane >= o) incl += u;
        }
        if (r <= m) out_rowptr[ro + r] = carry + incl - cnt;
        carry += __shfl_sync(FULLM, incl, 31);
    }
    if (lane == 0) out_nnz[p] = carry;
}

// the kept entries, in order (warp per pair, lanes over a row's entries)
__global__ void k_budget_copy(const int2* __restrict__ pairs, const int64_t* __restrict__ seq_off,
                              const int64_t* __restrict__ pair_row_off, const int64_t* __restrict__ in_off,
                              const int32_t* __restrict__ in_rowptr, const int32_t* __restrict__ in_col,
                              const float* in_val, const double* in_val64, const SelectState* s, int64_t n_pairs,
                              const int64_t* __restrict__ out_off, const int32_t* __restrict__ out_rowptr,
                              int32_t* __restrict__ out_col, float* __restrict__ out_val,
                              double* __restrict__ out_val64, int64_t out_cap, const Status* st) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= n_pairs || st->pool_overflow) return;   // the call runs again
    const int2 ab = pairs[p];
    const int m = (int)(seq_off[ab.x + 1] - seq_off[ab.x]);
    const int64_t ro = pair_row_off[p], bin = in_off[p], bout = out_off[p];
    const Cut cut(s);
    // a lane per row (32 rows in flight), each writing its kept entries in order
    for (int r = lane; r < m; r += 32) {
        const int beg = in_rowptr[ro + r], end = in_rowptr[ro + r + 1];
        int64_t o = bout + out_rowptr[ro + r];
        for (int e = beg; e < end; ++e) {
            if (!kept(in_val, in_val64, bin + e, cut)) continue;
            if (o < out_cap) {                   // always, unless the select failed (reported)
                out_col[o] = in_col[bin + e];
                out_val[o] = in_val[bin + e];
                if (out_val64) out_val64[o] = in_val64[bin + e];
            }
            ++o;
        }
    }
}

}  // namespace

cudaError_t prepare_budget_kernels() {
    const int hbytes = (int)(sizeof(unsigned) * kBins);
    cudaError_t e = cudaFuncSetAttribute(k_sel_hist<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, hbytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sel_hist<unsigned long long>, cudaFuncAttributeMaxDynamicSharedMemorySize, hbytes);
    return e;
}

cudaError_t launch_budget_select(const int64_t* total, int64_t n_keep, double theta, bool f64, const float* val,
                                 const double* val64, const unsigned long long* minmax, SelectState* s,
                                 unsigned* hist, Status* st, int grid, cudaStream_t str) {
    // passes for the worst case (only the sign bit shared); a pass with
    // nothing left to find returns at once, and one more pick writes the cut
    k_sel_init<<<1, 256, 0, str>>>(total, n_keep, theta, f64 ? 1 : 0, minmax, s, hist, st);
    const int passes = ((f64 ? 63 : 31) + kDigitBits - 1) / kDigitBits;
    const size_t hbytes = sizeof(unsigned) * kBins;
    for (int pass = 0; pass < passes; ++pass) {
        if (f64) k_sel_hist<unsigned long long><<<grid, 256, hbytes, str>>>(val64, s, hist);
        else k_sel_hist<uint32_t><<<grid, 256, hbytes, str>>>(val, s, hist);
        if (f64) k_sel_pick<unsigned long long><<<1, 1024, 0, str>>>(s, hist, st);
        else k_sel_pick<uint32_t><<<1, 1024, 0, str>>>(s, hist, st);
    }
    if (f64) k_sel_pick<unsigned long long><<<1, 1024, 0, str>>>(s, hist, st);
    else k_sel_pick<uint32_t><<<1, 1024, 0, str>>>(s, hist, st);
    return cudaGetLastError();
}

cudaError_t launch_budget_count(const int2* pairs, const int64_t* seq_off, const int64_t* pair_row_off,
                                const int64_t* in_off, const int32_t* in_rowptr, const float* in_val,
                                const double* in_val64, const SelectState* s, int64_t n_pairs, int32_t* out_rowptr,
                                int64_t* out_nnz, const Status* st, cudaStream_t str) {
    const int blocks = (int)((n_pairs * 32 + 255) / 256);
    if (blocks > 0)
        k_budget_count<<<blocks, 256, 0, str>>>(pairs, seq_off, pair_row_off, in_off, in_rowptr, in_val, in_val64,
                                                 s, n_pairs, out_rowptr, out_nnz, st);
    return cudaGetLastError();
}

cudaError_t launch_budget_copy(const int2* pairs, const int64_t* seq_off, const int64_t* pair_row_off,
                               const int64_t* in_off, const int32_t* in_rowptr, const int32_t* in_col,
                               const float* in_val, const double* in_val64, const SelectState* s, int64_t n_pairs,
                               const int64_t* out_off, const int32_t* out_rowptr, int32_t* out_col, float* out_val,
                               double* out_val64, int64_t out_cap, const Status* st, cudaStream_t str) {
    const int blocks = (int)((n_pairs * 32 + 255) / 256);
    if (blocks > 0)
        k_budget_copy<<<blocks, 256, 0, str>>>(pairs, seq_off, pair_row_off, in_off, in_rowptr, in_col, in_val,
                                                in_val64, s, n_pairs, out_off, out_rowptr, out_col, out_val,
                                                out_val64, out_cap, st);
    return cudaGetLastError();
}

}  // namespace qpk
