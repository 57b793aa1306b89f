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
// (N+1)-th largest is found by a radix select on the bit patterns, 11 bits a
// pass (3 passes for float, 6 for double), each pass a histogram of the keys
// that share the bits found so far.  Every kernel reads its counts from
// device memory, so the sequence needs no host decision (it runs inside the
// captured call).  The filtered CSR is then written from the full one.
#include "qp_internal.h"

namespace qpk {

namespace {

constexpr unsigned FULLM = 0xffffffffu;
constexpr int kDigitBits = 11;
constexpr int kBins = 1 << kDigitBits;

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

__global__ void k_sel_init(const int64_t* total, int64_t n_keep, double theta, int f64, SelectState* s,
                           unsigned* hist, Status* st) {
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) hist[i] = 0;
    if (threadIdx.x == 0) {
        s->total = *total;
        s->prefix = 0;
        s->bits_done = 0;
        s->rank = n_keep;                 // 0-based rank, from the top, of the (N+1)-th largest
        s->active = s->total > n_keep ? 1 : 0;
        s->theta_f = (float)theta;
        s->theta_d = theta;
        s->f64 = f64;
        st->theta_used = f64 ? theta : (double)(float)theta;
    }
}

// histogram of the next digit of the keys that carry the prefix found so far
template <typename K>
__global__ void k_sel_hist(const void* vals, const SelectState* s, unsigned* hist) {
    __shared__ unsigned h[kBins];
    if (!s->active) return;               // the same for every thread of the grid
    constexpr int KB = (int)sizeof(K) * 8;
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

// the digit whose bucket holds the wanted rank; after the last digit, the
// threshold one unit above the found key
template <typename K>
__global__ void k_sel_pick(SelectState* s, unsigned* hist, Status* st) {
    if (!s->active || threadIdx.x >= 32) return;
    constexpr int KB = (int)sizeof(K) * 8;
    const int lane = threadIdx.x;
    const int done = s->bits_done;
    const int dig = min(kDigitBits, KB - done);
    const int nb = 1 << dig;
    const int per = (nb + 31) / 32;       // bins a lane sums, counted from the top bin
    unsigned long long sum = 0;
    for (int q = 0; q < per; ++q) {
        const int j = lane * per + q;
        if (j < nb) sum += hist[nb - 1 - j];
    }
    unsigned long long incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(FULLM, incl, o);
        if (lane >= o) incl += u;
    }
    const unsigned long long excl = incl - sum;
    const unsigned long long rank = (unsigned long long)s->rank;
    const unsigned who = __ballot_sync(FULLM, excl <= rank && rank < incl);
    if (who == 0) {
        // the counts do not hold the rank: a logic error, reported to the host
        if (lane == 0) { st->select_error = 1; s->active = 0; }
        return;
    }
    const int l = __ffs(who) - 1;
    int digit = -1;
    unsigned long long left = 0;
    if (lane == l) {
        unsigned long long acc = excl;
        for (int q = 0; q < per; ++q) {
            const int j = lane * per + q;
            if (j >= nb) break;
            const unsigned c = hist[nb - 1 - j];
            if (rank < acc + c) { digit = nb - 1 - j; left = rank - acc; break; }
            acc += c;
        }
    }
    __syncwarp();
    for (int b = lane; b < kBins; b += 32) hist[b] = 0;   // ready for the next pass
    if (lane == l) {
        if (digit < 0) { st->select_error = 1; s->active = 0; return; }
        const unsigned long long prefix = (s->prefix << dig) | (unsigned long long)digit;
        s->prefix = prefix;
        s->rank = (long long)left;
        s->bits_done = done + dig;
        if (done + dig == KB) {
            // prefix is the (N+1)-th largest key: keep entries strictly above it
            if (KB == 32) {
                const float t = __uint_as_float((uint32_t)prefix + 1u);
                s->theta_f = t;
                st->theta_used = (double)t;
            } else {
                const double t = __longlong_as_double((long long)(prefix + 1ull));
                s->theta_d = t;
                st->theta_used = t;
            }
        }
    }
}

__device__ __forceinline__ bool kept(const float* val, const double* val64, int64_t i, const SelectState* s) {
    return val64 ? val64[i] >= s->theta_d : val[i] >= s->theta_f;
}

// row pointers and entry count of every pair after the filter (warp per pair)
__global__ void k_budget_count(const int2* __restrict__ pairs, const int64_t* __restrict__ seq_off,
                               const int64_t* __restrict__ pair_row_off, const int64_t* __restrict__ in_off,
                               const int32_t* __restrict__ in_rowptr, const float* in_val, const double* in_val64,
                               const SelectState* s, int64_t n_pairs, int32_t* __restrict__ out_rowptr,
                               int64_t* __restrict__ out_nnz) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= n_pairs) return;
    const int2 ab = pairs[p];
    const int m = (int)(seq_off[ab.x + 1] - seq_off[ab.x]);
    const int64_t ro = pair_row_off[p], base = in_off[p];
    int carry = 0;
    for (int r0 = 0; r0 <= m; r0 += 32) {
        const int r = r0 + lane;
        int cnt = 0;
        if (r < m) {
            const int beg = in_rowptr[ro + r], end = in_rowptr[ro + r + 1];
            for (int e = beg; e < end; ++e) cnt += kept(in_val, in_val64, base + e, s) ? 1 : 0;
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
                              double* __restrict__ out_val64, int64_t out_cap) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= n_pairs) return;
    const int2 ab = pairs[p];
    const int m = (int)(seq_off[ab.x + 1] - seq_off[ab.x]);
    const int64_t ro = pair_row_off[p], bin = in_off[p], bout = out_off[p];
    const unsigned below = (1u << lane) - 1u;
    for (int r = 0; r < m; ++r) {
        const int beg = in_rowptr[ro + r], end = in_rowptr[ro + r + 1];
        int64_t dst = bout + out_rowptr[ro + r];
        for (int e0 = beg; e0 < end; e0 += 32) {
            const int e = e0 + lane;
            const bool keep = e < end && kept(in_val, in_val64, bin + e, s);
            const unsigned mk = __ballot_sync(FULLM, keep);
            const int64_t o = dst + __popc(mk & below);
            if (keep && o < out_cap) {          // always, unless the select failed (reported)
                out_col[o] = in_col[bin + e];
                out_val[o] = in_val[bin + e];
                if (out_val64) out_val64[o] = in_val64[bin + e];
            }
            dst += __popc(mk);
        }
    }
}

}  // namespace

cudaError_t launch_budget_select(const int64_t* total, int64_t n_keep, double theta, bool f64, const float* val,
                                 const double* val64, SelectState* s, unsigned* hist, Status* st, int grid,
                                 cudaStream_t str) {
    k_sel_init<<<1, 256, 0, str>>>(total, n_keep, theta, f64 ? 1 : 0, s, hist, st);
    if (f64) {
        for (int pass = 0; pass < (64 + kDigitBits - 1) / kDigitBits; ++pass) {
            k_sel_hist<unsigned long long><<<grid, 256, 0, str>>>(val64, s, hist);
            k_sel_pick<unsigned long long><<<1, 32, 0, str>>>(s, hist, st);
        }
    } else {
        for (int pass = 0; pass < (32 + kDigitBits - 1) / kDigitBits; ++pass) {
            k_sel_hist<uint32_t><<<grid, 256, 0, str>>>(val, s, hist);
            k_sel_pick<uint32_t><<<1, 32, 0, str>>>(s, hist, st);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_budget_count(const int2* pairs, const int64_t* seq_off, const int64_t* pair_row_off,
                                const int64_t* in_off, const int32_t* in_rowptr, const float* in_val,
                                const double* in_val64, const SelectState* s, int64_t n_pairs, int32_t* out_rowptr,
                                int64_t* out_nnz, cudaStream_t str) {
    const int blocks = (int)((n_pairs * 32 + 255) / 256);
    if (blocks > 0)
        k_budget_count<<<blocks, 256, 0, str>>>(pairs, seq_off, pair_row_off, in_off, in_rowptr, in_val, in_val64,
                                                 s, n_pairs, out_rowptr, out_nnz);
    return cudaGetLastError();
}

cudaError_t launch_budget_copy(const int2* pairs, const int64_t* seq_off, const int64_t* pair_row_off,
                               const int64_t* in_off, const int32_t* in_rowptr, const int32_t* in_col,
                               const float* in_val, const double* in_val64, const SelectState* s, int64_t n_pairs,
                               const int64_t* out_off, const int32_t* out_rowptr, int32_t* out_col, float* out_val,
                               double* out_val64, int64_t out_cap, cudaStream_t str) {
    const int blocks = (int)((n_pairs * 32 + 255) / 256);
    if (blocks > 0)
        k_budget_copy<<<blocks, 256, 0, str>>>(pairs, seq_off, pair_row_off, in_off, in_rowptr, in_col, in_val,
                                                in_val64, s, n_pairs, out_off, out_rowptr, out_col, out_val,
                                                out_val64, out_cap);
    return cudaGetLastError();
}

}  // namespace qpk
