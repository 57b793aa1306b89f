// Internal definitions shared by the host orchestration (qp_api.cpp) and the
// kernels (qp_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace qpk {

constexpr int kWarp = 32;
constexpr int kRmax = 4;                     // DP rows per lane in a full strip
constexpr int kStripRows = kWarp * kRmax;    // 128 DP rows per strip
constexpr int kC = 16;                       // renormalisation period (steps); divides 32
constexpr int kTab = 21;                     // 20 residues + the empty row/column code
constexpr int kEmpty = 20;
constexpr int kNS = 9;                       // FP64 form: values per diagonal slot
#ifndef QP_RING_DEPTH
#define QP_RING_DEPTH 4
#endif
constexpr int kD_ring = QP_RING_DEPTH;       // FP32 form: depth of the stored-block ring (steps; a power of 2)

// Staging records a lane of the FP32 kernel may hold per strip: at most one
// per column it sweeps (L + 1), and at most R_max times a row's entry bound
// (every record holds at least one kept entry of one of its rows).
__host__ __device__ constexpr int group_capacity(int max_len, int row_cap) {
    return (max_len + 1) < kRmax * row_cap ? (max_len + 1) : kRmax * row_cap;
}

// Copies of the (odds, weight) table a block may hold in shared memory: with
// kTabCopies copies side by side, lane l reads copy l mod kTabCopies and the
// 8-byte lookups of a half-warp never share a bank.
constexpr int kTabCopies = 16;

// Per-call derived constants, written by k_setup on the device.
struct Consts {
    // (odds p(a,b)/(q(a)q(b)), Boltzmann weight exp(s(a,b)/T)), indexed [y][x]
    float2 ow[kTab * kTab];
    // FP64 form
    double tMMd, d1d, d2d, e1d, e2d, c1d, c2d, Wod, Wed;
    double pid[5], taud[5];
    double thetad;
    double oddsd[kTab * kTab];   // [y][x]
    double wd[kTab * kTab];      // [y][x]
    double logq[20];
    int32_t combine;
    int32_t err;
    int32_t n_alpha;             // letters of the alphabet (20 or 4)
};

// Host-side copy of the parameters the setup kernel needs (plain doubles).
struct RawParams {
    double pi[5], delta1, eps1, delta2, eps2;
    double emit_pair[400], emit_bg[20], end_w[5], score[400];
    double gap_open, gap_ext, temperature, threshold;
    int32_t combine;
    int32_t n_alpha;             // letters of the alphabet (20 or 4)
};

// Status words written by the kernels (device memory, zeroed per call).
struct Status {
    unsigned long long pool_used;   // entries reserved in the pool (single-family calls)
    int32_t pool_overflow;          // a reservation did not fit
    int32_t n_fallback;             // pairs queued for the FP64 form
    int32_t stage_overflow;         // a row had more entries than its staging
    int32_t bad_residue;            // encode saw a byte outside the alphabet
    int32_t work_f32;               // work counters of the persistent kernels
    int32_t work_f64;
    int32_t pad[2];
    int32_t diag[16];               // first guard event: site, strip, step, lane, exponents, m, n
    // device time stamps (ns, %globaltimer): first block start and last block
    // end of the FP32 and of the FP64 kernel (0: did not run)
    unsigned long long t_f32[2];
    unsigned long long t_f64[2];
    double theta_used;              // threshold the result was filtered at (entry budget)
    int32_t select_error;           // the budget's radix select lost its rank (logic error)
    int32_t pad2;
};

// State of the entry-budget selection (device memory; qp_budget.cu).
struct SelectState {
    unsigned long long prefix;      // high bits of the wanted key found so far
    long long rank;                 // rank from the top (0-based) among keys with that prefix
    long long total;                // entries at the call's threshold
    double theta_d;                 // threshold applied by the filter (FP64 form)
    float theta_f;                  // threshold applied by the filter (FP32 form)
    int bits_done;
    int active;                     // 1 while the entries exceed the budget
    int f64;
};

// Scalar coefficients passed by value (they live in the constant bank).
struct Coef {
    // pairs for the packed (HMM, PF) updates: gap opening (delta1, Wo), gap
    // extension (eps1, We), match continuation (1 - 2 delta1 - 2 delta2, 1),
    // gap closing (1 - eps1, 1)
    float2 k_open, k_ext, k_mm, k_close;
    float tMM, d1, d2, e1, e2, c1, c2, Wo, We;
    float pi[5];        // M, X, Y, X2, Y2
    float tau[5];
    float theta;
    float wh, wp;       // combination weights
    int32_t combine;    // 0 rms-family (sqrt(wh Ph^2 + wp Pp^2)), 1 linear (wh Ph + wp Pp)
    // FP32 kernel: bytes between table entries of consecutive row / column
    // residue codes (8 c and 8 kTab c for c table copies), and the polls of a
    // wait for another warp's strip (0: default)
    uint32_t tab_x, tab_y;
    int32_t spin_limit;
};

// One family resident on the device: inputs, plan and outputs.
struct FamDesc {
    const uint8_t* codes;          // residue codes 0..19, concatenated
    const int64_t* seq_off;        // [k+1]
    const double* seq_logq;        // [k] sum of log q over each sequence
    const int2* pairs;             // [n_pairs] (a, b), a < b
    const int64_t* pair_row_off;   // [n_pairs+1] first CSR row slot of the pair
    const int64_t* pair_strip_off; // [n_pairs+1] first strip slot of the pair
    int32_t k;
    int32_t pad0;
    int32_t* row_cnt;              // entries per CSR row, at pair_row_off[p] + r
    int64_t* chunk_off;            // absolute pool offset of each strip's entries
    int64_t* pair_nnz;             // [n_pairs]
    double* mea;                   // [n_pairs]
    double* logz_h;                // [n_pairs]
    double* logz_p;                // [n_pairs]
    float* dist;                   // [k*k]
    double* dist64;                // [k*k]
    int32_t* pair_flags;           // [n_pairs]
    // entry pool of this family (null: the launch's shared pool) and the
    // region of it that the family owns
    int2* pool;
    double* pool64;
    unsigned long long* pool_used; // entries reserved in the region
    int64_t pool_base;             // absolute first entry of the region
    int64_t pool_cap;              // entries in the region
    int32_t* n_done;               // pairs completed (atomic), may be null
};

struct Problem {
    Coef cf;
    const Consts* cst;
    const FamDesc* fams;           // family table
    const int2* items;             // [n_work] (family, pair), longest first
    int32_t n_work;
    int32_t cap;                   // staging capacity per row
    // pool of sparse entries (shared by all families)
    int2* pool;                    // (col, float bits of P)
    double* pool64;                // FP64 values (F64 form) or null
    Status* status;
    int2* fallback;                // (family, pair) items for the FP64 form
    // FP32 per-warp scratch
    float2* bst;  int64_t bst_stride;      // stored backward values
    int2* bex;    int64_t bex_stride;      // backward exponents per chunk
    float4* bnd;  int64_t bnd_stride;      // strip boundary rows (2 float4 / column)
    int2* stg;    int64_t stg_stride;      // staging records: 32 lanes x group_capacity x 32 bytes a warp
    // backward boundary rows (bck) and forward ones (bnd), per warp: one row
    // per strip when other warps or a recompute read them (checkpointed form,
    // wpp > 1), else one row.  bst / bex per warp: every strip of the pair
    // (stored form) or one strip (checkpointed form).  An item shared by a
    // group uses the buffers of the group's first warp.
    float4* bck;  int64_t bck_stride;
    int32_t ckpt;
    int32_t wpp;                   // warps per pair: 1, or 2 with at most 2 groups per block
    // FP64 per-CTA scratch
    double2* d_b; int64_t d_b_stride;      // dense backward (B_M, Zm_b)
    double* d_diag; int64_t d_diag_stride; // rotating diagonals
    int32_t* d_cnt; int64_t d_cnt_stride;  // per-row entry counts and exponents
    int2* d_stg;  double* d_stg64; int64_t d_stg_stride;
    int32_t f64_all;               // 1: F64 form over the whole item list
    int32_t f64_smem_diag;         // 1: the FP64 form's rotating diagonals in shared memory (else d_diag)
    int32_t max_len;
    int32_t tab_copies;            // copies of the emission table in shared memory: 1, or kTabCopies
    int32_t n_big;                 // wpp = 2: items [0, n_big) are shared by the two warps of a group
};

// launch wrappers (qp_kernels.cu)
// copies the parameters (host) into d_raw (device) and derives the tables
cudaError_t launch_setup(const RawParams* host_raw, RawParams* d_raw, Consts* dev_cst, cudaStream_t s);
cudaError_t launch_encode(const uint8_t* ascii, uint8_t* codes, int64_t n,
                          const int64_t* seq_off, int32_t k, double* seq_logq,
                          const Consts* cst, Status* status, cudaStream_t s);
// variant: 0 = at most 128 registers a thread (16 warps per SM),
//          1 = at most 168 registers a thread (12 warps per SM);
// P.ckpt picks the stored or the checkpointed form.
constexpr int kF32Variants = 2;
cudaError_t launch_posterior_f32(const Problem& P, int grid, int warps_per_block,
                                 cudaStream_t s, int variant = 0);
// Copies of the emission table for blocks of warps_per_block warps: kTabCopies
// when two such blocks with that many copies fit one SM's shared memory
// (smem_per_sm bytes) at sequence length max_len, else 1.
int posterior_f32_tab_copies(int warps_per_block, int max_len, int smem_per_sm);
// Scratch of the FP32 kernel for sequences up to L (elements of each buffer
// per warp), for wpp warps per pair.
struct F32Scratch {
    int64_t bst, bex, bnd, bck, stg;
    bool ckpt;
    int wpp;
    F32Scratch(int L, int cap, bool ckpt_, int wpp_ = 1) : ckpt(ckpt_), wpp(wpp_ > 1 ? wpp_ : 1) {
        const int64_t ns = (L + 1 + kStripRows - 1) / kStripRows;
        const int64_t strip = (int64_t)kStripRows * (L + 32);
        const int64_t ex = (int64_t)((L + 32 + kC - 1) / kC) * 32;
        const int64_t row = 2 * (int64_t)(L + 1);
        // pass 2 streams the stored blocks kD - 1 steps ahead of their use;
        // the blocks past a strip's end are never read (their copies are
        // zero-filled) but their addresses stay inside the buffer
        const int64_t pad = (int64_t)kD_ring * kWarp * kRmax;
        bst = (ckpt ? strip : ns * strip) + pad;
        bex = ckpt ? ex : ns * ex;
        bnd = (wpp > 1 ? ns : 1) * row;
        bck = (ckpt || wpp > 1 ? ns : 1) * row;
        stg = (int64_t)kWarp * 4 * group_capacity(L, cap);
        // (with wpp > 1 every buffer is per warp: a warp may run an item alone)
    }
    // bytes for a grid of `warps` warps
    size_t bytes(int64_t warps) const {
        return (size_t)warps * (sizeof(float2) * bst + sizeof(int2) * bex + sizeof(float4) * (bnd + bck) +
                                sizeof(int2) * stg);
    }
};
cudaError_t launch_posterior_f64(const Problem& P, int grid, cudaStream_t s);
// Whether the FP64 form keeps its rotating diagonals (3 x kNS x (L + 1)
// doubles) in shared memory at sequence length max_len.
bool posterior_f64_smem_diag(int max_len);
cudaError_t launch_compact(const int2* pairs, const int64_t* seq_off,
                           const int64_t* pair_row_off, const int64_t* pair_strip_off,
                           const int32_t* row_cnt, const int64_t* chunk_off, const int2* pool,
                           const double* pool64, int64_t n_pairs, const int64_t* pair_nnz_off,
                           int32_t* row_ptr, int32_t* col, float* val, double* val64,
                           cudaStream_t s, unsigned long long* minmax = nullptr,
                           const int32_t* overflow = nullptr);   // skip everything when *overflow
// Entry budget (qp_budget.cu): the threshold that fits n_keep entries, from
// the full CSR's values (total at *total); then the filtered row pointers and
// counts, and the filtered entries.
cudaError_t prepare_budget_kernels();       // before the first launch (not inside a capture)
cudaError_t launch_budget_select(const int64_t* total, int64_t n_keep, double theta, bool f64, const float* val,
                                 const double* val64, const unsigned long long* minmax, SelectState* s,
                                 unsigned* hist, Status* st, int grid, cudaStream_t str);
cudaError_t launch_budget_count(const int2* pairs, const int64_t* seq_off, const int64_t* pair_row_off,
                                const int64_t* in_off, const int32_t* in_rowptr, const float* in_val,
                                const double* in_val64, const SelectState* s, int64_t n_pairs, int32_t* out_rowptr,
                                int64_t* out_nnz, const Status* st, cudaStream_t str);
cudaError_t launch_budget_copy(const int2* pairs, const int64_t* seq_off, const int64_t* pair_row_off,
                               const int64_t* in_off, const int32_t* in_rowptr, const int32_t* in_col,
                               const float* in_val, const double* in_val64, const SelectState* s, int64_t n_pairs,
                               const int64_t* out_off, const int32_t* out_rowptr, int32_t* out_col, float* out_val,
                               double* out_val64, int64_t out_cap, const Status* st, cudaStream_t str);
constexpr int kBudgetBins = 16384;           // histogram bins of the select (14-bit digits)

cudaError_t launch_scan_nnz(const int64_t* pair_nnz, int64_t n_pairs, int64_t* pair_nnz_off,
                            cudaStream_t s);
int posterior_f32_regs(int variant = 0, bool ckpt = false);
int posterior_f32_occupancy(int warps_per_block, int max_len, int* blocks_per_sm, int variant = 0,
                            bool ckpt = false, int wpp = 1, int tab_copies = 1);
int posterior_f64_occupancy(int* blocks_per_sm);
size_t posterior_f32_smem(int warps_per_block, int max_len, int tab_copies = 1);

}  // namespace qpk
