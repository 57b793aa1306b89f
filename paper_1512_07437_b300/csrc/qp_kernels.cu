// Kernels of the all-pairs posterior stage (paper, Methods, stage I) for sm_103a.
//
//   k_setup            derived tables: pair-HMM odds p(a,b)/(q(a)q(b)) and
//                      partition-function weights exp(s(a,b)/T)
//   k_encode           ASCII residues -> codes 0..19, alphabet check
//   k_seqlogq          per-sequence sum of log q (turns the odds-scaled total
//                      back into the pair-HMM probability)
//   k_posterior_f32    the hot path: one warp per pair, FP32 recurrences with
//                      per-lane power-of-two rescaling; pass 1 = backward of both
//                      models (stored), pass 2 = forward of both models fused
//                      with posterior, combination, threshold, MEA, distance
//   k_posterior_f64    plain FP64 form (one CTA per pair, anti-diagonal
//                      wavefront, per-diagonal rescaling); also recomputes pairs
//                      whose FP32 range guards fired
//   k_scan_nnz / k_compact   CSR assembly from the per-strip entry chunks
//
// Model (the reading this library documents; the paper prints no model):
// a 5-state pair-HMM (M, X, Y, X2, Y2) with emissions taken relative to the
// background (M: p(a,b)/(q(a)q(b)), gap states: 1; every path emits every
// residue once, so posteriors are unchanged and the total differs by the
// product of q over both sequences), and a 3-state affine partition function
// (Zm, Ze, Zf) with Boltzmann weights.
#include "qp_internal.h"

#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include <cstdio>

namespace qpk {

#define FULL 0xffffffffu

// 2^e as a float for e in [-126, 127]; 0 below -126, 2^127 above.
__device__ __forceinline__ float pow2f(int e) {
    if (e < -126) return 0.f;
    if (e > 127) e = 127;
    return __int_as_float((e + 127) << 23);
}

// Square root with the single hardware approximation (relative error of a
// few ulp, far inside the 1e-5 posterior tolerance).
__device__ __forceinline__ float sqrt_approx(float v) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// floor(log2 v) for a positive normal float; -127 for zero / denormal.
__device__ __forceinline__ int ilog2f(float v) {
    return ((__float_as_int(v) >> 23) & 0xff) - 127;
}

// ---------------------------------------------------------------- set-up
__global__ void k_setup(const RawParams* __restrict__ rp, Consts* c) {
    const RawParams& raw = *rp;
    const int t = threadIdx.x;
    for (int idx = t; idx < kTab * kTab; idx += blockDim.x) {
        const int y = idx / kTab, x = idx % kTab;
        double o = 0.0, w = 0.0;
        if (x < raw.n_alpha && y < raw.n_alpha) {
            o = raw.emit_pair[x * 20 + y] / (raw.emit_bg[x] * raw.emit_bg[y]);
            w = exp(raw.score[x * 20 + y] / raw.temperature);
        }
        c->ow[idx] = make_float2((float)o, (float)w);
        c->oddsd[idx] = o;
        c->wd[idx] = w;
    }
    if (t < 20) c->logq[t] = t < raw.n_alpha ? log(raw.emit_bg[t]) : 0.0;
    if (t == 0) {
        c->tMMd = 1.0 - 2.0 * raw.delta1 - 2.0 * raw.delta2;
        c->d1d = raw.delta1; c->d2d = raw.delta2;
        c->e1d = raw.eps1;   c->e2d = raw.eps2;
        c->c1d = 1.0 - raw.eps1; c->c2d = 1.0 - raw.eps2;
        c->Wod = exp(raw.gap_open / raw.temperature);
        c->Wed = exp(raw.gap_ext / raw.temperature);
        for (int s = 0; s < 5; ++s) { c->pid[s] = raw.pi[s]; c->taud[s] = raw.end_w[s]; }
        c->thetad = raw.threshold;
        c->combine = raw.combine;
        c->err = 0;
        c->n_alpha = raw.n_alpha;
    }
}

cudaError_t launch_setup(const RawParams* raw, RawParams* d_raw, Consts* cst, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(d_raw, raw, sizeof(RawParams), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    k_setup<<<1, 512, 0, s>>>(d_raw, cst);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- encode
// letters -> codes: the 20 amino acids, or in nucleotide mode A, C, G, T
// (U read as T); the alphabet comes from the call's constants
__global__ void k_encode(const uint8_t* __restrict__ ascii, uint8_t* __restrict__ codes,
                         int64_t n, const Consts* __restrict__ cst, Status* st) {
    __shared__ uint8_t lut[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) lut[i] = 255;
    __syncthreads();
    const bool nuc = cst->n_alpha == 4;
    if (threadIdx.x < (nuc ? 5 : 20)) {
        const char* A = nuc ? "ACGTU" : "ACDEFGHIKLMNPQRSTVWY";
        const int c = A[threadIdx.x];
        const uint8_t code = (uint8_t)(nuc && threadIdx.x == 4 ? 3 : threadIdx.x);
        lut[c] = code;
        lut[c + 32] = code;                    // lower case
    }
    __syncthreads();
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint8_t c = lut[ascii[i]];
        if (c == 255) { bad = 1; c = 0; }
        codes[i] = c;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(&st->bad_residue, 1);
}

__global__ void k_seqlogq(const uint8_t* __restrict__ codes, const int64_t* __restrict__ off,
                          int k, const Consts* __restrict__ c, double* __restrict__ out) {
    const int w = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= k) return;
    double s = 0.0;
    for (int64_t i = off[w] + lane; i < off[w + 1]; i += 32) s += c->logq[codes[i]];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if (lane == 0) out[w] = s;
}

cudaError_t launch_encode(const uint8_t* ascii, uint8_t* codes, int64_t n,
                          const int64_t* seq_off, int32_t k, double* seq_logq,
                          const Consts* cst, Status* status, cudaStream_t s) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_encode<<<blocks, 256, 0, s>>>(ascii, codes, n, cst, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_seqlogq<<<(k * 32 + 255) / 256, 256, 0, s>>>(codes, seq_off, k, cst, seq_logq);
    return cudaGetLastError();
}

// ================================================================ FP32 path
//
// Geometry.  The DP grid has rows 0..m (row 0 and column 0 are the empty
// prefixes; their residue code is kEmpty, whose odds and weights are 0) and
// columns 0..n.  Rows are cut into strips of 128; in a strip lane l owns the
// R consecutive rows row0 + l*R + r (R = 4, fewer in a short last strip).
// A strip is swept column by column with the lanes skewed by one column:
// in the forward pass lane l is at column t - l at step t, so one step of the
// warp covers an anti-diagonal segment and the value a lane needs from the row
// above was produced by lane l-1 one step earlier (one shuffle per value).
// The row above lane 0 (the previous strip's last row) comes from a boundary
// row in global memory written by lane 31 of that strip.  The backward pass
// mirrors this (lane 31 leads, values come from lane l+1).
//
// Storage.  Pass 1 stores (B_M, Zm_b) of every cell in blocks indexed by the
// forward step T = j + l at which pass 2 visits the cell; a block is 32*R
// float2 in lane-major order, so both passes touch 256*R contiguous bytes per
// step.
//
// Scaling.  Every lane carries one power-of-two exponent per model.  All
// lanes renormalise on the same steps (every kC steps): the lane's largest
// carried value is brought into [1, 2); a lane that holds no value yet takes
// the new exponent of the nearest upstream lane that does, so a lane starts
// close to the magnitude of what will flow into it.  Values received from the
// row above are converted with 2^(e_above - e_me), which only changes on those
// steps.  A strip starts at the exponent of its boundary row's values.
// A lane whose upstream neighbour is zero for good (padding rows below row m
// in the backward pass, the missing row above the first strip in the forward
// pass) keeps the neighbour's exponent equal to its own.  Pass 1 records its
// exponent per lane and kC-step chunk; pass 2 combines the two exponents and
// the totals into one factor per lane and chunk, so the posterior of a cell
// is (F_M * factor) * B_M.
//
// Range guards (the pair is recomputed by the FP64 form when one fires), for
// lanes that own a row of the pair: a carried maximum >= 2^100 or not finite,
// an exponent gap beyond the float range, a posterior factor beyond the float
// range, a posterior above 1.001, forward and backward totals that disagree by
// more than 1e-3 in log.

struct PairCtx {
    const FamDesc* fd;
    Status* st;
    const uint8_t* x;
    const uint8_t* y;
    int m, n, p, nch;
    float2* bst;
    int2* bex;
    float4* bnd;
    float4* bck;     // checkpointed form: the backward boundary row of every strip
    int2* stg;
};

// Where one strip sweep reads and writes: the boundary row it starts from
// (null: none), the boundary row it leaves for the next strip (null: none),
// and the stored backward values and exponents of the strip.
struct StripIO {
    const float4* bnd_in;
    float4* bnd_out;
    float2* bst;
    int2* bex;
    // strips of one pair shared by several warps: the progress word of the
    // warp writing bnd_in and the value that marks its strip (null: the row
    // is complete), and this warp's own progress word for bnd_out (null: no
    // reader waits on it).  A word holds (strip tag << 32) | steps done.
    const volatile long long* wait;
    long long wait_tag;
    volatile long long* pub;
    long long pub_tag;
};

constexpr long long kStepsDone = 0x7fffffffLL;     // "strip complete" in a progress word
constexpr long long kPass2Tag = 1LL << 20;         // strip tags of pass 2 start here
constexpr int kSpinLimit = 1 << 22;                 // bounded wait for a progress word

// Waits (warp-uniform) until the progress word reaches need.  A wait that runs
// out sets the sync guard (bit 12), so the pair goes to the FP64 form; it
// never hangs, and once the guard is set the warp waits no more (the pair's
// FP32 values are discarded anyway).
__device__ __forceinline__ void wait_progress(const volatile long long* w, long long need, int& flag) {
    if (!w || (flag & (1 << 12))) return;
    int it = 0;
    while (*w < need) {
        if (++it > kSpinLimit) { flag |= (1 << 12); return; }
        __nanosleep(64);
    }
    __threadfence_block();
}

// Publishes this warp's progress (called by the lane that writes the row).
__device__ __forceinline__ void publish_progress(volatile long long* w, long long v) {
    __threadfence_block();
    *w = v;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Kernel time stamps without events (they also work inside a CUDA graph):
// the first block to start sets ts[0], every block raises ts[1] at its end.
__device__ __forceinline__ void stamp_begin(unsigned long long* ts) {
    if (threadIdx.x == 0) atomicCAS(&ts[0], 0ull, global_ns());
}
__device__ __forceinline__ void stamp_end(unsigned long long* ts) {
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(&ts[1], global_ns());
}

constexpr float kBig = 1.2676506002282294e30f;   // 2^100
constexpr int kNoExp = (int)0x80000000;           // "no exponent yet" in the fill scan

// Records the first guard event of a launch (site code and context) so that a
// fallback can be explained from the host.
__device__ __forceinline__ void note_guard(Status* st, int site, int s, int t, int lane, int a, int b,
                                           int c, int d, int m, int n) {
    if (atomicCAS(&st->diag[0], 0, site) == 0) {
        st->diag[1] = s; st->diag[2] = t; st->diag[3] = lane;
        st->diag[4] = a; st->diag[5] = b; st->diag[6] = c; st->diag[7] = d;
        st->diag[8] = m; st->diag[9] = n;
    }
}

// Reasons an FP32 pair is handed to the FP64 form (pair_flags bits 2..).
enum : int {
    kGuardRange = 1 << 2,    // a carried maximum >= 2^100 or not finite
    kGuardGap = 1 << 3,      // exponent gap between neighbouring lanes beyond float range
    kGuardFactor = 1 << 4,   // posterior factor 2^(eF + eB - eZ) beyond float range
    kGuardPost = 1 << 5,     // a posterior above 1.001
    kGuardAgreeH = 1 << 6,   // pair-HMM forward and backward totals disagree
    kGuardAgreeP = 1 << 7,   // partition-function totals disagree
    kGuardTotal = 1 << 8,    // a total is zero or not finite
    kGuardCorner = 1 << 9,   // a corner cell was reached with a non-zero exponent
    kGuardStage = 1 << 10,   // a row exceeded its staging capacity
    kGuardPool = 1 << 11,    // the entry pool region was full
    kGuardSync = 1 << 12,    // a wait for another warp's strip ran out
};

// ---------------------------------------------------------------- async copies
// cp.async moves the stored backward blocks and the boundary row into a small
// per-warp shared-memory ring kD steps ahead of their use.  Every lane copies
// and later reads only its own bytes, so waiting on its own copy groups is the
// only synchronisation needed.  A source size of 0 fills the slot with zeros.
constexpr int kD = 4;



__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(src), "r"(bytes));
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, int bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(src), "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// per-warp shared memory: stored-block ring, boundary ring, column residues
struct WarpSmem {
    float2* ring_b;   // [kD][kWarp * kRmax]
    float4* ring_e;   // [kD][2]
    uint8_t* sy;      // [max_len]
};

constexpr int kOwBytes = ((kTab * kTab * 8 + 255) / 256) * 256;

constexpr int kYPad = 33;   // empty codes before column 1 of the staged residues

__host__ __device__ constexpr int warp_smem_bytes(int max_len) {
    return kD * kWarp * kRmax * 8 + kD * 32 + ((max_len + 2 * kYPad + 15) / 16) * 16;
}

// Predicated stores without a branch: the address is only used when p holds.
__device__ __forceinline__ void st_pred_v4(bool p, float4* a, float x, float y, float z, float w) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q st.global.v4.f32 [%1], {%2, %3, %4, %5};\n\t}"
                 ::"r"((int)p), "l"(a), "f"(x), "f"(y), "f"(z), "f"(w));
}
__device__ __forceinline__ void st_pred_v2i(bool p, int2* a, int x, int y) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q st.global.v2.s32 [%1], {%2, %3};\n\t}"
                 ::"r"((int)p), "l"(a), "r"(x), "r"(y));
}

// Runs steps 0 .. nsteps-1 of a strip: the steps t_a and t_b (-1: none) with
// the corner-cell copy of the step, all others with the plain copy, which is
// the only one inside the hot loop.
template <class Step>
__device__ __forceinline__ void run_steps(int nsteps, int t_a, int t_b, Step& step) {
    int t = 0;
    while (t < nsteps) {
        int stop = nsteps;
        if (t_a >= t && t_a < stop) stop = t_a;
        if (t_b >= t && t_b < stop) stop = t_b;
        for (; t < stop; ++t) step(t, std::false_type{});
        if (t < nsteps) {
            step(t, std::true_type{});
            ++t;
        }
    }
}

// ---------------------------------------------------------------- pass 1
template <int R, bool SPEC, bool STORE>
__device__ __forceinline__ void bwd_step(
    const Coef& cf, const float2* __restrict__ s_ow, const PairCtx& c, int j, bool act, int lane,
    int Lend, int rend, bool first_strip, int yc,
    float2 (&DD)[R], float2& tV, float& tX2, float2 (&HB)[R], float (&BY2o)[R], const int (&xo)[R],
    float2& dDD, float2 cv, float2* __restrict__ bst_strip,
    const float4* __restrict__ ebnd, float4* __restrict__ bnd_out, int eH, int eP,
    float& Zh, float& Zp, int& eZh, int& eZp, int& flag)
{
    const int n = c.n;
    // values of the row below (lane+1's top row; lane 31: the boundary row):
    // (B_M, Zm_b) weighted by the emission of their cell, (B_X, Ze_b), B_X2
    float2 rDD = make_float2(__shfl_down_sync(FULL, DD[0].x, 1), __shfl_down_sync(FULL, DD[0].y, 1));
    float2 rV = make_float2(__shfl_down_sync(FULL, tV.x, 1), __shfl_down_sync(FULL, tV.y, 1));
    float rX2 = __shfl_down_sync(FULL, tX2, 1);
    if (lane == 31) {
        const float4 v0 = ebnd[0], v1 = ebnd[1];
        rDD = make_float2(v0.x, v0.y); rV = make_float2(v0.z, v0.w); rX2 = v1.x;
    }
    rDD = __fmul2_rn(rDD, cv); rV = __fmul2_rn(rV, cv); rX2 *= cv.x;
    const float2* __restrict__ owr = s_ow + yc * kTab;
    float2 D = dDD;
    float2 V = rV;
    float X2b = rX2;
    dDD = rDD;
    float2* blk = bst_strip + (int64_t)(j + lane) * (kWarp * R) + lane * R;
#pragma unroll
    for (int r = R - 1; r >= 0; --r) {
        const float2 H = HB[r];             // (B_Y, Zf_b) of the cell to the right
        const float Y2b = BY2o[r];
        // (B_X, Ze_b) and (B_Y, Zf_b) of this cell: gap closed by the match
        // below-right, or extended
        // (the carried operand enters last: one operation per row on the
        // vertical chain)
        const float2 cD = __fmul2_rn(cf.k_close, D);
        float2 nV = __ffma2_rn(cf.k_ext, V, cD);
        float2 nH = __ffma2_rn(cf.k_ext, H, cD);
        const float cX2 = cf.c2 * D.x;
        float BX2 = fmaf(cf.e2, X2b, cX2);
        float BY2 = fmaf(cf.e2, Y2b, cX2);
        // (B_M, Zm_b): continue the match, or open a gap
        float2 B = __ffma2_rn(cf.k_open, __fadd2_rn(V, H), __fmul2_rn(cf.k_mm, D));
        B.x = fmaf(cf.d2, X2b + Y2b, B.x);
        if (SPEC) {
            if (lane == Lend && r == rend && j == n) {
                // end of every path: B_s(m, n) = tau_s; the partition function ends with weight 1
                B = make_float2(cf.tau[0], 1.f);
                nV = make_float2(cf.tau[1], 1.f);
                nH = make_float2(cf.tau[2], 1.f);
                BX2 = cf.tau[3]; BY2 = cf.tau[4];
                if (eH != 0 || eP != 0) flag |= kGuardCorner;
            }
            if (first_strip && lane == 0 && r == 0 && j == 0) {
                // totals seen from the start: pi_s times the first emission of s
                Zh = cf.pi[0] * D.x + cf.pi[1] * V.x + cf.pi[2] * H.x + cf.pi[3] * X2b + cf.pi[4] * Y2b;
                Zp = B.y;
                eZh = eH; eZp = eP;
            }
        }
        const float2 w = owr[xo[r]];
        if (STORE && act) blk[r] = B;
        D = DD[r];
        V = nV; X2b = BX2;
        DD[r] = __fmul2_rn(w, B);
        HB[r] = nH; BY2o[r] = BY2;
        if (r == 0) { tV = nV; tX2 = BX2; }
    }
    {
        const bool wr = (lane == 0) && act && (bnd_out != nullptr);
        float4* q = bnd_out + 2 * j;
        st_pred_v4(wr, q, DD[0].x, DD[0].y, tV.x, tV.y);
        st_pred_v4(wr, q + 1, tX2, 0.f, __int_as_float(eH), __int_as_float(eP));
    }
}

template <int R, bool STORE>
__device__ __forceinline__ void bwd_strip(const Coef& cf, const float2* __restrict__ s_ow, const PairCtx& c,
                          const WarpSmem& ws, int s, int nstrips, const StripIO& io, float& Zh, float& Zp,
                          int& eZh, int& eZp, int& flag)
{
    const int lane = threadIdx.x & 31;
    const int m = c.m, n = c.n;
    const int row0 = s * kStripRows;
    const bool last_strip = (s == nstrips - 1);
    const bool first_strip = (s == 0);
    int xo[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = row0 + lane * R + r;
        xo[r] = (i >= 1 && i <= m) ? (int)__ldg(c.x + i - 1) : kEmpty;
    }
    // carried across steps: the diagonal outflow (B_M, Zm_b) and the
    // horizontal outflows (B_Y, Zf_b), B_Y2 of every row; the vertical
    // outflows (B_X, Ze_b), B_X2 of the top row (they go to the lane above)
    float2 DD[R], HB[R];
    float BY2o[R];
    float2 tV = make_float2(0.f, 0.f);
    float tX2 = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) { DD[r] = HB[r] = make_float2(0.f, 0.f); BY2o[r] = 0.f; }
    float2 dDD = make_float2(0.f, 0.f);
    // the boundary row below this strip (none for the last strip)
    const float4* bnd_in = io.bnd_in;
    float4* bnd_out = io.bnd_out;
    const bool owns_row = row0 + lane * R <= m;
    // the neighbour below is zero for good: padding rows, or no strip below
    const bool up_zero = (lane == 31) ? (bnd_in == nullptr) : (row0 + (lane + 1) * R > m);
    // starting exponent: the boundary row's exponent, moved to the magnitude of
    // its values at column n (every lane starts there)
    int eH = 0, eP = 0, eUpH = 0, eUpP = 0;
    // the row below is written by another warp: wait for its first columns
    wait_progress(io.wait, io.wait_tag | (64 + kD), flag);
    if (bnd_in) {
        const float4 v0 = bnd_in[2 * n], v1 = bnd_in[2 * n + 1];
        eUpH = __float_as_int(v1.z); eUpP = __float_as_int(v1.w);
        const float bh = fmaxf(v0.x, fmaxf(v0.z, v1.x)), bp = fmaxf(v0.y, v0.w);
        eH = eUpH + (bh > 0.f ? max(-126, min(126, ilog2f(bh))) : 0);
        eP = eUpP + (bp > 0.f ? max(-126, min(126, ilog2f(bp))) : 0);
        if (lane != 31) { eUpH = eH; eUpP = eP; }
    }
    float2 cv = make_float2(pow2f(eUpH - eH), pow2f(eUpP - eP));
    const int Lend = last_strip ? (m - row0) / R : -1;
    const int rend = last_strip ? (m - row0) % R : -1;
    const int t_end = last_strip ? 31 - Lend : -1;
    const int t_start = first_strip ? n + 31 : -1;
    // column n - t of the row below is written at the writer's step t + 31 and
    // fetched here kD - 1 steps ahead: stay 16 + kD + 32 steps behind it
    float2* bst_strip = io.bst;
    int2* bex = io.bex;
    const int nsteps = n + 32;
    // lane 31 streams the boundary row (column n - t at step t) into its ring
    const bool streams = (lane == 31) && (bnd_in != nullptr);
    auto fetch = [&](int t) {
        if (streams) {
            const int jb = n - t;
            const bool ok = (t < nsteps) && jb >= 0;
            const float4* src = bnd_in + 2 * (ok ? jb : 0);
            float4* dst = ws.ring_e + 2 * (t & (kD - 1));
            cp_async16(dst, src, ok ? 16 : 0);
            cp_async16(dst + 1, src + 1, ok ? 16 : 0);
        }
        cp_async_commit();
    };
    // without a strip below, lane 31 reads zeros from a ring slot
    if (!streams && lane == 31) {
#pragma unroll
        for (int q = 0; q < 2 * kD; ++q) ws.ring_e[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int t = 0; t < kD - 1; ++t) fetch(t);
    // column residue of the lane, one step ahead (padded: no range check)
    auto ycode = [&](int j) { return (int)ws.sy[j + kYPad - 1]; };
    int yc = ycode(n + 31 - lane);
    // one step; SPEC: the step holds a corner cell (its own copy of the step,
    // kept out of the loop below)
    auto step = [&](int t, auto spec) {
        constexpr bool SPEC = decltype(spec)::value;
        const int ph = t & (kC - 1);
        if (ph == 0) {
            wait_progress(io.wait, io.wait_tag | (t + 16 + kD + 32), flag);
            if (io.pub && lane == 0) publish_progress(io.pub, io.pub_tag | t);
        }
        fetch(t + kD - 1);
        cp_async_wait<kD - 1>();
        const float4* ebnd = ws.ring_e + 2 * (streams ? (t & (kD - 1)) : 0);
        const int j = n + 31 - lane - t;
        const bool act = (j >= 0) && (j <= n);
        if (ph == 0) {
            // renormalise: bring the lane's largest carried value into [1, 2)
            float mh = fmaxf(fmaxf(dDD.x, tV.x), tX2), mp = fmaxf(dDD.y, tV.y);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                mh = fmaxf(mh, fmaxf(DD[r].x, fmaxf(HB[r].x, BY2o[r])));
                mp = fmaxf(mp, fmaxf(DD[r].y, HB[r].y));
            }
            const bool live = owns_row && (j >= -1) && (j <= n);
            if (live && !(mh < kBig && mp < kBig)) flag |= kGuardRange;
            const int kh = mh > 0.f ? max(-126, min(126, ilog2f(mh))) : 0;
            const int kp = mp > 0.f ? max(-126, min(126, ilog2f(mp))) : 0;
            const float2 sc = make_float2(pow2f(-kh), pow2f(-kp));
#pragma unroll
            for (int r = 0; r < R; ++r) {
                DD[r] = __fmul2_rn(DD[r], sc); HB[r] = __fmul2_rn(HB[r], sc); BY2o[r] *= sc.x;
            }
            dDD = __fmul2_rn(dDD, sc); tV = __fmul2_rn(tV, sc); tX2 *= sc.x;
            int fh = mh > 0.f ? eH + kh : (lane == 31 ? eH : kNoExp);
            int fp = mp > 0.f ? eP + kp : (lane == 31 ? eP : kNoExp);
            // a lane without state takes the new exponent of the nearest lane
            // below it that has state (lane 31 keeps its own)
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int vh = __shfl_down_sync(FULL, fh, d), vp = __shfl_down_sync(FULL, fp, d);
                if (lane + d < 32) {
                    if (fh == kNoExp) fh = vh;
                    if (fp == kNoExp) fp = vp;
                }
            }
            eH = fh; eP = fp;
            const int uH = __shfl_down_sync(FULL, eH, 1);
            const int uP = __shfl_down_sync(FULL, eP, 1);
            if (lane != 31) { eUpH = uH; eUpP = uP; }
            if (up_zero) { eUpH = eH; eUpP = eP; }
            if (STORE) bex[(t / kC) * 32 + lane] = make_int2(eH, eP);
            const int gh = eUpH - eH, gp = eUpP - eP;
            if (live && (gh > 127 || gp > 127)) {
                flag |= kGuardGap;
                note_guard(c.st, 1, s, t, lane, eH, eUpH, eP, eUpP, m, n);
            }
            cv = make_float2(pow2f(gh), pow2f(gp));
        } else if (ph == 1) {
            // the boundary row's exponent changes on these steps
            if (streams && n - t >= 0) {
                const float4 e = ebnd[1];
                eUpH = __float_as_int(e.z); eUpP = __float_as_int(e.w);
                const int gh = eUpH - eH, gp = eUpP - eP;
                if (owns_row && (gh > 127 || gp > 127)) {
                    flag |= kGuardGap;
                    note_guard(c.st, 2, s, t, lane, eH, eUpH, eP, eUpP, m, n);
                }
                cv = make_float2(pow2f(gh), pow2f(gp));
            }
        }
        const int yc_now = yc;
        yc = ycode(j - 1);
        bwd_step<R, SPEC, STORE>(cf, s_ow, c, j, act, lane, Lend, rend, first_strip, yc_now, DD, tV, tX2,
                                 HB, BY2o, xo, dDD, cv, bst_strip, ebnd, bnd_out, eH, eP, Zh, Zp, eZh, eZp,
                                 flag);
    };
    run_steps(nsteps, t_start, t_end, step);
    cp_async_wait<0>();
    if (io.pub && lane == 0) publish_progress(io.pub, io.pub_tag | kStepsDone);
}

// ---------------------------------------------------------------- pass 2
struct FwdOut {      // per-lane results captured at the end corner
    float Zh, Zp;
    int eZh, eZp;
    int A;
};

template <int R, bool SPEC, bool LIN>
__device__ __forceinline__ void fwd_step(
    const Coef& cf, const float2* __restrict__ s_ow, const PairCtx& c, int j, bool act, int lane,
    int Lend, int rend, bool first_strip, int yc,
    float2 (&MZ)[R], float2& lV, float& lX2, float2 (&HY)[R], float (&Y2i)[R], int (&Aa)[R], int (&cnt)[R],
    const int (&xo)[R], float2& uMZ, int& uA, float2 cv, float2 ps, float scaleA,
    const float2* __restrict__ bs, const float4* __restrict__ ebnd, float4* __restrict__ bnd_out,
    int2* __restrict__ stg, int cap, int eH, int eP, float& pmax, FwdOut& fo, int& flag)
{
    const int n = c.n;
    // values of the row above (lane-1's bottom row; lane 0: the boundary row):
    // the diagonal outflow (M, Zm), the vertical outflow (X, Ze), X2, MEA
    float2 rMZ = make_float2(__shfl_up_sync(FULL, MZ[R - 1].x, 1), __shfl_up_sync(FULL, MZ[R - 1].y, 1));
    float2 rV = make_float2(__shfl_up_sync(FULL, lV.x, 1), __shfl_up_sync(FULL, lV.y, 1));
    float rX2 = __shfl_up_sync(FULL, lX2, 1);
    int rA = __shfl_up_sync(FULL, Aa[R - 1], 1);
    if (lane == 0) {
        // the previous strip's last row (zeros above the first strip)
        const float4 v0 = ebnd[0], v1 = ebnd[1];
        rMZ = make_float2(v0.x, v0.y); rV = make_float2(v0.z, v0.w); rX2 = v1.x; rA = __float_as_int(v1.y);
    }
    rMZ = __fmul2_rn(rMZ, cv); rV = __fmul2_rn(rV, cv); rX2 *= cv.x;
    const float2* __restrict__ owr = s_ow + yc * kTab;
    float2 dMZ = uMZ;
    int dA = uA;
    float2 aV = rV;
    float aX2 = rX2;
    int aA = rA;
    uMZ = rMZ; uA = rA;
    float Pv[R];
    bool any = false;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float2 w = owr[xo[r]];
        const float2 F = __fmul2_rn(w, dMZ);     // (M, Zm) of the cell
        const float2 V = aV, H = HY[r];         // (X, Ze), (Y, Zf) of the cell
        const float FX2 = aX2, FY2 = Y2i[r];
        // outflows: gaps opened from the match or extended; the match
        // continued or closing a gap (diagonal, weighted by the next cell's
        // emission when it is read)
        // (the carried operand enters last: one operation per row on the
        // vertical chain)
        const float2 oF = __fmul2_rn(cf.k_open, F);
        float2 nV = __ffma2_rn(cf.k_ext, V, oF);
        float2 nH = __ffma2_rn(cf.k_ext, H, oF);
        const float oX2 = cf.d2 * F.x;
        float nX2 = fmaf(cf.e2, FX2, oX2);
        float nY2 = fmaf(cf.e2, FY2, oX2);
        float2 nMZ = __ffma2_rn(cf.k_close, __fadd2_rn(V, H), __fmul2_rn(cf.k_mm, F));
        nMZ.x = fmaf(cf.c2, FX2 + FY2, nMZ.x);
        // posteriors of the cell and their combination
        const float2 Pq2 = __fmul2_rn(__fmul2_rn(F, ps), bs[(r >> 1) * 2 * kWarp + (r & 1)]);
        float P;
        if (!LIN) {         // the root-mean-square family (the default)
            const float2 sq = __fmul2_rn(Pq2, Pq2);
            P = sqrt_approx(fmaf(cf.wh, sq.x, cf.wp * sq.y));
        } else {            // linear combinations (mean, one model alone)
            P = fmaf(cf.wh, Pq2.x, cf.wp * Pq2.y);
        }
        pmax = fmaxf(pmax, P);
        Pv[r] = P;
        any |= (P >= cf.theta);
        // maximum expected accuracy, fixed point (scaleA * P < 2^22)
        const int Pq = __float_as_int(fmaf(P, scaleA, 12582912.0f)) - 0x4B400000;
        int nA = __vimax3_s32(dA + Pq, aA, Aa[r]);
        if (SPEC) {
            if (first_strip && lane == 0 && r == 0 && j == 0) {
                // empty prefixes: the start distribution and the empty alignment
                nMZ = make_float2(cf.pi[0], 1.f);
                nV = make_float2(cf.pi[1], cf.Wo);
                nH = make_float2(cf.pi[2], cf.Wo);
                nX2 = cf.pi[3]; nY2 = cf.pi[4];
                nA = 0;
                if (eH != 0 || eP != 0) flag |= kGuardCorner;
            }
            if (lane == Lend && r == rend && j == n) {
                fo.Zh = cf.tau[0] * F.x + cf.tau[1] * V.x + cf.tau[2] * H.x + cf.tau[3] * FX2 + cf.tau[4] * FY2;
                fo.Zp = F.y + V.y + H.y;
                fo.eZh = eH; fo.eZp = eP;
                fo.A = nA;
            }
        }
        dMZ = MZ[r]; dA = Aa[r];
        aV = nV; aX2 = nX2; aA = nA;
        MZ[r] = nMZ; HY[r] = nH; Y2i[r] = nY2; Aa[r] = nA;
        if (r == R - 1) { lV = nV; lX2 = nX2; }
    }
    // entries at or above the threshold: one vote per step (long rows have
    // few), then a predicated store per row without a branch
    if (__any_sync(FULL, any)) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const bool keep = Pv[r] >= cf.theta;
            const int q = cnt[r];
            st_pred_v2i(keep && q < cap, stg + ((lane * R + r) * cap + q), j - 1, __float_as_int(Pv[r]));
            cnt[r] = q + (keep ? 1 : 0);
        }
    }
    {
        const bool wr = (lane == 31) && act && (bnd_out != nullptr);
        float4* q = bnd_out + 2 * j;
        st_pred_v4(wr, q, MZ[R - 1].x, MZ[R - 1].y, lV.x, lV.y);
        st_pred_v4(wr, q + 1, lX2, __int_as_float(Aa[R - 1]), __int_as_float(eH), __int_as_float(eP));
    }
}

template <int R, bool LIN>
__device__ __forceinline__ void fwd_strip(const Problem& Pb, const float2* __restrict__ s_ow, const PairCtx& c,
                          const WarpSmem& ws, int s, int nstrips, const StripIO& io, float invZh,
                          float invZp, int eZh, int eZp, float scaleA, float& pmax, FwdOut& fo,
                          int64_t& pair_tot, int& flag)
{
    const Coef& cf = Pb.cf;
    const int lane = threadIdx.x & 31;
    const int m = c.m, n = c.n;
    const int row0 = s * kStripRows;
    const bool last_strip = (s == nstrips - 1);
    const bool first_strip = (s == 0);
    // rows outside 1..m get the empty code: their posteriors are 0, below any
    // threshold, so they never produce an entry
    int xo[R];
    int cnt[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = row0 + lane * R + r;
        xo[r] = (i >= 1 && i <= m) ? (int)__ldg(c.x + i - 1) : kEmpty;
        cnt[r] = 0;
    }
    // carried across steps: the diagonal outflow (M, Zm) and the horizontal
    // outflows (Y, Zf), Y2 of every row; the vertical outflows (X, Ze), X2 of
    // the bottom row (they go to the lane below)
    float2 MZ[R], HY[R];
    float Y2i[R];
    float2 lV = make_float2(0.f, 0.f);
    float lX2 = 0.f;
    int Aa[R];
#pragma unroll
    for (int r = 0; r < R; ++r) { MZ[r] = HY[r] = make_float2(0.f, 0.f); Y2i[r] = 0.f; Aa[r] = 0; }
    float2 uMZ = make_float2(0.f, 0.f);
    int uA = 0;
    const float4* bnd_in = io.bnd_in;
    float4* bnd_out = io.bnd_out;
    const bool owns_row = row0 + lane * R <= m;
    const bool up_zero = (lane == 0) && (bnd_in == nullptr);
    // starting exponent: the boundary row's exponent, moved to the magnitude of
    // its values at column 0 (every lane starts there)
    int eH = 0, eP = 0, eUpH = 0, eUpP = 0;
    // the row above is written by another warp: wait for its first columns
    wait_progress(io.wait, io.wait_tag | (64 + kD), flag);
    if (bnd_in) {
        const float4 v0 = bnd_in[0], v1 = bnd_in[1];
        eUpH = __float_as_int(v1.z); eUpP = __float_as_int(v1.w);
        const float bh = fmaxf(v0.x, fmaxf(v0.z, v1.x)), bp = fmaxf(v0.y, v0.w);
        eH = eUpH + (bh > 0.f ? max(-126, min(126, ilog2f(bh))) : 0);
        eP = eUpP + (bp > 0.f ? max(-126, min(126, ilog2f(bp))) : 0);
        if (lane != 0) { eUpH = eH; eUpP = eP; }
    }
    float2 cv = make_float2(pow2f(eUpH - eH), pow2f(eUpP - eP));
    const int Lend = last_strip ? (m - row0) / R : -1;
    const int rend = last_strip ? (m - row0) % R : -1;
    const int t_end = last_strip ? n + Lend : -1;
    const int t_start = first_strip ? 0 : -1;
    const float2* bst_strip = io.bst;
    const int2* bex = io.bex;
    int2* stg = c.stg;
    const int cap = Pb.cap;
    const int nsteps = n + 32;
    const int c2 = n & (kC - 1);
    // posterior factor of this lane: 2^(eF + eB - eZ) / Z for each model
    int2 eb = bex[((n + 31) / kC) * 32 + lane];
    float2 ps;
    int t_ps = 0;
    auto ps_update = [&]() {
        const int Eh = eH + eb.x - eZh, Ep = eP + eb.y - eZp;
        const int j0 = t_ps - lane;      // first column of the chunk for this lane
        if (owns_row && (Eh > 126 || Ep > 126) && j0 <= n && j0 + kC >= 0) {
            flag |= kGuardFactor;
            note_guard(c.st, 5, s, t_ps, lane, eH, eb.x, eP, eb.y, m, n);
        }
        ps = make_float2(pow2f(Eh) * invZh, pow2f(Ep) * invZp);
    };
    ps_update();
    // ring streams: this lane's stored block of step T, and (lane 0) the
    // boundary row column T
    const bool streams = (lane == 0) && (bnd_in != nullptr);
    const float2* bst_lane = bst_strip + lane * R;
    // ring slot layout: the lane's values of rows 2h, 2h+1 (16 bytes) at
    // h * 64 + lane * 2 (float2 units), so that the 16-byte reads of
    // consecutive lanes hit consecutive banks; one row: lane * 1
    float2* ring_lane = ws.ring_b + (R == 1 ? lane : lane * 2);
    auto fetch = [&](int T) {
        // the block of step T exists for this lane when 0 <= T - lane <= n
        const bool ok = (unsigned)(T - lane) <= (unsigned)n;
        const float2* src = ok ? bst_lane + T * (kWarp * R) : bst_lane;
        float2* dst = ring_lane + (T & (kD - 1)) * (kWarp * kRmax);
        if (R == 1) {
            cp_async8(dst, src, ok ? 8 : 0);
        } else {
#pragma unroll
            for (int h = 0; h < R / 2; ++h) cp_async16(dst + h * 2 * kWarp, src + 2 * h, ok ? 16 : 0);
        }
        if (streams) {
            const bool okb = (T < nsteps) && T <= n;
            const float4* sb = bnd_in + 2 * (okb ? T : 0);
            float4* db = ws.ring_e + 2 * (T & (kD - 1));
            cp_async16(db, sb, okb ? 16 : 0);
            cp_async16(db + 1, sb + 1, okb ? 16 : 0);
        }
        cp_async_commit();
    };
    // lanes without a boundary read zeros from their ring slots
    if (!streams && lane == 0) {
#pragma unroll
        for (int q = 0; q < 2 * kD; ++q) ws.ring_e[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int t = 0; t < kD - 1; ++t) fetch(t);
    auto ycode = [&](int j) { return (int)ws.sy[j + kYPad - 1]; };
    int yc = ycode(-lane);
    // one step; SPEC: the step holds a corner cell (its own copy of the step,
    // kept out of the loop below)
    auto step = [&](int t, auto spec) {
        constexpr bool SPEC = decltype(spec)::value;
        // column T of the row above is written at the writer's step T + 31 and
        // fetched here kD - 1 steps ahead: stay 16 + kD + 32 steps behind it
        if ((t & (kC - 1)) == 0) {
            wait_progress(io.wait, io.wait_tag | (t + 16 + kD + 32), flag);
            if (io.pub && lane == 31) publish_progress(io.pub, io.pub_tag | t);
        }
        fetch(t + kD - 1);
        cp_async_wait<kD - 1>();
        const float2* bs = ws.ring_b + (t & (kD - 1)) * (kWarp * kRmax) + (R == 1 ? lane : lane * 2);
        const float4* ebnd = ws.ring_e + 2 * (streams ? (t & (kD - 1)) : 0);
        const int j = t - lane;
        const bool act = (j >= 0) && (j <= n);
        const int ph = (t - c2) & (kC - 1);
        if (ph == 0) {
            float mh = fmaxf(fmaxf(uMZ.x, lV.x), lX2), mp = fmaxf(uMZ.y, lV.y);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                mh = fmaxf(mh, fmaxf(MZ[r].x, fmaxf(HY[r].x, Y2i[r])));
                mp = fmaxf(mp, fmaxf(MZ[r].y, HY[r].y));
            }
            const bool live = owns_row && (j >= 0) && (j <= n + 1);
            if (live && !(mh < kBig && mp < kBig)) flag |= kGuardRange;
            const int kh = mh > 0.f ? max(-126, min(126, ilog2f(mh))) : 0;
            const int kp = mp > 0.f ? max(-126, min(126, ilog2f(mp))) : 0;
            const float2 sc = make_float2(pow2f(-kh), pow2f(-kp));
#pragma unroll
            for (int r = 0; r < R; ++r) {
                MZ[r] = __fmul2_rn(MZ[r], sc); HY[r] = __fmul2_rn(HY[r], sc); Y2i[r] *= sc.x;
            }
            uMZ = __fmul2_rn(uMZ, sc); lV = __fmul2_rn(lV, sc); lX2 *= sc.x;
            int fh = mh > 0.f ? eH + kh : (lane == 0 ? eH : kNoExp);
            int fp = mp > 0.f ? eP + kp : (lane == 0 ? eP : kNoExp);
            // a lane without state takes the new exponent of the nearest lane
            // above it that has state (lane 0 keeps its own)
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int vh = __shfl_up_sync(FULL, fh, d), vp = __shfl_up_sync(FULL, fp, d);
                if (lane >= d) {
                    if (fh == kNoExp) fh = vh;
                    if (fp == kNoExp) fp = vp;
                }
            }
            eH = fh; eP = fp;
            const int uH = __shfl_up_sync(FULL, eH, 1);
            const int uP = __shfl_up_sync(FULL, eP, 1);
            if (lane != 0) { eUpH = uH; eUpP = uP; }
            if (up_zero) { eUpH = eH; eUpP = eP; }
            const int gh = eUpH - eH, gp = eUpP - eP;
            if (live && (gh > 127 || gp > 127)) {
                flag |= kGuardGap;
                note_guard(c.st, 3, s, t, lane, eH, eUpH, eP, eUpP, m, n);
            }
            cv = make_float2(pow2f(gh), pow2f(gp));
            const int kc = (n + 31 - t) / kC;
            eb = bex[kc * 32 + lane];
            t_ps = t;
            ps_update();
        } else if (ph == 1) {
            if (streams && t <= n) {
                const float4 e = ebnd[1];
                eUpH = __float_as_int(e.z); eUpP = __float_as_int(e.w);
                const int gh = eUpH - eH, gp = eUpP - eP;
                if (gh > 127 || gp > 127) {
                    flag |= kGuardGap;
                    note_guard(c.st, 4, s, t, lane, eH, eUpH, eP, eUpP, m, n);
                }
                cv = make_float2(pow2f(gh), pow2f(gp));
            }
        }
        const int yc_now = yc;
        yc = ycode(j + 1);
        fwd_step<R, SPEC, LIN>(cf, s_ow, c, j, act, lane, Lend, rend, first_strip, yc_now, MZ, lV, lX2, HY, Y2i,
                          Aa, cnt, xo, uMZ, uA, cv, ps, scaleA, bs, ebnd, bnd_out, stg, cap, eH, eP, pmax,
                          fo, flag);
    };
    run_steps(nsteps, t_start, t_end, step);
    cp_async_wait<0>();
    if (io.pub && lane == 31) publish_progress(io.pub, io.pub_tag | kStepsDone);
    // ---- flush this strip's entries into the pool (row-major, columns ascending)
    int tot = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (cnt[r] > cap) { flag |= kGuardStage; atomicExch(&Pb.status->stage_overflow, 1); cnt[r] = cap; }
        tot += cnt[r];
    }
    int incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += v;
    }
    const int strip_tot = __shfl_sync(FULL, incl, 31);
    const FamDesc& fd = *c.fd;
    unsigned long long off = 0;
    if (lane == 0 && strip_tot > 0) off = atomicAdd(fd.pool_used, (unsigned long long)strip_tot);
    off = __shfl_sync(FULL, off, 0);
    const bool fits = (int64_t)off + strip_tot <= fd.pool_cap;
    if (!fits) { flag |= kGuardPool; if (lane == 0) atomicExch(&Pb.status->pool_overflow, 1); }
    const int64_t base = fd.pool_base + (int64_t)off;
    int w = incl - tot;
    const int64_t row_slot = fd.pair_row_off[c.p];
    int2* pool = fd.pool ? fd.pool : Pb.pool;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = row0 + lane * R + r;
        if (i >= 1 && i <= m) fd.row_cnt[row_slot + i - 1] = cnt[r];
        if (fits) {
            const int2* src = stg + (lane * R + r) * cap;
            for (int q = 0; q < cnt[r]; ++q) pool[base + w + q] = src[q];
        }
        w += cnt[r];
    }
    if (lane == 0) fd.chunk_off[fd.pair_strip_off[c.p] + s] = base;
    pair_tot += strip_tot;
    __syncwarp();
}

// rows per lane of a strip with rows_in rows: the smallest of 1, 2, 4, 8 that covers it
__device__ __forceinline__ int rows_per_lane(int rows_in) {
    const int r = (rows_in + 31) / 32;
    return r <= 1 ? 1 : r <= 2 ? 2 : (r <= 4 || kRmax == 4) ? 4 : 8;
}

template <bool STORE>
__device__ __forceinline__ void bwd_dispatch(int Rs, const Coef& cf, const float2* s_ow, const PairCtx& c,
                                             const WarpSmem& ws, int s, int ns, const StripIO& io,
                                             float& Zh, float& Zp, int& eZh, int& eZp, int& flag) {
    switch (Rs) {
        case 1: bwd_strip<1, STORE>(cf, s_ow, c, ws, s, ns, io, Zh, Zp, eZh, eZp, flag); break;
        case 2: bwd_strip<2, STORE>(cf, s_ow, c, ws, s, ns, io, Zh, Zp, eZh, eZp, flag); break;
        case 4: bwd_strip<4, STORE>(cf, s_ow, c, ws, s, ns, io, Zh, Zp, eZh, eZp, flag); break;
        default: bwd_strip<kRmax, STORE>(cf, s_ow, c, ws, s, ns, io, Zh, Zp, eZh, eZp, flag); break;
    }
}

template <bool LIN>
__device__ __forceinline__ void fwd_dispatch(int Rs, const Problem& Pb, const float2* s_ow, const PairCtx& c,
                                             const WarpSmem& ws, int s, int ns, const StripIO& io,
                                             float invZh, float invZp, int eZh, int eZp, float scaleA,
                                             float& pmax, FwdOut& fo, int64_t& pair_tot, int& flag) {
    switch (Rs) {
        case 1: fwd_strip<1, LIN>(Pb, s_ow, c, ws, s, ns, io, invZh, invZp, eZh, eZp, scaleA, pmax, fo, pair_tot, flag); break;
        case 2: fwd_strip<2, LIN>(Pb, s_ow, c, ws, s, ns, io, invZh, invZp, eZh, eZp, scaleA, pmax, fo, pair_tot, flag); break;
        case 4: fwd_strip<4, LIN>(Pb, s_ow, c, ws, s, ns, io, invZh, invZp, eZh, eZp, scaleA, pmax, fo, pair_tot, flag); break;
        default: fwd_strip<kRmax, LIN>(Pb, s_ow, c, ws, s, ns, io, invZh, invZp, eZh, eZp, scaleA, pmax, fo, pair_tot, flag); break;
    }
}

// Control block of one group of warps working on one pair (shared memory).
struct GroupCtl {
    long long prog[4];          // progress word of each warp of the group
    int q;                      // the group's current work item
    int pad;
    float Zh, Zp;               // pass-1 totals (from the warp of strip 0)
    int eZh, eZp;
    float fZh, fZp;             // pass-2 corner values (from the warp of the last strip)
    int feh, fep, fA;
    int flag[4];
    float pmax[4];
    long long tot[4];
};

// Barrier of one group.  Groups of 2 warps use named barriers 1 and 2, a group
// of 4 barrier 1 (literal ids: a register id would reserve all 16 barriers of
// the block and cost occupancy).
__device__ __forceinline__ void group_sync(int gib, int W) {
    if (W == 1) { __syncwarp(); return; }
    if (gib == 0) asm volatile("bar.sync 1, %0;" ::"r"(32 * W) : "memory");
    else asm volatile("bar.sync 2, %0;" ::"r"(32 * W) : "memory");
}

// CKPT = false (stored form): pass 1 stores (B_M, Zm_b) of every strip, pass 2
// reads them back.  CKPT = true (checkpointed form, for long sequences): pass 1
// keeps only the boundary row at the top of every strip; pass 2 recomputes the
// backward values of one strip from the boundary row below it, then runs the
// forward sweep of that strip, so the per-warp scratch holds one strip instead
// of the whole matrix, for one more backward sweep of work.  Both forms give
// the same values: the recomputed strip starts from the same boundary row and
// runs the same instructions.
//
// W warps (1 or 2; Pb.wpp) share a pair: warp w of the group takes every
// W-th strip (pass 1 from the bottom, pass 2 from the top) and trails the warp
// of the neighbouring strip through that strip's boundary row and its
// progress word, so the strips of one pair run concurrently.
template <int MINB, bool CKPT, int W, bool LIN>
__global__ void __launch_bounds__(128, MINB) k_posterior_f32(Problem Pb) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    stamp_begin(Pb.status->t_f32);
    float2* s_ow = (float2*)s_raw;
    for (int i = threadIdx.x; i < kTab * kTab; i += blockDim.x) s_ow[i] = Pb.cst->ow[i];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int nwb = blockDim.x >> 5;
    const int gib = wib / W, wig = wib % W;
    WarpSmem ws;
    {
        unsigned char* p = s_raw + kOwBytes + (size_t)wib * warp_smem_bytes(Pb.max_len);
        ws.ring_b = (float2*)p;
        ws.ring_e = (float4*)(p + kD * kWarp * kRmax * 8);
        ws.sy = p + kD * kWarp * kRmax * 8 + kD * 32;
    }
    GroupCtl* gc = (GroupCtl*)(s_raw + kOwBytes + (size_t)nwb * warp_smem_bytes(Pb.max_len)) + gib;
    __syncthreads();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t gg = gw / W;
    PairCtx c;
    c.bst = Pb.bst + (CKPT ? gw : gg) * Pb.bst_stride;
    c.bex = Pb.bex + (CKPT ? gw : gg) * Pb.bex_stride;
    c.bnd = Pb.bnd + gg * Pb.bnd_stride;
    c.bck = Pb.bck + gg * Pb.bck_stride;
    c.stg = Pb.stg + gw * Pb.stg_stride;
    c.st = Pb.status;
    // boundary rows: one per strip when other warps or a later recompute read
    // them, else one row reused in place (the writer trails the reader)
    const bool bck_rows = CKPT || W > 1;
    const bool bnd_rows = W > 1;
    volatile long long* my_prog = W > 1 ? &gc->prog[wig] : nullptr;
    for (;;) {
        if (lane == 0) {
            if (my_prog) *my_prog = 0;
            if (wig == 0) gc->q = atomicAdd(&Pb.status->work_f32, 1);
        }
        group_sync(gib, W);
        const int q = *(volatile int*)&gc->q;
        if (q >= Pb.n_work) break;
        const int2 it = Pb.items[q];
        const FamDesc& fd = Pb.fams[it.x];
        const int p = it.y;
        const int2 ab = fd.pairs[p];
        const int64_t oa = fd.seq_off[ab.x], ob = fd.seq_off[ab.y];
        c.fd = &fd;
        c.m = (int)(fd.seq_off[ab.x + 1] - oa);
        c.n = (int)(fd.seq_off[ab.y + 1] - ob);
        c.x = fd.codes + oa;
        c.y = fd.codes + ob;
        c.p = p;
        c.nch = (c.n + 32 + kC - 1) / kC;
        const int m = c.m, n = c.n;
        const int nstrips = (m + 1 + kStripRows - 1) / kStripRows;
        // the column residues of the pair, staged once, with empty codes on
        // both sides so that every skewed column index reads a valid byte
        __syncwarp();
        for (int i = lane; i < n + 2 * kYPad; i += 32) {
            const int jj = i - kYPad;
            ws.sy[i] = (jj >= 0 && jj < n) ? c.y[jj] : (uint8_t)kEmpty;
        }
        __syncwarp();
        int flag = 0;
        // ---- pass 1: backward, bottom strip first (strip s: warp (ns-1-s) % W)
        float Zh = 0.f, Zp = 0.f;
        int eZh = 0, eZp = 0;
        const int64_t strip_vals = (int64_t)kStripRows * (n + 32), strip_exps = (int64_t)c.nch * 32;
        const int64_t row_len = 2 * (int64_t)(n + 1);
        for (int s = nstrips - 1 - wig, seq = 0; s >= 0; s -= W, ++seq) {
            const int rows_in = min(kStripRows, m + 1 - s * kStripRows);
            const int Rs = rows_per_lane(rows_in);
            StripIO io;
            io.bnd_in = (s == nstrips - 1) ? nullptr : c.bck + (bck_rows ? (s + 1) * row_len : 0);
            io.bnd_out = (s == 0) ? nullptr : c.bck + (bck_rows ? s * row_len : 0);
            io.wait = nullptr; io.pub = nullptr; io.wait_tag = io.pub_tag = 0;
            if (W > 1) {
                if (s < nstrips - 1) {
                    const int ps = nstrips - 2 - s;          // order of strip s + 1 in pass 1
                    io.wait = &gc->prog[ps % W];
                    io.wait_tag = (long long)(ps / W + 1) << 32;
                }
                if (s > 0) { io.pub = my_prog; io.pub_tag = (long long)(seq + 1) << 32; }
            }
            if (CKPT) {
                io.bst = nullptr;
                io.bex = nullptr;
                bwd_dispatch<false>(Rs, Pb.cf, s_ow, c, ws, s, nstrips, io, Zh, Zp, eZh, eZp, flag);
            } else {
                io.bst = c.bst + s * strip_vals;
                io.bex = c.bex + s * strip_exps;
                bwd_dispatch<true>(Rs, Pb.cf, s_ow, c, ws, s, nstrips, io, Zh, Zp, eZh, eZp, flag);
            }
            __syncwarp();
        }
        // the totals come from strip 0 (lane 0 of its warp)
        if (wig == (nstrips - 1) % W && lane == 0) {
            gc->Zh = Zh; gc->Zp = Zp; gc->eZh = eZh; gc->eZp = eZp;
        }
        group_sync(gib, W);
        Zh = *(volatile float*)&gc->Zh; Zp = *(volatile float*)&gc->Zp;
        eZh = *(volatile int*)&gc->eZh; eZp = *(volatile int*)&gc->eZp;
        // normalise the totals to [1, 2) * 2^e
        if (!(Zh > 0.f) || !(Zp > 0.f) || !(Zh < kBig) || !(Zp < kBig)) flag |= kGuardTotal;
        {
            const int kh = ilog2f(fmaxf(Zh, 1e-30f)), kp = ilog2f(fmaxf(Zp, 1e-30f));
            Zh *= pow2f(-kh); eZh += kh;
            Zp *= pow2f(-kp); eZp += kp;
        }
        const float invZh = 1.f / Zh, invZp = 1.f / Zp;
        // ---- pass 2: forward + posterior + threshold + MEA, top strip first
        // (strip s: warp s % W)
        const int mn = min(m, n);
        int sA = 30 - (32 - __clz(mn + 1));
        if (sA > 21) sA = 21;
        const float scaleA = (float)(1 << sA);
        float pmax = 0.f;
        FwdOut fo{0.f, 0.f, 0, 0, 0};
        int64_t pair_tot = 0;
        for (int s = wig, seq = 0; s < nstrips; s += W, ++seq) {
            const int rows_in = min(kStripRows, m + 1 - s * kStripRows);
            const int Rs = rows_per_lane(rows_in);
            StripIO io;
            io.bnd_in = (s == 0) ? nullptr : c.bnd + (bnd_rows ? (s - 1) * row_len : 0);
            io.bnd_out = (s == nstrips - 1) ? nullptr : c.bnd + (bnd_rows ? s * row_len : 0);
            io.wait = nullptr; io.pub = nullptr; io.wait_tag = io.pub_tag = 0;
            if (W > 1) {
                if (s > 0) {
                    io.wait = &gc->prog[(s - 1) % W];
                    io.wait_tag = (kPass2Tag + (s - 1) / W + 1) << 32;
                }
                if (s < nstrips - 1) { io.pub = my_prog; io.pub_tag = (kPass2Tag + seq + 1) << 32; }
            }
            if (CKPT) {
                // the strip's backward values again, from its checkpoint row
                StripIO bio;
                bio.bnd_in = (s == nstrips - 1) ? nullptr : c.bck + (s + 1) * row_len;
                bio.bnd_out = nullptr;
                bio.bst = c.bst;
                bio.bex = c.bex;
                bio.wait = nullptr; bio.pub = nullptr; bio.wait_tag = bio.pub_tag = 0;
                float dZh = 0.f, dZp = 0.f;
                int deZh = 0, deZp = 0;
                bwd_dispatch<true>(Rs, Pb.cf, s_ow, c, ws, s, nstrips, bio, dZh, dZp, deZh, deZp, flag);
                __syncwarp();
                io.bst = c.bst;
                io.bex = c.bex;
            } else {
                io.bst = c.bst + s * strip_vals;
                io.bex = c.bex + s * strip_exps;
            }
            fwd_dispatch<LIN>(Rs, Pb, s_ow, c, ws, s, nstrips, io, invZh, invZp, eZh, eZp, scaleA, pmax, fo,
                         pair_tot, flag);
            __syncwarp();
        }
        // ---- pair results: partial values of every warp of the group
        if (wig == (nstrips - 1) % W) {
            // corner values, held by the lane that owns row m
            const int lastRs = rows_per_lane(min(kStripRows, m + 1 - (nstrips - 1) * kStripRows));
            const int Lend = (m - (nstrips - 1) * kStripRows) / lastRs;
            const float fZh = __shfl_sync(FULL, fo.Zh, Lend), fZp = __shfl_sync(FULL, fo.Zp, Lend);
            const int feh = __shfl_sync(FULL, fo.eZh, Lend), fep = __shfl_sync(FULL, fo.eZp, Lend);
            const int Aend = __shfl_sync(FULL, fo.A, Lend);
            if (lane == 0) { gc->fZh = fZh; gc->fZp = fZp; gc->feh = feh; gc->fep = fep; gc->fA = Aend; }
        }
        for (int o = 16; o > 0; o >>= 1) pmax = fmaxf(pmax, __shfl_xor_sync(FULL, pmax, o));
        flag = __reduce_or_sync(FULL, flag);
        if (lane == 0) { gc->flag[wig] = flag; gc->pmax[wig] = pmax; gc->tot[wig] = pair_tot; }
        group_sync(gib, W);
        if (wig == 0 && lane == 0) {
            int fl = 0;
            float pm = 0.f;
            int64_t tot = 0;
            for (int w = 0; w < W; ++w) {
                fl |= ((volatile int*)gc->flag)[w];
                pm = fmaxf(pm, ((volatile float*)gc->pmax)[w]);
                tot += ((volatile long long*)gc->tot)[w];
            }
            if (pm > 1.001f) fl |= kGuardPost;
            const float fZh = *(volatile float*)&gc->fZh, fZp = *(volatile float*)&gc->fZp;
            const int feh = *(volatile int*)&gc->feh, fep = *(volatile int*)&gc->fep;
            const int Aend = *(volatile int*)&gc->fA;
            const double ln2 = 0.69314718055994530942;
            const double lzb_h = log((double)Zh) + (double)eZh * ln2;
            const double lzb_p = log((double)Zp) + (double)eZp * ln2;
            const double lzf_h = log((double)fZh) + (double)feh * ln2;
            const double lzf_p = log((double)fZp) + (double)fep * ln2;
            if (!(fabs(lzb_h - lzf_h) <= 1e-3)) fl |= kGuardAgreeH;
            if (!(fabs(lzb_p - lzf_p) <= 1e-3)) fl |= kGuardAgreeP;
            // a full entry pool is not a range problem: the pair keeps its FP32
            // results, its flag tells the host to grow the pool and run again
            if (fl & ~kGuardPool) {
                fd.pair_flags[p] = fl;
                const int slot = atomicAdd(&Pb.status->n_fallback, 1);
                Pb.fallback[slot] = it;
            } else {
                const double A = (double)Aend / (double)(1 << sA);
                fd.mea[p] = A;
                fd.logz_h[p] = lzb_h + fd.seq_logq[ab.x] + fd.seq_logq[ab.y];
                fd.logz_p[p] = lzb_p;
                fd.pair_nnz[p] = tot;
                fd.pair_flags[p] = fl;
                const double d = 1.0 - A / (double)mn;
                const int64_t k = fd.k;
                fd.dist[ab.x * k + ab.y] = (float)d;
                fd.dist[ab.y * k + ab.x] = (float)d;
                fd.dist64[ab.x * k + ab.y] = d;
                fd.dist64[ab.y * k + ab.x] = d;
                if (fd.n_done) { __threadfence(); atomicAdd(fd.n_done, 1); }
            }
        }
        group_sync(gib, W);
    }
    stamp_end(Pb.status->t_f32);
}

using F32Kernel = void (*)(Problem);

template <int W, bool LIN>
static F32Kernel f32_kernel_wl(int variant, bool ckpt) {
    if (ckpt) return variant == 1 ? k_posterior_f32<3, true, W, LIN> : k_posterior_f32<4, true, W, LIN>;
    return variant == 1 ? k_posterior_f32<3, false, W, LIN> : k_posterior_f32<4, false, W, LIN>;
}

// lin: a linear combination of the two posteriors (combine modes other than
// the root mean square), compiled as its own kernel so the default keeps no
// per-cell test of the mode
static F32Kernel f32_kernel(int variant, bool ckpt, int wpp = 1, bool lin = false) {
    if (lin) return wpp == 2 ? f32_kernel_wl<2, true>(variant, ckpt) : f32_kernel_wl<1, true>(variant, ckpt);
    return wpp == 2 ? f32_kernel_wl<2, false>(variant, ckpt) : f32_kernel_wl<1, false>(variant, ckpt);
}

// Raises a kernel's dynamic shared memory limit once per size (so that a
// launch inside a stream capture makes no attribute call).
static cudaError_t set_smem(F32Kernel k, size_t smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    static std::mutex mu;
    static std::map<std::pair<F32Kernel, int>, size_t> done;   // (kernel, device) -> limit set
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    size_t& cur = done[std::make_pair(k, dev)];
    if (smem <= cur) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) cur = smem;
    return e;
}

int posterior_f32_regs(int variant, bool ckpt) {
    cudaFuncAttributes a;
    const cudaError_t e = cudaFuncGetAttributes(&a, f32_kernel(variant, ckpt));
    return e == cudaSuccess ? a.numRegs : -1;
}

size_t posterior_f32_smem(int warps_per_block, int max_len) {
    return (size_t)kOwBytes + (size_t)warps_per_block * warp_smem_bytes(max_len) +
           (size_t)warps_per_block * sizeof(GroupCtl);
}

int posterior_f32_occupancy(int warps_per_block, int max_len, int* blocks_per_sm, int variant, bool ckpt,
                            int wpp) {
    const size_t smem = posterior_f32_smem(warps_per_block, max_len);
    const F32Kernel k = f32_kernel(variant, ckpt, wpp);
    set_smem(k, smem);
    set_smem(f32_kernel(variant, ckpt, wpp, true), smem);    // the linear-combination kernel too (no attribute
                                                             // call inside a later stream capture)
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, warps_per_block * 32, smem);
}

cudaError_t launch_posterior_f32(const Problem& P, int grid, int warps_per_block, cudaStream_t s,
                                 int variant) {
    const size_t smem = posterior_f32_smem(warps_per_block, P.max_len);
    if (P.wpp != 1 && P.wpp != 2) return cudaErrorInvalidValue;
    const F32Kernel k = f32_kernel(variant, P.ckpt != 0, P.wpp, P.cf.combine != 0);
    cudaError_t e = set_smem(k, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, warps_per_block * 32, smem, s>>>(P);
    return cudaGetLastError();
}

// ================================================================ FP64 form
//
// Plain FP64 evaluation: one CTA per pair, anti-diagonal wavefront over the
// (m+1) x (n+1) grid, values of each diagonal rescaled by a power of two so
// that its largest value is in [1, 2).  Pass 1 (backward) stores (B_M, Zm_b)
// densely; pass 2 (forward) forms the posteriors, the combination, the
// threshold and the MEA recurrence on each diagonal.
constexpr int kF64Threads = 256;

__device__ __forceinline__ double pow2d(int e) { return ldexp(1.0, e); }

__device__ double block_max(double v, double* red) {
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double r = red[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) r = fmax(r, red[i]);
    return r;
}

__device__ int block_sum(int v, int* red) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    int r = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += red[i];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kF64Threads) k_posterior_f64(Problem Pb) {
    stamp_begin(Pb.status->t_f64);
    __shared__ double sred[2][kF64Threads / 32];
    __shared__ int ired[kF64Threads / 32];
    __shared__ int s_q;
    __shared__ unsigned long long s_base;
    const Consts* __restrict__ C = Pb.cst;
    const int tid = threadIdx.x, nt = blockDim.x;
    double2* Bd = Pb.d_b + (int64_t)blockIdx.x * Pb.d_b_stride;
    double* dg = Pb.d_diag + (int64_t)blockIdx.x * Pb.d_diag_stride;
    int32_t* rc = Pb.d_cnt + (int64_t)blockIdx.x * Pb.d_cnt_stride;
    int2* stg = Pb.d_stg + (int64_t)blockIdx.x * Pb.d_stg_stride;
    double* stg64 = Pb.d_stg64 + (int64_t)blockIdx.x * Pb.d_stg_stride;
    const int L = Pb.max_len + 1;   // diagonal slot length (indexed by row)
    const int cap = Pb.cap;
    const double tMM = C->tMMd, d1 = C->d1d, d2 = C->d2d, e1 = C->e1d, e2 = C->e2d;
    const double c1 = C->c1d, c2 = C->c2d, Wo = C->Wod, We = C->Wed;
    for (;;) {
        if (tid == 0) s_q = atomicAdd(&Pb.status->work_f64, 1);
        __syncthreads();
        const int q = s_q;
        __syncthreads();
        const int n_items = Pb.f64_all ? Pb.n_work : *(volatile int*)&Pb.status->n_fallback;
        if (q >= n_items) break;
        const int2 it = Pb.f64_all ? Pb.items[q] : Pb.fallback[q];
        const FamDesc& fd = Pb.fams[it.x];
        const int p = it.y;
        const int2 ab = fd.pairs[p];
        const int64_t oa = fd.seq_off[ab.x], ob = fd.seq_off[ab.y];
        const int m = (int)(fd.seq_off[ab.x + 1] - oa), n = (int)(fd.seq_off[ab.y + 1] - ob);
        const uint8_t* x = fd.codes + oa;
        const uint8_t* y = fd.codes + ob;
        auto X = [&](int i) { return (i >= 1 && i <= m) ? (int)x[i - 1] : kEmpty; };
        auto Y = [&](int j) { return (j >= 1 && j <= n) ? (int)y[j - 1] : kEmpty; };
        auto slot = [&](int d, int v) -> double* { return dg + ((int64_t)((d % 3 + 3) % 3) * kNS + v) * L; };
        // ---- pass 1: backward over anti-diagonals d = m+n .. 0
        // slot values: 0 B_M, 1 B_X, 2 B_X2, 3 B_Y, 4 B_Y2, 5 Zm_b, 6 Ze_b, 7 Zf_b
        int Eh1 = 0, Ep1 = 0, Eh2 = 0, Ep2 = 0;   // exponents of diagonals d+1, d+2
        double Zh = 0.0, Zp = 0.0;
        int eZh = 0, eZp = 0;
        int32_t* EB = rc + L;            // [m+n+1] HMM exponents per diagonal
        int32_t* EP = EB + (2 * L + 2);  // [m+n+1] PF exponents per diagonal
        for (int d = m + n; d >= 0; --d) {
            const int ilo = max(0, d - n), ihi = min(m, d);
            double* cur[8];
            for (int v = 0; v < 8; ++v) cur[v] = slot(d, v);
            double mh = 0.0, mp = 0.0;
            const double f2 = pow2d(Eh2 - Eh1), g2 = pow2d(Ep2 - Ep1);
            for (int i = ilo + tid; i <= ihi; i += nt) {
                const int j = d - i;
                double D = 0, Dp = 0, Xb = 0, X2b = 0, Eb = 0, Yb = 0, Y2b = 0, Fb = 0;
                if (i < m && j < n) {
                    const int o = Y(j + 1) * kTab + X(i + 1);
                    D = C->oddsd[o] * slot(d + 2, 0)[i + 1] * f2;
                    Dp = C->wd[o] * slot(d + 2, 5)[i + 1] * g2;
                }
                if (i < m) { Xb = slot(d + 1, 1)[i + 1]; X2b = slot(d + 1, 2)[i + 1]; Eb = slot(d + 1, 6)[i + 1]; }
                if (j < n) { Yb = slot(d + 1, 3)[i]; Y2b = slot(d + 1, 4)[i]; Fb = slot(d + 1, 7)[i]; }
                double BM = tMM * D + d1 * (Xb + Yb) + d2 * (X2b + Y2b);
                double BX = c1 * D + e1 * Xb, BX2 = c2 * D + e2 * X2b;
                double BY = c1 * D + e1 * Yb, BY2 = c2 * D + e2 * Y2b;
                double ZMB = Dp + Wo * (Eb + Fb), ZEB = Dp + We * Eb, ZFB = Dp + We * Fb;
                if (i == m && j == n) {
                    BM = C->taud[0]; BX = C->taud[1]; BY = C->taud[2]; BX2 = C->taud[3]; BY2 = C->taud[4];
                    ZMB = ZEB = ZFB = 1.0;
                }
                if (i == 0 && j == 0) {
                    Zh = C->pid[0] * D + C->pid[1] * Xb + C->pid[2] * Yb + C->pid[3] * X2b + C->pid[4] * Y2b;
                    Zp = ZMB;
                }
                cur[0][i] = BM; cur[1][i] = BX; cur[2][i] = BX2; cur[3][i] = BY; cur[4][i] = BY2;
                cur[5][i] = ZMB; cur[6][i] = ZEB; cur[7][i] = ZFB;
                mh = fmax(mh, fmax(fmax(BM, BX), fmax(BX2, fmax(BY, BY2))));
                mp = fmax(mp, fmax(ZMB, fmax(ZEB, ZFB)));
            }
            const double MH = block_max(mh, sred[0]);
            const double MP = block_max(mp, sred[1]);
            int kh = 0, kp = 0;
            if (d != m + n) {
                if (MH > 0.0) { frexp(MH, &kh); kh -= 1; }
                if (MP > 0.0) { frexp(MP, &kp); kp -= 1; }
            }
            const double sh = pow2d(-kh), sp = pow2d(-kp);
            const int Ed = Eh1 + kh, Fd = Ep1 + kp;
            for (int i = ilo + tid; i <= ihi; i += nt) {
                const int j = d - i;
                for (int v = 0; v < 5; ++v) cur[v][i] *= sh;
                for (int v = 5; v < 8; ++v) cur[v][i] *= sp;
                Bd[(int64_t)i * (n + 1) + j] = make_double2(cur[0][i], cur[5][i]);
            }
            if (tid == 0) { EB[d] = (d == m + n) ? 0 : Ed; EP[d] = (d == m + n) ? 0 : Fd; }
            if (d == 0 && tid == 0) { eZh = Eh1; eZp = Ep1; }
            Eh2 = Eh1; Ep2 = Ep1;
            Eh1 = (d == m + n) ? 0 : Ed; Ep1 = (d == m + n) ? 0 : Fd;
            __syncthreads();
        }
        // totals (thread 0 computed them at d = 0, in units of diagonal 1)
        if (tid == 0) { sred[0][0] = Zh; sred[1][0] = Zp; ired[0] = eZh; ired[1] = eZp; }
        __syncthreads();
        Zh = sred[0][0]; Zp = sred[1][0]; eZh = ired[0]; eZp = ired[1];
        __syncthreads();
        // ---- pass 2: forward over d = 0 .. m+n
        // slot values: 0 Mdiag, 1 Xin, 2 X2in, 3 Yin, 4 Y2in, 5 Zd, 6 Ein, 7 Fin, 8 A
        for (int i = tid; i <= m; i += nt) rc[i] = 0;
        __syncthreads();
        int Fh1 = 0, Fp1 = 0, Fh2 = 0, Fp2 = 0;
        double fZh = 0, fZp = 0, Aend = 0;
        int feh = 0, fep = 0;
        const double theta = C->thetad;
        const int comb = C->combine;
        for (int d = 0; d <= m + n; ++d) {
            const int ilo = max(0, d - n), ihi = min(m, d);
            double* cur[9];
            for (int v = 0; v < 9; ++v) cur[v] = slot(d, v);
            const double f2 = pow2d(Fh2 - Fh1), g2 = pow2d(Fp2 - Fp1);
            double mh = 0.0, mp = 0.0;
            // the thread for row i is fixed: i = tid (mod nt)
            const int i0 = ilo + ((tid - ilo) % nt + nt) % nt;
            for (int i = i0; i <= ihi; i += nt) {
                const int j = d - i;
                double Md = 0, Xi = 0, X2i = 0, Yi = 0, Y2i = 0, Zd = 0, Ei = 0, Fi = 0;
                double Adg = 0, Aup = 0, Alf = 0;
                if (i >= 1 && j >= 1) { Md = slot(d - 2, 0)[i - 1] * f2; Zd = slot(d - 2, 5)[i - 1] * g2; Adg = slot(d - 2, 8)[i - 1]; }
                if (i >= 1) { Xi = slot(d - 1, 1)[i - 1]; X2i = slot(d - 1, 2)[i - 1]; Ei = slot(d - 1, 6)[i - 1]; Aup = slot(d - 1, 8)[i - 1]; }
                if (j >= 1) { Yi = slot(d - 1, 3)[i]; Y2i = slot(d - 1, 4)[i]; Fi = slot(d - 1, 7)[i]; Alf = slot(d - 1, 8)[i]; }
                const int o = Y(j) * kTab + X(i);
                const double FM = C->oddsd[o] * Md, FX = Xi, FX2 = X2i, FY = Yi, FY2 = Y2i;
                const double ZM = C->wd[o] * Zd, ZE = Ei, ZF = Fi;
                double nMd = tMM * FM + c1 * (FX + FY) + c2 * (FX2 + FY2);
                double nXi = d1 * FM + e1 * FX, nX2i = d2 * FM + e2 * FX2;
                double nYi = d1 * FM + e1 * FY, nY2i = d2 * FM + e2 * FY2;
                double nZd = ZM + ZE + ZF, nEi = Wo * ZM + We * ZE, nFi = Wo * ZM + We * ZF;
                double A = 0.0;
                if (i >= 1 && j >= 1) {
                    const double2 b = Bd[(int64_t)i * (n + 1) + j];
                    // F in units of the previous diagonal, B in units of its diagonal
                    const double ph = ldexp(FM * b.x / Zh, Fh1 + EB[d] - eZh);
                    const double pp = ldexp(ZM * b.y / Zp, Fp1 + EP[d] - eZp);
                    double P;
                    if (comb == 0) P = sqrt(0.5 * (ph * ph + pp * pp));
                    else if (comb == 1) P = 0.5 * (ph + pp);
                    else if (comb == 2) P = ph;
                    else P = pp;
                    if (P >= theta) {
                        const int qq = rc[i]++;
                        if (qq < cap) {
                            stg[(int64_t)(i - 1) * cap + qq] = make_int2(j - 1, __float_as_int((float)P));
                            stg64[(int64_t)(i - 1) * cap + qq] = P;
                        }
                    }
                    A = fmax(Adg + P, fmax(Aup, Alf));
                }
                if (i == 0 && j == 0) {
                    nMd = C->pid[0]; nXi = C->pid[1]; nYi = C->pid[2]; nX2i = C->pid[3]; nY2i = C->pid[4];
                    nZd = 1.0; nEi = Wo; nFi = Wo;
                }
                if (i == m && j == n) {
                    fZh = C->taud[0] * FM + C->taud[1] * FX + C->taud[2] * FY + C->taud[3] * FX2 + C->taud[4] * FY2;
                    fZp = ZM + ZE + ZF;
                    Aend = A;
                    feh = Fh1; fep = Fp1;
                }
                cur[0][i] = nMd; cur[1][i] = nXi; cur[2][i] = nX2i; cur[3][i] = nYi; cur[4][i] = nY2i;
                cur[5][i] = nZd; cur[6][i] = nEi; cur[7][i] = nFi; cur[8][i] = A;
                mh = fmax(mh, fmax(fmax(nMd, nXi), fmax(nX2i, fmax(nYi, nY2i))));
                mp = fmax(mp, fmax(nZd, fmax(nEi, nFi)));
            }
            const double MH = block_max(mh, sred[0]);
            const double MP = block_max(mp, sred[1]);
            int kh = 0, kp = 0;
            if (MH > 0.0) { frexp(MH, &kh); kh -= 1; }
            if (MP > 0.0) { frexp(MP, &kp); kp -= 1; }
            const double sh = pow2d(-kh), sp = pow2d(-kp);
            for (int i = i0; i <= ihi; i += nt) {
                for (int v = 0; v < 5; ++v) cur[v][i] *= sh;
                for (int v = 5; v < 8; ++v) cur[v][i] *= sp;
            }
            Fh2 = Fh1; Fp2 = Fp1;
            Fh1 += kh; Fp1 += kp;
            __syncthreads();
        }
        // gather the corner values from the thread that held row m
        if (tid == m % nt) {
            sred[0][0] = fZh; sred[1][0] = fZp; sred[0][1] = Aend; ired[0] = feh; ired[1] = fep;
        }
        __syncthreads();
        fZh = sred[0][0]; fZp = sred[1][0]; Aend = sred[0][1]; feh = ired[0]; fep = ired[1];
        __syncthreads();
        // ---- flush entries per 128-row strip
        const int nstrips = (m + 1 + kStripRows - 1) / kStripRows;
        const int64_t row_slot = fd.pair_row_off[p];
        int64_t pair_tot = 0;
        for (int s = 0; s < nstrips; ++s) {
            const int r0 = max(1, s * kStripRows), r1 = min(m, s * kStripRows + kStripRows - 1);
            int my = 0;
            for (int i = r0 + tid; i <= r1; i += nt) {
                if (rc[i] > cap) { atomicExch(&Pb.status->stage_overflow, 1); rc[i] = cap; }
                my += rc[i];
            }
            const int tot = block_sum(my, ired);
            if (tid == 0) s_base = tot ? atomicAdd(fd.pool_used, (unsigned long long)tot) : 0ull;
            __syncthreads();
            const bool fits = (int64_t)s_base + tot <= fd.pool_cap;
            const int64_t base = fd.pool_base + (int64_t)s_base;
            if (!fits && tid == 0) atomicExch(&Pb.status->pool_overflow, 1);
            // serial prefix over the strip's rows by thread 0 (plain form), then copy
            if (tid == 0) {
                int64_t w = 0;
                for (int i = r0; i <= r1; ++i) {
                    fd.row_cnt[row_slot + i - 1] = rc[i];
                    const int c0 = rc[i];
                    rc[i] = (int)w;   // reused as the row's offset within the strip
                    w += c0;
                }
                fd.chunk_off[fd.pair_strip_off[p] + s] = base;
            }
            __syncthreads();
            if (fits) {
                int2* pool = fd.pool ? fd.pool : Pb.pool;
                double* pool64 = fd.pool ? fd.pool64 : Pb.pool64;
                for (int i = r0 + tid; i <= r1; i += nt) {
                    const int cnt = fd.row_cnt[row_slot + i - 1];
                    const int o = rc[i];
                    for (int qq = 0; qq < cnt; ++qq) {
                        pool[base + o + qq] = stg[(int64_t)(i - 1) * cap + qq];
                        if (pool64) pool64[base + o + qq] = stg64[(int64_t)(i - 1) * cap + qq];
                    }
                }
            }
            pair_tot += tot;
            __syncthreads();
        }
        if (tid == 0) {
            const double ln2 = 0.69314718055994530942;
            const double lzb_h = log(Zh) + (double)eZh * ln2;
            const double lzb_p = log(Zp) + (double)eZp * ln2;
            fd.mea[p] = Aend;
            fd.logz_h[p] = lzb_h + fd.seq_logq[ab.x] + fd.seq_logq[ab.y];
            fd.logz_p[p] = lzb_p;
            fd.pair_nnz[p] = pair_tot;
            const double lzf_h = log(fZh) + (double)feh * ln2;
            const double lzf_p = log(fZp) + (double)fep * ln2;
            const bool agree = fabs(lzb_h - lzf_h) <= 1e-8 * fmax(1.0, fabs(lzb_h)) &&
                               fabs(lzb_p - lzf_p) <= 1e-8 * fmax(1.0, fabs(lzb_p));
            fd.pair_flags[p] = (Pb.f64_all ? 0 : (fd.pair_flags[p] | 1)) | (agree ? 0 : 2);
            const int mn = min(m, n);
            const double dd = 1.0 - Aend / (double)mn;
            const int64_t kk = fd.k;
            fd.dist[ab.x * kk + ab.y] = (float)dd;
            fd.dist[ab.y * kk + ab.x] = (float)dd;
            fd.dist64[ab.x * kk + ab.y] = dd;
            fd.dist64[ab.y * kk + ab.x] = dd;
            if (fd.n_done) { __threadfence(); atomicAdd(fd.n_done, 1); }
        }
        __syncthreads();
    }
    stamp_end(Pb.status->t_f64);
}

int posterior_f64_occupancy(int* blocks_per_sm) {
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_posterior_f64,
                                                              kF64Threads, 0);
}

cudaError_t launch_posterior_f64(const Problem& P, int grid, cudaStream_t s) {
    k_posterior_f64<<<grid, kF64Threads, 0, s>>>(P);
    return cudaGetLastError();
}

// ================================================================ CSR assembly
__global__ void k_scan_nnz(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ out) {
    // single CTA: each thread scans a contiguous segment, then the CTA scans
    // the segment totals
    __shared__ int64_t part[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t per = (n + nt - 1) / nt;
    const int64_t lo = min(n, per * tid), hi = min(n, lo + per);
    int64_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += in[i];
    part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        int64_t acc = 0;
        for (int i = 0; i < nt; ++i) { const int64_t v = part[i]; part[i] = acc; acc += v; }
        out[n] = acc;
    }
    __syncthreads();
    int64_t acc = part[tid];
    for (int64_t i = lo; i < hi; ++i) { out[i] = acc; acc += in[i]; }
}

__global__ void k_compact(const int2* __restrict__ pairs, const int64_t* __restrict__ seq_off,
                          const int64_t* __restrict__ pair_row_off, const int64_t* __restrict__ pair_strip_off,
                          const int32_t* __restrict__ row_cnt, const int64_t* __restrict__ chunk_off,
                          const int2* __restrict__ pool, const double* __restrict__ pool64, int64_t n_pairs,
                          const int64_t* __restrict__ pair_nnz_off, int32_t* __restrict__ row_ptr,
                          int32_t* __restrict__ col, float* __restrict__ val, double* __restrict__ val64,
                          unsigned long long* __restrict__ minmax, const int32_t* __restrict__ overflow) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    // a pool that overflowed holds chunks beyond its end: nothing to assemble
    // (the call runs again with a larger pool)
    if (p >= n_pairs || (overflow && *overflow)) return;
    const int2 ab = pairs[p];
    const int m = (int)(seq_off[ab.x + 1] - seq_off[ab.x]);
    const int64_t ro = pair_row_off[p];
    // row pointers: exclusive scan of the row counts, 32 rows at a time
    int carry = 0;
    for (int r0 = 0; r0 <= m; r0 += 32) {
        const int r = r0 + lane;
        const int v = (r < m) ? row_cnt[ro + r] : 0;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += u;
        }
        if (r <= m) row_ptr[ro + r] = carry + incl - v;
        carry += __shfl_sync(FULL, incl, 31);
    }
    __syncwarp();
    const int64_t base = pair_nnz_off[p];
    const int nstrips = (m + 1 + kStripRows - 1) / kStripRows;
    // smallest and largest key (bit pattern of the compared value), for the
    // entry budget's select
    unsigned long long kmin = ~0ull, kmax = 0ull;
    for (int s = 0; s < nstrips; ++s) {
        const int r0 = max(1, s * kStripRows) - 1;
        const int r1 = min(m + 1, s * kStripRows + kStripRows) - 1;
        const int beg = row_ptr[ro + r0], end = row_ptr[ro + r1];
        const int64_t src = chunk_off[pair_strip_off[p] + s];
        for (int e = lane; e < end - beg; e += 32) {
            const int2 v = pool[src + e];
            col[base + beg + e] = v.x;
            val[base + beg + e] = __int_as_float(v.y);
            unsigned long long key = (unsigned)v.y;
            if (val64) {
                const double d = pool64[src + e];
                val64[base + beg + e] = d;
                key = (unsigned long long)__double_as_longlong(d);
            }
            kmin = key < kmin ? key : kmin;
            kmax = key > kmax ? key : kmax;
        }
    }
    if (minmax) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long a = __shfl_xor_sync(FULL, kmin, o), b = __shfl_xor_sync(FULL, kmax, o);
            kmin = a < kmin ? a : kmin;
            kmax = b > kmax ? b : kmax;
        }
        if (lane == 0 && kmax >= kmin) {
            atomicMin(&minmax[0], kmin);
            atomicMax(&minmax[1], kmax);
        }
    }
}

cudaError_t launch_scan_nnz(const int64_t* pair_nnz, int64_t n_pairs, int64_t* pair_nnz_off,
                            cudaStream_t s) {
    k_scan_nnz<<<1, 1024, 0, s>>>(pair_nnz, n_pairs, pair_nnz_off);
    return cudaGetLastError();
}

cudaError_t launch_compact(const int2* pairs, const int64_t* seq_off,
                           const int64_t* pair_row_off, const int64_t* pair_strip_off,
                           const int32_t* row_cnt, const int64_t* chunk_off, const int2* pool,
                           const double* pool64, int64_t n_pairs, const int64_t* pair_nnz_off,
                           int32_t* row_ptr, int32_t* col, float* val, double* val64,
                           cudaStream_t s, unsigned long long* minmax, const int32_t* overflow) {
    const int64_t threads = n_pairs * 32;
    const int blocks = (int)((threads + 255) / 256);
    if (blocks > 0)
        k_compact<<<blocks, 256, 0, s>>>(pairs, seq_off, pair_row_off, pair_strip_off, row_cnt, chunk_off,
                                         pool, pool64, n_pairs, pair_nnz_off, row_ptr, col, val, val64, minmax,
                                         overflow);
    return cudaGetLastError();
}

}  // namespace qpk
