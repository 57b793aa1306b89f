// The FP32 posterior kernel, k_posterior_f32: the hot path of the all-pairs
// posterior stage (paper, Methods, stage I).  One warp (or two) per pair, FP32
// recurrences with per-lane power-of-two rescaling; pass 1 = backward of the
// pair-HMM and the partition function (stored, or checkpointed per strip),
// pass 2 = forward of both models fused with the posterior, the combination,
// the threshold, the MEA recurrence and the distance.
//
// Included by the translation units that instantiate the kernel's forms
// (qp_f32_w1.cu: one warp per pair, qp_f32_w2.cu: two), so that they compile
// in parallel.
//
// Geometry.  The DP grid has rows 0..m (row 0 and column 0 are the empty
// prefixes; their residue code is kEmpty, whose odds and weights are 0) and
// columns 0..n.  Rows are cut into strips of kStripRows; in a strip lane l
// owns the R consecutive rows row0 + l*R + r (R = 4, fewer in a short last
// strip).  A strip is swept column by column with the lanes skewed by one
// column: in the forward pass lane l is at column t - l at step t, so one step
// of the warp covers an anti-diagonal segment and the value a lane needs from
// the row above was produced by lane l-1 one step earlier (one shuffle per
// value).  The row above lane 0 (the previous strip's last row) comes from a
// boundary row in global memory written by lane 31 of that strip.  The
// backward pass mirrors this (lane 31 leads, values come from lane l+1).
//
// Storage.  Pass 1 stores (B_M, Zm_b) of every cell in blocks indexed by the
// forward step T = j + l at which pass 2 visits the cell; a block is 32*R
// float2 laid out [half][lane][2 rows] (rows 2h and 2h + 1 of every lane,
// then the next pair of rows), so that every 16-byte store of pass 1 and
// every 16-byte copy of pass 2 covers 512 contiguous bytes.  Pass 2 streams
// the blocks into a per-warp shared-memory ring kD steps ahead of their use,
// in the same layout.
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
// exponent per lane and kC-step chunk; pass 2 combines the two exponents, the
// totals and the combination weights into one factor per lane and chunk, so
// the weighted posterior of a cell is (F * factor) * B.
//
// Threshold.  The cells of a lane's rows at one step form a group; when the
// largest posterior of the group reaches the threshold the lane writes the
// whole group (column and R values, one 32-byte record) to its staging area.
// At the end of the strip each lane counts its entries per row, the warp
// reserves their place in the family's entry pool, and each lane copies its
// entries there in CSR order in one pass over its records.
//
// Range guards (the pair is recomputed by the FP64 form when one fires), for
// lanes that own a row of the pair: a carried maximum >= 2^100 or not finite,
// an exponent gap beyond the float range, a posterior factor beyond the float
// range, a posterior above 1.001, forward and backward totals that disagree by
// more than 1e-3 in log.
#pragma once
#include "qp_internal.h"

#include <type_traits>

namespace qpk {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------- scalar helpers
// 2^e as a float for e in [-126, 127]; 0 below -126, 2^127 above.
__device__ __forceinline__ float pow2f(int e) {
    if (e < -126) return 0.f;
    if (e > 127) e = 127;
    return __int_as_float((e + 127) << 23);
}

// Square root with the single hardware approximation (sqrt.approx.ftz.f32);
// its relative error is a few units in the last place, far inside the 1e-5
// posterior tolerance.
__device__ __forceinline__ float sqrt_approx(float v) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// Largest of three floats in one instruction (sm_100 and later).
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// floor(log2 v) for a positive normal float; -127 for zero / denormal.
__device__ __forceinline__ int ilog2f(float v) {
    return ((__float_as_int(v) >> 23) & 0xff) - 127;
}

// ---------------------------------------------------------------- shared memory
// Shared-memory accesses through 32-bit shared-window addresses.  Loads of
// data that cp.async or other lanes write are volatile (ordered against the
// waits); the read-only table loads are not, so the compiler may schedule them.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ float2 lds_tab(unsigned a) {
    float2 v;
    asm("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ float4 lds_v4(unsigned a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ float2 lds_v2(unsigned a) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ int lds_u8(unsigned a) {
    unsigned v;
    asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(a));
    return (int)v;
}
__device__ __forceinline__ void sts_v4(unsigned a, float4 v) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// ---------------------------------------------------------------- async copies
// cp.async moves the stored backward blocks into a small per-warp
// shared-memory ring kD steps ahead of their use; every lane copies and later
// reads only its own bytes, so waiting on its own copy groups is the only
// synchronisation needed.  The boundary row, which one lane reads, comes in
// chunks of kBndChunk columns, one 16-byte copy per lane for a whole chunk,
// issued on the renormalisation steps one chunk ahead into a two-chunk ring;
// the lanes then meet at a warp barrier before the reading lane uses it.  A
// source size of 0 fills the slot with zeros.
constexpr int kD = kD_ring;
constexpr int kBndChunk = kC;                 // boundary-row columns per chunk (one per step)
constexpr int kBndSlots = 2 * kBndChunk;      // the two-chunk ring of boundary columns (32 bytes each)
static_assert(kWarp == 2 * kBndChunk, "a chunk is one 16-byte copy per lane");

__device__ __forceinline__ void cp_async16(unsigned dst, const void* src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async8(unsigned dst, const void* src, int bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ---------------------------------------------------------------- global stores
// Predicated stores without a branch, each predicate formed inside the asm
// from the column j: the address is only used when 0 <= j <= n.
__device__ __forceinline__ void st_v4_if_in(int j, int n, void* a, float x, float y, float z, float w) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.le.u32 q, %0, %1;\n\t@q st.global.v4.f32 [%2], {%3, %4, %5, %6};\n\t}"
                 ::"r"(j), "r"(n), "l"(a), "f"(x), "f"(y), "f"(z), "f"(w) : "memory");
}
__device__ __forceinline__ void st_v2_if_in(int j, int n, void* a, float x, float y) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.le.u32 q, %0, %1;\n\t@q st.global.v2.f32 [%2], {%3, %4};\n\t}"
                 ::"r"(j), "r"(n), "l"(a), "f"(x), "f"(y) : "memory");
}
// 32 bytes of a boundary row (column j, one 256-bit store) when this lane
// writes the row (on != 0) and 0 <= j <= n.
__device__ __forceinline__ void st_bnd_if(int on, int j, int n, float4* a, float4 v, float4 u) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\tsetp.le.and.u32 q, %1, %2, q;\n\t"
                 "@q st.global.v8.f32 [%3], {%4, %5, %6, %7, %8, %9, %10, %11};\n\t}"
                 ::"r"(on), "r"(j), "r"(n), "l"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w),
                 "f"(u.x), "f"(u.y), "f"(u.z), "f"(u.w) : "memory");
}
// One staging record of a lane (column j, then the values of its R rows)
// when the step's largest value reaches the threshold and the area has room;
// ng counts the records wanted (it may pass the capacity: the caller checks).
template <int R>
__device__ __forceinline__ void stage_record(int4* g, int& ng, int capg, float pst, float theta, int j,
                                             const float (&Pv)[R]) {
    if (R == 1) {
        asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ge.f32 p, %1, %2;\n\tsetp.lt.and.s32 q, %0, %3, p;\n\t"
                     "@q st.global.v2.b32 [%4], {%5, %6};\n\t@p add.s32 %0, %0, 1;\n\t}"
                     : "+r"(ng) : "f"(pst), "f"(theta), "r"(capg), "l"(g), "r"(j), "f"(Pv[0]) : "memory");
    } else if (R == 2) {
        asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ge.f32 p, %1, %2;\n\tsetp.lt.and.s32 q, %0, %3, p;\n\t"
                     "@q st.global.v4.b32 [%4], {%5, %6, %7, %5};\n\t@p add.s32 %0, %0, 1;\n\t}"
                     : "+r"(ng) : "f"(pst), "f"(theta), "r"(capg), "l"(g), "r"(j), "r"(__float_as_int(Pv[0])),
                       "r"(__float_as_int(Pv[1])) : "memory");
    } else {
        asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ge.f32 p, %1, %2;\n\tsetp.lt.and.s32 q, %0, %3, p;\n\t"
                     "@q st.global.v8.b32 [%4], {%5, %6, %7, %8, %9, %5, %5, %5};\n\t"
                     "@p add.s32 %0, %0, 1;\n\t}"
                     : "+r"(ng) : "f"(pst), "f"(theta), "r"(capg), "l"(g), "r"(j), "r"(__float_as_int(Pv[0])),
                       "r"(__float_as_int(Pv[1])), "r"(__float_as_int(Pv[2])), "r"(__float_as_int(Pv[R - 1]))
                     : "memory");
    }
}

// ---------------------------------------------------------------- progress words
// Strips of one pair shared by several warps: a warp waits on the progress
// word of the warp writing its input boundary row.  A word holds (strip tag
// << 32) | steps done.  What a strip waits on and publishes sits in a slot in
// shared memory (read on the renormalisation steps only, so the sweep keeps
// one 32-bit address for it).
struct SyncSlot {
    long long wait_tag;   // tag of the strip whose row bnd_in is
    long long pub_tag;    // tag of this strip
    unsigned wait_addr;   // shared address of the writer's progress word (0: the row is complete)
    unsigned pub_addr;    // shared address of this warp's progress word (0: nobody waits)
};

struct StripIO {
    const float4* bnd_in;
    float4* bnd_out;
    float2* bst;
    int2* bex;
    unsigned sync;        // shared address of this strip's SyncSlot (0: the strip waits on nobody)
};

constexpr long long kStepsDone = 0x7fffffffLL;     // "strip complete" in a progress word
constexpr long long kPass2Tag = 1LL << 20;         // strip tags of pass 2 start here
constexpr int kSpinLimitDefault = 1 << 22;          // bounded wait for a progress word

// Waits (warp-uniform) until the progress word reaches need.  A wait that runs
// out after `limit` polls sets the sync guard, so the pair goes to the FP64
// form; it never hangs, and once the guard is set the warp waits no more (the
// pair's FP32 values are discarded anyway).
__device__ __forceinline__ void wait_progress(const volatile long long* w, long long need, int& flag, int limit);

__device__ __forceinline__ void publish_progress(volatile long long* w, long long v) {
    __threadfence_block();
    *w = v;
}

__device__ __forceinline__ long long lds_vol_s64(unsigned a) {
    long long v;
    asm volatile("ld.volatile.shared.s64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ unsigned lds_vol_u32(unsigned a) {
    unsigned v;
    asm volatile("ld.volatile.shared.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
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
    kGuardStage = 1 << 10,   // a lane's staging area was full
    kGuardPool = 1 << 11,    // the entry pool region was full
    kGuardSync = 1 << 12,    // a wait for another warp's strip ran out
};

__device__ __forceinline__ void wait_progress(const volatile long long* w, long long need, int& flag, int limit) {
    if (!w || (flag & kGuardSync)) return;
    if (limit <= 0) limit = kSpinLimitDefault;
    int it = 0;
    while (*w < need) {
        if (++it > limit) { flag |= kGuardSync; return; }
        __nanosleep(64);
    }
    __threadfence_block();
}

// The strip's wait (warp-uniform) until its writer has done `steps` steps of
// the strip in the slot (nothing without a slot or a writer).
__device__ __forceinline__ void strip_wait(unsigned slot, long long steps, int& flag, int limit) {
    if (!slot || (flag & kGuardSync)) return;
    const unsigned wa = lds_vol_u32(slot + 16);
    if (!wa) return;
    const long long need = lds_vol_s64(slot) | steps;
    if (limit <= 0) limit = kSpinLimitDefault;
    int it = 0;
    while (lds_vol_s64(wa) < need) {
        if (++it > limit) { flag |= kGuardSync; return; }
        __nanosleep(64);
    }
    __threadfence_block();
}

// Publishes this strip's progress (called by the lane that writes the row).
__device__ __forceinline__ void strip_publish(unsigned slot, long long steps) {
    if (!slot) return;
    const unsigned pa = lds_vol_u32(slot + 20);
    if (!pa) return;
    const long long v = lds_vol_s64(slot + 8) | steps;
    __threadfence_block();
    asm volatile("st.volatile.shared.s64 [%0], %1;" ::"r"(pa), "l"(v) : "memory");
}

// ---------------------------------------------------------------- per-warp state
struct GroupCtl;
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
    int4* stg;       // this lane's staging area: capg records of 32 bytes
    int capg;
    const struct GroupCtl* pc;   // the warp's control block (flush targets)
};

// per-warp shared memory (32-bit shared-window addresses): stored-block ring,
// boundary ring, column residues
struct WarpSmem {
    unsigned ring_b;  // [kD][kWarp * kRmax] float2
    unsigned ring_e;  // [kBndSlots][2] float4
    unsigned sy;      // [max_len + 2 kYPad] residue codes
};

// bytes of the (odds, weight) table with `copies` copies: entry e of copy c
// at (e * copies + c) * 8
__host__ __device__ constexpr int tab_bytes(int copies) { return ((kTab * kTab * 8 * copies + 255) / 256) * 256; }
constexpr int kYPad = 33;   // empty codes before column 1 of the staged residues
constexpr unsigned kRingSlot = kWarp * kRmax * 8;   // bytes of one ring slot

__host__ __device__ constexpr int warp_smem_bytes(int max_len) {
    return kD * kWarp * kRmax * 8 + kBndSlots * 32 + ((max_len + 2 * kYPad + 15) / 16) * 16;
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

// Brings the lane's carried values into [1, 2) * 2^e: returns the new
// exponent (or kNoExp for a lane without state, lane `keep` excepted) and the
// factor (1 / 2^k) to apply.
__device__ __forceinline__ int renorm_exp(float mx, int e, bool keep, float& sc) {
    const int k = mx > 0.f ? max(-126, min(126, ilog2f(mx))) : 0;
    sc = pow2f(-k);
    return mx > 0.f ? e + k : (keep ? e : kNoExp);
}

// ---------------------------------------------------------------- pass 1
template <int R, bool STORE>
__device__ __forceinline__ void bwd_strip(const Coef& cf, unsigned s_ow, const PairCtx& c, const WarpSmem& ws,
                                          int s, int nstrips, const StripIO& io, float& Zh, float& Zp,
                                          int& eZh, int& eZp, int& flag)
{
    const int lane = threadIdx.x & 31;
    const int m = c.m, n = c.n;
    const int row0 = s * kStripRows;
    const bool last_strip = (s == nstrips - 1);
    const bool first_strip = (s == 0);
    // byte offset of each row's residue within a table row (in this lane's
    // copy of the table: lane mod copies, 8 bytes apart)
    const unsigned lane_copy = (8u * (unsigned)lane) & (cf.tab_x - 8u);
    unsigned xo[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = row0 + lane * R + r;
        xo[r] = cf.tab_x * (unsigned)((i >= 1 && i <= m) ? (int)__ldg(c.x + i - 1) : kEmpty) + lane_copy;
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
    const float4* bnd_in = io.bnd_in;
    float4* bnd_out = io.bnd_out;
    const bool owns_row = row0 + lane * R <= m;
    // the neighbour below is zero for good: padding rows, or no strip below
    const bool up_zero = (lane == 31) ? (bnd_in == nullptr) : (row0 + (lane + 1) * R > m);
    // starting exponent: the boundary row's exponent, moved to the magnitude of
    // its values at column n (every lane starts there)
    int eH = 0, eP = 0, eUpH = 0, eUpP = 0;
    // the row below is written by another warp: wait for its first columns
    strip_wait(io.sync, 64 + kD, flag, cf.spin_limit);
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
    // the stored block of step t is T = n + 31 - t: this lane's part of it
    // (rows 2h, 2h + 1 at h * 64 + lane * 2 float2; one row: lane)
    float2* blk = STORE ? io.bst + (int64_t)(n + 31) * (kWarp * R) + (R == 1 ? lane : 2 * lane) : nullptr;
    int2* bex = io.bex;
    const int nsteps = n + 32;
    // lane 31 reads the boundary row (column n - t at step t) from the ring,
    // slot t mod kBndSlots
    const bool streams = (lane == 31) && (bnd_in != nullptr);
    // lane 0 writes the boundary row above the strip (none above strip 0;
    // the base then points at the staging area and no store is made)
    const int bnd_lane = (lane == 0 && bnd_out != nullptr) ? 1 : 0;
    float4* const bnd_base = bnd_lane ? bnd_out : (float4*)c.stg;
    // the chunk of steps t0 .. t0 + kBndChunk - 1: lane l copies half l & 1 of
    // the column of step t0 + l / 2 (zeros left of column 0)
    auto fetch_chunk = [&](int t0) {
        const int tl = t0 + (lane >> 1);
        const int jb = n - tl;
        const float4* src = bnd_in + 2 * max(jb, 0) + (lane & 1);
        const unsigned dst = ws.ring_e + 32u * (unsigned)(tl & (kBndSlots - 1)) + 16u * (unsigned)(lane & 1);
        cp_async16(dst, src, jb >= 0 ? 16 : 0);
        cp_async_commit();
    };
    // without a strip below, lane 31 reads zeros from slot 0
    if (!streams && lane == 31) {
        sts_v4(ws.ring_e, make_float4(0.f, 0.f, 0.f, 0.f));
        sts_v4(ws.ring_e + 16u, make_float4(0.f, 0.f, 0.f, 0.f));
    }
    if (bnd_in) {
        fetch_chunk(0);
        cp_async_wait<0>();
        __syncwarp();
    }
    // column residue of the lane, one step ahead (padded: no range check)
    unsigned ya = ws.sy + (unsigned)(n + 31 - lane + kYPad - 1);
    int yc = lds_u8(ya);
    // one step; SPEC: the step holds a corner cell (its own copy of the step,
    // kept out of the loop below)
    auto step = [&](int t, auto spec) {
        constexpr bool SPEC = decltype(spec)::value;
        const int ph = t & (kC - 1);
        const unsigned eba = ws.ring_e + 32u * (unsigned)(streams ? (t & (kBndSlots - 1)) : 0);
        const int j = n + 31 - lane - t;
        if (ph == 0) {
            // the row below is written by another warp: stay 64 steps behind
            // it (column n - T of the row below is written at the writer's
            // step T + 31 and fetched here up to 31 steps ahead)
            strip_wait(io.sync, t + 64, flag, cf.spin_limit);
            if (lane == 0) strip_publish(io.sync, t);
            // this chunk of the boundary row has landed (issued a chunk ago);
            // fetch the next one into the other half of the ring
            if (bnd_in) {
                cp_async_wait<0>();
                __syncwarp();
                fetch_chunk(t + kBndChunk);
            }
            // renormalise: bring the lane's largest carried value into [1, 2)
            float mh = max3f(dDD.x, tV.x, tX2), mp = fmaxf(dDD.y, tV.y);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                mh = max3f(mh, DD[r].x, fmaxf(HB[r].x, BY2o[r]));
                mp = max3f(mp, DD[r].y, HB[r].y);
            }
            const bool live = owns_row && (j >= -1) && (j <= n);
            if (live && !(mh < kBig && mp < kBig)) flag |= kGuardRange;
            float2 sc;
            int fh = renorm_exp(mh, eH, lane == 31, sc.x);
            int fp = renorm_exp(mp, eP, lane == 31, sc.y);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                DD[r] = __fmul2_rn(DD[r], sc); HB[r] = __fmul2_rn(HB[r], sc); BY2o[r] *= sc.x;
            }
            dDD = __fmul2_rn(dDD, sc); tV = __fmul2_rn(tV, sc); tX2 *= sc.x;
            // a lane without state takes the new exponent of the nearest lane
            // below it that has state (lane 31 keeps its own); nothing to do
            // when every lane has state
            if (!__all_sync(kFull, fh != kNoExp && fp != kNoExp)) {
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int vh = __shfl_down_sync(kFull, fh, d), vp = __shfl_down_sync(kFull, fp, d);
                    if (lane + d < 32) {
                        if (fh == kNoExp) fh = vh;
                        if (fp == kNoExp) fp = vp;
                    }
                }
            }
            eH = fh; eP = fp;
            const int uH = __shfl_down_sync(kFull, eH, 1);
            const int uP = __shfl_down_sync(kFull, eP, 1);
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
                const float4 e = lds_v4(eba + 16);
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
        ya -= 1;
        yc = lds_u8(ya);
        // ---- the step proper
        // values of the row below (lane+1's top row; lane 31: the boundary row):
        // (B_M, Zm_b) weighted by the emission of their cell, (B_X, Ze_b), B_X2
        float2 rDD = make_float2(__shfl_down_sync(kFull, DD[0].x, 1), __shfl_down_sync(kFull, DD[0].y, 1));
        float2 rV = make_float2(__shfl_down_sync(kFull, tV.x, 1), __shfl_down_sync(kFull, tV.y, 1));
        float rX2 = __shfl_down_sync(kFull, tX2, 1);
        // lane 31 replaces them by the boundary row's (predicated loads)
        asm volatile("{\n\t.reg .pred q;\n\tsetp.eq.u32 q, %5, 31;\n\t"
                     "@q ld.shared.v4.f32 {%0, %1, %2, %3}, [%6];\n\t@q ld.shared.f32 %4, [%6+16];\n\t}"
                     : "+f"(rDD.x), "+f"(rDD.y), "+f"(rV.x), "+f"(rV.y), "+f"(rX2) : "r"(lane), "r"(eba));
        rDD = __fmul2_rn(rDD, cv); rV = __fmul2_rn(rV, cv); rX2 *= cv.x;
        const unsigned owr = s_ow + (unsigned)yc_now * cf.tab_y;
        float2 D = dDD;
        float2 V = rV;
        float X2b = rX2;
        dDD = rDD;
        float2 Bprev = make_float2(0.f, 0.f);
#pragma unroll
        for (int r = R - 1; r >= 0; --r) {
            const float2 H = HB[r];             // (B_Y, Zf_b) of the cell to the right
            const float Y2b = BY2o[r];
            // (B_X, Ze_b) and (B_Y, Zf_b) of this cell: gap closed by the match
            // below-right, or extended (the carried operand enters last: one
            // operation per row on the vertical chain)
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
            const float2 w = lds_tab(owr + xo[r]);
            if (STORE) {
                // rows (r, r + 1) go out as one 16-byte store
                if (R == 1) st_v2_if_in(j, n, blk, B.x, B.y);
                else if (r & 1) Bprev = B;
                else st_v4_if_in(j, n, blk + r * kWarp, B.x, B.y, Bprev.x, Bprev.y);
            }
            D = DD[r];
            V = nV; X2b = BX2;
            DD[r] = __fmul2_rn(w, B);
            HB[r] = nH; BY2o[r] = BY2;
            if (r == 0) { tV = nV; tX2 = BX2; }
        }
        if (STORE) blk -= kWarp * R;
        st_bnd_if(bnd_lane, j, n, bnd_base + 2 * j, make_float4(DD[0].x, DD[0].y, tV.x, tV.y),
                  make_float4(tX2, 0.f, __int_as_float(eH), __int_as_float(eP)));
    };
    run_steps(nsteps, t_start, t_end, step);
    cp_async_wait<0>();
    __syncwarp();
    if (lane == 0) strip_publish(io.sync, kStepsDone);
}

// The column and the R values of a staging record (16-byte loads).
template <int R>
__device__ __forceinline__ int rec_values(const int4* g, float (&v)[R]) {
    const int4 a = g[0];
    if (R == 1) { v[0] = __int_as_float(a.y); }
    else if (R == 2) { v[0] = __int_as_float(a.y); v[1] = __int_as_float(a.z); }
    else {
        const int4 b = g[1];
        v[0] = __int_as_float(a.y); v[1] = __int_as_float(a.z); v[2] = __int_as_float(a.w); v[R - 1] = __int_as_float(b.x);
    }
    return a.x;
}

// ---------------------------------------------------------------- pass 2
struct FwdOut {      // per-lane results captured at the end corner
    float Zh, Zp;
    int eZh, eZp;
    int A;
};

template <int R, bool LIN>
__device__ __forceinline__ void fwd_strip(const Problem& Pb, unsigned s_ow, const PairCtx& c, const WarpSmem& ws,
                                          int s, int nstrips, const StripIO& io, float2 zfac, int eZh, int eZp,
                                          float scaleA, float& pmax, FwdOut& fo, int64_t& pair_tot, int& flag)
{
    const Coef& cf = Pb.cf;
    const int lane = threadIdx.x & 31;
    const int m = c.m, n = c.n;
    const int row0 = s * kStripRows;
    const bool last_strip = (s == nstrips - 1);
    const bool first_strip = (s == 0);
    // rows outside 1..m get the empty code: their posteriors are 0, below any
    // threshold, so they never produce an entry (offsets in this lane's copy
    // of the table: lane mod copies, 8 bytes apart)
    const unsigned lane_copy = (8u * (unsigned)lane) & (cf.tab_x - 8u);
    unsigned xo[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = row0 + lane * R + r;
        xo[r] = cf.tab_x * (unsigned)((i >= 1 && i <= m) ? (int)__ldg(c.x + i - 1) : kEmpty) + lane_copy;
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
    strip_wait(io.sync, 64 + kD, flag, cf.spin_limit);
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
    const int2* bex = io.bex;
    const float theta = cf.theta;
    const int nsteps = n + 32;
    const int c2 = n & (kC - 1);
    // posterior factor of this lane: 2^(eF + eB - eZ) times zfac (the inverse
    // totals with the combination weights folded in) for each model.  The
    // renormalisation step t (t = c2 mod kC) reads the backward exponents of
    // chunk (n + 31 - t) / kC; they are loaded one renormalisation ahead
    int2 eb = bex[((n + 31) / kC) * 32 + lane];              // step 0
    int2 eb_next = bex[((n + 31 - c2) / kC) * 32 + lane];    // the first renormalisation (t = c2)
    float2 ps;
    // t: the step that starts the chunk
    auto ps_update = [&](int t) {
        const int Eh = eH + eb.x - eZh, Ep = eP + eb.y - eZp;
        const int j0 = t - lane;      // first column of the chunk for this lane
        if (owns_row && (Eh > 126 || Ep > 126) && j0 <= n && j0 + kC >= 0) {
            flag |= kGuardFactor;
            note_guard(c.st, 5, s, t, lane, eH, eb.x, eP, eb.y, m, n);
        }
        ps = make_float2(pow2f(Eh) * zfac.x, pow2f(Ep) * zfac.y);
    };
    ps_update(0);
    // staging of kept entries: one 32-byte record (column, R values; two
    // int4) per step in which the lane's largest posterior reaches the
    // threshold
    int4* grp = c.stg;
    int ng = 0;
    // ring streams: this lane's stored block of step T; lane 0 reads the
    // boundary row (column T at step T) from the boundary ring, slot
    // (T - c2 + kBndChunk) mod kBndSlots: chunks start on the renormalisation
    // steps
    const bool streams = (lane == 0) && (bnd_in != nullptr);
    // lane 31 writes the boundary row below the strip (none below the last;
    // the base then points at the staging area and no store is made)
    const int bnd_lane = (lane == 31 && bnd_out != nullptr) ? 1 : 0;
    float4* const bnd_base = bnd_lane ? bnd_out : (float4*)c.stg;
    const float2* src_b = io.bst + (R == 1 ? lane : 2 * lane);    // block 0, this lane's first rows
    // ring slot layout: the lane's values of rows 2h, 2h+1 (16 bytes) at
    // h * 512 + lane * 16 bytes, so that the 16-byte reads of consecutive
    // lanes hit consecutive banks; one row: lane * 8
    const unsigned ring_lane = ws.ring_b + (R == 1 ? 8u : 16u) * (unsigned)lane;
    auto fetch = [&](int T) {
        // the block of step T exists for this lane when 0 <= T - lane <= n
        const int sz = ((unsigned)(T - lane) <= (unsigned)n) ? 16 : 0;
        const float2* src = src_b + (int64_t)T * (kWarp * R);
        const unsigned dst = ring_lane + kRingSlot * (unsigned)(T & (kD - 1));
        if (R == 1) {
            cp_async8(dst, src, sz >> 1);
        } else {
#pragma unroll
            for (int h = 0; h < R / 2; ++h) cp_async16(dst + 512u * h, src + 2 * kWarp * h, sz);
        }
        cp_async_commit();
    };
    // the boundary chunk of steps T0 .. T0 + kBndChunk - 1: lane l copies half
    // l & 1 of column T0 + l / 2 (zeros outside 0 .. n); it joins the next
    // copy group
    auto fetch_chunk = [&](int T0) {
        const int Tl = T0 + (lane >> 1);
        const float4* src = bnd_in + 2 * min(max(Tl, 0), n) + (lane & 1);
        const unsigned dst = ws.ring_e + 32u * (unsigned)((Tl - c2 + kBndChunk) & (kBndSlots - 1)) +
                             16u * (unsigned)(lane & 1);
        cp_async16(dst, src, (unsigned)Tl <= (unsigned)n ? 16 : 0);
    };
    // lane 0 without a boundary reads zeros from slot 0
    if (!streams && lane == 0) {
        sts_v4(ws.ring_e, make_float4(0.f, 0.f, 0.f, 0.f));
        sts_v4(ws.ring_e + 16u, make_float4(0.f, 0.f, 0.f, 0.f));
    }
    if (bnd_in) {
        // the chunks before and from the first renormalisation step
        fetch_chunk(c2 - kBndChunk);
        fetch_chunk(c2);
        cp_async_commit();
        cp_async_wait<0>();
        __syncwarp();
    }
#pragma unroll
    for (int t = 0; t < kD - 1; ++t) fetch(t);
    unsigned ya = ws.sy + (unsigned)(kYPad - 1 - lane);
    int yc = lds_u8(ya);
    // one step; SPEC: the step holds a corner cell (its own copy of the step,
    // kept out of the loop below)
    auto step = [&](int t, auto spec) {
        constexpr bool SPEC = decltype(spec)::value;
        fetch(t + kD - 1);
        cp_async_wait<kD - 1>();
        const unsigned slot = kRingSlot * (unsigned)(t & (kD - 1));
        const unsigned bsa = ring_lane + slot;
        const unsigned eba = ws.ring_e + (streams ? 32u * (unsigned)((t - c2 + kBndChunk) & (kBndSlots - 1)) : 0u);
        const int j = t - lane;
        const int ph = (t - c2) & (kC - 1);
        if (ph == 0) {
            // the row above is written by another warp: stay 64 steps behind
            // it (column T of the row above is written at the writer's step
            // T + 31 and fetched here up to 31 steps ahead; a writer
            // publishes its progress every kC steps)
            strip_wait(io.sync, t + 64, flag, cf.spin_limit);
            if (lane == 31) strip_publish(io.sync, t);
            // this chunk of the boundary row has landed (its group is older
            // than the kD - 1 the step's wait leaves pending); fetch the next
            // one into the other half of the ring
            if (bnd_in) {
                __syncwarp();
                fetch_chunk(t + kBndChunk);
            }
            float mh = max3f(uMZ.x, lV.x, lX2), mp = fmaxf(uMZ.y, lV.y);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                mh = max3f(mh, MZ[r].x, fmaxf(HY[r].x, Y2i[r]));
                mp = max3f(mp, MZ[r].y, HY[r].y);
            }
            const bool live = owns_row && (j >= 0) && (j <= n + 1);
            if (live && !(mh < kBig && mp < kBig)) flag |= kGuardRange;
            float2 sc;
            int fh = renorm_exp(mh, eH, lane == 0, sc.x);
            int fp = renorm_exp(mp, eP, lane == 0, sc.y);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                MZ[r] = __fmul2_rn(MZ[r], sc); HY[r] = __fmul2_rn(HY[r], sc); Y2i[r] *= sc.x;
            }
            uMZ = __fmul2_rn(uMZ, sc); lV = __fmul2_rn(lV, sc); lX2 *= sc.x;
            // a lane without state takes the new exponent of the nearest lane
            // above it that has state (lane 0 keeps its own); nothing to do
            // when every lane has state
            if (!__all_sync(kFull, fh != kNoExp && fp != kNoExp)) {
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int vh = __shfl_up_sync(kFull, fh, d), vp = __shfl_up_sync(kFull, fp, d);
                    if (lane >= d) {
                        if (fh == kNoExp) fh = vh;
                        if (fp == kNoExp) fp = vp;
                    }
                }
            }
            eH = fh; eP = fp;
            const int uH = __shfl_up_sync(kFull, eH, 1);
            const int uP = __shfl_up_sync(kFull, eP, 1);
            if (lane != 0) { eUpH = uH; eUpP = uP; }
            if (up_zero) { eUpH = eH; eUpP = eP; }
            const int gh = eUpH - eH, gp = eUpP - eP;
            if (live && (gh > 127 || gp > 127)) {
                flag |= kGuardGap;
                note_guard(c.st, 3, s, t, lane, eH, eUpH, eP, eUpP, m, n);
            }
            cv = make_float2(pow2f(gh), pow2f(gp));
            eb = eb_next;
            eb_next = bex[(max(n + 15 - t, 0) / kC) * 32 + lane];   // step t + kC
            ps_update(t);
        } else if (ph == 1) {
            if (streams && t <= n) {
                const float4 e = lds_v4(eba + 16);
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
        ya += 1;
        yc = lds_u8(ya);
        // ---- the step proper
        // values of the row above (lane-1's bottom row; lane 0: the boundary
        // row): the diagonal outflow (M, Zm), the vertical outflow (X, Ze),
        // X2, MEA
        float2 rMZ = make_float2(__shfl_up_sync(kFull, MZ[R - 1].x, 1), __shfl_up_sync(kFull, MZ[R - 1].y, 1));
        float2 rV = make_float2(__shfl_up_sync(kFull, lV.x, 1), __shfl_up_sync(kFull, lV.y, 1));
        float rX2 = __shfl_up_sync(kFull, lX2, 1);
        int rA = __shfl_up_sync(kFull, Aa[R - 1], 1);
        if (lane == 0) {
            const float4 v0 = lds_v4(eba), v1 = lds_v4(eba + 16);
            rMZ = make_float2(v0.x, v0.y); rV = make_float2(v0.z, v0.w); rX2 = v1.x; rA = __float_as_int(v1.y);
        }
        rMZ = __fmul2_rn(rMZ, cv); rV = __fmul2_rn(rV, cv); rX2 *= cv.x;
        const unsigned owr = s_ow + (unsigned)yc_now * cf.tab_y;
        // this step's stored backward values of the lane's rows
        float2 bsv[R];
        if (R == 1) {
            bsv[0] = lds_v2(bsa);
        } else {
#pragma unroll
            for (int h = 0; h < R / 2; ++h) {
                const float4 b = lds_v4(bsa + 512u * h);
                bsv[2 * h] = make_float2(b.x, b.y);
                bsv[2 * h + 1] = make_float2(b.z, b.w);
            }
        }
        float2 dMZ = uMZ;
        int dA = uA;
        float2 aV = rV;
        float aX2 = rX2;
        int aA = rA;
        uMZ = rMZ; uA = rA;
        float Pv[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float2 w = lds_tab(owr + xo[r]);
            const float2 F = __fmul2_rn(w, dMZ);     // (M, Zm) of the cell
            const float2 V = aV, H = HY[r];         // (X, Ze), (Y, Zf) of the cell
            const float FX2 = aX2, FY2 = Y2i[r];
            // outflows: gaps opened from the match or extended; the match
            // continued or closing a gap (diagonal, weighted by the next cell's
            // emission when it is read) (the carried operand enters last: one
            // operation per row on the vertical chain)
            const float2 oF = __fmul2_rn(cf.k_open, F);
            float2 nV = __ffma2_rn(cf.k_ext, V, oF);
            float2 nH = __ffma2_rn(cf.k_ext, H, oF);
            const float oX2 = cf.d2 * F.x;
            float nX2 = fmaf(cf.e2, FX2, oX2);
            float nY2 = fmaf(cf.e2, FY2, oX2);
            float2 nMZ = __ffma2_rn(cf.k_close, __fadd2_rn(V, H), __fmul2_rn(cf.k_mm, F));
            nMZ.x = fmaf(cf.c2, FX2 + FY2, nMZ.x);
            // posteriors of the cell, each with its combination weight folded
            // into the lane's factor, and their combination
            const float2 u = __fmul2_rn(__fmul2_rn(F, ps), bsv[r]);
            const float P = LIN ? (u.x + u.y) : sqrt_approx(fmaf(u.x, u.x, u.y * u.y));
            Pv[r] = P;
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
        // the step's largest posterior of the lane: the guard maximum, and the
        // test for a staging record
        float pst = Pv[0];
        if (R == 2) pst = fmaxf(Pv[0], Pv[1]);
        if (R == 4) pst = fmaxf(max3f(Pv[0], Pv[1], Pv[2]), Pv[3]);
        pmax = fmaxf(pmax, pst);
        stage_record<R>(grp + 2 * ng, ng, c.capg, pst, theta, j, Pv);
        st_bnd_if(bnd_lane, j, n, bnd_base + 2 * j, make_float4(MZ[R - 1].x, MZ[R - 1].y, lV.x, lV.y),
                  make_float4(lX2, __int_as_float(Aa[R - 1]), __int_as_float(eH), __int_as_float(eP)));
    };
    run_steps(nsteps, t_start, t_end, step);
    cp_async_commit();       // a chunk issued on the last step joins no step's group
    cp_async_wait<0>();
    if (lane == 31) strip_publish(io.sync, kStepsDone);
    // ---- flush this strip's entries into the pool (row-major, columns ascending)
    if (ng > c.capg) {
        flag |= kGuardStage;
        ng = c.capg;
    }
    int cnt[R];
#pragma unroll
    for (int r = 0; r < R; ++r) cnt[r] = 0;
    // (unrolled so that several records' loads are in flight at once)
#pragma unroll 4
    for (int g = 0; g < ng; ++g) {
        float v[R];
        rec_values<R>(grp + 2 * g, v);
#pragma unroll
        for (int r = 0; r < R; ++r) cnt[r] += v[r] >= theta ? 1 : 0;
    }
    int tot = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) tot += cnt[r];
    int incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    const int strip_tot = __shfl_sync(kFull, incl, 31);
    const GroupCtl& pc = *c.pc;
    unsigned long long off = 0;
    if (lane == 0 && strip_tot > 0) off = atomicAdd(pc.pool_used, (unsigned long long)strip_tot);
    off = __shfl_sync(kFull, off, 0);
    const bool fits = (int64_t)off + strip_tot <= pc.pool_cap;
    if (!fits) { flag |= kGuardPool; if (lane == 0) atomicExch(&Pb.status->pool_overflow, 1); }
    const int64_t base = pc.pool_base + (int64_t)off;
    int w = incl - tot;
    int2* pool = pc.pool;
    int2* dst[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = row0 + lane * R + r;
        if (i >= 1 && i <= m) pc.rowc[i - 1] = cnt[r];
        dst[r] = pool + base + w;
        w += cnt[r];
    }
    // one pass over the records: every kept value goes to the next place of its row
    if (fits) {
#pragma unroll 2
        for (int g = 0; g < ng; ++g) {
            float v[R];
            const int col = rec_values<R>(grp + 2 * g, v) - 1;
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (v[r] >= theta) { *dst[r] = make_int2(col, __float_as_int(v[r])); ++dst[r]; }
        }
    }
    if (lane == 0) pc.chunk[s] = base;
    pair_tot += strip_tot;
    __syncwarp();
}

// rows per lane of a strip with rows_in rows: the smallest of 1, 2, 4 that covers it
__device__ __forceinline__ int rows_per_lane(int rows_in) {
    const int r = (rows_in + 31) / 32;
    return r <= 1 ? 1 : r <= 2 ? 2 : 4;
}

template <bool STORE>
__device__ __forceinline__ void bwd_dispatch(int Rs, const Coef& cf, unsigned s_ow, const PairCtx& c,
                                             const WarpSmem& ws, int s, int ns, const StripIO& io,
                                             float& Zh, float& Zp, int& eZh, int& eZp, int& flag) {
    switch (Rs) {
        case 1: bwd_strip<1, STORE>(cf, s_ow, c, ws, s, ns, io, Zh, Zp, eZh, eZp, flag); break;
        case 2: bwd_strip<2, STORE>(cf, s_ow, c, ws, s, ns, io, Zh, Zp, eZh, eZp, flag); break;
        default: bwd_strip<4, STORE>(cf, s_ow, c, ws, s, ns, io, Zh, Zp, eZh, eZp, flag); break;
    }
}

template <bool LIN>
__device__ __forceinline__ void fwd_dispatch(int Rs, const Problem& Pb, unsigned s_ow, const PairCtx& c,
                                             const WarpSmem& ws, int s, int ns, const StripIO& io, float2 zfac,
                                             int eZh, int eZp, float scaleA, float& pmax, FwdOut& fo,
                                             int64_t& pair_tot, int& flag) {
    switch (Rs) {
        case 1: fwd_strip<1, LIN>(Pb, s_ow, c, ws, s, ns, io, zfac, eZh, eZp, scaleA, pmax, fo, pair_tot, flag); break;
        case 2: fwd_strip<2, LIN>(Pb, s_ow, c, ws, s, ns, io, zfac, eZh, eZp, scaleA, pmax, fo, pair_tot, flag); break;
        default: fwd_strip<4, LIN>(Pb, s_ow, c, ws, s, ns, io, zfac, eZh, eZp, scaleA, pmax, fo, pair_tot, flag); break;
    }
}

// Control block of one group of warps working on one pair (shared memory).
struct GroupCtl {
    long long prog[4];          // progress word of each warp of the group
    SyncSlot slot[4];           // what each warp's current strip waits on and publishes
    int q;                      // the group's current work item
    int pad;
    float Zh, Zp;               // pass-1 totals (from the warp of strip 0)
    int eZh, eZp;
    float fZh, fZp;             // pass-2 corner values (from the warp of the last strip)
    int feh, fep, fA;
    int flag[4];
    float pmax[4];
    long long tot[4];
    // the pair's flush targets (written once per pair by the warp's lane 0)
    int2* pool;
    unsigned long long* pool_used;
    int64_t* chunk;             // chunk_off of the pair's first strip
    int32_t* rowc;              // row_cnt of the pair's first row (row i at rowc[i - 1])
    long long pool_base, pool_cap;
};

// Barrier of one group.  Group g of W warps uses named barrier g + 1 (literal
// ids: a register id would reserve all 16 barriers of the block and cost
// occupancy); a block holds at most 4 groups.
__device__ __forceinline__ void group_sync(int gib, int W) {
    if (W == 1) { __syncwarp(); return; }
    switch (gib) {
        case 0: asm volatile("bar.sync 1, %0;" ::"r"(32 * W) : "memory"); break;
        case 1: asm volatile("bar.sync 2, %0;" ::"r"(32 * W) : "memory"); break;
        case 2: asm volatile("bar.sync 3, %0;" ::"r"(32 * W) : "memory"); break;
        default: asm volatile("bar.sync 4, %0;" ::"r"(32 * W) : "memory"); break;
    }
}

__host__ __device__ constexpr size_t posterior_f32_smem_bytes(int warps_per_block, int max_len, int copies) {
    return (size_t)tab_bytes(copies) + (size_t)warps_per_block * warp_smem_bytes(max_len) +
           (size_t)2 * warps_per_block * sizeof(GroupCtl);
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
// progress word, so the strips of one pair run concurrently.  With W = 2 only
// the first Pb.n_big work items (the longest: items come longest first) are
// shared; once a group draws a later item, its first warp runs that item alone
// and both warps go on drawing items one warp each.  Scratch is then laid out
// per warp (a shared item uses the region of its group's first warp).
template <bool CKPT, int W, bool LIN>
__device__ __forceinline__ void posterior_f32_body(const Problem& Pb) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    stamp_begin(Pb.status->t_f32);
    // the table, tab_copies copies side by side (entry e of copy q at e * copies + q)
    const int copies = Pb.tab_copies > 1 ? kTabCopies : 1;
    float2* s_ow_p = (float2*)s_raw;
    for (int i = threadIdx.x; i < kTab * kTab * copies; i += blockDim.x) s_ow_p[i] = Pb.cst->ow[i / copies];
    const unsigned s_ow = smem_u32(s_raw);
    const unsigned tab_end = tab_bytes(copies);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int nwb = blockDim.x >> 5;
    const int gib = wib / W, wig = wib % W;
    WarpSmem ws;
    {
        const unsigned p = smem_u32(s_raw) + tab_end + (unsigned)wib * (unsigned)warp_smem_bytes(Pb.max_len);
        ws.ring_b = p;
        ws.ring_e = p + kD * kWarp * kRmax * 8;
        ws.sy = p + kD * kWarp * kRmax * 8 + kBndSlots * 32;
    }
    uint8_t* sy_p = s_raw + tab_end + (size_t)wib * warp_smem_bytes(Pb.max_len) + kD * kWarp * kRmax * 8 + kBndSlots * 32;
    // control blocks: one per group, and (W > 1) one per warp for items it runs alone
    GroupCtl* gc = (GroupCtl*)(s_raw + tab_end + (size_t)nwb * warp_smem_bytes(Pb.max_len)) + gib;
    GroupCtl* gcs = W == 1 ? gc : gc - gib + nwb + wib;
    __syncthreads();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t gg0 = gw - wig;          // the first warp of the group
    PairCtx c;
    c.capg = group_capacity(Pb.max_len, Pb.cap);
    if (W == 1) {
        c.bst = Pb.bst + gw * Pb.bst_stride;
        c.bex = Pb.bex + gw * Pb.bex_stride;
        c.bnd = Pb.bnd + gw * Pb.bnd_stride;
        c.bck = Pb.bck + gw * Pb.bck_stride;
    }
    c.stg = (int4*)(Pb.stg + gw * Pb.stg_stride) + (int64_t)lane * 2 * c.capg;
    c.st = Pb.status;

    // boundary rows: one per strip when other warps or a later recompute read
    // them, else one row reused in place (the writer trails the reader)
    const bool bck_rows = CKPT || W > 1;
    const bool bnd_rows = W > 1;
    volatile long long* my_prog = W > 1 ? &gc->prog[wig] : nullptr;
    bool solo = W == 1;                    // drawing items one warp each
    for (;;) {
        int q;
        if (!solo) {
            if (lane == 0) {
                *my_prog = 0;
                if (wig == 0) gc->q = atomicAdd(&Pb.status->work_f32, 1);
            }
            group_sync(gib, W);
            q = *(volatile int*)&gc->q;
            if (q >= Pb.n_work) break;
            if (q >= Pb.n_big) {
                // a one-warp item: the first warp runs it, then both draw alone
                solo = true;
                if (wig != 0) continue;
            }
        } else {
            if (lane == 0) gcs->q = atomicAdd(&Pb.status->work_f32, 1);
            __syncwarp();
            q = *(volatile int*)&gcs->q;
            __syncwarp();
            if (q >= Pb.n_work) break;
        }
        // warps on this item and this warp's place among them
        const int nw = solo ? 1 : W;
        const int wg = solo ? 0 : wig;
        if (W > 1) {
            const int64_t unit = solo ? gw : gg0;
            c.bst = Pb.bst + (CKPT ? gw : unit) * Pb.bst_stride;
            c.bex = Pb.bex + (CKPT ? gw : unit) * Pb.bex_stride;
            c.bnd = Pb.bnd + unit * Pb.bnd_stride;
            c.bck = Pb.bck + unit * Pb.bck_stride;
        }
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
        // what the strip flushes write to, read from shared memory there
        // (no chain of dependent global loads at the end of every strip)
        if (lane == 0) {
            gcs->pool = fd.pool ? fd.pool : Pb.pool;
            gcs->pool_used = fd.pool_used;
            gcs->chunk = fd.chunk_off + fd.pair_strip_off[p];
            gcs->rowc = fd.row_cnt + fd.pair_row_off[p];
            gcs->pool_base = fd.pool_base;
            gcs->pool_cap = fd.pool_cap;
        }
        c.pc = gcs;
        const int m = c.m, n = c.n;
        const int nstrips = (m + 1 + kStripRows - 1) / kStripRows;
        // the column residues of the pair, staged once, with empty codes on
        // both sides so that every skewed column index reads a valid byte
        // (four loads of a lane in flight)
        __syncwarp();
#pragma unroll 4
        for (int i = lane; i < n + 2 * kYPad; i += 32) {
            const int jj = i - kYPad;
            sy_p[i] = (jj >= 0 && jj < n) ? c.y[jj] : (uint8_t)kEmpty;
        }
        __syncwarp();
        int flag = 0;
        // ---- pass 1: backward, bottom strip first (strip s: warp (ns-1-s) % nw)
        float Zh = 0.f, Zp = 0.f;
        int eZh = 0, eZp = 0;
        const int64_t strip_vals = (int64_t)kStripRows * (n + 32), strip_exps = (int64_t)c.nch * 32;
        const int64_t row_len = 2 * (int64_t)(n + 1);
        for (int s = nstrips - 1 - wg, seq = 0; s >= 0; s -= nw, ++seq) {
            const int rows_in = min(kStripRows, m + 1 - s * kStripRows);
            const int Rs = rows_per_lane(rows_in);
            StripIO io;
            io.bnd_in = (s == nstrips - 1) ? nullptr : c.bck + (bck_rows ? (s + 1) * row_len : 0);
            io.bnd_out = (s == 0) ? nullptr : c.bck + (bck_rows ? s * row_len : 0);
            io.sync = 0;
            if (nw > 1) {
                SyncSlot* sl = &gc->slot[wg];
                if (lane == 0) {
                    const int ps = nstrips - 2 - s;          // order of strip s + 1 in pass 1
                    sl->wait_addr = s < nstrips - 1 ? smem_u32(&gc->prog[ps % nw]) : 0u;
                    sl->wait_tag = (long long)(ps / nw + 1) << 32;
                    sl->pub_addr = s > 0 ? smem_u32((const void*)my_prog) : 0u;
                    sl->pub_tag = (long long)(seq + 1) << 32;
                }
                __syncwarp();
                io.sync = smem_u32(sl);
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
        GroupCtl* cb = nw > 1 ? gc : gcs;
        if (wg == (nstrips - 1) % nw && lane == 0) {
            cb->Zh = Zh; cb->Zp = Zp; cb->eZh = eZh; cb->eZp = eZp;
        }
        if (nw > 1) group_sync(gib, W);
        else __syncwarp();
        Zh = *(volatile float*)&cb->Zh; Zp = *(volatile float*)&cb->Zp;
        eZh = *(volatile int*)&cb->eZh; eZp = *(volatile int*)&cb->eZp;
        // normalise the totals to [1, 2) * 2^e
        if (!(Zh > 0.f) || !(Zp > 0.f) || !(Zh < kBig) || !(Zp < kBig)) flag |= kGuardTotal;
        {
            const int kh = ilog2f(fmaxf(Zh, 1e-30f)), kp = ilog2f(fmaxf(Zp, 1e-30f));
            Zh *= pow2f(-kh); eZh += kh;
            Zp *= pow2f(-kp); eZp += kp;
        }
        // the inverse totals with the combination weights folded in: the
        // root-mean-square family combines sqrt(wh P_hmm^2 + wp P_pf^2), so
        // each factor carries the root of its weight; the linear family
        // combines wh P_hmm + wp P_pf
        const float2 zfac = LIN ? make_float2(Pb.cf.wh / Zh, Pb.cf.wp / Zp)
                                : make_float2(sqrtf(Pb.cf.wh) / Zh, sqrtf(Pb.cf.wp) / Zp);
        // ---- pass 2: forward + posterior + threshold + MEA, top strip first
        // (strip s: warp s % nw)
        const int mn = min(m, n);
        int sA = 30 - (32 - __clz(mn + 1));
        if (sA > 21) sA = 21;
        const float scaleA = (float)(1 << sA);
        float pmax = 0.f;
        FwdOut fo{0.f, 0.f, 0, 0, 0};
        int64_t pair_tot = 0;
        for (int s = wg, seq = 0; s < nstrips; s += nw, ++seq) {
            const int rows_in = min(kStripRows, m + 1 - s * kStripRows);
            const int Rs = rows_per_lane(rows_in);
            StripIO io;
            io.bnd_in = (s == 0) ? nullptr : c.bnd + (bnd_rows ? (s - 1) * row_len : 0);
            io.bnd_out = (s == nstrips - 1) ? nullptr : c.bnd + (bnd_rows ? s * row_len : 0);
            io.sync = 0;
            if (nw > 1) {
                SyncSlot* sl = &gc->slot[wg];
                if (lane == 0) {
                    sl->wait_addr = s > 0 ? smem_u32(&gc->prog[(s - 1) % nw]) : 0u;
                    sl->wait_tag = (kPass2Tag + (s - 1) / nw + 1) << 32;
                    sl->pub_addr = s < nstrips - 1 ? smem_u32((const void*)my_prog) : 0u;
                    sl->pub_tag = (kPass2Tag + seq + 1) << 32;
                }
                __syncwarp();
                io.sync = smem_u32(sl);
            }
            if (CKPT) {
                // the strip's backward values again, from its checkpoint row
                StripIO bio;
                bio.bnd_in = (s == nstrips - 1) ? nullptr : c.bck + (s + 1) * row_len;
                bio.bnd_out = nullptr;
                bio.bst = c.bst;
                bio.bex = c.bex;
                bio.sync = 0;
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
            fwd_dispatch<LIN>(Rs, Pb, s_ow, c, ws, s, nstrips, io, zfac, eZh, eZp, scaleA, pmax, fo,
                              pair_tot, flag);
            __syncwarp();
        }
        // ---- pair results: partial values of every warp on the item
        float fZh = 0.f, fZp = 0.f;
        int feh = 0, fep = 0, Aend = 0;
        if (wg == (nstrips - 1) % nw) {
            // corner values, held by the lane that owns row m
            const int lastRs = rows_per_lane(min(kStripRows, m + 1 - (nstrips - 1) * kStripRows));
            const int Lend = (m - (nstrips - 1) * kStripRows) / lastRs;
            fZh = __shfl_sync(kFull, fo.Zh, Lend); fZp = __shfl_sync(kFull, fo.Zp, Lend);
            feh = __shfl_sync(kFull, fo.eZh, Lend); fep = __shfl_sync(kFull, fo.eZp, Lend);
            Aend = __shfl_sync(kFull, fo.A, Lend);
            if (nw > 1 && lane == 0) { gc->fZh = fZh; gc->fZp = fZp; gc->feh = feh; gc->fep = fep; gc->fA = Aend; }
        }
        for (int o = 16; o > 0; o >>= 1) pmax = fmaxf(pmax, __shfl_xor_sync(kFull, pmax, o));
        flag = __reduce_or_sync(kFull, flag);
        int fl = flag;
        float pm = pmax;
        int64_t tot = pair_tot;
        if (nw > 1) {
            if (lane == 0) { gc->flag[wg] = flag; gc->pmax[wg] = pmax; gc->tot[wg] = pair_tot; }
            group_sync(gib, W);
            if (wg == 0 && lane == 0) {
                fl = 0; pm = 0.f; tot = 0;
                for (int w = 0; w < nw; ++w) {
                    fl |= ((volatile int*)gc->flag)[w];
                    pm = fmaxf(pm, ((volatile float*)gc->pmax)[w]);
                    tot += ((volatile long long*)gc->tot)[w];
                }
                fZh = *(volatile float*)&gc->fZh; fZp = *(volatile float*)&gc->fZp;
                feh = *(volatile int*)&gc->feh; fep = *(volatile int*)&gc->fep;
                Aend = *(volatile int*)&gc->fA;
            }
        }
        if (wg == 0 && lane == 0) {
            if (pm > 1.001f) fl |= kGuardPost;
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
        if (nw > 1) group_sync(gib, W);
        else __syncwarp();
    }
    stamp_end(Pb.status->t_f32);
}

// The two occupancy variants: at most 128 registers a thread (16 warps per
// SM, blocks of up to 8 warps), and at most 168 (12 warps per SM).
template <bool CKPT, int W, bool LIN>
__global__ void __launch_bounds__(256, 2) k_posterior_f32_v0(Problem Pb) { posterior_f32_body<CKPT, W, LIN>(Pb); }
template <bool CKPT, int W, bool LIN>
__global__ void __maxnreg__(168) k_posterior_f32_v1(Problem Pb) { posterior_f32_body<CKPT, W, LIN>(Pb); }

using F32Kernel = void (*)(Problem);

// The kernel's forms for one number of warps per pair (defined in
// qp_f32_w1.cu and qp_f32_w2.cu): variant 0 = at most 128 registers (4 blocks
// of 128 threads per SM), 1 = at most 168 (3 blocks); stored or checkpointed;
// root-mean-square or linear combination.
F32Kernel f32_kernel_w1(int variant, bool ckpt, bool lin);
F32Kernel f32_kernel_w2(int variant, bool ckpt, bool lin);

}  // namespace qpk
