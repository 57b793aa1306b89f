// Kernels of the all-pairs posterior stage (paper, Methods, stage I) for sm_103a.
//
//   k_setup            derived tables: pair-HMM odds p(a,b)/(q(a)q(b)) and
//                      partition-function weights exp(s(a,b)/T)
//   k_encode           ASCII residues -> codes 0..19, alphabet check
//   k_seqlogq          per-sequence sum of log q (turns the odds-scaled total
//                      back into the pair-HMM probability)
//   k_posterior_f32    the hot path (qp_f32.cuh, instantiated in qp_f32_w1.cu
//                      and qp_f32_w2.cu): launch configuration and wrappers here
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
#include "qp_f32.cuh"

#include <map>
#include <mutex>
#include <utility>

#include <cstdio>

namespace qpk {

#define FULL 0xffffffffu

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

// lin: a linear combination of the two posteriors (combine modes other than
// the root mean square), compiled as its own kernel so the default keeps no
// per-cell test of the mode
static F32Kernel f32_kernel(int variant, bool ckpt, int wpp = 1, bool lin = false) {
    return wpp == 2 ? f32_kernel_w2(variant, ckpt, lin) : f32_kernel_w1(variant, ckpt, lin);
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

size_t posterior_f32_smem(int warps_per_block, int max_len, int tab_copies) {
    return posterior_f32_smem_bytes(warps_per_block, max_len, tab_copies > 1 ? kTabCopies : 1);
}

int posterior_f32_tab_copies(int warps_per_block, int max_len, int smem_per_sm) {
    // (1 KB of every block's shared memory is reserved by the system)
    const size_t need = 2 * (posterior_f32_smem(warps_per_block, max_len, kTabCopies) + 1024);
    return need <= (size_t)smem_per_sm ? kTabCopies : 1;
}

int posterior_f32_occupancy(int warps_per_block, int max_len, int* blocks_per_sm, int variant, bool ckpt,
                            int wpp, int tab_copies) {
    const size_t smem = posterior_f32_smem(warps_per_block, max_len, tab_copies);
    const F32Kernel k = f32_kernel(variant, ckpt, wpp);
    set_smem(k, smem);
    set_smem(f32_kernel(variant, ckpt, wpp, true), smem);    // the linear-combination kernel too (no attribute
                                                             // call inside a later stream capture)
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, warps_per_block * 32, smem);
}

cudaError_t launch_posterior_f32(const Problem& P, int grid, int warps_per_block, cudaStream_t s,
                                 int variant) {
    const size_t smem = posterior_f32_smem(warps_per_block, P.max_len, P.tab_copies);
    if (P.wpp != 1 && P.wpp != 2) return cudaErrorInvalidValue;
    // at most 8 warps a block (the launch bounds) and 4 groups of several
    // warps (the named barriers)
    if (warps_per_block > 8 || warps_per_block % P.wpp || (P.wpp > 1 && warps_per_block / P.wpp > 4))
        return cudaErrorInvalidValue;
    const F32Kernel k = f32_kernel(variant, P.ckpt != 0, P.wpp, P.cf.combine != 0);
    cudaError_t e = set_smem(k, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, warps_per_block * 32, smem, s>>>(P);
    return cudaGetLastError();
}

// ================================================================ FP64 form
//
// Plain FP64 evaluation: one CTA per pair, anti-diagonal wavefront over the
// (m+1) x (n+1) grid.  Pass 1 (backward) stores (B_M, Zm_b) densely; pass 2
// (forward) forms the posteriors, the combination, the threshold and the MEA
// recurrence on each diagonal.
//
// Scaling (per model, per diagonal): a diagonal is computed in the units of
// its predecessor's largest value ("normalised units"), and stored as it is;
// its readers bring it to their own units with one power of two per operand
// (exact), so each diagonal needs one block-wide maximum and one barrier.
// The stored backward values carry the units they were stored in.
constexpr int kF64Threads = 128;
constexpr int kF64Warps = kF64Threads / 32;

// floor(log2 v) for a positive normal double, 0 for 0 (exponent field only)
__device__ __forceinline__ int exp2_of(double v) {
    return v > 0.0 ? (int)((__double_as_longlong(v) >> 52) & 0x7ff) - 1023 : 0;
}
// 2^e for e in the normal range (clamped to it)
__device__ __forceinline__ double pow2d(int e) {
    e = max(-1022, min(1023, e));
    return __longlong_as_double((long long)(e + 1023) << 52);
}

// Largest (mh, mp) over the block: warp maxima go to red[w], and after the
// barrier every thread reads all of them.  red alternates between two
// buffers on consecutive diagonals, so one barrier per diagonal suffices.
__device__ __forceinline__ double2 block_max2(double mh, double mp, double2* red) {
    for (int o = 16; o; o >>= 1) {
        mh = fmax(mh, __shfl_xor_sync(FULL, mh, o));
        mp = fmax(mp, __shfl_xor_sync(FULL, mp, o));
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[w] = make_double2(mh, mp);
    __syncthreads();
    double2 r = red[0];
#pragma unroll
    for (int i = 1; i < kF64Warps; ++i) { const double2 v = red[i]; r.x = fmax(r.x, v.x); r.y = fmax(r.y, v.y); }
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
    __shared__ double2 sred2[2][kF64Warps];
    __shared__ double sred[2][2];
    __shared__ int ired[kF64Warps];
    __shared__ int s_q;
    __shared__ unsigned long long s_base;
    const Consts* __restrict__ C = Pb.cst;
    extern __shared__ double s_diag[];
    const int tid = threadIdx.x, nt = blockDim.x;
    double2* Bd = Pb.d_b + (int64_t)blockIdx.x * Pb.d_b_stride;
    // the three rotating diagonals: shared memory when they fit, else global
    double* dg = Pb.f64_smem_diag ? s_diag : Pb.d_diag + (int64_t)blockIdx.x * Pb.d_diag_stride;
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
        // units (HMM, PF): stored units of diagonals d+1 (u1) and d+2 (u2),
        // normalised units of d+1 (v1) = the units diagonal d is computed in
        int u1h = 0, u1p = 0, u2h = 0, u2p = 0, v1h = 0, v1p = 0;
        double Zh = 0.0, Zp = 0.0;
        int eZh = 0, eZp = 0;
        int32_t* EB = rc + L;            // [m+n+1] HMM units of the stored diagonal
        int32_t* EP = EB + (2 * L + 2);  // [m+n+1] PF units of the stored diagonal
        for (int d = m + n; d >= 0; --d) {
            const int ilo = max(0, d - n), ihi = min(m, d);
            double* cur[8];
            for (int v = 0; v < 8; ++v) cur[v] = slot(d, v);
            const double f1h = pow2d(u1h - v1h), f1p = pow2d(u1p - v1p);
            const double f2h = pow2d(u2h - v1h), f2p = pow2d(u2p - v1p);
            double mh = 0.0, mp = 0.0;
            for (int i = ilo + tid; i <= ihi; i += nt) {
                const int j = d - i;
                double D = 0, Dp = 0, Xb = 0, X2b = 0, Eb = 0, Yb = 0, Y2b = 0, Fb = 0;
                if (i < m && j < n) {
                    const int o = Y(j + 1) * kTab + X(i + 1);
                    D = C->oddsd[o] * (slot(d + 2, 0)[i + 1] * f2h);
                    Dp = C->wd[o] * (slot(d + 2, 5)[i + 1] * f2p);
                }
                if (i < m) {
                    Xb = slot(d + 1, 1)[i + 1] * f1h; X2b = slot(d + 1, 2)[i + 1] * f1h;
                    Eb = slot(d + 1, 6)[i + 1] * f1p;
                }
                if (j < n) {
                    Yb = slot(d + 1, 3)[i] * f1h; Y2b = slot(d + 1, 4)[i] * f1h;
                    Fb = slot(d + 1, 7)[i] * f1p;
                }
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
                    eZh = v1h; eZp = v1p;
                }
                cur[0][i] = BM; cur[1][i] = BX; cur[2][i] = BX2; cur[3][i] = BY; cur[4][i] = BY2;
                cur[5][i] = ZMB; cur[6][i] = ZEB; cur[7][i] = ZFB;
                Bd[(int64_t)i * (n + 1) + j] = make_double2(BM, ZMB);
                mh = fmax(mh, fmax(fmax(BM, BX), fmax(BX2, fmax(BY, BY2))));
                mp = fmax(mp, fmax(ZMB, fmax(ZEB, ZFB)));
            }
            if (tid == 0) { EB[d] = v1h; EP[d] = v1p; }
            const double2 M = block_max2(mh, mp, sred2[d & 1]);
            u2h = u1h; u2p = u1p;
            u1h = v1h; u1p = v1p;
            v1h += exp2_of(M.x); v1p += exp2_of(M.y);
        }
        // totals (thread 0 computed them at d = 0)
        if (tid == 0) { sred[0][0] = Zh; sred[1][0] = Zp; ired[0] = eZh; ired[1] = eZp; }
        __syncthreads();
        Zh = sred[0][0]; Zp = sred[1][0]; eZh = ired[0]; eZp = ired[1];
        __syncthreads();
        // ---- pass 2: forward over d = 0 .. m+n
        // slot values: 0 Mdiag, 1 Xin, 2 X2in, 3 Yin, 4 Y2in, 5 Zd, 6 Ein, 7 Fin, 8 A
        // units as in pass 1, of diagonals d-1 (u1, v1) and d-2 (u2)
        for (int i = tid; i <= m; i += nt) rc[i] = 0;
        __syncthreads();
        u1h = u1p = u2h = u2p = v1h = v1p = 0;
        double fZh = 0, fZp = 0, Aend = 0;
        int feh = 0, fep = 0;
        const double theta = C->thetad;
        const int comb = C->combine;
        const double invZh = 1.0 / Zh, invZp = 1.0 / Zp;
        // the thread for row i is fixed, i = tid (mod nt); with at most two
        // rows a thread, the stored backward values of the next diagonal are
        // loaded one diagonal ahead
        const bool ahead = (m + 1) <= 2 * nt;
        auto bload = [&](int i, int d) -> double2 {
            const int j = d - i;
            return (i >= 1 && i <= m && j >= 1 && j <= n) ? Bd[(int64_t)i * (n + 1) + j] : make_double2(0.0, 0.0);
        };
        double2 bq0 = make_double2(0.0, 0.0), bq1 = bq0;
        for (int d = 0; d <= m + n; ++d) {
            const int ilo = max(0, d - n), ihi = min(m, d);
            double* cur[9];
            for (int v = 0; v < 9; ++v) cur[v] = slot(d, v);
            const double f1h = pow2d(u1h - v1h), f1p = pow2d(u1p - v1p);
            const double f2h = pow2d(u2h - v1h), f2p = pow2d(u2p - v1p);
            // posterior factors of the diagonal: F in the diagonal's units
            // (v1), B in the units it was stored in, over the totals
            const double sph = ldexp(invZh, v1h + EB[d] - eZh), spp = ldexp(invZp, v1p + EP[d] - eZp);
            double2 bn0 = make_double2(0.0, 0.0), bn1 = bn0;
            if (ahead) { bn0 = bload(tid, d + 1); bn1 = bload(tid + nt, d + 1); }
            double mh = 0.0, mp = 0.0;
            const int i0 = ilo + ((tid - ilo) % nt + nt) % nt;
            for (int i = i0; i <= ihi; i += nt) {
                const int j = d - i;
                double Md = 0, Xi = 0, X2i = 0, Yi = 0, Y2i = 0, Zd = 0, Ei = 0, Fi = 0;
                double Adg = 0, Aup = 0, Alf = 0;
                if (i >= 1 && j >= 1) { Md = slot(d - 2, 0)[i - 1] * f2h; Zd = slot(d - 2, 5)[i - 1] * f2p; Adg = slot(d - 2, 8)[i - 1]; }
                if (i >= 1) {
                    Xi = slot(d - 1, 1)[i - 1] * f1h; X2i = slot(d - 1, 2)[i - 1] * f1h;
                    Ei = slot(d - 1, 6)[i - 1] * f1p; Aup = slot(d - 1, 8)[i - 1];
                }
                if (j >= 1) {
                    Yi = slot(d - 1, 3)[i] * f1h; Y2i = slot(d - 1, 4)[i] * f1h;
                    Fi = slot(d - 1, 7)[i] * f1p; Alf = slot(d - 1, 8)[i];
                }
                const int o = Y(j) * kTab + X(i);
                const double FM = C->oddsd[o] * Md, FX = Xi, FX2 = X2i, FY = Yi, FY2 = Y2i;
                const double ZM = C->wd[o] * Zd, ZE = Ei, ZF = Fi;
                double nMd = tMM * FM + c1 * (FX + FY) + c2 * (FX2 + FY2);
                double nXi = d1 * FM + e1 * FX, nX2i = d2 * FM + e2 * FX2;
                double nYi = d1 * FM + e1 * FY, nY2i = d2 * FM + e2 * FY2;
                double nZd = ZM + ZE + ZF, nEi = Wo * ZM + We * ZE, nFi = Wo * ZM + We * ZF;
                double A = 0.0;
                if (i >= 1 && j >= 1) {
                    const double2 b = ahead ? (i == tid ? bq0 : bq1) : Bd[(int64_t)i * (n + 1) + j];
                    const double ph = FM * b.x * sph;
                    const double pp = ZM * b.y * spp;
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
                    feh = v1h; fep = v1p;
                }
                cur[0][i] = nMd; cur[1][i] = nXi; cur[2][i] = nX2i; cur[3][i] = nYi; cur[4][i] = nY2i;
                cur[5][i] = nZd; cur[6][i] = nEi; cur[7][i] = nFi; cur[8][i] = A;
                mh = fmax(mh, fmax(fmax(nMd, nXi), fmax(nX2i, fmax(nYi, nY2i))));
                mp = fmax(mp, fmax(nZd, fmax(nEi, nFi)));
            }
            bq0 = bn0; bq1 = bn1;
            const double2 M = block_max2(mh, mp, sred2[d & 1]);
            u2h = u1h; u2p = u1p;
            u1h = v1h; u1p = v1p;
            v1h += exp2_of(M.x); v1p += exp2_of(M.y);
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

// Shared memory the FP64 form may use for its diagonals: two CTAs per SM.
constexpr size_t kF64DiagSmem = 100 * 1024;

static size_t f64_diag_bytes(int max_len) { return sizeof(double) * 3 * kNS * (size_t)(max_len + 1); }

bool posterior_f64_smem_diag(int max_len) { return f64_diag_bytes(max_len) <= kF64DiagSmem; }

int posterior_f64_occupancy(int* blocks_per_sm) {
    // the attribute is raised once, before any launch (none inside a capture)
    cudaError_t e = cudaFuncSetAttribute(k_posterior_f64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kF64DiagSmem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_posterior_f64,
                                                              kF64Threads, kF64DiagSmem);
}

cudaError_t launch_posterior_f64(const Problem& P, int grid, cudaStream_t s) {
    const size_t smem = P.f64_smem_diag ? f64_diag_bytes(P.max_len) : 0;
    if (smem > kF64DiagSmem) return cudaErrorInvalidValue;
    k_posterior_f64<<<grid, kF64Threads, smem, s>>>(P);
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
