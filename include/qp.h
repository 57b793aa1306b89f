/*
 * qp.h -- C ABI of the all-pairs posterior stage (libqp.so, sm_103a).
 *
 * Operation (paper, Methods, stage I): for every pair of sequences of a
 * family, posterior probability matrices are computed from a pair hidden
 * Markov model and a partition function; maximum expected accuracy (MEA)
 * alignment scores on those matrices give the pairwise distances that feed
 * the guide tree.  The matrices are kept sparse (Methods, "Selective
 * consistency", footnote: sparsity coefficient beta < 1).
 *
 * The paper prints neither models nor parameters.  This library computes,
 * for each pair (x, y) with lengths m, n:
 *   - the 5-state pair-HMM (M, X, Y, X2, Y2) forward/backward and the match
 *     posterior P_hmm(i,j);
 *   - the 3-state affine partition function forward/backward and the
 *     aligned-pair posterior P_pf(i,j);
 *   - the combination P(i,j) (root mean square by default);
 *   - the sparse matrix {(i,j): P(i,j) >= threshold} in CSR form;
 *   - the MEA score A = max over monotone matchings of sum P, and the
 *     distance d = 1 - A / min(m, n).
 *
 * Conventions
 *   Pairs: a < b, linear index p = a*k - a(a+1)/2 + (b - a - 1).  Rows of
 *   pair p index sequence a (row i-1 <-> residue x_i), columns index
 *   sequence b.  The pair (b, a) is the transpose.
 *   Residues: ASCII letters of the 20-letter alphabet ACDEFGHIKLMNPQRSTVWY,
 *   or in nucleotide mode (params->alphabet = QP_NUCLEOTIDE) of A, C, G, T
 *   with U read as T (lower case accepted).  Any other byte -> QP_EINVAL.
 *   Ownership: inputs are borrowed for the duration of the call.  A
 *   qp_result is owned by the library and released with qp_result_free.
 *   Errors: every entry point returns a qp_status; qp_last_error() gives a
 *   thread-local message for the last failure on the calling thread.
 *   Streams: work is issued on params->stream (a cudaStream_t), or on a
 *   library-owned stream of params->device when it is NULL; that stream
 *   first waits for all work issued so far to the legacy default stream,
 *   so inputs written there are complete.  qp_posteriors
 *   returns after the results are complete on the device.
 */
#ifndef QP_H
#define QP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QP_OK = 0,
    QP_EINVAL = 1,      /* malformed family or parameters */
    QP_ENOMEM = 2,      /* device or host allocation failed */
    QP_ECUDA = 3,       /* a CUDA call failed (message has the CUDA error) */
    QP_ETIMEOUT = 4,    /* a bounded wait ran out (server poll) */
    QP_ECANCELLED = 5,  /* the request was cancelled or the server shut down */
    QP_ENOTREADY = 6    /* server poll: the request has not finished yet */
} qp_status;

enum { QP_COMBINE_RMS = 0, QP_COMBINE_MEAN = 1, QP_COMBINE_HMM = 2, QP_COMBINE_PF = 3 };
enum { QP_F32_SCALED = 0, QP_F64_PLAIN = 1 };
enum { QP_PROTEIN = 0, QP_NUCLEOTIDE = 1 };

/* A family of k sequences laid out as one buffer.
 *   residues : concatenated ASCII residues, offsets[k] bytes; host memory,
 *              or device memory of params->device when residues_on_device.
 *   offsets  : HOST array of k+1 int64, offsets[0] = 0, strictly increasing
 *              (every sequence non-empty).  2 <= k <= 46340. */
typedef struct qp_family {
    int32_t k;
    int32_t residues_on_device;
    const uint8_t* residues;
    const int64_t* offsets;
} qp_family;

/* Model and run parameters (all host memory).
 *   Pair-HMM: start distribution pi over (M, X, Y, X2, Y2); M->M = 1 - 2 d1 - 2 d2,
 *   M->X = M->Y = delta1, M->X2 = M->Y2 = delta2, X->X = Y->Y = eps1,
 *   X2->X2 = Y2->Y2 = eps2, every gap state returns to M; emit_pair[a*20+b]
 *   = p(a,b) (sums to 1), emit_bg[a] = q(a) > 0 (sums to 1), end weights
 *   end_w[s] >= 0.
 *   Partition function: score[a*20+b] = s(a,b), weight exp(s/T); a gap of
 *   length g weighs exp((gap_open + (g-1) gap_ext)/T); temperature T > 0;
 *   end_gap_mode must be 0 (terminal gaps scored as internal ones).
 *   combine: QP_COMBINE_*.  threshold: keep P >= threshold, 0 < threshold <= 1.
 *   precision: QP_F32_SCALED (FP32 recurrences with power-of-two rescaling,
 *   FP64 totals) or QP_F64_PLAIN (FP64 recurrences, one CTA per pair).
 *   device: CUDA ordinal.  stream: cudaStream_t or NULL.
 *   entry_budget: bytes the sparse entries of all pairs may take (col + val,
 *   plus val64 for QP_F64_PLAIN: 8 or 16 bytes an entry); 0 = no budget.  When
 *   the entries at `threshold` exceed it, the threshold is raised to the
 *   smallest value whose entries fit (paper, Methods, "Other algorithmic
 *   improvements": the posterior matrices are fitted into a given amount of
 *   memory by lowering the sparsity coefficient).  That value, one unit in the
 *   last place above the (N+1)-th largest entry (N = entry_budget / bytes an
 *   entry), in the precision the entries are compared in, is reported as
 *   qp_result.threshold_used; entries equal to the (N+1)-th are all dropped.
 *   Must be >= 0.  Servers reject it (QP_EINVAL) and
 *   qp_pair_posteriors_static ignores it.
 *   alphabet: QP_PROTEIN (20 letters, codes in the order ACDEFGHIKLMNPQRSTVWY)
 *   or QP_NUCLEOTIDE (paper, Methods, "Other algorithmic improvements":
 *   nucleotide mode; letters A, C, G, T = codes 0..3, U read as T).  The
 *   tables keep their layout, [a*20+b] and [a]; in nucleotide mode only
 *   entries with a, b < 4 are read, emit_pair over that block and
 *   emit_bg[0..3] sum to 1, and the rest is ignored.  reserved_ must be 0. */
typedef struct qp_params {
    double pi[5];
    double delta1, eps1, delta2, eps2;
    double emit_pair[400];
    double emit_bg[20];
    double end_w[5];
    double score[400];
    double gap_open, gap_ext, temperature;
    int32_t end_gap_mode;
    int32_t combine;
    double threshold;
    int32_t precision;
    int32_t device;
    void* stream;
    int64_t entry_budget;
    int32_t alphabet;
    int32_t reserved_;
} qp_params;

/* Results.  When on_device, every pointer is device memory of the call's
 * device; otherwise host memory.  Layout:
 *   pair_row_off [n_pairs+1] : row_ptr block of pair p starts at
 *                              pair_row_off[p] and has m_a + 1 entries;
 *   row_ptr      [n_rows]    : within pair p, CSR row r (residue x_{r+1})
 *                              holds entries [row_ptr[o+r], row_ptr[o+r+1])
 *                              counted from pair_nnz_off[p];
 *   pair_nnz_off [n_pairs+1] : first entry of pair p in col / val;
 *   col          [nnz]       : 0-based column (residue y_{c+1}), ascending
 *                              within a row;
 *   val          [nnz]       : P(i,j) as float;
 *   val64        [nnz]       : P(i,j) as double (QP_F64_PLAIN only, else NULL);
 *   dist, dist64 [k*k]       : symmetric MEA distances, zero diagonal;
 *   mea          [n_pairs]   : MEA score A(m, n);
 *   log_z_hmm    [n_pairs]   : natural log of the pair-HMM total probability;
 *   log_z_pf     [n_pairs]   : natural log of the partition function;
 *   pair_flags   [n_pairs]   : bit 0 set when an FP32 range guard fired and
 *                              the pair was recomputed by the FP64 form; bits
 *                              2.. name the guard;
 *   kernel_ms[0..3]           : device time of the FP32 posterior kernel and
 *                              of the FP64 kernel (CUDA events around them
 *                              with plain launches; with a CUDA graph, time
 *                              stamps the kernels take themselves), of the
 *                              rest of the call (input staging, CSR
 *                              assembly), and of the whole call (CUDA events
 *                              around it);
 *   n_fallback                : pairs recomputed by the FP64 form;
 *   guard_info[12]            : the first FP32 range-guard event of the call
 *                              (site, strip, step, lane, HMM exponent and its
 *                              neighbour's, PF exponent and its neighbour's,
 *                              m, n), all zero when no guard fired;
 *   threshold_used            : the threshold the entries were kept at, in
 *                              the precision they were compared in (float
 *                              for QP_F32_SCALED): params.threshold, or the
 *                              raised one when params.entry_budget applied. */
typedef struct qp_result {
    int32_t k;
    int32_t on_device;
    int32_t precision;
    int32_t device;
    int64_t n_pairs;
    int64_t n_rows;
    int64_t nnz;
    int64_t* pair_row_off;
    int32_t* row_ptr;
    int64_t* pair_nnz_off;
    int32_t* col;
    float* val;
    double* val64;
    float* dist;
    double* dist64;
    double* mea;
    double* log_z_hmm;
    double* log_z_pf;
    int32_t* pair_flags;
    double kernel_ms[4];
    int64_t n_fallback;
    int32_t guard_info[12];
    double threshold_used;
    void* owner_;            /* library bookkeeping; do not touch */
} qp_result;

/* All-pairs posterior stage of one family (Methods, stage I).
 * On success *out holds a complete result (device or host per
 * out_on_device).  With host output a large family is computed in pair
 * ranges, each range's arrays copied to host memory while the next range
 * computes (option "host_chunks"); the result is the same.
 * Lengths: 1 to 2^20 residues; with FP32 precision at most the device's
 * limit, the counter "f32_max_len" (each warp stages its pair's column
 * residues in shared memory: about 108,000 on B300), else QP_EINVAL before
 * anything runs.
 * Errors: QP_EINVAL (family/params), QP_ENOMEM, QP_ECUDA.
 * On error *out is NULL. */
int qp_posteriors(const qp_family* family, const qp_params* params,
                  int32_t out_on_device, qp_result** out);

/* The pairs p_begin <= p < p_end of one family (the same computation as
 * qp_posteriors, restricted to a range of the linear pair order; paper,
 * Methods, stage I: every pair is independent, so a family's pairs can be
 * split over several GPUs and the pieces gathered).
 *   p_begin, p_end : 0 <= p_begin < p_end <= k(k-1)/2, else QP_EINVAL;
 *   out            : a result of n_pairs = p_end - p_begin pairs, numbered
 *                    from 0 (local pair q is pair p_begin + q of the family);
 *                    pair_row_off and pair_nnz_off start at 0 for the first
 *                    pair of the range; row_ptr, col, val, mea, log totals
 *                    and flags as for qp_posteriors; dist / dist64 are k x k
 *                    with only the range's pairs (both triangles) filled and
 *                    zeros elsewhere, so that the matrices of disjoint ranges
 *                    add up to the family's.
 * Every value equals the one qp_posteriors gives for the same pair.  Errors
 * as for qp_posteriors. */
int qp_posteriors_range(const qp_family* family, const qp_params* params, int64_t p_begin,
                        int64_t p_end, int32_t out_on_device, qp_result** out);

/* Equal-work split of a family's pairs over n_parts ranks (host only, no
 * device needed): bounds[0] = 0 < bounds[1] < ... < bounds[n_parts] =
 * k(k-1)/2, part i = pairs bounds[i] <= p < bounds[i+1] of the linear order,
 * each boundary placed where the cumulative work (sum of m n over the pairs
 * before it) is nearest to i / n_parts of the family's total.
 *   offsets : HOST int64[k + 1] as in qp_family (every sequence non-empty);
 *   bounds  : HOST int64[n_parts + 1], written;
 *   1 <= n_parts <= k(k-1)/2 (every part holds a pair), else QP_EINVAL. */
int qp_split_pairs(int32_t k, const int64_t* offsets, int32_t n_parts, int64_t* bounds);

/* Releases a result and everything it points to.  NULL is ignored.  Device
 * blocks of a result may be kept by the library for the next call of the same
 * shape: call it after the caller's own work that reads the result (on any
 * stream) has completed. */
void qp_result_free(qp_result* result);

/* Serving loop with continuous batching: many families in one run under a
 * device memory limit (Methods, "Other algorithmic improvements": bulk mode
 * and the user-specified memory limit).
 *
 * A server owns three streams of params->device and two threads.  Submitted
 * families are admitted while one of 64 family slots is free and mem_budget
 * holds their bytes (sequences, pair plan, entry pool, results, plus the
 * kernels' per-warp scratch, which grows with the longest admitted
 * sequence): in arrival order, except that a family that does not fit is
 * passed by later ones that do until it has waited past the aging bound.
 * Admitted families stay resident on the device.  The server keeps two
 * persistent launches of the FP32 kernel queued back to back; every launch
 * takes pairs from all admitted families (the family with the least
 * remaining work first; families admitted more than the aging bound ago
 * get up to half of every launch, oldest first), so a family that arrives
 * while others run shares the next launch with them.  Results equal those of qp_posteriors on the same
 * family and parameters.
 *
 *   qp_server_create : params as for qp_posteriors (precision must be
 *                      QP_F32_SCALED; params->stream is ignored); mem_budget
 *                      > 0 bytes; out_on_device 0: results are copied to host
 *                      memory, 1: results stay in device memory (and no
 *                      longer count against the budget once polled).
 *   qp_server_submit : copies the family; returns a ticket.  QP_EINVAL for a
 *                      malformed family, a residue outside the alphabet, a
 *                      sequence longer than the server's FP32 launches take
 *                      (blocks of four warps: about half of "f32_max_len"),
 *                      or a family that can never fit the budget.
 *   qp_server_poll   : waits up to timeout_ms (0: no wait, <0: forever) for
 *                      the ticket; QP_ENOTREADY / QP_ETIMEOUT when not done.
 *                      On success the caller owns *out (qp_result_free); a
 *                      ticket is consumed by the poll that returns its end.
 *                      Server results use kernel_ms as: [0] ms queued before
 *                      admission, [1] ms from admission to the last pair,
 *                      [2] ms of CSR assembly and copy-out, [3] ms from
 *                      submit to completion.
 *   qp_server_cancel : cancels a ticket not yet finished (QP_ECANCELLED on
 *                      poll); pairs already on the device finish first.
 *   qp_server_get_stats : counters below.
 *   qp_server_destroy: cancels pending work, waits for the device, frees
 *                      everything, including results never polled.
 * Environment knobs: QP_SERVER_LAUNCH_MS (target device time of one launch,
 * default 30), QP_SERVER_AGING_MS (aging bound, default 5000). */
typedef struct qp_server qp_server;
typedef struct qp_server_stats {
    int64_t submitted;       /* tickets issued */
    int64_t completed;       /* finished with a result */
    int64_t failed;          /* finished with an error */
    int64_t cancelled;
    int64_t pairs_done;      /* pairs of completed families */
    double cells_done;       /* sum of m*n over those pairs */
    int64_t launches_f32;    /* persistent FP32 launches */
    int64_t launches_f64;    /* FP64 follow-up launches */
    double kernel_ms;        /* device time of all those launches */
    int32_t resident;        /* families holding device memory now */
    int32_t max_resident;    /* most families resident at once */
    int32_t max_families_per_launch;  /* most families sharing one launch */
    int32_t queued;          /* submitted and not yet admitted */
    int64_t reserved_bytes;  /* device bytes held for admitted families */
    int64_t scratch_bytes;   /* device bytes of the kernels' scratch */
} qp_server_stats;
int qp_server_create(const qp_params* params, size_t mem_budget, int32_t out_on_device,
                     qp_server** out);
int qp_server_submit(qp_server* server, const qp_family* family, uint64_t* ticket);
int qp_server_poll(qp_server* server, uint64_t ticket, int32_t timeout_ms,
                   qp_result** out);
int qp_server_cancel(qp_server* server, uint64_t ticket);
int qp_server_get_stats(qp_server* server, qp_server_stats* out);
void qp_server_destroy(qp_server* server);

/* Launch knobs of the FP32 kernel on one device, for benchmarks and tests
 * (no counterpart in the paper).  value -1 (or 0 for the sizes) restores the
 * automatic choice.  Names:
 *   "variant"         0: at most 128 registers a thread (16 warps per SM),
 *                     1: at most 168 registers (12 warps per SM);
 *   "ckpt"            0: stored form (pass 1 keeps the backward values of the
 *                     whole matrix), 1: checkpointed form (pass 1 keeps one
 *                     boundary row per 128-row strip; pass 2 recomputes each
 *                     strip's backward values before its forward sweep);
 *   "wpp"             warps sharing one pair: 1, or 2 (each takes every
 *                     second 128-row strip, trailing the other through the
 *                     boundary row between them); by default the autotuner
 *                     tries 2 when pairs are too few to fill the grid;
 *   "graph"           1 (default): run each call as one captured CUDA graph;
 *                     0: plain launches;
 *   "blocks_per_sm", "warps_per_block" (qp_posteriors: by default the
 *                     autotuner picks blocks of 2 warps with one emission
 *                     table, or, for launches that fill the grid, blocks of
 *                     8 warps with 16 table copies; setting this or
 *                     "tab_copies" fixes the layout; 4 in a server);
 *   "scratch_bytes"   device bytes the kernels' scratch may take (default:
 *                     45% of free memory, at most 48 GiB); the stored form is
 *                     chosen while it fits a full grid, else the checkpointed
 *                     form, on a grid cut to the budget if need be;
 *   "tree_form"       qp_guide_tree: 2 the cluster form (matrix in the
 *                     shared memory of a thread-block cluster; QP_EINVAL from
 *                     qp_guide_tree when it does not fit), 1 one CTA with
 *                     per-slot state in shared memory (k <= 8192), 0 one CTA
 *                     with the state in global memory; automatic: the first
 *                     that fits, in that order;
 *   "tree_ctas"       qp_guide_tree cluster form: CTAs of the cluster (1, 2,
 *                     4, 8 or 16; automatic: about 8 rows per CTA);
 *   "pool_entries"    releases the entry pool and starts later calls from a
 *                     pool of at most this many entries (a call whose entries
 *                     overflow it grows it and runs again; 0: estimated).
 *   "cons_form"       qp_consistency: 1 the staged form (a CTA per row chunk
 *                     of a pair, each third sequence's matrices copied into
 *                     shared memory, 32-bit fixed-point sums), 0 the row form
 *                     (a CTA per pair, matrices read from global memory,
 *                     64-bit fixed-point sums); automatic: the staged form
 *                     when T <= 256 and the sums' bound allows its unit;
 *   "cons_chunk_rows" qp_consistency staged form: at most this many rows of
 *                     x per CTA (0: as many as the shared memory holds);
 *   "cons_ctas_per_sm" qp_consistency staged form: CTAs per SM (1 or 2;
 *                     the shared memory is split between them; automatic: 2
 *                     unless their accumulators would hold fewer than 32
 *                     rows of the longest sequence);
 *   "cons_wait_polls" qp_consistency staged form: waits (each suspends the
 *                     thread for up to 20 us) on a stage buffer's barrier
 *                     before a warp gives up; its CTA then leaves, CTAs
 *                     that start later leave at once, and the call fails
 *                     with QP_ECUDA (default 65536, about a second);
 *   "cons_stall_test" testing only: 1 withholds the first batch's arrival,
 *                     so the first waits run out (the call fails with
 *                     QP_ECUDA and the device stays usable);
 *   "tab_copies"      copies of the emission table each block keeps in
 *                     shared memory: 16 (bank-sliced: lane l reads copy
 *                     l mod 16, so a half-warp's lookups never share a bank;
 *                     56 KB) or 1; -1 automatic (chosen with the block
 *                     layout, see "warps_per_block").  Results are
 *                     identical either way;
 *   "host_chunks"     qp_posteriors with host output: the family's pairs are
 *                     computed in this many ranges of equal work, the
 *                     arrays of a finished range copied to host memory
 *                     while the next range computes (1: never; 0
 *                     automatic: FP32 families of at least 2e9 cells
 *                     without an entry budget, one range per 1.5e9 cells,
 *                     2 to 8).  The result is identical either way;
 *   "spin_limit"      testing only: polls (each about 64 ns of sleep) of a
 *                     warp waiting for the other warp of its pair (wpp = 2)
 *                     before it gives up and the pair is recomputed by the
 *                     FP64 form (0: the default, about 4 million);
 *   "cons_min_unit"   qp_consistency staged form: the coarsest fixed-point
 *                     unit 2^-u it accepts (default 21); a call whose bound
 *                     on the sums needs a coarser unit runs the row form;
 * Applies to later qp_posteriors calls and servers created afterwards.
 * QP_EINVAL for an unknown name or device. */
int qp_set_option(int32_t device, const char* name, int64_t value);

/* Counters of qp_posteriors calls on one device (no counterpart in the
 * paper): "graph_captures" (calls that captured their sequence as a new CUDA
 * graph), "graph_relaunches" (calls that relaunched the cached graph as it
 * was), "plain_calls" (calls with plain launches), "pool_retries" (calls run again because their entries
 * overflowed the entry pool), "consistency_fma" (multiply-adds of the last
 * qp_consistency relaxation), "consistency_form" (form of the last
 * qp_consistency relaxation: 1 staged, 0 row form), "f32_variant",
 * "f32_wpp", "f32_warps_per_block", "f32_tab_copies" (launch configuration
 * of the last qp_posteriors call's FP32 kernel; -1 before the first),
 * "f32_max_len" (the longest sequence the FP32 form takes on the device).
 * QP_EINVAL for an unknown name or device. */
int qp_get_counter(int32_t device, const char* name, int64_t* value);

/* Allocation-free variant for callers that cannot allocate device memory.
 * There is no counterpart in the paper: it exists for code that must not call
 * cudaMalloc / cudaFree while it runs -- for instance a host program whose
 * device memory is all handed to another allocator (a framework's caching
 * pool or a fixed arena) so that a stray cudaMalloc can fail or fragment it,
 * or a latency-critical loop that cannot afford the device-wide
 * synchronisation that cudaMalloc and cudaFree imply.
 *
 * It runs ONE pair (x, y) through the same FP32 posterior kernel as
 * qp_posteriors, taking every piece of scratch memory from a fixed array
 * compiled into libqp.so (about 5.5 MiB, held on every GPU that loads the
 * library until the process exits).  No cudaMalloc, cudaFree or other
 * allocating call is made.
 *   residues : DEVICE memory of params->device, m + n ASCII residues: x
 *              (m letters) immediately followed by y (n letters);
 *   m, n     : 1 <= m, n <= QP_STATIC_MAX_LEN, else QP_EINVAL;
 *   params   : as for qp_posteriors; precision must be QP_F32_SCALED;
 *   row_ptr  : DEVICE int32[m + 1], CSR row pointers of P (rows = x);
 *   col, val : DEVICE int32 / float [nnz_capacity], entries P >= threshold,
 *              columns ascending within a row;
 *   pair_out : DEVICE double[4] = MEA score, MEA distance, log Z_hmm, log Z_pf;
 *   nnz_out  : HOST, the number of entries (also set when nnz_capacity is too
 *              small, in which case QP_EINVAL is returned and the outputs are
 *              left untouched).
 * Values equal those of qp_posteriors for the same pair.  A pair that trips
 * an FP32 range guard returns QP_ENOMEM (its FP64 recomputation needs more
 * scratch than the fixed array holds; call qp_posteriors instead).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) for that device; make that first call before any
 * stream capture.  All calls share the one array: the call clears what has to
 * start at zero, but two calls that overlap on the GPU (other host threads,
 * other streams) race and corrupt each other.  The call returns after its
 * work on params->stream (or the legacy default stream when NULL) is done,
 * with the caller's current device as it was. */
#define QP_STATIC_MAX_LEN 512
int qp_pair_posteriors_static(const uint8_t* residues, int32_t m, int32_t n,
                              const qp_params* params, int32_t* row_ptr, int32_t* col,
                              float* val, int64_t nnz_capacity, double* pair_out,
                              int64_t* nnz_out);

/* Guide tree by weighted UPGMA (paper, Methods, stage II: the distances of
 * stage I feed weighted UPGMA, after Sneath and Sokal).  Repeatedly joins the
 * two clusters at the smallest distance; the distance from the joined cluster
 * to any other is the mean of the distances from its two parts, whatever
 * their sizes.  Clusters live in slots 0..k-1 (slot i starts as leaf i);
 * joining slots i < j puts the new cluster in slot i and empties slot j.
 * Ties: the smallest distance, then the smallest i, then the smallest j.
 * Arithmetic is FP64; the result is bit-identical to any FP64 implementation
 * of the same rule.
 *   dist      : k x k row-major FP64 distances (for instance
 *               qp_result.dist64); only the upper triangle (i < j) is read, so
 *               the matrix is taken as symmetric.  HOST memory, or DEVICE
 *               memory of `device` when on_device != 0.  Entries should be
 *               finite (NaN gives a valid tree of unspecified shape).  Not
 *               modified;
 *   k         : 2 <= k <= 46340, else QP_EINVAL;
 *   merges    : int32[(k - 1) * 2], the ids joined at step s; leaves are
 *               0..k-1 and the cluster formed at step s has id k + s;
 *   heights   : double[k - 1], half the joining distance of step s
 *               (non-decreasing: weighted UPGMA has no inversions);
 *   merges and heights are in the same memory as dist (host or device).
 *   stream    : cudaStream_t to run on, or NULL for the library's stream
 *               (ordered after the legacy default stream, as for
 *               qp_posteriors).
 * Device working memory: 8 k^2 bytes (plus 8 k^2 more for a host matrix),
 * taken and released within the call.  Returns after the outputs are
 * written.  QP_EINVAL for a bad k, NULL pointer or device; QP_ENOMEM when the
 * working memory cannot be allocated; QP_ECUDA otherwise. */
int qp_guide_tree(const double* dist, int32_t k, int32_t on_device, int32_t device, void* stream,
                  int32_t* merges, double* heights);

/* Selective consistency (paper, Methods, stage III and "Selective
 * consistency").  Every posterior matrix S_xy is relaxed through the third
 * sequences z whose tree distances to x and y both stay within T, and its own
 * signal is amplified:
 *   S'_xy = (2 h_xy S_xy + sum_{z in Z_xy} S_xz S_zy) / (2 + |Z_xy|),
 *   Z_xy  = {z not in {x, y} : max(d_xz, d_zy) <= T},
 *   h_xy  = 1 + (h - 1) min(|Z_xy|, n_max) / n_max,
 * where d_xy is the number of sequences in the smallest subtree of the guide
 * tree holding x and y, S_yx is S_xy transposed, and the 2 counts x and y
 * themselves (S_xx = I: the ProbCons relaxation restricted to Z).  Entries
 * below `threshold` are dropped.  FP32 arithmetic; the sum over z runs in
 * the guide tree's leaf order.
 *   T         : tree-distance threshold (the paper: about 200);
 *   n_max     : relaxations at which the amplification reaches h (200);
 *   h         : amplification, >= 1 (the paper: 3);
 *   threshold : entries kept, 0 < threshold <= 1. */
typedef struct qp_consistency_params {
    int32_t T;
    int32_t n_max;
    double h;
    double threshold;
} qp_consistency_params;

/*   posteriors : a qp_posteriors result (host or device, either precision; its
 *                float values are used);
 *   offsets    : HOST int64[k + 1], the family's sequence offsets (lengths
 *                1 .. 51200);
 *   merges     : int32[(k - 1) * 2], a guide tree's joins as qp_guide_tree
 *                writes them (leaves 0..k-1, node of step s = k + s); HOST,
 *                or DEVICE memory of the result's device when
 *                merges_on_device;
 *   out        : a new result in the layout of the posteriors (the relaxed
 *                matrices; dist, dist64, mea, log totals and flags copied
 *                from the input; kernel_ms[0] the device time of the stage).
 * k <= 16384.  QP_EINVAL for bad arguments or merges that are not a join
 * sequence of k leaves, QP_ENOMEM, QP_ECUDA.  Runs on the library's stream
 * and returns after the result is complete. */
int qp_consistency(const qp_result* posteriors, const int64_t* offsets, const int32_t* merges,
                   int32_t merges_on_device, const qp_consistency_params* params, int32_t out_on_device,
                   qp_result** out);

/* Thread-local message of the last failure on the calling thread. */
const char* qp_last_error(void);

/* Library version string. */
const char* qp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* QP_H */
