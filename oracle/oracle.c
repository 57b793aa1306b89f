/*
 * Oracle for the all-pairs posterior stage -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark load this file's library.  The product path never calls it and
 * shares no code, header, table or helper with it.
 *
 * What it computes (paper, Methods, stage (I)): for every pair of sequences,
 * posterior probability matrices from a pair hidden Markov model (Durbin et
 * al.) and from a partition function (Miyazawa), a maximum expected accuracy
 * (MEA) alignment score computed on the posterior matrix, and a pairwise
 * distance from that score.  The matrices are stored sparsely (Methods,
 * "Selective consistency", footnote on the sparsity coefficient).
 *
 * The paper prints neither the models nor their parameters.  The readings
 * adopted here (5-state pair-HMM, 3-state affine partition function,
 * root-mean-square combination, threshold P >= theta, distance
 * 1 - A/min(m,n)) are the ones the repository documents; they are written
 * out below as plain definitions in natural-log space, FP64, one cell at a
 * time, with no blocking, fusion or reordering.
 *
 * Parity pins: brute-force enumeration of all paths / alignments / matchings
 * for tiny pairs, forward total = backward total, row and column posterior
 * identities, closed forms for m = n = 1 and m = 1, the ungapped and
 * zero-temperature limits, and the swap symmetry (tests/test_oracle_*.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ---- parameters (own layout; mirrors nothing in the product headers) ---- */
typedef struct {
    double pi[5];           /* start over (M, X, Y, X2, Y2) */
    double delta1, eps1, delta2, eps2;
    double emit_pair[400];  /* p(a,b), a*20+b */
    double emit_bg[20];     /* q(a) */
    double end_w[5];        /* tau_s */
    double score[400];      /* s(a,b) */
    double gap_open, gap_ext, temperature;
    int32_t combine;        /* 0 rms, 1 mean, 2 hmm only, 3 pf only */
    int32_t pad_;
} or_params;

enum { SM = 0, SX = 1, SY = 2, SX2 = 3, SY2 = 4 };

static const double NEG_INF = -INFINITY;

/* log(exp(a) + exp(b)) with -inf handled */
static double lse2(double a, double b) {
    if (a == NEG_INF) return b;
    if (b == NEG_INF) return a;
    if (a > b) return a + log1p(exp(b - a));
    return b + log1p(exp(a - b));
}

static double safe_log(double v) { return v > 0.0 ? log(v) : NEG_INF; }

/* transition t(s -> s') of the 5-state pair-HMM, in log space */
static void transitions(const or_params* p, double lt[5][5]) {
    double t[5][5];
    memset(t, 0, sizeof t);
    t[SM][SM] = 1.0 - 2.0 * p->delta1 - 2.0 * p->delta2;
    t[SM][SX] = p->delta1;  t[SM][SY] = p->delta1;
    t[SM][SX2] = p->delta2; t[SM][SY2] = p->delta2;
    t[SX][SX] = p->eps1;    t[SX][SM] = 1.0 - p->eps1;
    t[SY][SY] = p->eps1;    t[SY][SM] = 1.0 - p->eps1;
    t[SX2][SX2] = p->eps2;  t[SX2][SM] = 1.0 - p->eps2;
    t[SY2][SY2] = p->eps2;  t[SY2][SM] = 1.0 - p->eps2;
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b) lt[a][b] = safe_log(t[a][b]);
}

/* which states consume x_i (X, X2) and which consume y_j (Y, Y2) */
static int eats_x(int s) { return s == SX || s == SX2; }
static int eats_y(int s) { return s == SY || s == SY2; }

#define IDX(i, j) ((size_t)(i) * (size_t)(n + 1) + (size_t)(j))

/*
 * Pair-HMM forward / backward (Durbin et al., cited in Methods, stage I).
 * F_s(i,j): log probability of emitting x_1..x_i, y_1..y_j with the last
 * emission made by state s.  B_s(i,j): log probability of emitting the rest
 * given state s at (i,j).  Emissions: M emits (x_i, y_j) with p; X/X2 emit
 * x_i with q; Y/Y2 emit y_j with q.  Returns log Z from both directions.
 */
static void hmm_fwd_bwd(const uint8_t* x, int m, const uint8_t* y, int n,
                        const or_params* p, double* F[5], double* B[5],
                        double* logz_f, double* logz_b) {
    double lt[5][5];
    transitions(p, lt);
    double lpi[5], ltau[5], lq[20], lp[400];
    for (int s = 0; s < 5; ++s) { lpi[s] = safe_log(p->pi[s]); ltau[s] = safe_log(p->end_w[s]); }
    for (int a = 0; a < 20; ++a) lq[a] = safe_log(p->emit_bg[a]);
    for (int a = 0; a < 400; ++a) lp[a] = safe_log(p->emit_pair[a]);

    /* forward */
    for (int i = 0; i <= m; ++i) {
        for (int j = 0; j <= n; ++j) {
            for (int s = 0; s < 5; ++s) {
                int di = (s == SM || eats_x(s)) ? 1 : 0;
                int dj = (s == SM || eats_y(s)) ? 1 : 0;
                double v = NEG_INF;
                if (i - di < 0 || j - dj < 0 || (i == 0 && j == 0)) { F[s][IDX(i, j)] = NEG_INF; continue; }
                int pi_ = i - di, pj = j - dj;
                if (pi_ == 0 && pj == 0) v = lpi[s];     /* first emission */
                for (int r = 0; r < 5; ++r) {
                    double prev = F[r][IDX(pi_, pj)];
                    if (prev == NEG_INF || lt[r][s] == NEG_INF) continue;
                    v = lse2(v, prev + lt[r][s]);
                }
                double e;
                if (s == SM) e = lp[x[i - 1] * 20 + y[j - 1]];
                else if (eats_x(s)) e = lq[x[i - 1]];
                else e = lq[y[j - 1]];
                F[s][IDX(i, j)] = (v == NEG_INF) ? NEG_INF : v + e;
            }
        }
    }
    double z = NEG_INF;
    for (int s = 0; s < 5; ++s)
        if (F[s][IDX(m, n)] != NEG_INF && ltau[s] != NEG_INF) z = lse2(z, F[s][IDX(m, n)] + ltau[s]);
    *logz_f = z;

    /* backward */
    for (int i = m; i >= 0; --i) {
        for (int j = n; j >= 0; --j) {
            for (int s = 0; s < 5; ++s) {
                if (i == m && j == n) { B[s][IDX(i, j)] = ltau[s]; continue; }
                double v = NEG_INF;
                for (int r = 0; r < 5; ++r) {
                    if (lt[s][r] == NEG_INF) continue;
                    int di = (r == SM || eats_x(r)) ? 1 : 0;
                    int dj = (r == SM || eats_y(r)) ? 1 : 0;
                    int ni = i + di, nj = j + dj;
                    if (ni > m || nj > n) continue;
                    double e;
                    if (r == SM) e = lp[x[ni - 1] * 20 + y[nj - 1]];
                    else if (eats_x(r)) e = lq[x[ni - 1]];
                    else e = lq[y[nj - 1]];
                    double nb = B[r][IDX(ni, nj)];
                    if (nb == NEG_INF || e == NEG_INF) continue;
                    v = lse2(v, lt[s][r] + e + nb);
                }
                B[s][IDX(i, j)] = v;
            }
        }
    }
    /* total from the start: pi_s times the first emission of s */
    double zb = NEG_INF;
    for (int s = 0; s < 5; ++s) {
        int di = (s == SM || eats_x(s)) ? 1 : 0;
        int dj = (s == SM || eats_y(s)) ? 1 : 0;
        if (di > m || dj > n || lpi[s] == NEG_INF) continue;
        double e;
        if (s == SM) e = lp[x[0] * 20 + y[0]];
        else if (eats_x(s)) e = lq[x[0]];
        else e = lq[y[0]];
        double nb = B[s][IDX(di, dj)];
        if (nb == NEG_INF || e == NEG_INF) continue;
        zb = lse2(zb, lpi[s] + e + nb);
    }
    *logz_b = zb;
}

/*
 * Partition function over all alignments (Miyazawa, cited in Methods,
 * stage I; VTML200 scores, trained gap penalties and temperature in the
 * paper, "Other algorithmic improvements").  Boltzmann weights
 * w(a,b) = exp(s(a,b)/T); a gap of length g weighs exp((go + (g-1) ge)/T).
 * Zm: alignments of the prefixes ending in the aligned pair (x_i, y_j);
 * Ze: ending in a gap in y (x_i unaligned); Zf: ending in a gap in x.
 * Zm(0,0) = 1 is the empty alignment; Ze and Zf never follow one another.
 */
static void pf_fwd_bwd(const uint8_t* x, int m, const uint8_t* y, int n,
                       const or_params* p, double* Zm, double* Ze, double* Zf,
                       double* Bm, double* Be, double* Bf,
                       double* logz_f, double* logz_b) {
    const double T = p->temperature;
    const double lo = p->gap_open / T, le = p->gap_ext / T;
    for (int i = 0; i <= m; ++i) {
        for (int j = 0; j <= n; ++j) {
            size_t c = IDX(i, j);
            if (i == 0 && j == 0) { Zm[c] = 0.0; Ze[c] = NEG_INF; Zf[c] = NEG_INF; continue; }
            double vm = NEG_INF, ve = NEG_INF, vf = NEG_INF;
            if (i >= 1 && j >= 1) {
                size_t d = IDX(i - 1, j - 1);
                double s = lse2(lse2(Zm[d], Ze[d]), Zf[d]);
                if (s != NEG_INF) vm = s + p->score[x[i - 1] * 20 + y[j - 1]] / T;
            }
            if (i >= 1) {
                size_t u = IDX(i - 1, j);
                ve = lse2(Zm[u] == NEG_INF ? NEG_INF : Zm[u] + lo,
                          Ze[u] == NEG_INF ? NEG_INF : Ze[u] + le);
            }
            if (j >= 1) {
                size_t l = IDX(i, j - 1);
                vf = lse2(Zm[l] == NEG_INF ? NEG_INF : Zm[l] + lo,
                          Zf[l] == NEG_INF ? NEG_INF : Zf[l] + le);
            }
            Zm[c] = vm; Ze[c] = ve; Zf[c] = vf;
        }
    }
    size_t e = IDX(m, n);
    *logz_f = lse2(lse2(Zm[e], Ze[e]), Zf[e]);

    for (int i = m; i >= 0; --i) {
        for (int j = n; j >= 0; --j) {
            size_t c = IDX(i, j);
            if (i == m && j == n) { Bm[c] = 0.0; Be[c] = 0.0; Bf[c] = 0.0; continue; }
            double dm = NEG_INF, de = NEG_INF, df = NEG_INF;
            if (i < m && j < n) {
                size_t d = IDX(i + 1, j + 1);
                if (Bm[d] != NEG_INF) dm = Bm[d] + p->score[x[i] * 20 + y[j]] / T;
            }
            if (i < m) de = Be[IDX(i + 1, j)];
            if (j < n) df = Bf[IDX(i, j + 1)];
            /* from M: next is M, or open a gap of either kind */
            Bm[c] = lse2(lse2(dm, de == NEG_INF ? NEG_INF : de + lo),
                         df == NEG_INF ? NEG_INF : df + lo);
            /* from E: next is M, or extend the same gap */
            Be[c] = lse2(dm, de == NEG_INF ? NEG_INF : de + le);
            Bf[c] = lse2(dm, df == NEG_INF ? NEG_INF : df + le);
        }
    }
    *logz_b = Bm[IDX(0, 0)];
}

/*
 * One pair, everything dense.  Outputs (all optional except P):
 *   P_hmm, P_pf, P : [m*n], row-major over residues (row i-1 for x_i,
 *                    column j-1 for y_j);
 *   gx_hmm [m], gy_hmm [n] : posterior of the gap states at each row /
 *                    column (X + X2, Y + Y2); gx_pf, gy_pf likewise (E, F);
 *   logz[4] : log Z_hmm forward, backward, log Z_pf forward, backward;
 *   mea, dist : MEA score A(m,n) on the dense combined P and 1 - A/min(m,n).
 * Returns 0, or -1 if memory ran out.
 */
int or_pair(const uint8_t* x, int m, const uint8_t* y, int n, const or_params* p,
            double* P_hmm, double* P_pf, double* P,
            double* gx_hmm, double* gy_hmm, double* gx_pf, double* gy_pf,
            double* logz, double* mea, double* dist) {
    size_t cells = (size_t)(m + 1) * (size_t)(n + 1);
    double* buf = (double*)malloc(sizeof(double) * cells * 16);
    if (!buf) return -1;
    double *F[5], *Bk[5];
    for (int s = 0; s < 5; ++s) { F[s] = buf + cells * s; Bk[s] = buf + cells * (5 + s); }
    double *Zm = buf + cells * 10, *Ze = buf + cells * 11, *Zf = buf + cells * 12;
    double *Bm = buf + cells * 13, *Be = buf + cells * 14, *Bf = buf + cells * 15;

    double zhf, zhb, zpf, zpb;
    hmm_fwd_bwd(x, m, y, n, p, F, Bk, &zhf, &zhb);
    pf_fwd_bwd(x, m, y, n, p, Zm, Ze, Zf, Bm, Be, Bf, &zpf, &zpb);
    if (logz) { logz[0] = zhf; logz[1] = zhb; logz[2] = zpf; logz[3] = zpb; }

    /* posteriors of the match state / aligned pair, and their combination */
    double* Pc = P;
    for (int i = 1; i <= m; ++i) {
        for (int j = 1; j <= n; ++j) {
            size_t c = IDX(i, j);
            double ph = (F[SM][c] == NEG_INF || Bk[SM][c] == NEG_INF) ? 0.0
                        : exp(F[SM][c] + Bk[SM][c] - zhf);
            double pp = (Zm[c] == NEG_INF || Bm[c] == NEG_INF) ? 0.0
                        : exp(Zm[c] + Bm[c] - zpf);
            double v;
            switch (p->combine) {
                case 1: v = 0.5 * (ph + pp); break;
                case 2: v = ph; break;
                case 3: v = pp; break;
                default: v = sqrt(0.5 * (ph * ph + pp * pp)); break;
            }
            size_t o = (size_t)(i - 1) * (size_t)n + (size_t)(j - 1);
            if (P_hmm) P_hmm[o] = ph;
            if (P_pf) P_pf[o] = pp;
            Pc[o] = v;
        }
    }
    /* gap-state posteriors (used by the row / column identity pins) */
    if (gx_hmm || gx_pf) {
        for (int i = 1; i <= m; ++i) {
            double gh = 0.0, gp = 0.0;
            for (int j = 0; j <= n; ++j) {
                size_t c = IDX(i, j);
                if (F[SX][c] != NEG_INF && Bk[SX][c] != NEG_INF) gh += exp(F[SX][c] + Bk[SX][c] - zhf);
                if (F[SX2][c] != NEG_INF && Bk[SX2][c] != NEG_INF) gh += exp(F[SX2][c] + Bk[SX2][c] - zhf);
                if (Ze[c] != NEG_INF && Be[c] != NEG_INF) gp += exp(Ze[c] + Be[c] - zpf);
            }
            if (gx_hmm) gx_hmm[i - 1] = gh;
            if (gx_pf) gx_pf[i - 1] = gp;
        }
    }
    if (gy_hmm || gy_pf) {
        for (int j = 1; j <= n; ++j) {
            double gh = 0.0, gp = 0.0;
            for (int i = 0; i <= m; ++i) {
                size_t c = IDX(i, j);
                if (F[SY][c] != NEG_INF && Bk[SY][c] != NEG_INF) gh += exp(F[SY][c] + Bk[SY][c] - zhf);
                if (F[SY2][c] != NEG_INF && Bk[SY2][c] != NEG_INF) gh += exp(F[SY2][c] + Bk[SY2][c] - zhf);
                if (Zf[c] != NEG_INF && Bf[c] != NEG_INF) gp += exp(Zf[c] + Bf[c] - zpf);
            }
            if (gy_hmm) gy_hmm[j - 1] = gh;
            if (gy_pf) gy_pf[j - 1] = gp;
        }
    }
    free(buf);

    /*
     * Maximum expected accuracy (Methods, stage I): the largest sum of
     * posteriors over monotone matchings of x and y,
     * A(i,j) = max(A(i-1,j-1) + P(i,j), A(i-1,j), A(i,j-1)), A(0,.) = A(.,0) = 0.
     */
    double* A = (double*)malloc(sizeof(double) * cells);
    if (!A) return -1;
    for (int j = 0; j <= n; ++j) A[IDX(0, j)] = 0.0;
    for (int i = 1; i <= m; ++i) {
        A[IDX(i, 0)] = 0.0;
        for (int j = 1; j <= n; ++j) {
            double diag = A[IDX(i - 1, j - 1)] + Pc[(size_t)(i - 1) * n + (j - 1)];
            double best = A[IDX(i - 1, j)];
            if (A[IDX(i, j - 1)] > best) best = A[IDX(i, j - 1)];
            if (diag > best) best = diag;
            A[IDX(i, j)] = best;
        }
    }
    double score = A[IDX(m, n)];
    free(A);
    if (mea) *mea = score;
    /* distance from the alignment score, normalised by the shorter length */
    if (dist) *dist = 1.0 - score / (double)(m < n ? m : n);
    return 0;
}

/* ---- family level: all listed pairs on a thread pool (CPU baseline) ---- */
typedef struct {
    const uint8_t* codes; const int64_t* off; const int32_t* pa; const int32_t* pb;
    int64_t n_pairs; const or_params* p; double theta;
    double* logz; double* mea; double* dist; int64_t* nnz;
    int64_t next; pthread_mutex_t mu; int err;
} or_job;

static void* or_worker(void* arg) {
    or_job* J = (or_job*)arg;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t q = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (q >= J->n_pairs) break;
        int a = J->pa[q], b = J->pb[q];
        const uint8_t* x = J->codes + J->off[a];
        const uint8_t* y = J->codes + J->off[b];
        int m = (int)(J->off[a + 1] - J->off[a]), n = (int)(J->off[b + 1] - J->off[b]);
        double* P = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
        double lz[4], me, d;
        if (!P || or_pair(x, m, y, n, J->p, NULL, NULL, P, NULL, NULL, NULL, NULL, lz, &me, &d) != 0) {
            free(P);
            pthread_mutex_lock(&J->mu); J->err = 1; pthread_mutex_unlock(&J->mu);
            continue;
        }
        int64_t cnt = 0;
        for (size_t c = 0; c < (size_t)m * (size_t)n; ++c) cnt += P[c] >= J->theta;
        free(P);
        if (J->logz) { J->logz[2 * q] = lz[0]; J->logz[2 * q + 1] = lz[2]; }
        if (J->mea) J->mea[q] = me;
        if (J->dist) J->dist[q] = d;
        if (J->nnz) J->nnz[q] = cnt;
    }
    return NULL;
}

/* Runs or_pair on the listed pairs (codes are residue indices 0..19). */
int or_pairs(const uint8_t* codes, const int64_t* off, const int32_t* pa, const int32_t* pb,
             int64_t n_pairs, const or_params* p, double theta, int threads,
             double* logz /* [2*n_pairs] */, double* mea, double* dist, int64_t* nnz) {
    or_job J;
    memset(&J, 0, sizeof J);
    J.codes = codes; J.off = off; J.pa = pa; J.pb = pb; J.n_pairs = n_pairs; J.p = p;
    J.theta = theta; J.logz = logz; J.mea = mea; J.dist = dist; J.nnz = nnz;
    pthread_mutex_init(&J.mu, NULL);
    if (threads < 1) threads = 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
    for (int t = 0; t < threads; ++t) pthread_create(&th[t], NULL, or_worker, &J);
    for (int t = 0; t < threads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&J.mu);
    return J.err ? -1 : 0;
}
