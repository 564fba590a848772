/*
 * abft_oracle.c -- plain, slow, FP64 CPU oracle for ABFT one-sided decompositions.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, imports or
 * executes this file: only tests/, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or constant with the CUDA path.
 *
 * What it computes (paper: "Improving Energy Saving of One-sided Matrix
 * Decompositions on CPU-GPU Heterogeneous Systems", PPoPP'23):
 *   - Sec. 2.1: the blocked right-looking decomposition skeleton, one iteration
 *     per column block: (1) panel decomposition PD, (2) panel update PU,
 *     (3) trailing matrix update TMU, for Cholesky, LU and QR.
 *   - Sec. 3.1.2: ABFT -- checksums encoded per matrix block before the
 *     operation, the same operation applied to the checksums, the checksum
 *     relation verified after every iteration, errors located and corrected;
 *     single-side (one dimension) and full (both dimensions) checksums; the
 *     0D / 1D / 2D error-propagation classes.
 * The paper gives the checksum scheme only in prose, so the formulas below are
 * a reading: the Huang-Abraham row/column checksum code applied per g x g
 * block (g = the block size b), carried through PU and TMU, with a weighted
 * column checksum (weights 1..g) as the locator for single-side mode.
 *
 * Conventions: row-major storage, leading dimension lda >= n; 0-based indices.
 * Every routine is written as plain loops in the order of the algorithm; there
 * is no blocking, fusion or reordering beyond the algorithm's own blocks.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ types */
typedef struct {
    int32_t step, kind;
    int64_t row, col;
    double delta;
} orc_event;

typedef struct {
    int64_t detected, corrected, uncorrectable, checksum_repaired;
    int32_t nloc, info;
    orc_event loc[64];
    double max_ratio; /* max |d| / tau over tiles that raised no flag */
    double tau;       /* threshold used at the last verified step       */
} orc_report;

enum { M_NONE = 0, M_SINGLE = 1, M_FULL = 2 };
/* injected fault kinds */
enum { F_MEMORY = 0, F_COMPUTE = 1, F_ROW1D = 2, F_COL1D = 3, F_PANEL = 4 };
/* reported event kinds */
enum { E_0D = 0, E_ROW = 1, E_COL = 2, E_UNCORR = 3, E_CKSUM = 4, E_PD = 5 };

#define U64 (0x1p-53)

static double* dalloc(int64_t n) {
    double* p = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    return p;
}
static int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }

/* ------------------------------------------------ unblocked definitions */

/* Cholesky, lower, A = L L^T (the plain definition, column by column):
 * l_jj = sqrt(a_jj - sum_{p<j} l_jp^2), l_ij = (a_ij - sum_{p<j} l_ip l_jp) / l_jj.
 * Reads and writes the lower triangle only.  Returns 0 or the 1-based column
 * of the first non-positive (or NaN) radicand. */
int orc_potf2(int64_t n, double* A, int64_t lda) {
    for (int64_t j = 0; j < n; ++j) {
        double s = A[j * lda + j];
        for (int64_t p = 0; p < j; ++p) s -= A[j * lda + p] * A[j * lda + p];
        if (!(s > 0.0)) return (int)(j + 1);
        double ljj = sqrt(s);
        A[j * lda + j] = ljj;
        for (int64_t i = j + 1; i < n; ++i) {
            double t = A[i * lda + j];
            for (int64_t p = 0; p < j; ++p) t -= A[i * lda + p] * A[j * lda + p];
            A[i * lda + j] = t / ljj;
        }
    }
    return 0;
}

/* LU with partial pivoting on an m x n block (m >= n not required), the plain
 * right-looking definition: pivot = FIRST index of the largest |a| in the
 * column (strict > comparison, so ties keep the earlier row and NaN never
 * wins), whole-row interchange, multipliers by division, rank-1 update.
 * ipiv[j] = 0-based row swapped with row j.  Returns 0 or the 1-based column
 * of the first exactly-zero pivot (the factorization continues, as LAPACK). */
int orc_getf2(int64_t m, int64_t n, double* A, int64_t lda, int64_t* ipiv) {
    int info = 0;
    int64_t kmax = imin(m, n);
    for (int64_t j = 0; j < kmax; ++j) {
        int64_t p = j;
        double best = fabs(A[j * lda + j]);
        for (int64_t i = j + 1; i < m; ++i) {
            double v = fabs(A[i * lda + j]);
            if (v > best) { best = v; p = i; }
        }
        ipiv[j] = p;
        if (p != j)
            for (int64_t c = 0; c < n; ++c) {
                double t = A[j * lda + c]; A[j * lda + c] = A[p * lda + c]; A[p * lda + c] = t;
            }
        double piv = A[j * lda + j];
        if (piv == 0.0) { if (!info) info = (int)(j + 1); continue; }
        for (int64_t i = j + 1; i < m; ++i) A[i * lda + j] /= piv;
        for (int64_t i = j + 1; i < m; ++i) {
            double l = A[i * lda + j];
            for (int64_t c = j + 1; c < n; ++c) A[i * lda + c] -= l * A[j * lda + c];
        }
    }
    return info;
}

/* Householder reflector (LAPACK larfg convention) for x = [alpha; x1] of
 * length len stored with stride ld: beta = -sign(alpha) * ||x||_2 (sign(0) = +),
 * tau = (beta - alpha)/beta, v = [1; x1 / (alpha - beta)]; tau = 0 and H = I
 * when ||x1|| = 0.  On return x holds [beta; v(2:)]. */
static double larfg(int64_t len, double* x, int64_t ld) {
    double alpha = x[0], ss = 0.0;
    for (int64_t i = 1; i < len; ++i) ss += x[i * ld] * x[i * ld];
    if (ss == 0.0) return 0.0;
    double nrm = sqrt(alpha * alpha + ss);
    double beta = alpha >= 0.0 ? -nrm : nrm;
    double tau = (beta - alpha) / beta;
    double scal = alpha - beta;
    for (int64_t i = 1; i < len; ++i) x[i * ld] /= scal;
    x[0] = beta;
    return tau;
}

/* Householder QR, m x n block: for each column j, reflector on A[j:m, j],
 * then H_j^T applied to A[j:m, j+1:n] (w = v^T a, a -= tau v w).  R is left
 * in the upper triangle, v(2:) below the diagonal, tau[j] per column. */
int orc_geqr2(int64_t m, int64_t n, double* A, int64_t lda, double* tau) {
    int64_t kmax = imin(m, n);
    for (int64_t j = 0; j < kmax; ++j) {
        double* x = A + j * lda + j;
        double t = larfg(m - j, x, lda);
        tau[j] = t;
        if (t == 0.0) continue;
        for (int64_t c = j + 1; c < n; ++c) {
            double w = A[j * lda + c];
            for (int64_t i = j + 1; i < m; ++i) w += A[i * lda + j] * A[i * lda + c];
            A[j * lda + c] -= t * w;
            for (int64_t i = j + 1; i < m; ++i) A[i * lda + c] -= t * A[i * lda + j] * w;
        }
    }
    return 0;
}

/* ------------------------------------------------------ checksum verify */

typedef struct {
    int mode;
    int step;
    int64_t g;
    double tau;
    orc_report* rep;
    double tau_used;   /* largest per-component threshold applied (mixed form) */
} vctx;

static void add_event(vctx* c, int kind, int64_t row, int64_t col, double d) {
    orc_report* r = c->rep;
    if (r->nloc < 64) {
        orc_event* e = &r->loc[r->nloc++];
        e->step = c->step; e->kind = kind; e->row = row; e->col = col; e->delta = d;
    }
}

/* Verify one tile T (nr x nc at global origin (r0, c0), leading dim ldt)
 * against its carried checksums, then locate and correct (Sec. 3.1.2: full
 * checksums tolerate 0D and 1D errors, single-side checksums 0D only).
 *   cc[j]        carried column sums   1^T T      (both modes)
 *   cw[j]        carried weighted sums w^T T, w = (1..nr)  (single mode)
 *   cr[i*crs]    carried row sums      T 1        (full mode)
 * d^c = recomputed - carried; a component is flagged when |d| > tau.
 * Full mode: 1 row + 1 col -> 0D, T[i][j] -= d^c_j (and d^c_j must agree with
 * d^r_i within tau); 1 row + >=2 cols -> 1D row, T[i][j] -= d^c_j for every
 * flagged j; >=2 rows + 1 col -> 1D column, T[i][j] -= d^r_i; flags on one
 * side only -> the checksum itself is wrong, re-encode it from the data;
 * >=2 rows and >=2 cols -> 2D, uncorrectable.
 * Single mode: every flagged column j is located at row
 * i = round(d^w_j / d^c_j) - 1 (accepted when within 0.05 of an integer and
 * inside the tile) and corrected by d^c_j; otherwise uncorrectable. */
static void verify_tile_t(vctx* c, double* T, int64_t ldt, int64_t r0, int64_t c0,
                          int64_t nr, int64_t nc, double* cc, double* cw,
                          double* cr, int64_t crs, const double* tc, const double* tr) {
    if (c->mode == M_NONE || nr <= 0 || nc <= 0) return;
    double tau = c->tau;
#define TC(j) (tc ? tc[j] : tau)
#define TR(i) (tr ? tr[(i) * crs] : tau)
    double* dc = dalloc(nc);
    double* dw = dalloc(nc);
    double* dr = dalloc(nr);
    for (int64_t j = 0; j < nc; ++j) {
        double s = 0.0, sw = 0.0;
        for (int64_t i = 0; i < nr; ++i) {
            s += T[i * ldt + j];
            sw += (double)(i + 1) * T[i * ldt + j];
        }
        dc[j] = s - cc[j];
        if (c->mode == M_SINGLE) dw[j] = sw - cw[j];
    }
    if (c->mode == M_FULL)
        for (int64_t i = 0; i < nr; ++i) {
            double s = 0.0;
            for (int64_t j = 0; j < nc; ++j) s += T[i * ldt + j];
            dr[i] = s - cr[i * crs];
        }
    int64_t nfc = 0, nfr = 0, fc = -1, fr = -1;
    double dmax = 0.0, rmax = 0.0;   /* largest |d|; largest |d| / threshold */
    for (int64_t j = 0; j < nc; ++j) {
        double a = fabs(dc[j]);
        if (!(a <= TC(j))) { ++nfc; if (fc < 0) fc = j; }
        if (a > dmax) dmax = a;
        if (tc && tc[j] > 0.0 && a / tc[j] > rmax) rmax = a / tc[j];
        if (tc && tc[j] > c->tau_used) c->tau_used = tc[j];
    }
    if (c->mode == M_FULL)
        for (int64_t i = 0; i < nr; ++i) {
            double a = fabs(dr[i]);
            if (!(a <= TR(i))) { ++nfr; if (fr < 0) fr = i; }
            if (a > dmax) dmax = a;
            if (tr && tr[i * crs] > 0.0 && a / tr[i * crs] > rmax) rmax = a / tr[i * crs];
            if (tr && tr[i * crs] > c->tau_used) c->tau_used = tr[i * crs];
        }
    orc_report* rep = c->rep;
    if (nfc == 0 && nfr == 0) {
        double ratio = tc ? rmax : (tau > 0.0 ? dmax / tau : 0.0);
        if (ratio > rep->max_ratio) rep->max_ratio = ratio;
        free(dc); free(dw); free(dr);
        return;
    }
    rep->detected += 1;
    if (c->mode == M_SINGLE) {
        for (int64_t j = 0; j < nc; ++j) {
            if (fabs(dc[j]) <= TC(j)) continue;
            double rho = dw[j] / dc[j];
            double ri = nearbyint(rho);
            int64_t i = (int64_t)ri - 1;
            if (fabs(rho - ri) <= 0.05 && i >= 0 && i < nr) {
                T[i * ldt + j] -= dc[j];
                rep->corrected += 1;
                add_event(c, E_0D, r0 + i, c0 + j, dc[j]);
            } else {
                rep->uncorrectable += 1;
                add_event(c, E_UNCORR, r0, c0 + j, dc[j]);
            }
        }
    } else if (nfr == 1 && nfc == 1) {
        if (fabs(dc[fc] - dr[fr]) <= (tc ? TC(fc) + TR(fr) : tau)) {
            T[fr * ldt + fc] -= dc[fc];
            rep->corrected += 1;
            add_event(c, E_0D, r0 + fr, c0 + fc, dc[fc]);
        } else {
            rep->uncorrectable += 1;
            add_event(c, E_UNCORR, r0, c0, dc[fc]);
        }
    } else if (nfr == 1 && nfc >= 2) {
        for (int64_t j = 0; j < nc; ++j) {
            if (fabs(dc[j]) <= TC(j)) continue;
            T[fr * ldt + j] -= dc[j];
            rep->corrected += 1;
            add_event(c, E_ROW, r0 + fr, c0 + j, dc[j]);
        }
    } else if (nfr >= 2 && nfc == 1) {
        for (int64_t i = 0; i < nr; ++i) {
            if (fabs(dr[i]) <= TR(i)) continue;
            T[i * ldt + fc] -= dr[i];
            rep->corrected += 1;
            add_event(c, E_COL, r0 + i, c0 + fc, dr[i]);
        }
    } else if (nfr == 0 || nfc == 0) {
        for (int64_t j = 0; j < nc; ++j) {
            double s = 0.0;
            for (int64_t i = 0; i < nr; ++i) s += T[i * ldt + j];
            cc[j] = s;
        }
        for (int64_t i = 0; i < nr; ++i) {
            double s = 0.0;
            for (int64_t j = 0; j < nc; ++j) s += T[i * ldt + j];
            cr[i * crs] = s;
        }
        rep->checksum_repaired += 1;
        add_event(c, E_CKSUM, r0, c0, 0.0);
    } else {
        rep->uncorrectable += 1;
        add_event(c, E_UNCORR, r0, c0, 0.0);
    }
    free(dc); free(dw); free(dr);
#undef TC
#undef TR
}

static void verify_tile(vctx* c, double* T, int64_t ldt, int64_t r0, int64_t c0,
                        int64_t nr, int64_t nc, double* cc, double* cw,
                        double* cr, int64_t crs) {
    verify_tile_t(c, T, ldt, r0, c0, nr, nc, cc, cw, cr, crs, NULL, NULL);
}

/* Encode the checksums of one tile (Sec. 3.1.2: encode before the operation). */
static void encode_tile(const double* T, int64_t ldt, int64_t nr, int64_t nc,
                        double* cc, double* cw, double* cr, int64_t crs) {
    for (int64_t j = 0; j < nc; ++j) {
        double s = 0.0, sw = 0.0;
        for (int64_t i = 0; i < nr; ++i) {
            s += T[i * ldt + j];
            sw += (double)(i + 1) * T[i * ldt + j];
        }
        cc[j] = s; cw[j] = sw;
    }
    for (int64_t i = 0; i < nr; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < nc; ++j) s += T[i * ldt + j];
        cr[i * crs] = s;
    }
}

static int cmp_event(const void* a, const void* b) {
    const orc_event* x = (const orc_event*)a;
    const orc_event* y = (const orc_event*)b;
    if (x->step != y->step) return x->step < y->step ? -1 : 1;
    if (x->row != y->row) return x->row < y->row ? -1 : 1;
    if (x->col != y->col) return x->col < y->col ? -1 : 1;
    if (x->kind != y->kind) return x->kind < y->kind ? -1 : 1;
    return 0;
}

/* Add an injected fault to the working matrix W (n x n, ld n).  A 0D kind
 * touches one element; ROW1D runs along the row from col to the end of col's
 * g-tile; COL1D runs down the column from row to the end of row's g-tile. */
static void apply_fault(double* W, int64_t n, int64_t g, const orc_event* f) {
    if (f->kind == F_ROW1D) {
        int64_t end = imin((f->col / g + 1) * g, n);
        for (int64_t j = f->col; j < end; ++j) W[f->row * n + j] += f->delta;
    } else if (f->kind == F_COL1D) {
        int64_t end = imin((f->row / g + 1) * g, n);
        for (int64_t i = f->row; i < end; ++i) W[i * n + f->col] += f->delta;
    } else {
        W[f->row * n + f->col] += f->delta;
    }
}

/* tau = tau_scale * 8 * u * n * g * M, multiplied left to right. */
static double threshold(double tau_scale, int64_t n, int64_t g, double M) {
    double t = tau_scale * 8.0;
    t *= U64;
    t *= (double)n;
    t *= (double)g;
    t *= M;
    return t;
}

/* ------------------------------------------------ blocked ABFT Cholesky */

/* Validate a fault against the region the algorithm touches at its step.
 * Cholesky TMU region: row, col >= T0 and blk(col) <= blk(row) (the lower
 * block triangle; diagonal blocks are kept full).  PANEL: the panel below the
 * diagonal block.  Returns 1 if valid. */
static int chol_fault_ok(const orc_event* f, int64_t n, int64_t nb, int64_t N) {
    if (f->step < 0 || f->step >= N - 1) return 0;
    int64_t K0 = (int64_t)f->step * nb, T0 = imin(K0 + nb, n);
    if (f->row < 0 || f->row >= n || f->col < 0 || f->col >= n) return 0;
    if (f->kind == F_PANEL) return f->row >= T0 && f->col >= K0 && f->col < T0;
    if (f->kind < F_MEMORY || f->kind > F_PANEL) return 0;
    return f->row >= T0 && f->col >= T0 && f->col / nb <= f->row / nb;
}

/*
 * Blocked right-looking Cholesky with ABFT (Sec. 2.1 skeleton; Sec. 3.1.2
 * checksums).  Per iteration k (K0 = k b, T0 = K0 + kb):
 *   PD : L_kk = chol(A_kk).  PD check: 1^T A_kk (carried) vs (1^T L_kk) L_kk^T.
 *   PU : L_Ik = A_Ik L_kk^{-T} for the panel below.  The checksum rows are
 *        carried through the same solve: s_I = c_Ik L_kk^{-T} and the weighted
 *        row s^w_I = w_Ik L_kk^{-T} (both modes).  A triangular solve works row
 *        by row, so an error in its output is 0D or spreads along its row; both
 *        are located by the weighted column checksum, so every panel tile is
 *        verified with the single-side rule (no row sums: a row-sum check would
 *        need L_kk^{-T} 1, whose use cancels badly for ill-conditioned L_kk).
 *   TMU: A_IJ -= L_Ik L_Jk^T on the lower block triangle (diagonal blocks in
 *        full), with c_IJ -= s_I L_Jk^T and r_IJ -= L_Ik s_J^T.
 *        Verify / correct every trailing tile.
 * Faults listed for step k are added after the TMU (PANEL faults after the
 * PU).  tau = tau_scale * 8 u n g max_i a_ii.  Returns 0, the 1-based info of
 * a non-positive pivot, or -(argument index) for an invalid argument.
 * The strict upper triangle of A is left untouched.
 */
/*
 * orc_potrf_sched -- orc_potrf with a checksum mode per step (the adaptive
 * ABFT of Sec. 3.1.2, Alg. alg-abft: each iteration runs with no check, the
 * single-side check or the full check).  modes[k] is the mode of step k
 * (N = ceil(n / nb) entries).  A step with mode NONE neither carries nor
 * verifies checksums; when checking starts again, or moves from SINGLE to
 * FULL, the checksums of the trailing block triangle are encoded afresh from
 * the current data at the start of that step (so an error that struck during
 * unchecked steps is part of the new checksums and is not detected).
 */
int orc_potrf_sched(int64_t n, int64_t nb, const int* modes, double* A, int64_t lda,
                    const orc_event* faults, int32_t nfaults, double tau_scale,
                    orc_report* rep) {
    memset(rep, 0, sizeof(*rep));
    if (n < 0) return -1;
    if (nb <= 0) return -2;
    if (lda < (n > 1 ? n : 1)) return -5;
    if (n == 0) return 0;
    int64_t g = nb, nt = (n + g - 1) / g, N = nt;
    for (int64_t k = 0; k < N; ++k)
        if (modes[k] < M_NONE || modes[k] > M_FULL) return -3;
    for (int32_t f = 0; f < nfaults; ++f)
        if (!chol_fault_ok(&faults[f], n, nb, N)) return -6;

    double* W = dalloc(n * n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j <= i; ++j) W[i * n + j] = W[j * n + i] = A[i * lda + j];
    double dmax = 0.0;
    for (int64_t i = 0; i < n; ++i) if (A[i * lda + i] > dmax) dmax = A[i * lda + i];
    vctx c = { M_NONE, 0, g, threshold(tau_scale, n, g, dmax), rep };
    rep->tau = c.tau;

    double* Cc = dalloc(nt * n);  /* Cc[I*n + j]: column sums of tile-row I   */
    double* Cw = dalloc(nt * n);  /* weighted column sums (single mode)        */
    double* Cr = dalloc(n * nt);  /* Cr[i*nt + J]: row sums of tile-column J   */
    double* xr = dalloc(n);       /* carried row sums of the panel             */
    double* v = dalloc(g);
    int info = 0;
    for (int64_t k = 0; k < N; ++k) {
        const int mode = modes[k];
        const int prev = k > 0 ? modes[k - 1] : M_NONE;
        c.step = (int)k;
        c.mode = mode;
        int64_t K0 = k * g, kb = imin(g, n - K0), T0 = K0 + kb;
        double* Lkk = W + K0 * n + K0;
        /* (re-)encode the trailing block triangle when checking starts or
           moves from single-side to full checksums */
        if (mode != M_NONE && (prev == M_NONE || (mode == M_FULL && prev != M_FULL)))
            for (int64_t I = k; I < nt; ++I)
                for (int64_t J = k; J <= I; ++J) {
                    int64_t r0 = I * g, c0 = J * g;
                    encode_tile(W + r0 * n + c0, n, imin(g, n - r0), imin(g, n - c0),
                                Cc + I * n + c0, Cw + I * n + c0, Cr + r0 * nt + J, nt);
                }
        /* PD */
        int pinfo = orc_potf2(kb, Lkk, n);
        if (pinfo) { info = (int)(K0 + pinfo); break; }
        if (mode != M_NONE) { /* PD check on column sums */
            for (int64_t j = 0; j < kb; ++j) {
                double y = 0.0;
                for (int64_t p = 0; p <= j; ++p) {
                    double colsum = 0.0;
                    for (int64_t q = p; q < kb; ++q) colsum += Lkk[q * n + p];
                    y += colsum * Lkk[j * n + p];
                }
                double d = y - Cc[k * n + K0 + j];
                if (!(fabs(d) <= c.tau)) {
                    rep->detected += 1; rep->uncorrectable += 1;
                    add_event(&c, E_PD, K0 + j, K0 + j, d);
                }
            }
        }
        /* PU: checksum rows and panel rows through x L_kk^T = b */
        if (mode != M_NONE) {
            for (int64_t I = k + 1; I < nt; ++I)
                for (int w = 0; w < 2; ++w) {
                    double* s = (w ? Cw : Cc) + I * n + K0;
                    for (int64_t j = 0; j < kb; ++j) {
                        double t = s[j];
                        for (int64_t p = 0; p < j; ++p) t -= s[p] * Lkk[j * n + p];
                        s[j] = t / Lkk[j * n + j];
                    }
                }
        }
        for (int64_t i = T0; i < n; ++i) {
            double* a = W + i * n + K0;
            for (int64_t j = 0; j < kb; ++j) {
                double t = a[j];
                for (int64_t p = 0; p < j; ++p) t -= a[p] * Lkk[j * n + p];
                a[j] = t / Lkk[j * n + j];
            }
        }
        for (int32_t f = 0; f < nfaults; ++f)
            if (faults[f].step == k && faults[f].kind == F_PANEL) apply_fault(W, n, g, &faults[f]);
        {
            vctx cp = c;   /* panel tiles: single-side rule in both checksum modes */
            if (cp.mode == M_FULL) cp.mode = M_SINGLE;
            for (int64_t I = k + 1; I < nt; ++I) {
                int64_t r0 = I * g;
                verify_tile(&cp, W + r0 * n + K0, n, r0, K0, imin(g, n - r0), kb,
                            Cc + I * n + K0, Cw + I * n + K0, xr + r0, 1);
            }
        }
        /* TMU */
        for (int64_t i = T0; i < n; ++i)
            for (int64_t j = T0; j < n; ++j) {
                if (j / g > i / g) continue;
                double t = W[i * n + j];
                for (int64_t p = 0; p < kb; ++p) t -= W[i * n + K0 + p] * W[j * n + K0 + p];
                W[i * n + j] = t;
            }
        if (mode != M_NONE) {
            for (int64_t I = k + 1; I < nt; ++I)
                for (int w = 0; w < 2; ++w) {
                    double* C = (w ? Cw : Cc) + I * n;
                    for (int64_t j = T0; j < n; ++j) {
                        if (j / g > I) continue;
                        double t = C[j];
                        for (int64_t p = 0; p < kb; ++p) t -= C[K0 + p] * W[j * n + K0 + p];
                        C[j] = t;
                    }
                }
            if (mode == M_FULL)
                for (int64_t i = T0; i < n; ++i)
                    for (int64_t J = k + 1; J <= i / g; ++J) {
                        double t = Cr[i * nt + J];
                        for (int64_t p = 0; p < kb; ++p) t -= W[i * n + K0 + p] * Cc[J * n + K0 + p];
                        Cr[i * nt + J] = t;
                    }
        }
        for (int32_t f = 0; f < nfaults; ++f)
            if (faults[f].step == k && faults[f].kind != F_PANEL) apply_fault(W, n, g, &faults[f]);
        for (int64_t I = k + 1; I < nt; ++I)
            for (int64_t J = k + 1; J <= I; ++J) {
                int64_t r0 = I * g, c0 = J * g;
                verify_tile(&c, W + r0 * n + c0, n, r0, c0, imin(g, n - r0), imin(g, n - c0),
                            Cc + I * n + c0, Cw + I * n + c0, Cr + r0 * nt + J, nt);
            }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j <= i; ++j) A[i * lda + j] = W[i * n + j];
    rep->info = info;
    qsort(rep->loc, (size_t)rep->nloc, sizeof(orc_event), cmp_event);
    free(W); free(Cc); free(Cw); free(Cr); free(xr); free(v);
    return info;
}

/* orc_potrf: every step in the same checksum mode (the algorithm described
 * above orc_potrf_sched). */
int orc_potrf(int64_t n, int64_t nb, int mode, double* A, int64_t lda,
              const orc_event* faults, int32_t nfaults, double tau_scale,
              orc_report* rep) {
    memset(rep, 0, sizeof(*rep));
    if (n < 0) return -1;
    if (nb <= 0) return -2;
    if (mode < M_NONE || mode > M_FULL) return -3;
    int64_t N = n > 0 ? (n + nb - 1) / nb : 1;
    int* modes = (int*)malloc(sizeof(int) * (size_t)N);
    for (int64_t k = 0; k < N; ++k) modes[k] = mode;
    int r = orc_potrf_sched(n, nb, modes, A, lda, faults, nfaults, tau_scale, rep);
    free(modes);
    return r;
}

/* ------------------------------------ mixed-precision ABFT Cholesky (16-bit TMU) */
/*
 * The mixed form is not in the paper.  It keeps the blocked skeleton of
 * Sec. 2.1 and the checksum scheme of Sec. 3.1.2, and runs the trailing
 * matrix update on 16-bit operands whose products are accumulated in FP32
 * (what a tensor core computes).  Readings, written out in this section:
 *  - the 16-bit formats: BF16 (8 significand bits, exponents -126..127) and
 *    FP16 (11 significand bits, exponents -14..15), both with subnormals;
 *    rounding to nearest, ties to the even significand, overflow to infinity;
 *  - per g-row tile I of the panel L_Ik: sigma_I = 2^(ceil(log2 max|L_I|) - e_t),
 *    e_t = 0 (BF16, the tile maximum maps to at most 1) or 14 (FP16, at most
 *    2^14); sigma_I = 1 for an all-zero tile; Lq_I = RN16(L_I / sigma_I);
 *  - TMU: A_IJ -= sigma_I sigma_J (Lq_I Lq_J^T).  Here the products of the
 *    16-bit operands are summed in FP64 (exact products, p in order); the GPU
 *    accumulates them in FP32, which the thresholds below allow for;
 *  - the checksums are carried with the same quantized operands, so that the
 *    quantization cancels from the checksum relation: with t_I = 1^T Lq_I and
 *    tw_I = (1..g)^T Lq_I, c_IJ -= sigma_I sigma_J t_I Lq_J^T (and the weighted
 *    rows with tw_I), r_IJ -= sigma_I sigma_J Lq_I t_J^T;
 *  - abs-checksums bound what the FP32 accumulation can do to that relation:
 *    |c|_IJ += sigma_I sigma_J (1^T |Lq_I|) |Lq_J|^T and
 *    |r|_IJ += sigma_I sigma_J |Lq_I| (1^T |Lq_J|)^T, zero when the tile is
 *    encoded; the threshold of column j (row i) of tile IJ is
 *    tau_j = coef |c|_IJ,j + tau64, coef = tau_scale * 4 * gamma_g(2^-24),
 *    gamma_g(u) = g u / (1 - g u), and tau64 the FP64 threshold
 *    tau_scale * 8 * 2^-53 * n * g * max a_ii (the FP64 rounding of the
 *    FP64 parts: C, the checksums, the verification sums).  The factor 4
 *    covers both sides of the relation (data and checksum products) and a
 *    factor 2 for an accumulation that does not round to nearest;
 *  - PD in FP64; PU in FP32: L_kk and each right-hand side rounded to FP32,
 *    x_j = (b_j - sum_{p<j} x_p l_jp) / l_jj with the sum one fused
 *    multiply-add chain in p order starting from b_j, correctly rounded
 *    division; the checksum rows (plain and weighted) go through the same
 *    solve;
 *  - the PD check and the panel verification use the scalar threshold
 *    tau_scale * 8 * 2^-24 * n * g * max a_ii (the FP32 panel solve).
 */
#define U32 (0x1p-24)

/* x rounded to BF16 (is_bf16 != 0) or FP16, to nearest with ties to even;
 * *bits receives the 16-bit encoding (sign, biased exponent, fraction). */
double orc_round16(double x, int is_bf16, uint16_t* bits) {
    const int p = is_bf16 ? 8 : 11;          /* significand bits, hidden bit included */
    const int emin = is_bf16 ? -126 : -14;   /* smallest normal exponent */
    const int emax = is_bf16 ? 127 : 15;
    const int fbits = p - 1, bias = emax;
    const uint16_t sign = signbit(x) ? 0x8000u : 0u;
    const uint16_t expall = (uint16_t)(((1u << (is_bf16 ? 8 : 5)) - 1u) << fbits);
    if (isnan(x)) { *bits = (uint16_t)(sign | expall | (1u << (fbits - 1))); return x; }
    if (isinf(x)) { *bits = (uint16_t)(sign | expall); return x; }
    double a = fabs(x);
    if (a == 0.0) { *bits = sign; return x; }
    int E;
    frexp(a, &E);                             /* a = f 2^E, f in [0.5, 1): exponent E - 1 */
    int e = E - 1;
    int qe = (e < emin ? emin : e) - fbits;   /* spacing of the format around a: 2^qe */
    double r = nearbyint(ldexp(a, -qe));      /* default mode: nearest, ties to even */
    double v = ldexp(r, qe);
    double maxf = ldexp(ldexp(1.0, p) - 1.0, emax - fbits);
    if (v > maxf) { *bits = (uint16_t)(sign | expall); return sign ? -INFINITY : INFINITY; }
    uint16_t code;
    if (v < ldexp(1.0, emin)) {               /* subnormal: fraction = v / 2^(emin - fbits) */
        code = (uint16_t)ldexp(v, -(emin - fbits));
    } else {
        int E2;
        frexp(v, &E2);
        int e2 = E2 - 1;
        uint16_t frac = (uint16_t)(ldexp(v, fbits - e2) - ldexp(1.0, fbits));
        code = (uint16_t)(((unsigned)(e2 + bias) << fbits) | frac);
    }
    *bits = (uint16_t)(sign | code);
    return sign ? -v : v;
}

/* sigma = 2^(ceil(log2 m) - et) for the tile maximum m = max |x| > 0, else 1. */
double orc_tile_sigma(double m, int is_bf16) {
    const int et = is_bf16 ? 0 : 14;
    if (!(m > 0.0)) return 1.0;
    int E;
    double f = frexp(m, &E);                  /* m = f 2^E, f in [0.5, 1) */
    int c = (f == 0.5) ? E - 1 : E;           /* ceil(log2 m) */
    return ldexp(1.0, c - et);
}

/* Quantize one tile (rows x cols, leading dimension ldp): *sigma, the 16-bit
 * encodings (bits, rows x cols, may be NULL) and their values (q, rows x cols). */
void orc_quantize(int64_t rows, int64_t cols, const double* P, int64_t ldp, int is_bf16,
                  double* sigma, uint16_t* bits, double* q) {
    double m = 0.0;
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < cols; ++j)
            if (fabs(P[i * ldp + j]) > m) m = fabs(P[i * ldp + j]);
    double s = orc_tile_sigma(m, is_bf16);
    *sigma = s;
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < cols; ++j) {
            uint16_t b;
            q[i * cols + j] = orc_round16(P[i * ldp + j] / s, is_bf16, &b);
            if (bits) bits[i * cols + j] = b;
        }
}

/* The mixed trailing update on its own: the m x k panel P quantized per g-row
 * tile (sigma[I], bits m x k), then C -= sigma_I sigma_J (Lq_I Lq_J^T) on the
 * lower block triangle of the m x m matrix C (blocks g x g, J <= I); each
 * entry's products summed in FP64 in p order, then subtracted once. */
void orc_syrk_mixed(int64_t m, int64_t k, int64_t g, int is_bf16, const double* P, int64_t ldp,
                    double* C, int64_t ldc, uint16_t* bits, double* sigma) {
    int64_t nt = (m + g - 1) / g;
    double* q = dalloc(m * k);
    for (int64_t I = 0; I < nt; ++I) {
        int64_t r0 = I * g, rows = imin(g, m - r0);
        orc_quantize(rows, k, P + r0 * ldp, ldp, is_bf16, &sigma[I], bits ? bits + r0 * k : NULL,
                     q + r0 * k);
    }
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < m; ++j) {
            if (j / g > i / g) continue;
            double s = 0.0;
            for (int64_t p = 0; p < k; ++p) s += q[i * k + p] * q[j * k + p];
            C[i * ldc + j] = C[i * ldc + j] - (sigma[i / g] * sigma[j / g]) * s;
        }
    free(q);
}

/* One right-hand side of x L^T = b in FP32 (the mixed form's panel solve):
 * Lf holds L (kb x kb, lower) rounded to FP32; b is overwritten with x. */
static void solve_row_f32(double* b, const float* Lf, int64_t kb) {
    float x[512];
    for (int64_t j = 0; j < kb; ++j) {
        float v = (float)b[j];
        for (int64_t p = 0; p < j; ++p) v = fmaf(-x[p], Lf[j * kb + p], v);
        x[j] = v / Lf[j * kb + j];
    }
    for (int64_t j = 0; j < kb; ++j) b[j] = (double)x[j];
}

static double threshold_u(double tau_scale, double u, int64_t n, int64_t g, double M) {
    double t = tau_scale * 8.0;
    t *= u;
    t *= (double)n;
    t *= (double)g;
    t *= M;
    return t;
}

/* coef of the abs-checksum thresholds: tau_scale * 4 * gamma_g(2^-24). */
double orc_mixed_coef(double tau_scale, int64_t g) {
    double gam = ((double)g * U32) / (1.0 - (double)g * U32);
    double t = tau_scale * 4.0;
    t *= gam;
    return t;
}

/*
 * orc_potrf_mixed -- the blocked ABFT Cholesky in the mixed form described
 * above, with a checksum mode per step (modes[k], N = ceil(n / nb) entries,
 * the same schedule semantics as orc_potrf_sched).  is_bf16 selects BF16 or
 * FP16 operands.  rep->tau is the largest threshold applied to a trailing
 * tile (an error larger than it plus the clean |d| is always flagged);
 * rep->max_ratio the largest |d| / threshold over tiles without flags.
 */
int orc_potrf_mixed(int64_t n, int64_t nb, const int* modes, int is_bf16, double* A, int64_t lda,
                    const orc_event* faults, int32_t nfaults, double tau_scale,
                    orc_report* rep) {
    memset(rep, 0, sizeof(*rep));
    if (n < 0) return -1;
    if (nb <= 0 || nb > 512) return -2;
    if (lda < (n > 1 ? n : 1)) return -5;
    if (n == 0) return 0;
    int64_t g = nb, nt = (n + g - 1) / g, N = nt;
    for (int64_t k = 0; k < N; ++k)
        if (modes[k] < M_NONE || modes[k] > M_FULL) return -3;
    for (int32_t f = 0; f < nfaults; ++f)
        if (!chol_fault_ok(&faults[f], n, nb, N)) return -6;

    double* W = dalloc(n * n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j <= i; ++j) W[i * n + j] = W[j * n + i] = A[i * lda + j];
    double dmax = 0.0;
    for (int64_t i = 0; i < n; ++i) if (A[i * lda + i] > dmax) dmax = A[i * lda + i];
    const double tau64 = threshold_u(tau_scale, U64, n, g, dmax);
    const double coef = orc_mixed_coef(tau_scale, g);
    vctx c = { M_NONE, 0, g, threshold_u(tau_scale, U32, n, g, dmax), rep, 0.0 };

    double* Cc = dalloc(nt * n);   /* column sums of tile-row I: Cc[I*n + j]      */
    double* Cw = dalloc(nt * n);   /* weighted column sums                          */
    double* Cr = dalloc(n * nt);   /* row sums of tile-column J: Cr[i*nt + J]      */
    double* Ca = dalloc(nt * n);   /* abs-checksums of the column sums             */
    double* Ra = dalloc(n * nt);   /* abs-checksums of the row sums                */
    double* Tc = dalloc(g);        /* thresholds of one tile's columns             */
    double* Tr = dalloc(n * nt);   /* thresholds of the row sums (laid out as Cr)  */
    double* xr = dalloc(n);
    double* q = dalloc(n * g);     /* quantized panel values, row i at q[i*g]      */
    double* sig = dalloc(nt);
    double* t = dalloc(nt * g);    /* t_I = 1^T Lq_I                               */
    double* tw = dalloc(nt * g);   /* tw_I = (1..g)^T Lq_I                         */
    double* ta = dalloc(nt * g);   /* 1^T |Lq_I|                                   */
    float* Lf = (float*)calloc((size_t)(g * g), sizeof(float));
    int info = 0;
    for (int64_t k = 0; k < N; ++k) {
        const int mode = modes[k];
        const int prev = k > 0 ? modes[k - 1] : M_NONE;
        c.step = (int)k;
        c.mode = mode;
        int64_t K0 = k * g, kb = imin(g, n - K0), T0 = K0 + kb;
        double* Lkk = W + K0 * n + K0;
        if (mode != M_NONE && (prev == M_NONE || (mode == M_FULL && prev != M_FULL)))
            for (int64_t I = k; I < nt; ++I)
                for (int64_t J = k; J <= I; ++J) {
                    int64_t r0 = I * g, c0 = J * g, nr = imin(g, n - r0), ncl = imin(g, n - c0);
                    encode_tile(W + r0 * n + c0, n, nr, ncl, Cc + I * n + c0, Cw + I * n + c0,
                                Cr + r0 * nt + J, nt);
                    for (int64_t j = 0; j < ncl; ++j) Ca[I * n + c0 + j] = 0.0;
                    for (int64_t i = 0; i < nr; ++i) Ra[(r0 + i) * nt + J] = 0.0;
                }
        /* PD (FP64) and its check */
        int pinfo = orc_potf2(kb, Lkk, n);
        if (pinfo) { info = (int)(K0 + pinfo); break; }
        if (mode != M_NONE) {
            for (int64_t j = 0; j < kb; ++j) {
                double y = 0.0;
                for (int64_t p = 0; p <= j; ++p) {
                    double colsum = 0.0;
                    for (int64_t r = p; r < kb; ++r) colsum += Lkk[r * n + p];
                    y += colsum * Lkk[j * n + p];
                }
                double d = y - Cc[k * n + K0 + j];
                if (!(fabs(d) <= c.tau)) {
                    rep->detected += 1; rep->uncorrectable += 1;
                    add_event(&c, E_PD, K0 + j, K0 + j, d);
                }
            }
        }
        if (T0 >= n) break;
        /* PU in FP32: checksum rows and panel rows through x L_kk^T = b */
        for (int64_t i = 0; i < kb; ++i)
            for (int64_t j = 0; j < kb; ++j) Lf[i * kb + j] = j <= i ? (float)Lkk[i * n + j] : 0.0f;
        if (mode != M_NONE)
            for (int64_t I = k + 1; I < nt; ++I) {
                solve_row_f32(Cc + I * n + K0, Lf, kb);
                solve_row_f32(Cw + I * n + K0, Lf, kb);
            }
        for (int64_t i = T0; i < n; ++i) solve_row_f32(W + i * n + K0, Lf, kb);
        for (int32_t f = 0; f < nfaults; ++f)
            if (faults[f].step == k && faults[f].kind == F_PANEL) apply_fault(W, n, g, &faults[f]);
        {
            vctx cp = c;   /* panel tiles: single-side rule, scalar FP32 threshold */
            if (cp.mode == M_FULL) cp.mode = M_SINGLE;
            for (int64_t I = k + 1; I < nt; ++I) {
                int64_t r0 = I * g;
                verify_tile(&cp, W + r0 * n + K0, n, r0, K0, imin(g, n - r0), kb,
                            Cc + I * n + K0, Cw + I * n + K0, xr + r0, 1);
            }
        }
        /* quantize the panel per tile-row, with the sums the checksums use */
        for (int64_t I = k + 1; I < nt; ++I) {
            int64_t r0 = I * g, rows = imin(g, n - r0);
            orc_quantize(rows, kb, W + r0 * n + K0, n, is_bf16, &sig[I], NULL, q + r0 * g);
            for (int64_t p = 0; p < kb; ++p) {
                double s = 0.0, sw = 0.0, sa = 0.0;
                for (int64_t r = 0; r < rows; ++r) {
                    double v = q[(r0 + r) * g + p];
                    s += v;
                    sw += (double)(r + 1) * v;
                    sa += fabs(v);
                }
                t[I * g + p] = s; tw[I * g + p] = sw; ta[I * g + p] = sa;
            }
        }
        /* TMU on the quantized operands (products summed in FP64) */
        for (int64_t i = T0; i < n; ++i)
            for (int64_t j = T0; j < n; ++j) {
                if (j / g > i / g) break;   /* lower block triangle, diagonal blocks full */
                double s = 0.0;
                for (int64_t p = 0; p < kb; ++p) s += q[i * g + p] * q[j * g + p];
                W[i * n + j] = W[i * n + j] - (sig[i / g] * sig[j / g]) * s;
            }
        /* checksum carries with the same operands, abs-checksums beside them */
        if (mode != M_NONE) {
            for (int64_t I = k + 1; I < nt; ++I)
                for (int64_t j = T0; j < n; ++j) {
                    if (j / g > I) break;
                    double sc = sig[I] * sig[j / g], s = 0.0, sw = 0.0, sa = 0.0;
                    for (int64_t p = 0; p < kb; ++p) {
                        s += t[I * g + p] * q[j * g + p];
                        sw += tw[I * g + p] * q[j * g + p];
                        sa += ta[I * g + p] * fabs(q[j * g + p]);
                    }
                    Cc[I * n + j] = Cc[I * n + j] - sc * s;
                    Cw[I * n + j] = Cw[I * n + j] - sc * sw;
                    Ca[I * n + j] = Ca[I * n + j] + sc * sa;
                }
            if (mode == M_FULL)
                for (int64_t i = T0; i < n; ++i)
                    for (int64_t J = k + 1; J <= i / g; ++J) {
                        double sc = sig[i / g] * sig[J], s = 0.0, sa = 0.0;
                        for (int64_t p = 0; p < kb; ++p) {
                            s += q[i * g + p] * t[J * g + p];
                            sa += fabs(q[i * g + p]) * ta[J * g + p];
                        }
                        Cr[i * nt + J] = Cr[i * nt + J] - sc * s;
                        Ra[i * nt + J] = Ra[i * nt + J] + sc * sa;
                    }
        }
        for (int32_t f = 0; f < nfaults; ++f)
            if (faults[f].step == k && faults[f].kind != F_PANEL) apply_fault(W, n, g, &faults[f]);
        /* verify every trailing tile against per-column / per-row thresholds */
        if (mode != M_NONE)
            for (int64_t I = k + 1; I < nt; ++I)
                for (int64_t J = k + 1; J <= I; ++J) {
                    int64_t r0 = I * g, c0 = J * g, nr = imin(g, n - r0), ncl = imin(g, n - c0);
                    for (int64_t j = 0; j < ncl; ++j) Tc[j] = coef * Ca[I * n + c0 + j] + tau64;
                    for (int64_t i = 0; i < nr; ++i)
                        Tr[(r0 + i) * nt + J] = coef * Ra[(r0 + i) * nt + J] + tau64;
                    verify_tile_t(&c, W + r0 * n + c0, n, r0, c0, nr, ncl, Cc + I * n + c0,
                                  Cw + I * n + c0, Cr + r0 * nt + J, nt, Tc, Tr + r0 * nt + J);
                }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j <= i; ++j) A[i * lda + j] = W[i * n + j];
    rep->info = info;
    rep->tau = c.tau_used;
    qsort(rep->loc, (size_t)rep->nloc, sizeof(orc_event), cmp_event);
    free(W); free(Cc); free(Cw); free(Cr); free(Ca); free(Ra); free(Tc); free(Tr); free(xr);
    free(q); free(sig); free(t); free(tw); free(ta); free(Lf);
    return info;
}

/* ------------------------------------------------------ blocked ABFT LU */

static int lu_fault_ok(const orc_event* f, int64_t n, int64_t nb, int64_t N) {
    if (f->step < 0 || f->step >= N - 1) return 0;
    int64_t K0 = (int64_t)f->step * nb, T0 = imin(K0 + nb, n);
    if (f->row < 0 || f->row >= n || f->col < 0 || f->col >= n) return 0;
    if (f->kind == F_PANEL) return f->row >= K0 && f->row < T0 && f->col >= T0;
    if (f->kind < F_MEMORY || f->kind > F_PANEL) return 0;
    return f->row >= T0 && f->col >= T0;
}

/*
 * Blocked right-looking LU with partial pivoting and ABFT (Sec. 2.1:
 * PD  L.1 x U11 <- A.1,  PU  U12 <- L11^{-1} A12,  TMU  A22 <- A22 - L21 U12).
 * Per iteration k:
 *   PD : getf2 on the panel A[K0:n, K0:T0] (first-max pivot), each interchange
 *        applied to the whole row.  Row checksums move with their rows; each
 *        interchange i <-> p adds the row difference to the column checksums
 *        of the two tile-rows (trailing columns only).
 *        PD check: the total column sums of the panel are invariant under
 *        row interchanges: sum_{I>=k} c_Ik (carried) vs (1^T L_panel) U_kk.
 *   PU : U_kJ = L_kk^{-1} A_kJ (unit lower).  Row checksums carried through
 *        the same solve: t_J = L_kk^{-1} r_kJ.  Column checksums of U taken
 *        from the row block before the solve: z^T A_kJ with L_kk^T z = 1
 *        (and L_kk^T z_w = w in single mode).  Verify / correct the U tiles.
 *   TMU: A_IJ -= L_Ik U_kJ; c_IJ -= (1^T L_Ik) U_kJ; r_IJ -= L_Ik t_J.
 *        Verify / correct every trailing tile.
 * tau_k = tau_scale * 8 u n g max(max|A|, max|U so far|).
 * ipiv is 0-based, length n.
 */
int orc_getrf(int64_t n, int64_t nb, int mode, double* A, int64_t lda, int64_t* ipiv,
              const orc_event* faults, int32_t nfaults, double tau_scale, orc_report* rep) {
    memset(rep, 0, sizeof(*rep));
    if (n < 0) return -1;
    if (nb <= 0) return -2;
    if (mode < M_NONE || mode > M_FULL) return -3;
    if (lda < (n > 1 ? n : 1)) return -5;
    if (n == 0) return 0;
    int64_t g = nb, nt = (n + g - 1) / g, N = nt;
    for (int32_t f = 0; f < nfaults; ++f)
        if (!lu_fault_ok(&faults[f], n, nb, N)) return -7;
    double* W = dalloc(n * n);
    double amax = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            W[i * n + j] = A[i * lda + j];
            if (fabs(W[i * n + j]) > amax) amax = fabs(W[i * n + j]);
        }
    double umax = 0.0;
    vctx c = { mode, 0, g, 0.0, rep };
    double* Cc = dalloc(nt * n);
    double* Cw = dalloc(nt * n);
    double* Cr = dalloc(n * nt);
    double* s = dalloc(g);
    double* sw = dalloc(g);
    double* z = dalloc(g);
    double* zw = dalloc(g);
    double* tt = dalloc(g * nt);   /* t_J, column J of the carried U row sums */
    double* colchk = dalloc(n);    /* column sums of U from the pre-PU row block */
    double* colchkw = dalloc(n);
    if (mode != M_NONE)
        for (int64_t I = 0; I < nt; ++I)
            for (int64_t J = 0; J < nt; ++J) {
                int64_t r0 = I * g, c0 = J * g;
                encode_tile(W + r0 * n + c0, n, imin(g, n - r0), imin(g, n - c0),
                            Cc + I * n + c0, Cw + I * n + c0, Cr + r0 * nt + J, nt);
            }
    int info = 0;
    for (int64_t k = 0; k < N; ++k) {
        c.step = (int)k;
        int64_t K0 = k * g, kb = imin(g, n - K0), T0 = K0 + kb;
        /* panel column totals before the PD (invariant under interchanges) */
        for (int64_t j = 0; j < kb; ++j) {
            double t = 0.0;
            for (int64_t I = k; I < nt; ++I) t += Cc[I * n + K0 + j];
            s[j] = t;
        }
        /* PD: getf2 on the panel with whole-row interchanges */
        for (int64_t j = 0; j < kb; ++j) {
            int64_t col = K0 + j, p = col;
            double best = fabs(W[col * n + col]);
            for (int64_t i = col + 1; i < n; ++i) {
                double a = fabs(W[i * n + col]);
                if (a > best) { best = a; p = i; }
            }
            ipiv[col] = p;
            if (p != col) {
                if (mode != M_NONE) {
                    int64_t Ii = col / g, Ip = p / g;
                    double wi = (double)(col - Ii * g + 1), wp = (double)(p - Ip * g + 1);
                    for (int64_t cc2 = T0; cc2 < n; ++cc2) {
                        double a = W[col * n + cc2], b = W[p * n + cc2];
                        Cc[Ii * n + cc2] += b - a; Cc[Ip * n + cc2] += a - b;
                        Cw[Ii * n + cc2] += wi * (b - a); Cw[Ip * n + cc2] += wp * (a - b);
                    }
                    for (int64_t J = 0; J < nt; ++J) {
                        double t = Cr[col * nt + J]; Cr[col * nt + J] = Cr[p * nt + J]; Cr[p * nt + J] = t;
                    }
                }
                for (int64_t cc2 = 0; cc2 < n; ++cc2) {
                    double t = W[col * n + cc2]; W[col * n + cc2] = W[p * n + cc2]; W[p * n + cc2] = t;
                }
            }
            double piv = W[col * n + col];
            if (piv == 0.0) { if (!info) info = (int)(col + 1); continue; }
            for (int64_t i = col + 1; i < n; ++i) W[i * n + col] /= piv;
            for (int64_t i = col + 1; i < n; ++i) {
                double l = W[i * n + col];
                for (int64_t c2 = col + 1; c2 < T0; ++c2) W[i * n + c2] -= l * W[col * n + c2];
            }
        }
        double* Lkk = W + K0 * n + K0;
        for (int64_t i = 0; i < kb; ++i)
            for (int64_t j = i; j < kb; ++j)
                if (fabs(Lkk[i * n + j]) > umax) umax = fabs(Lkk[i * n + j]);
        c.tau = threshold(tau_scale, n, g, amax > umax ? amax : umax);
        rep->tau = c.tau;
        if (mode != M_NONE) { /* PD check */
            for (int64_t j = 0; j < kb; ++j) {
                double y = 0.0;
                for (int64_t q = 0; q <= j; ++q) {
                    double lsum = 1.0; /* unit diagonal */
                    for (int64_t i = K0 + q + 1; i < n; ++i) lsum += W[i * n + K0 + q];
                    y += lsum * Lkk[q * n + j];
                }
                double d = y - s[j];
                if (!(fabs(d) <= c.tau)) {
                    rep->detected += 1; rep->uncorrectable += 1;
                    add_event(&c, E_PD, K0 + j, K0 + j, d);
                }
            }
        }
        if (T0 < n) {
            /* PU: checksums first (from the row block before the solve) */
            if (mode != M_NONE) {
                for (int64_t i = kb - 1; i >= 0; --i) { /* L_kk^T z = 1, L_kk^T z_w = w */
                    double t = 1.0, tw = (double)(i + 1);
                    for (int64_t p = i + 1; p < kb; ++p) {
                        t -= Lkk[p * n + i] * z[p];
                        tw -= Lkk[p * n + i] * zw[p];
                    }
                    z[i] = t; zw[i] = tw;
                }
                for (int64_t c2 = T0; c2 < n; ++c2) {
                    double t = 0.0, tw = 0.0;
                    for (int64_t i = 0; i < kb; ++i) {
                        t += z[i] * W[(K0 + i) * n + c2];
                        tw += zw[i] * W[(K0 + i) * n + c2];
                    }
                    colchk[c2] = t; colchkw[c2] = tw;
                }
                for (int64_t J = k + 1; J < nt; ++J) /* t_J = L_kk^{-1} r_kJ */
                    for (int64_t i = 0; i < kb; ++i) {
                        double t = Cr[(K0 + i) * nt + J];
                        for (int64_t p = 0; p < i; ++p) t -= Lkk[i * n + p] * tt[p * nt + J];
                        tt[i * nt + J] = t;
                    }
            }
            for (int64_t c2 = T0; c2 < n; ++c2)
                for (int64_t i = 0; i < kb; ++i) {
                    double t = W[(K0 + i) * n + c2];
                    for (int64_t p = 0; p < i; ++p) t -= Lkk[i * n + p] * W[(K0 + p) * n + c2];
                    W[(K0 + i) * n + c2] = t;
                }
            for (int32_t f = 0; f < nfaults; ++f)
                if (faults[f].step == k && faults[f].kind == F_PANEL) apply_fault(W, n, g, &faults[f]);
            for (int64_t J = k + 1; J < nt; ++J) {
                int64_t c0 = J * g;
                verify_tile(&c, W + K0 * n + c0, n, K0, c0, kb, imin(g, n - c0),
                            colchk + c0, colchkw + c0, tt + J, nt);
            }
            for (int64_t i = 0; i < kb; ++i)
                for (int64_t c2 = T0; c2 < n; ++c2)
                    if (fabs(W[(K0 + i) * n + c2]) > umax) umax = fabs(W[(K0 + i) * n + c2]);
            /* TMU */
            for (int64_t i = T0; i < n; ++i)
                for (int64_t c2 = T0; c2 < n; ++c2) {
                    double t = W[i * n + c2];
                    for (int64_t q = 0; q < kb; ++q) t -= W[i * n + K0 + q] * W[(K0 + q) * n + c2];
                    W[i * n + c2] = t;
                }
            if (mode != M_NONE) {
                for (int64_t I = k + 1; I < nt; ++I) {
                    int64_t r0 = I * g, r1 = imin(r0 + g, n);
                    for (int64_t q = 0; q < kb; ++q) {
                        double t = 0.0, tw = 0.0;
                        for (int64_t i = r0; i < r1; ++i) {
                            t += W[i * n + K0 + q];
                            tw += (double)(i - r0 + 1) * W[i * n + K0 + q];
                        }
                        s[q] = t; sw[q] = tw;
                    }
                    for (int64_t c2 = T0; c2 < n; ++c2) {
                        double t = Cc[I * n + c2], tw = Cw[I * n + c2];
                        for (int64_t q = 0; q < kb; ++q) {
                            t -= s[q] * W[(K0 + q) * n + c2];
                            tw -= sw[q] * W[(K0 + q) * n + c2];
                        }
                        Cc[I * n + c2] = t; Cw[I * n + c2] = tw;
                    }
                }
                if (mode == M_FULL)
                    for (int64_t i = T0; i < n; ++i)
                        for (int64_t J = k + 1; J < nt; ++J) {
                            double t = Cr[i * nt + J];
                            for (int64_t q = 0; q < kb; ++q) t -= W[i * n + K0 + q] * tt[q * nt + J];
                            Cr[i * nt + J] = t;
                        }
            }
            for (int32_t f = 0; f < nfaults; ++f)
                if (faults[f].step == k && faults[f].kind != F_PANEL) apply_fault(W, n, g, &faults[f]);
            for (int64_t I = k + 1; I < nt; ++I)
                for (int64_t J = k + 1; J < nt; ++J) {
                    int64_t r0 = I * g, c0 = J * g;
                    verify_tile(&c, W + r0 * n + c0, n, r0, c0, imin(g, n - r0), imin(g, n - c0),
                                Cc + I * n + c0, Cw + I * n + c0, Cr + r0 * nt + J, nt);
                }
        }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) A[i * lda + j] = W[i * n + j];
    rep->info = info;
    qsort(rep->loc, (size_t)rep->nloc, sizeof(orc_event), cmp_event);
    free(W); free(Cc); free(Cw); free(Cr); free(s); free(sw); free(z); free(zw);
    free(tt); free(colchk); free(colchkw);
    return info;
}

/* ------------------------------------------------------ blocked ABFT QR */

static int qr_fault_ok(const orc_event* f, int64_t n, int64_t nb, int64_t N) {
    if (f->step < 0 || f->step >= N - 1) return 0;
    int64_t K0 = (int64_t)f->step * nb, T0 = imin(K0 + nb, n);
    if (f->row < 0 || f->row >= n || f->col < 0 || f->col >= n) return 0;
    if (f->kind < F_MEMORY || f->kind > F_COL1D) return 0;
    return f->row >= K0 && f->col >= T0;
}

/*
 * Blocked Householder QR with ABFT.  Per iteration k:
 *   PD : geqr2 on the panel A[K0:n, K0:T0] (larfg convention), then the
 *        triangular factor T of the block reflector H = I - V T V^T
 *        (forward, columnwise: T_jj = tau_j, T[0:j, j] = -tau_j T[0:j,0:j] V[:,0:j]^T v_j).
 *        PD check: column 2-norms are preserved by the reflectors:
 *        ||R_kk[0:j+1, j]|| vs ||A_panel[:, j]|| taken before the PD.
 *   TMU: C = A[K0:n, T0:n];  W = V^T C;  W = T^T W;  C -= V W.
 *        Row checksums ride along as extra columns: r -= V T^T V^T r.
 *        Column checksums: c_I -= (1^T V_I) W (weighted: (w^T V_I) W).
 *        Verify / correct every updated tile (tile-rows >= k).
 * tau = tau_scale * 8 u n g max_j ||a_j||_2.
 */
int orc_geqrf(int64_t n, int64_t nb, int mode, double* A, int64_t lda, double* tau,
              const orc_event* faults, int32_t nfaults, double tau_scale, orc_report* rep) {
    memset(rep, 0, sizeof(*rep));
    if (n < 0) return -1;
    if (nb <= 0) return -2;
    if (mode < M_NONE || mode > M_FULL) return -3;
    if (lda < (n > 1 ? n : 1)) return -5;
    if (n == 0) return 0;
    int64_t g = nb, nt = (n + g - 1) / g, N = nt;
    for (int32_t f = 0; f < nfaults; ++f)
        if (!qr_fault_ok(&faults[f], n, nb, N)) return -7;
    double* W = dalloc(n * n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) W[i * n + j] = A[i * lda + j];
    double cmax = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += W[i * n + j] * W[i * n + j];
        if (sqrt(s) > cmax) cmax = sqrt(s);
    }
    vctx c = { mode, 0, g, threshold(tau_scale, n, g, cmax), rep };
    rep->tau = c.tau;
    double* Cc = dalloc(nt * n);
    double* Cw = dalloc(nt * n);
    double* Cr = dalloc(n * nt);
    double* T = dalloc(g * g);
    double* Wm = dalloc(g * (n + nt));  /* g x (n + nt): W for data + checksum columns */
    double* nrm = dalloc(g);
    double* s = dalloc(g);
    double* sw = dalloc(g);
    double* y = dalloc(g);
    if (mode != M_NONE)
        for (int64_t I = 0; I < nt; ++I)
            for (int64_t J = 0; J < nt; ++J) {
                int64_t r0 = I * g, c0 = J * g;
                encode_tile(W + r0 * n + c0, n, imin(g, n - r0), imin(g, n - c0),
                            Cc + I * n + c0, Cw + I * n + c0, Cr + r0 * nt + J, nt);
            }
    for (int64_t k = 0; k < N; ++k) {
        c.step = (int)k;
        int64_t K0 = k * g, kb = imin(g, n - K0), T0 = K0 + kb, m = n - K0;
        for (int64_t j = 0; j < kb; ++j) {
            double t = 0.0;
            for (int64_t i = K0; i < n; ++i) t += W[i * n + K0 + j] * W[i * n + K0 + j];
            nrm[j] = sqrt(t);
        }
        /* PD: geqr2 on the panel */
        double* P = W + K0 * n + K0;
        for (int64_t j = 0; j < kb; ++j) {
            double t = larfg(m - j, P + j * n + j, n);
            tau[K0 + j] = t;
            if (t == 0.0) continue;
            for (int64_t c2 = j + 1; c2 < kb; ++c2) {
                double w = P[j * n + c2];
                for (int64_t i = j + 1; i < m; ++i) w += P[i * n + j] * P[i * n + c2];
                P[j * n + c2] -= t * w;
                for (int64_t i = j + 1; i < m; ++i) P[i * n + c2] -= t * P[i * n + j] * w;
            }
        }
        if (mode != M_NONE)
            for (int64_t j = 0; j < kb; ++j) {
                double t = 0.0;
                for (int64_t i = 0; i <= j; ++i) t += P[i * n + j] * P[i * n + j];
                double d = sqrt(t) - nrm[j];
                if (!(fabs(d) <= c.tau)) {
                    rep->detected += 1; rep->uncorrectable += 1;
                    add_event(&c, E_PD, K0 + j, K0 + j, d);
                }
            }
        if (T0 >= n) break;
        /* larft: V is unit lower trapezoidal, v_j(i) = 1 at i = j, 0 above */
#define VV(i, j) ((i) == (j) ? 1.0 : ((i) < (j) ? 0.0 : P[(i) * n + (j)]))
        for (int64_t j = 0; j < kb; ++j) {
            double tj = tau[K0 + j];
            for (int64_t i = 0; i < j; ++i) {
                double t = 0.0;
                for (int64_t r = 0; r < m; ++r) t += VV(r, i) * VV(r, j);
                y[i] = t;
            }
            for (int64_t i = 0; i < j; ++i) {
                double t = 0.0;
                for (int64_t q = i; q < j; ++q) t += T[i * g + q] * y[q];
                T[i * g + j] = -tj * t;
            }
            T[j * g + j] = tj;
            for (int64_t i = j + 1; i < kb; ++i) T[i * g + j] = 0.0;
        }
        /* TMU (larfb) on data columns T0..n and, in full mode, on the
         * row-checksum columns J > k, which are extra columns of C. */
        int64_t ncs = (mode == M_FULL) ? nt - (k + 1) : 0;
        int64_t ncol = (n - T0) + ncs;
#define CC(i, c2) ((c2) < n - T0 ? &W[(K0 + (i)) * n + T0 + (c2)] : &Cr[(K0 + (i)) * nt + (k + 1) + ((c2) - (n - T0))])
        for (int64_t c2 = 0; c2 < ncol; ++c2) {
            for (int64_t j = 0; j < kb; ++j) { /* W = V^T C */
                double t = 0.0;
                for (int64_t r = 0; r < m; ++r) t += VV(r, j) * *CC(r, c2);
                y[j] = t;
            }
            for (int64_t j = 0; j < kb; ++j) { /* W = T^T W */
                double t = 0.0;
                for (int64_t q = 0; q <= j; ++q) t += T[q * g + j] * y[q];
                Wm[j * (n + nt) + c2] = t;
            }
            for (int64_t r = 0; r < m; ++r) { /* C -= V W */
                double t = *CC(r, c2);
                for (int64_t j = 0; j < kb; ++j) t -= VV(r, j) * Wm[j * (n + nt) + c2];
                *CC(r, c2) = t;
            }
        }
        if (mode != M_NONE)
            for (int64_t I = k; I < nt; ++I) {
                int64_t r0 = I * g, r1 = imin(r0 + g, n);
                for (int64_t j = 0; j < kb; ++j) {
                    double t = 0.0, tw = 0.0;
                    for (int64_t i = r0; i < r1; ++i) {
                        t += VV(i - K0, j);
                        tw += (double)(i - r0 + 1) * VV(i - K0, j);
                    }
                    s[j] = t; sw[j] = tw;
                }
                for (int64_t c2 = T0; c2 < n; ++c2) {
                    double t = Cc[I * n + c2], tw = Cw[I * n + c2];
                    for (int64_t j = 0; j < kb; ++j) {
                        t -= s[j] * Wm[j * (n + nt) + (c2 - T0)];
                        tw -= sw[j] * Wm[j * (n + nt) + (c2 - T0)];
                    }
                    Cc[I * n + c2] = t; Cw[I * n + c2] = tw;
                }
            }
#undef CC
#undef VV
        for (int32_t f = 0; f < nfaults; ++f)
            if (faults[f].step == k) apply_fault(W, n, g, &faults[f]);
        for (int64_t I = k; I < nt; ++I)
            for (int64_t J = k + 1; J < nt; ++J) {
                int64_t r0 = I * g, c0 = J * g;
                verify_tile(&c, W + r0 * n + c0, n, r0, c0, imin(g, n - r0), imin(g, n - c0),
                            Cc + I * n + c0, Cw + I * n + c0, Cr + r0 * nt + J, nt);
            }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) A[i * lda + j] = W[i * n + j];
    qsort(rep->loc, (size_t)rep->nloc, sizeof(orc_event), cmp_event);
    free(W); free(Cc); free(Cw); free(Cr); free(T); free(Wm); free(nrm);
    free(s); free(sw); free(y);
    return 0;
}

/* ------------------------------------------------------------- solves */

/* X = L^{-T} L^{-1} B for a lower Cholesky factor L (forward then backward
 * substitution, column by column of the n x nrhs row-major B, in place). */
int orc_potrs(int64_t n, int64_t nrhs, const double* L, int64_t ldl, double* B, int64_t ldb) {
    for (int64_t r = 0; r < nrhs; ++r) {
        for (int64_t i = 0; i < n; ++i) {
            double t = B[i * ldb + r];
            for (int64_t p = 0; p < i; ++p) t -= L[i * ldl + p] * B[p * ldb + r];
            B[i * ldb + r] = t / L[i * ldl + i];
        }
        for (int64_t i = n - 1; i >= 0; --i) {
            double t = B[i * ldb + r];
            for (int64_t p = i + 1; p < n; ++p) t -= L[p * ldl + i] * B[p * ldb + r];
            B[i * ldb + r] = t / L[i * ldl + i];
        }
    }
    return 0;
}
