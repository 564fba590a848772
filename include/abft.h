/*
 * abft.h -- C ABI of the B300 ABFT one-sided decomposition library (libabft.so).
 *
 * The library factors dense matrices resident in GPU memory with blocked
 * right-looking algorithms (Sec. 2.1 of "Improving Energy Saving of One-sided
 * Matrix Decompositions on CPU-GPU Heterogeneous Systems", PPoPP'23: each
 * iteration runs the panel decomposition PD, the panel update PU and the
 * trailing-matrix update TMU) and protects every iteration with ABFT
 * checksums (Sec. 3.1.2: checksums encoded per matrix block before the
 * operation, carried through it, verified after each iteration; errors are
 * located and corrected; single-side checksums tolerate 0D errors, full
 * checksums 0D and 1D errors; error classes 0D / 1D / 2D).
 *
 * Conventions shared by every entry point
 *  - Matrices are dense, ROW-MAJOR, FP64, with leading dimension ld >= max(1, n).
 *  - All matrix, vector and workspace pointers are DEVICE pointers owned by the
 *    caller; the library never allocates device memory.  `faults` and `rep`
 *    are HOST pointers.  `stream` is a cudaStream_t (NULL = legacy stream).
 *  - Workspace protocol: call with ws == NULL to receive the required size in
 *    *ws_bytes (nothing is launched); then call again with ws pointing to at
 *    least that many bytes (256-byte aligned) and *ws_bytes set to its size.
 *  - Work is enqueued on `stream` asynchronously.  If rep != NULL the call
 *    synchronizes the stream at the end and fills *rep; with rep == NULL the
 *    call only enqueues work (no host synchronization).
 *  - Return value: 0 on success; > 0 is the LAPACK-style info (1-based index
 *    of the first non-positive pivot of potrf, or of the first exactly-zero
 *    pivot of getrf; known only when rep != NULL); -i when argument i
 *    (1-based) is invalid; ABFT_ERR_* below for the remaining failures.
 *  - Checksum block size g equals the block size nb (one checksum tile per
 *    matrix block, Sec. 3.1.2).  nb must be a positive multiple of 32 and at
 *    most 512.
 *  - One GPU per process: several launchers raise their kernels' dynamic
 *    shared-memory limit once per process (a per-device attribute), and the
 *    look-ahead and the no-allocation entry point keep per-device state for
 *    device indices below 16.  Several GPUs are driven by one process each
 *    (the batched form splits its matrices over them with
 *    abft_batched_partition).
 */
#ifndef ABFT_H
#define ABFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Arithmetic of the trailing update (the PD, verify and correction always run in FP64). */
typedef enum {
    ABFT_F64 = 0,        /* FP64 everywhere */
    ABFT_F32 = 1,        /* reserved */
    ABFT_MIXED_BF16 = 2, /* TMU inputs BF16 with per-tile power-of-two scales, FP32 accumulate */
    ABFT_MIXED_F16 = 3,  /* TMU inputs FP16 with per-tile power-of-two scales, FP32 accumulate */
    ABFT_F64_EMU = 4     /* abft_potrf / getrf / geqrf (and posv_ir's residual): FP64-accurate
                            TMU from exact products of BF16 slices on the tensor cores (8
                            balanced base-128 digits per element under a power-of-two row
                            scale, the 36 digit pairs of weight <= 7, FP32 group sums exact
                            for K <= 256, integer recombination; nb <= 256); PD, pivoting,
                            checksum verification and correction in FP64 */
} abft_dtype;

/* Checksum strength (Sec. 3.1.2: single-side vs full checksum ABFT). */
typedef enum {
    ABFT_MODE_NONE = 0,   /* no checksums: the plain blocked factorization   */
    ABFT_MODE_SINGLE = 1, /* column checksums + weighted column checksums    */
    ABFT_MODE_FULL = 2    /* column and row checksums                        */
} abft_mode;

/* Kinds of injected fault (host-listed, numeric; Sec. 3.1.2 error classes). */
typedef enum {
    ABFT_FAULT_MEMORY = 0,  /* +delta at (row, col) after the TMU has stored its result   */
    ABFT_FAULT_COMPUTE = 1, /* +delta added to (row, col) inside the TMU epilogue          */
    ABFT_FAULT_ROW1D = 2,   /* +delta along row `row`, from col to the end of col's block  */
    ABFT_FAULT_COL1D = 3,   /* +delta down column `col`, from row to the end of row's block */
    ABFT_FAULT_PANEL = 4    /* +delta at (row, col) of the panel-update output, before its verify */
} abft_fault_kind;

/* Kinds of reported event. */
typedef enum {
    ABFT_EV_0D = 0,            /* single element located and corrected                    */
    ABFT_EV_ROW = 1,           /* element of a 1D row error corrected                     */
    ABFT_EV_COL = 2,           /* element of a 1D column error corrected                  */
    ABFT_EV_UNCORRECTABLE = 3, /* block with a 2D (or unlocatable) error; row/col = origin */
    ABFT_EV_CHECKSUM = 4,      /* checksum itself wrong, re-encoded; row/col = block origin */
    ABFT_EV_PD = 5             /* panel-decomposition check failed (detect only)          */
} abft_event_kind;

/* A fault to inject (input) or an event that was handled (output).
 * step: 0-based iteration; row, col: 0-based global indices; delta: the
 * injected value, or for events the error size the checksums estimated. */
typedef struct {
    int32_t step;
    int32_t kind;
    int64_t row;
    int64_t col;
    double delta;
} abft_fault;

#define ABFT_MAX_LOC 64

/* Result of one call (host memory, filled when rep != NULL). */
typedef struct {
    int64_t detected;          /* blocks (or PD checks) that raised a flag            */
    int64_t corrected;         /* elements corrected                                  */
    int64_t uncorrectable;     /* blocks or PD checks that could not be corrected     */
    int64_t checksum_repaired; /* blocks whose checksums were re-encoded              */
    int32_t nloc;              /* number of entries in loc (<= ABFT_MAX_LOC)          */
    int32_t info;              /* as the return value's info                          */
    abft_fault loc[ABFT_MAX_LOC]; /* events sorted by (step, row, col, kind); if more
                                     than ABFT_MAX_LOC occurred, which ones are kept
                                     is unspecified (the counters stay exact)         */
    double max_ratio;          /* max |d| / tau over verified blocks without a flag   */
    double tau;                /* detection threshold of the last verified step       */
    int32_t ir_iters;          /* iterative refinement iterations (posv_ir)           */
    int32_t reserved;
    double backward_err;       /* final normwise backward error (posv_ir)             */
    int32_t gmres_iters;       /* GMRES iterations over all refinement steps          */
    int32_t attempts;          /* factorizations tried (posv_gmres_ir shift retries)  */
    double shift;              /* diagonal shift of the factored matrix               */
} abft_report;

#define ABFT_OK 0
#define ABFT_ERR_UNCORRECTABLE (-1000) /* rep != NULL and an uncorrectable error was reported */
#define ABFT_ERR_TIMEOUT (-1001)       /* a bounded device wait gave up                    */
#define ABFT_ERR_CUDA (-1002)          /* a CUDA launch or runtime call failed             */
#define ABFT_ERR_UNSUPPORTED (-1003)   /* valid but unsupported combination (e.g. dtype)   */
#define ABFT_ERR_TOO_LARGE (-1004)     /* the problem needs more than the built-in scratch */

/*
 * abft_potrf -- ABFT-protected blocked Cholesky A = L L^T (lower).
 * Sec. 2.1 (PD = Cholesky of the diagonal block, PU = triangular solve of the
 * panel, TMU = symmetric rank-nb update); Sec. 3.1.2 (checksums).
 *   n, nb      order and block size (nb multiple of 32, <= 512)
 *   dtype      abft_dtype of the TMU
 *   mode       abft_mode
 *   A, lda     n x n row-major; only the lower triangle is read; on return it
 *              holds L; the strict upper triangle is left as it was
 *   faults     host array of nfaults faults to inject (NULL if nfaults == 0);
 *              each must lie in the region its step updates: TMU kinds need
 *              row, col >= (step+1) nb with col/nb <= row/nb; PANEL needs
 *              row >= (step+1) nb and step nb <= col < (step+1) nb; step < N-1
 *   tau_scale  multiplies the detection threshold tau = 8 u n nb max_i a_ii
 *   rep        host report or NULL (see conventions)
 *   ws, ws_bytes  workspace protocol (see conventions)
 * Errors: -1 n < 0; -2 nb invalid; -3 dtype; -4 mode; -5 A NULL with n > 0;
 * -6 lda < max(1,n); -7 faults invalid (or more than 4 COMPUTE faults in one
 * step); -8 nfaults < 0; -9 tau_scale <= 0;
 * -12 workspace too small.
 */
int abft_potrf(int64_t n, int64_t nb, int32_t dtype, int32_t mode, double* A, int64_t lda,
               const abft_fault* faults, int32_t nfaults, double tau_scale,
               abft_report* rep, void* ws, size_t* ws_bytes, void* stream);

/*
 * abft_getrf -- ABFT-protected blocked LU with partial pivoting, P A = L U.
 * Sec. 2.1 (PD = pivoted factorization of the n-K0 x nb panel, PU = unit
 * lower triangular solve of the block row, TMU = rank-nb GEMM update);
 * Sec. 3.1.2 (checksums; row interchanges move the row checksums and add the
 * row difference to the column checksums of the two block rows).
 *   A, lda     n x n row-major; on return L (unit, strictly below the
 *              diagonal) and U (on and above), LAPACK getrf layout
 *   ipiv       device int64[n]: 0-based row interchanged with row i at step i
 *              (first index of the largest |a|, as LAPACK)
 *   faults     TMU kinds need row, col >= (step+1) nb; PANEL faults hit the
 *              block row of U: step nb <= row < (step+1) nb, col >= (step+1) nb
 *   tau_scale  tau_k = tau_scale * 8 u n nb max(max|a_ij|, max|u_ij| so far)
 * Returns as abft_potrf; info > 0 is the first exactly-zero pivot (the
 * factorization is completed, as LAPACK).  dtype ABFT_F64 or ABFT_F64_EMU
 * (nb <= 256: the trailing update and its checksum borders FP64-accurate from
 * BF16 slices on the tensor cores, the rows of L21 and the columns of U12
 * sliced each step; the panel, pivoting and verification stay FP64); other
 * dtypes ABFT_ERR_UNSUPPORTED.  Errors: -1 n; -2 nb; -3 dtype;
 * -4 mode; -5 A; -6 lda; -7 ipiv NULL; -8 faults; -9 nfaults; -10 tau_scale;
 * -13 workspace.
 */
int abft_getrf(int64_t n, int64_t nb, int32_t dtype, int32_t mode, double* A, int64_t lda,
               int64_t* ipiv, const abft_fault* faults, int32_t nfaults, double tau_scale,
               abft_report* rep, void* ws, size_t* ws_bytes, void* stream);

/*
 * abft_geqrf -- ABFT-protected blocked Householder QR, A = Q R.
 * Sec. 2.1 (PD = Householder factorization of the n-K0 x nb panel and the
 * triangular factor T of its block reflector I - V T V^T; TMU = block
 * reflector applied to the trailing columns, C -= V T^T V^T C); Sec. 3.1.2
 * (the row checksums ride through the update as extra columns, the column
 * checksums of each block row are updated by (1^T V_I) T^T V^T C).
 * dtype ABFT_F64, or ABFT_F64_EMU with nb <= 256: V^T V and V^T [C, r]
 * (reduced over the panel rows in 256-row pieces, one exact slice product
 * per piece, summed in FP64 in piece order) and [C, r] -= V X with the
 * checksum rows FP64-accurate from BF16 slices on the tensor cores; the
 * panel, T, X = T^T W and verification in FP64.  Other dtypes
 * ABFT_ERR_UNSUPPORTED.
 *   A, lda     n x n row-major; on return R on and above the diagonal and the
 *              reflectors v (unit leading entry implicit) below, LAPACK
 *              geqrf layout; reflectors follow LAPACK larfg:
 *              beta = -sign(alpha) ||x||, sign(0) = +, tau = (beta - alpha)/beta
 *   tau        device double[n], the reflector scalars
 *   faults     TMU kinds (no PANEL kind): row >= step nb, col >= (step+1) nb
 *   tau_scale  tau = tau_scale * 8 u n nb max_j ||a_j||_2
 * Returns as abft_potrf (no info).  Errors: -1 n; -2 nb; -3 dtype; -4 mode;
 * -5 A; -6 lda; -7 tau NULL; -8 faults; -9 nfaults; -10 tau_scale;
 * -13 workspace.
 */
int abft_geqrf(int64_t n, int64_t nb, int32_t dtype, int32_t mode, double* A, int64_t lda,
               double* tau, const abft_fault* faults, int32_t nfaults, double tau_scale,
               abft_report* rep, void* ws, size_t* ws_bytes, void* stream);

/*
 * abft_potrf_sched -- abft_potrf with one checksum mode per step: the
 * adaptive ABFT of Sec. 3.1.2 (Alg. alg-abft), where each iteration of the
 * decomposition runs without a check, with the single-side or with the full
 * check.  modes: host int32[ceil(n / nb)], ABFT_MODE_* per step.  A step in
 * mode NONE neither carries nor verifies checksums; at a step that checks
 * after an unchecked one, or that moves from SINGLE to FULL, the checksums of
 * the trailing block triangle are encoded afresh from the data (so an error
 * that struck while nothing was checked is not detected).  The workspace is
 * that of abft_potrf in the strongest mode of the schedule.  Returns and
 * errors as abft_potrf (-4: modes NULL or an entry out of range).
 */
int abft_potrf_sched(int64_t n, int64_t nb, int32_t dtype, const int32_t* modes, double* A,
                     int64_t lda, const abft_fault* faults, int32_t nfaults, double tau_scale,
                     abft_report* rep, void* ws, size_t* ws_bytes, void* stream);

/*
 * Fault coverage of one detection interval (Sec. 3.1.2): the probability
 * that single-side (abft_fc_single) or full (abft_fc_full) checksums correct
 * every error, with errors of type 0D / 1D / 2D arriving as independent
 * Poisson processes with mean counts mu0 / mu1 / mu2 in the interval
 * (lambda T) and striking S blocks uniformly; a block corrects at most one
 * error per interval, single-side checksums 0D errors only, full checksums
 * 0D and 1D.  The product of the paper's formulas is read as
 * prod_{i=0}^{k-1} (S - i) / S (k errors in k distinct blocks).  Host only
 * (no GPU needed).  Returns NaN for S <= 0 or a negative or NaN mean.
 */
double abft_fc_single(int64_t S, double mu0, double mu1, double mu2);
double abft_fc_full(int64_t S, double mu0, double mu1, double mu2);

/*
 * abft_adaptive_modes -- the mode policy of Alg. alg-abft without its clock
 * loop (changing clocks is out of scope): for step k with predicted duration
 * step_seconds[k], NONE when every rate is zero, else SINGLE when
 * FC_single >= fc_desired, else FULL (also when FC_full < fc_desired, where
 * the paper would lower the clock; coverage[k] then reports the shortfall).
 * S = ceil(n / nb)^2.  lambda: host double[3], error rates of 0D, 1D, 2D
 * errors per second; modes: host int32[ceil(n / nb)] out; coverage: host
 * double[ceil(n / nb)] out or NULL.  Host only.  Errors: -1 n; -2 nb;
 * -3 lambda; -4 fc_desired outside [0, 1]; -5 step_seconds / modes.
 */
int abft_adaptive_modes(int64_t n, int64_t nb, const double* lambda, double fc_desired,
                        const double* step_seconds, int32_t* modes, double* coverage);

/*
 * abft_potrs -- solve A X = B with the Cholesky factor L of abft_potrf
 * (X = L^{-T} L^{-1} B, forward then backward block substitution).  Not in
 * the paper; the solve that the factorization serves.
 *   n, nrhs    order and number of right-hand sides (processed 16 at a time)
 *   nb         block size of the substitution (multiple of 32, <= 512)
 *   dtype      ABFT_F64: FP64 arithmetic; ABFT_F32 / ABFT_MIXED_*: FP32
 *              arithmetic (the lower triangle of L is rounded to FP32 once,
 *              into the workspace, which then holds n x n floats more)
 *   L, ldl     lower factor (device, row-major); the upper triangle is not read
 *   B, ldb     n x nrhs row-major (device); overwritten by X
 * Errors: -1 n; -2 nrhs; -3 nb; -4 dtype; -5 L; -6 ldl; -7 B; -8 ldb;
 * -10 workspace.
 */
int abft_potrs(int64_t n, int64_t nrhs, int64_t nb, int32_t dtype, const double* L, int64_t ldl,
               double* B, int64_t ldb, void* ws, size_t* ws_bytes, void* stream);

/*
 * abft_syrk_mixed -- the trailing-matrix update (TMU, Sec. 2.1) of abft_potrf
 * in its mixed-precision form (ABFT_MIXED_BF16 / ABFT_MIXED_F16; the form is
 * not in the paper), on its own and without checksums, so that it can be
 * checked element by element.  For each g-row tile I of the m x k panel P:
 * sigma_I = 2^(ceil(log2 max|P_I|) - e_t) (e_t = 0 for BF16, 14 for FP16;
 * 1 for an all-zero tile) and Pq_I = P_I / sigma_I rounded to the 16-bit
 * format (nearest, ties to even); then C -= sigma_I sigma_J (Pq_I Pq_J^T) on
 * the lower block triangle of the m x m matrix C (g x g blocks with J <= I,
 * diagonal blocks in full), the products of the 16-bit operands accumulated
 * in FP32 on the tensor cores and subtracted from C in FP64 (one rounding).
 * Entries outside the lower block triangle are not touched.
 *   m, k       panel rows and width; k a multiple of 64, at most 512
 *   g          tile order, a multiple of 128
 *   dtype      ABFT_MIXED_BF16 or ABFT_MIXED_F16
 *   P, ldp     m x k FP64 row-major (device), read only
 *   C, ldc     m x m FP64 row-major (device), updated in place
 *   Pq         m x k 16-bit codes (device, row-major with ld k, 16-byte
 *              aligned), written
 *   sigma      ceil(m / g) doubles (device), written
 *   timed_out  host int32 or NULL; when given, the call synchronizes its
 *              stream and sets it to 1 if a bounded wait of the update kernel
 *              gave up (then ABFT_ERR_TIMEOUT is returned), else 0
 *   ws, ws_bytes   workspace query protocol as abft_potrf (a status block and
 *              ceil(m / g) x k doubles)
 * Asynchronous on stream unless timed_out is given.  Errors: -1 m; -2 k;
 * -3 g; -4 dtype; -5 P; -6 ldp; -7 C; -8 ldc; -9 Pq; -10 sigma; -13 workspace.
 */
int abft_syrk_mixed(int64_t m, int64_t k, int64_t g, int32_t dtype, const double* P, int64_t ldp,
                    double* C, int64_t ldc, uint16_t* Pq, double* sigma, int32_t* timed_out,
                    void* ws, size_t* ws_bytes, void* stream);

/*
 * abft_symm_emu -- Y = A X for symmetric A (lower triangle read), FP64-accurate
 * on the BF16 tensor cores (the product of the refinement residuals; not in the
 * paper).  A is split into 8 BF16 slices of its full rows (a power-of-two
 * scale per row, balanced base-128 digits), each block of up to 16 columns of
 * X into 8 slices per column; the 36 slice pairs whose weights add up to at
 * most 7 are summed exactly (FP32 accumulation over 256 terms, 64-bit integer
 * combination), the 256-term chunks in FP64.  Error per element at most about
 * n 2^-55 (row scale of A)(column scale of X), below the rounding of the same
 * dot product in FP64; exact when every product and partial sum is an integer
 * below 2^53 whose digits fit the slices (e.g. small integers).
 *   n          order, a multiple of 32 (ABFT_ERR_UNSUPPORTED otherwise)
 *   A, lda     device, row-major, lower triangle read, not modified
 *   X, ldx     n x nrhs device, row-major;  Y, ldy  n x nrhs device output
 *   ws, ws_bytes   workspace query protocol (ws = NULL: *ws_bytes = the
 *              size, 16 n^2 + O(n) bytes)
 * Returns 0 or an argument error: -1 n; -2 nrhs; -3 A; -4 lda; -5 X; -6 ldx;
 * -7 Y; -8 ldy; -10 workspace.
 */
int abft_symm_emu(int64_t n, int64_t nrhs, const double* A, int64_t lda, const double* X,
                  int64_t ldx, double* Y, int64_t ldy, void* ws, size_t* ws_bytes, void* stream);

/*
 * abft_posv_ir -- solve A X = B for SPD A by an ABFT Cholesky in the given
 * dtype followed by iterative refinement (not in the paper: the precision
 * form added on top of it).  L := A (lower triangle copied), abft_potrf(L),
 * X = L^{-T} L^{-1} B, then repeat: R = B - A X in FP64 (A symmetric, read
 * from its lower triangle; for the 16-bit dtypes and ABFT_F64_EMU with n a
 * multiple of 32 the products A X are FP64-accurate sums of exact BF16 slice
 * products on the
 * tensor cores -- A split once per call into 8 slices of its full rows, n^2
 * 16 bytes of workspace -- with an error below that of the same dot products
 * in FP64 arithmetic), eta = max_r ||R_r||_inf / (||A||_inf ||X_r||_inf +
 * ||B_r||_inf); stop when eta <= tol or after maxit corrections; otherwise
 * D = L^{-T} L^{-1} R (FP32 for the mixed dtypes, FP64 for ABFT_F64 and
 * ABFT_F64_EMU, whose factor an FP32 solve would not use) and X += D.
 * ABFT_F64_EMU (nb 128 or 256) suits ill-conditioned A: its factor is as
 * accurate as the FP64 one, so refinement converges while kappa u64 << 1.  rep (optional) receives the factorization report plus ir_iters and
 * backward_err (max over right-hand sides).  The call synchronizes the stream
 * once per refinement step (to read eta).
 *   A, lda     SPD matrix (device, lower triangle read, not modified)
 *   L, ldl     n x n device buffer receiving the factor
 *   B, ldb / X, ldx   n x nrhs right-hand sides / solution (device, row-major)
 * Returns the factorization's code (0, info > 0 on a non-positive pivot,
 * ABFT_ERR_UNCORRECTABLE) or an argument error: -1 n; -2 nrhs; -3 nb;
 * -4 dtype; -5 mode; -6 A; -7 lda; -8 L; -9 ldl; -10 B; -11 ldb; -12 X;
 * -13 ldx; -14 tol; -15 maxit; -16 faults; -22 workspace.
 */
int abft_posv_ir(int64_t n, int64_t nrhs, int64_t nb, int32_t dtype, int32_t mode, const double* A,
                 int64_t lda, double* L, int64_t ldl, const double* B, int64_t ldb, double* X,
                 int64_t ldx, double tol, int32_t maxit, const abft_fault* faults, int32_t nfaults,
                 double tau_scale, abft_report* rep, void* ws, size_t* ws_bytes, void* stream);

/*
 * abft_posv_gmres_ir -- solve A X = B for SPD A by GMRES-based iterative
 * refinement (Carson and Higham, SISC 2017 / 2018) preconditioned by an ABFT
 * Cholesky factor in the given dtype, with the diagonal scaling and shift of
 * Higham and Pranesh (SISC 2021) for low-precision factorizations.  Not in
 * the paper: the precision form added on top of it, for ill-conditioned A.
 *   S = diag(s_i), s_i = 2^-t_i, t_i = e_i / 2 rounded toward zero, with
 *       a_ii = f 2^e_i, f in [1/2, 1) (scale != 0; else S = I), so S A S is
 *       formed exactly and its diagonal lies in [1/4, 2);
 *   L := lower(S A S + delta I) (the upper triangle of L is not written),
 *       abft_potrf(L) in dtype; with shift < 0 a
 *       non-positive pivot restarts the factorization with delta = u_f, then
 *       4 delta (at most 8 attempts; u_f = 2^-8 BF16, 2^-11 FP16, 2^-53 FP64);
 *       shift >= 0 fixes delta = shift;
 *   M^{-1} v = S L^{-T} L^{-1} S v (FP64 substitution if precond_f64, else FP32);
 *   inner_f32 != 0: GMRES's products with A use an FP32 copy of A and FP32
 *       arithmetic (the five-precision GMRES-IR of Amestoy, Buttari, Higham,
 *       L'Excellent, Mary and Vieuble, SIMAX 2024, with GMRES and the
 *       preconditioner in FP32); the residual R and the update of X stay FP64;
 *       the workspace then holds n x n floats more;
 *   X = M^{-1} B; repeat: R = B - A X in FP64, eta as abft_posv_ir; stop at
 *       eta <= tol or after maxit refinement steps; else run GMRES (left
 *       preconditioned, Arnoldi with classical Gram-Schmidt applied twice,
 *       Givens rotations, FP64) on M^{-1} A D = M^{-1} R from D = 0 until its
 *       residual falls to inner_tol times the initial one for every
 *       right-hand side or m iterations, and X += D.
 *   m          GMRES iterations per refinement step, 1 .. 64
 * rep (optional) receives the factorization report plus ir_iters, gmres_iters,
 * attempts, shift (delta) and backward_err.  The call synchronizes the stream
 * once per GMRES iteration.  Returns as abft_posv_ir; argument errors as
 * abft_posv_ir plus -16 m; -17 inner_tol; -18 shift NaN; -19 faults.
 */
int abft_posv_gmres_ir(int64_t n, int64_t nrhs, int64_t nb, int32_t dtype, int32_t mode,
                       const double* A, int64_t lda, double* L, int64_t ldl, const double* B,
                       int64_t ldb, double* X, int64_t ldx, double tol, int32_t maxit, int32_t m,
                       double inner_tol, double shift, int32_t scale, int32_t precond_f64,
                       int32_t inner_f32, const abft_fault* faults, int32_t nfaults,
                       double tau_scale, abft_report* rep, void* ws, size_t* ws_bytes,
                       void* stream);

/*
 * Reverse mode (adjoints) of potrf, potrs and logdet -- not in the paper: the
 * differentiation form added on top of it.  Convention: a function of a
 * symmetric A that reads only its lower triangle has the lower-triangular
 * adjoint Abar (df = sum_{i >= j} Abar[i][j] dA[i][j]); the symmetric gradient
 * is (Abar + Abar^T) / 2.  All matrices are device, row-major FP64.
 *
 * abft_potrf_backward: given the factor L (lower triangle read) and the
 * adjoint Lbar of L (lower triangle read), writes Abar: with sym == 0 the
 * lower-triangle adjoint (strict upper triangle set to zero), with sym != 0
 * the symmetric gradient (Abar + Abar^T) / 2 in both triangles.  Blocked reverse sweep of the
 * right-looking algorithm (Murray, "Differentiation of the Cholesky
 * decomposition", 2016), block size nb, from the last block to the first:
 * Lbar21 -= (Abar22 + Abar22^T) L21; Abar21 = Lbar21 L11^{-1};
 * Lbar11 -= tril(Abar21^T L21); Abar11 = Phi(S + S^T) with
 * S = L11^{-T} Phi(L11^T Lbar11) L11^{-1}, Phi = lower triangle with halved
 * diagonal.  Only L and Lbar are read: no forward intermediates are stored.
 * Errors: -1 n; -2 nb; -3 L; -4 ldl; -5 Lbar; -6 ldlb; -7 Abar; -8 ldab; -11 ws.
 *
 * abft_potrf_backward_ex: the same with the arithmetic of the dominant
 * product chosen by dtype: ABFT_F64 (FP64 FMA; abft_potrf_backward) or
 * ABFT_F64_EMU, where Lbar21 -= (Abar22 + Abar22^T) L21 -- about two thirds
 * of the sweep's flops -- is FP64-accurate from exact BF16 slice products on
 * the tensor cores (the splitting of abft_potrf's ABFT_F64_EMU: per block
 * column of Abar22 + Abar22^T, sliced once when the sweep finalizes it, and
 * per block row of L21; error per term below the FP64 rounding of the same
 * product).  ABFT_F64_EMU needs nb = 128 or 256 and n a multiple of nb
 * (ABFT_ERR_UNSUPPORTED otherwise) and 16 n (n + nb) more bytes of workspace;
 * it synchronizes the stream once at the end (to read the status of its
 * bounded waits; ABFT_ERR_TIMEOUT if one gave up).  Errors as
 * abft_potrf_backward, plus -12 dtype.
 *
 * abft_potrs_backward: for X = A^{-1} B computed with the factor L and the
 * adjoint Xbar of X (n x nrhs, nrhs <= 16): Bbar = A^{-1} Xbar, and
 * Lbar -= tril((Bbar X^T + X Bbar^T) L) (accumulated into Lbar's lower
 * triangle).  Errors: -1 n; -2 nrhs; -3 nb; -4..-13 pointers and leading
 * dimensions in argument order; -15 ws.
 *
 * abft_logdet: *out (device double) = log det A = 2 sum_i log L[i][i].
 * abft_logdet_backward: Lbar[i][i] += 2 gbar / L[i][i] for the adjoint gbar
 * of log det A.
 * abft_tril: zero the strict upper triangle of A (n x n).
 */
int abft_potrf_backward(int64_t n, int64_t nb, const double* L, int64_t ldl, const double* Lbar,
                        int64_t ldlb, double* Abar, int64_t ldab, int32_t sym, void* ws,
                        size_t* ws_bytes, void* stream);
int abft_potrf_backward_ex(int64_t n, int64_t nb, int32_t dtype, const double* L, int64_t ldl,
                           const double* Lbar, int64_t ldlb, double* Abar, int64_t ldab,
                           int32_t sym, void* ws, size_t* ws_bytes, void* stream);
int abft_potrs_backward(int64_t n, int64_t nrhs, int64_t nb, const double* L, int64_t ldl,
                        const double* X, int64_t ldx, const double* Xbar, int64_t ldxb,
                        double* Bbar, int64_t ldbb, double* Lbar, int64_t ldlb, void* ws,
                        size_t* ws_bytes, void* stream);
int abft_logdet(int64_t n, const double* L, int64_t ldl, double* out, void* stream);
int abft_logdet_backward(int64_t n, const double* L, int64_t ldl, double gbar, double* Lbar,
                         int64_t ldlb, void* stream);
int abft_tril(int64_t n, double* A, int64_t lda, void* stream);

/*
 * Batched ABFT Cholesky -- many independent small SPD matrices in one
 * persistent launch (not in the paper: the batching form added on top of it).
 * Each matrix is factored by one CTA with the same blocked algorithm and full
 * (or no) checksums as abft_potrf, block size nb = 32 or 64 per matrix.
 * Descriptors and statuses live in DEVICE memory; a CTA takes the next
 * descriptor from an atomic queue, so order the descriptors by decreasing n
 * (longest first).  At most one fault per matrix (kinds MEMORY, COMPUTE,
 * PANEL; fstep = -1 for none) with the same placement rules as abft_potrf.
 */
typedef struct {
    void* A;          /* device, row-major, FP64 (dtype ABFT_F64) or FP32 (ABFT_F32) */
    int64_t lda;
    int32_t n;        /* 1 .. 512 */
    int32_t id;       /* index of this matrix's status entry */
    int32_t nb;       /* 32 or 64 */
    int32_t fstep;    /* injected fault: step (-1 = none), kind, row, col, delta */
    int32_t fkind;
    int32_t frow;
    int32_t fcol;
    int32_t pad;
    double fdelta;
} abft_batch_item;

typedef struct {
    int32_t info;          /* 1-based first non-positive pivot, 0 = factored */
    int32_t detected;
    int32_t corrected;
    int32_t uncorrectable;
    int32_t ev_step;       /* first event of this matrix (-1 = none) */
    int32_t ev_kind;
    int32_t ev_row;
    int32_t ev_col;
} abft_batch_status;

/*
 * abft_potrf_batched: factor `count` matrices described by the device array
 * `items`; per-matrix results go to the device array `status` (indexed by
 * item.id).  dtype: ABFT_F64 or ABFT_F32 (arithmetic and storage); mode:
 * ABFT_MODE_NONE or ABFT_MODE_FULL; tau = tau_scale * 8 u n nb max_i a_ii
 * with u the unit roundoff of dtype.  use_graph != 0: the launch sequence
 * (queue reset + persistent kernel) is captured once into a CUDA graph per
 * (items, count, dtype, mode, status, workspace, stream) and replayed.
 * Workspace protocol as abft_potrf.  The arguments of the descriptors are
 * not validated on the host (they are device memory); invalid n is skipped.
 * Errors: -1 count; -2 items; -3 dtype; -4 mode; -6 status; -9 ws.
 */
int abft_potrf_batched(int32_t count, const abft_batch_item* items, int32_t dtype, int32_t mode,
                       double tau_scale, abft_batch_status* status, int32_t use_graph, void* ws,
                       size_t* ws_bytes, void* stream);

/* Destroy the CUDA graphs cached by abft_potrf_batched (call before freeing
 * the memory their keys refer to, if the same addresses may be reused). */
int abft_batched_graph_reset(void);

/*
 * abft_batched_set_ctas_per_sm: how many persistent CTAs per SM the next
 * abft_potrf_batched launches use (the launch-level knob of the tuner in
 * tune.py; the per-matrix knob is the block size item.nb).  0 restores the
 * default, the most that fit (FP64 2, FP32 4); larger values are clamped to
 * it.  Process-wide; a cached graph is keyed by the grid it was captured
 * with.  The factors do not depend on it (each matrix is factored by one
 * CTA).  Not in the paper.  Returns the previous setting, or -1 for a
 * negative argument.
 */
int abft_batched_set_ctas_per_sm(int32_t ctas);

/*
 * abft_batched_partition -- split a batch of independent factorizations
 * (abft_potrf_batched) over G GPUs, one process per GPU, so that every GPU
 * gets about the same work.  Not in the paper (the batched form's multi-GPU
 * split; the matrices are independent, so nothing is exchanged on the data
 * path: each GPU factors its share, the statuses are gathered on the host).
 * Longest processing time first on the work n_i^3 / 3: the matrices in
 * decreasing work (ties: lower index first), each to the GPU with the least
 * work so far (ties: lower GPU index).  The largest share exceeds the
 * smallest by at most one matrix's work.  Host only, deterministic.
 *   count, n   number of matrices and their orders (host, n_i >= 0)
 *   G          number of GPUs (>= 1)
 *   owner      host int32[count] out: the GPU of each matrix
 *   load       host double[G] out, or NULL: each GPU's work in flops
 * Errors: -1 count; -2 n; -3 G; -4 owner.
 */
int abft_batched_partition(int32_t count, const int64_t* n, int32_t G, int32_t* owner,
                           double* load);

/*
 * abft_wait_selftest -- exercises the give-up path of the library's bounded
 * waits on purpose-built cases (no counterpart in the paper; the failure
 * path of every persistent and cooperative kernel).  Every device-side wait
 * of the library is bounded: the cooperative kernels' grid barrier gives up
 * after 2 s, the tensor-core kernels' mbarrier waits after 1 s; a CTA that
 * gives up records a timeout in the call's status block, releases its tensor
 * memory and returns, and the call returns ABFT_ERR_TIMEOUT.  Here the limit
 * is limit_ns (1 .. 2e9) and the case is one of
 *   0  two CTAs at one grid barrier, one never arrives  -> ABFT_ERR_TIMEOUT
 *   1  one CTA holding 32 TMEM columns waits on an mbarrier that gets one of
 *      its two arrivals (it frees the columns after giving up) -> ABFT_ERR_TIMEOUT
 *   2, 3  the same with every arrival (the waits complete)  -> 0
 * error_out (host, nullable) receives the status block's error code (0 none,
 * 1 grid barrier, 2 mbarrier).  Synchronizes the stream.  Workspace query
 * protocol as abft_potrf (one status block).  Errors: -1 which; -2 limit_ns;
 * -5 workspace.
 */
int abft_wait_selftest(int32_t which, int64_t limit_ns, int32_t* error_out, void* ws,
                       size_t* ws_bytes, void* stream);

/*
 * abft_fp64_pipe_probe -- diagnostics (no counterpart in the paper): the
 * FP64 multiply-add rate of this GPU measured two ways, which = 0 the FP64
 * FMA of the CUDA cores, which = 1 the FP64 tensor-core MMA (mma.sync
 * m8n8k4); four CTAs of 256 threads per SM, 8 independent chains per thread
 * (4 accumulators per warp for the MMA), iters steps each.  *tflops_out
 * receives the rate of the second of two launches (CUDA events).  Behind the
 * library's choice of the FMA for its FP64 arithmetic.  Synchronizes the
 * stream.  Errors: -1 which; -2 iters (1 .. 2^24); -3 tflops_out.
 */
int abft_fp64_pipe_probe(int32_t which, int64_t iters, double* tflops_out, void* stream);

/* Size of the built-in device scratch array used by abft_potrf_noalloc. */
#define ABFT_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)   /* 16 MiB per GPU */

/*
 * abft_potrf_noalloc -- abft_potrf for callers that cannot allocate device
 * memory.  The paper has no counterpart: it exists for host programs whose
 * own allocator or arena owns the whole GPU (or that may not grow the
 * process's device footprint) and therefore can neither call cudaMalloc nor
 * pass a workspace.  Arguments and results are those of abft_potrf without
 * ws / ws_bytes; A is still the caller's.  The workspace is a built-in device
 * array of ABFT_NOALLOC_SCRATCH_BYTES (16 MiB), present on every GPU where
 * the library's device code is loaded and kept there until the process
 * exits; a problem whose abft_potrf workspace would exceed it is rejected with
 * ABFT_ERR_TOO_LARGE before anything is launched (for example, ABFT_F64 in
 * FULL mode fits n = 4096 with nb <= 256; the other dtypes need more).  The first call on a device looks up the array's
 * device address (with that device current); make that first call before any
 * stream capture.  Every call reuses the same array and it keeps the previous
 * call's contents (the status block at its start is cleared by each call,
 * everything else is written before it is read), so calls whose GPU work
 * overlaps (on different streams, or from different threads) race; serialize
 * them.  The call makes no cudaMalloc, cudaFree or other device-memory
 * allocation; like abft_potrf, a thread's first factorization on a device
 * creates the look-ahead's side stream and its two events once.  Like the
 * rest of the library it assumes one GPU per process (device index < 16).
 */
int abft_potrf_noalloc(int64_t n, int64_t nb, int32_t dtype, int32_t mode, double* A, int64_t lda,
                       const abft_fault* faults, int32_t nfaults, double tau_scale,
                       abft_report* rep, void* stream);

/*
 * abft_set_lookahead(on): look-ahead of the blocked Cholesky (Sec. 2.1, the
 *   look-ahead of Fig. example-lu (b), here on one GPU).  On (the default),
 *   abft_potrf / abft_posv_* with one checksum mode for all steps split each
 *   trailing update: the next block column is updated and verified first,
 *   then the next diagonal block is factored (PD of the next step, with its
 *   checksum check) on the caller's stream while the rest of the update and
 *   its verification run on an internal stream of the calling thread; the
 *   caller's stream waits for both before the next panel solve.  Every kernel
 *   performs the same arithmetic either way: factors, reports and return codes
 *   are identical with look-ahead on and off.  Per-step schedules
 *   (abft_potrf_sched) always run sequentially.  The internal stream and its
 *   events are created on the first call that uses them on a device (make it
 *   before any stream capture).  Returns the previous setting (0 or 1).
 */
int abft_set_lookahead(int32_t on);

/*
 * Diagnostics (no counterpart in the paper; the paper profiles per-operation
 * times only to predict slack, Sec. 3.2.1).
 * abft_timing_enable(on): when on != 0, every entry point records CUDA events
 *   around its phases on its stream (0 PD + PD check, 1 PU + panel verify,
 *   2 TMU, 3 fault injection + trailing verify, 4 encode / set-up, 5 solves
 *   and refinement), then
 *   synchronizes its stream before returning; resets the accumulators.
 * abft_timing_read(ms, count, nphase): accumulated milliseconds (and number of
 *   timed intervals) per phase since the last enable.
 * abft_launch_count(): number of kernels this library has launched so far.
 */
int abft_timing_enable(int32_t on);
int abft_timing_read(double* ms, int64_t* count, int32_t nphase);

/*
 * abft_timing_marks(phase, step, ms, max): the timed intervals recorded since
 *   the last abft_timing_enable, in recording order: phase (as above), the
 *   Cholesky iteration the interval belongs to (-1 outside the step loop;
 *   the look-ahead PD is attributed to the iteration it factors) and its
 *   milliseconds.  Writes at most max entries (host arrays); returns the
 *   number of intervals, or -1 on bad arguments.
 *
 * abft_predict_step_times(T, W, nsteps, pred): the enhanced algorithmic
 *   per-iteration time prediction of Sec. 3.2.1 (host only):
 *   pred[k] = sum_i w_i (W[k] / W[k-i]) T[k-i], i = 1 .. 4, w = 1/2, 1/4,
 *   1/8, 1/8, over the previous iterations j = k - i with W[j] > 0 and
 *   T[j] >= 0; when fewer than four are usable their weights are
 *   renormalized to sum to one (the paper is silent on the first
 *   iterations); pred[k] = NaN when none is.  T: measured times, W: the
 *   operation's work per iteration (any unit).  Returns 0, or -1 on bad
 *   arguments.
 *
 * abft_chol_step_work(n, nb, phase, k): the work of one operation of
 *   iteration k of the blocked Cholesky as this library performs it, for
 *   abft_predict_step_times: PD kb^3/3, PU m kb^2, TMU 2 kb E (flops), verify
 *   E + m kb (elements), with kb the block width, m the trailing order and E
 *   the elements of the trailing lower block triangle (diagonal blocks
 *   full); phase as in abft_timing_read; 0 for other phases or past the end.
 */
int abft_timing_marks(int32_t* phase, int64_t* step, double* ms, int32_t max);
int abft_predict_step_times(const double* T, const double* W, int64_t nsteps, double* pred);
double abft_chol_step_work(int64_t n, int64_t nb, int32_t phase, int64_t k);
int64_t abft_launch_count(void);

/* Library version string. */
const char* abft_version(void);

/* Text for a return code. */
const char* abft_strerror(int32_t code);

#ifdef __cplusplus
}
#endif

#endif /* ABFT_H */
