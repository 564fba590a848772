// common.cuh -- internal declarations shared by the CUDA translation units of
// libabft.so (device status block, tile sets, kernel launchers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "abft.h"

namespace abft {

// Device-resident status of one factorization call.  Lives at the start of
// the caller's workspace; zeroed at the start of every call.
struct DevStatus {
    int info;                          // 1-based first bad pivot (0 = none)
    int nloc;                          // events appended (may exceed ABFT_MAX_LOC)
    unsigned long long detected;
    unsigned long long corrected;
    unsigned long long uncorrectable;
    unsigned long long repaired;
    unsigned long long max_ratio_bits; // bit pattern of a non-negative double
    double tau;                        // current detection threshold
    double amax;                       // max |a_ij| of the input (LU) / max column norm (QR)
    double umax;                       // running max |u_ij| (LU)
    int error;                         // internal error code (timeouts)
    int lu_info;                       // LU: 1-based first exactly-zero pivot (factorization continues)
    int vexp;                          // > 0: biased exponent bound of the verified entries (fixed-point sums)
    unsigned long long bar_count;      // grid barrier of the cooperative panel kernels:
                                       // arrivals since the launch (zeroed by the launcher)
    // mixed-precision Cholesky: trailing tiles are checked against per-column
    // (per-row) thresholds tau_coef |c| + tau64 from the abs-checksums
    double tau64;                      // FP64 part of those thresholds
    double tau_coef;                   // tau_scale * 4 * gamma_g(2^-24); 0 = scalar tau
    unsigned long long tau_max_bits;   // largest such threshold applied (bits of a double >= 0)
    abft_fault loc[ABFT_MAX_LOC];
};

// Grid-wide barrier for cooperative launches (all CTAs co-resident).  The
// wait is bounded: after kBarrierNs of spinning the CTA records a timeout in
// st->error and the barrier returns false, so no CTA can wait forever.
constexpr unsigned long long kBarrierNs = 2000000000ull;  // 2 s
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool grid_barrier(DevStatus* st, unsigned int nblocks,
                                             unsigned long long& passed,
                                             unsigned long long limit_ns = kBarrierNs) {
    // bar_count only grows during a launch: barrier number `passed` (1, 2, ...)
    // is complete once every CTA has added its arrival, i.e. at passed * nblocks,
    // so the last arrival's own increment releases the waiters (no reset and no
    // generation flag on the critical path).  A CTA that gives up never arrives
    // again, so the others give up at their next wait as well.
    __shared__ int s_ok;
    __syncthreads();
    ++passed;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long target = passed * nblocks;
        __threadfence();
        const unsigned long long seen = atomicAdd(&st->bar_count, 1ull) + 1ull;
        if (seen < target) {
            volatile unsigned long long* vc = &st->bar_count;
            const unsigned long long t0 = global_ns();
            while (*vc < target) {
                if (global_ns() - t0 > limit_ns) {
                    atomicExch(&st->error, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

enum { MODE_NONE = 0, MODE_SINGLE = 1, MODE_FULL = 2 };
enum { EV_0D = 0, EV_ROW = 1, EV_COL = 2, EV_UNCORR = 3, EV_CKSUM = 4, EV_PD = 5 };

__device__ __forceinline__ void record_event(DevStatus* st, int step, int kind, int64_t row,
                                             int64_t col, double d) {
    int idx = atomicAdd(&st->nloc, 1);
    if (idx < ABFT_MAX_LOC) {
        abft_fault& e = st->loc[idx];
        e.step = step;
        e.kind = kind;
        e.row = row;
        e.col = col;
        e.delta = d;
    }
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
    if (!(v >= 0.0)) return;
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// A set of g x g checksum tiles (I, J), I in [I0, I1), J in [J0, J1),
// optionally restricted to J <= I (lower block triangle).  Element pointers:
//   T(I,J)  = A  + (I g) lda + (J g)
//   cc(I,J) = cc + I ccI + J g           (column sums, a row vector)
//   cw(I,J) = cw + I ccI + J g           (weighted column sums)
//   cr(I,J) = cr + (I g) crs + J crJ     (row sums, stride crs)
// Rows end at nrow_end, columns at ncol_end (global indices).
struct TileSet {
    double* A;
    int64_t lda;
    double* cc;
    double* cw;
    int64_t ccI;
    double* cr;
    int64_t crs, crJ;
    int64_t g;
    int64_t I0, I1, J0, J1;
    int lower;
    int64_t nrow_end, ncol_end;
    int weighted;   // encode also writes the weighted column sums (cw)
    // verify only, mixed-precision Cholesky: abs-checksums (FP32) laid out as
    // cc and cr (ca(I,J) = ca + I caI + J g, ra(I,J) = ra + (I g) crs + J crJ);
    // when set, column j is flagged above tau_coef ca_j + tau64 and row i above
    // tau_coef ra_i + tau64 (formed in FP32) instead of the scalar tau
    const float* ca;
    int64_t caI;
    const float* ra;
};

cudaError_t launch_encode(const TileSet& ts, int mode, cudaStream_t s);
cudaError_t launch_verify(const TileSet& ts, int mode, int step, DevStatus* st, cudaStream_t s);
cudaError_t launch_inject(double* A, int64_t lda, int64_t n, int64_t g, const abft_fault& f,
                          cudaStream_t s);
cudaError_t launch_mirror_diag(double* A, int64_t lda, int64_t n, int64_t nb, double* save,
                               int restore, cudaStream_t s);
// tau_coef > 0 (mixed precision): also stores tau64 (the FP64 threshold) and
// tau_coef for the per-column thresholds.
cudaError_t launch_tau_chol(const double* A, int64_t lda, int64_t n, int64_t g, double tau_scale,
                            DevStatus* st, cudaStream_t s, double unit_roundoff = 0x1p-53,
                            double tau_coef = 0.0);

// FP64 update C -= A_op * B_op^T (NT) or A_op * B_op (NN), over up to three
// segments (the main tiles and the checksum border rows / columns).
struct GemmSeg {
    const double* A;   // A[i*lda + p] (K-major: A[p*lda + i])
    int64_t lda;
    const double* B;   // NT: B[j*ldb + p];  NN: B[p*ldb + j]
    int64_t ldb;
    double* C;
    int64_t ldc;
    int64_t M, N, K;
    // lower-block mask: element (i, j) is updated only when
    // (i + row0) / g >= (j + col0) / g  (g == 0: no mask)
    int64_t g, row0, col0;
};
struct ComputeFault {
    int64_t row, col;  // indices local to segment 0, -1 = none
    double delta;
};
enum { MAX_CF = 4 };
// a_kmajor: 0 row-major A, 1 K-major A, 2 symmetric A + A^T read from its lower triangle.
cudaError_t launch_gemm_f64(const GemmSeg* segs, int nseg, int a_kmajor, int b_kmajor,
                            const ComputeFault* cf, int ncf, const DevStatus* st, cudaStream_t s);
// One segment, K split over kparts CTAs (partials in `part`, kparts x M x N), then reduced
// in a fixed order into C (with the lower-block mask).
cudaError_t launch_gemm_f64_splitk(const GemmSeg& seg, int a_kmajor, int b_kmajor, int kparts,
                                   double* part, const DevStatus* st, cudaStream_t s);

cudaError_t launch_potf2_small(double* A, int64_t lda, int64_t nb, int64_t info_base,
                               DevStatus* st, cudaStream_t s);
// FP64 factorization of a kb x kb (kb <= 256) diagonal block by one thread-block
// cluster; check != 0 then tests it against the carried column checksum cc
// (k_pd_cluster.cu).  A non-positive pivot sets info = K0 + column + 1.
int pd_cluster_size();   // CTAs of the cluster PD (16 where supported, else 8)
cudaError_t launch_potrf_pd_cluster(double* A, int64_t lda, int64_t kb, int64_t K0,
                                    const double* cc, int step, int check, DevStatus* st,
                                    cudaStream_t s);
// X L^T = B (nt = false) or X L = B (nt = true, FP64 only) for the rows of up
// to two row segments (in place); L lower nb x nb.
// If v != NULL, x[i] = B_i . v is stored for the rows of segment 0 before the solve.
struct TrsmSeg {
    double* B;
    int64_t ldb;
    int64_t rows;
};
cudaError_t launch_trsm_rows(const double* L, int64_t ldl, int64_t nb, const TrsmSeg* segs,
                             int nseg, const DevStatus* st, cudaStream_t s, bool f32 = false,
                             bool rev = false);
// lf (FP32 X L^T = B only): L rounded to FP32 beforehand by launch_l_to_f32.
cudaError_t launch_trsm_rlt(const double* L, int64_t ldl, int64_t nb, const TrsmSeg* segs,
                            int nseg, const double* v, double* x, const DevStatus* st,
                            cudaStream_t s, bool f32 = false, bool nt = false,
                            const float* lf = nullptr);
cudaError_t launch_l_to_f32(const double* L, int64_t ldl, int64_t nb, float* Lf, cudaStream_t s);
cudaError_t launch_chol_pd_check(const double* L, int64_t ldl, int64_t nb, const double* cc,
                                 int64_t K0, int step, double* v, int mode, DevStatus* st,
                                 cudaStream_t s);

// LU kernels (k_lu.cu).
int num_sms();
size_t getf2_stage_bytes(int64_t kb);   // pivot-row copies of launch_getf2_coop
cudaError_t launch_getf2_coop(double* P, int64_t lda, int64_t m, int64_t kb, int64_t K0,
                              int64_t* ipiv, DevStatus* st, double* part_v, int64_t* part_i,
                              double* stage, cudaStream_t s);
cudaError_t launch_laswp(double* A, int64_t lda, int64_t n, int64_t K0, int64_t kb,
                         const int64_t* ipiv, double* CS, int64_t ldcs, int64_t nc, int64_t g,
                         double* Cr, int64_t nt, int mode, cudaStream_t s);
cudaError_t launch_coltot(const double* CS, int64_t ldcs, int64_t nc, int64_t k, int64_t nt,
                          int64_t K0, int64_t kb, double* ptot, cudaStream_t s);
cudaError_t launch_lu_colsums(const double* P, int64_t lda, int64_t m, int64_t kb, int64_t g,
                              int64_t k, int64_t nt, int64_t K0, double* CS, int64_t ldcs,
                              int64_t nc, int mode, double* part, int64_t ldpart, cudaStream_t s);
cudaError_t launch_lu_pd_check(const double* P, int64_t lda, int64_t kb, const double* ptot,
                               const double* part, int64_t ldpart, int nparts, int step,
                               int64_t K0, int64_t n, int64_t g, double tau_scale, double* z,
                               double* zw, int mode, DevStatus* st, cudaStream_t s);
cudaError_t launch_trsm_llu(const double* L, int64_t ldl, int64_t kb, double* B0, int64_t ldb0,
                            int64_t ncols0, double* B1, int64_t ldb1, int64_t ncols1,
                            const double* z, const double* zw, double* colchk, double* colchkw,
                            cudaStream_t s, bool colchk_only = false);
cudaError_t launch_absmax(const double* A, int64_t lda, int64_t rows, int64_t cols, double* out,
                          cudaStream_t s);

// QR kernels (k_qr.cu).
cudaError_t launch_geqr2_coop(double* P, int64_t lda, int64_t m, int64_t kb, double* tau,
                              double* nrm, double* part, double* wv, DevStatus* st,
                              cudaStream_t s);
cudaError_t launch_qr_pd_check(const double* P, int64_t lda, int64_t kb, const double* nrm,
                               int step, int64_t K0, DevStatus* st, cudaStream_t s);
cudaError_t launch_qr_prep_v(const double* P, int64_t lda, int64_t m, int64_t kb, double* V,
                             cudaStream_t s);
cudaError_t launch_qr_vsums(const double* V, int64_t m, int64_t kb, int64_t g, int64_t k,
                            int64_t nt, int64_t K0, double* CS, int64_t ldcs, int64_t nc, int mode,
                            cudaStream_t s);
cudaError_t launch_larft(const double* Gneg, int64_t kb, const double* tau, double* T,
                         cudaStream_t s);
cudaError_t launch_qr_tau(const double* A, int64_t lda, int64_t n, int64_t g, double tau_scale,
                          DevStatus* st, cudaStream_t s);

// Mixed-precision TMU kernels (k_mixed.cu).
// Checksum borders of the mixed update of trailing rows T0 + [0, m): the
// products of the quantized panel rows Lq_j with the FP32 checksum vectors of
// blocks [Jb, Je) (nc signed sums per block in tq, one abs sum in ta).  Rows
// j in [c0, c1) update the column-checksum rows CS / Ca; blocks J in [J0, J1)
// update the row-checksum columns Cr / Ra (null: single-side checksums).
struct BorderSymHost {
    const uint16_t* Lq;
    int64_t m, K;
    int bf16;
    const float* tq;
    const float* ta;
    int nc;
    int64_t Jb, Je;
    double* CS;
    float* Ca;
    int64_t ldcs, T0;
    double* Cr;
    float* Ra;
    int64_t ldr;
    int64_t c0, c1, J0, J1;
    int64_t g;
    const double* sig;
};
// tabs32 (nullable): 1^T |Lq_I| per tile-row, FP32, at tabs32[I kb + p].
cudaError_t launch_quant_panel(const double* P, int64_t lda, int64_t T0, int64_t n, int64_t kb,
                               int64_t g, int64_t I0, int64_t I1, int bf16, uint16_t* Lq,
                               double* sig, double* tsum, int64_t tstride, int weighted,
                               cudaStream_t s, float* tsum32 = nullptr, float* tabs32 = nullptr);
cudaError_t launch_tmu_mixed(const uint16_t* Lq, int64_t m, int64_t kb, int bf16, double* C,
                             int64_t ldc, int64_t g, int64_t off, const double* sig,
                             const ComputeFault* cf, int ncf, DevStatus* st, cudaStream_t s,
                             int64_t o = 0, int strip = 0, int max_grid = 0);
cudaError_t launch_border_sym(const BorderSymHost& h, const DevStatus* st, cudaStream_t s);

// Solves and iterative refinement (k_solve.cu).
int potrs_max_rhs();
// inv: scratch for the inverses of the diagonal blocks and the sweep's tickets
// and ready flags (potrs_inv_bytes).  have_inv: the inverses of this L (in this
// arithmetic) are already in inv from an earlier call.
cudaError_t launch_potrs_f64(int64_t n, int nrhs, int64_t nb, const double* L, int64_t ldl,
                             double* B, int64_t ldb, double* inv, cudaStream_t s,
                             bool have_inv = false);
// L32 (nullable): the lower triangle of L rounded to FP32, n x n with ld n
// (launch_tril_to_f32); with it the FP32 sweeps stream FP32 tiles.
cudaError_t launch_potrs_f32(int64_t n, int nrhs, int64_t nb, const double* L, int64_t ldl,
                             float* B, int64_t ldb, float* inv, cudaStream_t s,
                             bool have_inv = false, const float* L32 = nullptr);
cudaError_t launch_tril_to_f32(const double* L, int64_t ldl, int64_t n, float* L32,
                               cudaStream_t s);
size_t potrs_inv_bytes(int64_t n, bool f64);
// Nonzero when a wait of the last solve using `inv` gave up (reads one word and
// synchronizes the stream; *ce receives the copy's status).
int potrs_error(const void* inv, int64_t n, bool f64, cudaStream_t s, cudaError_t* ce);
cudaError_t launch_copy_d2f(const double* src, int64_t lds, float* dst, int64_t ldd, int64_t rows,
                            int cols, cudaStream_t s);
cudaError_t launch_copy_d2d(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t rows,
                            int cols, cudaStream_t s);
cudaError_t launch_residual(const double* A, int64_t lda, int64_t n, const double* X, int64_t ldx,
                            const double* B, int64_t ldb, int nrhs, double* R, int64_t ldr,
                            double* P, int nsplit, unsigned long long* rmax,
                            unsigned long long* xmax, cudaStream_t s);
// Y = A X for symmetric A (lower triangle read), X / Y n x 16 (ld 16), split-K
// partials in P (nsplit x n x 16).
cudaError_t launch_symv(const double* A, int64_t lda, int64_t n, const double* X, double* Y,
                        double* P, int nsplit, cudaStream_t s);
// The same product in FP32 arithmetic from an FP32 copy of A (Y in FP64).
cudaError_t launch_symv_f32(const float* A, int64_t lda, int64_t n, const double* X, double* Y,
                            double* P, int nsplit, cudaStream_t s);
cudaError_t launch_inf_norms(const double* A, int64_t lda, int64_t n, const double* B, int64_t ldb,
                             int nrhs, double* rs, unsigned long long* anorm,
                             unsigned long long* bmax, double* scratch, cudaStream_t s);   // scratch: 16 n doubles
cudaError_t launch_eta(const unsigned long long* rmax, const unsigned long long* xmax,
                       const unsigned long long* anorm, const unsigned long long* bmax, int nrhs,
                       double* eta, cudaStream_t s);
cudaError_t launch_add_f32(double* X, int64_t ldx, const float* D, int64_t ldd, int64_t n, int nrhs,
                           cudaStream_t s);
cudaError_t launch_add_f64(double* X, int64_t ldx, const double* D, int64_t ldd, int64_t n,
                           int nrhs, cudaStream_t s);
cudaError_t launch_copy_f2d(const float* src, int64_t lds, double* dst, int64_t ldd, int64_t rows,
                            int cols, cudaStream_t s);

// Adjoint kernels (k_adjoint.cu).
cudaError_t launch_copy_lower(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t n,
                              cudaStream_t s);
cudaError_t launch_phi_neg(double* P, int64_t ld, int64_t kb, cudaStream_t s);
// D (kb x kb, ld kb) = A + A^T for the lower-stored block A (diagonal doubled).
cudaError_t launch_sym_diag(const double* A, int64_t lda, int64_t kb, double* D, cudaStream_t s);
cudaError_t launch_add_tril(const double* P, double* A, int64_t lda, int64_t kb, cudaStream_t s);
cudaError_t launch_transpose(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t kb,
                             cudaStream_t s);
cudaError_t launch_assemble_diag(const double* St, int64_t lds, double* A, int64_t lda, int64_t kb,
                                 cudaStream_t s);
cudaError_t launch_ltx(const double* L, int64_t ldl, int64_t n, const double* X, int64_t ldx,
                       int nrhs, double* U, int64_t ldu, cudaStream_t s);
cudaError_t launch_syr2k_lower(const double* Bb, const double* X, const double* U, const double* V,
                               int64_t ld16, int64_t n, int nrhs, double* Lbar, int64_t ldlb,
                               cudaStream_t s);
cudaError_t launch_logdet(const double* L, int64_t ldl, int64_t n, double* out, cudaStream_t s);
cudaError_t launch_logdet_backward(const double* L, int64_t ldl, int64_t n, double gbar,
                                   double* Lbar, int64_t ldlb, cudaStream_t s);
cudaError_t launch_tril_zero(double* A, int64_t lda, int64_t n, cudaStream_t s);
cudaError_t launch_symmetrize_half(double* A, int64_t lda, int64_t n, cudaStream_t s);

// Batched kernel (k_batched.cu).
size_t batched_scratch_bytes(int grid, bool f64);
int batched_grid(bool f64);       // CTAs of the persistent batched launch
int batched_max_grid(bool f64);   // the most CTAs it can have (workspace sizing)
int batched_set_ctas_per_sm(int c);   // returns the previous setting
cudaError_t batched_prepare();
cudaError_t launch_potrf_batched(const abft_batch_item* items, int count, bool f64, int mode,
                                 double tau_scale, abft_batch_status* status, void* scratch,
                                 unsigned int* queue, cudaStream_t s);

// Kernel launch accounting (every launcher calls note_launch once per kernel).
void note_launch();

// Per-phase GPU time accounting with CUDA events on the launch stream.
enum { PH_PD = 0, PH_PU = 1, PH_TMU = 2, PH_VERIFY = 3, PH_OTHER = 4, PH_SOLVE = 5, PH_COUNT = 6 };
bool timing_on();
void timing_mark(int phase, int begin, cudaStream_t s);
void timing_step(int64_t k);   // iteration index recorded with the next marks (-1: none)
cudaError_t timing_collect(cudaStream_t s);

// FP64-accurate trailing update from BF16 slices (k_emu.cu).  The slice
// tensor holds emu_rows(n, nb) rows: the panel rows, then the checksum rows.
struct EmuRectHost {
    double* C;              // C[i * ldc + j / cdiv] for i < na, j < nb with j % cdiv == 0
    int64_t ldc;
    int64_t a0, na;         // A operand: slice rows a0 .. a0 + na - 1
    int64_t b0, nb;         // B operand: slice rows b0 .. b0 + nb - 1
    int cdiv;
    int64_t frow, fcol;     // trailing coordinates of (0, 0) for compute faults (-1: none)
};
int64_t emu_rows(int64_t n, int64_t nb);
size_t emu_slice_bytes(int64_t n, int64_t nb);
cudaError_t launch_slice_cols(const double* P, int64_t ld, int64_t K, int64_t ncols, uint16_t* S,
                              int64_t Mtot, int64_t row0, int* ex, cudaStream_t s);
// The columns of an mrows x ncols matrix in K-row pieces (zero past mrows):
// piece c at slice rows row0 + c rstride .. + ncols - 1, one scale per column and piece.
cudaError_t launch_slice_cols_chunked(const double* P, int64_t ld, int64_t K, int64_t mrows,
                                      int64_t ncols, uint16_t* S, int64_t Mtot, int64_t row0,
                                      int64_t rstride, int* ex, cudaStream_t s);
cudaError_t launch_slice_panel(const double* P, int64_t lda, int64_t m, int64_t kb, uint16_t* S,
                               int64_t Mtot, int64_t row0, int* ex, cudaStream_t s);
cudaError_t launch_tmu_emu(const uint16_t* S, const int* ex, int64_t mtot, int64_t kb, double* C,
                           int64_t ldc, int64_t M, int64_t o, int64_t g, const EmuRectHost* rects,
                           int nrect, const ComputeFault* cf, int ncf, int max_grid, DevStatus* st,
                           cudaStream_t s);

// FP64-accurate refinement residual on the tensor cores (k_resid_emu.cu).
bool resid_emu_supported(int64_t n);
size_t resid_emu_bytes(int64_t n);
cudaError_t launch_resid_emu_prepare(const double* A, int64_t lda, int64_t n, void* ws,
                                     cudaStream_t s);
// B == nullptr: R = A X (n x 16, ld 16) instead of the residual.
cudaError_t launch_resid_emu(int64_t n, const double* X, int64_t ldx, const double* B, int64_t ldb,
                             int nr, double* R, int64_t ldr, void* ws, unsigned long long* rmax,
                             unsigned long long* xmax, cudaStream_t s);
cudaError_t launch_symv_reduce(const double* P, int nsplit, int64_t n, double* Y, cudaStream_t s);
cudaError_t launch_resid_reduce(const double* P, int nsplit, int64_t n, const double* B,
                                int64_t ldb, const double* X, int64_t ldx, int nrhs, double* R,
                                int64_t ldr, unsigned long long* rmax, unsigned long long* xmax,
                                cudaStream_t s);

// GMRES-IR pieces (k_gmres.cu); vectors are n x 16 blocks (ld 16), basis
// vector i at V + i * vstride.
int gmres_dot_blocks(int64_t n);
cudaError_t launch_gm_dots(const double* V, int64_t vstride, int nv, const double* W, int64_t n,
                           double* part, double* h, int acc, cudaStream_t s);
cudaError_t launch_gm_subtract(const double* V, int64_t vstride, int nv, const double* h,
                               double* W, int64_t n, cudaStream_t s);
cudaError_t launch_gm_scale(const double* x, const double* nrm2, double* out, int64_t n,
                            cudaStream_t s);
cudaError_t launch_gm_rowscale(const double* sc, const double* x, double* y, int64_t n,
                               cudaStream_t s);
cudaError_t launch_gm_givens(double* H, int m, const double* hnew, double* cs, double* sn,
                             double* g, int j, double* res, cudaStream_t s);
cudaError_t launch_gm_init_g(const double* nrm2, double* g, int m, double* res, cudaStream_t s);
cudaError_t launch_gm_update(const double* H, int m, const double* g, int k, double* y,
                             const double* V, int64_t vstride, double* X, int64_t ldx, int nrhs,
                             int64_t n, cudaStream_t s);
cudaError_t launch_gm_diag_scale(const double* A, int64_t lda, int64_t n, double* sc, int on,
                                 cudaStream_t s);
cudaError_t launch_gm_scaled_copy(const double* A, int64_t lda, const double* sc, double delta,
                                  double* L, int64_t ldl, int64_t n, cudaStream_t s);

}  // namespace abft

#define ABFT_CUDA_TRY(expr)                                  \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) return ABFT_ERR_CUDA;         \
    } while (0)
