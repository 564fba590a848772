// k_gmres.cu -- kernels of GMRES-based iterative refinement (Carson and
// Higham's GMRES-IR; not in the paper): the correction equation A d = r is
// solved by GMRES on the left-preconditioned operator M^{-1} A, with
// M = S^{-1} L L^T S^{-1} built from the low-precision Cholesky factor L of
// the scaled and shifted matrix S A S + delta I (S diagonal, powers of two, so
// the scaling is exact).  All vectors are blocks of 16 right-hand sides stored
// row-major (n x 16), and every right-hand side runs its own Arnoldi process
// in lockstep.  Everything here is FP64.  Reductions are two-stage with a
// fixed order, so repeated runs give identical results.
#include <math.h>

#include "common.cuh"

namespace abft {

namespace {

constexpr int NR = 16;          // right-hand sides per block
constexpr int GT = 256;         // threads: 16 row groups x 16 right-hand sides

// part[(i * nblk + b) * 16 + r] = sum over this block's rows p of
// V_i[p][r] * W[p][r], for i = blockIdx.y (V_i = V + i * vstride).
__global__ void __launch_bounds__(GT) k_gm_dots(const double* V, int64_t vstride, const double* W,
                                               int64_t n, int64_t rows_per_blk, double* part) {
    __shared__ double red[GT / NR][NR];
    const int t = threadIdx.x, pg = t >> 4, r = t & 15;
    const int64_t b = blockIdx.x, i = blockIdx.y;
    const double* Vi = V + i * vstride;
    const int64_t p0 = b * rows_per_blk, p1 = (p0 + rows_per_blk < n) ? p0 + rows_per_blk : n;
    double acc = 0.0;
    for (int64_t p = p0 + pg; p < p1; p += GT / NR) acc = fma(Vi[p * NR + r], W[p * NR + r], acc);
    red[pg][r] = acc;
    __syncthreads();
    if (t < NR) {
        double s = 0.0;
        for (int q = 0; q < GT / NR; ++q) s += red[q][t];
        part[(i * gridDim.x + b) * NR + t] = s;
    }
}

// h[i][r] = sum_b part[i][b][r] (block order); acc != 0 adds into h.
__global__ void k_gm_dots_reduce(const double* part, int nblk, int nv, double* h, int acc) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nv * NR) return;
    const int i = e / NR, r = e % NR;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[((int64_t)i * nblk + b) * NR + r];
    h[e] = acc ? h[e] + s : s;
}

// W[p][r] -= sum_{i < nv} V_i[p][r] h[i][r]
__global__ void k_gm_subtract(const double* V, int64_t vstride, int nv, const double* h, double* W,
                              int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * NR) return;
    const int r = (int)(e % NR);
    double w = W[e];
    for (int i = 0; i < nv; ++i) w = fma(-V[i * vstride + e], h[i * NR + r], w);
    W[e] = w;
}

// out = x / nrm[r] (a zero norm gives a zero vector: breakdown is handled by
// the Givens step, which then reports a zero residual for that column)
__global__ void k_gm_scale(const double* x, const double* nrm2, double* out, int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * NR) return;
    const int r = (int)(e % NR);
    const double nr = sqrt(nrm2[r]);
    out[e] = nr > 0.0 ? x[e] / nr : 0.0;
}

// x[p][r] *= s[p] (s = nullptr: identity), optionally into y
__global__ void k_gm_rowscale(const double* s, const double* x, double* y, int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * NR) return;
    y[e] = s ? s[e / NR] * x[e] : x[e];
}

// One Arnoldi column per right-hand side: the new column h (length j + 2,
// h[j + 1] = ||w||^2 on entry, replaced by ||w||) gets the previous Givens
// rotations, a new rotation zeroes h[j + 1], and g (the rotated residual
// vector) advances.  State per right-hand side r: H column-major (m + 1) x m,
// cs / sn (m), g (m + 1).  res[r] = |g[j + 1]|.
__global__ void k_gm_givens(double* H, int m, const double* hnew, double* cs, double* sn,
                            double* g, int j, double* res) {
    const int r = threadIdx.x;
    if (r >= NR) return;
    double* Hc = H + ((int64_t)r * m + j) * (m + 1);
    for (int i = 0; i <= j; ++i) Hc[i] = hnew[i * NR + r];
    Hc[j + 1] = sqrt(hnew[(j + 1) * NR + r]);
    for (int i = 0; i < j; ++i) {
        const double c = cs[r * m + i], s = sn[r * m + i];
        const double a = Hc[i], b = Hc[i + 1];
        Hc[i] = c * a + s * b;
        Hc[i + 1] = -s * a + c * b;
    }
    const double a = Hc[j], b = Hc[j + 1];
    const double d = hypot(a, b);
    const double c = d > 0.0 ? a / d : 1.0, s = d > 0.0 ? b / d : 0.0;
    cs[r * m + j] = c;
    sn[r * m + j] = s;
    Hc[j] = d;
    Hc[j + 1] = 0.0;
    double* gr = g + (int64_t)r * (m + 1);
    const double gj = gr[j];
    gr[j] = c * gj;
    gr[j + 1] = -s * gj;
    res[r] = fabs(gr[j + 1]);
}

// g = (beta_r, 0, ...), beta from ||z0||^2
__global__ void k_gm_init_g(const double* nrm2, double* g, int m, double* res) {
    const int r = threadIdx.x;
    if (r >= NR) return;
    double* gr = g + (int64_t)r * (m + 1);
    for (int i = 0; i <= m; ++i) gr[i] = 0.0;
    gr[0] = sqrt(nrm2[r]);
    res[r] = gr[0];
}

// y = R^{-1} g for the k x k upper triangle R of the rotated H (per r);
// right-hand sides with a zero initial residual get y = 0.
__global__ void k_gm_backsolve(const double* H, int m, const double* g, int k, double* y) {
    const int r = threadIdx.x;
    if (r >= NR) return;
    const double* Hr = H + (int64_t)r * m * (m + 1);
    const double* gr = g + (int64_t)r * (m + 1);
    for (int i = k - 1; i >= 0; --i) {
        double s = gr[i];
        for (int l = i + 1; l < k; ++l) s -= Hr[(int64_t)l * (m + 1) + i] * y[l * NR + r];
        const double d = Hr[(int64_t)i * (m + 1) + i];
        y[i * NR + r] = d != 0.0 ? s / d : 0.0;
    }
}

// X[p][r] += sum_{i < k} V_i[p][r] y[i][r]
__global__ void k_gm_combine(const double* V, int64_t vstride, int k, const double* y, double* X,
                             int64_t ldx, int nrhs, int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * NR) return;
    const int64_t p = e / NR;
    const int r = (int)(e % NR);
    if (r >= nrhs) return;
    double s = 0.0;
    for (int i = 0; i < k; ++i) s = fma(V[i * vstride + e], y[i * NR + r], s);
    X[p * ldx + r] += s;
}

// s_i = 2^(-t_i), t_i = e_i / 2 rounded toward zero, with a_ii = f 2^e_i,
// f in [1/2, 1), so that s_i^2 a_ii lies in [1/4, 2); on = 0, a non-positive
// or a non-finite diagonal give s_i = 1 (the factorization then reports the
// pivot).
__global__ void k_gm_diag_scale(const double* A, int64_t lda, int64_t n, double* s, int on) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double d = A[i * lda + i];
    double v = 1.0;
    if (on && d > 0.0 && isfinite(d)) {
        int e = 0;
        frexp(d, &e);                 // d = f 2^e, f in [0.5, 1)
        v = ldexp(1.0, -(e / 2));
    }
    s[i] = v;
}

// L[i][j] = s_i A[i][j] s_j (+ delta on the diagonal) for j <= i; the upper
// triangle of L is not written (the factorization reads the lower one).
__global__ void k_gm_scaled_copy(const double* A, int64_t lda, const double* s, double delta,
                                 double* L, int64_t ldl, int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int64_t i = e / n, j = e % n;
    if (j > i) return;
    double v = s[i] * A[i * lda + j] * s[j];
    if (i == j) v += delta;
    L[i * ldl + j] = v;
}

unsigned nb_blocks(int64_t tot) { return (unsigned)((tot + 255) / 256); }

}  // namespace

int gmres_dot_blocks(int64_t n) {
    int64_t b = (n + 127) / 128;
    return (int)(b < 296 ? (b > 0 ? b : 1) : 296);
}

cudaError_t launch_gm_dots(const double* V, int64_t vstride, int nv, const double* W, int64_t n,
                           double* part, double* h, int acc, cudaStream_t s) {
    if (nv <= 0) return cudaSuccess;
    const int nblk = gmres_dot_blocks(n);
    const int64_t rpb = (n + nblk - 1) / nblk;
    k_gm_dots<<<dim3((unsigned)nblk, (unsigned)nv), GT, 0, s>>>(V, vstride, W, n, rpb, part);
    note_launch();
    k_gm_dots_reduce<<<nb_blocks((int64_t)nv * NR), 256, 0, s>>>(part, nblk, nv, h, acc);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gm_subtract(const double* V, int64_t vstride, int nv, const double* h,
                               double* W, int64_t n, cudaStream_t s) {
    if (nv <= 0) return cudaSuccess;
    k_gm_subtract<<<nb_blocks(n * NR), 256, 0, s>>>(V, vstride, nv, h, W, n);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gm_scale(const double* x, const double* nrm2, double* out, int64_t n,
                            cudaStream_t s) {
    k_gm_scale<<<nb_blocks(n * NR), 256, 0, s>>>(x, nrm2, out, n);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gm_rowscale(const double* sc, const double* x, double* y, int64_t n,
                               cudaStream_t s) {
    k_gm_rowscale<<<nb_blocks(n * NR), 256, 0, s>>>(sc, x, y, n);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gm_givens(double* H, int m, const double* hnew, double* cs, double* sn,
                             double* g, int j, double* res, cudaStream_t s) {
    k_gm_givens<<<1, 32, 0, s>>>(H, m, hnew, cs, sn, g, j, res);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gm_init_g(const double* nrm2, double* g, int m, double* res, cudaStream_t s) {
    k_gm_init_g<<<1, 32, 0, s>>>(nrm2, g, m, res);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gm_update(const double* H, int m, const double* g, int k, double* y,
                             const double* V, int64_t vstride, double* X, int64_t ldx, int nrhs,
                             int64_t n, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    k_gm_backsolve<<<1, 32, 0, s>>>(H, m, g, k, y);
    note_launch();
    k_gm_combine<<<nb_blocks(n * NR), 256, 0, s>>>(V, vstride, k, y, X, ldx, nrhs, n);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gm_diag_scale(const double* A, int64_t lda, int64_t n, double* sc, int on,
                                 cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_gm_diag_scale<<<nb_blocks(n), 256, 0, s>>>(A, lda, n, sc, on);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gm_scaled_copy(const double* A, int64_t lda, const double* sc, double delta,
                                  double* L, int64_t ldl, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_gm_scaled_copy<<<nb_blocks(n * n), 256, 0, s>>>(A, lda, sc, delta, L, ldl, n);
    note_launch();
    return cudaGetLastError();
}

}  // namespace abft
