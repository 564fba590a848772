// k_solve.cu -- triangular solves with a Cholesky factor (potrs) and the
// pieces of iterative refinement: the FP64 residual R = B - A X, the
// normwise backward error, and X += D.
//
// potrs runs block by block: a one-CTA solve of the nb x nb diagonal block
// (32-row chunks: an update from the solved rows by all threads, then a short
// substitution inside the chunk), and a many-CTA update of the remaining rows
// with the just-solved block.  T is the arithmetic type (double for the FP64
// solve, float for the correction solves of iterative refinement); L is read
// in FP64 and converted on load.
#include <math.h>

#include "common.cuh"

namespace abft {

namespace {

constexpr int MAXRHS = 16;

// Inverses of the 32 x 32 diagonal chunks of L (lower), one warp per chunk:
// lane j computes column j of the inverse by substitution with the chunk in
// shared memory.  Used by the diagonal-block solves below.
template <typename T>
__global__ void __launch_bounds__(32) k_chunk_inv(const double* L, int64_t ldl, int64_t n, T* Inv) {
    __shared__ T Lc[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32;
    const int w = (int)((n - c0) < 32 ? (n - c0) : 32);
    const int lane = threadIdx.x;
    for (int i = 0; i < 32; ++i)
        Lc[i][lane] = (i < w && lane <= i) ? (T)L[(c0 + i) * ldl + c0 + lane] : (T)0;
    __syncwarp();
    T x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        T v = (i == lane) ? (T)1 : (T)0;
#pragma unroll
        for (int p = 0; p < i; ++p) v -= Lc[i][p] * x[p];
        x[i] = (i < w) ? v / Lc[i][i] : (T)0;
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) Inv[(c0 + i) * 32 + lane] = (i < w && lane < w) ? x[i] : (T)0;
}

// Solve the kb x kb diagonal block in place: L Y = Y (TRANS = 0) or
// L^T X = X (TRANS = 1) for nrhs <= 16 right-hand sides (Y row-major, ld ldy).
// 32-row chunks: the chunk is updated from the already solved rows, then
// multiplied by its precomputed inverse (Inv: the block's chunks, 32 x 32 each).
template <typename T, int TRANS>
__global__ void __launch_bounds__(512) k_trsv_diag(const double* L, int64_t ldl, int kb, T* Y,
                                                   int64_t ldy, int nrhs, const T* Inv) {
    extern __shared__ __align__(16) unsigned char sb[];
    T* y = (T*)sb;                        // kb x MAXRHS
    T* Lr = y + (size_t)kb * MAXRHS;      // 32 x (kb + 1): the chunk's rows (or columns) of L
    const int ldr = kb + 1;
    __shared__ T Ic[32][33];
    __shared__ T tmp[32][MAXRHS];
    const int t = threadIdx.x;
    for (int e = t; e < kb * nrhs; e += blockDim.x) {
        int i = e / nrhs, r = e % nrhs;
        y[i * MAXRHS + r] = Y[(int64_t)i * ldy + r];
    }
    __syncthreads();
    const int nch = (kb + 31) / 32;
    const int q = t >> 4, r = t & 15;     // this thread's (row in chunk, rhs)
    for (int ci = 0; ci < nch; ++ci) {
        const int c = TRANS ? nch - 1 - ci : ci;
        const int c0 = c * 32, c1 = (c0 + 32 < kb) ? c0 + 32 : kb, w = c1 - c0;
        // the chunk's inverse (transposed for the backward solve)
        for (int e = t; e < 32 * 32; e += blockDim.x) {
            int a = e >> 5, b = e & 31;
            Ic[a][b] = TRANS ? Inv[(int64_t)(c0 + b) * 32 + a] : Inv[(int64_t)(c0 + a) * 32 + b];
        }
        // stage the part of L that couples the chunk to the solved rows in one
        // coalesced pass: rows c0..c1 x cols 0..c0 (forward), or rows c1..kb x
        // cols c0..c1 stored transposed (backward)
        if (!TRANS) {
            for (int e = t; e < w * c0; e += blockDim.x) {
                int a = e / c0, b = e % c0;
                Lr[a * ldr + b] = (T)L[(int64_t)(c0 + a) * ldl + b];
            }
        } else {
            const int h = kb - c1;
            for (int e = t; e < h * 32; e += blockDim.x) {
                int b = e >> 5, a = e & 31;
                if (a < w) Lr[a * ldr + b] = (T)L[(int64_t)(c1 + b) * ldl + c0 + a];
            }
        }
        __syncthreads();
        // update the chunk from the solved rows
        if (q < w && r < nrhs) {
            const int i = c0 + q;
            T acc = 0;
            if (!TRANS) {
                for (int p = 0; p < c0; ++p) acc += Lr[q * ldr + p] * y[p * MAXRHS + r];
            } else {
                for (int p = c1; p < kb; ++p) acc += Lr[q * ldr + (p - c1)] * y[p * MAXRHS + r];
            }
            tmp[q][r] = y[i * MAXRHS + r] - acc;
        }
        __syncthreads();
        if (q < w && r < nrhs) {
            T v = 0;
            for (int p = 0; p < w; ++p) v += Ic[q][p] * tmp[p][r];
            y[(c0 + q) * MAXRHS + r] = v;
        }
        __syncthreads();
    }
    for (int e = t; e < kb * nrhs; e += blockDim.x) {
        int i = e / nrhs, rr = e % nrhs;
        Y[(int64_t)i * ldy + rr] = y[i * MAXRHS + rr];
    }
}

// Rows update with a solved block: Y[i][r] -= sum_p Lop[i][p] Ys[p][r], i < M,
// p < K; Lop[i][p] = L[i][p] (TRANS = 0) or L[p][i] (TRANS = 1).
template <typename T, int TRANS>
__global__ void __launch_bounds__(256) k_trsv_update(const double* L, int64_t ldl, int64_t M,
                                                     int K, const T* Ys, int64_t ldys, T* Y,
                                                     int64_t ldy, int nrhs) {
    __shared__ T As[64][65];
    __shared__ T Bs[64][MAXRHS];
    const int t = threadIdx.x;
    const int64_t i0 = blockIdx.x * 64;
    const int row = t & 63, cg = t >> 6;   // 4 column groups
    T acc[4] = {0, 0, 0, 0};
    for (int k0 = 0; k0 < K; k0 += 64) {
        for (int e = t; e < 64 * 64; e += 256) {
            int a = e >> 6, b = e & 63;   // coalesced along b
            if (!TRANS) {   // As[p][i] = L[i0+a][k0+b] stored as As[b][a]
                int64_t i = i0 + a; int p = k0 + b;
                As[b][a] = (i < M && p < K) ? (T)L[i * ldl + p] : (T)0;
            } else {        // As[p][i] = L[k0+a][i0+b]
                int p = k0 + a; int64_t i = i0 + b;
                As[a][b] = (i < M && p < K) ? (T)L[(int64_t)p * ldl + i] : (T)0;
            }
        }
        for (int e = t; e < 64 * MAXRHS; e += 256) {
            int p = e / MAXRHS, r = e % MAXRHS;
            Bs[p][r] = (k0 + p < K && r < nrhs) ? Ys[(int64_t)(k0 + p) * ldys + r] : (T)0;
        }
        __syncthreads();
#pragma unroll 8
        for (int p = 0; p < 64; ++p) {
            T a = As[p][row];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] += a * Bs[p][cg + 4 * u];
        }
        __syncthreads();
    }
    const int64_t i = i0 + row;
    if (i < M)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int r = cg + 4 * u;
            if (r < nrhs) Y[i * ldy + r] -= acc[u];
        }
}

template <typename S, typename D>
__global__ void k_copy2d(const S* src, int64_t lds, D* dst, int64_t ldd, int64_t rows, int cols) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * cols) return;
    int64_t i = e / cols;
    int j = (int)(e % cols);
    dst[i * ldd + j] = (D)src[i * lds + j];
}

// Split-K partial products of the residual: P[s][i][r] = sum_{p in chunk s} A[i][p] X[p][r].
__global__ void __launch_bounds__(256) k_resid_partial(const double* A, int64_t lda, int64_t n,
                                                       const double* X, int64_t ldx, int nrhs,
                                                       int64_t kchunk, double* P) {
    __shared__ double As[32][65];
    __shared__ double Xs[32][MAXRHS];
    const int t = threadIdx.x;
    const int64_t i0 = blockIdx.x * 64;
    const int64_t kbeg = blockIdx.y * kchunk;
    const int64_t kend = (kbeg + kchunk < n) ? kbeg + kchunk : n;
    const int row = t & 63, cg = t >> 6;
    double acc[4] = {0, 0, 0, 0};
    for (int64_t k0 = kbeg; k0 < kend; k0 += 32) {
        // A is symmetric and only its lower triangle is read: A[i][p] for p <= i,
        // A[p][i] above; whole tiles on one side load coalesced.
        if (k0 + 31 <= i0) {
            for (int e = t; e < 64 * 32; e += 256) {
                int a = e >> 5, b = e & 31;
                int64_t i = i0 + a, p = k0 + b;
                As[b][a] = (i < n && p < kend) ? A[i * lda + p] : 0.0;
            }
        } else if (k0 >= i0 + 64) {
            for (int e = t; e < 64 * 32; e += 256) {
                int b = e >> 6, a = e & 63;
                int64_t i = i0 + a, p = k0 + b;
                As[b][a] = (i < n && p < kend) ? A[p * lda + i] : 0.0;
            }
        } else {
            for (int e = t; e < 64 * 32; e += 256) {
                int a = e >> 5, b = e & 31;
                int64_t i = i0 + a, p = k0 + b;
                As[b][a] = (i < n && p < kend) ? (p <= i ? A[i * lda + p] : A[p * lda + i]) : 0.0;
            }
        }
        for (int e = t; e < 32 * MAXRHS; e += 256) {
            int p = e / MAXRHS, r = e % MAXRHS;
            Xs[p][r] = (k0 + p < kend && r < nrhs) ? X[(k0 + p) * ldx + r] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int p = 0; p < 32; ++p) {
            double a = As[p][row];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fma(a, Xs[p][cg + 4 * u], acc[u]);
        }
        __syncthreads();
    }
    const int64_t i = i0 + row;
    if (i < n)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int r = cg + 4 * u;
            if (r < nrhs) P[((int64_t)blockIdx.y * n + i) * MAXRHS + r] = acc[u];
        }
}

// R = B - sum_s P[s] (fixed order) and the per-column max |R|, max |X|.
__global__ void k_resid_reduce(const double* P, int nsplit, int64_t n, const double* B,
                               int64_t ldb, const double* X, int64_t ldx, int nrhs, double* R,
                               int64_t ldr, unsigned long long* rmax, unsigned long long* xmax) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * nrhs) return;
    int64_t i = e / nrhs;
    int r = (int)(e % nrhs);
    double s = 0.0;
    for (int k = 0; k < nsplit; ++k) s += P[((int64_t)k * n + i) * MAXRHS + r];
    double v = B[i * ldb + r] - s;
    R[i * ldr + r] = v;
    atomic_max_nonneg(&rmax[r], fabs(v));
    atomic_max_nonneg(&xmax[r], fabs(X[i * ldx + r]));
}

// Row sums of |A| for symmetric A read from its lower triangle: the part
// j <= i of row i (one warp per row) plus the strict column part i > j of
// column i (one thread per column); both passes are coalesced.
__global__ void k_abs_rowsum_lower(const double* A, int64_t lda, int64_t n, double* rs) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    double s = 0.0;
    for (int64_t j = lane; j <= i; j += 32) s += fabs(A[i * lda + j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) rs[i] = s;
}

__global__ void k_abs_colsum_strict(const double* A, int64_t lda, int64_t n, const double* rs,
                                    const double* B, int64_t ldb, int nrhs,
                                    unsigned long long* anorm, unsigned long long* bmax) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s = rs[j];
    for (int64_t i = j + 1; i < n; ++i) s += fabs(A[i * lda + j]);
    atomic_max_nonneg(anorm, s);
    for (int r = 0; r < nrhs; ++r) atomic_max_nonneg(&bmax[r], fabs(B[j * ldb + r]));
}

// eta = max_r ||R_r||_inf / (||A||_inf ||X_r||_inf + ||B_r||_inf)
__global__ void k_eta(const unsigned long long* rmax, const unsigned long long* xmax,
                      const unsigned long long* anorm, const unsigned long long* bmax, int nrhs,
                      double* eta) {
    double a = __longlong_as_double((long long)*anorm), m = 0.0;
    for (int r = 0; r < nrhs; ++r) {
        double rr = __longlong_as_double((long long)rmax[r]);
        double xx = __longlong_as_double((long long)xmax[r]);
        double bb = __longlong_as_double((long long)bmax[r]);
        double d = a * xx + bb;
        double e = d > 0.0 ? rr / d : (rr > 0.0 ? INFINITY : 0.0);
        m = fmax(m, e);
    }
    *eta = m;
}

template <typename T>
__global__ void k_add(double* X, int64_t ldx, const T* D, int64_t ldd, int64_t n, int nrhs) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * nrhs) return;
    int64_t i = e / nrhs;
    int r = (int)(e % nrhs);
    X[i * ldx + r] += (double)D[i * ldd + r];
}

template <typename T>
cudaError_t set_attrs() {
    static bool done = false;
    if (done) return cudaSuccess;
    const int bytes = (512 * MAXRHS + 32 * 513) * (int)sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(k_trsv_diag<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_trsv_diag<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bytes);
    if (e == cudaSuccess) done = true;
    return e;
}

template <typename T>
cudaError_t potrs_t(int64_t n, int nrhs, int64_t nb, const double* L, int64_t ldl, T* Y,
                    int64_t ldy, T* Inv, cudaStream_t s) {
    cudaError_t e = set_attrs<T>();
    if (e != cudaSuccess) return e;
    const int64_t N = (n + nb - 1) / nb;
    const size_t smem = (size_t)(nb * MAXRHS + 32 * (nb + 1)) * sizeof(T);
    k_chunk_inv<T><<<(unsigned)((n + 31) / 32), 32, 0, s>>>(L, ldl, n, Inv);
    note_launch();
    for (int64_t k = 0; k < N; ++k) {   // L Y = B
        const int64_t K0 = k * nb, kb = (K0 + nb < n) ? nb : n - K0, T0 = K0 + kb;
        k_trsv_diag<T, 0><<<1, 512, smem, s>>>(L + K0 * ldl + K0, ldl, (int)kb, Y + K0 * ldy, ldy,
                                               nrhs, Inv + K0 * 32);
        note_launch();
        if (T0 < n) {
            k_trsv_update<T, 0><<<(unsigned)((n - T0 + 63) / 64), 256, 0, s>>>(
                L + T0 * ldl + K0, ldl, n - T0, (int)kb, Y + K0 * ldy, ldy, Y + T0 * ldy, ldy, nrhs);
            note_launch();
        }
    }
    for (int64_t k = N - 1; k >= 0; --k) {   // L^T X = Y
        const int64_t K0 = k * nb, kb = (K0 + nb < n) ? nb : n - K0;
        k_trsv_diag<T, 1><<<1, 512, smem, s>>>(L + K0 * ldl + K0, ldl, (int)kb, Y + K0 * ldy, ldy,
                                               nrhs, Inv + K0 * 32);
        note_launch();
        if (K0 > 0) {
            k_trsv_update<T, 1><<<(unsigned)((K0 + 63) / 64), 256, 0, s>>>(
                L + K0 * ldl, ldl, K0, (int)kb, Y + K0 * ldy, ldy, Y, ldy, nrhs);
            note_launch();
        }
    }
    return cudaGetLastError();
}

}  // namespace

int potrs_max_rhs() { return MAXRHS; }

cudaError_t launch_potrs_f64(int64_t n, int nrhs, int64_t nb, const double* L, int64_t ldl,
                             double* B, int64_t ldb, double* inv, cudaStream_t s) {
    return potrs_t<double>(n, nrhs, nb, L, ldl, B, ldb, inv, s);
}

cudaError_t launch_potrs_f32(int64_t n, int nrhs, int64_t nb, const double* L, int64_t ldl,
                             float* B, int64_t ldb, float* inv, cudaStream_t s) {
    return potrs_t<float>(n, nrhs, nb, L, ldl, B, ldb, inv, s);
}

size_t potrs_inv_bytes(int64_t n, bool f64) {
    return (size_t)((n + 31) / 32) * 32 * 32 * (f64 ? sizeof(double) : sizeof(float));
}

cudaError_t launch_copy_d2f(const double* src, int64_t lds, float* dst, int64_t ldd, int64_t rows,
                            int cols, cudaStream_t s) {
    int64_t tot = rows * cols;
    if (tot <= 0) return cudaSuccess;
    k_copy2d<double, float><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, lds, dst, ldd, rows, cols);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_copy_d2d(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t rows,
                            int cols, cudaStream_t s) {
    int64_t tot = rows * cols;
    if (tot <= 0) return cudaSuccess;
    k_copy2d<double, double><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, lds, dst, ldd, rows, cols);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_residual(const double* A, int64_t lda, int64_t n, const double* X, int64_t ldx,
                            const double* B, int64_t ldb, int nrhs, double* R, int64_t ldr,
                            double* P, int nsplit, unsigned long long* rmax,
                            unsigned long long* xmax, cudaStream_t s) {
    const int64_t kchunk = ((n + nsplit - 1) / nsplit + 31) / 32 * 32;
    dim3 grid((unsigned)((n + 63) / 64), (unsigned)nsplit);
    k_resid_partial<<<grid, 256, 0, s>>>(A, lda, n, X, ldx, nrhs, kchunk, P);
    note_launch();
    int64_t tot = n * nrhs;
    k_resid_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(P, nsplit, n, B, ldb, X, ldx, nrhs,
                                                                 R, ldr, rmax, xmax);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_inf_norms(const double* A, int64_t lda, int64_t n, const double* B, int64_t ldb,
                             int nrhs, double* rs, unsigned long long* anorm,
                             unsigned long long* bmax, cudaStream_t s) {
    k_abs_rowsum_lower<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(A, lda, n, rs);
    note_launch();
    k_abs_colsum_strict<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(A, lda, n, rs, B, ldb, nrhs,
                                                                   anorm, bmax);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_eta(const unsigned long long* rmax, const unsigned long long* xmax,
                       const unsigned long long* anorm, const unsigned long long* bmax, int nrhs,
                       double* eta, cudaStream_t s) {
    k_eta<<<1, 1, 0, s>>>(rmax, xmax, anorm, bmax, nrhs, eta);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_add_f64(double* X, int64_t ldx, const double* D, int64_t ldd, int64_t n,
                           int nrhs, cudaStream_t s) {
    int64_t tot = n * nrhs;
    if (tot <= 0) return cudaSuccess;
    k_add<double><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, ldx, D, ldd, n, nrhs);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_copy_f2d(const float* src, int64_t lds, double* dst, int64_t ldd, int64_t rows,
                            int cols, cudaStream_t s) {
    int64_t tot = rows * cols;
    if (tot <= 0) return cudaSuccess;
    k_copy2d<float, double><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, lds, dst, ldd, rows, cols);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_add_f32(double* X, int64_t ldx, const float* D, int64_t ldd, int64_t n, int nrhs,
                           cudaStream_t s) {
    int64_t tot = n * nrhs;
    if (tot <= 0) return cudaSuccess;
    k_add<float><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, ldx, D, ldd, n, nrhs);
    note_launch();
    return cudaGetLastError();
}

}  // namespace abft
