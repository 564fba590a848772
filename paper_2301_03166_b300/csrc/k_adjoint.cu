// k_adjoint.cu -- small kernels of the Cholesky adjoint (reverse mode of
// potrf, potrs and logdet).  The heavy parts of the blocked reverse sweep
// reuse the FP64 tile GEMM (symmetric operand, split-K) and the panel solve.
//
// Convention: a function of a symmetric A that reads only its lower triangle
// has the lower-triangular adjoint Abar_L (d f = sum_{i >= j} Abar_L[i][j]
// dA[i][j]); its symmetric gradient is (Abar_L + Abar_L^T) / 2.
#include <math.h>

#include "common.cuh"

namespace abft {

namespace {

// dst = tril(src), zero above the diagonal.
__global__ void k_copy_lower(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int64_t i = e / n, j = e % n;
    dst[i * ldd + j] = (j <= i) ? src[i * lds + j] : 0.0;
}

// P holds -(L11^T Lbar11); replace it by Phi(L11^T Lbar11): lower triangle,
// diagonal halved, zero above.
__global__ void k_phi_neg(double* P, int64_t ld, int kb) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kb * kb) return;
    const int i = e / kb, j = e % kb;
    double v = -P[(int64_t)i * ld + j];
    P[(int64_t)i * ld + j] = (j < i) ? v : (j == i ? 0.5 * v : 0.0);
}

__global__ void k_transpose(const double* src, int64_t lds, double* dst, int64_t ldd, int kb) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kb * kb) return;
    const int i = e / kb, j = e % kb;
    dst[(int64_t)j * ldd + i] = src[(int64_t)i * lds + j];
}

// Abar11 = Phi(S + S^T) from St = S^T: lower triangle (S + S^T)_ij, the
// diagonal halved, zero above.
__global__ void k_assemble_diag(const double* St, int64_t lds, double* A, int64_t lda, int kb) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kb * kb) return;
    const int i = e / kb, j = e % kb;
    double v = 0.0;
    if (j <= i) {
        v = St[(int64_t)i * lds + j] + St[(int64_t)j * lds + i];
        if (i == j) v *= 0.5;
    }
    A[(int64_t)i * lda + j] = v;
}

// D = A + A^T of a lower-stored kb x kb block A (the diagonal doubled): the
// diagonal block of F = Abar_L + Abar_L^T, in full, for the FP64-accurate sweep.
__global__ void k_sym_diag(const double* A, int64_t lda, int kb, double* D) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kb * kb) return;
    const int i = e / kb, j = e % kb;
    D[e] = i > j ? A[(int64_t)i * lda + j] : (i < j ? A[(int64_t)j * lda + i] : 2.0 * A[(int64_t)i * lda + i]);
}

// A += tril(P) for a kb x kb block (P dense, ld kb).
__global__ void k_add_tril(const double* P, double* A, int64_t lda, int kb) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kb * kb) return;
    const int i = e / kb, j = e % kb;
    if (j <= i) A[(int64_t)i * lda + j] += P[e];
}

// U = L^T X for lower L (only p >= i of column i used): U[i][r] = sum_{p >= i} L[p][i] X[p][r].
__global__ void __launch_bounds__(256) k_ltx(const double* L, int64_t ldl, int64_t n,
                                             const double* X, int64_t ldx, int nrhs, double* U,
                                             int64_t ldu) {
    __shared__ double As[32][65];
    __shared__ double Xs[32][16];
    const int t = threadIdx.x;
    const int64_t i0 = blockIdx.x * 64;
    const int row = t & 63, cg = t >> 6;
    double acc[4] = {0, 0, 0, 0};
    for (int64_t k0 = (i0 / 32) * 32; k0 < n; k0 += 32) {
        for (int e = t; e < 32 * 64; e += 256) {
            int b = e >> 6, a = e & 63;     // coalesced along a (= i)
            int64_t p = k0 + b, i = i0 + a;
            As[b][a] = (p < n && i < n && p >= i) ? L[p * ldl + i] : 0.0;
        }
        for (int e = t; e < 32 * 16; e += 256) {
            int b = e >> 4, r = e & 15;
            Xs[b][r] = (k0 + b < n && r < nrhs) ? X[(k0 + b) * ldx + r] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int b = 0; b < 32; ++b) {
            double a = As[b][row];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fma(a, Xs[b][cg + 4 * u], acc[u]);
        }
        __syncthreads();
    }
    const int64_t i = i0 + row;
    if (i < n)
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (cg + 4 * u < nrhs) U[i * ldu + cg + 4 * u] = acc[u];
}

// Lbar[i][j] -= sum_r (Bb[i][r] U[j][r] + X[i][r] V[j][r]) for j <= i
// (the lower part of (Bb X^T + X Bb^T) L with U = L^T X, V = L^T Bb).
__global__ void __launch_bounds__(256) k_syr2k_lower(const double* Bb, const double* X,
                                                     const double* U, const double* V,
                                                     int64_t ld16, int64_t n, int nrhs,
                                                     double* Lbar, int64_t ldlb) {
    __shared__ double sB[64][17], sX[64][17], sU[64][17], sV[64][17];
    const int64_t i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
    if (j0 > i0 + 63) return;
    const int t = threadIdx.x;
    for (int e = t; e < 64 * 16; e += 256) {
        int a = e >> 4, r = e & 15;
        int64_t i = i0 + a, j = j0 + a;
        bool ri = i < n && r < nrhs, rj = j < n && r < nrhs;
        sB[a][r] = ri ? Bb[i * ld16 + r] : 0.0;
        sX[a][r] = ri ? X[i * ld16 + r] : 0.0;
        sU[a][r] = rj ? U[j * ld16 + r] : 0.0;
        sV[a][r] = rj ? V[j * ld16 + r] : 0.0;
    }
    __syncthreads();
    const int tx = t & 15, ty = t >> 4;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int li = ty + 16 * a, lj = tx + 16 * b;
            const int64_t i = i0 + li, j = j0 + lj;
            if (i >= n || j >= n || j > i) continue;
            double s = 0.0;
            for (int r = 0; r < nrhs; ++r) s += sB[li][r] * sU[lj][r] + sX[li][r] * sV[lj][r];
            Lbar[i * ldlb + j] -= s;
        }
}

// out = 2 sum_i log L[i][i] (one CTA, fixed reduction order).
__global__ void k_logdet(const double* L, int64_t ldl, int64_t n, double* out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += log(L[i * ldl + i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *out = 2.0 * t;
    }
}

__global__ void k_logdet_backward(const double* L, int64_t ldl, int64_t n, double gbar,
                                  double* Lbar, int64_t ldlb) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) Lbar[i * ldlb + i] += 2.0 * gbar / L[i * ldl + i];
}

// Symmetric gradient from the lower-triangle adjoint: G = (Abar + Abar^T) / 2.
__global__ void k_symmetrize_half(double* A, int64_t lda, int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int64_t i = e / n, j = e % n;
    if (j < i) {
        const double v = 0.5 * A[i * lda + j];
        A[i * lda + j] = v;
        A[j * lda + i] = v;
    }
}

__global__ void k_tril_zero(double* A, int64_t lda, int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int64_t i = e / n, j = e % n;
    if (j > i) A[i * lda + j] = 0.0;
}

unsigned blocks_for(int64_t tot) { return (unsigned)((tot + 255) / 256); }

}  // namespace

cudaError_t launch_copy_lower(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t n,
                              cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_copy_lower<<<blocks_for(n * n), 256, 0, s>>>(src, lds, dst, ldd, n);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_add_tril(const double* P, double* A, int64_t lda, int64_t kb, cudaStream_t s) {
    if (kb <= 0) return cudaSuccess;
    k_add_tril<<<blocks_for(kb * kb), 256, 0, s>>>(P, A, lda, (int)kb);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_sym_diag(const double* A, int64_t lda, int64_t kb, double* D, cudaStream_t s) {
    if (kb <= 0) return cudaSuccess;
    k_sym_diag<<<blocks_for(kb * kb), 256, 0, s>>>(A, lda, (int)kb, D);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_phi_neg(double* P, int64_t ld, int64_t kb, cudaStream_t s) {
    k_phi_neg<<<blocks_for(kb * kb), 256, 0, s>>>(P, ld, (int)kb);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_transpose(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t kb,
                             cudaStream_t s) {
    k_transpose<<<blocks_for(kb * kb), 256, 0, s>>>(src, lds, dst, ldd, (int)kb);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_assemble_diag(const double* St, int64_t lds, double* A, int64_t lda, int64_t kb,
                                 cudaStream_t s) {
    k_assemble_diag<<<blocks_for(kb * kb), 256, 0, s>>>(St, lds, A, lda, (int)kb);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_ltx(const double* L, int64_t ldl, int64_t n, const double* X, int64_t ldx,
                       int nrhs, double* U, int64_t ldu, cudaStream_t s) {
    k_ltx<<<(unsigned)((n + 63) / 64), 256, 0, s>>>(L, ldl, n, X, ldx, nrhs, U, ldu);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_syr2k_lower(const double* Bb, const double* X, const double* U, const double* V,
                               int64_t ld16, int64_t n, int nrhs, double* Lbar, int64_t ldlb,
                               cudaStream_t s) {
    const unsigned tiles = (unsigned)((n + 63) / 64);
    k_syr2k_lower<<<dim3(tiles, tiles), 256, 0, s>>>(Bb, X, U, V, ld16, n, nrhs, Lbar, ldlb);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_logdet(const double* L, int64_t ldl, int64_t n, double* out, cudaStream_t s) {
    k_logdet<<<1, 1024, 0, s>>>(L, ldl, n, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_logdet_backward(const double* L, int64_t ldl, int64_t n, double gbar,
                                   double* Lbar, int64_t ldlb, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_logdet_backward<<<blocks_for(n), 256, 0, s>>>(L, ldl, n, gbar, Lbar, ldlb);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_symmetrize_half(double* A, int64_t lda, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_symmetrize_half<<<blocks_for(n * n), 256, 0, s>>>(A, lda, n);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_tril_zero(double* A, int64_t lda, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_tril_zero<<<blocks_for(n * n), 256, 0, s>>>(A, lda, n);
    note_launch();
    return cudaGetLastError();
}

}  // namespace abft
