// k_solve.cu -- triangular solves with a Cholesky factor (potrs) and the
// pieces of iterative refinement: the FP64 residual R = B - A X, the
// normwise backward error, and X += D.
//
// potrs is two launches of a persistent sweep kernel (forward with L, backward
// with L^T), each covering all 64-row blocks with flag-ordered block solves.
// T is the arithmetic type (double for the FP64 solve, float for the
// correction solves of iterative refinement); L is read in FP64 and converted
// on load.
#include <math.h>

#include <algorithm>

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

// One triangular sweep in a single launch: L Y = Y (TRANS = 0) or L^T X = X
// (TRANS = 1) for nrhs <= 16 right-hand sides, Y row-major (ld ldy), solved in
// place.  Rows are cut into 64-row blocks.  CTAs take blocks from a ticket
// counter in solve order (first to last for L, last to first for L^T); the CTA
// of block i streams the 64 x 64 tiles of L that couple it to the blocks solved
// before it, waiting on each block's ready flag, then solves its diagonal block
// with the precomputed 32 x 32 chunk inverses and publishes its rows and flag.
// A CTA only waits on blocks whose tickets were handed out before its own, so
// the sweep completes whatever the number of resident CTAs.  Every wait gives
// up after one second: it sets sync[2] and the remaining CTAs drain.
// sync: [0] / [1] tickets (L, L^T), [2] error, [4, 4 + NB) flags of the L
// sweep, [4 + NB, 4 + 2 NB) flags of the L^T sweep; zeroed before the solve.
constexpr int RB = 64;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename T>
size_t sweep_smem_bytes() {
    return sizeof(T) * ((size_t)RB * (RB + 1) + 2 * (size_t)RB * MAXRHS + 2 * 32 * 33);
}

template <typename T, int TRANS>
__global__ void __launch_bounds__(256, 2) k_trsv_sweep(const double* __restrict__ L, int64_t ldl,
                                                    int64_t n, T* Y, int64_t ldy, int nrhs,
                                                    const T* __restrict__ Inv, unsigned* sync) {
    extern __shared__ __align__(16) unsigned char sb[];
    T* sA = (T*)sb;                         // tile of L^T (or L): sA[p * (RB + 1) + a]
    T* sY = sA + RB * (RB + 1);             // solved rows of the tile / rhs of the diagonal
    T* sX = sY + RB * MAXRHS;               // solution of the diagonal block
    T* sI = sX + RB * MAXRHS;               // two 32 x 32 chunk inverses, ld 33
    __shared__ int s_blk, s_ok, s_known;
    const int NB = (int)((n + RB - 1) / RB);
    const int nchunk = (int)((n + 31) / 32);
    unsigned* ticket = sync + TRANS;
    unsigned* err = sync + 2;
    unsigned* flag = sync + 4 + (TRANS ? NB : 0);
    const int t = threadIdx.x, row = t & 63, cg = t >> 6;
    for (;;) {
        if (t == 0) {
            const unsigned tk = atomicAdd(ticket, 1u);
            const bool live = *(volatile unsigned*)err == 0u;
            s_blk = (live && tk < (unsigned)NB) ? (TRANS ? NB - 1 - (int)tk : (int)tk) : -1;
        }
        __syncthreads();
        const int bi = s_blk;
        if (bi < 0) return;
        const int64_t i0 = (int64_t)bi * RB;
        const int nj = TRANS ? NB - 1 - bi : bi;     // coupling tiles, in solve order
        auto jblk = [&](int k) { return TRANS ? NB - 1 - k : k; };
        // this thread's 16 elements of tile (bi, jb) of the operator (jb == bi: diagonal)
        auto load_tile = [&](int jb, double (&v)[16]) {
            const int64_t j0 = (int64_t)jb * RB;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int e = t + 256 * q, a = e >> 6, b = e & 63;
                const int64_t gr = TRANS ? j0 + a : i0 + a, gc = TRANS ? i0 + b : j0 + b;
                v[q] = (gr < n && gc < n) ? L[gr * ldl + gc] : 0.0;
            }
        };
        auto store_tile = [&](const double (&v)[16]) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int e = t + 256 * q, a = e >> 6, b = e & 63;
                if (TRANS) sA[a * (RB + 1) + b] = (T)v[q];    // sA[p][a] = L[j0 + p][i0 + a]
                else sA[b * (RB + 1) + a] = (T)v[q];          // sA[p][a] = L[i0 + a][j0 + p]
            }
        };
        auto load_y = [&](int jb, T (&v)[4]) {
            const int64_t j0 = (int64_t)jb * RB;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = t + 256 * q, p = e >> 4, r = e & 15;
                v[q] = (j0 + p < n && r < nrhs) ? __ldcg(&Y[(j0 + p) * ldy + r]) : (T)0;
            }
        };
        auto store_y = [&](const T (&v)[4]) {
#pragma unroll
            for (int q = 0; q < 4; ++q) sY[t + 256 * q] = v[q];
        };
        T acc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t i = i0 + row;
            const int r = cg + 4 * u;
            acc[u] = (i < n && r < nrhs) ? __ldcg(&Y[i * ldy + r]) : (T)0;
        }
        if (t == 0) s_known = (nj > 0 && ld_acquire_u32(&flag[jblk(nj - 1)]) != 0u) ? nj - 1 : -1;
        __syncthreads();
        int known = s_known;
        double preL[16];
        T preY[4];
        load_tile(nj > 0 ? jblk(0) : bi, preL);
        bool hy = false;
        if (nj > 0 && known >= 0) { load_y(jblk(0), preY); hy = true; }
        for (int k = 0; k < nj; ++k) {
            store_tile(preL);
            if (hy) store_y(preY);
            bool next_y = false;
            if (k + 1 < nj) {
                load_tile(jblk(k + 1), preL);
                if (k + 1 <= known) { load_y(jblk(k + 1), preY); next_y = true; }
            } else {
                load_tile(bi, preL);                  // the diagonal tile comes next
            }
            if (!hy) {
                if (t == 0) {
                    int ok = 1;
                    const unsigned long long t_start = global_ns();
                    while (ld_acquire_u32(&flag[jblk(k)]) == 0u) {
                        if (*(volatile unsigned*)err != 0u) { ok = 0; break; }
                        if (global_ns() - t_start > 1000000000ull) {
                            atomicExch(err, 1u);
                            ok = 0;
                            break;
                        }
                        __nanosleep(32);
                    }
                    int kn = k;
                    if (ok && ld_acquire_u32(&flag[jblk(nj - 1)]) != 0u) kn = nj - 1;
                    s_known = kn;
                    s_ok = ok;
                }
                __syncthreads();
                if (!s_ok) return;
                known = s_known;
                T v[4];
                load_y(jblk(k), v);
                store_y(v);
            }
            __syncthreads();
#pragma unroll 8
            for (int p = 0; p < RB; ++p) {
                const T a = sA[p * (RB + 1) + row];
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u] -= a * sY[p * MAXRHS + cg + 4 * u];
            }
            __syncthreads();
            hy = next_y;
        }
        // diagonal block
        store_tile(preL);
        for (int e = t; e < 2 * 32 * 32; e += 256) {
            const int c = e >> 10, a = (e >> 5) & 31, b = e & 31;
            const int ci = (int)(i0 / 32) + c;
            sI[(c * 32 + a) * 33 + b] = (ci < nchunk) ? Inv[((int64_t)ci * 32 + a) * 32 + b] : (T)0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) sY[row * MAXRHS + cg + 4 * u] = acc[u];
        __syncthreads();
        const int q = t >> 3, r0 = t & 7;
        // first chunk (rows 0..31 for L, 32..63 for L^T)
        {
            const int c = TRANS ? 1 : 0, o = 32 * c;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = r0 + 8 * h;
                T v = 0;
                for (int p = 0; p < 32; ++p) {
                    const T m = TRANS ? sI[(c * 32 + p) * 33 + q] : sI[(c * 32 + q) * 33 + p];
                    v += m * sY[(o + p) * MAXRHS + r];
                }
                sX[(o + q) * MAXRHS + r] = v;
            }
        }
        __syncthreads();
        // couple the second chunk to the first
        {
            const int o2 = TRANS ? 0 : 32, o1 = TRANS ? 32 : 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = r0 + 8 * h;
                T v = 0;
                for (int p = 0; p < 32; ++p) {
                    // L: L[32 + q][p] = sA[p][32 + q];  L^T: L[32 + p][q] = sA[32 + p][q]
                    const T m = sA[(o1 + p) * (RB + 1) + o2 + q];
                    v += m * sX[(o1 + p) * MAXRHS + r];
                }
                sY[(o2 + q) * MAXRHS + r] -= v;
            }
        }
        __syncthreads();
        {
            const int c = TRANS ? 0 : 1, o = 32 * c;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = r0 + 8 * h;
                T v = 0;
                for (int p = 0; p < 32; ++p) {
                    const T m = TRANS ? sI[(c * 32 + p) * 33 + q] : sI[(c * 32 + q) * 33 + p];
                    v += m * sY[(o + p) * MAXRHS + r];
                }
                sX[(o + q) * MAXRHS + r] = v;
            }
        }
        __syncthreads();
        for (int e = t; e < RB * MAXRHS; e += 256) {
            const int a = e >> 4, r = e & 15;
            if (i0 + a < n && r < nrhs) Y[(i0 + a) * ldy + r] = sX[e];
        }
        __syncthreads();
        if (t == 0) {
            __threadfence();
            st_release_u32(&flag[bi], 1u);
        }
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

// Y = sum_s P[s] (fixed order): the product A X from the split-K partials.
__global__ void k_symv_reduce(const double* P, int nsplit, int64_t n, double* Y) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * MAXRHS) return;
    const int64_t i = e / MAXRHS;
    const int r = (int)(e % MAXRHS);
    double s = 0.0;
    for (int k = 0; k < nsplit; ++k) s += P[((int64_t)k * n + i) * MAXRHS + r];
    Y[e] = s;
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
    const int bytes = (int)sweep_smem_bytes<T>();
    cudaError_t e = cudaFuncSetAttribute(k_trsv_sweep<T, 0>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_trsv_sweep<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bytes);
    if (e == cudaSuccess) done = true;
    return e;
}

size_t inv_region(int64_t n, bool f64) {
    const size_t b = (size_t)((n + 31) / 32) * 32 * 32 * (f64 ? sizeof(double) : sizeof(float));
    return (b + 255) / 256 * 256;
}

size_t sync_words(int64_t n) { return 4 + 2 * (size_t)((n + RB - 1) / RB); }

template <typename T>
cudaError_t potrs_t(int64_t n, int nrhs, const double* L, int64_t ldl, T* Y, int64_t ldy, T* Inv,
                    cudaStream_t s) {
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    cudaError_t e = set_attrs<T>();
    if (e != cudaSuccess) return e;
    unsigned* sync = (unsigned*)((char*)Inv + inv_region(n, sizeof(T) == sizeof(double)));
    e = cudaMemsetAsync(sync, 0, sizeof(unsigned) * sync_words(n), s);
    if (e != cudaSuccess) return e;
    k_chunk_inv<T><<<(unsigned)((n + 31) / 32), 32, 0, s>>>(L, ldl, n, Inv);
    note_launch();
    const int NB = (int)((n + RB - 1) / RB);
    const unsigned grid = (unsigned)std::min<int64_t>(NB, 2 * (int64_t)num_sms());
    const size_t smem = sweep_smem_bytes<T>();
    k_trsv_sweep<T, 0><<<grid, 256, smem, s>>>(L, ldl, n, Y, ldy, nrhs, Inv, sync);
    note_launch();
    k_trsv_sweep<T, 1><<<grid, 256, smem, s>>>(L, ldl, n, Y, ldy, nrhs, Inv, sync);
    note_launch();
    return cudaGetLastError();
}

}  // namespace

int potrs_max_rhs() { return MAXRHS; }

cudaError_t launch_potrs_f64(int64_t n, int nrhs, int64_t nb, const double* L, int64_t ldl,
                             double* B, int64_t ldb, double* inv, cudaStream_t s) {
    (void)nb;
    return potrs_t<double>(n, nrhs, L, ldl, B, ldb, inv, s);
}

cudaError_t launch_potrs_f32(int64_t n, int nrhs, int64_t nb, const double* L, int64_t ldl,
                             float* B, int64_t ldb, float* inv, cudaStream_t s) {
    (void)nb;
    return potrs_t<float>(n, nrhs, L, ldl, B, ldb, inv, s);
}

int potrs_error(const void* inv, int64_t n, bool f64, cudaStream_t s, cudaError_t* ce) {
    unsigned h = 0;
    const unsigned* sync = (const unsigned*)((const char*)inv + inv_region(n, f64));
    *ce = cudaMemcpyAsync(&h, sync + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (*ce == cudaSuccess) *ce = cudaStreamSynchronize(s);
    return (int)h;
}

size_t potrs_inv_bytes(int64_t n, bool f64) {
    return inv_region(n, f64) + sizeof(unsigned) * sync_words(n);
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

cudaError_t launch_symv(const double* A, int64_t lda, int64_t n, const double* X, double* Y,
                        double* P, int nsplit, cudaStream_t s) {
    const int64_t kchunk = ((n + nsplit - 1) / nsplit + 31) / 32 * 32;
    dim3 grid((unsigned)((n + 63) / 64), (unsigned)nsplit);
    k_resid_partial<<<grid, 256, 0, s>>>(A, lda, n, X, MAXRHS, MAXRHS, kchunk, P);
    note_launch();
    const int64_t tot = n * MAXRHS;
    k_symv_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(P, nsplit, n, Y);
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
