// k_solve.cu -- triangular solves with a Cholesky factor (potrs) and the
// pieces of iterative refinement: the FP64 residual R = B - A X, the
// normwise backward error, and X += D.
//
// potrs is the inverses of the diagonal blocks (128 rows in FP32, 64 in FP64)
// and two launches of a persistent sweep kernel (forward with L, backward
// with L^T), each covering all blocks with flag-ordered block solves.
// T is the arithmetic type (double for the FP64 solve, float for the
// correction solves of iterative refinement); L is read in FP64 and converted
// on load.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace abft {

namespace {

constexpr int MAXRHS = 16;

// Block geometry of the sweeps: 128-row blocks and 512 threads in FP32, 64-row
// blocks and 256 threads in FP64 (shared memory holds one tile of L and the
// inverse of the block's diagonal part).
template <typename T>
struct SweepCfg;
template <>
struct SweepCfg<float> {
    static constexpr int RB = 128;
};
template <>
struct SweepCfg<double> {
    static constexpr int RB = 64;
};

template <typename T>
size_t inv_smem_bytes() {
    constexpr int RB = SweepCfg<T>::RB;
    return sizeof(T) * 2 * (size_t)RB * (RB + 1);
}

// Inverse of each RB x RB diagonal block of L (rows past n are the identity),
// one CTA of RB threads per block: thread j computes column j by forward
// substitution with true divisions, X[j][j] = 1 / L[j][j] and
// X[i][j] = -(sum_{p=j}^{i-1} L[i][p] X[p][j]) / L[i][i].  Inv holds the
// blocks one after the other, RB x RB row-major each.
template <typename T>
__global__ void k_block_inv(const double* L, int64_t ldl, int64_t n, T* Inv) {
    constexpr int RB = SweepCfg<T>::RB;
    extern __shared__ __align__(16) unsigned char bsb[];
    T* Ls = (T*)bsb;                      // RB x (RB + 1)
    T* Xs = Ls + RB * (RB + 1);           // column j written by thread j
    const int64_t b0 = (int64_t)blockIdx.x * RB;
    const int t = threadIdx.x;
    for (int e = t; e < RB * RB; e += RB) {
        const int i = e / RB, j = e % RB;
        const int64_t gi = b0 + i, gj = b0 + j;
        T v;
        if (gi < n && gj < n) v = (j <= i) ? (T)L[gi * ldl + gj] : (T)0;
        else v = (i == j) ? (T)1 : (T)0;
        Ls[i * (RB + 1) + j] = v;
    }
    __syncthreads();
    const int j = t;
    for (int i = 0; i < RB; ++i) {
        T x = 0;
        if (i == j) {
            x = (T)1 / Ls[i * (RB + 1) + i];
        } else if (i > j) {
            T s0 = 0, s1 = 0;
            int p = j;
            for (; p + 1 < i; p += 2) {
                s0 += Ls[i * (RB + 1) + p] * Xs[p * (RB + 1) + j];
                s1 += Ls[i * (RB + 1) + p + 1] * Xs[(p + 1) * (RB + 1) + j];
            }
            if (p < i) s0 += Ls[i * (RB + 1) + p] * Xs[p * (RB + 1) + j];
            x = -(s0 + s1) / Ls[i * (RB + 1) + i];
        }
        Xs[i * (RB + 1) + j] = x;
    }
    __syncthreads();
    T* out = Inv + (int64_t)blockIdx.x * RB * RB;
    for (int e = t; e < RB * RB; e += RB) out[e] = Xs[(e / RB) * (RB + 1) + e % RB];
}

// Coupling of each block with the block solved just before it, folded with
// the block's inverse: P_i = Inv_i L_{i,i-1} for the L sweep (block 0 has
// none) and P_i = Inv_i^T L_{i+1,i}^T for the L^T sweep (the last block has
// none); RB x RB row-major per block, at P + i RB^2.  With them the last step
// of a block's solve is y_i = w_i - P_i y_prev, w_i = M_i (b_i - the older
// couplings) formed before y_prev is ready: one product on the sweep's
// critical path instead of two.  One CTA of RB threads per block; thread b
// forms column b, each entry one FMA chain over p in order.
template <typename T, int TRANS>
__global__ void k_block_couple(const double* L, int64_t ldl, int64_t n, const T* Inv, T* P) {
    constexpr int RB = SweepCfg<T>::RB;
    extern __shared__ __align__(16) unsigned char csb[];
    T* Ms = (T*)csb;                      // RB x (RB + 1): M[a][p]
    T* Cs = Ms + RB * (RB + 1);           // RB x (RB + 1): C[p][b]
    const int NB = (int)((n + RB - 1) / RB);
    const int i = blockIdx.x;
    const bool has = TRANS ? i + 1 < NB : i > 0;
    T* out = P + (int64_t)i * RB * RB;
    const int t = threadIdx.x;
    if (!has) {
        for (int e = t; e < RB * RB; e += RB) out[e] = (T)0;
        return;
    }
    const int64_t i0 = (int64_t)i * RB, jn0 = (int64_t)(TRANS ? i + 1 : i - 1) * RB;
    const T* Ib = Inv + (int64_t)i * RB * RB;
    for (int e = t; e < RB * RB; e += RB) {
        const int a = e / RB, q = e % RB;
        Ms[a * (RB + 1) + q] = TRANS ? Ib[q * RB + a] : Ib[e];   // M = Inv_i^T or Inv_i
        // C[p][b]: L_{i,i-1}[p][b] = L[i0 + p][jn0 + b], or L_{i+1,i}^T[p][b] = L[jn0 + b][i0 + p]
        const int64_t gr = TRANS ? jn0 + q : i0 + a, gc = TRANS ? i0 + a : jn0 + q;
        Cs[a * (RB + 1) + q] = (gr < n && gc < n) ? (T)L[gr * ldl + gc] : (T)0;
    }
    __syncthreads();
    const int b = t;
    for (int a = 0; a < RB; ++a) {
        T acc = 0;
        for (int q = 0; q < RB; ++q) acc = fma(Ms[a * (RB + 1) + q], Cs[q * (RB + 1) + b], acc);
        out[a * RB + b] = acc;
    }
}

// One triangular sweep in a single launch: L Y = Y (TRANS = 0) or L^T X = X
// (TRANS = 1) for nrhs <= 16 right-hand sides, Y row-major (ld ldy), solved in
// place.  Rows are cut into RB-row blocks.  CTAs take blocks from a ticket
// counter in solve order (first to last for L, last to first for L^T); the CTA
// of block i loads the block's precomputed inverse, streams the RB x RB tiles
// of L that couple it to the blocks solved before it, waiting on each block's
// ready flag, then forms y_i = Inv_i (b_i - sum_j L_ij y_j) (Inv_i^T for L^T)
// and publishes its rows and flag.  A CTA only waits on blocks whose tickets
// were handed out before its own, so the sweep completes whatever the number
// of resident CTAs.  Every wait gives up after one second: it sets sync[2] and
// the remaining CTAs drain.
// sync: [0] / [1] tickets (L, L^T), [2] error, [4, 4 + NB) flags of the L
// sweep, [4 + NB, 4 + 2 NB) flags of the L^T sweep; zeroed before the solve.
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
    constexpr int RB = SweepCfg<T>::RB;
    return sizeof(T) * (2 * (size_t)RB * (RB + 1) + (size_t)RB * MAXRHS);
}

template <typename T, int TRANS, typename LT>
__global__ void __launch_bounds__(4 * SweepCfg<T>::RB) k_trsv_sweep(
    const LT* __restrict__ L, int64_t ldl, int64_t n, T* Y, int64_t ldy, int nrhs,
    const T* __restrict__ Inv, const T* __restrict__ Pc, unsigned* sync) {
    constexpr int RB = SweepCfg<T>::RB, NT = 4 * RB, PER = RB * RB / NT, YPER = RB * MAXRHS / NT;
    extern __shared__ __align__(16) unsigned char sb[];
    T* sA = (T*)sb;                         // tile, sA[p * (RB + 1) + a] = op(L)[a][p]
    T* sI = sA + RB * (RB + 1);             // sI[p * (RB + 1) + a] = M[a][p], M = Inv_i or Inv_i^T
    T* sY = sI + RB * (RB + 1);             // solved rows of the tile / rhs of the diagonal
    __shared__ int s_blk, s_ok, s_known;
    const int NB = (int)((n + RB - 1) / RB);
    unsigned* ticket = sync + TRANS;
    unsigned* err = sync + 2;
    unsigned* flag = sync + 4 + (TRANS ? NB : 0);
    // compute roles: 4 groups split the RB-long inner dimension into quarters;
    // in a group, thread (rg, cg) owns rows rg + c RB / 4 (c < 4) and
    // right-hand sides 4 cg .. 4 cg + 3 (a 4 x 4 register block)
    constexpr int Q = RB / 4;
    const int t = threadIdx.x, g = t / RB, rg = t % Q, cg = (t / Q) % 4;
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
        auto load_tile = [&](int jb, LT (&v)[PER]) {
            const int64_t j0 = (int64_t)jb * RB;
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int e = t + NT * q, a = e / RB, b = e % RB;
                const int64_t gr = TRANS ? j0 + a : i0 + a, gc = TRANS ? i0 + b : j0 + b;
                v[q] = (gr < n && gc < n) ? L[gr * ldl + gc] : (LT)0;
            }
        };
        auto store_tile = [&](const LT (&v)[PER]) {
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int e = t + NT * q, a = e / RB, b = e % RB;
                if (TRANS) sA[a * (RB + 1) + b] = (T)v[q];    // sA[p][a] = L[j0 + p][i0 + a]
                else sA[b * (RB + 1) + a] = (T)v[q];          // sA[p][a] = L[i0 + a][j0 + p]
            }
        };
        auto load_y = [&](int jb, T (&v)[YPER]) {
            const int64_t j0 = (int64_t)jb * RB;
#pragma unroll
            for (int q = 0; q < YPER; ++q) {
                const int e = t + NT * q, p = e >> 4, r = e & 15;
                v[q] = (j0 + p < n && r < nrhs) ? __ldcg(&Y[(j0 + p) * ldy + r]) : (T)0;
            }
        };
        auto store_y = [&](const T (&v)[YPER]) {
#pragma unroll
            for (int q = 0; q < YPER; ++q) sY[t + NT * q] = v[q];
        };
        // the block's inverse, off the critical path of the sweep
        {
            const T* Ib = Inv + (int64_t)bi * RB * RB;
            for (int e = t; e < RB * RB; e += NT) {
                const int i = e / RB, j = e % RB;
                if (TRANS) sI[i * (RB + 1) + j] = Ib[e];     // M[a][p] = Inv[p][a]
                else sI[j * (RB + 1) + i] = Ib[e];           // M[a][p] = Inv[a][p]
            }
        }
        T acc[4][4];            // partial sum over this group's quarter of every tile
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[c][u] = 0;
        T bv[RB * MAXRHS / NT];  // this thread's right-hand side entries of block i
#pragma unroll
        for (int q = 0; q < RB * MAXRHS / NT; ++q) {
            const int e = t + NT * q, i = e / MAXRHS, r = e % MAXRHS;
            bv[q] = (i0 + i < n && r < nrhs) ? __ldcg(&Y[(i0 + i) * ldy + r]) : (T)0;
        }
        if (t == 0) s_known = (nj > 0 && ld_acquire_u32(&flag[jblk(nj - 1)]) != 0u) ? nj - 1 : -1;
        __syncthreads();
        int known = s_known;
        // with the coupling products, the block solved just before this one
        // (the last in solve order) is taken through P_i at the end
        const bool usep = Pc != nullptr && nj > 0;
        const int nk = usep ? nj - 1 : nj;
        // wait until block jblk(k) is solved; false when the sweep gives up
        auto wait_block = [&](int k) -> bool {
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
                }
                int kn = k;
                if (ok && ld_acquire_u32(&flag[jblk(nj - 1)]) != 0u) kn = nj - 1;
                s_known = kn;
                s_ok = ok;
            }
            __syncthreads();
            known = s_known;
            return s_ok != 0;
        };
        // acc += sA^T sY over this group's quarter of the inner dimension
        auto tile_product = [&]() {
#pragma unroll 8
            for (int pp = 0; pp < Q; ++pp) {
                const int p = g * Q + pp;
                T a[4], yv[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) a[c] = sA[p * (RB + 1) + rg + c * Q];
#pragma unroll
                for (int u = 0; u < 4; ++u) yv[u] = sY[p * MAXRHS + 4 * cg + u];
#pragma unroll
                for (int c = 0; c < 4; ++c)
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc[c][u] += a[c] * yv[u];
            }
        };
        LT preL[PER];
        T preY[YPER];
        if (nk > 0) load_tile(jblk(0), preL);
        bool hy = false;
        if (nk > 0 && known >= 0) { load_y(jblk(0), preY); hy = true; }
        for (int k = 0; k < nk; ++k) {
            store_tile(preL);
            if (hy) store_y(preY);
            bool next_y = false;
            if (k + 1 < nk) {
                load_tile(jblk(k + 1), preL);
                if (k + 1 <= known) { load_y(jblk(k + 1), preY); next_y = true; }
            }
            if (!hy) {
                if (!wait_block(k)) return;
                T v[YPER];
                load_y(jblk(k), v);
                store_y(v);
            }
            __syncthreads();
            tile_product();
            __syncthreads();
            hy = next_y;
        }
        // y_i = M (b_i - sum_j L_ij y_j): combine the groups' partial sums in
        // group order, then the same split product with M
        T* red = sA;                             // [4][RB][16], reuses the tile buffer
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int u = 0; u < 4; ++u)
                red[(g * RB + rg + c * Q) * MAXRHS + 4 * cg + u] = acc[c][u];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < RB * MAXRHS / NT; ++q) {
            const int e = t + NT * q;
            T sum = red[e];
#pragma unroll
            for (int h = 1; h < 4; ++h) sum += red[h * RB * MAXRHS + e];
            sY[e] = bv[q] - sum;
        }
        __syncthreads();
        T out[4][4];
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int u = 0; u < 4; ++u) out[c][u] = 0;
#pragma unroll 8
        for (int pp = 0; pp < Q; ++pp) {
            const int p = g * Q + pp;
            T m[4], yv[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) m[c] = sI[p * (RB + 1) + rg + c * Q];
#pragma unroll
            for (int u = 0; u < 4; ++u) yv[u] = sY[p * MAXRHS + 4 * cg + u];
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int u = 0; u < 4; ++u) out[c][u] += m[c] * yv[u];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int u = 0; u < 4; ++u)
                red[(g * RB + rg + c * Q) * MAXRHS + 4 * cg + u] = out[c][u];
        __syncthreads();
        T wv[YPER];   // w_i (usep) or y_i, entries t + NT q of the block's RB x 16
#pragma unroll
        for (int q = 0; q < YPER; ++q) {
            const int e = t + NT * q;
            T sum = red[e];
#pragma unroll
            for (int h = 1; h < 4; ++h) sum += red[h * RB * MAXRHS + e];
            wv[q] = sum;
        }
        if (usep) {
            // y_i = w_i - P_i y_prev: P_i in the tile buffer as a tile
            // (sA[p][a] = P_i[a][p]), y_prev once its block is solved
            __syncthreads();   // red (the tile buffer) has been read
            const T* Pb = Pc + (int64_t)bi * RB * RB;
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int e = t + NT * q, aa = e / RB, pq = e % RB;
                sA[pq * (RB + 1) + aa] = Pb[e];
            }
            if (known < nj - 1 && !wait_block(nj - 1)) return;
            {
                T v[YPER];
                load_y(jblk(nj - 1), v);
                store_y(v);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[c][u] = 0;
            __syncthreads();
            tile_product();
            __syncthreads();   // P_i (the tile buffer) has been read: reuse it for the sums
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    red[(g * RB + rg + c * Q) * MAXRHS + 4 * cg + u] = acc[c][u];
            __syncthreads();
#pragma unroll
            for (int q = 0; q < YPER; ++q) {
                const int e = t + NT * q;
                T sum = red[e];
#pragma unroll
                for (int h = 1; h < 4; ++h) sum += red[h * RB * MAXRHS + e];
                wv[q] -= sum;
            }
        }
#pragma unroll
        for (int q = 0; q < YPER; ++q) {
            const int e = t + NT * q, i = e / MAXRHS, r = e % MAXRHS;
            if (i0 + i < n && r < nrhs) Y[(i0 + i) * ldy + r] = wv[q];
        }
        __syncthreads();
        // the release store orders the CTA's stores of y_i (made visible to
        // thread 0 by the barrier) before the flag
        if (t == 0) st_release_u32(&flag[bi], 1u);
    }
}

// L32[i][j] = RN(L[i][j]) for j <= i (the strict upper triangle is not
// written); one CTA per row (grid-stride), four loads in flight per thread.
__global__ void k_tril_to_f32(const double* L, int64_t ldl, int64_t n, float* L32, int64_t ld32) {
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const double* src = L + i * ldl;
        float* dst = L32 + i * ld32;
        for (int64_t j0 = threadIdx.x; j0 <= i; j0 += 4 * (int64_t)blockDim.x) {
            double v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t j = j0 + u * (int64_t)blockDim.x;
                v[u] = j <= i ? src[j] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t j = j0 + u * (int64_t)blockDim.x;
                if (j <= i) dst[j] = (float)v[u];
            }
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

// Split-K partial products of the residual: P[s][i][r] = sum_{p in chunk s} A[i][p] X[p][r],
// in the arithmetic of T (double: the FP64 residual and product; float: the
// FP32 product of GMRES-IR's inner solver, from an FP32 copy of A).
template <typename T>
__global__ void __launch_bounds__(256) k_resid_partial(const T* A, int64_t lda, int64_t n,
                                                       const double* X, int64_t ldx, int nrhs,
                                                       int64_t kchunk, double* P) {
    __shared__ T As[32][65];
    __shared__ T Xs[32][MAXRHS];
    const int t = threadIdx.x;
    const int64_t i0 = blockIdx.x * 64;
    const int64_t kbeg = blockIdx.y * kchunk;
    const int64_t kend = (kbeg + kchunk < n) ? kbeg + kchunk : n;
    const int row = t & 63, cg = t >> 6;
    T acc[4] = {0, 0, 0, 0};
    for (int64_t k0 = kbeg; k0 < kend; k0 += 32) {
        // A is symmetric and only its lower triangle is read: A[i][p] for p <= i,
        // A[p][i] above; whole tiles on one side load coalesced.
        if (k0 + 31 <= i0) {
            for (int e = t; e < 64 * 32; e += 256) {
                int a = e >> 5, b = e & 31;
                int64_t i = i0 + a, p = k0 + b;
                As[b][a] = (i < n && p < kend) ? A[i * lda + p] : (T)0;
            }
        } else if (k0 >= i0 + 64) {
            for (int e = t; e < 64 * 32; e += 256) {
                int b = e >> 6, a = e & 63;
                int64_t i = i0 + a, p = k0 + b;
                As[b][a] = (i < n && p < kend) ? A[p * lda + i] : (T)0;
            }
        } else {
            for (int e = t; e < 64 * 32; e += 256) {
                int a = e >> 5, b = e & 31;
                int64_t i = i0 + a, p = k0 + b;
                As[b][a] = (i < n && p < kend) ? (p <= i ? A[i * lda + p] : A[p * lda + i]) : (T)0;
            }
        }
        for (int e = t; e < 32 * MAXRHS; e += 256) {
            int p = e / MAXRHS, r = e % MAXRHS;
            Xs[p][r] = (k0 + p < kend && r < nrhs) ? (T)X[(k0 + p) * ldx + r] : (T)0;
        }
        __syncthreads();
#pragma unroll 8
        for (int p = 0; p < 32; ++p) {
            const T a = As[p][row];
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
            if (r < nrhs) P[((int64_t)blockIdx.y * n + i) * MAXRHS + r] = (double)acc[u];
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

// The strict column part of the row sums of |A| (i > j of column j) in
// kNormChunks row ranges per column (P[c][j]), so that many threads stream
// each column; then ||A||_inf = max_j (rs[j] + sum_c P[c][j]) in a fixed order.
constexpr int kNormChunks = 16;

__global__ void k_abs_colsum_part(const double* A, int64_t lda, int64_t n, double* P) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int64_t chunk = (n + kNormChunks - 1) / kNormChunks;
    const int64_t i0 = blockIdx.y * chunk, i1 = i0 + chunk < n ? i0 + chunk : n;
    double s0 = 0.0, s1 = 0.0;
    int64_t i = i0 > j + 1 ? i0 : j + 1;
    for (; i + 1 < i1; i += 2) {
        s0 += fabs(A[i * lda + j]);
        s1 += fabs(A[(i + 1) * lda + j]);
    }
    if (i < i1) s0 += fabs(A[i * lda + j]);
    P[blockIdx.y * n + j] = s0 + s1;
}

__global__ void k_abs_colsum_strict(const double* rs, const double* P, int64_t n, const double* B,
                                    int64_t ldb, int nrhs, unsigned long long* anorm,
                                    unsigned long long* bmax) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s = rs[j];
    for (int c = 0; c < kNormChunks; ++c) s += P[c * n + j];
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
    cudaError_t e = cudaFuncSetAttribute(k_trsv_sweep<T, 0, double>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_trsv_sweep<T, 1, double>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && sizeof(T) == sizeof(float))
        e = cudaFuncSetAttribute(k_trsv_sweep<T, 0, float>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && sizeof(T) == sizeof(float))
        e = cudaFuncSetAttribute(k_trsv_sweep<T, 1, float>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_block_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)inv_smem_bytes<T>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_block_couple<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)inv_smem_bytes<T>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_block_couple<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)inv_smem_bytes<T>());
    if (e == cudaSuccess) done = true;
    return e;
}

template <typename T>
int64_t sweep_blocks(int64_t n) {
    return (n + SweepCfg<T>::RB - 1) / SweepCfg<T>::RB;
}

size_t inv_region(int64_t n, bool f64) {
    const size_t b = f64 ? (size_t)sweep_blocks<double>(n) * 64 * 64 * sizeof(double)
                         : (size_t)sweep_blocks<float>(n) * 128 * 128 * sizeof(float);
    return (b + 255) / 256 * 256;
}

// The solve's precomputed region: the diagonal blocks' inverses, then the
// coupling products of the L sweep and of the L^T sweep (each the size of the
// inverses), then the sweeps' tickets and flags.
size_t pre_region(int64_t n, bool f64) { return 3 * inv_region(n, f64); }

size_t sync_words(int64_t n, bool f64) {
    return 4 + 2 * (size_t)(f64 ? sweep_blocks<double>(n) : sweep_blocks<float>(n));
}

template <typename T>
cudaError_t potrs_t(int64_t n, int nrhs, const double* L, int64_t ldl, const float* L32, T* Y,
                    int64_t ldy, T* Inv, bool have_inv, cudaStream_t s) {
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    constexpr bool F64 = sizeof(T) == sizeof(double);
    cudaError_t e = set_attrs<T>();
    if (e != cudaSuccess) return e;
    unsigned* sync = (unsigned*)((char*)Inv + pre_region(n, F64));
    T* P0 = (T*)((char*)Inv + inv_region(n, F64));
    T* P1 = (T*)((char*)Inv + 2 * inv_region(n, F64));
    e = cudaMemsetAsync(sync, 0, sizeof(unsigned) * sync_words(n, F64), s);
    if (e != cudaSuccess) return e;
    const int64_t NB = sweep_blocks<T>(n);
    if (!have_inv) {
        k_block_inv<T><<<(unsigned)NB, SweepCfg<T>::RB, inv_smem_bytes<T>(), s>>>(L, ldl, n, Inv);
        note_launch();
        k_block_couple<T, 0><<<(unsigned)NB, SweepCfg<T>::RB, inv_smem_bytes<T>(), s>>>(L, ldl, n, Inv, P0);
        note_launch();
        k_block_couple<T, 1><<<(unsigned)NB, SweepCfg<T>::RB, inv_smem_bytes<T>(), s>>>(L, ldl, n, Inv, P1);
        note_launch();
    }
    const int per_sm = F64 ? 2 : 1;
    const unsigned grid = (unsigned)std::min<int64_t>(NB, per_sm * (int64_t)num_sms());
    const size_t smem = sweep_smem_bytes<T>();
    constexpr int NT = 4 * SweepCfg<T>::RB;
    if (!F64 && L32 != nullptr) {   // FP32 tiles: no conversion in the sweep
        k_trsv_sweep<T, 0, float><<<grid, NT, smem, s>>>(L32, n, n, Y, ldy, nrhs, Inv, P0, sync);
        note_launch();
        k_trsv_sweep<T, 1, float><<<grid, NT, smem, s>>>(L32, n, n, Y, ldy, nrhs, Inv, P1, sync);
        note_launch();
    } else {
        k_trsv_sweep<T, 0, double><<<grid, NT, smem, s>>>(L, ldl, n, Y, ldy, nrhs, Inv, P0, sync);
        note_launch();
        k_trsv_sweep<T, 1, double><<<grid, NT, smem, s>>>(L, ldl, n, Y, ldy, nrhs, Inv, P1, sync);
        note_launch();
    }
    return cudaGetLastError();
}

}  // namespace

int potrs_max_rhs() { return MAXRHS; }

cudaError_t launch_potrs_f64(int64_t n, int nrhs, int64_t nb, const double* L, int64_t ldl,
                             double* B, int64_t ldb, double* inv, cudaStream_t s, bool have_inv) {
    (void)nb;
    return potrs_t<double>(n, nrhs, L, ldl, nullptr, B, ldb, inv, have_inv, s);
}

cudaError_t launch_potrs_f32(int64_t n, int nrhs, int64_t nb, const double* L, int64_t ldl,
                             float* B, int64_t ldb, float* inv, cudaStream_t s, bool have_inv,
                             const float* L32) {
    (void)nb;
    return potrs_t<float>(n, nrhs, L, ldl, L32, B, ldb, inv, have_inv, s);
}

cudaError_t launch_tril_to_f32(const double* L, int64_t ldl, int64_t n, float* L32,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_tril_to_f32<<<(unsigned)std::min<int64_t>(n, 1 << 20), 256, 0, s>>>(L, ldl, n, L32, n);
    note_launch();
    return cudaGetLastError();
}

int potrs_error(const void* inv, int64_t n, bool f64, cudaStream_t s, cudaError_t* ce) {
    unsigned h = 0;
    const unsigned* sync = (const unsigned*)((const char*)inv + pre_region(n, f64));
    *ce = cudaMemcpyAsync(&h, sync + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (*ce == cudaSuccess) *ce = cudaStreamSynchronize(s);
    return (int)h;
}

size_t potrs_inv_bytes(int64_t n, bool f64) {
    (void)f64;   // room for either arithmetic, so one region serves both
    return std::max(pre_region(n, true) + sizeof(unsigned) * sync_words(n, true),
                    pre_region(n, false) + sizeof(unsigned) * sync_words(n, false));
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
    k_resid_partial<double><<<grid, 256, 0, s>>>(A, lda, n, X, ldx, nrhs, kchunk, P);
    note_launch();
    int64_t tot = n * nrhs;
    k_resid_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(P, nsplit, n, B, ldb, X, ldx, nrhs,
                                                                 R, ldr, rmax, xmax);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_symv_reduce(const double* P, int nsplit, int64_t n, double* Y, cudaStream_t s) {
    const int64_t tot = n * MAXRHS;
    if (tot <= 0) return cudaSuccess;
    k_symv_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(P, nsplit, n, Y);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_resid_reduce(const double* P, int nsplit, int64_t n, const double* B,
                                int64_t ldb, const double* X, int64_t ldx, int nrhs, double* R,
                                int64_t ldr, unsigned long long* rmax, unsigned long long* xmax,
                                cudaStream_t s) {
    const int64_t tot = n * nrhs;
    if (tot <= 0) return cudaSuccess;
    k_resid_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(P, nsplit, n, B, ldb, X, ldx, nrhs,
                                                                 R, ldr, rmax, xmax);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_symv(const double* A, int64_t lda, int64_t n, const double* X, double* Y,
                        double* P, int nsplit, cudaStream_t s) {
    const int64_t kchunk = ((n + nsplit - 1) / nsplit + 31) / 32 * 32;
    dim3 grid((unsigned)((n + 63) / 64), (unsigned)nsplit);
    k_resid_partial<double><<<grid, 256, 0, s>>>(A, lda, n, X, MAXRHS, MAXRHS, kchunk, P);
    note_launch();
    const int64_t tot = n * MAXRHS;
    k_symv_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(P, nsplit, n, Y);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_symv_f32(const float* A, int64_t lda, int64_t n, const double* X, double* Y,
                            double* P, int nsplit, cudaStream_t s) {
    const int64_t kchunk = ((n + nsplit - 1) / nsplit + 31) / 32 * 32;
    dim3 grid((unsigned)((n + 63) / 64), (unsigned)nsplit);
    k_resid_partial<float><<<grid, 256, 0, s>>>(A, lda, n, X, MAXRHS, MAXRHS, kchunk, P);
    note_launch();
    const int64_t tot = n * MAXRHS;
    k_symv_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(P, nsplit, n, Y);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_inf_norms(const double* A, int64_t lda, int64_t n, const double* B, int64_t ldb,
                             int nrhs, double* rs, unsigned long long* anorm,
                             unsigned long long* bmax, double* scratch, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_abs_rowsum_lower<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(A, lda, n, rs);
    note_launch();
    k_abs_colsum_part<<<dim3((unsigned)((n + 255) / 256), kNormChunks), 256, 0, s>>>(A, lda, n,
                                                                                  scratch);
    note_launch();
    k_abs_colsum_strict<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rs, scratch, n, B, ldb, nrhs,
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
