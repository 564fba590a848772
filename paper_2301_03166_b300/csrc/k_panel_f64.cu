// k_panel_f64.cu -- FP64 panel kernels of the blocked Cholesky (Sec. 2.1:
// PD = factorization of the diagonal block, PU = triangular solve of the
// panel below it) and the PD checksum check (Sec. 3.1.2).
//
// The diagonal block is factored by the host in 64-column chunks: a one-CTA
// Cholesky of the 64 x 64 leaf in shared memory, a solve of the rows below
// it, and a rank-64 update (the DFMA tile kernel).  Solves use true division
// by the diagonal, never a reciprocal, so integer inputs stay exact.
#include <math.h>

#include <type_traits>

#include "common.cuh"
#include "fp_bits.cuh"

namespace abft {

namespace {

constexpr int LEAF = 64;

// Unblocked right-looking Cholesky of an nb x nb (nb <= 64) lower block in
// shared memory.  On a non-positive or NaN pivot at column j the first such
// index info_base + j + 1 is recorded and the block is left as it is.
__global__ void __launch_bounds__(256) k_potf2_small(double* A, int64_t lda, int nb,
                                                     int64_t info_base, DevStatus* st) {
    __shared__ double a[LEAF][LEAF + 1];
    __shared__ int fail;
    if (st->info != 0) return;
    const int t = threadIdx.x;
    for (int e = t; e < nb * nb; e += blockDim.x) {
        int i = e / nb, j = e % nb;
        if (j <= i) a[i][j] = A[(int64_t)i * lda + j];
    }
    if (t == 0) fail = -1;
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (t == 0) {
            double d = a[j][j];
            if (!(d > 0.0)) fail = j;
            else a[j][j] = sqrt(d);
        }
        __syncthreads();
        if (fail >= 0) break;
        const double djj = a[j][j];
        for (int i = j + 1 + t; i < nb; i += blockDim.x) a[i][j] = a[i][j] / djj;
        __syncthreads();
        // rank-1 update of the remaining lower triangle on a 16 x 16 thread grid
        const int tx = t & 15, ty = t >> 4;
        for (int i = j + 1 + ty; i < nb; i += 16) {
            const double aij = a[i][j];
            for (int l = j + 1 + tx; l <= i; l += 16) a[i][l] -= aij * a[l][j];
        }
        __syncthreads();
    }
    if (fail >= 0) {
        if (t == 0) atomicCAS(&st->info, 0, (int)(info_base + fail + 1));
        return;
    }
    for (int e = t; e < nb * nb; e += blockDim.x) {
        int i = e / nb, j = e % nb;
        if (j <= i) A[(int64_t)i * lda + j] = a[i][j];
    }
}

constexpr int RB = 32;     // rows per CTA
constexpr int CW = 32;     // column chunk
constexpr int TT = 256;

struct TrsmArgs {
    const double* L;
    int64_t ldl;
    int nb;
    TrsmSeg seg[2];
    int64_t start[3];
    int nseg;
    const double* v;
    double* x;
    const DevStatus* st;
    const float* Lf;    // FP32 solves: L rounded to FP32 once (nb x nb, ld nb), or null
    int rev;            // k_trsm_rows2 only: solve X L = B instead of X L^T = B
};

// The lower triangle of L rounded to FP32 (ld nb), once per panel solve
// instead of once per CTA (an FP64 -> FP32 conversion runs on the FP64 pipe).
__global__ void k_l_to_f32(const double* L, int64_t ldl, int nb, float* Lf) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)nb * nb) return;
    const int i = (int)(e / nb), j = (int)(e % nb);
    Lf[e] = j <= i ? (float)L[(int64_t)i * ldl + j] : 0.f;
}

// Solve X L^T = B (NT = false) or X L = B (NT = true) for RB rows at a time
// (in place), L lower nb x nb.  Columns are processed in chunks of 32, left to
// right for L^T (X[:, c] -= X[:, :c] L[c, :c]^T) and right to left for L
// (X[:, c] -= X[:, c1:] L[c1:, c]), the update by all threads, then a per-row
// substitution inside the chunk.
template <typename T, bool NT>
__global__ void __launch_bounds__(TT) k_trsm_rlt(TrsmArgs a) {
    extern __shared__ __align__(16) unsigned char smem_bytes[];
    T* smem = (T*)smem_bytes;
    const int ldx = a.nb + 1;
    T* X = smem;                            // RB x (nb + 1)
    T* Ls = smem + RB * ldx;                // CW x (CW + 1)
    if (a.st && a.st->info != 0) return;
    const int64_t bid = blockIdx.x;
    const int s = (a.nseg > 1 && bid >= a.start[1]) ? 1 : 0;
    const TrsmSeg& g = a.seg[s];
    const int64_t r0 = (bid - a.start[s]) * RB;
    const int nr = (int)((g.rows - r0) < RB ? (g.rows - r0) : RB);
    const int nb = a.nb, t = threadIdx.x;
    for (int e = t; e < RB * nb; e += TT) {
        int r = e / nb, p = e % nb;
        X[r * ldx + p] = (r < nr) ? (T)g.B[(r0 + r) * g.ldb + p] : (T)0;
    }
    __syncthreads();
    if (a.v != nullptr && s == 0) {  // carried row sums x = B v, before the solve
        const int warp = t >> 5, lane = t & 31;
        for (int r = warp; r < nr; r += TT / 32) {
            T acc = 0;
            for (int p = lane; p < nb; p += 32) acc = fma(X[r * ldx + p], (T)a.v[p], acc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) a.x[r0 + r] = (double)acc;
        }
        __syncthreads();
    }
    const int gr = t >> 3, gq = (t & 7) * 4;  // GEMM part: row gr, cols gq..gq+3
    const int nch = (nb + CW - 1) / CW;
    for (int ci = 0; ci < nch; ++ci) {
        const int c0 = (NT ? nch - 1 - ci : ci) * CW;
        const int w = (nb - c0) < CW ? (nb - c0) : CW;
        const int c1 = c0 + w;
        // each unknown's terms form one fused multiply-add chain in p order,
        // starting from its right-hand side: the chunk's columns continue here
        // from X and the substitution inside the chunk continues from them
        T acc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = (gq + u < w) ? X[gr * ldx + c0 + gq + u] : (T)0;
        const int pbeg = NT ? c1 : 0, pend = NT ? nb : c0;
        // the L piece of columns p0 .. p0 + CW - 1 of the chunk's rows: each
        // thread's CW * CW / TT values, loaded into registers one piece ahead
        // (the next piece's loads are in flight during this piece's products)
        constexpr int PPT = CW * CW / TT;
        auto load_piece = [&](int p0, T (&v)[PPT]) {
#pragma unroll
            for (int i = 0; i < PPT; ++i) {
                const int e = t + TT * i, q = e / CW, pp = e % CW;
                T x = 0;
                if (q < w && p0 + pp < pend) {
                    if (std::is_same<T, float>::value && !NT && a.Lf)
                        x = (T)a.Lf[(c0 + q) * nb + p0 + pp];
                    else
                        x = NT ? (T)a.L[(int64_t)(p0 + pp) * a.ldl + c0 + q]
                               : (T)a.L[(int64_t)(c0 + q) * a.ldl + p0 + pp];
                }
                v[i] = x;
            }
        };
        T lnext[PPT];
        if (pbeg < pend) load_piece(pbeg, lnext);
        for (int p0 = pbeg; p0 < pend; p0 += CW) {
            __syncthreads();
#pragma unroll
            for (int i = 0; i < PPT; ++i) {
                const int e = t + TT * i;
                Ls[(e / CW) * (CW + 1) + e % CW] = lnext[i];
            }
            __syncthreads();
            if (p0 + CW < pend) load_piece(p0 + CW, lnext);
#pragma unroll 8
            for (int pp = 0; pp < CW; ++pp) {
                T xv = (p0 + pp < pend) ? X[gr * ldx + p0 + pp] : (T)0;
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u] = fma(-xv, Ls[(gq + u) * (CW + 1) + pp], acc[u]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (gq + u < w) X[gr * ldx + c0 + gq + u] = acc[u];
        // the chunk's diagonal block: Ls[q][p] = L[c0+q][c0+p] (p <= q) for L^T,
        // L[c0+p][c0+q] (p >= q) for L
        for (int e = t; e < CW * CW; e += TT) {
            int q = e / CW, pp = e % CW;
            T v = 0;
            if (q < w && pp < w) {
                if (!NT && pp <= q)
                    v = (std::is_same<T, float>::value && a.Lf)
                            ? (T)a.Lf[(c0 + q) * nb + c0 + pp]
                            : (T)a.L[(int64_t)(c0 + q) * a.ldl + c0 + pp];
                if (NT && pp >= q) v = (T)a.L[(int64_t)(c0 + pp) * a.ldl + c0 + q];
            }
            Ls[q * (CW + 1) + pp] = v;
        }
        __syncthreads();
        if (t < RB) {
            T* xr = X + t * ldx + c0;
            if (std::is_same<T, float>::value && !NT && w == CW) {
                // FP32, a full chunk: the row's 32 unknowns in registers (fully
                // unrolled; the same terms, order and division as the loop below)
                T xv[CW];
#pragma unroll
                for (int jj = 0; jj < CW; ++jj) {
                    T v = xr[jj];
#pragma unroll
                    for (int p = 0; p < jj; ++p) v = fma(-xv[p], Ls[jj * (CW + 1) + p], v);
                    xv[jj] = v / Ls[jj * (CW + 1) + jj];
                }
#pragma unroll
                for (int jj = 0; jj < CW; ++jj) xr[jj] = xv[jj];
            } else if (!NT) {
                for (int jj = 0; jj < w; ++jj) {
                    T v = xr[jj];
                    for (int p = 0; p < jj; ++p) v = fma(-xr[p], Ls[jj * (CW + 1) + p], v);
                    xr[jj] = v / Ls[jj * (CW + 1) + jj];
                }
            } else {
                for (int jj = w - 1; jj >= 0; --jj) {
                    T v = xr[jj];
                    for (int p = jj + 1; p < w; ++p) v = fma(-xr[p], Ls[jj * (CW + 1) + p], v);
                    xr[jj] = v / Ls[jj * (CW + 1) + jj];
                }
            }
        }
        __syncthreads();
    }
    for (int e = t; e < nr * nb; e += TT) {
        int r = e / nb, p = e % nb;
        // FP32 results widen with integer operations (off the FP64 pipe)
        if (std::is_same<T, float>::value)
            g.B[(r0 + r) * g.ldb + p] = f32_to_f64_exact((float)X[r * ldx + p]);
        else
            g.B[(r0 + r) * g.ldb + p] = (double)X[r * ldx + p];
    }
}

// Solve X L^T = B in place for a narrow L (nb <= 64), one thread per row:
// four warps of 32 rows per CTA (one per SM sub-partition), each thread
// substituting its own row once L and the reciprocals of its diagonal are in
// shared memory; one warp per sub-partition keeps its FP64 unit busy
// (k_trsm_rlt's one-warp substitution next to seven waiting warps left most
// of it idle).  x_j = (b_j - sum_{p<j} x_p L_jp) / L_jj
// with the division by L_jj a multiplication by its reciprocal, formed once per
// CTA (exact for the power-of-two pivots of exact integer cases).  Two
// partial sums per row shorten the dependent chain.
constexpr int RW_ROWS = 128;
constexpr int RW_MAXNB = 64;
constexpr int RW_LD = RW_MAXNB + 1;

template <typename T>
__global__ void __launch_bounds__(RW_ROWS) k_trsm_rows(TrsmArgs a) {
    extern __shared__ __align__(16) unsigned char smem_bytes[];
    T* X = (T*)smem_bytes;                 // RW_ROWS x RW_LD
    T* Ls = X + RW_ROWS * RW_LD;           // nb x RW_LD
    T* rinv = Ls + RW_MAXNB * RW_LD;       // nb
    if (a.st && a.st->info != 0) return;
    const int64_t bid = blockIdx.x;
    const int s = (a.nseg > 1 && bid >= a.start[1]) ? 1 : 0;
    const TrsmSeg g = s ? a.seg[1] : a.seg[0];   // static indices: no local copy
    const int64_t r0 = (bid - (s ? a.start[1] : a.start[0])) * RW_ROWS;
    const int nr = (int)((g.rows - r0) < RW_ROWS ? (g.rows - r0) : RW_ROWS);
    const int nb = a.nb, t = threadIdx.x;
    for (int e = t; e < RW_ROWS * nb; e += RW_ROWS) {
        const int r = e / nb, p = e % nb;
        X[r * RW_LD + p] = r < nr ? (T)g.B[(r0 + r) * g.ldb + p] : (T)0;
    }
    for (int e = t; e < nb * nb; e += RW_ROWS) {
        const int j = e / nb, p = e % nb;
        Ls[j * RW_LD + p] = p <= j ? (T)a.L[(int64_t)j * a.ldl + p] : (T)0;
    }
    for (int j = t; j < nb; j += RW_ROWS) rinv[j] = (T)1 / (T)a.L[(int64_t)j * a.ldl + j];
    __syncthreads();
    T* xr = X + t * RW_LD;
    if (nb == RW_MAXNB) {
        // full width: the row's unknowns in registers (fully unrolled; the same
        // terms, pairing and order as the loop below), one shared load per term
        T xv[RW_MAXNB];
#pragma unroll
        for (int j = 0; j < RW_MAXNB; ++j) {
            const T* lj = Ls + j * RW_LD;
            T v0 = xr[j], v1 = 0;
#pragma unroll
            for (int p = 0; p + 1 < j; p += 2) {
                v0 -= xv[p] * lj[p];
                v1 -= xv[p + 1] * lj[p + 1];
            }
            if (j & 1) v0 -= xv[j - 1] * lj[j - 1];
            xv[j] = (v0 + v1) * rinv[j];
        }
#pragma unroll
        for (int j = 0; j < RW_MAXNB; ++j) xr[j] = xv[j];
    } else {
        for (int j = 0; j < nb; ++j) {
            const T* lj = Ls + j * RW_LD;
            T v0 = xr[j], v1 = 0;
            int p = 0;
            for (; p + 1 < j; p += 2) {
                v0 -= xr[p] * lj[p];
                v1 -= xr[p + 1] * lj[p + 1];
            }
            if (p < j) v0 -= xr[p] * lj[p];
            xr[j] = (v0 + v1) * rinv[j];
        }
    }
    __syncthreads();
    for (int e = t; e < nr * nb; e += RW_ROWS) {
        const int r = e / nb, p = e % nb;
        g.B[(r0 + r) * g.ldb + p] = (double)X[r * RW_LD + p];
    }
}

// The full-width FP64 case (nb = 64) with two threads per row, lanes 2 r and
// 2 r + 1: thread h sums the terms p = h (mod 2) of every unknown, in two
// partial sums, and keeps those x_p in registers; one shuffle per unknown adds
// the pair's sums (even + odd, the same order on both threads).
// rev: X L = B (the reverse sweep's panel solve).  With j' = 63 - j, that is
// x'_j' = (b'_j' - sum_{p' < j'} x'_p' M_j'p') / M_j'j' for M_j'p' = L_(63-p')(63-j')
// (lower triangular again): the same recurrence on the reversed columns of X
// and B with the anti-transpose of L.  Twice the
// warps of k_trsm_rows and half the dependent chain per thread: at these
// orders one thread per row leaves a quarter of the sub-partitions without a
// warp and the rest waiting on dependent FP64 FMAs.
constexpr int RW2_ROWS = 64;   // rows per CTA (128 threads)

__global__ void __launch_bounds__(2 * RW2_ROWS) k_trsm_rows2(TrsmArgs a) {
    extern __shared__ __align__(16) unsigned char smem_bytes[];
    double* X = (double*)smem_bytes;             // RW2_ROWS x RW_LD
    double* Ls = X + RW2_ROWS * RW_LD;           // 64 x RW_LD
    double* rinv = Ls + RW_MAXNB * RW_LD;        // 64
    if (a.st && a.st->info != 0) return;
    const int64_t bid = blockIdx.x;
    const int sg = (a.nseg > 1 && bid >= a.start[1]) ? 1 : 0;
    const TrsmSeg g = sg ? a.seg[1] : a.seg[0];   // static indices: no local copy
    const int64_t r0 = (bid - (sg ? a.start[1] : a.start[0])) * RW2_ROWS;
    const int nr = (int)((g.rows - r0) < RW2_ROWS ? (g.rows - r0) : RW2_ROWS);
    const int t = threadIdx.x;
    const int rv = a.rev ? RW_MAXNB - 1 : 0;   // column p of X, B is column |rv - p|
    for (int e = t; e < RW2_ROWS * RW_MAXNB; e += 2 * RW2_ROWS) {
        const int r = e / RW_MAXNB, p = e % RW_MAXNB;
        X[r * RW_LD + p] = r < nr ? g.B[(r0 + r) * g.ldb + (rv ? rv - p : p)] : 0.0;
    }
    for (int e = t; e < RW_MAXNB * RW_MAXNB; e += 2 * RW2_ROWS) {
        const int j = e / RW_MAXNB, p = e % RW_MAXNB;
        Ls[j * RW_LD + p] = p > j ? 0.0
                            : rv  ? a.L[(int64_t)(rv - p) * a.ldl + (rv - j)]
                                  : a.L[(int64_t)j * a.ldl + p];
    }
    for (int j = t; j < RW_MAXNB; j += 2 * RW2_ROWS)
        rinv[j] = 1.0 / a.L[(int64_t)(rv ? rv - j : j) * a.ldl + (rv ? rv - j : j)];
    __syncthreads();
    const int r = t >> 1, h = t & 1;
    double* xr = X + r * RW_LD;
    double xv[RW_MAXNB / 2];   // x_p, p = 2 q + h
#pragma unroll
    for (int j = 0; j < RW_MAXNB; ++j) {
        const double* lj = Ls + j * RW_LD;
        double s0 = 0.0, s1 = 0.0;
#pragma unroll
        for (int q = 0; 2 * q < j; ++q) {
            const int p = 2 * q + h;
            if (p < j) {
                if (q & 1) s1 = fma(xv[q], lj[p], s1);
                else s0 = fma(xv[q], lj[p], s0);
            }
        }
        const double sh = s0 + s1;
        const double so = __shfl_xor_sync(0xffffffffu, sh, 1);
        const double tot = h == 0 ? sh + so : so + sh;
        const double xj = (xr[j] - tot) * rinv[j];
        if ((j & 1) == h) xv[j >> 1] = xj;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < RW_MAXNB / 2; ++q) xr[2 * q + h] = xv[q];
    __syncthreads();
    for (int e = t; e < nr * RW_MAXNB; e += 2 * RW2_ROWS) {
        const int rr = e / RW_MAXNB, p = e % RW_MAXNB;
        g.B[(r0 + rr) * g.ldb + (rv ? rv - p : p)] = X[rr * RW_LD + p];
    }
}

// PD check on column sums: 1^T A_kk (carried, cc) vs (1^T L) L^T, and, when
// v != NULL, v = L^{-T} 1 (blocked back substitution, chunks of 32).
__global__ void __launch_bounds__(512) k_chol_pd_check(const double* L, int64_t ldl, int nb,
                                                       const double* cc, int64_t K0, int step,
                                                       double* v, int check, DevStatus* st) {
    __shared__ double cs[512];
    __shared__ double tv[512];
    if (st->info != 0) return;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
    if (check) {
        for (int p = t; p < nb; p += blockDim.x) {
            double s = 0.0;
            for (int q = p; q < nb; ++q) s += L[(int64_t)q * ldl + p];
            cs[p] = s;
        }
        __syncthreads();
        const double tau = st->tau;
        for (int j = warp; j < nb; j += nw) {
            double y = 0.0;
            for (int p = lane; p <= j; p += 32) y = fma(cs[p], L[(int64_t)j * ldl + p], y);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
            if (lane == 0) {
                double d = y - cc[j];
                if (!(fabs(d) <= tau)) {
                    atomicAdd(&st->detected, 1ull);
                    atomicAdd(&st->uncorrectable, 1ull);
                    record_event(st, step, EV_PD, K0 + j, K0 + j, d);
                }
            }
        }
    }
    if (v == nullptr) return;
    for (int p = t; p < nb; p += blockDim.x) tv[p] = 1.0;
    __syncthreads();
    for (int c1 = nb; c1 > 0; c1 -= 32) {
        const int c0 = c1 - 32 > 0 ? c1 - 32 : 0;
        if (warp == 0) {
            const int p = c0 + lane;
            double tp = (p < c1) ? tv[p] : 0.0;
            for (int j = c1 - 1; j >= c0; --j) {
                double tj = __shfl_sync(0xffffffffu, tp, j - c0);
                double vj = tj / L[(int64_t)j * ldl + j];
                if (p == j) tp = vj;
                if (p < j) tp -= L[(int64_t)j * ldl + p] * vj;
            }
            if (p < c1) tv[p] = tp;
        }
        __syncthreads();
        for (int p = t; p < c0; p += blockDim.x) {
            double s = tv[p];
            for (int j = c0; j < c1; ++j) s -= L[(int64_t)j * ldl + p] * tv[j];
            tv[p] = s;
        }
        __syncthreads();
    }
    for (int p = t; p < nb; p += blockDim.x) v[p] = tv[p];
}

}  // namespace

cudaError_t launch_potf2_small(double* A, int64_t lda, int64_t nb, int64_t info_base,
                               DevStatus* st, cudaStream_t s) {
    k_potf2_small<<<1, 256, 0, s>>>(A, lda, (int)nb, info_base, st);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_l_to_f32(const double* L, int64_t ldl, int64_t nb, float* Lf,
                            cudaStream_t s) {
    const int64_t tot = nb * nb;
    if (tot <= 0) return cudaSuccess;
    k_l_to_f32<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(L, ldl, (int)nb, Lf);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_trsm_rlt(const double* L, int64_t ldl, int64_t nb, const TrsmSeg* segs,
                            int nseg, const double* v, double* x, const DevStatus* st,
                            cudaStream_t s, bool f32, bool nt, const float* lf) {
    TrsmArgs a{};
    a.L = L;
    a.Lf = (f32 && !nt) ? lf : nullptr;
    a.ldl = ldl;
    a.nb = (int)nb;
    a.nseg = 0;
    int64_t total = 0;
    for (int i = 0; i < nseg; ++i) {
        if (segs[i].rows <= 0) {
            if (i == 0) v = nullptr;  // x belongs to segment 0
            continue;
        }
        a.seg[a.nseg] = segs[i];
        a.start[a.nseg] = total;
        total += (segs[i].rows + RB - 1) / RB;
        a.nseg++;
    }
    if (total == 0) return cudaSuccess;
    a.start[a.nseg] = total;
    a.v = v;
    a.x = x;
    a.st = st;
    static bool attr_set = false;
    if (!attr_set) {
        const int bd = (int)((RB * 513 + CW * (CW + 1)) * sizeof(double));
        const int bf = (int)((RB * 513 + CW * (CW + 1)) * sizeof(float));
        cudaError_t e = cudaFuncSetAttribute(k_trsm_rlt<double, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, bd);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_trsm_rlt<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bd);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_trsm_rlt<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bf);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const size_t sd = (size_t)(RB * (nb + 1) + CW * (CW + 1)) * sizeof(double);
    const size_t sf = (size_t)(RB * (nb + 1) + CW * (CW + 1)) * sizeof(float);
    if (nt) k_trsm_rlt<double, true><<<(unsigned)total, TT, sd, s>>>(a);
    else if (f32) k_trsm_rlt<float, false><<<(unsigned)total, TT, sf, s>>>(a);
    else k_trsm_rlt<double, false><<<(unsigned)total, TT, sd, s>>>(a);
    note_launch();
    return cudaGetLastError();
}

// X L^T = B for nb <= 64 with k_trsm_rows (f32: in FP32, the FP64 B and L
// rounded on load).
cudaError_t launch_trsm_rows(const double* L, int64_t ldl, int64_t nb, const TrsmSeg* segs,
                             int nseg, const DevStatus* st, cudaStream_t s, bool f32, bool rev) {
    if (nb <= 0) return cudaSuccess;
    if (nb > RW_MAXNB || nseg < 1 || nseg > 2) return cudaErrorInvalidValue;
    if (rev && (f32 || nb != RW_MAXNB)) return cudaErrorInvalidValue;
    TrsmArgs a{};
    a.rev = rev ? 1 : 0;
    a.L = L;
    a.ldl = ldl;
    a.nb = (int)nb;
    int64_t total = 0;
    for (int i = 0; i < nseg; ++i) {
        if (segs[i].rows <= 0) continue;
        a.seg[a.nseg] = segs[i];
        a.start[a.nseg] = total;
        total += (segs[i].rows + RW_ROWS - 1) / RW_ROWS;
        a.nseg++;
    }
    if (total == 0) return cudaSuccess;
    a.start[a.nseg] = total;
    a.st = st;
    if (!f32 && nb == RW_MAXNB) {   // two threads per row
        int64_t t2 = 0;
        for (int i = 0; i < a.nseg; ++i) {
            a.start[i] = t2;
            t2 += (a.seg[i].rows + RW2_ROWS - 1) / RW2_ROWS;
        }
        a.start[a.nseg] = t2;
        const size_t s2 = (size_t)(RW2_ROWS * RW_LD + RW_MAXNB * RW_LD + RW_MAXNB) * sizeof(double);
        static bool attr2 = false;
        if (!attr2) {
            cudaError_t e = cudaFuncSetAttribute(k_trsm_rows2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)s2);
            if (e != cudaSuccess) return e;
            attr2 = true;
        }
        k_trsm_rows2<<<(unsigned)t2, 2 * RW2_ROWS, s2, s>>>(a);
        note_launch();
        return cudaGetLastError();
    }
    const size_t sd = (size_t)(RW_ROWS * RW_LD + RW_MAXNB * RW_LD + RW_MAXNB) * sizeof(double);
    const size_t sf = (size_t)(RW_ROWS * RW_LD + RW_MAXNB * RW_LD + RW_MAXNB) * sizeof(float);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_trsm_rows<double>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sd);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_trsm_rows<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sf);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (f32) k_trsm_rows<float><<<(unsigned)total, RW_ROWS, sf, s>>>(a);
    else k_trsm_rows<double><<<(unsigned)total, RW_ROWS, sd, s>>>(a);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_chol_pd_check(const double* L, int64_t ldl, int64_t nb, const double* cc,
                                 int64_t K0, int step, double* v, int mode, DevStatus* st,
                                 cudaStream_t s) {
    k_chol_pd_check<<<1, 512, 0, s>>>(L, ldl, (int)nb, cc, K0, step, v, mode != MODE_NONE ? 1 : 0,
                                      st);
    note_launch();
    return cudaGetLastError();
}

}  // namespace abft
