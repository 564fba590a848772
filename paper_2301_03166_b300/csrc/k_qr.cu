// k_qr.cu -- kernels of the blocked ABFT Householder QR (Sec. 2.1 PD / TMU;
// Sec. 3.1.2 checksums).  PD = geqr2 on the (n - K0) x kb panel (LAPACK larfg
// convention) as one cooperative launch, then the triangular factor T of the
// block reflector I - V T V^T; the TMU is three FP64 GEMM launches of
// k_gemm_f64 (W = V^T C, X = T^T W, C -= V X) issued by the host, or, in the
// FP64-accurate form, the same three products as exact BF16 slice products
// on the tensor cores (k_emu.cu).
#include <math.h>

#include "common.cuh"
#include "fp_bits.cuh"

namespace abft {

namespace {

constexpr int QT = 256;
constexpr int QMAXR = 1024;
constexpr int QT_PF = 8;   // partials per lane held by k_geqr2_smem's phase B (G <= 256)

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    return s;
}

// sum_{b<G} p[b * stride] in the order b = 0, 1, ..., with eight loads in
// flight (the partials live in L2; a load-add chain would pay its latency G times)
__device__ __forceinline__ double ordered_sum(const double* p, int64_t stride, unsigned G) {
    double s = 0.0;
    for (unsigned b = 0; b < G; b += 8) {
        double x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = (b + u < G) ? p[(int64_t)(b + u) * stride] : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (b + u < G) s += x[u];
    }
    return s;
}

// The same sum taken by one warp: lane l adds b = l, l + 32, ... in order, then
// an xor butterfly (a + b == b + a, so every lane ends with the same value, and
// every CTA that calls it on the same data gets the same bits).  The dependent
// FP64 chain is ceil(G/32) + 5 adds instead of G: on this FP64 pipe one
// warp-instruction occupies a sub-partition for tens of cycles, so a G-long
// chain per column was a large part of the panel's time.
__device__ __forceinline__ double warp_tree_sum(const double* p, int64_t stride, unsigned G) {
    const unsigned lane = threadIdx.x & 31;
    double s = 0.0;
    for (unsigned b = lane; b < G; b += 32) s += p[(int64_t)b * stride];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Cooperative geqr2 on the panel P (m x kb, row-major, ld lda).  part is a
// G x (kb + 1) scratch of per-CTA partial sums, wv a kb scratch for the
// reflector's row vector w, nrm receives the column norms before the PD.
// Each CTA owns a contiguous block of panel rows.  Per column j: (A) every
// CTA forms its partial |x(2:)|^2 and x(2:)^T a_c for c > j; grid barrier;
// (B) every CTA forms beta and tau from the partials (one warp tree, the
// same bits in every CTA), and the CTAs' warps share the reductions of the
// dot products into w; grid barrier; (C) every CTA scales its part of v and
// applies a_c -= tau v w_c to its rows.  The dot products and the update map
// threads to (column, row chunk) pairs, so that late columns keep every
// thread busy.
__global__ void __launch_bounds__(QT) k_geqr2_coop(double* P, int64_t lda, int64_t m, int kb,
                                                   double* tau, double* nrm, double* part,
                                                   double* wv, DevStatus* st) {
    __shared__ double red[QT / 32];
    __shared__ double wl[512];
    __shared__ double vloc[QMAXR];
    __shared__ double dpart[512];   // (row chunk, column) partial dot products
    __shared__ double s_sst;
    const unsigned G = gridDim.x;
    const int64_t R = (m + G - 1) / G;
    const int64_t r0 = blockIdx.x * R, r1 = (r0 + R < m) ? r0 + R : m;
    const int ld = kb + 1;
    double* mypart = part + (int64_t)blockIdx.x * ld;
    unsigned long long nbar = 0;   // grid barriers passed
    // column norms before the PD (for the norm-preservation check)
    for (int c = threadIdx.x; c < kb; c += QT) {
        double s = 0.0;
        for (int64_t i = r0; i < r1; ++i) s += P[i * lda + c] * P[i * lda + c];
        mypart[c] = s;
    }
    if (!grid_barrier(st, G, nbar)) return;
    if (blockIdx.x == 0)
        for (int c = threadIdx.x; c < kb; c += QT) {
            nrm[c] = sqrt(ordered_sum(part + c, ld, G));
        }
    if (!grid_barrier(st, G, nbar)) return;
    for (int j = 0; j < kb; ++j) {
        // A: partial |x(2:)|^2 and partial dots x(2:)^T P[:, c] over my rows i > j
        const int64_t ibeg = r0 > j + 1 ? r0 : j + 1;
        double ss = 0.0;
        for (int64_t i = ibeg + threadIdx.x; i < r1; i += QT) {
            double x = P[i * lda + j];
            ss += x * x;
        }
        ss = block_sum(ss, red);
        if (threadIdx.x == 0) mypart[0] = ss;
        {
            // x(2:)^T a_c: thread t takes column j + 1 + t % w over row chunk t / w
            // (rows split when fewer columns than threads remain), eight rows of
            // operands loaded ahead and accumulated in row order; the chunks'
            // partial sums are then added in chunk order
            const int w = kb - j - 1;
            const int64_t nrow = r1 - ibeg;
            int rsp = w > 0 ? QT / w : 1;
            if ((int64_t)rsp > (nrow + 7) / 8) rsp = (int)((nrow + 7) / 8);
            if (rsp < 1) rsp = 1;
            const int64_t rch = (nrow + rsp - 1) / rsp;
            for (int t = threadIdx.x; t < w * rsp; t += QT) {
                const int c = j + 1 + t % w;
                const int64_t ia = ibeg + (int64_t)(t / w) * rch;
                const int64_t ie = ia + rch < r1 ? ia + rch : r1;
                double d = 0.0;
                for (int64_t i = ia; i < ie; i += 8) {
                    double xv[8], av[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (i + u < ie) { xv[u] = P[(i + u) * lda + j]; av[u] = P[(i + u) * lda + c]; }
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (i + u < ie) d += xv[u] * av[u];
                }
                dpart[t] = d;
            }
            __syncthreads();
            for (int c = j + 1 + threadIdx.x; c < kb; c += QT) {
                double d = 0.0;
                for (int q = 0; q < rsp; ++q) d += dpart[q * w + (c - j - 1)];
                mypart[1 + c] = d;
            }
        }
        if (!grid_barrier(st, G, nbar)) return;
        // B: every CTA forms beta, tau; warp q of CTA b reduces the dots of
        // columns c = j + 1 + 8 b + q, then + 8 G, ...
        if (threadIdx.x < 32) {
            const double t = warp_tree_sum(part, ld, G);
            if (threadIdx.x == 0) s_sst = t;
        }
        __syncthreads();
        const double sst = s_sst;
        const double alpha = P[(int64_t)j * lda + j];
        double tj = 0.0, beta = alpha, scal = 1.0;
        if (sst != 0.0) {
            double nr = sqrt(alpha * alpha + sst);
            beta = alpha >= 0.0 ? -nr : nr;
            tj = (beta - alpha) / beta;
            scal = alpha - beta;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) tau[j] = tj;
        if (tj != 0.0) {
            const int nw = QT / 32;
            for (int c = j + 1 + (int)blockIdx.x * nw + (int)(threadIdx.x >> 5); c < kb;
                 c += (int)G * nw) {
                const double d = warp_tree_sum(part + 1 + c, ld, G);
                if ((threadIdx.x & 31) == 0) wv[c] = P[(int64_t)j * lda + c] + d / scal;
            }
        }
        if (!grid_barrier(st, G, nbar)) return;
        // C: v_i = x_i / (alpha - beta); a -= tau v w on my rows
        if (tj == 0.0) continue;
        for (int c = j + 1 + threadIdx.x; c < kb; c += QT) wl[c] = wv[c];
        for (int64_t i = ibeg + threadIdx.x; i < r1; i += QT) {
            double v = P[i * lda + j] / scal;
            P[i * lda + j] = v;
            vloc[i - r0] = __dmul_rn(tj, v);  // tau_j v_i, once per row
        }
        __syncthreads();
        const int w = kb - j - 1;
        if (w > 0) {
            // thread t: column j + 1 + t % w, row chunk t / w (rows split when
            // there are fewer columns than threads), eight rows at a time
            // (coalesced along the rows, eight loads in flight)
            const int64_t nrow = r1 - ibeg;
            int rsp = QT / w;
            if ((int64_t)rsp > (nrow + 7) / 8) rsp = (int)((nrow + 7) / 8);
            if (rsp < 1) rsp = 1;
            const int64_t rch = (nrow + rsp - 1) / rsp;
            for (int t = threadIdx.x; t < w * rsp && ibeg < r1; t += QT) {
                const int c = j + 1 + t % w;
                const int64_t ia = ibeg + (int64_t)(t / w) * rch;
                const int64_t ie = ia + rch < r1 ? ia + rch : r1;
                const double wc = wl[c];
                for (int64_t i = ia; i < ie; i += 8) {
                    double av[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (i + u < ie) av[u] = P[(i + u) * lda + c];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (i + u < ie)
                            P[(i + u) * lda + c] = fma(-vloc[i + u - r0], wc, av[u]);
                }
            }
            if (j >= r0 && j < r1)
                for (int c = j + 1 + threadIdx.x; c < kb; c += QT) {
                    double* a = P + (int64_t)j * lda + c;
                    *a = __dsub_rn(*a, __dmul_rn(tj, wl[c]));
                }
        }
        if (threadIdx.x == 0 && j >= r0 && j < r1) P[(int64_t)j * lda + j] = beta;
        __syncthreads();
    }
}

// k_geqr2_coop with the CTA's rows r0 .. r1 - 1 of the panel in shared memory
// (sp[(i - r0) kb + c]), then vloc[R] and wl[kb]: the norms, the partial dot
// products, the scaling and the update read and write shared memory, and only
// the partial sums, w and the current row j (published by its owner before
// the first barrier of column j) go through global memory.  The same CTA
// count, row chunks and operation order as k_geqr2_coop: identical panels.
__global__ void __launch_bounds__(QT) k_geqr2_smem(double* P, int64_t lda, int64_t m, int kb,
                                                   double* tau, double* nrm, double* part,
                                                   double* wv, DevStatus* st) {
    extern __shared__ double qsm[];
    __shared__ double red[QT / 32];
    __shared__ double dpart[QT];    // (row chunk, column) partial dot products
    __shared__ double s_sst;
    const unsigned G = gridDim.x;
    const int64_t R = (m + G - 1) / G;
    const int64_t r0 = blockIdx.x * R < m ? blockIdx.x * R : m;
    const int64_t r1 = (r0 + R < m) ? r0 + R : m;
    const int ld = kb + 1;          // row stride of part
    double* sp = qsm;
    double* vloc = qsm + (size_t)R * kb;
    double* wl = vloc + R;
    double* mypart = part + (int64_t)blockIdx.x * ld;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t r = warp; r < r1 - r0; r += QT / 32)
        for (int c = lane; c < kb; c += 32) sp[r * kb + c] = P[(r0 + r) * lda + c];
    __syncthreads();
#define SP(i, c) sp[((i) - r0) * kb + (c)]
    unsigned long long nbar = 0;   // grid barriers passed
    // column norms before the PD (for the norm-preservation check)
    for (int c = threadIdx.x; c < kb; c += QT) {
        double s = 0.0;
        for (int64_t i = r0; i < r1; ++i) s += SP(i, c) * SP(i, c);
        mypart[c] = s;
    }
    if (!grid_barrier(st, G, nbar)) return;
    if (blockIdx.x == 0)
        for (int c = threadIdx.x; c < kb; c += QT) {
            nrm[c] = sqrt(ordered_sum(part + c, ld, G));
        }
    if (!grid_barrier(st, G, nbar)) return;
    for (int j = 0; j < kb; ++j) {
        // row j as it stands, for every CTA's beta, tau and w
        if (j >= r0 && j < r1)
            for (int c = j + threadIdx.x; c < kb; c += QT) P[(int64_t)j * lda + c] = SP(j, c);
        // A: partial |x(2:)|^2 and partial dots x(2:)^T P[:, c] over my rows i > j
        const int64_t ibeg = r0 > j + 1 ? r0 : j + 1;
        double ss = 0.0;
        for (int64_t i = ibeg + threadIdx.x; i < r1; i += QT) {
            double x = SP(i, j);
            ss += x * x;
        }
        ss = block_sum(ss, red);
        if (threadIdx.x == 0) mypart[0] = ss;
        {
            const int w = kb - j - 1;
            const int64_t nrow = r1 - ibeg;
            int rsp = w > 0 ? QT / w : 1;
            if ((int64_t)rsp > (nrow + 7) / 8) rsp = (int)((nrow + 7) / 8);
            if (rsp < 1) rsp = 1;
            const int64_t rch = (nrow + rsp - 1) / rsp;
            for (int t = threadIdx.x; t < w * rsp; t += QT) {
                const int c = j + 1 + t % w;
                const int64_t ia = ibeg + (int64_t)(t / w) * rch;
                const int64_t ie = ia + rch < r1 ? ia + rch : r1;
                double d = 0.0;
                for (int64_t i = ia; i < ie; i += 8) {
                    double xv[8], av[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (i + u < ie) { xv[u] = SP(i + u, j); av[u] = SP(i + u, c); }
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (i + u < ie) d += xv[u] * av[u];
                }
                dpart[t] = d;
            }
            __syncthreads();
            for (int c = j + 1 + threadIdx.x; c < kb; c += QT) {
                double d = 0.0;
                for (int q = 0; q < rsp; ++q) d += dpart[q * w + (c - j - 1)];
                mypart[1 + c] = d;
            }
        }
        if (!grid_barrier(st, G, nbar)) return;
        // B: every CTA forms beta, tau; warp q of CTA b reduces the dots of
        // columns c = j + 1 + 8 b + q, then + 8 G, ...  Every load of this phase
        // (the |x|^2 partials, alpha, the first column's dot partials and a_jc)
        // is issued before the first sum, and each sum adds its values in the
        // order of warp_tree_sum, so the results are those of k_geqr2_coop
        const int nw = QT / 32;
        const int c1 = j + 1 + (int)blockIdx.x * nw + warp;   // this warp's first column
        double sv[QT_PF], dv[QT_PF];
#pragma unroll
        for (int q = 0; q < QT_PF; ++q) {
            const unsigned bq = lane + 32u * q;
            sv[q] = (warp == 0 && bq < G) ? part[(int64_t)bq * ld] : 0.0;
            dv[q] = (c1 < kb && bq < G) ? part[(int64_t)bq * ld + 1 + c1] : 0.0;
        }
        const double alpha = P[(int64_t)j * lda + j];
        const double ajc1 = c1 < kb ? P[(int64_t)j * lda + c1] : 0.0;
        if (warp == 0) {
            double t = 0.0;
#pragma unroll
            for (int q = 0; q < QT_PF; ++q)
                if (lane + 32u * q < G) t += sv[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) s_sst = t;
        }
        __syncthreads();
        const double sst = s_sst;
        double tj = 0.0, beta = alpha, scal = 1.0;
        if (sst != 0.0) {
            double nr = sqrt(alpha * alpha + sst);
            beta = alpha >= 0.0 ? -nr : nr;
            tj = (beta - alpha) / beta;
            scal = alpha - beta;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) tau[j] = tj;
        if (tj != 0.0) {
            if (c1 < kb) {
                double d = 0.0;
#pragma unroll
                for (int q = 0; q < QT_PF; ++q)
                    if (lane + 32u * q < G) d += dv[q];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
                if (lane == 0) wv[c1] = ajc1 + d / scal;
            }
            for (int c = c1 + (int)G * nw; c < kb; c += (int)G * nw) {
                const double d = warp_tree_sum(part + 1 + c, ld, G);
                if (lane == 0) wv[c] = P[(int64_t)j * lda + c] + d / scal;
            }
        }
        if (!grid_barrier(st, G, nbar)) return;
        // C: v_i = x_i / (alpha - beta); a -= tau v w on my rows
        if (tj == 0.0) continue;
        for (int c = j + 1 + threadIdx.x; c < kb; c += QT) wl[c] = wv[c];
        for (int64_t i = ibeg + threadIdx.x; i < r1; i += QT) {
            double v = SP(i, j) / scal;
            SP(i, j) = v;
            vloc[i - r0] = __dmul_rn(tj, v);  // tau_j v_i, once per row
        }
        __syncthreads();
        const int w = kb - j - 1;
        if (w > 0) {
            const int64_t nrow = r1 - ibeg;
            int rsp = QT / w;
            if ((int64_t)rsp > (nrow + 7) / 8) rsp = (int)((nrow + 7) / 8);
            if (rsp < 1) rsp = 1;
            const int64_t rch = (nrow + rsp - 1) / rsp;
            for (int t = threadIdx.x; t < w * rsp && ibeg < r1; t += QT) {
                const int c = j + 1 + t % w;
                const int64_t ia = ibeg + (int64_t)(t / w) * rch;
                const int64_t ie = ia + rch < r1 ? ia + rch : r1;
                const double wc = wl[c];
                for (int64_t i = ia; i < ie; ++i) SP(i, c) = fma(-vloc[i - r0], wc, SP(i, c));
            }
            if (j >= r0 && j < r1)
                for (int c = j + 1 + threadIdx.x; c < kb; c += QT)
                    SP(j, c) = __dsub_rn(SP(j, c), __dmul_rn(tj, wl[c]));
        }
        if (threadIdx.x == 0 && j >= r0 && j < r1) SP(j, j) = beta;
        __syncthreads();
    }
    for (int64_t r = warp; r < r1 - r0; r += QT / 32)
        for (int c = lane; c < kb; c += 32) P[(r0 + r) * lda + c] = sp[r * kb + c];
#undef SP
}

// PD check: column norms preserved, ||R[0:j+1, j]|| vs the norm before the PD.
__global__ void k_qr_pd_check(const double* P, int64_t lda, int kb, const double* nrm, int step,
                              int64_t K0, DevStatus* st) {
    const double tau = st->tau;
    for (int j = threadIdx.x; j < kb; j += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i <= j; ++i) s += P[(int64_t)i * lda + j] * P[(int64_t)i * lda + j];
        double d = sqrt(s) - nrm[j];
        if (!(fabs(d) <= tau)) {
            atomicAdd(&st->detected, 1ull);
            atomicAdd(&st->uncorrectable, 1ull);
            record_event(st, step, EV_PD, K0 + j, K0 + j, d);
        }
    }
}

// V (unit lower trapezoidal, explicit ones and zeros) from the panel, and the
// border rows 1^T V_I (and weighted) per tile-row I >= k.
__global__ void k_qr_prep_v(const double* P, int64_t lda, int64_t m, int kb, double* V) {
    const int64_t tot = m * kb;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e / kb;
        int q = (int)(e % kb);
        V[e] = (i == q) ? 1.0 : (i < q ? 0.0 : P[i * lda + q]);
    }
}

__global__ void k_qr_vsums(const double* V, int64_t m, int kb, int64_t g, int64_t k, int64_t K0,
                           double* CS, int64_t ldcs, int64_t nc, int mode) {
    const int64_t I = k + blockIdx.x;
    const int64_t gr0 = I * g, gr1 = (gr0 + g < K0 + m) ? gr0 + g : K0 + m;
    for (int q = threadIdx.x; q < kb; q += blockDim.x) {
        double s = 0.0, sw = 0.0;
        for (int64_t gi = gr0; gi < gr1; ++gi) {
            double v = V[(gi - K0) * kb + q];
            s += v;
            sw += (double)(gi - gr0 + 1) * v;
        }
        CS[(I * nc) * ldcs + K0 + q] = s;
        if (mode == MODE_SINGLE) CS[(I * nc + 1) * ldcs + K0 + q] = sw;
    }
}

// larft (forward, columnwise) from Gneg = -V^T V: T[j][j] = tau_j,
// T[0:j, j] = -tau_j T[0:j, 0:j] (V^T v_j)[0:j].  One CTA, columns in order.
// T of the compact WY form: T(j, j) = tau_j and, for i < j,
// T(i, j) = -tau_j sum_{q=i}^{j-1} T(i, q) (V^T V)(q, j)  (Gneg = -V^T V).
// Row i depends on nothing but its own earlier entries, so one warp takes one
// row: lane l keeps the running sums S_j of the columns j = l, l + 32, ...
// and, as soon as T(i, q) is final, adds T(i, q) (V^T V)(q, j) to every S_j,
// j > q -- the terms of each sum in the order q = i, i + 1, ..., as a
// column-by-column evaluation takes them, and row q of Gneg read contiguously.
constexpr int LARFT_W = 4;   // rows (warps) per CTA
__global__ void __launch_bounds__(32 * LARFT_W) k_larft(const double* Gneg, int kb,
                                                       const double* tau, double* T) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * LARFT_W + (threadIdx.x >> 5);
    if (i >= kb) return;
    double S[16];   // kb <= 512
#pragma unroll
    for (int t = 0; t < 16; ++t) S[t] = 0.0;
    double* Ti = T + (int64_t)i * kb;
    for (int j = lane; j < i; j += 32) Ti[j] = 0.0;
    for (int q = i; q < kb; ++q) {
        // T(i, q): the diagonal, or -tau_q times the finished sum S_q
        const int own = q & 31, slot = q >> 5;
        double mine = 0.0;
#pragma unroll
        for (int t = 0; t < 16; ++t)
            if (t == slot) mine = S[t];
        const double sq = __shfl_sync(0xffffffffu, mine, own);
        const double tq = tau[q];
        const double tiq = (q == i) ? tq : -tq * sq;
        if (lane == own) Ti[q] = tiq;
        const double* Gq = Gneg + (int64_t)q * kb;
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int j = lane + 32 * t;
            if (j > q && j < kb) S[t] = fma(tiq, -Gq[j], S[t]);
        }
    }
}

__global__ void k_colnorm_max(const double* A, int64_t lda, int64_t n, DevStatus* st) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double s = 0.0;
    if (c < n)
        for (int64_t i = 0; i < n; ++i) s += A[i * lda + c] * A[i * lda + c];
    double v = sqrt(s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg((unsigned long long*)&st->amax, v);
}

__global__ void k_set_tau(double tau_scale, int64_t n, int64_t g, DevStatus* st) {
    double t = tau_scale * 8.0;
    t *= 0x1p-53;
    t *= (double)n;
    t *= (double)g;
    t *= st->amax;
    st->tau = t;
    // fixed-point bound of the verify sums: orthogonal updates keep every
    // column's norm, so no trailing entry exceeds the largest column norm
    // (twice it, for rounding)
    const double bnd = 2.0 * st->amax;
    const int ve = (int)((__double_as_longlong(bnd) >> 52) & 0x7ff);
    st->vexp = (bnd > 0.0 && bnd < 1e300 && ve >= kFixedMinExp) ? ve : 0;
}

}  // namespace

cudaError_t launch_geqr2_coop(double* P, int64_t lda, int64_t m, int64_t kb, double* tau,
                              double* nrm, double* part, double* wv, DevStatus* st,
                              cudaStream_t s) {
    int64_t want = (m + 63) / 64;
    int64_t G = want < num_sms() ? want : num_sms();
    if (G < 1) G = 1;
    while ((m + G - 1) / G > QMAXR) ++G;
    if (G > num_sms()) return cudaErrorInvalidValue;
    int kbi = (int)kb;
    cudaError_t e0 = cudaMemsetAsync(&st->bar_count, 0, sizeof(st->bar_count), s);
    if (e0 != cudaSuccess) return e0;
    void* args[] = {&P, &lda, &m, &kbi, &tau, &nrm, &part, &wv, &st};
    // the rows of every CTA in shared memory when they fit (with the kernel's
    // static shared memory, about 2.2 KB)
    static int cap = -1, attr = -1;
    if (cap < 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            v = 0;
        cap = v;
    }
    const int64_t R = (m + G - 1) / G;
    const size_t sm = sizeof(double) * ((size_t)R * (size_t)kb + (size_t)R + (size_t)kb);
    if (kb <= 512 && G <= 32 * QT_PF && sm + 2304 <= (size_t)cap) {
        if ((int)sm > attr) {
            cudaError_t ea = cudaFuncSetAttribute(k_geqr2_smem,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (ea != cudaSuccess) return ea;
            attr = (int)sm;
        }
        cudaError_t e = cudaLaunchCooperativeKernel((void*)k_geqr2_smem, dim3((unsigned)G),
                                                    dim3(QT), args, sm, s);
        note_launch();
        return e;
    }
    cudaError_t e = cudaLaunchCooperativeKernel((void*)k_geqr2_coop, dim3((unsigned)G), dim3(QT),
                                                args, 0, s);
    note_launch();
    return e;
}

cudaError_t launch_qr_pd_check(const double* P, int64_t lda, int64_t kb, const double* nrm,
                               int step, int64_t K0, DevStatus* st, cudaStream_t s) {
    k_qr_pd_check<<<1, 512, 0, s>>>(P, lda, (int)kb, nrm, step, K0, st);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_qr_prep_v(const double* P, int64_t lda, int64_t m, int64_t kb, double* V,
                             cudaStream_t s) {
    int64_t blocks = (m * kb + 255) / 256;
    if (blocks > 8 * num_sms()) blocks = 8 * num_sms();
    k_qr_prep_v<<<(unsigned)blocks, 256, 0, s>>>(P, lda, m, (int)kb, V);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_qr_vsums(const double* V, int64_t m, int64_t kb, int64_t g, int64_t k,
                            int64_t nt, int64_t K0, double* CS, int64_t ldcs, int64_t nc, int mode,
                            cudaStream_t s) {
    k_qr_vsums<<<(unsigned)(nt - k), 256, 0, s>>>(V, m, (int)kb, g, k, K0, CS, ldcs, nc, mode);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_larft(const double* Gneg, int64_t kb, const double* tau, double* T,
                         cudaStream_t s) {
    if (kb > 512) return cudaErrorInvalidValue;
    k_larft<<<(unsigned)((kb + LARFT_W - 1) / LARFT_W), 32 * LARFT_W, 0, s>>>(Gneg, (int)kb, tau,
                                                                           T);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_qr_tau(const double* A, int64_t lda, int64_t n, int64_t g, double tau_scale,
                          DevStatus* st, cudaStream_t s) {
    k_colnorm_max<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(A, lda, n, st);
    note_launch();
    k_set_tau<<<1, 1, 0, s>>>(tau_scale, n, g, st);
    note_launch();
    return cudaGetLastError();
}

}  // namespace abft
