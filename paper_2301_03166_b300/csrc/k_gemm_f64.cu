// k_gemm_f64.cu -- FP64 trailing-matrix update tiles (Sec. 2.1 TMU:
// A22 <- A22 - L21 U12; SYRK for Cholesky, GEMM for LU / QR) with the
// checksum rows and columns folded into the same launch (Sec. 3.1.2: the
// operation is applied to the checksums as well).
//
// B300 note: the FP64 pipe is ~2 DFMA/clk/SM (measured 1.13 TFLOP/s for the
// whole GPU) and mma.sync .f64 runs no faster than DFMA, so this kernel is a
// register-tiled DFMA kernel.  With 64x64 tiles the arithmetic intensity is
// 8 flop/B against HBM -- two orders of magnitude above the FP64 balance
// point -- so the only goal is to keep the DFMA pipe issuing every cycle.
//
// Operands may be row-major over K or K-major (A^T or B^T layouts).
// A launch carries up to three segments; CTAs are numbered over the 64x64
// tiles of segment 0, then 1, then 2.  Segment 0 is the main trailing block
// (with a lower-block mask for the symmetric update: diagonal blocks are
// updated in full), segments 1 and 2 are the checksum border rows and columns.
#include "common.cuh"

namespace abft {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NTH = 256;

struct GemmArgs {
    int kparts;         // split-K factor (1 = none)
    double* part;       // kparts x M x N partial products when kparts > 1
    GemmSeg seg[3];
    int64_t tn[3];      // tiles along N per segment
    int64_t start[4];   // first CTA of each segment
    int nseg;
    int ncf;
    ComputeFault cf[MAX_CF];
    const DevStatus* st;
};

// KMAJOR_A: 0 = A[i*lda + p]; 1 = A[p*lda + i]; 2 = the symmetric matrix
// A + A^T whose lower triangle (with the diagonal) is stored: element (i, p) is
// A[i][p] for p < i, A[p][i] for p > i, 2 A[i][i] on the diagonal.
// With kparts > 1 the CTA computes only its share of K and writes the partial
// product to part[kpart][i][j] (no mask, no faults); a reduce pass applies it.
template <int KMAJOR_A, int KMAJOR_B>
__global__ void __launch_bounds__(NTH) k_gemm_f64(GemmArgs args) {
    __shared__ double As[2][BK][BM + 1];
    __shared__ double Bs[2][BK][BN + 1];
    if (args.st && args.st->info != 0) return;
    const int64_t bid = blockIdx.x;
    int s = 0;
    while (s + 1 < args.nseg && bid >= args.start[s + 1]) ++s;
    const GemmSeg& g = args.seg[s];
    const int64_t local = bid - args.start[s];
    const int kpart = blockIdx.y;
    const int64_t kchunk = ((g.K + args.kparts - 1) / args.kparts + BK - 1) / BK * BK;
    const int64_t kbeg = kpart * kchunk;
    const int64_t kend = (kbeg + kchunk < g.K) ? kbeg + kchunk : g.K;
    const int64_t tm = local / args.tn[s], tn = local % args.tn[s];
    const int64_t i0 = tm * BM, j0 = tn * BN;
    if (g.g > 0) {
        int64_t rlast = (i0 + BM - 1 < g.M - 1 ? i0 + BM - 1 : g.M - 1) + g.row0;
        if (rlast / g.g < (j0 + g.col0) / g.g) return;
    }
    if (kbeg >= kend && args.kparts == 1) return;
    const int t = threadIdx.x;
    const int tx = t & 15, ty = t >> 4;
    // loader coordinates
    const int la_r = t >> 2, la_k = (t & 3) * 4;          // A (and NT B): 64 rows x 16 k
    const int lb_k = t >> 4, lb_c = (t & 15) * 4;         // NN B: 16 k x 64 cols
    double ra[4], rb[4];
    double acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;

    auto load = [&](int64_t k0) {
        if (KMAJOR_A == 1) {  // A[p*lda + i]
            const int64_t k = k0 + lb_k;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int64_t i = i0 + lb_c + u;
                ra[u] = (k < kend && i < g.M) ? g.A[k * g.lda + i] : 0.0;
            }
        } else if (KMAJOR_A == 2) {  // symmetric A + A^T from the lower triangle
            const int64_t ia = i0 + la_r;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int64_t k = k0 + la_k + u;
                double v = 0.0;
                if (ia < g.M && k < kend) {
                    if (k < ia) v = g.A[ia * g.lda + k];
                    else if (k > ia) v = g.A[k * g.lda + ia];
                    else v = 2.0 * g.A[ia * g.lda + k];
                }
                ra[u] = v;
            }
        } else {
            const int64_t ia = i0 + la_r;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int64_t k = k0 + la_k + u;
                ra[u] = (ia < g.M && k < kend) ? g.A[ia * g.lda + k] : 0.0;
            }
        }
        if (KMAJOR_B) {
            const int64_t k = k0 + lb_k;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int64_t j = j0 + lb_c + u;
                rb[u] = (k < kend && j < g.N) ? g.B[k * g.ldb + j] : 0.0;
            }
        } else {
            const int64_t jb = j0 + la_r;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int64_t k = k0 + la_k + u;
                rb[u] = (jb < g.N && k < kend) ? g.B[jb * g.ldb + k] : 0.0;
            }
        }
    };
    auto store = [&](int buf) {
        if (KMAJOR_A == 1) {
#pragma unroll
            for (int u = 0; u < 4; ++u) As[buf][lb_k][lb_c + u] = ra[u];
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) As[buf][la_k + u][la_r] = ra[u];
        }
        if (KMAJOR_B) {
#pragma unroll
            for (int u = 0; u < 4; ++u) Bs[buf][lb_k][lb_c + u] = rb[u];
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) Bs[buf][la_k + u][la_r] = rb[u];
        }
    };

    const int64_t nk = (kend - kbeg + BK - 1) / BK;
    if (nk > 0) {
    load(kbeg);
    store(0);
    __syncthreads();
    for (int64_t kt = 0; kt < nk; ++kt) {
        const int buf = (int)(kt & 1);
        if (kt + 1 < nk) load(kbeg + (kt + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[buf][kk][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[buf][kk][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        if (kt + 1 < nk) store(buf ^ 1);
        __syncthreads();
    }
    }
    if (args.kparts > 1) {
        double* P = args.part + (int64_t)kpart * g.M * g.N;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t i = i0 + ty + 16 * r;
            if (i >= g.M) continue;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t j = j0 + tx + 16 * c;
                if (j < g.N) P[i * g.N + j] = acc[r][c];
            }
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t i = i0 + ty + 16 * r;
        if (i >= g.M) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t j = j0 + tx + 16 * c;
            if (j >= g.N) continue;
            if (g.g > 0 && (i + g.row0) / g.g < (j + g.col0) / g.g) continue;
            double* p = g.C + i * g.ldc + j;
            double v = *p - acc[r][c];
            if (s == 0)
                for (int f = 0; f < args.ncf; ++f)
                    if (args.cf[f].row == i && args.cf[f].col == j) v += args.cf[f].delta;
            *p = v;
        }
    }
}

// C[i][j] -= sum_s part[s][i][j] (fixed order) under the lower-block mask.
__global__ void k_splitk_reduce(GemmSeg g, int kparts, const double* part) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= g.M * g.N) return;
    const int64_t i = e / g.N, j = e % g.N;
    if (g.g > 0 && (i + g.row0) / g.g < (j + g.col0) / g.g) return;
    double s = 0.0;
    for (int k = 0; k < kparts; ++k) s += part[(int64_t)k * g.M * g.N + e];
    g.C[i * g.ldc + j] -= s;
}

}  // namespace

cudaError_t launch_gemm_f64_splitk(const GemmSeg& seg, int a_kmajor, int b_kmajor, int kparts,
                                   double* part, const DevStatus* st, cudaStream_t s) {
    if (seg.M <= 0 || seg.N <= 0 || seg.K <= 0) return cudaSuccess;
    GemmArgs a{};
    a.kparts = kparts;
    a.part = part;
    a.nseg = 1;
    a.seg[0] = seg;
    a.tn[0] = (seg.N + BN - 1) / BN;
    a.start[0] = 0;
    const int64_t total = ((seg.M + BM - 1) / BM) * a.tn[0];
    a.start[1] = total;
    a.ncf = 0;
    a.st = st;
    dim3 grid((unsigned)total, (unsigned)kparts);
    if (a_kmajor == 1 && b_kmajor) k_gemm_f64<1, 1><<<grid, NTH, 0, s>>>(a);
    else if (a_kmajor == 2 && b_kmajor) k_gemm_f64<2, 1><<<grid, NTH, 0, s>>>(a);
    else if (a_kmajor == 1) k_gemm_f64<1, 0><<<grid, NTH, 0, s>>>(a);
    else if (b_kmajor) k_gemm_f64<0, 1><<<grid, NTH, 0, s>>>(a);
    else k_gemm_f64<0, 0><<<grid, NTH, 0, s>>>(a);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || kparts == 1) return e;
    const int64_t tot = seg.M * seg.N;
    k_splitk_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(seg, kparts, part);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gemm_f64(const GemmSeg* segs, int nseg, int a_kmajor, int b_kmajor,
                            const ComputeFault* cf, int ncf, const DevStatus* st, cudaStream_t s) {
    GemmArgs a{};
    a.kparts = 1;
    a.part = nullptr;
    a.nseg = 0;
    int64_t total = 0;
    for (int i = 0; i < nseg; ++i) {
        if (segs[i].M <= 0 || segs[i].N <= 0 || segs[i].K <= 0) continue;
        int k = a.nseg++;
        a.seg[k] = segs[i];
        int64_t tm = (segs[i].M + BM - 1) / BM;
        a.tn[k] = (segs[i].N + BN - 1) / BN;
        a.start[k] = total;
        total += tm * a.tn[k];
    }
    if (total == 0) return cudaSuccess;
    a.start[a.nseg] = total;
    a.ncf = 0;
    // compute faults are indexed in the coordinates of the caller's segment 0;
    // they only apply when segment 0 was kept
    if (nseg > 0 && segs[0].M > 0 && segs[0].N > 0 && segs[0].K > 0)
        for (int f = 0; f < ncf && f < MAX_CF; ++f) a.cf[a.ncf++] = cf[f];
    a.st = st;
    if (a_kmajor == 2 && b_kmajor) k_gemm_f64<2, 1><<<(unsigned)total, NTH, 0, s>>>(a);
    else if (a_kmajor && b_kmajor) k_gemm_f64<1, 1><<<(unsigned)total, NTH, 0, s>>>(a);
    else if (a_kmajor) k_gemm_f64<1, 0><<<(unsigned)total, NTH, 0, s>>>(a);
    else if (b_kmajor) k_gemm_f64<0, 1><<<(unsigned)total, NTH, 0, s>>>(a);
    else k_gemm_f64<0, 0><<<(unsigned)total, NTH, 0, s>>>(a);
    note_launch();
    return cudaGetLastError();
}

}  // namespace abft
