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
    GemmSeg seg[3];
    int64_t tn[3];      // tiles along N per segment
    int64_t start[4];   // first CTA of each segment
    int nseg;
    int ncf;
    ComputeFault cf[MAX_CF];
    const DevStatus* st;
};

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
    const int64_t tm = local / args.tn[s], tn = local % args.tn[s];
    const int64_t i0 = tm * BM, j0 = tn * BN;
    if (g.g > 0) {
        int64_t rlast = (i0 + BM - 1 < g.M - 1 ? i0 + BM - 1 : g.M - 1) + g.row0;
        if (rlast / g.g < (j0 + g.col0) / g.g) return;
    }
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
        if (KMAJOR_A) {  // A[p*lda + i]
            const int64_t k = k0 + lb_k;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int64_t i = i0 + lb_c + u;
                ra[u] = (k < g.K && i < g.M) ? g.A[k * g.lda + i] : 0.0;
            }
        } else {
            const int64_t ia = i0 + la_r;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int64_t k = k0 + la_k + u;
                ra[u] = (ia < g.M && k < g.K) ? g.A[ia * g.lda + k] : 0.0;
            }
        }
        if (KMAJOR_B) {
            const int64_t k = k0 + lb_k;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int64_t j = j0 + lb_c + u;
                rb[u] = (k < g.K && j < g.N) ? g.B[k * g.ldb + j] : 0.0;
            }
        } else {
            const int64_t jb = j0 + la_r;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int64_t k = k0 + la_k + u;
                rb[u] = (jb < g.N && k < g.K) ? g.B[jb * g.ldb + k] : 0.0;
            }
        }
    };
    auto store = [&](int buf) {
        if (KMAJOR_A) {
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

    const int64_t nk = (g.K + BK - 1) / BK;
    load(0);
    store(0);
    __syncthreads();
    for (int64_t kt = 0; kt < nk; ++kt) {
        const int buf = (int)(kt & 1);
        if (kt + 1 < nk) load((kt + 1) * BK);
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

}  // namespace

cudaError_t launch_gemm_f64(const GemmSeg* segs, int nseg, int a_kmajor, int b_kmajor,
                            const ComputeFault* cf, int ncf, const DevStatus* st, cudaStream_t s) {
    GemmArgs a{};
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
    if (a_kmajor && b_kmajor) k_gemm_f64<1, 1><<<(unsigned)total, NTH, 0, s>>>(a);
    else if (a_kmajor) k_gemm_f64<1, 0><<<(unsigned)total, NTH, 0, s>>>(a);
    else if (b_kmajor) k_gemm_f64<0, 1><<<(unsigned)total, NTH, 0, s>>>(a);
    else k_gemm_f64<0, 0><<<(unsigned)total, NTH, 0, s>>>(a);
    note_launch();
    return cudaGetLastError();
}

}  // namespace abft
