// k_mixed.cu -- mixed-precision trailing update of the ABFT Cholesky.
//
// The TMU C -= L_I L_J^T runs on the 5th-generation tensor cores: the panel
// is quantized per g-row tile with a power-of-two scale sigma_I (BF16: the
// tile maximum maps to at most 1; FP16: to at most 2^14), the products of the
// quantized operands accumulate in FP32 in tensor memory (tcgen05.mma
// kind::f16, M = N = 128, K = 16), and the epilogue applies
// C_f64 -= sigma_I sigma_J acc in FP64.  The checksum borders use the same
// quantized operands (their column sums t_I = 1^T Lq_I), so that the checksum
// relation holds up to the FP32 accumulation error only; they are small and
// run as an FP32 SIMT GEMM.  The panel solve runs in FP32 (k_trsm_rlt<float>),
// the diagonal-block factorization, verification and correction stay in FP64.
//
// Kernel anatomy: persistent, one CTA per SM (576 threads), the 128 x 128
// output tiles of the lower block triangle dealt round-robin to the CTAs:
//   warp 0   TMA producer: 128x64 BF16 boxes of A (rows i0..) and B (rows j0..)
//            with 128-byte swizzle into a 4-stage ring of shared buffers
//   warp 1   TMEM allocation (2 x 128 columns) and the single-thread MMA
//            issuer, alternating between the two accumulators so the next
//            tile's MMAs run while the previous tile drains;
//            tcgen05.commit releases each stage and signals the epilogue
//   warps 2-17 tcgen05.ld of the FP32 accumulator (warp w reads lane quarter
//            w % 4, column quarter (w - 2) / 4), staged in shared memory, the
//            accumulator released, then a coalesced FP64 read-modify-write
//            of C with the scales, 16 loads in flight per thread (sixteen
//            epilogue warps: the read-modify-write is latency-bound; eight
//            had made the BF16 solve at n = 16384 1.7 ms slower).
// Every mbarrier wait is bounded: on timeout the CTA records an error in the
// status block, skips the rest of its work, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cooperative_groups.h>
#include <math.h>

#include "common.cuh"
#include "fp_bits.cuh"
#include "tc_util.cuh"

namespace abft {

namespace cg = cooperative_groups;
using namespace tc;

namespace {

constexpr int TM = 128, TN = 128, KC = 64;
constexpr int STAGES = 4;
constexpr int HALF_BYTES = TM * KC * 2;              // one 128 x 64 16-bit box
constexpr int STAGE_BYTES = 2 * HALF_BYTES;          // A box + B box
constexpr int EPI_WARPS = 16;
constexpr int MIX_THREADS = 64 + EPI_WARPS * 32;     // producer, MMA, 16 epilogue warps
constexpr uint32_t TMEM_COLS = 256;                  // two 128-column FP32 accumulators
constexpr int STG_LD = TN + 1;                       // epilogue staging row stride (floats)
constexpr int STG_BYTES = TM * STG_LD * 4;
constexpr size_t MIX_SMEM = (size_t)STAGES * STAGE_BYTES + STG_BYTES + 1024 + 256;

struct MixArgs {
    double* C;
    int64_t ldc;
    int64_t M;          // trailing order
    int64_t K;          // panel width (multiple of 64)
    int64_t g, off;     // lower-block mask and scale index: tile-row of row i is (i + off) / g
    const double* sig;  // per tile-row scale (global tile-row index)
    int ncf;
    ComputeFault cf[MAX_CF];
    DevStatus* st;
    int64_t ntiles;     // tiles of the block pairs (r x r per block pair)
    int64_t r;          // 128-tiles per g
    int64_t o;          // triangle origin (a multiple of g)
    int strip;          // 1: only the first block column (all block rows), no triangle
    uint32_t idesc;
};

// Decode the idx-th tile of the lower block triangle: block pairs (BI >= BJ)
// in row-major order, r x r 128-tiles inside each g x g block pair.  (The
// epilogue widens FP32 to FP64 without the FP64 pipe: f32_to_f64_exact.)
__device__ __forceinline__ void lower_tile(int64_t idx, int64_t r, int64_t& ti, int64_t& tj) {
    const int64_t r2 = r * r, pair = idx / r2, sub = idx % r2;
    int64_t a = (int64_t)((sqrt(8.0 * (double)pair + 1.0) - 1.0) * 0.5);
    while (a * (a + 1) / 2 > pair) --a;
    while ((a + 1) * (a + 2) / 2 <= pair) ++a;
    const int64_t b = pair - a * (a + 1) / 2;
    ti = a * r + sub / r;
    tj = b * r + sub % r;
}

// The idx-th tile: of the lower block triangle of [o, M) (strip = 0), or of the
// first block column of [0, M) (strip = 1, the look-ahead part).
__device__ __forceinline__ void mix_tile(const MixArgs& a, int64_t idx, int64_t& ti, int64_t& tj) {
    if (a.strip) {
        const int64_t r2 = a.r * a.r, pair = idx / r2, sub = idx % r2;
        ti = pair * a.r + sub / a.r;
        tj = sub % a.r;
    } else {
        lower_tile(idx, a.r, ti, tj);
        ti += a.o / TM;
        tj += a.o / TM;
    }
}

// Persistent warp-specialized update: CTA c handles tiles c, c + G, c + 2G, ...
__global__ void __launch_bounds__(MIX_THREADS, 1) k_tmu_mixed(const __grid_constant__ CUtensorMap tmap,
                                                             MixArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    float* stg = (float*)(smem + STAGES * STAGE_BYTES);
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES + STG_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* accf = empty + STAGES;   // [2]
    uint64_t* acce = accf + 2;         // [2]
    uint32_t* tmem_slot = (uint32_t*)(acce + 2);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    if (a.st->info != 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], EPI_WARPS);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int nk = (int)(a.K / KC);
    const int64_t G = gridDim.x;

    if (warp == 0) {
        if (lane == 0) {   // TMA producer
            int64_t c = 0;
            for (int64_t idx = blockIdx.x; idx < a.ntiles && !*abort_flag; idx += G) {
                int64_t ti, tj;
                mix_tile(a, idx, ti, tj);
                if (ti * TM >= a.M || tj * TN >= a.M) continue;
                for (int kc = 0; kc < nk; ++kc, ++c) {
                    const int s = (int)(c % STAGES);
                    if (c >= STAGES && !mbar_wait(&empty[s], (uint32_t)(((c - STAGES) / STAGES) & 1))) {
                        *abort_flag = 1;
                        atomicExch(&a.st->error, 2);
                        break;
                    }
                    mbar_expect_tx(&full[s], STAGE_BYTES);
                    uint8_t* dst = smem + s * STAGE_BYTES;
                    tma_load_2d(dst, &tmap, &full[s], kc * KC, (int)(ti * TM));
                    tma_load_2d(dst + HALF_BYTES, &tmap, &full[s], kc * KC, (int)(tj * TN));
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            int64_t c = 0, it = 0;
            for (int64_t idx = blockIdx.x; idx < a.ntiles && !*abort_flag; idx += G) {
                int64_t ti, tj;
                mix_tile(a, idx, ti, tj);
                if (ti * TM >= a.M || tj * TN >= a.M) continue;
                const int b = (int)(it & 1);
                if (it >= 2 && !mbar_wait(&acce[b], (uint32_t)(((it >> 1) - 1) & 1))) {
                    *abort_flag = 1;
                    atomicExch(&a.st->error, 2);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dt = tmem + (uint32_t)(b * TN);
                bool ok = true;
                for (int kc = 0; kc < nk; ++kc, ++c) {
                    const int s = (int)(c % STAGES);
                    if (!mbar_wait(&full[s], (uint32_t)((c / STAGES) & 1))) {
                        *abort_flag = 1;
                        atomicExch(&a.st->error, 2);
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t abase = smem_u32(smem + s * STAGE_BYTES);
                    const uint32_t bbase = abase + HALF_BYTES;
#pragma unroll
                    for (int kk = 0; kk < KC / 16; ++kk)
                        mma_f16(dt, smem_desc(abase + kk * 32), smem_desc(bbase + kk * 32), a.idesc,
                                (kc | kk) != 0 ? 1u : 0u);
                    mma_commit(&empty[s]);
                }
                if (!ok) break;
                mma_commit(&accf[b]);
                ++it;
            }
        }
    } else {
        // epilogue warps: TMEM lane quarter q = warp % 4, column half h
        const int ew = warp - 2;               // 0 .. EPI_WARPS-1
        const int q = warp & 3;
        constexpr int CPW = TN / (EPI_WARPS / 4);   // accumulator columns drained per warp
        const int h = ew >> 2;                 // columns [CPW h, CPW h + CPW)
        int64_t it = 0;
        for (int64_t idx = blockIdx.x; idx < a.ntiles; idx += G) {
            int64_t ti, tj;
            mix_tile(a, idx, ti, tj);
            if (ti * TM >= a.M || tj * TN >= a.M) continue;
            const int b = (int)(it & 1);
            bool ok = !*abort_flag && mbar_wait(&accf[b], (uint32_t)((it >> 1) & 1));
            if (!ok) {
                *abort_flag = 1;
                atomicExch(&a.st->error, 2);
            } else {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int r = q * 32 + lane;
#pragma unroll
                for (int cc = 0; cc < CPW / 32; ++cc) {
                    uint32_t v[32];
                    const int col = h * CPW + cc * 32;
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * TN + col), v);
#pragma unroll
                    for (int u = 0; u < 32; ++u) stg[r * STG_LD + col + u] = __uint_as_float(v[u]);
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[b])) : "memory");
            }
            asm volatile("bar.sync 1, %0;" ::"r"(EPI_WARPS * 32) : "memory");
            if (!*abort_flag) {
                const int64_t i0 = ti * TM, j0 = tj * TN;
                // a 128 x 128 tile lies in one g x g block (g is a multiple of 128 and
                // the trailing matrix starts on a block boundary): one scale per tile
                const double sc = a.sig[(i0 + a.off) / a.g] * a.sig[(j0 + a.off) / a.g];
                // FP64 read-modify-write of the tile: warp ew takes rows
                // ew + 4 E g + E u (E = EPI_WARPS; groups g < NG, u < 4) x 128
                // columns; the next
                // group's 16 loads are issued before this group's FMAs and
                // stores (32 loads in flight per thread); C - sc * acc is one
                // FMA on the FP64 pipe per element
                constexpr int NG = TM / (EPI_WARPS * 4);
                double cv[2][4][TN / 32];
                auto load_group = [&](int gq, double (&c)[4][TN / 32]) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int64_t i = i0 + ew + 4 * EPI_WARPS * gq + EPI_WARPS * u;
#pragma unroll
                        for (int t4 = 0; t4 < TN / 32; ++t4) {
                            const int64_t j = j0 + lane + 32 * t4;
                            c[u][t4] = (i < a.M && j < a.M) ? a.C[i * a.ldc + j] : 0.0;
                        }
                    }
                };
                load_group(0, cv[0]);
#pragma unroll
                for (int gq = 0; gq < NG; ++gq) {
                    if (gq + 1 < NG) load_group(gq + 1, cv[(gq + 1) & 1]);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int rr = ew + 4 * EPI_WARPS * gq + EPI_WARPS * u;
                        const int64_t i = i0 + rr;
                        if (i >= a.M) continue;
#pragma unroll
                        for (int t4 = 0; t4 < TN / 32; ++t4) {
                            const int64_t j = j0 + lane + 32 * t4;
                            if (j >= a.M) continue;
                            const double x = f32_to_f64_exact(stg[rr * STG_LD + lane + 32 * t4]);
                            double v = fma(-sc, x, cv[gq & 1][u][t4]);
                            for (int f = 0; f < a.ncf; ++f)
                                if (a.cf[f].row == i && a.cf[f].col == j) v += a.cf[f].delta;
                            a.C[i * a.ldc + j] = v;
                        }
                    }
                }
            }
            asm volatile("bar.sync 1, %0;" ::"r"(EPI_WARPS * 32) : "memory");
            ++it;
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS));
    }
}

// Quantize the panel per g-row tile: sigma_I = 2^(ceil(log2 max|L_I|) - e_t),
// Lq = RN(L / sigma_I) in BF16 (e_t = 0) or FP16 (e_t = 14); t_I = 1^T Lq_I
// and (single-side mode) tw_I = (1..g)^T Lq_I, in FP64.
// One cluster of QCL CTAs per tile, each CTA a slab of g / QCL rows: the tile
// maximum and the column sums are combined in rank 0's shared memory (the
// slab partial sums in rank order).  The panel was just written by the panel
// solve, so both passes over it are served mostly from L2.
constexpr int QCL = 8;

template <bool BF16>
__global__ void __cluster_dims__(QCL, 1, 1) __launch_bounds__(256)
    k_quant_panel(const double* __restrict__ P, int64_t lda, int64_t T0, int64_t n, int kb,
                  int64_t g, int64_t I0, uint16_t* __restrict__ Lq, double* __restrict__ sig,
                  double* __restrict__ tsum, int64_t tstride, int weighted,
                  float* __restrict__ tsum32, float* __restrict__ tabs32) {
    extern __shared__ double qpart[];     // rank 0: [QCL][3][kb] slab column sums
    __shared__ double red[8];
    __shared__ double cmax[QCL];          // rank 0: slab maxima
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int t = threadIdx.x;
    const int64_t I = I0 + blockIdx.x / QCL;
    const int64_t r0 = I * g, r1 = (r0 + g < n) ? r0 + g : n;
    const int64_t rps = (g + QCL - 1) / QCL;
    const int64_t s0 = (r0 + rank * rps < r1) ? r0 + rank * rps : r1;
    const int64_t s1 = (s0 + rps < r1) ? s0 + rps : r1;
    double m = 0.0;
    for (int p = t; p < kb; p += 256) {
        for (int64_t r = s0; r < s1; r += 8) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = (r + u < s1) ? P[(r + u) * lda + p] : 0.0;
#pragma unroll
            for (int u = 0; u < 8; ++u) m = fmax(m, fabs(v[u]));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((t & 31) == 0) red[t >> 5] = m;
    __syncthreads();
    if (t == 0) {
        double mc = red[0];
        for (int w = 1; w < 8; ++w) mc = fmax(mc, red[w]);
        double* rc = cl.map_shared_rank(cmax, 0);
        rc[rank] = mc;
    }
    cl.sync();
    {
        const double* rc = cl.map_shared_rank(cmax, 0);
        m = rc[0];
        for (int c = 1; c < QCL; ++c) m = fmax(m, rc[c]);
    }
    int e2 = 0;
    const double f = frexp(m, &e2);                 // m = f 2^e2, f in [0.5, 1)
    const int cexp = (f == 0.5) ? e2 - 1 : e2;      // ceil(log2 m)
    const int ex = cexp - (BF16 ? 0 : 14);
    const double sigma = (m > 0.0) ? ldexp(1.0, ex) : 1.0;
    // x / sigma is exact scaling by a power of two; multiply by the exact
    // reciprocal unless it would leave the normal range
    const bool use_mul = m > 0.0 && ex > -1000 && ex < 1000;
    const double rsig = use_mul ? ldexp(1.0, -ex) : 1.0;
    double* qp = cl.map_shared_rank(qpart, 0);
    for (int p = t; p < kb; p += 256) {
        double s = 0.0, sw = 0.0, sa = 0.0;
        for (int64_t r = s0; r < s1; ++r) {
            const double x = use_mul ? P[r * lda + p] * rsig : P[r * lda + p] / sigma;
            double xq;
            uint16_t bits;
            if (BF16) {
                __nv_bfloat16 h = __double2bfloat16(x);
                bits = __bfloat16_as_ushort(h);
                xq = (double)__bfloat162float(h);
            } else {
                __half h = __double2half(x);
                bits = __half_as_ushort(h);
                xq = (double)__half2float(h);
            }
            Lq[(r - T0) * kb + p] = bits;
            s += xq;
            sw += (double)(r - r0 + 1) * xq;
            sa += fabs(xq);
        }
        qp[(3 * rank) * kb + p] = s;
        qp[(3 * rank + 1) * kb + p] = sw;
        qp[(3 * rank + 2) * kb + p] = sa;
    }
    cl.sync();
    if (rank != 0) return;
    if (t == 0) sig[I] = sigma;
    for (int p = t; p < kb; p += 256) {
        double s = 0.0, sw = 0.0, sa = 0.0;
        for (int c = 0; c < QCL; ++c) {
            s += qpart[(3 * c) * kb + p];
            sw += qpart[(3 * c + 1) * kb + p];
            sa += qpart[(3 * c + 2) * kb + p];
        }
        if (tabs32) tabs32[I * kb + p] = (float)sa;
        tsum[I * tstride + p] = s;
        if (weighted) tsum[I * tstride + kb + p] = sw;
        if (tsum32) {   // the FP32 operand of the border products, rounded once here
            tsum32[I * tstride + p] = (float)s;
            if (weighted) tsum32[I * tstride + kb + p] = (float)sw;
        }
    }
}

// Small FP32 GEMM for the checksum borders of the mixed update:
// C_f64[i][j] -= sr(i) sc(j) sum_p A[i][p] B[j][p], A rows FP64 (t sums) or
// 16-bit (the quantized panel), B likewise; sr / sc are tile scales.
struct BorderSeg {
    const void* A;      // rows of K
    int a_half;         // 1: A is 16-bit (BF16 / FP16 per `bf16`), 0: FP64, 2: FP32
    int64_t lda;
    const void* B;
    int b_half;
    int64_t ldb;
    double* C;
    int64_t ldc;
    int64_t M, N, K;
    // scale index of row i: (i + r_off) / r_div + r_base; of column j likewise
    int64_t r_off, r_div, r_base, c_off, c_div, c_base;
    int a_abs, b_abs;   // the abs-checksum products use |A| and |B|
    int plus;           // abs-checksums grow: C += instead of C -=
    float* C32;         // FP32 output instead of C (the abs-checksums)
};
constexpr int MAX_BSEG = 4;
struct BorderArgs {
    BorderSeg seg[MAX_BSEG];
    int64_t tn[MAX_BSEG], start[MAX_BSEG + 1];
    int nseg;
    int bf16;
    const double* sig;
    const DevStatus* st;
};

__device__ __forceinline__ float ld_op(const void* p, int half, int bf16, int64_t idx) {
    if (half == 2) return ((const float*)p)[idx];
    if (!half) return (float)((const double*)p)[idx];
    uint16_t b = ((const uint16_t*)p)[idx];
    return bf16 ? __bfloat162float(__ushort_as_bfloat16(b)) : __half2float(__ushort_as_half(b));
}

__global__ void __launch_bounds__(256) k_border_mixed(BorderArgs a) {
    __shared__ float As[16][65], Bs[16][65];
    if (a.st->info != 0) return;
    const int64_t bid = blockIdx.x;
    int s = 0;
    while (s + 1 < a.nseg && bid >= a.start[s + 1]) ++s;
    const BorderSeg& g = a.seg[s];
    const int64_t local = bid - a.start[s];
    const int64_t i0 = (local / a.tn[s]) * 64, j0 = (local % a.tn[s]) * 64;
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int lr = t >> 2, lk = (t & 3) * 4;
    float acc[4][4] = {};
    // the next K chunk's operands are loaded into registers while the current
    // chunk is multiplied from shared memory
    float pa[4], pb[4];
    auto fetch = [&](int64_t k0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t k = k0 + lk + u, i = i0 + lr, j = j0 + lr;
            pa[u] = (i < g.M && k < g.K) ? ld_op(g.A, g.a_half, a.bf16, i * g.lda + k) : 0.f;
            pb[u] = (j < g.N && k < g.K) ? ld_op(g.B, g.b_half, a.bf16, j * g.ldb + k) : 0.f;
            if (g.a_abs) pa[u] = fabsf(pa[u]);
            if (g.b_abs) pb[u] = fabsf(pb[u]);
        }
    };
    fetch(0);
    for (int64_t k0 = 0; k0 < g.K; k0 += 16) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            As[lk + u][lr] = pa[u];
            Bs[lk + u][lr] = pb[u];
        }
        __syncthreads();
        if (k0 + 16 < g.K) fetch(k0 + 16);
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float av[4], bv[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) av[r] = As[kk][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t i = i0 + ty + 16 * r;
        if (i >= g.M) continue;
        const double sr = a.sig[(i + g.r_off) / g.r_div + g.r_base];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t j = j0 + tx + 16 * c;
            if (j >= g.N) continue;
            const double sc = a.sig[(j + g.c_off) / g.c_div + g.c_base];
            if (g.C32) {   // abs-checksums: FP32 (they only scale a threshold)
                g.C32[i * g.ldc + j] += (float)(sr * sc) * acc[r][c];
                continue;
            }
            const double v = (sr * sc) * (double)acc[r][c];
            if (g.plus) g.C[i * g.ldc + j] += v;
            else g.C[i * g.ldc + j] -= v;
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t get_encoder() {
    if (g_encode) return cudaSuccess;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || fn == nullptr || q != cudaDriverEntryPointSuccess)
        return e != cudaSuccess ? e : cudaErrorNotSupported;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_quant_panel(const double* P, int64_t lda, int64_t T0, int64_t n, int64_t kb,
                               int64_t g, int64_t I0, int64_t I1, int bf16, uint16_t* Lq,
                               double* sig, double* tsum, int64_t tstride, int weighted,
                               cudaStream_t s, float* tsum32, float* tabs32) {
    if (I1 <= I0) return cudaSuccess;
    if (kb > 512) return cudaErrorInvalidValue;
    static bool attr = false;
    const size_t smem = sizeof(double) * 3 * QCL * 512;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_quant_panel<true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_quant_panel<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const size_t need = sizeof(double) * 3 * QCL * (size_t)kb;
    const unsigned grid = (unsigned)((I1 - I0) * QCL);
    if (bf16)
        k_quant_panel<true><<<grid, 256, need, s>>>(P, lda, T0, n, (int)kb, g, I0, Lq, sig, tsum,
                                                    tstride, weighted, tsum32, tabs32);
    else
        k_quant_panel<false><<<grid, 256, need, s>>>(P, lda, T0, n, (int)kb, g, I0, Lq, sig, tsum,
                                                     tstride, weighted, tsum32, tabs32);
    note_launch();
    return cudaGetLastError();
}

// C (m x m, trailing, FP64) -= sigma sigma^T o (Lq Lq^T) on the lower block
// triangle of [o, m) (strip = 0) or on the first block column (strip = 1);
// max_grid > 0 caps the persistent grid.
cudaError_t launch_tmu_mixed(const uint16_t* Lq, int64_t m, int64_t kb, int bf16, double* C,
                             int64_t ldc, int64_t g, int64_t off, const double* sig,
                             const ComputeFault* cf, int ncf, DevStatus* st, cudaStream_t s,
                             int64_t o, int strip, int max_grid) {
    if (m <= 0 || (!strip && o >= m)) return cudaSuccess;
    if (o % g != 0 || (strip && o != 0)) return cudaErrorInvalidValue;
    if (kb % KC != 0) return cudaErrorInvalidValue;
    cudaError_t e = get_encoder();
    if (e != cudaSuccess) return e;
    CUtensorMap map;
    cuuint64_t dims[2] = {(cuuint64_t)kb, (cuuint64_t)m};
    cuuint64_t strides[1] = {(cuuint64_t)kb * 2};
    cuuint32_t box[2] = {KC, TM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(&map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                          2, (void*)Lq, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        e = cudaFuncSetAttribute(k_tmu_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)MIX_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    MixArgs a{};
    a.C = C; a.ldc = ldc; a.M = m; a.K = kb; a.g = g; a.off = off; a.sig = sig; a.st = st;
    a.ncf = 0;
    for (int f = 0; f < ncf && f < MAX_CF; ++f) a.cf[a.ncf++] = cf[f];
    a.r = g / TM;
    a.o = o;
    a.strip = strip;
    if (strip) {
        a.ntiles = (m + g - 1) / g * a.r * a.r;
    } else {
        const int64_t q = (m - o + g - 1) / g;
        a.ntiles = q * (q + 1) / 2 * a.r * a.r;
    }
    // kind::f16 instruction descriptor: D F32 (bits 4-5), A/B format BF16 = 1 or
    // F16 = 0 (bits 7-9, 10-12), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
    const uint32_t fmt = bf16 ? 1u : 0u;
    a.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(TN >> 3) << 17) |
              ((uint32_t)(TM >> 4) << 24);
    int64_t grid = num_sms();
    if (max_grid > 0 && grid > max_grid) grid = max_grid;
    if (grid > a.ntiles) grid = a.ntiles;
    k_tmu_mixed<<<(unsigned)grid, MIX_THREADS, MIX_SMEM, s>>>(map, a);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_border_mixed(const BorderSegHost* segs, int nseg, int bf16, const double* sig,
                                const DevStatus* st, cudaStream_t s) {
    BorderArgs a{};
    a.bf16 = bf16;
    a.sig = sig;
    a.st = st;
    int64_t total = 0;
    a.nseg = 0;
    if (nseg > MAX_BSEG) return cudaErrorInvalidValue;
    for (int i = 0; i < nseg; ++i) {
        const BorderSegHost& h = segs[i];
        if (h.M <= 0 || h.N <= 0 || h.K <= 0) continue;
        BorderSeg& b = a.seg[a.nseg];
        b.A = h.A; b.a_half = h.a_half; b.lda = h.lda;
        b.B = h.B; b.b_half = h.b_half; b.ldb = h.ldb;
        b.C = h.C; b.ldc = h.ldc; b.M = h.M; b.N = h.N; b.K = h.K;
        b.r_off = h.r_off; b.r_div = h.r_div; b.r_base = h.r_base;
        b.c_off = h.c_off; b.c_div = h.c_div; b.c_base = h.c_base;
        b.a_abs = h.a_abs; b.b_abs = h.b_abs; b.plus = h.plus; b.C32 = h.C32;
        a.tn[a.nseg] = (h.N + 63) / 64;
        a.start[a.nseg] = total;
        total += ((h.M + 63) / 64) * a.tn[a.nseg];
        a.nseg++;
    }
    if (total == 0) return cudaSuccess;
    a.start[a.nseg] = total;
    k_border_mixed<<<(unsigned)total, 256, 0, s>>>(a);
    note_launch();
    return cudaGetLastError();
}

}  // namespace abft
