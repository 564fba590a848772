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
#include <algorithm>
#include <climits>
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

// exponent of a power of two (sigma), or INT_MIN for 0 / Inf / NaN / subnormal
__device__ __forceinline__ int pow2_exp(double s) {
    const int e = (__double2hiint(s) >> 20) & 0x7ff;
    return (e == 0 || e == 0x7ff) ? INT_MIN : e - 1023;
}

// x 2^e (|e| < 1000, so 2^e is a normal double): by exponent arithmetic when
// x and the result are normal, else as the FP64 product with 2^e
__device__ __forceinline__ double scale_f64(double x, int e) {
    const int hi = __double2hiint(x);
    const int ex = (hi >> 20) & 0x7ff;
    if (ex != 0 && ex != 0x7ff && ex + e > 0 && ex + e < 0x7ff)
        return __hiloint2double(hi + (e << 20), __double2loint(x));
    return x * __hiloint2double((e + 1023) << 20, 0);
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
    // the largest |x| by an integer maximum of the bit patterns of |x| (the
    // order of non-negative doubles), NaN ignored as fmax ignores it: no FP64
    // pipe instruction per element
    unsigned long long mbits = 0ull;
    for (int p = t; p < kb; p += 256) {
        for (int64_t r = s0; r < s1; r += 8) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = (r + u < s1) ? P[(r + u) * lda + p] : 0.0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                unsigned long long a = (unsigned long long)__double_as_longlong(v[u]) &
                                       0x7fffffffffffffffull;
                if (a > 0x7ff0000000000000ull) a = 0ull;
                mbits = a > mbits ? a : mbits;
            }
        }
    }
    double m = __longlong_as_double((long long)mbits);
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
    // x / sigma is exact scaling by a power of two: x 2^-ex (exponent
    // arithmetic, scale_f64) unless 2^-ex would leave the normal range
    const bool use_mul = m > 0.0 && ex > -1000 && ex < 1000;
    double* qp = cl.map_shared_rank(qpart, 0);
    // FP64-pipe work per element (slow on B300): the rounding to 16 bits and
    // the sums.  The power-of-two scaling is an exponent addition and the
    // 16-bit value is widened to FP64 with integer operations (the same
    // values as the FP64 product and conversion); the weighted sums are formed
    // only where they are kept.
    for (int p = t; p < kb; p += 256) {
        double s = 0.0, sw = 0.0, sa = 0.0;
        for (int64_t r = s0; r < s1; ++r) {
            const double x = use_mul ? scale_f64(P[r * lda + p], -ex) : P[r * lda + p] / sigma;
            double xq;
            uint16_t bits;
            bool okr;
            // round to nearest even in 16 bits by integer operations (the
            // conversion instruction runs on the FP64 pipe); NaN, infinities
            // and overflow take the instruction
            if (BF16) {
                uint32_t b16 = f64_to_small_rn<8, 7>(x, okr);
                if (!okr) b16 = __bfloat16_as_ushort(__double2bfloat16(x));
                bits = (uint16_t)b16;
                xq = f32_to_f64_exact(__uint_as_float(b16 << 16));
            } else {
                uint32_t b16 = f64_to_small_rn<5, 10>(x, okr);
                if (!okr) b16 = __half_as_ushort(__double2half(x));
                bits = (uint16_t)b16;
                xq = f32_to_f64_exact(__half2float(__ushort_as_half((unsigned short)b16)));
            }
            Lq[(r - T0) * kb + p] = bits;
            s += xq;
            if (weighted) sw += (double)(r - r0 + 1) * xq;
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

// Checksum borders of the mixed update.  Every border product is a dot
// product of one trailing panel row Lq_j (16-bit, K values) with one checksum
// vector of a block J: the column sums t_J and weighted sums tw_J (FP32,
// signed) or the abs sums 1^T |Lq_J| (FP32, against |Lq_j|).  By the symmetry
// of L L^T the column-checksum rows (c_J -= sigma_J sigma_I t_J Lq_j^T, for
// the columns j of the part) and the row-checksum columns (r_I -= sigma_I
// sigma_J Lq_j t_J^T, for the blocks J of the part) are the same dot
// products, so each is computed once and written to both borders.
// A job is a range of panel rows times a range of vectors of one kind; a CTA
// computes an RT x VC tile of it as an FP32 SIMT GEMM over K in chunks of 32
// (the next chunk copied by cp.async while this one is multiplied, the 16-bit
// rows widened to FP32 in shared memory), every dot product summed with fmaf
// in order of increasing k.
// The scales are powers of two: sigma_I sigma_J acc is formed by exponent
// arithmetic, so the epilogue's only FP64 operation is the update of C.
struct BJob {
    int64_t r0, r1;     // panel rows [r0, r1)
    int v0, v1;         // vectors [v0, v1) of the kind's list
    int vstep;          // list index v is vector u = v vstep (2: plain sums only)
    int kind;           // 0: signed (t, tw), 1: abs
    int cfg;            // tile shape (BCfg)
    int64_t nvc;        // vector chunks
    int64_t cta0;       // first CTA of the job
};
constexpr int MAX_BJOB = 6;
struct BSymArgs {
    const uint16_t* Lq;
    int64_t m, K;
    int bf16;
    const float* tq;    // signed vectors: u-th at tq + (Jb nc + u) K
    const float* ta;    // abs vectors: u-th at ta + (Jb + u) K
    int nc;             // signed vectors per block
    int64_t Jb;         // block of vector 0
    double* CS;         // column-checksum rows: (J nc + s, T0 + j), leading dimension ldcs
    float* Ca;          // abs-checksum rows: (J, T0 + j), leading dimension ldcs
    int64_t ldcs, T0;
    double* Cr;         // row-checksum columns: (T0 + j, J), leading dimension ldr; null: none
    float* Ra;          // abs row-checksum columns
    int64_t ldr;
    int64_t c0, c1;     // rows j in [c0, c1) update the column-checksum rows
    int64_t J0, J1;     // blocks J in [J0, J1) update the row-checksum columns
    int64_t g;
    const double* sig;
    const DevStatus* st;
    int njob;
    BJob job[MAX_BJOB];
};

constexpr int BKC = 32;            // K chunk
constexpr int BLD = BKC + 4;       // shared row stride (floats): conflict-free float4 reads
constexpr int BTHREADS = 256;
// Tile shapes: TR x TV threads, each RPT rows x VPT vectors.  Per 4 k a thread
// reads RPT + VPT float4 from shared memory (a 128-bit shared load costs four
// wavefronts even when broadcast) for 4 RPT VPT FMAs, so the bulk shape 8 x 4
// keeps the shared pipe at two thirds of the FMA rate; its 128 x 64 tile does
// 16 FMAs per byte brought from L2.
template <int TR_, int TV_, int RPT_, int VPT_>
struct BShape {
    static constexpr int TR = TR_, TV = TV_, RPT = RPT_, VPT = VPT_;
    static constexpr int RT = TR * RPT, VC = TV * VPT;
    static_assert(TR * TV == BTHREADS, "threads");
    static constexpr int LU = RT * BKC / 8;           // 8-value units of the Lq chunk
    static constexpr int TU = VC * BKC / 4;           // float4 units of the vector chunk
    static constexpr int LPT = (LU + BTHREADS - 1) / BTHREADS, TPT = (TU + BTHREADS - 1) / BTHREADS;
};
using BBulk = BShape<16, 16, 8, 4>;    // 128 rows x 64 vectors
using BTiny = BShape<16, 16, 2, 1>;    // 32 x 16: jobs too small to fill the GPU in bulk tiles
using BSkinny = BShape<64, 4, 2, 1>;   // 128 x 4: a handful of vectors (the look-ahead's row sums)
constexpr int BLR = BKC + 8;       // raw 16-bit row stride (elements): 16-byte aligned rows
// widened rows, two vector buffers and the raw rows, in floats
constexpr int bsmem(int rt, int vc) { return (rt + 2 * vc) * BLD + rt * BLR / 2; }
constexpr int BSMEM_FLOATS = bsmem(128, 64);   // the largest shape (BBulk)
static_assert(bsmem(128, 4) <= BSMEM_FLOATS && bsmem(32, 16) <= BSMEM_FLOATS, "shared");
constexpr int bcfg_rt(int c) { return c == 0 ? BBulk::RT : (c == 1 ? BTiny::RT : BSkinny::RT); }
constexpr int bcfg_vc(int c) { return c == 0 ? BBulk::VC : (c == 1 ? BTiny::VC : BSkinny::VC); }

// 16-byte global -> shared copy (cp.async), zero-filled when !pred
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool pred) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
                 "r"(pred ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <class S>
__device__ __forceinline__ void border_tile(const BSymArgs& a, const BJob& jb, int64_t rtile,
                                            int64_t vchunk, float* sm) {
    float* const Ls = sm;                               // [RT][BLD] FP32 (widened, |.| for abs jobs)
    float* const Tb = sm + S::RT * BLD;                 // [2][VC][BLD] FP32 vectors
    uint16_t* const Lr = (uint16_t*)(Tb + 2 * S::VC * BLD);   // [RT][BLR] raw 16-bit rows
    const int t = threadIdx.x, tv = t % S::TV, tr = t / S::TV;
    const int64_t r0 = jb.r0 + rtile * S::RT;
    const int vbase = jb.v0 + (int)vchunk * S::VC;
    const int ncK = jb.kind ? 1 : a.nc;
    const float* vecs = jb.kind ? a.ta + a.Jb * a.K : a.tq + a.Jb * a.nc * a.K;
    const bool absl = jb.kind != 0;
    // chunk k0 -> shared memory by cp.async: raw panel rows to Lr, vectors to Td
    auto fetch = [&](int64_t k0, float* Td) {
#pragma unroll
        for (int q = 0; q < S::LPT; ++q) {
            const int u = t + BTHREADS * q;
            if (u < S::LU) {
                const int64_t row = r0 + u / (BKC / 8);
                const bool ok = row < jb.r1;
                const uint16_t* src = a.Lq + (ok ? row : jb.r0) * a.K + k0 + (u % (BKC / 8)) * 8;
                cp_async16(Lr + (u / (BKC / 8)) * BLR + (u % (BKC / 8)) * 8, src, ok);
            }
        }
#pragma unroll
        for (int q = 0; q < S::TPT; ++q) {
            const int u = t + BTHREADS * q;
            if (u < S::TU) {
                const int v = vbase + u / (BKC / 4);
                const bool ok = v < jb.v1;
                const float* src = vecs + (int64_t)(ok ? v : jb.v0) * jb.vstep * a.K + k0 + (u % (BKC / 4)) * 4;
                cp_async16(Td + (u / (BKC / 4)) * BLD + (u % (BKC / 4)) * 4, src, ok);
            }
        }
        cp_async_commit();
    };
    auto widen = [&](uint32_t h) -> float {
        const uint16_t b = (uint16_t)h;
        const float f = a.bf16 ? __uint_as_float((uint32_t)b << 16) : __half2float(__ushort_as_half(b));
        return absl ? fabsf(f) : f;
    };
    float acc[S::RPT][S::VPT];
#pragma unroll
    for (int i = 0; i < S::RPT; ++i)
#pragma unroll
        for (int j = 0; j < S::VPT; ++j) acc[i][j] = 0.f;
    fetch(0, Tb);
    int buf = 0;
    for (int64_t k0 = 0; k0 < a.K; k0 += BKC, buf ^= 1) {
        cp_async_wait_all();
        __syncthreads();   // chunk k0 landed; the previous chunk's products are done
#pragma unroll
        for (int q = 0; q < S::LPT; ++q) {
            const int u = t + BTHREADS * q;
            if (u < S::LU) {
                const int row = u / (BKC / 8), c8 = (u % (BKC / 8)) * 8;
                const uint4 raw = *(const uint4*)(Lr + row * BLR + c8);
                const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
                float f[8];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    f[2 * e] = widen(w[e] & 0xffffu);
                    f[2 * e + 1] = widen(w[e] >> 16);
                }
                float* d = Ls + row * BLD + c8;
                *(float4*)d = make_float4(f[0], f[1], f[2], f[3]);
                *(float4*)(d + 4) = make_float4(f[4], f[5], f[6], f[7]);
            }
        }
        __syncthreads();   // Ls ready, Lr free
        if (k0 + BKC < a.K) fetch(k0 + BKC, Tb + (buf ^ 1) * (S::VC * BLD));
        const float* Ts = Tb + buf * (S::VC * BLD);
#pragma unroll
        for (int k4 = 0; k4 < BKC; k4 += 4) {
            float4 tt[S::VPT];
#pragma unroll
            for (int j = 0; j < S::VPT; ++j) tt[j] = *(const float4*)(Ts + (tv + S::TV * j) * BLD + k4);
#pragma unroll
            for (int i = 0; i < S::RPT; ++i) {
                const float4 l = *(const float4*)(Ls + (tr + S::TR * i) * BLD + k4);
#pragma unroll
                for (int j = 0; j < S::VPT; ++j) {
                    acc[i][j] = fmaf(tt[j].x, l.x, acc[i][j]);
                    acc[i][j] = fmaf(tt[j].y, l.y, acc[i][j]);
                    acc[i][j] = fmaf(tt[j].z, l.z, acc[i][j]);
                    acc[i][j] = fmaf(tt[j].w, l.w, acc[i][j]);
                }
            }
        }
    }
    // epilogue: scatter each product to the borders that hold it.  The
    // read-modify-writes go in groups of G rows: all loads of a group are
    // issued before its first store (the borders may alias as far as the
    // compiler knows, so one load per store would serialize on latency).
    const bool rowsums = a.Cr != nullptr;
    int64_t Jv[S::VPT];
    int sv[S::VPT], eJ[S::VPT];
    bool vok[S::VPT];
#pragma unroll
    for (int j = 0; j < S::VPT; ++j) {
        const int v = vbase + tv + S::TV * j;
        vok[j] = v < jb.v1;
        const int uu = (vok[j] ? v : jb.v0) * jb.vstep;
        Jv[j] = a.Jb + uu / ncK;
        sv[j] = uu % ncK;
        eJ[j] = pow2_exp(a.sig[Jv[j]]);
    }
    constexpr int G = S::RPT < 2 ? S::RPT : 2;
#pragma unroll
    for (int i0 = 0; i0 < S::RPT; i0 += G) {
        int64_t jr[G];
        int eI[G];
        bool rok[G], toc[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            jr[g] = r0 + tr + S::TR * (i0 + g);
            rok[g] = jr[g] < jb.r1;
            eI[g] = rok[g] ? pow2_exp(a.sig[(a.T0 + jr[g]) / a.g]) : 0;
            toc[g] = rok[g] && jr[g] >= a.c0 && jr[g] < a.c1;
        }
        auto cpos = [&](int g, int j) -> int64_t {
            return (jb.kind ? Jv[j] : Jv[j] * a.nc + sv[j]) * a.ldcs + a.T0 + jr[g];
        };
        auto rpos = [&](int g, int j) -> int64_t { return (a.T0 + jr[g]) * a.ldr + Jv[j]; };
        auto wc = [&](int g, int j) { return toc[g] && vok[j]; };
        auto wr = [&](int g, int j) {
            return rok[g] && vok[j] && rowsums && sv[j] == 0 && Jv[j] >= a.J0 && Jv[j] < a.J1;
        };
        // sigma_I sigma_J acc: exponent arithmetic, else the FP64 product
        auto exact_e = [&](int g, int j) {
            return (eI[g] != INT_MIN && eJ[j] != INT_MIN) ? eI[g] + eJ[j] : 4096;
        };
        auto s2 = [&](int g, int j) {
            return a.sig[(a.T0 + jr[g]) / a.g] * a.sig[Jv[j]];
        };
        if (jb.kind == 0) {
            double cv[G][S::VPT], rv[G][S::VPT];
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int j = 0; j < S::VPT; ++j) {
                    cv[g][j] = wc(g, j) ? a.CS[cpos(g, j)] : 0.0;
                    rv[g][j] = wr(g, j) ? a.Cr[rpos(g, j)] : 0.0;
                }
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int j = 0; j < S::VPT; ++j) {
                    if (!rok[g] || !vok[j]) continue;
                    const int e = exact_e(g, j);
                    const double x = f32_to_f64_exact(acc[i0 + g][j]);
                    const double val = (e > -1000 && e < 1000) ? scale_f64(x, e) : s2(g, j) * x;
                    if (wc(g, j)) a.CS[cpos(g, j)] = cv[g][j] - val;
                    if (wr(g, j)) a.Cr[rpos(g, j)] = rv[g][j] - val;
                }
        } else {
            float cv[G][S::VPT], rv[G][S::VPT];
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int j = 0; j < S::VPT; ++j) {
                    cv[g][j] = wc(g, j) ? a.Ca[cpos(g, j)] : 0.f;
                    rv[g][j] = wr(g, j) ? a.Ra[rpos(g, j)] : 0.f;
                }
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int j = 0; j < S::VPT; ++j) {
                    if (!rok[g] || !vok[j]) continue;
                    const int e = exact_e(g, j);
                    const float f = (e >= -126 && e <= 127) ? __int_as_float((e + 127) << 23)
                                                            : (float)s2(g, j);
                    const float val = f * acc[i0 + g][j];
                    if (wc(g, j)) a.Ca[cpos(g, j)] = cv[g][j] + val;
                    if (wr(g, j)) a.Ra[rpos(g, j)] = rv[g][j] + val;
                }
        }
    }
}

__global__ void __launch_bounds__(BTHREADS, 2) k_border_sym(BSymArgs a) {
    __shared__ __align__(16) float sm[BSMEM_FLOATS];
    if (a.st->info != 0) return;
    const int64_t b = blockIdx.x;
    int q = 0;
    while (q + 1 < a.njob && b >= a.job[q + 1].cta0) ++q;
    const BJob& jb = a.job[q];
    const int64_t loc = b - jb.cta0;
    const int64_t rtile = loc / jb.nvc, vchunk = loc % jb.nvc;
    if (jb.cfg == 0) border_tile<BBulk>(a, jb, rtile, vchunk, sm);
    else if (jb.cfg == 1) border_tile<BTiny>(a, jb, rtile, vchunk, sm);
    else border_tile<BSkinny>(a, jb, rtile, vchunk, sm);
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

cudaError_t launch_border_sym(const BorderSymHost& h, const DevStatus* st, cudaStream_t s) {
    if (h.m <= 0 || h.K <= 0 || h.Je <= h.Jb) return cudaSuccess;
    if (h.K % BKC != 0 || h.nc < 1 || h.nc > 2) return cudaErrorInvalidValue;
    BSymArgs a{};
    a.Lq = h.Lq; a.m = h.m; a.K = h.K; a.bf16 = h.bf16;
    a.tq = h.tq; a.ta = h.ta; a.nc = h.nc; a.Jb = h.Jb;
    a.CS = h.CS; a.Ca = h.Ca; a.ldcs = h.ldcs; a.T0 = h.T0;
    a.Cr = h.Cr; a.Ra = h.Ra; a.ldr = h.ldr;
    a.c0 = std::max<int64_t>(0, h.c0); a.c1 = std::min(h.m, h.c1);
    a.J0 = h.J0; a.J1 = h.J1; a.g = h.g; a.sig = h.sig; a.st = st;
    const int nblk = (int)(h.Je - h.Jb);
    int64_t total = 0;
    auto add = [&](int64_t r0, int64_t r1, int v0, int v1, int vstep, int kind) {
        if (r1 <= r0 || v1 <= v0) return;
        BJob& j = a.job[a.njob++];
        j.r0 = r0; j.r1 = r1; j.v0 = v0; j.v1 = v1; j.vstep = vstep; j.kind = kind;
        const int nv = v1 - v0;
        const int64_t bulk = ((r1 - r0 + BBulk::RT - 1) / BBulk::RT) * ((nv + BBulk::VC - 1) / BBulk::VC);
        j.cfg = nv <= BSkinny::VC ? 2 : (bulk < num_sms() ? 1 : 0);
        const int rt = bcfg_rt(j.cfg), vc = bcfg_vc(j.cfg);
        j.nvc = (nv + vc - 1) / vc;
        j.cta0 = total;
        total += ((r1 - r0 + rt - 1) / rt) * j.nvc;
    };
    // rows of the part: every vector; the other rows: the row sums of blocks [J0, J1)
    add(a.c0, a.c1, 0, nblk * h.nc, 1, 0);
    add(a.c0, a.c1, 0, nblk, 1, 1);
    if (h.Cr && h.J1 > h.J0) {
        const int v0 = (int)(h.J0 - h.Jb), v1 = (int)(h.J1 - h.Jb);
        add(0, a.c0, v0, v1, h.nc, 0);
        add(0, a.c0, v0, v1, 1, 1);
        add(a.c1, h.m, v0, v1, h.nc, 0);
        add(a.c1, h.m, v0, v1, 1, 1);
    }
    if (total == 0) return cudaSuccess;
    k_border_sym<<<(unsigned)total, BTHREADS, 0, s>>>(a);
    note_launch();
    return cudaGetLastError();
}

}  // namespace abft
