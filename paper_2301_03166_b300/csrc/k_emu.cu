// k_emu.cu -- FP64-accurate trailing update of the Cholesky on the BF16
// tensor cores by splitting the panel into small-integer slices (the Ozaki
// scheme: Ozaki, Ogita, Oishi, Rump 2012; not in the paper).  B300's FP64 pipe
// runs the FP64 update at ~1.1 TFLOP/s; the slice products below run on
// tcgen05 and are exact.
//
// Splitting (k_slice_panel, integer operations only): row i of the m x kb
// panel gets the power-of-two scale sigma_i = 2^e_i, e_i = E_max - 1022 with
// E_max its largest biased exponent, so |x| < 1 for x = L[i][k] / sigma_i.
// |x| 2^56 rounded to an integer F is written in balanced base 128:
// x ~ sign(x) sum_{p=0}^{7} d_p 2^(-7 (p + 1)), d_p in [-64, 63] for p >= 1 and
// d_0 in [0, 128] (digits taken from the least significant end with a carry),
// and the eight signed digits are stored as BF16 (exact).
//
// Update (k_tmu_emu): C_ij -= sigma_i sigma_j 2^-14 sum_d 2^(-7 d) G_d with
// G_d = sum_{p + q = d} sum_k s_p(i, k) s_q(j, k) over the 36 pairs with
// p + q <= 7.  The omitted pairs weigh <= ~2^-47 sigma_i sigma_j and the
// rounding of F <= 2^-57 sigma per element, both at or below the rounding of
// the same product in FP64.  For kb <= 256 a slice product is an integer below
// 2^21 (2^20 unless it involves d_0), so all d + 1 <= 8 pairs of weight d
// accumulate exactly in one FP32 TMEM accumulator: eight groups per tile.
// Each group is drained into a 64-bit integer fixed-point sum
// A = sum_d G_d 2^(40 - 7 d) (exact for d <= 5, truncated for d = 6, 7 below
// 2^-40), and C_ij -= A 2^(e_i + e_j - 54) is one FP64 update per element.
//
// Kernel anatomy (persistent, one CTA per SM, 128 x 64 tiles of C): the pairs
// of a tile run p-major, so slice p of the tile's rows (the A operand, 128 x kb,
// 64 KB) is loaded once and stays in shared memory (two slots) while slices
// q = 0 .. 7 - p of the tile's columns (B, 64 x kb, one pair per stage) stream
// through a 3-stage ring; the eight weight groups accumulate in eight 64-column FP32
// TMEM accumulators (all 512 columns).  Group d is complete after pair
// (d, 0), so the epilogue drains it while the MMAs of larger p continue, and
// the next tile's first MMA into group d waits only for that drain.
// Warp 0 issues the TMA loads (lane 0 the B chunks, lane 1 the A slices, each
// running ahead as far as its buffers allow), warp 1 allocates TMEM and
// issues the MMAs,
// warps 2-9 drain the groups into 64-bit integers (registers) and update C.
// Every wait is bounded.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"
#include "tc_util.cuh"

namespace abft {

using namespace tc;

namespace {

constexpr int ES = 8;                       // slices per element
constexpr int ETM = 128, ETN = 64, EKC = 64;
constexpr int EKMAX = 256;                  // panel width limit (exact FP32 accumulation)
constexpr int ACHUNK = ETM * EKC * 2;       // 128 x 64 BF16 box
constexpr int ASLOT = ACHUNK * (EKMAX / EKC);   // one slice of the tile rows, whole K
constexpr int BCHUNK = ETN * EKC * 2;       // 64 x 64 BF16 box
constexpr int BSTAGE = BCHUNK * (EKMAX / EKC);   // one slice of the tile columns, whole K
constexpr int BSTAGES = 3;
constexpr int EPI_W = 8;
constexpr int ETHREADS = 64 + EPI_W * 32;
constexpr int NGROUP = 8;
constexpr uint32_t ETMEM_COLS = 512;        // eight 64-column FP32 accumulators
constexpr size_t E_SMEM = 2 * (size_t)ASLOT + (size_t)BSTAGES * BSTAGE + 1024 + 512;
constexpr int FIXB = 40;                    // fraction bits of the fixed-point sum

struct EmuArgs {
    double* C;
    int64_t ldc;
    int64_t M;          // trailing order (rows of the panel slices)
    int64_t K;          // panel width, multiple of 64, <= 256
    const int* ex;      // e_i per panel row
    int ncf;
    ComputeFault cf[MAX_CF];
    DevStatus* st;
    int64_t ntiles;     // tiles of the lower block triangle (rm x rn per block pair)
    int64_t rm, rn;     // 128-row and 64-column tiles per g
    uint32_t idesc;
};

__device__ __forceinline__ void emu_tile(int64_t idx, int64_t rm, int64_t rn, int64_t& ti,
                                         int64_t& tj) {
    const int64_t per = rm * rn, pair = idx / per, sub = idx % per;
    int64_t a = (int64_t)((sqrt(8.0 * (double)pair + 1.0) - 1.0) * 0.5);
    while (a * (a + 1) / 2 > pair) --a;
    while ((a + 1) * (a + 2) / 2 <= pair) ++a;
    const int64_t b = pair - a * (a + 1) / 2;
    ti = a * rm + sub / rn;
    tj = b * rn + sub % rn;
}

// 2^k as a double for the normal range, 0 below it (k > 1023 does not occur:
// the scales are bounded by the largest finite double).
__device__ __forceinline__ double pow2(int k) {
    if (k < -1022) return 0.0;
    return __hiloint2double((k + 1023) << 20, 0);
}

__global__ void __launch_bounds__(256) k_slice_panel(const double* __restrict__ P, int64_t lda,
                                                     int64_t m, int kb, uint16_t* __restrict__ S,
                                                     int* __restrict__ ex) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * 8 + warp;
    if (row >= m) return;
    const int nt = kb >> 5;                 // kb <= 256: at most 8 per lane
    unsigned long long b[8];
    int emax = 1;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        b[t] = 0ull;
        if (t < nt) {
            b[t] = (unsigned long long)__double_as_longlong(P[row * lda + lane + 32 * t]);
            const int e = (int)((b[t] >> 52) & 0x7ffull);
            emax = e > emax ? e : emax;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int other = __shfl_xor_sync(0xffffffffu, emax, o);
        emax = other > emax ? other : emax;
    }
    if (lane == 0) ex[row] = emax - 1022;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        if (t >= nt) continue;
        const int e = (int)((b[t] >> 52) & 0x7ffull);
        const unsigned long long mant = (b[t] & 0xfffffffffffffull) | (e ? (1ull << 52) : 0ull);
        // F = round(|x| 2^56) = round(mant 2^(E - E_max + 3)), E of a subnormal taken
        // as 1: a right shift by E_max - 3 - E (a left shift for the largest elements)
        const int sh = emax - 3 - (e ? e : 1);
        unsigned long long F;
        if (sh <= 0) F = mant << (-sh);
        else if (sh >= 64) F = 0ull;
        else F = (mant >> sh) + ((mant >> (sh - 1)) & 1ull);
        const bool neg = (b[t] >> 63) != 0ull;
        const int64_t k = lane + 32 * t;
        int carry = 0;
#pragma unroll
        for (int p = ES - 1; p >= 0; --p) {
            int d = (int)((F >> (7 * (ES - 1 - p))) & 127ull) + carry;
            carry = 0;
            if (p > 0 && d >= 64) {
                d -= 128;
                carry = 1;
            }
            const float v = (float)(neg ? -d : d);
            S[((int64_t)p * m + row) * kb + k] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
        }
    }
}

__global__ void __launch_bounds__(ETHREADS, 1) k_tmu_emu(const __grid_constant__ CUtensorMap mapA,
                                                         const __grid_constant__ CUtensorMap mapB,
                                                         EmuArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* abuf = smem;                                  // [2][ASLOT]
    uint8_t* bring = smem + 2 * ASLOT;                     // [BSTAGES][BSTAGE]
    uint64_t* fullA = (uint64_t*)(bring + BSTAGES * BSTAGE);
    uint64_t* emptyA = fullA + 2;
    uint64_t* fullB = emptyA + 2;
    uint64_t* emptyB = fullB + BSTAGES;
    uint64_t* accf = emptyB + BSTAGES;                     // [NGROUP]
    uint64_t* acce = accf + NGROUP;                        // [NGROUP]
    uint32_t* tmem_slot = (uint32_t*)(acce + NGROUP);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    if (a.st->info != 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s2 = 0; s2 < 2; ++s2) {
            mbar_init(&fullA[s2], 1);
            mbar_init(&emptyA[s2], 1);
        }
        for (int s2 = 0; s2 < BSTAGES; ++s2) {
            mbar_init(&fullB[s2], 1);
            mbar_init(&emptyB[s2], 1);
        }
        for (int d = 0; d < NGROUP; ++d) {
            mbar_init(&accf[d], 1);
            mbar_init(&acce[d], EPI_W);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(ETMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int nk = (int)(a.K / EKC);
    const int64_t G = gridDim.x;
    auto fail = [&]() {
        *abort_flag = 1;
        atomicExch(&a.st->error, 3);
    };

    if (warp == 0) {
        if (lane == 1) {          // TMA producer of the A slices (tile rows, whole K)
            int64_t ca = 0;
            bool ok = true;
            for (int64_t idx = blockIdx.x; idx < a.ntiles && ok && !*abort_flag; idx += G) {
                int64_t ti, tj;
                emu_tile(idx, a.rm, a.rn, ti, tj);
                if (ti * ETM >= a.M || tj * ETN >= a.M) continue;
                for (int p = 0; p < ES; ++p, ++ca) {
                    const int slot = (int)(ca & 1);
                    if (ca >= 2 && !mbar_wait(&emptyA[slot], (uint32_t)(((ca >> 1) - 1) & 1))) {
                        fail();
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&fullA[slot], (uint32_t)(ACHUNK * nk));
                    const int ya = (int)((int64_t)p * a.M + ti * ETM);
                    for (int kc = 0; kc < nk; ++kc)
                        tma_load_2d(abuf + slot * ASLOT + kc * ACHUNK, &mapA, &fullA[slot], kc * EKC, ya);
                }
            }
        } else if (lane == 0) {   // TMA producer of the B chunks (tile columns)
            int64_t cb = 0;
            bool ok = true;
            for (int64_t idx = blockIdx.x; idx < a.ntiles && ok && !*abort_flag; idx += G) {
                int64_t ti, tj;
                emu_tile(idx, a.rm, a.rn, ti, tj);
                if (ti * ETM >= a.M || tj * ETN >= a.M) continue;
                for (int p = 0; p < ES && ok; ++p) {
                    for (int q = 0; q < ES - p; ++q, ++cb) {
                        const int yb = (int)((int64_t)q * a.M + tj * ETN);
                        const int s2 = (int)(cb % BSTAGES);
                        if (cb >= BSTAGES &&
                            !mbar_wait(&emptyB[s2], (uint32_t)(((cb / BSTAGES) - 1) & 1))) {
                            fail();
                            ok = false;
                            break;
                        }
                        mbar_expect_tx(&fullB[s2], (uint32_t)(BCHUNK * nk));
                        for (int kc = 0; kc < nk; ++kc)
                            tma_load_2d(bring + s2 * BSTAGE + kc * BCHUNK, &mapB, &fullB[s2],
                                        kc * EKC, yb);
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            int64_t ca = 0, cb = 0, tc = 0;
            bool ok = true;
            for (int64_t idx = blockIdx.x; idx < a.ntiles && ok && !*abort_flag; idx += G) {
                int64_t ti, tj;
                emu_tile(idx, a.rm, a.rn, ti, tj);
                if (ti * ETM >= a.M || tj * ETN >= a.M) continue;
                for (int p = 0; p < ES && ok; ++p, ++ca) {
                    const int slot = (int)(ca & 1);
                    if (!mbar_wait(&fullA[slot], (uint32_t)((ca >> 1) & 1))) {
                        fail();
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t abase = smem_u32(abuf + slot * ASLOT);
                    for (int q = 0; q < ES - p && ok; ++q, ++cb) {
                        const int d = p + q;
                        // first MMA of group d in this tile: its accumulator must be drained
                        if (p == 0 && tc >= 1 && !mbar_wait(&acce[d], (uint32_t)((tc - 1) & 1))) {
                            fail();
                            ok = false;
                            break;
                        }
                        const int s2 = (int)(cb % BSTAGES);
                        if (!mbar_wait(&fullB[s2], (uint32_t)((cb / BSTAGES) & 1))) {
                            fail();
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t dt = tmem + (uint32_t)(d * ETN);
                        // descriptors advance by 32 bytes per K = 16 step (field in 16-byte units)
                        const uint64_t adesc0 = smem_desc(abase);
                        const uint64_t bdesc0 = smem_desc(smem_u32(bring + s2 * BSTAGE));
                        for (int kc = 0; kc < nk; ++kc) {
#pragma unroll
                            for (int kk = 0; kk < EKC / 16; ++kk)
                                mma_f16(dt, adesc0 + (uint64_t)((kc * ACHUNK + kk * 32) >> 4),
                                        bdesc0 + (uint64_t)((kc * BCHUNK + kk * 32) >> 4), a.idesc,
                                        (p > 0 || kc > 0 || kk > 0) ? 1u : 0u);
                        }
                        mma_commit(&emptyB[s2]);
                        if (q == 0) mma_commit(&accf[p]);   // pair (p, 0) ends group p
                    }
                    if (ok) mma_commit(&emptyA[slot]);
                }
                ++tc;
            }
        }
    } else {
        // epilogue: TMEM lane quarter q (rows 32 q ..), column half h (32 columns)
        const int ew = warp - 2;
        const int q = warp & 3;
        const int h = ew >> 2;
        const int r = q * 32 + lane;
        int64_t tc = 0;
        for (int64_t idx = blockIdx.x; idx < a.ntiles; idx += G) {
            int64_t ti, tj;
            emu_tile(idx, a.rm, a.rn, ti, tj);
            if (ti * ETM >= a.M || tj * ETN >= a.M) continue;
            long long acc[32];
#pragma unroll
            for (int u = 0; u < 32; ++u) acc[u] = 0;
            bool ok = true;
            for (int d = 0; d < NGROUP; ++d) {
                if (ok && !*abort_flag && mbar_wait(&accf[d], (uint32_t)(tc & 1))) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    uint32_t v[32];
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(d * ETN + h * 32), v);
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0)
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                                         smem_u32(&acce[d]))
                                     : "memory");
                    const int sh = FIXB - 7 * d;
#pragma unroll
                    for (int u = 0; u < 32; ++u) {
                        // an exact integer below 2^24 in magnitude
                        const long long iv = (long long)__float2int_rn(__uint_as_float(v[u]));
                        acc[u] += sh >= 0 ? iv * (1ll << sh) : (iv >> (-sh));
                    }
                } else {
                    if (ok && !*abort_flag) fail();
                    ok = false;
                }
            }
            // C[i][j] -= A 2^(e_i + e_j - 54): this thread's row, 32 columns, all
            // loads first
            const int64_t gi = ti * ETM + r, jb = tj * ETN + h * 32;
            if (ok && !*abort_flag && gi < a.M) {
                double* crow = a.C + gi * a.ldc;
                const int ei = a.ex[gi];
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    double cv[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int64_t gj = jb + 16 * half + u;
                        cv[u] = gj < a.M ? crow[gj] : 0.0;
                    }
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int64_t gj = jb + 16 * half + u;
                        if (gj >= a.M) continue;
                        double v = cv[u] - (double)acc[16 * half + u] * pow2(ei + a.ex[gj] - 54);
                        for (int f = 0; f < a.ncf; ++f)
                            if (a.cf[f].row == gi && a.cf[f].col == gj) v += a.cf[f].delta;
                        crow[gj] = v;
                    }
                }
            }
            ++tc;
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(ETMEM_COLS));
    }
}

bool encode_slices(CUtensorMap* map, const uint16_t* S, int64_t rows, int64_t kb, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)kb, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kb * 2};
    cuuint32_t box[2] = {(cuuint32_t)EKC, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)S, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t emu_slice_bytes(int64_t n, int64_t nb) {
    return sizeof(uint16_t) * (size_t)ES * (size_t)n * (size_t)nb;
}

cudaError_t launch_slice_panel(const double* P, int64_t lda, int64_t m, int64_t kb, uint16_t* S,
                               int* ex, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    if (kb % 32 != 0 || kb > 256) return cudaErrorInvalidValue;
    k_slice_panel<<<(unsigned)((m + 7) / 8), 256, 0, s>>>(P, lda, m, (int)kb, S, ex);
    note_launch();
    return cudaGetLastError();
}

// C (m x m, trailing, FP64) -= L L^T on the lower block triangle (blocks of g),
// from the slices S (7 x m x kb BF16) and row exponents ex of the panel L.
cudaError_t launch_tmu_emu(const uint16_t* S, const int* ex, int64_t m, int64_t kb, double* C,
                           int64_t ldc, int64_t g, const ComputeFault* cf, int ncf, DevStatus* st,
                           cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    if (kb % EKC != 0 || kb > EKMAX || g % ETM != 0) return cudaErrorInvalidValue;
    CUtensorMap mapA, mapB;
    if (!encode_slices(&mapA, S, ES * m, kb, ETM) || !encode_slices(&mapB, S, ES * m, kb, ETN))
        return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_tmu_emu, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)E_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    EmuArgs a{};
    a.C = C; a.ldc = ldc; a.M = m; a.K = kb; a.ex = ex; a.st = st;
    a.ncf = 0;
    for (int f = 0; f < ncf && f < MAX_CF; ++f) a.cf[a.ncf++] = cf[f];
    const int64_t qb = (m + g - 1) / g;
    a.rm = g / ETM;
    a.rn = g / ETN;
    a.ntiles = qb * (qb + 1) / 2 * a.rm * a.rn;
    // kind::f16 instruction descriptor: D F32, A/B BF16, K-major, N >> 3, M >> 4
    a.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(ETN >> 3) << 17) |
              ((uint32_t)(ETM >> 4) << 24);
    int64_t grid = num_sms();
    if (grid > a.ntiles) grid = a.ntiles;
    k_tmu_emu<<<(unsigned)grid, ETHREADS, E_SMEM, s>>>(mapA, mapB, a);
    note_launch();
    return cudaGetLastError();
}

}  // namespace abft
