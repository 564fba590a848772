// k_resid_emu.cu -- FP64-accurate refinement residual R = B - A X on the BF16
// tensor cores, with the splitting of k_emu.cu (Ozaki et al. 2012; not in the
// paper): the FP64 residual of iterative refinement is B300's slowest step
// (two FP64 operations per element of A per right-hand side on its FP64
// pipe), so A is split once per solve into eight BF16 slices of its full rows
// (one power-of-two scale per row, both triangles from the stored lower one)
// and X once per refinement step into eight slices of each column (one scale
// per right-hand side).
//
// The product: group d of a 128-row tile of A X collects the slice pairs
// p + q = d.  With only 16 right-hand sides, the B operand of one MMA is a
// zero-padded stack of the X slices ([0 x 7, X_0, ..., X_7], 16 columns each):
// the MMA for slice p of A reads the window of eight blocks starting at block
// 7 - p, so accumulator column block c receives A_p X_(c - p), i.e. group c,
// for all pairs p + q <= 7 at once (M = 128, N = 128; blocks c < p are zero).
// FP32 accumulation is exact for K <= 256 (see k_emu.cu), so each 256-wide
// chunk of K is drained into a 64-bit fixed-point sum, converted to FP64 with
// integer operations (one rounding) and added to an FP64 running sum; two
// 128-column TMEM accumulators let the drain of one chunk overlap the MMAs of
// the next.  A work item is one 128-row tile and one 1024-wide range of K,
// written as a partial sum; R = B - sum of the partials in a fixed order.
//
// Error of the products (relative to the row scale of A times the column scale
// of X): the omitted slice pairs and the rounding of the slices leave about
// 2^-55 per term, so a length-n dot product is off by at most n 2^-55 (about
// sqrt(n) 2^-55 for independent signs), below the accumulated rounding of the
// same dot product in FP64.
//
// Kernel anatomy (persistent, one CTA per SM): warp 0 lane 0 issues the TMA
// loads (two 79 KB stages of K = 32: eight A slices and eight X blocks behind
// seven zero blocks), warp 1 allocates TMEM and issues the MMAs, warps 2-5
// drain the accumulators (one TMEM lane quarter each; thread = row).  Every
// wait is bounded; a wait that gives up makes the CTA's partial sums NaN, so
// the refinement stops with a NaN backward error.
#include <cuda.h>
#include <math.h>

#include "common.cuh"
#include "emu_slice.cuh"
#include "fp_bits.cuh"
#include "tc_util.cuh"

namespace abft {

using namespace tc;

namespace {

constexpr int RS = EMU_SLICES;
constexpr int RTM = 128;                 // rows per tile
constexpr int RKC = 32;                  // K per stage (64-byte rows)
constexpr int RNR = 16;                  // right-hand sides: one 16-row block per X slice
constexpr int RZ = 7;                    // zero blocks ahead of X_0
constexpr int R_ASL = RTM * RKC * 2;     // 8 KB: one A slice of the tile
constexpr int R_XBL = RNR * RKC * 2;     // 1 KB: one X block
constexpr int R_STA = RS * R_ASL;
constexpr int R_STAGE = R_STA + (RZ + RS) * R_XBL;   // 79 KB
constexpr int R_NST = 2;
constexpr uint32_t R_TX = (uint32_t)(RS * R_ASL + RS * R_XBL);
constexpr int RCH = 256;                 // K per exact FP32 accumulation
constexpr int RITEM = 1024;              // K per work item
constexpr int R_EPI = 4;
constexpr int R_THREADS = 64 + 32 * R_EPI;
constexpr uint32_t R_TMEM = 256;         // two 128-column accumulators
constexpr size_t R_SMEM = (size_t)R_NST * R_STAGE + 1024 + 256;
constexpr int FIXB = 40;                 // fraction bits of the fixed-point chunk sum

struct RArgs {
    int64_t n;
    int nr;
    const int* exA;     // e_i per row of A
    const int* exX;     // e_r per right-hand side
    double* P;          // partials [nsplit][n][16]
    int64_t ntile, nsplit;
    uint32_t idesc;
    int* err;
};

__global__ void __launch_bounds__(R_THREADS, 1) k_resid_emu(const __grid_constant__ CUtensorMap mapA,
                                                            const __grid_constant__ CUtensorMap mapX,
                                                            RArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + R_NST * R_STAGE);
    uint64_t* empty = full + R_NST;
    uint64_t* accf = empty + R_NST;     // [2]
    uint64_t* acce = accf + 2;          // [2]
    uint32_t* tmem_slot = (uint32_t*)(acce + 2);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int s2 = 0; s2 < R_NST; ++s2)   // zero blocks of the X stacks
        for (int i = threadIdx.x; i < RZ * R_XBL / 16; i += R_THREADS)
            *(uint4*)(smem + s2 * R_STAGE + R_STA + 16 * i) = make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x == 0) {
        for (int s2 = 0; s2 < R_NST; ++s2) {
            mbar_init(&full[s2], 1);
            mbar_init(&empty[s2], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], R_EPI);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(R_TMEM));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int64_t G = gridDim.x, items = a.ntile * a.nsplit;
    auto fail = [&]() {
        *abort_flag = 1;
        atomicExch(a.err, 1);
    };

    if (warp == 0) {
        if (lane == 0) {   // TMA producer
            int64_t c = 0;
            bool ok = true;
            for (int64_t idx = blockIdx.x; idx < items && ok && !*abort_flag; idx += G) {
                const int64_t tile = idx / a.nsplit, ks = idx % a.nsplit;
                const int64_t k0 = ks * RITEM, k1 = k0 + RITEM < a.n ? k0 + RITEM : a.n;
                for (int64_t kc = k0; kc < k1; kc += RKC, ++c) {
                    const int s2 = (int)(c % R_NST);
                    if (c >= R_NST && !mbar_wait(&empty[s2], (uint32_t)(((c / R_NST) - 1) & 1))) {
                        fail();
                        ok = false;
                        break;
                    }
                    uint8_t* st = smem + s2 * R_STAGE;
                    mbar_expect_tx(&full[s2], R_TX);
                    for (int p = 0; p < RS; ++p)
                        tma_load_2d(st + p * R_ASL, &mapA, &full[s2], (int)kc,
                                    (int)(p * a.n + tile * RTM));
                    for (int q = 0; q < RS; ++q)
                        tma_load_2d(st + R_STA + (RZ + q) * R_XBL, &mapX, &full[s2], (int)kc, q * RNR);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            int64_t c = 0, cc = 0;
            bool ok = true;
            for (int64_t idx = blockIdx.x; idx < items && ok && !*abort_flag; idx += G) {
                const int64_t ks = idx % a.nsplit;
                const int64_t k0 = ks * RITEM, k1 = k0 + RITEM < a.n ? k0 + RITEM : a.n;
                for (int64_t kch = k0; kch < k1 && ok; kch += RCH, ++cc) {
                    const int b = (int)(cc & 1);
                    if (cc >= 2 && !mbar_wait(&acce[b], (uint32_t)(((cc >> 1) - 1) & 1))) {
                        fail();
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t dt = tmem + (uint32_t)(b * 128);
                    const int64_t kend = kch + RCH < k1 ? kch + RCH : k1;
                    for (int64_t kc = kch; kc < kend; kc += RKC, ++c) {
                        const int s2 = (int)(c % R_NST);
                        if (!mbar_wait(&full[s2], (uint32_t)((c / R_NST) & 1))) {
                            fail();
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t sa = smem_u32(smem + s2 * R_STAGE);
                        const uint64_t adesc = smem_desc64(sa), bdesc = smem_desc64(sa + R_STA);
#pragma unroll 1
                        for (int kk = 0; kk < RKC / 16; ++kk)
#pragma unroll 1
                            for (int p = 0; p < RS; ++p)   // X window from block RZ - p
                                mma_f16(dt, adesc + (uint64_t)((p * R_ASL + kk * 32) >> 4),
                                        bdesc + (uint64_t)(((RZ - p) * R_XBL + kk * 32) >> 4),
                                        a.idesc, (kc > kch || kk > 0 || p > 0) ? 1u : 0u);
                        mma_commit(&empty[s2]);
                    }
                    if (ok) mma_commit(&accf[b]);
                }
            }
        }
    } else {
        // epilogue: TMEM lane quarter q, thread = row of the tile
        const int q = warp & 3;
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16);
        int64_t cc = 0;
        bool good = true;   // after a wait gives up, every remaining item of the CTA is NaN
        for (int64_t idx = blockIdx.x; idx < items; idx += G) {
            const int64_t tile = idx / a.nsplit, ks = idx % a.nsplit;
            const int64_t k0 = ks * RITEM, k1 = k0 + RITEM < a.n ? k0 + RITEM : a.n;
            const int64_t i = tile * RTM + q * 32 + lane;
            const int ei = i < a.n ? a.exA[i] : 0;
            double sum[RNR];
#pragma unroll
            for (int r = 0; r < RNR; ++r) sum[r] = 0.0;
            for (int64_t kch = k0; kch < k1 && good; kch += RCH, ++cc) {
                const int b = (int)(cc & 1);
                if (*abort_flag || !mbar_wait(&accf[b], (uint32_t)((cc >> 1) & 1))) {
                    if (!*abort_flag) fail();
                    good = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                long long acc[RNR];
#pragma unroll
                for (int r = 0; r < RNR; ++r) acc[r] = 0;
#pragma unroll
                for (int d = 0; d < RS; ++d) {
                    uint32_t v[RNR];
                    tmem_ld16(taddr + (uint32_t)(b * 128 + d * RNR), v);
                    if (d == RS - 1) {   // the accumulator has been read
                        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                        __syncwarp();
                        if (lane == 0)
                            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                                             smem_u32(&acce[b]))
                                         : "memory");
                    }
                    const int sh = FIXB - 7 * d;
#pragma unroll
                    for (int r = 0; r < RNR; ++r) {
                        // an exact integer below 2^24 in magnitude
                        const long long iv = (long long)__float2int_rn(__uint_as_float(v[r]));
                        acc[r] += sh >= 0 ? iv * (1ll << sh) : (iv >> (-sh));
                    }
                }
                // chunk value acc 2^(e_i + e_r - 54), added in FP64
#pragma unroll
                for (int r = 0; r < RNR; ++r) {
                    const int sc = ei + a.exX[r] - 54;
                    bool normal;
                    double y = i64_scaled_to_f64(acc[r], sc, normal);
                    if (!normal) y = ldexp((double)acc[r], sc);
                    sum[r] += y;
                }
            }
            if (i < a.n)
#pragma unroll
                for (int r = 0; r < RNR; ++r)   // static indices keep sum in registers
                    if (r < a.nr)
                        a.P[(ks * a.n + i) * RNR + r] =
                            good ? sum[r] : __longlong_as_double(0x7ff8000000000000ll);
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(R_TMEM));
    }
}

// Largest biased exponent of each full row of the symmetric A (lower triangle
// stored), over 256 x 256 tiles (I >= J) of the lower triangle: a tile's entries
// count for their rows and, mirrored, for the rows of their columns.  Thread t
// reads column t of the tile row by row (coalesced rows, eight loads in flight)
// and keeps that column's maximum in a register; a row's maximum is a warp
// reduction per warp and a maximum over the eight warps.  Two global atomics
// per row and column of a tile (8 per 1024 entries with 32 x 32 tiles).
__global__ void __launch_bounds__(256) k_sym_exp(const double* __restrict__ A, int64_t lda,
                                                 int64_t n, int* __restrict__ emax) {
    __shared__ unsigned rpart[8][256];
    const int64_t idx = blockIdx.x;
    int64_t I = (int64_t)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
    while (I * (I + 1) / 2 > idx) --I;
    while ((I + 1) * (I + 2) / 2 <= idx) ++I;
    const int64_t J = idx - I * (I + 1) / 2;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t r0 = I * 256, c = J * 256 + t;
    const int rows = n - r0 < 256 ? (int)(n - r0) : 256;
    unsigned cm = 0u;
    for (int r = 0; r < rows; r += 8) {
        unsigned long long b[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int rr = r + u;
            const bool ok = rr < rows && c < n && !(I == J && t > rr);
            b[u] = ok ? (unsigned long long)__double_as_longlong(A[(r0 + rr) * lda + c]) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const unsigned ex = (unsigned)((b[u] >> 52) & 0x7ffull);
            cm = ex > cm ? ex : cm;
            const unsigned rm = __reduce_max_sync(0xffffffffu, ex);
            if (lane == 0) rpart[warp][(r + u) & 255] = rm;
        }
    }
    __syncthreads();
    if (t < rows) {
        unsigned m = 0u;
#pragma unroll
        for (int w = 0; w < 8; ++w) m = rpart[w][t] > m ? rpart[w][t] : m;
        atomicMax(&emax[r0 + t], (int)m);
    }
    if (c < n) atomicMax(&emax[c], (int)cm);
}

// Slices of the full rows of A: S[p][i][k] for all i, k < n, written per lower
// 64 x 64 tile directly and (off the diagonal) mirrored through shared memory
// (n a multiple of 64).  A thread slices two adjacent entries of a row and
// stores each slice's two digits as one 32-bit word, so that a warp writes one
// 128-byte row piece per slice.
__global__ void __launch_bounds__(256) k_sym_slice(const double* __restrict__ A, int64_t lda,
                                                   int64_t n, const int* __restrict__ emax,
                                                   uint16_t* __restrict__ S) {
    __shared__ double T[64][65];
    const int64_t idx = blockIdx.x;
    int64_t I = (int64_t)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
    while (I * (I + 1) / 2 > idx) --I;
    while ((I + 1) * (I + 2) / 2 <= idx) ++I;
    const int64_t J = idx - I * (I + 1) / 2;
    for (int e = threadIdx.x; e < 4096; e += 256) {
        const int r = e >> 6, c = e & 63;
        T[r][c] = (I == J && c > r) ? 0.0 : A[(I * 64 + r) * lda + J * 64 + c];
    }
    __syncthreads();
    // direct: row I*64 + r, columns J*64 + c, c + 1 (the diagonal tile mirrored in place)
    for (int e = threadIdx.x; e < 2048; e += 256) {
        const int r = e >> 5, c = 2 * (e & 31);
        const double v0 = (I == J && c > r) ? T[c][r] : T[r][c];
        const double v1 = (I == J && c + 1 > r) ? T[c + 1][r] : T[r][c + 1];
        const int64_t row = I * 64 + r;
        const int em = emax[row] > 1 ? emax[row] : 1;
        uint16_t d0[EMU_SLICES], d1[EMU_SLICES];
        slice_digits((unsigned long long)__double_as_longlong(v0), em, d0);
        slice_digits((unsigned long long)__double_as_longlong(v1), em, d1);
#pragma unroll
        for (int p = 0; p < EMU_SLICES; ++p)
            *reinterpret_cast<uint32_t*>(S + ((int64_t)p * n + row) * n + J * 64 + c) =
                (uint32_t)d0[p] | ((uint32_t)d1[p] << 16);
    }
    if (I == J) return;
    // mirrored: row J*64 + c, columns I*64 + r, r + 1
    for (int e = threadIdx.x; e < 2048; e += 256) {
        const int c = e >> 5, r = 2 * (e & 31);
        const double v0 = T[r][c], v1 = T[r + 1][c];
        const int64_t row = J * 64 + c;
        const int em = emax[row] > 1 ? emax[row] : 1;
        uint16_t d0[EMU_SLICES], d1[EMU_SLICES];
        slice_digits((unsigned long long)__double_as_longlong(v0), em, d0);
        slice_digits((unsigned long long)__double_as_longlong(v1), em, d1);
#pragma unroll
        for (int p = 0; p < EMU_SLICES; ++p)
            *reinterpret_cast<uint32_t*>(S + ((int64_t)p * n + row) * n + I * 64 + r) =
                (uint32_t)d0[p] | ((uint32_t)d1[p] << 16);
    }
}

// The same for orders that are a multiple of 32 only (32 x 32 tiles).
__global__ void __launch_bounds__(256) k_sym_slice32(const double* __restrict__ A, int64_t lda,
                                                     int64_t n, const int* __restrict__ emax,
                                                     uint16_t* __restrict__ S) {
    __shared__ double T[32][33];
    const int64_t idx = blockIdx.x;
    int64_t I = (int64_t)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
    while (I * (I + 1) / 2 > idx) --I;
    while ((I + 1) * (I + 2) / 2 <= idx) ++I;
    const int64_t J = idx - I * (I + 1) / 2;
    for (int e = threadIdx.x; e < 1024; e += 256) {
        const int r = e >> 5, c = e & 31;
        T[r][c] = (I == J && c > r) ? 0.0 : A[(I * 32 + r) * lda + J * 32 + c];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 1024; e += 256) {
        const int r = e >> 5, c = e & 31;
        const double v = (I == J && c > r) ? T[c][r] : T[r][c];
        const int64_t row = I * 32 + r;
        const int em = emax[row] > 1 ? emax[row] : 1;
        uint16_t d[EMU_SLICES];
        slice_digits((unsigned long long)__double_as_longlong(v), em, d);
#pragma unroll
        for (int p = 0; p < EMU_SLICES; ++p) S[((int64_t)p * n + row) * n + J * 32 + c] = d[p];
    }
    if (I == J) return;
    for (int e = threadIdx.x; e < 1024; e += 256) {
        const int c = e >> 5, r = e & 31;
        const double v = T[r][c];
        const int64_t row = J * 32 + c;
        const int em = emax[row] > 1 ? emax[row] : 1;
        uint16_t d[EMU_SLICES];
        slice_digits((unsigned long long)__double_as_longlong(v), em, d);
#pragma unroll
        for (int p = 0; p < EMU_SLICES; ++p) S[((int64_t)p * n + row) * n + I * 32 + r] = d[p];
    }
}

// Column exponents and slices of X (n x nr, row-major, ld ldx) as 16 rows of
// length n per slice: SX[q][r][k] (zero for r >= nr).
__global__ void __launch_bounds__(256) k_xcol_exp(const double* __restrict__ X, int64_t ldx,
                                                  int64_t n, int nr, int* __restrict__ ex) {
    __shared__ int m[RNR];
    if (threadIdx.x < RNR) m[threadIdx.x] = 0;
    __syncthreads();
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t k = e / RNR;
    const int r = (int)(e % RNR);
    if (k < n && r < nr) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(X[k * ldx + r]);
        atomicMax(&m[r], (int)((b >> 52) & 0x7ffull));
    }
    __syncthreads();
    if (threadIdx.x < RNR) atomicMax(&ex[threadIdx.x], m[threadIdx.x]);
}

__global__ void __launch_bounds__(256) k_xcol_slice(const double* __restrict__ X, int64_t ldx,
                                                    int64_t n, int nr, const int* __restrict__ ex,
                                                    uint16_t* __restrict__ SX) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t k = e / RNR;
    const int r = (int)(e % RNR);
    if (k >= n) return;
    const double v = r < nr ? X[k * ldx + r] : 0.0;
    const int em = ex[r] > 1 ? ex[r] : 1;
    uint16_t d[EMU_SLICES];
    slice_digits((unsigned long long)__double_as_longlong(v), em, d);
#pragma unroll
    for (int q = 0; q < EMU_SLICES; ++q) SX[((int64_t)q * RNR + r) * n + k] = d[q];
}

// e = emax - 1022 per entry (the scale exponent of the splitting).
__global__ void k_exp_to_scale(int* __restrict__ e, int64_t count) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) e[i] = (e[i] > 1 ? e[i] : 1) - 1022;
}

bool encode_rows(CUtensorMap* map, const uint16_t* S, int64_t rows, int64_t n, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)n * 2};
    cuuint32_t box[2] = {(cuuint32_t)RKC, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)S, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool resid_emu_supported(int64_t n) { return n >= RKC && n % RKC == 0 && (int64_t)RS * n < INT32_MAX; }

size_t resid_emu_bytes(int64_t n) {
    if (!resid_emu_supported(n)) return 0;
    const int64_t nsplit = (n + RITEM - 1) / RITEM;
    const size_t sa = sizeof(uint16_t) * (size_t)RS * (size_t)n * (size_t)n;
    const size_t sx = sizeof(uint16_t) * (size_t)RS * RNR * (size_t)n;
    const size_t ex = sizeof(int) * ((size_t)n + RNR + 16);
    const size_t p = sizeof(double) * (size_t)nsplit * (size_t)n * RNR;
    return ((sa + 255) / 256 + (sx + 255) / 256 + (ex + 255) / 256 + (p + 255) / 256) * 256;
}

namespace {
struct ResidPtrs {
    uint16_t* SA;
    uint16_t* SX;
    int* exA;
    int* exX;
    int* err;
    double* P;
};
ResidPtrs resid_ptrs(void* ws, int64_t n) {
    char* b = (char*)ws;
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    ResidPtrs r;
    size_t off = 0;
    r.SA = (uint16_t*)(b + off); off += up(sizeof(uint16_t) * (size_t)RS * n * n);
    r.SX = (uint16_t*)(b + off); off += up(sizeof(uint16_t) * (size_t)RS * RNR * n);
    r.exA = (int*)(b + off);
    r.exX = r.exA + n;
    r.err = r.exX + RNR;
    off += up(sizeof(int) * ((size_t)n + RNR + 16));
    r.P = (double*)(b + off);
    return r;
}
}  // namespace

// Split A (n x n symmetric, lower triangle read) into its slices, once per solve.
cudaError_t launch_resid_emu_prepare(const double* A, int64_t lda, int64_t n, void* ws,
                                     cudaStream_t s) {
    if (!resid_emu_supported(n)) return cudaErrorInvalidValue;
    const ResidPtrs r = resid_ptrs(ws, n);
    cudaError_t e = cudaMemsetAsync(r.exA, 0, sizeof(int) * ((size_t)n + RNR + 16), s);
    if (e != cudaSuccess) return e;
    const int64_t ne = (n + 255) / 256;
    k_sym_exp<<<(unsigned)(ne * (ne + 1) / 2), 256, 0, s>>>(A, lda, n, r.exA);
    note_launch();
    if (n % 64 == 0) {
        const int64_t nt = n / 64;
        k_sym_slice<<<(unsigned)(nt * (nt + 1) / 2), 256, 0, s>>>(A, lda, n, r.exA, r.SA);
    } else {
        const int64_t nt = n / 32;
        k_sym_slice32<<<(unsigned)(nt * (nt + 1) / 2), 256, 0, s>>>(A, lda, n, r.exA, r.SA);
    }
    note_launch();
    k_exp_to_scale<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(r.exA, n);
    note_launch();
    return cudaGetLastError();
}

// R = B - A X for up to 16 right-hand sides from the slices of A made by
// launch_resid_emu_prepare (which must have run on the same workspace), with
// the per-column maxima of |R| and |X| as launch_residual; with B == nullptr,
// R = A X (16 columns, ld 16) as launch_symv.
cudaError_t launch_resid_emu(int64_t n, const double* X, int64_t ldx, const double* B, int64_t ldb,
                             int nr, double* R, int64_t ldr, void* ws, unsigned long long* rmax,
                             unsigned long long* xmax, cudaStream_t s) {
    if (!resid_emu_supported(n) || nr < 1 || nr > RNR) return cudaErrorInvalidValue;
    const ResidPtrs r = resid_ptrs(ws, n);
    cudaError_t e = cudaMemsetAsync(r.exX, 0, sizeof(int) * (RNR + 1), s);
    if (e != cudaSuccess) return e;
    const int64_t nx = n * RNR;
    k_xcol_exp<<<(unsigned)((nx + 255) / 256), 256, 0, s>>>(X, ldx, n, nr, r.exX);
    note_launch();
    k_xcol_slice<<<(unsigned)((nx + 255) / 256), 256, 0, s>>>(X, ldx, n, nr, r.exX, r.SX);
    note_launch();
    k_exp_to_scale<<<1, RNR, 0, s>>>(r.exX, RNR);
    note_launch();
    CUtensorMap mapA, mapX;
    if (!encode_rows(&mapA, r.SA, (int64_t)RS * n, n, RTM) ||
        !encode_rows(&mapX, r.SX, (int64_t)RS * RNR, n, RNR))
        return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        e = cudaFuncSetAttribute(k_resid_emu, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)R_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    RArgs a{};
    a.n = n;
    a.nr = nr;
    a.exA = r.exA;
    a.exX = r.exX;
    a.P = r.P;
    a.err = r.err;
    a.ntile = (n + RTM - 1) / RTM;
    a.nsplit = (n + RITEM - 1) / RITEM;
    // kind::f16 instruction descriptor: D F32, A/B BF16, K-major, N = 128, M = 128
    a.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 3) << 17) |
              ((uint32_t)(RTM >> 4) << 24);
    const int64_t items = a.ntile * a.nsplit;
    int64_t grid = num_sms();
    if (grid > items) grid = items;
    k_resid_emu<<<(unsigned)grid, R_THREADS, R_SMEM, s>>>(mapA, mapX, a);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (B == nullptr) {   // the product A X (n x 16, ld 16)
        if (ldr != RNR) return cudaErrorInvalidValue;
        return launch_symv_reduce(r.P, (int)a.nsplit, n, R, s);
    }
    return launch_resid_reduce(r.P, (int)a.nsplit, n, B, ldb, X, ldx, nr, R, ldr, rmax, xmax, s);
}

}  // namespace abft
