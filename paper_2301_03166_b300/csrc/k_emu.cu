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
// Tensor-core shape (measured on B300): one tcgen05.mma of M = 128, K = 16
// takes the same time for every N up to 256, so every MMA here has N = 256.
// The eight weight groups of a 128 x 64 tile of C fill the 512 TMEM columns
// (group d at columns 64 d), split into two 256-column windows X (groups 0-3)
// and Y (groups 4-7).  For slice p of the tile rows, the MMA into a window
// takes as its 256-row B operand four consecutive 64-row blocks of the stack
// [0, 0, 0, B_0, B_1, ..., B_7] (B_q = slice q of the tile columns): the block
// under group c is B_(c - p), or zero when c < p.  X needs slices p = 0..3,
// Y all eight: 12 MMAs per K step for the 36 pairs (75% of the MMA work useful,
// against 25% for N = 64 MMAs).
//
// Kernel anatomy (persistent, one CTA per SM): the K dimension streams through
// two 108 KB stages (K = 32 per stage, 64-byte swizzled rows) holding all eight
// slices of the tile rows (A) and of the tile columns (B, behind its three
// zero blocks).  Warp 0 lane 0 issues the TMA loads, warp 1 allocates TMEM and
// issues the MMAs (per stage the X MMAs, then the Y MMAs), warps 2-17 drain X
// and then Y into 64-bit integers and update C (each warp a TMEM lane quarter
// and 16 columns, read in the 16x256b shape so that C moves in 64-byte row
// segments).  The MMAs of the next tile
// start on X as soon as the epilogue has read X (it does so while the last Y
// MMAs of the tile run) and on Y once Y has been read; the FP64 update of C
// overlaps the next tile's MMAs.  One launch also carries the two checksum
// borders of the ABFT update (Sec. 3.1.2): the checksum rows are sliced into
// the same tensor behind the panel rows, and their tiles (checksum rows x
// panel rows, panel rows x checksum rows) join the work list as rectangles;
// a rectangle also carries the next block column alone when the update is
// split for look-ahead.
// Every wait is bounded.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"
#include "emu_slice.cuh"
#include "fp_bits.cuh"
#include "tc_util.cuh"

namespace abft {

using namespace tc;

namespace {

constexpr int ES = 8;                       // slices per element
constexpr int ETM = 128, ETN = 64;          // C tile
constexpr int EKC = 32;                     // K per stage (64-byte rows)
constexpr int EKMAX = 256;                  // panel width limit (exact FP32 accumulation)
constexpr int A_SL = ETM * EKC * 2;         // 8 KB: one slice of the tile rows
constexpr int B_BL = ETN * EKC * 2;         // 4 KB: one 64-row block of the B stack
constexpr int NZ = 3;                       // zero blocks ahead of B_0
constexpr int ST_A = ES * A_SL;
constexpr int STAGE = ST_A + (NZ + ES) * B_BL;   // 108 KB
constexpr int NSTAGE = 2;
constexpr int ECOLS = ETN / 4;             // columns per epilogue thread
constexpr uint32_t STAGE_TX = (uint32_t)(ES * A_SL + ES * B_BL);
constexpr int EPI_W = 16;                   // 4 TMEM lane quarters x 4 column quarters
constexpr int ETHREADS = 64 + EPI_W * 32;
constexpr uint32_t ETMEM_COLS = 512;        // eight 64-column FP32 group accumulators
constexpr size_t E_SMEM = (size_t)NSTAGE * STAGE + 1024 + 256;
constexpr int FIXB = 40;                    // fraction bits of the fixed-point sum

struct EmuRect {
    double* C;          // C[i * ldc + j / cdiv] for local row i < na, column j < nb, j % cdiv == 0
    int64_t ldc;
    int a0, na;         // A operand: slice rows a0 .. a0 + na - 1
    int b0, nb;         // B operand: slice rows b0 .. b0 + nb - 1
    int cdiv;
    int ntj;            // 64-column tiles
    int frow, fcol;     // trailing coordinates of local (0, 0) for compute faults (-1: none)
    bool vec;           // double2 access (cdiv 1, rows 16-byte aligned)
};

struct EmuArgs {
    double* C;          // trailing matrix: the triangle covers rows and columns [o, M)
    int64_t ldc;
    int64_t M, o;
    int64_t Mtot;       // rows per slice
    int64_t K;          // panel width, multiple of 32, <= 256
    const int* ex;      // e_i per slice row
    int ncf;
    ComputeFault cf[MAX_CF];   // trailing coordinates
    DevStatus* st;
    int64_t n1;         // tiles of the lower block triangle
    int64_t rm, rn;     // 128-row and 64-column tiles per g
    int nrect;
    EmuRect rect[3];
    int64_t rend[3];    // cumulative rectangle tile counts
    bool vec1;          // triangle rows 16-byte aligned at even columns
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

// rect[r] with static indices (a runtime index into the parameter block would
// copy it to local memory)
__device__ __forceinline__ EmuRect rect_of(const EmuArgs& a, int r) {
    return r == 0 ? a.rect[0] : (r == 1 ? a.rect[1] : a.rect[2]);
}

struct EmuItem {
    int seg;            // -1 triangle, else the rectangle
    int64_t ti, tj;     // tile indices within the segment
    int64_t arow, brow; // first slice row of the A and B tiles
    bool valid;
};

__device__ __forceinline__ EmuItem emu_item(int64_t idx, const EmuArgs& a) {
    EmuItem t;
    if (idx < a.n1) {
        emu_tile(idx, a.rm, a.rn, t.ti, t.tj);
        t.seg = -1;
        t.arow = a.o + t.ti * ETM;
        t.brow = a.o + t.tj * ETN;
        t.valid = t.arow < a.M && t.brow < a.M;
    } else {
        int64_t j = idx - a.n1;
        int r = 0;
        if (a.nrect > 1 && j >= a.rend[0]) r = 1;
        if (a.nrect > 2 && j >= a.rend[1]) r = 2;
        j -= r == 0 ? 0 : (r == 1 ? a.rend[0] : a.rend[1]);
        const EmuRect e = rect_of(a, r);
        t.seg = r;
        t.ti = j / e.ntj;
        t.tj = j % e.ntj;
        t.arow = e.a0 + t.ti * ETM;
        t.brow = e.b0 + t.tj * ETN;
        t.valid = true;
    }
    return t;
}

__global__ void __launch_bounds__(256) k_slice_panel(const double* __restrict__ P, int64_t lda,
                                                     int64_t m, int kb, uint16_t* __restrict__ S,
                                                     int64_t Mtot, int64_t row0,
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
    if (lane == 0) ex[row0 + row] = emax - 1022;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        if (t >= nt) continue;
        uint16_t d[EMU_SLICES];
        slice_digits(b[t], emax, d);
        const int64_t k = lane + 32 * t;
#pragma unroll
        for (int p = 0; p < ES; ++p) S[((int64_t)p * Mtot + row0 + row) * kb + k] = d[p];
    }
}

// Slices of the columns of a row-major K x ncols matrix P (K <= 256, a
// multiple of 32) as rows row0 .. row0 + ncols - 1 of S (row stride K): the
// B operand of an update whose right factor is stored by rows (the LU's
// U12).  One CTA per 32 columns: the K x 32 tile goes through shared memory
// so that the reads (along rows of P) and the writes (along rows of S) are
// coalesced; one scale per column.
// Chunked form (blockIdx.y = chunk c): rows c K .. c K + K - 1 of an
// mrows-row matrix, rows past mrows taken as zero, written at row0 + c rstride:
// the operands of a product whose reduction runs over the rows of P (the
// QR's V^T C), cut into K-long pieces with a scale per column and piece.
constexpr int SC_COLS = 32;
__global__ void __launch_bounds__(256) k_slice_cols(const double* __restrict__ P, int64_t ld,
                                                    int K, int64_t mrows, int64_t ncols,
                                                    uint16_t* __restrict__ S, int64_t Mtot,
                                                    int64_t row0, int64_t rstride,
                                                    int* __restrict__ ex) {
    extern __shared__ __align__(16) unsigned char sc_smem[];
    double* T = (double*)sc_smem;                     // K x (SC_COLS + 1)
    __shared__ int emax_s[SC_COLS];
    const int64_t c0 = (int64_t)blockIdx.x * SC_COLS;
    const int nc = (int)(ncols - c0 < SC_COLS ? ncols - c0 : SC_COLS);
    P += (int64_t)blockIdx.y * K * ld;
    row0 += (int64_t)blockIdx.y * rstride;
    const int64_t left = mrows - (int64_t)blockIdx.y * K;
    const int kv = (int)(left < K ? left : K);
    if (threadIdx.x < SC_COLS) emax_s[threadIdx.x] = 1;
    __syncthreads();
    {   // lane j of warp w reads rows w, w + 8, ... of column c0 + j (a warp: 32
        // consecutive doubles of one row), eight loads in flight; the largest
        // exponent is kept in a register and merged once per thread
        const int j = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
        int em = 1;
        for (int k0 = w; k0 < K; k0 += 8 * nw) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + u * nw;
                v[u] = (j < nc && k < kv) ? P[(int64_t)k * ld + c0 + j] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + u * nw;
                if (k < K) {
                    T[k * (SC_COLS + 1) + j] = v[u];
                    const int e = (int)(((unsigned long long)__double_as_longlong(v[u]) >> 52) & 0x7ffull);
                    em = e > em ? e : em;
                }
            }
        }
        atomicMax(&emax_s[j], em);
    }
    __syncthreads();
    if (threadIdx.x < nc) ex[row0 + c0 + threadIdx.x] = emax_s[threadIdx.x] - 1022;
    // two consecutive k per thread: each digit pair leaves in one 32-bit store
    const int kh = K >> 1;
    for (int e = threadIdx.x; e < nc * kh; e += blockDim.x) {
        const int j = e / kh, k = 2 * (e % kh);
        uint16_t d0[EMU_SLICES], d1[EMU_SLICES];
        slice_digits((unsigned long long)__double_as_longlong(T[k * (SC_COLS + 1) + j]),
                     emax_s[j], d0);
        slice_digits((unsigned long long)__double_as_longlong(T[(k + 1) * (SC_COLS + 1) + j]),
                     emax_s[j], d1);
#pragma unroll
        for (int p = 0; p < ES; ++p)
            *(uint32_t*)(S + ((int64_t)p * Mtot + row0 + c0 + j) * K + k) =
                (uint32_t)d0[p] | ((uint32_t)d1[p] << 16);
    }
}

// Drain group accumulators d0 .. d0 + 3 (one window) into the 64-bit
// fixed-point sums acc.  taddr addresses this warp's 32 TMEM lanes and 16
// columns; acc[8 hh + k] holds element k of the 16x256b fragment of lanes
// 16 hh .. 16 hh + 15.
__device__ __forceinline__ void drain_window(uint32_t taddr, int d0, long long (&acc)[ECOLS],
                                             uint64_t* freed, int lane) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int d = d0 + i;
        uint32_t v0[8], v1[8];
        tmem_ld16x256_x2(taddr + (uint32_t)(d * ETN), v0);
        tmem_ld16x256_x2(taddr + (16u << 16) + (uint32_t)(d * ETN), v1);
        tmem_wait_ld();
        if (i == 3) {   // the window has been read: the next tile's MMAs may overwrite it
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(freed))
                             : "memory");
        }
        const int sh = FIXB - 7 * d;
#pragma unroll
        for (int u = 0; u < ECOLS; ++u) {
            // an exact integer below 2^24 in magnitude
            const float f = __uint_as_float(u < 8 ? v0[u] : v1[u - 8]);
            const long long iv = (long long)__float2int_rn(f);
            acc[u] += sh >= 0 ? iv * (1ll << sh) : (iv >> (-sh));
        }
    }
}

__global__ void __launch_bounds__(ETHREADS, 1) k_tmu_emu(const __grid_constant__ CUtensorMap mapA,
                                                         const __grid_constant__ CUtensorMap mapB,
                                                         EmuArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* fullS = (uint64_t*)(smem + NSTAGE * STAGE);
    uint64_t* emptyS = fullS + NSTAGE;
    uint64_t* xdone = emptyS + NSTAGE;      // tile's X window complete
    uint64_t* ydone = xdone + 1;
    uint64_t* xfree = ydone + 1;            // X window read by the epilogue
    uint64_t* yfree = xfree + 1;
    uint32_t* tmem_slot = (uint32_t*)(yfree + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    if (a.st->info != 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // zero blocks of the B stacks
    for (int s2 = 0; s2 < NSTAGE; ++s2)
        for (int i = threadIdx.x; i < NZ * B_BL / 16; i += ETHREADS)
            *(uint4*)(smem + s2 * STAGE + ST_A + 16 * i) = make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x == 0) {
        for (int s2 = 0; s2 < NSTAGE; ++s2) {
            mbar_init(&fullS[s2], 1);
            mbar_init(&emptyS[s2], 1);
        }
        mbar_init(xdone, 1);
        mbar_init(ydone, 1);
        mbar_init(xfree, EPI_W);
        mbar_init(yfree, EPI_W);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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
    const int64_t G = gridDim.x, nitems = a.n1 + (a.nrect == 0 ? 0 : (a.nrect == 1 ? a.rend[0] : (a.nrect == 2 ? a.rend[1] : a.rend[2])));
    auto fail = [&]() {
        *abort_flag = 1;
        atomicExch(&a.st->error, 3);
    };

    if (warp == 0) {
        if (lane == 0) {   // TMA producer: per stage all eight A slices and B blocks
            int64_t c = 0;
            bool ok = true;
            for (int64_t idx = blockIdx.x; idx < nitems && ok && !*abort_flag; idx += G) {
                const EmuItem t = emu_item(idx, a);
                if (!t.valid) continue;
                for (int kc = 0; kc < nk; ++kc, ++c) {
                    const int s2 = (int)(c % NSTAGE);
                    if (c >= NSTAGE &&
                        !mbar_wait(&emptyS[s2], (uint32_t)(((c / NSTAGE) - 1) & 1))) {
                        fail();
                        ok = false;
                        break;
                    }
                    uint8_t* st = smem + s2 * STAGE;
                    mbar_expect_tx(&fullS[s2], STAGE_TX);
                    for (int p = 0; p < ES; ++p)
                        tma_load_2d(st + p * A_SL, &mapA, &fullS[s2], kc * EKC,
                                    (int)(p * a.Mtot + t.arow));
                    for (int q = 0; q < ES; ++q)
                        tma_load_2d(st + ST_A + (NZ + q) * B_BL, &mapB, &fullS[s2], kc * EKC,
                                    (int)(q * a.Mtot + t.brow));
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            int64_t c = 0, tc = 0;
            bool ok = true;
            const uint32_t tx = tmem, ty = tmem + 4 * ETN;
            for (int64_t idx = blockIdx.x; idx < nitems && ok && !*abort_flag; idx += G) {
                const EmuItem t = emu_item(idx, a);
                if (!t.valid) continue;
                for (int kc = 0; kc < nk && ok; ++kc, ++c) {
                    const int s2 = (int)(c % NSTAGE);
                    if (!mbar_wait(&fullS[s2], (uint32_t)((c / NSTAGE) & 1)) ||
                        (kc == 0 && tc >= 1 && !mbar_wait(xfree, (uint32_t)((tc - 1) & 1)))) {
                        fail();
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = smem_u32(smem + s2 * STAGE);
                    const uint64_t adesc = smem_desc64(sa), bdesc = smem_desc64(sa + ST_A);
                    // descriptors advance by 32 bytes per K = 16 step (field in 16-byte units)
#pragma unroll 1
                    for (int kk = 0; kk < EKC / 16; ++kk)
#pragma unroll 1
                        for (int p = 0; p < 4; ++p)   // X: groups 0-3, B blocks from NZ - p
                            mma_f16(tx, adesc + (uint64_t)((p * A_SL + kk * 32) >> 4),
                                    bdesc + (uint64_t)(((NZ - p) * B_BL + kk * 32) >> 4), a.idesc,
                                    (kc > 0 || kk > 0 || p > 0) ? 1u : 0u);
                    if (kc == nk - 1) mma_commit(xdone);
                    if (kc == 0 && tc >= 1 && !mbar_wait(yfree, (uint32_t)((tc - 1) & 1))) {
                        fail();
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
                    for (int kk = 0; kk < EKC / 16; ++kk)
#pragma unroll 1
                        for (int p = 0; p < ES; ++p)  // Y: groups 4-7, B blocks from NZ + 4 - p
                            mma_f16(ty, adesc + (uint64_t)((p * A_SL + kk * 32) >> 4),
                                    bdesc + (uint64_t)(((NZ + 4 - p) * B_BL + kk * 32) >> 4),
                                    a.idesc, (kc > 0 || kk > 0 || p > 0) ? 1u : 0u);
                    mma_commit(&emptyS[s2]);
                    if (kc == nk - 1) mma_commit(ydone);
                }
                ++tc;
            }
        }
    } else {
        // epilogue: warp (q, cq) drains TMEM lanes 32 q .. 32 q + 31 (tile rows)
        // and columns 16 cq .. 16 cq + 15 of every group in the 16x256b shape:
        // four neighbouring threads hold eight consecutive columns of one row,
        // so C moves in full 64-byte row segments
        const int ew = warp - 2;
        const int q = warp & 3;
        const int cq = ew >> 2;
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(cq * ECOLS);
        int64_t tc = 0;
        for (int64_t idx = blockIdx.x; idx < nitems; idx += G) {
            const EmuItem t = emu_item(idx, a);
            if (!t.valid) continue;
            long long acc[ECOLS];
#pragma unroll
            for (int u = 0; u < ECOLS; ++u) acc[u] = 0;
            if (*abort_flag || !mbar_wait(xdone, (uint32_t)(tc & 1))) {
                if (!*abort_flag) fail();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            drain_window(taddr, 0, acc, xfree, lane);
            if (*abort_flag || !mbar_wait(ydone, (uint32_t)(tc & 1))) {
                if (!*abort_flag) fail();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            drain_window(taddr, 4, acc, yfree, lane);
            ++tc;
            // C[i][j] -= A 2^(e_i + e_j - 54) over rows 32 q + 16 hh + 8 rr + lane / 4
            // and column pairs 16 cq + 8 j + 2 (lane % 4)
#pragma unroll
            for (int hr = 0; hr < 4; ++hr) {
                const int hh = hr >> 1, rr = hr & 1;
                const int ri = (int)(t.ti * ETM) + 32 * q + 16 * hh + 8 * rr + (lane >> 2);
                double* crow = nullptr;
                int ei = 0, colmax = 0, ej0 = 0, cdiv = 1, frow = -1, fcol = 0;
                bool vec = false;
                if (t.seg < 0) {
                    const int gi = (int)a.o + ri;
                    if (gi < a.M) {
                        crow = a.C + (int64_t)gi * a.ldc + a.o; ei = a.ex[gi];
                        colmax = (int)(a.M - a.o); ej0 = (int)a.o; vec = a.vec1;
                        frow = gi; fcol = (int)a.o;
                    }
                } else {
                    const EmuRect e = rect_of(a, t.seg);
                    if (ri < e.na) {
                        crow = e.C + (int64_t)ri * e.ldc; ei = a.ex[e.a0 + ri];
                        colmax = e.nb; ej0 = e.b0; cdiv = e.cdiv; vec = e.vec;
                        frow = e.frow >= 0 ? e.frow + ri : -1; fcol = e.fcol;
                    }
                }
                if (!crow) continue;
                double2 cv[2];
                const int gj0 = (int)(t.tj * ETN) + 16 * cq + 2 * (lane & 3);
#pragma unroll
                for (int j = 0; j < 2; ++j) {   // loads first
                    const int gj = gj0 + 8 * j;
                    if (vec && gj + 1 < colmax) {
                        cv[j] = *(const double2*)(crow + gj);
                    } else {
                        cv[j].x = (gj < colmax && (cdiv == 1 || gj % cdiv == 0))
                                      ? crow[cdiv == 1 ? gj : gj / cdiv] : 0.0;
                        cv[j].y = (gj + 1 < colmax && (cdiv == 1 || (gj + 1) % cdiv == 0))
                                      ? crow[cdiv == 1 ? gj + 1 : (gj + 1) / cdiv] : 0.0;
                    }
                }
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int gj = gj0 + 8 * j;
                    double v[2] = {cv[j].x, cv[j].y};
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        if (gj + c >= colmax) continue;
                        // A 2^(e_i + e_j - 54) assembled with integer operations
                        // (one FP64 instruction per element: the subtraction)
                        const long long av = acc[8 * hh + 4 * j + 2 * rr + c];
                        const int sc = ei + a.ex[ej0 + gj + c] - 54;
                        bool normal;
                        double y = i64_scaled_to_f64(av, sc, normal);
                        if (!normal) y = ldexp((double)av, sc);
                        v[c] -= y;
                        if (frow >= 0)
#pragma unroll
                            for (int f = 0; f < MAX_CF; ++f)   // static indices: no local copy
                                if (f < a.ncf && a.cf[f].row == frow && a.cf[f].col == fcol + gj + c)
                                    v[c] += a.cf[f].delta;
                    }
                    if (vec && gj + 1 < colmax) {
                        *(double2*)(crow + gj) = make_double2(v[0], v[1]);
                    } else {
#pragma unroll
                        for (int c = 0; c < 2; ++c)
                            if (gj + c < colmax && (cdiv == 1 || (gj + c) % cdiv == 0))
                                crow[cdiv == 1 ? gj + c : (gj + c) / cdiv] = v[c];
                    }
                }
            }
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
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int64_t emu_rows(int64_t n, int64_t nb) {
    return n + 2 * ((n + nb - 1) / nb);
}

size_t emu_slice_bytes(int64_t n, int64_t nb) {
    return sizeof(uint16_t) * (size_t)ES * (size_t)emu_rows(n, nb) * (size_t)nb;
}

cudaError_t launch_slice_cols(const double* P, int64_t ld, int64_t K, int64_t ncols, uint16_t* S,
                              int64_t Mtot, int64_t row0, int* ex, cudaStream_t s) {
    return launch_slice_cols_chunked(P, ld, K, K, ncols, S, Mtot, row0, 0, ex, s);
}

cudaError_t launch_slice_cols_chunked(const double* P, int64_t ld, int64_t K, int64_t mrows,
                                      int64_t ncols, uint16_t* S, int64_t Mtot, int64_t row0,
                                      int64_t rstride, int* ex, cudaStream_t s) {
    if (ncols <= 0 || mrows <= 0) return cudaSuccess;
    const int64_t nch = (mrows + K - 1) / K;
    if (K % 32 != 0 || K > 256 || nch > 65535 || row0 + (nch - 1) * rstride + ncols > Mtot)
        return cudaErrorInvalidValue;
    const size_t smem = sizeof(double) * (size_t)K * (SC_COLS + 1);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_slice_cols, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(sizeof(double) * 256 * (SC_COLS + 1)));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const dim3 grid((unsigned)((ncols + SC_COLS - 1) / SC_COLS), (unsigned)nch);
    k_slice_cols<<<grid, 256, smem, s>>>(P, ld, (int)K, mrows, ncols, S, Mtot, row0, rstride, ex);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_slice_panel(const double* P, int64_t lda, int64_t m, int64_t kb, uint16_t* S,
                               int64_t Mtot, int64_t row0, int* ex, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    if (kb % 32 != 0 || kb > 256 || row0 + m > Mtot) return cudaErrorInvalidValue;
    k_slice_panel<<<(unsigned)((m + 7) / 8), 256, 0, s>>>(P, lda, m, (int)kb, S, Mtot, row0, ex);
    note_launch();
    return cudaGetLastError();
}

// One launch of the emulated update: the lower block triangle of the trailing
// matrix C (rows and columns [o, M), blocks of g; M <= o: none) and up to three
// rectangles, all from the slice tensor S (8 x mtot x kb BF16) and the row
// exponents ex.  Compute faults are in trailing coordinates.  max_grid > 0
// caps the persistent grid (SMs left to a concurrent panel factorization).
cudaError_t launch_tmu_emu(const uint16_t* S, const int* ex, int64_t mtot, int64_t kb, double* C,
                           int64_t ldc, int64_t M, int64_t o, int64_t g, const EmuRectHost* rects,
                           int nrect, const ComputeFault* cf, int ncf, int max_grid, DevStatus* st,
                           cudaStream_t s) {
    if (kb % EKC != 0 || kb > EKMAX || g % ETM != 0 || nrect < 0 || nrect > 3 || o % g != 0)
        return cudaErrorInvalidValue;
    if ((int64_t)ES * mtot + ETM > INT32_MAX) return cudaErrorInvalidValue;
    EmuArgs a{};
    a.C = C; a.ldc = ldc; a.M = M; a.o = o; a.K = kb; a.ex = ex; a.st = st; a.Mtot = mtot;
    a.vec1 = ((uintptr_t)C % 16 == 0) && ldc % 2 == 0;
    a.ncf = 0;
    for (int f = 0; f < ncf && f < MAX_CF; ++f) a.cf[a.ncf++] = cf[f];
    const int64_t qb = M > o ? (M - o + g - 1) / g : 0;
    a.rm = g / ETM;
    a.rn = g / ETN;
    a.n1 = qb * (qb + 1) / 2 * a.rm * a.rn;
    int64_t tot = 0;
    for (int r = 0; r < nrect; ++r) {
        const EmuRectHost& h = rects[r];
        if (h.na <= 0 || h.nb <= 0) continue;
        if (h.a0 < 0 || h.b0 < 0 || h.a0 + h.na > mtot || h.b0 + h.nb > mtot || h.cdiv < 1)
            return cudaErrorInvalidValue;
        EmuRect& e = a.rect[a.nrect];
        e.C = h.C; e.ldc = h.ldc;
        e.a0 = (int)h.a0; e.na = (int)h.na; e.b0 = (int)h.b0; e.nb = (int)h.nb;
        e.cdiv = h.cdiv;
        e.ntj = (int)((h.nb + ETN - 1) / ETN);
        e.frow = (int)h.frow; e.fcol = (int)h.fcol;
        e.vec = h.cdiv == 1 && ((uintptr_t)h.C % 16 == 0) && h.ldc % 2 == 0;
        tot += (h.na + ETM - 1) / ETM * e.ntj;
        a.rend[a.nrect] = tot;
        ++a.nrect;
    }
    const int64_t items = a.n1 + tot;
    if (items == 0) return cudaSuccess;
    CUtensorMap mapA, mapB;
    if (!encode_slices(&mapA, S, ES * mtot, kb, ETM) || !encode_slices(&mapB, S, ES * mtot, kb, ETN))
        return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_tmu_emu, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)E_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    // kind::f16 instruction descriptor: D F32, A/B BF16, K-major, N = 256, M = 128
    a.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(256 >> 3) << 17) |
              ((uint32_t)(ETM >> 4) << 24);
    int64_t grid = num_sms();
    if (max_grid > 0 && grid > max_grid) grid = max_grid;
    if (grid > items) grid = items;
    k_tmu_emu<<<(unsigned)grid, ETHREADS, E_SMEM, s>>>(mapA, mapB, a);
    note_launch();
    return cudaGetLastError();
}

}  // namespace abft
