// k_batched.cu -- batched ABFT Cholesky of many small SPD matrices in one
// persistent launch (Sec. 2.1 blocked algorithm and Sec. 3.1.2 checksums at
// the scope of one CTA per matrix).
//
// Each CTA repeatedly takes the next matrix from an atomic queue (the host
// orders the descriptors by decreasing n, so the longest factorizations
// start first) and factors it with block size B (32 or 64, per descriptor):
//   PD   the B x B diagonal block in shared memory (right-looking potf2 with
//        one reciprocal square root per pivot; FP32 two columns per barrier,
//        FP64 full-warp packed updates) and its column-sum check;
//   PU   one thread per panel row (and per checksum row) solves x L^T = a with
//        L_kk's rows read four values at a time from shared memory; panel
//        tiles are verified with the weighted column checksums;
//   TMU  B x B output tiles of the lower block triangle (diagonal tiles kept
//        full: FP64 computes the groups on and below the diagonal and mirrors
//        them), L_I and L_J staged transposed in shared memory by cp.async, C
//        read-modify-written in global memory (L2-resident for these sizes),
//        checksum borders updated from the carried panel checksums;
//   then the optional injected fault and the verify / locate / correct of
//   every trailing tile (full checksums: 0D, 1D, checksum-only, 2D classes).
// T is the arithmetic type (double or float); the threshold uses its unit
// roundoff.  There are no spin waits: the only cross-CTA interaction is the
// atomic queue counter.
#include <math.h>

#include <atomic>

#include "common.cuh"
#include "fp_bits.cuh"

namespace abft {

namespace {

constexpr int BT = 256;   // threads per CTA
constexpr int MAXN = 512;
constexpr int MAXB = 64;
constexpr int MAXNT = MAXN / 32;

template <typename T>
__device__ __forceinline__ T tabs(T x) { return x < (T)0 ? -x : x; }

// 1 / sqrt(x) (CUDA's rsqrtf / rsqrt)
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }

// Element e of a lower triangle enumerated row by row ((0,0), (1,0), (1,1),
// (2,0), ...) as (row << 8) | column.
__device__ __forceinline__ int tri_pair(int e) {
    int i = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
    if ((i + 1) * (i + 2) / 2 <= e) ++i;
    if (i * (i + 1) / 2 > e) --i;
    return (i << 8) | (e - i * (i + 1) / 2);
}

// Transposed panels in shared memory: element (j, p) of a block's panel rows
// at p LDT + j, rows of LDT values (16-byte aligned for the vector reads).
constexpr int LDT = MAXB + 4;

// Register tile of the update, R = B / 16 outputs per thread and direction.
// FP32: thread (tx, ty) owns rows R ty + a and columns R tx + b, so that each
// operand row is one R-wide vector read per p (scalar reads would make the
// shared-memory pipe, not the FMA pipe, the bound); C is loaded before the
// product.  FP64: rows ty + 16 a and columns tx + 16 b, so that whole 16 x 16
// groups can be skipped (the FP64 pipe is the bound).
template <typename T, int B>
struct TileMap {
    static constexpr int R = B / 16;
    static constexpr bool CONTIG = sizeof(T) == 4;
    static constexpr bool PREF_C = sizeof(T) == 4;
    __device__ static int row(int ty, int a) { return CONTIG ? R * ty + a : ty + 16 * a; }
    __device__ static int col(int tx, int b) { return CONTIG ? R * tx + b : tx + 16 * b; }
    __device__ static void load(const T* rowp, int tt, T (&v)[R]) {
        if constexpr (CONTIG && R == 4) {
            const float4 q = *reinterpret_cast<const float4*>(rowp + 4 * tt);
            v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
        } else if constexpr (CONTIG && R == 2) {
            const float2 q = *reinterpret_cast<const float2*>(rowp + 2 * tt);
            v[0] = q.x; v[1] = q.y;
        } else {
#pragma unroll
            for (int a = 0; a < R; ++a) v[a] = rowp[tt + 16 * a];
        }
    }
};

// acc[a][b] += sum_p sA[p][row a] sB[p][col b] over the thread's register
// tile, p in increasing order.  SEL picks the 16 x 16 groups (FP64 mapping):
// 0 every group, 1 those on or below the diagonal (b <= a: a full diagonal
// tile), 2 those inside the tile's edge (a < ra, b < rb) and, on a diagonal
// tile, on or below it.  The choice is made once per tile, outside the loop.
template <typename Map, int SEL, typename T, int R>
__device__ __forceinline__ void tile_product(const T* sA, const T* sB, int tx, int ty, int ra, int rb,
                                             bool diag, T (&acc)[R][R]) {
    constexpr int B = 16 * R;
#pragma unroll 8
    for (int p = 0; p < B; ++p) {
        T av[R], bv[R];
        Map::load(sA + p * LDT, ty, av);
        Map::load(sB + p * LDT, tx, bv);
#pragma unroll
        for (int a = 0; a < R; ++a)
#pragma unroll
            for (int b = 0; b < R; ++b) {
                if (SEL == 1 && b > a) continue;
                if (SEL == 2 && !(a < ra && b < rb && !(diag && b > a))) continue;
                acc[a][b] = fma(av[a], bv[b], acc[a][b]);
            }
    }
}

// Four consecutive values from 16-byte aligned shared memory.
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// 4- or 8-byte global -> shared copy (cp.async), zero-filled when !pred
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src, bool pred) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src),
                 "n"((int)sizeof(T)), "r"(pred ? (int)sizeof(T) : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Panel rows q0 + [0, nq) of block column K0 (B values each) into dst,
// transposed: dst[p LDT + j] = A[(q0 + j) lda + K0 + p], zero for j >= nq.  A
// warp copies 4 rows x 8 consecutive values (a 32-byte stretch of each row);
// for FP32 its transposed stores fall in 32 distinct banks (LDT = 4 mod 32).
template <typename T, int B>
__device__ __forceinline__ void stage_panel_t(T* dst, const T* A, int64_t lda, int q0, int nq, int K0) {
#pragma unroll
    for (int e = threadIdx.x; e < B * B; e += BT) {
        const int lane = e & 31, grp = e >> 5;
        const int j = (grp / (B / 8)) * 4 + (lane >> 3);
        const int p = (grp % (B / 8)) * 8 + (lane & 7);
        const bool ok = j < nq;
        cp_async_elem<T>(dst + p * LDT + j, A + (int64_t)(q0 + (ok ? j : 0)) * lda + K0 + p, ok);
    }
}

// Per-CTA global scratch: checksums and the saved diagonal-block upper triangles.
template <typename T>
struct Scratch {
    T* Cc;    // MAXNT x MAXN column sums (row I: block row I)
    T* Cw;    // MAXNT x MAXN weighted column sums
    T* Cr;    // MAXN x MAXNT row sums
    T* save;  // MAXN x MAXB saved strict upper triangles of the diagonal blocks
};

template <typename T>
__device__ void record(abft_batch_status* st, int step, int kind, int row, int col, int* s_first) {
    if (atomicCAS(s_first, 0, 1) == 0) {
        st->ev_step = step;
        st->ev_kind = kind;
        st->ev_row = row;
        st->ev_col = col;
    }
}

// Sums of one tile (nr x nc at P, ld; nc <= 64) into shared memory: colsum[j],
// wsum[j] (weights 1..nr) and rowsum[i].  Warp w takes rows w, w + 8, ...;
// lane l holds columns l and l + 32, so each row is one coalesced load per
// warp and its sum is a warp shuffle reduction; the eight warps' column
// partials are added in warp order through shared memory (part: 8 x 64).
template <typename T>
__device__ void tile_sums(const T* P, int64_t ld, int nr, int nc, T* colsum, T* wsum, T* rowsum,
                          T* part) {
    const int t = threadIdx.x, w = t >> 5, l = t & 31;
    T c0 = 0, c1 = 0, w0 = 0, w1 = 0;
    // all of the warp's rows (at most MAXB / 8) loaded before they are summed
    T va[MAXB / 8], vb[MAXB / 8];
#pragma unroll
    for (int q = 0; q < MAXB / 8; ++q) {
        const int i = w + 8 * q;
        const T* row = P + (int64_t)i * ld;
        va[q] = (i < nr && l < nc) ? row[l] : (T)0;
        vb[q] = (i < nr && l + 32 < nc) ? row[l + 32] : (T)0;
    }
#pragma unroll
    for (int q = 0; q < MAXB / 8; ++q) {
        const int i = w + 8 * q;
        if (i >= nr) break;
        const T v0 = va[q], v1 = vb[q];
        const T wi = (T)(i + 1);
        c0 += v0;
        c1 += v1;
        w0 = fma(wi, v0, w0);
        w1 = fma(wi, v1, w1);
        T rs = v0 + v1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
        if (l == 0) rowsum[i] = rs;
    }
    T* pc = part;            // [8][64] column partials
    T* pw = part + 8 * 64;   // [8][64] weighted partials
    pc[w * 64 + l] = c0;
    pc[w * 64 + l + 32] = c1;
    pw[w * 64 + l] = w0;
    pw[w * 64 + l + 32] = w1;
    __syncthreads();
    for (int j = t; j < nc; j += BT) {
        T s = 0, sw = 0;
        for (int q = 0; q < BT / 32; ++q) {
            s += pc[q * 64 + j];
            sw += pw[q * 64 + j];
        }
        colsum[j] = s;
        wsum[j] = sw;
    }
    __syncthreads();
}

// tile_sums for FP64 tiles in exact 64-bit fixed point: every entry truncated to
// a multiple of 2^(vexp - 1075) (vexp bounds every entry's biased exponent:
// the Schur complements of an SPD matrix are bounded by max a_ii, the panel by
// its square root), the weighted sums in units 2^10 larger so that they stay
// inside 64 bits; the integer pipes instead of the FP64 pipe, which the
// update needs.  Returns false, with nothing written, when an entry exceeds
// the bound (an injected error, a NaN): the caller then sums in FP64.
__device__ bool tile_sums_fixed(const double* P, int64_t ld, int nr, int nc, int vexp,
                                double* colsum, double* wsum, double* rowsum, double* part) {
    const int t = threadIdx.x, w = t >> 5, l = t & 31;
    long long c0 = 0, c1 = 0, w0 = 0, w1 = 0;
    int emax = 0;
    long long* irow = reinterpret_cast<long long*>(rowsum);
#pragma unroll 4
    for (int i = w; i < nr; i += BT / 32) {
        const double* row = P + (int64_t)i * ld;
        const long long q0 = l < nc ? to_fixed(row[l], vexp, emax) : 0ll;
        const long long q1 = l + 32 < nc ? to_fixed(row[l + 32], vexp, emax) : 0ll;
        c0 += q0;
        c1 += q1;
        w0 += (long long)(i + 1) * (q0 >> 10);
        w1 += (long long)(i + 1) * (q1 >> 10);
        const long long rs = warp_sum_ll(q0 + q1);
        if (l == 0) irow[i] = rs;
    }
    if (__syncthreads_or(emax > vexp ? 1 : 0)) return false;
    long long* pc = reinterpret_cast<long long*>(part);   // [8][64] column partials
    long long* pw = pc + 8 * 64;                          // [8][64] weighted partials
    pc[w * 64 + l] = c0;
    pc[w * 64 + l + 32] = c1;
    pw[w * 64 + l] = w0;
    pw[w * 64 + l + 32] = w1;
    __syncthreads();
    const double unit = ldexp(1.0, vexp - 1075), wunit = ldexp(1.0, vexp - 1065);
    for (int j = t; j < nc; j += BT) {
        long long s = 0, sw = 0;
        for (int q = 0; q < BT / 32; ++q) {
            s += pc[q * 64 + j];
            sw += pw[q * 64 + j];
        }
        colsum[j] = (double)s * unit;
        wsum[j] = (double)sw * wunit;
    }
    for (int i = t; i < nr; i += BT) rowsum[i] = (double)irow[i] * unit;
    __syncthreads();
    return true;
}

template <typename T>
__device__ void tile_sums_any(const T* P, int64_t ld, int nr, int nc, int vexp, T* colsum, T* wsum,
                              T* rowsum, T* part) {
    if constexpr (sizeof(T) == 8) {
        if (vexp > 0 && tile_sums_fixed((const double*)P, ld, nr, nc, vexp, (double*)colsum,
                                        (double*)wsum, (double*)rowsum, (double*)part))
            return;
    }
    tile_sums<T>(P, ld, nr, nc, colsum, wsum, rowsum, part);
}

// Verify one tile against its carried checksums and correct it (same rules as
// the large-matrix kernel).  single = 1: weighted column checksums only.
template <typename T>
__device__ void verify_tile(T* P, int64_t ld, int r0, int c0, int nr, int nc, T* cc, T* cw, T* cr,
                            int crs, T tau, int single, int step, abft_batch_status* st,
                            T* colsum, T* wsum, T* rowsum, T* part, int* sflag, int* s_first,
                            int vexp) {
    const int t = threadIdx.x;
    // the carried checksums of this thread's column / row (nr, nc <= MAXB <= BT),
    // loaded before the sums so that their latency overlaps them
    const T ccv = t < nc ? cc[t] : (T)0, cwv = t < nc ? cw[t] : (T)0;
    const T crv = (!single && t < nr) ? cr[t * crs] : (T)0;
    tile_sums_any<T>(P, ld, nr, nc, vexp, colsum, wsum, rowsum, part);
    if (t == 0) { sflag[0] = 0; sflag[1] = 0; sflag[2] = 1 << 30; sflag[3] = 1 << 30; }
    __syncthreads();
    if (t < nc) {
        colsum[t] -= ccv;
        wsum[t] -= cwv;
        if (!(tabs(colsum[t]) <= tau)) { atomicAdd(&sflag[0], 1); atomicMin(&sflag[2], t); }
    }
    if (!single && t < nr) {
        rowsum[t] -= crv;
        if (!(tabs(rowsum[t]) <= tau)) { atomicAdd(&sflag[1], 1); atomicMin(&sflag[3], t); }
    }
    __syncthreads();
    const int nfc = sflag[0], nfr = sflag[1], fc = sflag[2], fr = sflag[3];
    if (nfc == 0 && nfr == 0) return;
    if (t == 0) atomicAdd(&st->detected, 1);
    if (single) {
        for (int j = t; j < nc; j += BT) {
            T dc = colsum[j];
            if (tabs(dc) <= tau) continue;
            T rho = wsum[j] / dc;
            T ri = rint(rho);
            int i = (int)ri - 1;
            if (tabs(rho - ri) <= (T)0.05 && i >= 0 && i < nr) {
                P[(int64_t)i * ld + j] -= dc;
                atomicAdd(&st->corrected, 1);
                record<T>(st, step, EV_0D, r0 + i, c0 + j, s_first);
            } else {
                atomicAdd(&st->uncorrectable, 1);
                record<T>(st, step, EV_UNCORR, r0, c0 + j, s_first);
            }
        }
    } else if (nfr == 1 && nfc == 1) {
        if (t == 0) {
            T dc = colsum[fc], dr = rowsum[fr];
            if (tabs(dc - dr) <= tau) {
                P[(int64_t)fr * ld + fc] -= dc;
                atomicAdd(&st->corrected, 1);
                record<T>(st, step, EV_0D, r0 + fr, c0 + fc, s_first);
            } else {
                atomicAdd(&st->uncorrectable, 1);
                record<T>(st, step, EV_UNCORR, r0, c0, s_first);
            }
        }
    } else if (nfr == 1 && nfc >= 2) {
        for (int j = t; j < nc; j += BT)
            if (!(tabs(colsum[j]) <= tau)) {
                P[(int64_t)fr * ld + j] -= colsum[j];
                atomicAdd(&st->corrected, 1);
                record<T>(st, step, EV_ROW, r0 + fr, c0 + j, s_first);
            }
    } else if (nfr >= 2 && nfc == 1) {
        for (int i = t; i < nr; i += BT)
            if (!(tabs(rowsum[i]) <= tau)) {
                P[(int64_t)i * ld + fc] -= rowsum[i];
                atomicAdd(&st->corrected, 1);
                record<T>(st, step, EV_COL, r0 + i, c0 + fc, s_first);
            }
    } else if (nfr == 0 || nfc == 0) {
        for (int j = t; j < nc; j += BT) cc[j] += colsum[j];
        for (int i = t; i < nr; i += BT) cr[i * crs] += rowsum[i];
        if (t == 0) record<T>(st, step, EV_CKSUM, r0, c0, s_first);
    } else if (t == 0) {
        atomicAdd(&st->uncorrectable, 1);
        record<T>(st, step, EV_UNCORR, r0, c0, s_first);
    }
    __syncthreads();
}

template <typename T, int B>
__device__ void factor_one(const abft_batch_item& it, int mode, T tau_scale, Scratch<T> S,
                           abft_batch_status* st, T (*sL)[MAXB + 1], T* sIt, T* sJt, T* colsum, T* wsum, T* rowsum, T* rdiag, int* sflag,
                           int* s_first, int* s_fail) {
    T* A = (T*)it.A;
    const int64_t lda = it.lda;
    const int n = it.n;
    const int nt = (n + B - 1) / B;
    const int t = threadIdx.x;
    const bool check = mode != MODE_NONE;
    using Map = TileMap<T, B>;
    const T u = sizeof(T) == 8 ? (T)0x1p-53 : (T)0x1p-24;
    // an injected fault is used only when it lies inside this matrix
    const bool fok = it.fstep >= 0 && it.frow >= 0 && it.frow < n && it.fcol >= 0 && it.fcol < n;
    // threshold tau = tau_scale * 8 u n B max_i a_ii
    if (t == 0) { *s_first = 0; *s_fail = -1; }
    T m = 0;
    for (int i = t; i < n; i += BT) m = fmax(m, A[(int64_t)i * lda + i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((t & 31) == 0) colsum[t >> 5] = m;
    __syncthreads();
    T dmax = 0;
    for (int w = 0; w < BT / 32; ++w) dmax = fmax(dmax, colsum[w]);
    const T tau = tau_scale * (T)8 * u * (T)n * (T)B * dmax;
    // fixed-point bound of the FP64 sums: max(max a_ii, sqrt(max a_ii))
    int vexp = 0;
    if (sizeof(T) == 8) {
        const double bnd = fmax((double)dmax, sqrt((double)dmax));
        const int ve = (int)((__double_as_longlong(bnd) >> 52) & 0x7ff);
        if (bnd > 0.0 && bnd < 1e300 && ve >= kFixedMinExp) vexp = ve;
    }
    __syncthreads();
    // mirror the diagonal blocks (save their strict upper triangles), each
    // block through shared memory: read row by row, the mirrored upper
    // triangle written row by row
    for (int K = 0; K < nt; ++K) {
        const int K0 = K * B, kb = min(B, n - K0);
#pragma unroll 4
        for (int e = t; e < kb * kb; e += BT) {
            const int i = e / kb, j = e % kb;
            sL[i][j] = A[(int64_t)(K0 + i) * lda + K0 + j];
        }
        __syncthreads();
        for (int e = t; e < kb * kb; e += BT) {
            const int i = e / kb, j = e % kb;
            if (j > i) {
                S.save[(K0 + i) * MAXB + j] = sL[i][j];
                A[(int64_t)(K0 + i) * lda + K0 + j] = sL[j][i];
            }
        }
        __syncthreads();
    }
    if (check)
        for (int I = 0; I < nt; ++I)
            for (int J = 0; J <= I; ++J) {
                const int r0 = I * B, c0 = J * B, nr = min(B, n - r0), nc = min(B, n - c0);
                tile_sums_any<T>(A + (int64_t)r0 * lda + c0, lda, nr, nc, vexp, colsum, wsum,
                                 rowsum, sJt);
                for (int j = t; j < nc; j += BT) {
                    S.Cc[I * MAXN + c0 + j] = colsum[j];
                    S.Cw[I * MAXN + c0 + j] = wsum[j];
                }
                for (int i = t; i < nr; i += BT) S.Cr[(r0 + i) * MAXNT + J] = rowsum[i];
                __syncthreads();
            }
    for (int k = 0; k < nt; ++k) {
        const int K0 = k * B, kb = min(B, n - K0), T0 = K0 + kb, mrows = n - T0;
        // ---- PD: right-looking potf2 of the diagonal block in shared memory.
        // Phase j updates the lower triangle of rows and columns j + 1 .. kb - 1
        // with column j.  The pivot's reciprocal square root r is taken once
        // (CUDA's rsqrt), l_jj = d r, and r scales the column: one long
        // operation per column on the dependent chain instead of a square
        // root and a division.  Thread 0 updates the next pivot first and
        // publishes l_jj and r for the next phase.
        //   FP32: two columns per barrier on a 16 x 16 thread grid (below).
        //   FP64: column j is scaled first (one FP64 multiply per element
        //   instead of two per update), then a second barrier; the update's
        //   elements are spread over all threads in row-major order (thread t
        //   takes elements t, t + BT, ...: full warps, which is what the FP64
        //   pipe charges for; the pairs are recomputed per phase, which keeps
        //   registers free).
        for (int e = t; e < kb * kb; e += BT) {
            int i = e / kb, j = e % kb;
            if (j <= i) sL[i][j] = A[(int64_t)(K0 + i) * lda + K0 + j];
        }
        __syncthreads();
        if constexpr (sizeof(T) == 4) {
            // Two columns per barrier.  Phase j (columns j and j + 1, whose
            // 2 x 2 diagonal block thread 0 has factored: r_j, r_j+1 and the
            // scaled l_j+1,j published) applies the rank-2 update to rows and
            // columns from j + 2 with both columns scaled where they are used
            // (l_i,j+1 = (a_i,j+1 - l_ij l_j+1,j) r_j+1), stores the previous
            // pair scaled, and thread 0 updates and factors the next 2 x 2
            // block itself.  Every element sees the same fused multiply-adds
            // in the same order as with one column per barrier.
            const int tx = t & 15, ty = t >> 4;
            if (t == 0) {
                const T d = sL[0][0];
                if (!(d > (T)0)) *s_fail = 0;
                else {
                    const T r = rsqrt_t(d);
                    sL[0][0] = d * r;
                    rdiag[0] = r;
                    if (kb > 1) {
                        const T l = sL[1][0] * r;
                        sL[1][0] = l;
                        const T e = fma(-l, l, sL[1][1]);
                        if (!(e > (T)0)) *s_fail = 1;
                        else { const T r1 = rsqrt_t(e); sL[1][1] = e * r1; rdiag[1] = r1; }
                    }
                }
            }
            for (int j = 0; j < kb; j += 2) {
                __syncthreads();
                if (*s_fail >= 0) break;
                const bool two = j + 1 < kb;
                const T r0 = rdiag[j];
                const T r1 = two ? rdiag[j + 1] : (T)0;
                const T l10 = two ? sL[j + 1][j] : (T)0;
                if (j > 0) {   // the previous pair, rows >= j, stored scaled
                    const T p0 = rdiag[j - 2], p1 = rdiag[j - 1], pl = sL[j - 1][j - 2];
                    for (int i = j + t; i < kb; i += BT) {
                        const T a0 = sL[i][j - 2] * p0;
                        sL[i][j - 1] = fma(-a0, pl, sL[i][j - 1]) * p1;
                        sL[i][j - 2] = a0;
                    }
                }
                if (!two) continue;
                if (t == 0 && j + 2 < kb) {   // the next diagonal block, rows j + 2 (.. j + 3)
                    const int g = j + 2;
                    const T c0 = sL[g][j] * r0;
                    const T c1 = fma(-c0, l10, sL[g][j + 1]) * r1;
                    T d = fma(-c0, c0, sL[g][g]);
                    d = fma(-c1, c1, d);
                    if (!(d > (T)0)) *s_fail = g;
                    else {
                        const T r = rsqrt_t(d);
                        sL[g][g] = d * r;
                        rdiag[g] = r;
                        if (g + 1 < kb) {
                            const T e0 = sL[g + 1][j] * r0;
                            const T e1 = fma(-e0, l10, sL[g + 1][j + 1]) * r1;
                            T x = fma(-e0, c0, sL[g + 1][g]);
                            x = fma(-e1, c1, x);
                            const T l32 = x * r;
                            sL[g + 1][g] = l32;
                            T y = fma(-e0, e0, sL[g + 1][g + 1]);
                            y = fma(-e1, e1, y);
                            y = fma(-l32, l32, y);
                            if (!(y > (T)0)) *s_fail = g + 1;
                            else { const T r3 = rsqrt_t(y); sL[g + 1][g + 1] = y * r3; rdiag[g + 1] = r3; }
                        }
                    }
                }
                // rank-2 update of rows j + 4 .. kb - 1 (rows j + 2, j + 3 belong
                // to thread 0's block), columns j + 2 .. i
                T lv0[4], lv1[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int l = j + 2 + tx + 16 * u;
                    const T v0 = l < kb ? sL[l][j] * r0 : (T)0;
                    lv0[u] = v0;
                    lv1[u] = l < kb ? fma(-v0, l10, sL[l][j + 1]) * r1 : (T)0;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = j + 2 + ty + 16 * q;
                    if (i >= kb) break;
                    if (i < j + 4) continue;
                    const T li0 = sL[i][j] * r0;
                    const T li1 = fma(-li0, l10, sL[i][j + 1]) * r1;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int l = j + 2 + tx + 16 * u;
                        if (l > i) break;
                        T v = fma(-li0, lv0[u], sL[i][l]);
                        sL[i][l] = fma(-li1, lv1[u], v);
                    }
                }
            }
        } else {
            if (t == 0) {
                const T d = sL[0][0];
                if (!(d > (T)0)) *s_fail = 0;
                else { const T r = rsqrt_t(d); sL[0][0] = d * r; rdiag[0] = r; }
            }
            for (int j = 0; j < kb; ++j) {
                __syncthreads();
                if (*s_fail >= 0) break;
                const T rj = rdiag[j];
                for (int i = j + 1 + t; i < kb; i += BT) sL[i][j] = sL[i][j] * rj;
                const int m = kb - j - 1, M = m * (m + 1) / 2;
                __syncthreads();
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (t + BT * q >= M) break;
                    const int pq = tri_pair(t + BT * q);
                    const int i = j + 1 + (pq >> 8), l = j + 1 + (pq & 255);
                    if (t + BT * q == 0) {
                        const T d = sL[i][i] - sL[i][j] * sL[i][j];
                        if (!(d > (T)0)) *s_fail = j + 1;
                        else { const T r = rsqrt_t(d); sL[i][i] = d * r; rdiag[i] = r; }
                    } else {
                        sL[i][l] -= sL[i][j] * sL[l][j];
                    }
                }
            }
        }
        __syncthreads();
        if (*s_fail >= 0) {
            if (t == 0) st->info = K0 + *s_fail + 1;
            break;
        }
        for (int e = t; e < kb * kb; e += BT) {
            int i = e / kb, j = e % kb;
            if (j <= i) A[(int64_t)(K0 + i) * lda + K0 + j] = sL[i][j];
        }
        // rdiag holds the pivots' reciprocals for the panel solve
        if (check) {   // PD check on column sums
            for (int p = t; p < kb; p += BT) {
                T s = 0;
                for (int q = p; q < kb; ++q) s += sL[q][p];
                colsum[p] = s;
            }
            __syncthreads();
            for (int j = t; j < kb; j += BT) {
                T y = 0;
                for (int p = 0; p <= j; ++p) y += colsum[p] * sL[j][p];
                if (!(tabs(y - S.Cc[k * MAXN + K0 + j]) <= tau)) {
                    atomicAdd(&st->detected, 1);
                    atomicAdd(&st->uncorrectable, 1);
                    record<T>(st, k, EV_PD, K0 + j, K0 + j, s_first);
                }
            }
        }
        // L_kk row by row at stride LDT (16-byte aligned rows) for the panel
        // solve's vector reads; sIt is free until the update
        T* const sLr = sIt;
        for (int e = t; e < kb * kb; e += BT) {
            const int i = e / kb, j = e % kb;
            sLr[i * LDT + j] = j <= i ? sL[i][j] : (T)0;
        }
        __syncthreads();
        if (mrows <= 0) break;
        // ---- PU: x L^T = a for the panel rows and the checksum rows, one thread
        // per row.  A block with rows below it is never ragged (kb = B, a
        // multiple of 32), so the row's unknowns are solved CH at a time in
        // registers (16 for FP32, whose 64 registers per thread cannot hold
        // 32 of them without spilling; 32 for FP64): each chunk first takes
        // the terms of the earlier chunks (re-read from the row, which this
        // thread wrote), then substitutes inside the chunk; every unknown's
        // terms form one fused multiply-add chain in p order.  L_kk's rows are
        // read four values at a time.
        constexpr int CH = sizeof(T) == 4 ? 16 : 32;
        const int ncs = check ? 2 * (nt - k - 1) : 0;
        for (int rr = t; rr < mrows + ncs; rr += BT) {
            T* row;
            if (rr < mrows) row = A + (int64_t)(T0 + rr) * lda + K0;
            else {
                int c = rr - mrows, I = k + 1 + c / 2;
                row = ((c & 1) ? S.Cw : S.Cc) + I * MAXN + K0;
            }
            for (int c0 = 0; c0 < B; c0 += CH) {
                T x[CH];
#pragma unroll
                for (int q = 0; q < CH; ++q) x[q] = row[c0 + q];
                for (int p = 0; p < c0; p += 4) {
                    const T x0 = row[p], x1 = row[p + 1], x2 = row[p + 2], x3 = row[p + 3];
#pragma unroll
                    for (int q = 0; q < CH; ++q) {
                        T l[4];
                        ld4(sLr + (c0 + q) * LDT + p, l);
                        x[q] = fma(-x0, l[0], x[q]);
                        x[q] = fma(-x1, l[1], x[q]);
                        x[q] = fma(-x2, l[2], x[q]);
                        x[q] = fma(-x3, l[3], x[q]);
                    }
                }
#pragma unroll
                for (int q = 0; q < CH; ++q) {
                    T v = x[q];
#pragma unroll
                    for (int p4 = 0; p4 < q; p4 += 4) {
                        T l[4];
                        ld4(sLr + (c0 + q) * LDT + c0 + p4, l);
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (p4 + u < q) v = fma(-x[p4 + u], l[u], v);
                    }
                    x[q] = v * rdiag[c0 + q];
                }
#pragma unroll
                for (int q = 0; q < CH; ++q) row[c0 + q] = x[q];
            }
        }
        __syncthreads();
        if (fok && it.fstep == k && it.fkind == ABFT_FAULT_PANEL && t == 0)
            A[(int64_t)it.frow * lda + it.fcol] += (T)it.fdelta;
        __syncthreads();
        if (check)
            for (int I = k + 1; I < nt; ++I) {
                const int r0 = I * B, nr = min(B, n - r0);
                verify_tile<T>(A + (int64_t)r0 * lda + K0, lda, r0, K0, nr, kb,
                               S.Cc + I * MAXN + K0, S.Cw + I * MAXN + K0, nullptr, 0, tau, 1, k,
                               st, colsum, wsum, rowsum, sJt, sflag, s_first, vexp);
            }
        // ---- TMU over the lower block triangle with the checksum borders.
        // sL is free from here to the next PD: it holds the carried checksum
        // rows of the panel (c_I, w_I of block row I; c_J of block row J) and
        // the border dot products' partial sums.  The panel rows of blocks I
        // and J sit transposed in sIt / sJt (element (j, p) at p LDT + j),
        // copied by cp.async.  A diagonal tile (J = I) takes its B operand
        // from sIt.
        T* sCI = &sL[0][0];
        T* sWI = sCI + MAXB;
        T* sCJ = sWI + MAXB;
        T* red = sCJ + MAXB;   // [3][BT / B][MAXB] partial sums of the border products
        for (int I = k + 1; I < nt; ++I) {
            const int r0 = I * B, nr = min(B, n - r0);
            // a block with rows below it is full: kb = B from here on
            stage_panel_t<T, B>(sIt, A, lda, r0, nr, K0);
            cp_async_commit();
            if (check)
                for (int p = t; p < kb; p += BT) {
                    sCI[p] = S.Cc[I * MAXN + K0 + p];
                    sWI[p] = S.Cw[I * MAXN + K0 + p];
                }
            for (int J = k + 1; J <= I; ++J) {
                const int c0 = J * B, nc = min(B, n - c0);
                const bool diag = J == I;
                if (!diag) stage_panel_t<T, B>(sJt, A, lda, c0, nc, K0);
                cp_async_commit();
                const T* sB = diag ? sIt : sJt;
                constexpr int R = B / 16;
                const int tx = t & 15, ty = t >> 4;
                // the tile's C values, loaded before the product so that their
                // latency is hidden behind it and the staging (FP32)
                T cv[R][R];
                if (Map::PREF_C) {
#pragma unroll
                    for (int a = 0; a < R; ++a)
#pragma unroll
                        for (int b = 0; b < R; ++b) {
                            const int i = Map::row(ty, a), j = Map::col(tx, b);
                            cv[a][b] = (i < nr && j < nc) ? A[(int64_t)(r0 + i) * lda + c0 + j] : (T)0;
                        }
                }
                if (check)
                    for (int p = t; p < kb; p += BT) sCJ[p] = S.Cc[J * MAXN + K0 + p];
                cp_async_wait<0>();
                __syncthreads();
                // register tile: thread (tx, ty) owns R x R outputs (Map); per p
                // it reads R values of each operand row of the transposed panels
                // and does R^2 fused multiply-adds in p order.  FP64 skips the
                // 16-row / 16-column groups beyond the tile's edge and, on a
                // diagonal tile, the groups above the diagonal, whose values the
                // mirrored groups below write (the same products: C is
                // symmetric there and a b = b a).
                T acc[R][R];
#pragma unroll
                for (int a = 0; a < R; ++a)
#pragma unroll
                    for (int b = 0; b < R; ++b) acc[a][b] = 0;
                const int ra = (nr + 15) / 16, rb = (nc + 15) / 16;
                if constexpr (Map::CONTIG) {
                    tile_product<Map, 0>(sIt, sB, tx, ty, ra, rb, diag, acc);
                } else {
                    const bool full = ra == R && rb == R;
                    if (full && !diag) tile_product<Map, 0>(sIt, sB, tx, ty, ra, rb, diag, acc);
                    else if (full) tile_product<Map, 1>(sIt, sB, tx, ty, ra, rb, diag, acc);
                    else tile_product<Map, 2>(sIt, sB, tx, ty, ra, rb, diag, acc);
                }
#pragma unroll
                for (int a = 0; a < R; ++a)
#pragma unroll
                    for (int b = 0; b < R; ++b) {
                        if (!Map::CONTIG && diag && b > a) continue;
                        const int i = Map::row(ty, a), j = Map::col(tx, b);
                        if (i >= nr || j >= nc) continue;
                        T* c = A + (int64_t)(r0 + i) * lda + c0 + j;
                        const T v = (Map::PREF_C ? cv[a][b] : *c) - acc[a][b];
                        T w = v;
                        if (fok && it.fstep == k && it.fkind == ABFT_FAULT_COMPUTE && it.frow == r0 + i &&
                            it.fcol == c0 + j)
                            w += (T)it.fdelta;
                        *c = w;
                        if (!Map::CONTIG && diag && b < a) {   // the mirrored element (j, i)
                            T wm = v;
                            if (fok && it.fstep == k && it.fkind == ABFT_FAULT_COMPUTE &&
                                it.frow == r0 + j && it.fcol == c0 + i)
                                wm += (T)it.fdelta;
                            A[(int64_t)(r0 + j) * lda + c0 + i] = wm;
                        }
                    }
                if (check) {
                    // border products on every thread: column j (or row j) and
                    // a quarter q of the panel's columns; the quarters are
                    // then added in order.  c_IJ -= s_I L_J^T, w_IJ likewise,
                    // r_IJ -= L_I s_J^T.
                    constexpr int NQ = BT / B;   // parts of the panel's columns
                    constexpr int np = B / NQ;
                    const int j = t % B, q = t / B;
                    const int p0 = q * np;
                    T a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
                    for (int p = p0; p < p0 + np; ++p) {
                        a1 = fma(sCI[p], sB[p * LDT + j], a1);
                        a2 = fma(sWI[p], sB[p * LDT + j], a2);
                        a3 = fma(sIt[p * LDT + j], sCJ[p], a3);
                    }
                    red[(0 * NQ + q) * MAXB + j] = a1;
                    red[(1 * NQ + q) * MAXB + j] = a2;
                    red[(2 * NQ + q) * MAXB + j] = a3;
                    __syncthreads();
                    if (t < nc) {
                        T s1 = 0, s2 = 0;
                        for (int qq = 0; qq < NQ; ++qq) {
                            s1 += red[(0 * NQ + qq) * MAXB + t];
                            s2 += red[(1 * NQ + qq) * MAXB + t];
                        }
                        S.Cc[I * MAXN + c0 + t] -= s1;
                        S.Cw[I * MAXN + c0 + t] -= s2;
                    }
                    if (t < nr) {
                        T s3 = 0;
                        for (int qq = 0; qq < NQ; ++qq) s3 += red[(2 * NQ + qq) * MAXB + t];
                        S.Cr[(r0 + t) * MAXNT + J] -= s3;
                    }
                }
                __syncthreads();
            }
        }
        if (fok && it.fstep == k && it.fkind == ABFT_FAULT_MEMORY && t == 0)
            A[(int64_t)it.frow * lda + it.fcol] += (T)it.fdelta;
        __syncthreads();
        if (check)
            for (int I = k + 1; I < nt; ++I)
                for (int J = k + 1; J <= I; ++J) {
                    const int r0 = I * B, c0 = J * B, nr = min(B, n - r0), nc = min(B, n - c0);
                    verify_tile<T>(A + (int64_t)r0 * lda + c0, lda, r0, c0, nr, nc,
                                   S.Cc + I * MAXN + c0, S.Cw + I * MAXN + c0,
                                   S.Cr + r0 * MAXNT + J, MAXNT, tau, 0, k, st, colsum, wsum,
                                   rowsum, sJt, sflag, s_first, vexp);
                }
    }
    __syncthreads();
    for (int K = 0; K < nt; ++K) {   // restore the diagonal blocks' upper triangles
        const int K0 = K * B, kb = min(B, n - K0);
        for (int e = t; e < kb * kb; e += BT) {
            int i = e / kb, j = e % kb;
            if (j > i) A[(int64_t)(K0 + i) * lda + K0 + j] = S.save[(K0 + i) * MAXB + j];
        }
    }
    __syncthreads();
}

// CTAs per SM: two for FP64 (the FP64 pipe is the limit), four for FP32 (as
// many as the shared memory holds; measured faster than three CTAs with a
// second J panel buffer, whose next tile's rows would be copied during the
// product)
template <typename T>
struct CtasPerSm { static constexpr int v = sizeof(T) == 8 ? 2 : 4; };

template <typename T>
__global__ void __launch_bounds__(BT, CtasPerSm<T>::v) k_potrf_batched(const abft_batch_item* items, int count,
                                                      int mode, double tau_scale,
                                                      abft_batch_status* status, T* scratch,
                                                      unsigned int* queue) {
    extern __shared__ __align__(16) unsigned char smb[];
    T (*sL)[MAXB + 1] = (T (*)[MAXB + 1])smb;
    T* sIt = (T*)(sL + MAXB);
    T* sJt = sIt + MAXB * LDT;
    T* colsum = sJt + MAXB * LDT;
    T* wsum = colsum + MAXB;
    T* rowsum = wsum + MAXB;
    T* rdiag = rowsum + MAXB;
    __shared__ int sflag[4], s_first, s_fail, s_item;
    const size_t per = (size_t)(3 * MAXNT * MAXN + MAXN * MAXB);
    Scratch<T> S;
    T* base = scratch + per * blockIdx.x;
    S.Cc = base;
    S.Cw = base + MAXNT * MAXN;
    S.Cr = base + 2 * MAXNT * MAXN;
    S.save = base + 3 * MAXNT * MAXN;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int idx = s_item;
        __syncthreads();
        if (idx >= count) break;
        const abft_batch_item it = items[idx];
        abft_batch_status* st = status + it.id;
        if (threadIdx.x == 0) {
            st->info = 0; st->detected = 0; st->corrected = 0; st->uncorrectable = 0;
            st->ev_step = -1; st->ev_kind = -1; st->ev_row = -1; st->ev_col = -1;
        }
        __syncthreads();
        if (it.n <= 0 || it.n > MAXN) continue;
        if (it.nb == 64)
            factor_one<T, 64>(it, mode, (T)tau_scale, S, st, sL, sIt, sJt, colsum, wsum, rowsum,
                              rdiag, sflag, &s_first, &s_fail);
        else
            factor_one<T, 32>(it, mode, (T)tau_scale, S, st, sL, sIt, sJt, colsum, wsum, rowsum,
                              rdiag, sflag, &s_first, &s_fail);
    }
}

}  // namespace

size_t batched_smem(bool f64) {
    return (size_t)(MAXB * (MAXB + 1) + 2 * MAXB * LDT + 4 * MAXB) *
           (f64 ? sizeof(double) : sizeof(float));
}

size_t batched_scratch_bytes(int grid, bool f64) {
    const size_t per = (size_t)(3 * MAXNT * MAXN + MAXN * MAXB);
    return per * (size_t)grid * (f64 ? sizeof(double) : sizeof(float));
}

// CTAs per SM of the persistent launch, set by abft_batched_set_ctas_per_sm
// (0: as many as fit, which the kernel's launch bounds fix).
std::atomic<int> g_batched_cps{0};

int batched_max_ctas_per_sm(bool f64) { return f64 ? CtasPerSm<double>::v : CtasPerSm<float>::v; }

int batched_set_ctas_per_sm(int c) { return g_batched_cps.exchange(c); }

int batched_grid(bool f64) {
    const int mx = batched_max_ctas_per_sm(f64);
    const int c = g_batched_cps.load();
    return (c <= 0 || c > mx ? mx : c) * num_sms();
}

int batched_max_grid(bool f64) { return batched_max_ctas_per_sm(f64) * num_sms(); }

// Kernel attributes (set once, outside any stream capture).
cudaError_t batched_prepare() {
    static bool attr = false;
    if (attr) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_potrf_batched<double>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)batched_smem(true));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_potrf_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)batched_smem(false));
    if (e == cudaSuccess) attr = true;
    return e;
}

cudaError_t launch_potrf_batched(const abft_batch_item* items, int count, bool f64, int mode,
                                 double tau_scale, abft_batch_status* status, void* scratch,
                                 unsigned int* queue, cudaStream_t s) {
    cudaError_t e = batched_prepare();
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(queue, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    const int grid = batched_grid(f64);
    if (f64)
        k_potrf_batched<double><<<grid, BT, batched_smem(true), s>>>(items, count, mode, tau_scale,
                                                                    status, (double*)scratch, queue);
    else
        k_potrf_batched<float><<<grid, BT, batched_smem(false), s>>>(items, count, mode, tau_scale,
                                                                    status, (float*)scratch, queue);
    note_launch();
    return cudaGetLastError();
}

}  // namespace abft
