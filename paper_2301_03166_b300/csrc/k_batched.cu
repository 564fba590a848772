// k_batched.cu -- batched ABFT Cholesky of many small SPD matrices in one
// persistent launch (Sec. 2.1 blocked algorithm and Sec. 3.1.2 checksums at
// the scope of one CTA per matrix).
//
// Each CTA repeatedly takes the next matrix from an atomic queue (the host
// orders the descriptors by decreasing n, so the longest factorizations
// start first) and factors it with block size B (32 or 64, per descriptor):
//   PD   the B x B diagonal block in shared memory (right-looking potf2) and
//        its column-sum check;
//   PU   one thread per panel row (and per checksum row) solves x L^T = a with
//        L_kk in shared memory; panel tiles are verified with the weighted
//        column checksums;
//   TMU  B x B output tiles of the lower block triangle (diagonal tiles in
//        full), L_I and L_J staged in shared memory, C read-modify-written in
//        global memory (L2-resident for these sizes), checksum borders
//        updated from the carried panel checksums;
//   then the optional injected fault and the verify / locate / correct of
//   every trailing tile (full checksums: 0D, 1D, checksum-only, 2D classes).
// T is the arithmetic type (double or float); the threshold uses its unit
// roundoff.  There are no spin waits: the only cross-CTA interaction is the
// atomic queue counter.
#include <math.h>

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
#pragma unroll 4
    for (int i = w; i < nr; i += BT / 32) {
        const T* row = P + (int64_t)i * ld;
        const T v0 = l < nc ? row[l] : (T)0;
        const T v1 = l + 32 < nc ? row[l + 32] : (T)0;
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

// tile_sums for FP64 tiles in exact 64-bit fixed point: every entry rounded to
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
    bool bad = false;
    long long* irow = reinterpret_cast<long long*>(rowsum);
#pragma unroll 4
    for (int i = w; i < nr; i += BT / 32) {
        const double* row = P + (int64_t)i * ld;
        const long long q0 = l < nc ? to_fixed(row[l], vexp, bad) : 0ll;
        const long long q1 = l + 32 < nc ? to_fixed(row[l + 32], vexp, bad) : 0ll;
        c0 += q0;
        c1 += q1;
        w0 += (long long)(i + 1) * (q0 >> 10);
        w1 += (long long)(i + 1) * (q1 >> 10);
        const long long rs = warp_sum_ll(q0 + q1);
        if (l == 0) irow[i] = rs;
    }
    if (__syncthreads_or(bad ? 1 : 0)) return false;
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
    tile_sums_any<T>(P, ld, nr, nc, vexp, colsum, wsum, rowsum, part);
    const int t = threadIdx.x;
    if (t == 0) { sflag[0] = 0; sflag[1] = 0; sflag[2] = 1 << 30; sflag[3] = 1 << 30; }
    __syncthreads();
    for (int j = t; j < nc; j += BT) {
        colsum[j] -= cc[j];
        wsum[j] -= cw[j];
        if (!(tabs(colsum[j]) <= tau)) { atomicAdd(&sflag[0], 1); atomicMin(&sflag[2], j); }
    }
    if (!single)
        for (int i = t; i < nr; i += BT) {
            rowsum[i] -= cr[i * crs];
            if (!(tabs(rowsum[i]) <= tau)) { atomicAdd(&sflag[1], 1); atomicMin(&sflag[3], i); }
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
                           abft_batch_status* st, T (*sL)[MAXB + 1], T (*sI)[MAXB + 1],
                           T (*sJ)[MAXB + 1], T* colsum, T* wsum, T* rowsum, T* rdiag, int* sflag,
                           int* s_first, int* s_fail) {
    T* A = (T*)it.A;
    const int64_t lda = it.lda;
    const int n = it.n;
    const int nt = (n + B - 1) / B;
    const int t = threadIdx.x;
    const bool check = mode != MODE_NONE;
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
        if (bnd > 0.0 && bnd < 1e300) vexp = (int)((__double_as_longlong(bnd) >> 52) & 0x7ff);
    }
    __syncthreads();
    // mirror the diagonal blocks (save their strict upper triangles)
    for (int K = 0; K < nt; ++K) {
        const int K0 = K * B, kb = min(B, n - K0);
        for (int e = t; e < kb * kb; e += BT) {
            int i = e / kb, j = e % kb;
            if (j > i) {
                S.save[(K0 + i) * MAXB + j] = A[(int64_t)(K0 + i) * lda + K0 + j];
                A[(int64_t)(K0 + i) * lda + K0 + j] = A[(int64_t)(K0 + j) * lda + K0 + i];
            }
        }
    }
    __syncthreads();
    if (check)
        for (int I = 0; I < nt; ++I)
            for (int J = 0; J <= I; ++J) {
                const int r0 = I * B, c0 = J * B, nr = min(B, n - r0), nc = min(B, n - c0);
                tile_sums_any<T>(A + (int64_t)r0 * lda + c0, lda, nr, nc, vexp, colsum, wsum,
                                 rowsum, &sJ[0][0]);
                for (int j = t; j < nc; j += BT) {
                    S.Cc[I * MAXN + c0 + j] = colsum[j];
                    S.Cw[I * MAXN + c0 + j] = wsum[j];
                }
                for (int i = t; i < nr; i += BT) S.Cr[(r0 + i) * MAXNT + J] = rowsum[i];
                __syncthreads();
            }
    for (int k = 0; k < nt; ++k) {
        const int K0 = k * B, kb = min(B, n - K0), T0 = K0 + kb, mrows = n - T0;
        // ---- PD: potf2 of the diagonal block in shared memory
        for (int e = t; e < kb * kb; e += BT) {
            int i = e / kb, j = e % kb;
            if (j <= i) sL[i][j] = A[(int64_t)(K0 + i) * lda + K0 + j];
        }
        __syncthreads();
        for (int j = 0; j < kb; ++j) {
            if (t == 0) {
                T d = sL[j][j];
                if (!(d > (T)0)) *s_fail = j;
                else sL[j][j] = sqrt(d);
            }
            __syncthreads();
            if (*s_fail >= 0) break;
            const T rjj = (T)1 / sL[j][j];   // one division per column, products below
            for (int i = j + 1 + t; i < kb; i += BT) sL[i][j] = sL[i][j] * rjj;
            __syncthreads();
            {   // rank-1 update of the remaining lower triangle on a 16 x 16 thread grid
                const int tx = t & 15, ty = t >> 4;
                for (int i = j + 1 + ty; i < kb; i += 16) {
                    const T aij = sL[i][j];
                    for (int l = j + 1 + tx; l <= i; l += 16) sL[i][l] -= aij * sL[l][j];
                }
            }
            __syncthreads();
        }
        if (*s_fail >= 0) {
            if (t == 0) st->info = K0 + *s_fail + 1;
            break;
        }
        for (int e = t; e < kb * kb; e += BT) {
            int i = e / kb, j = e % kb;
            if (j <= i) A[(int64_t)(K0 + i) * lda + K0 + j] = sL[i][j];
        }
        for (int j = t; j < kb; j += BT) rdiag[j] = (T)1 / sL[j][j];   // the panel solve's reciprocals
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
        __syncthreads();
        if (mrows <= 0) break;
        // ---- PU: x L^T = a for the panel rows and the checksum rows, one thread
        // per row.  A block with rows below it is never ragged (kb = B, a
        // multiple of 32), so the row's unknowns are solved 32 at a time in
        // registers: each chunk first takes the terms of the earlier chunks
        // (re-read from the row, which this thread wrote), then substitutes
        // inside the chunk; every unknown's terms form one fused multiply-add
        // chain in p order.
        const int ncs = check ? 2 * (nt - k - 1) : 0;
        for (int rr = t; rr < mrows + ncs; rr += BT) {
            T* row;
            if (rr < mrows) row = A + (int64_t)(T0 + rr) * lda + K0;
            else {
                int c = rr - mrows, I = k + 1 + c / 2;
                row = ((c & 1) ? S.Cw : S.Cc) + I * MAXN + K0;
            }
            for (int c0 = 0; c0 < B; c0 += 32) {
                T x[32];
#pragma unroll
                for (int q = 0; q < 32; ++q) x[q] = row[c0 + q];
                for (int p = 0; p < c0; ++p) {
                    const T xp = row[p];
#pragma unroll
                    for (int q = 0; q < 32; ++q) x[q] = fma(-xp, sL[c0 + q][p], x[q]);
                }
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    T v = x[q];
#pragma unroll
                    for (int pp = 0; pp < q; ++pp) v = fma(-x[pp], sL[c0 + q][c0 + pp], v);
                    x[q] = v * rdiag[c0 + q];
                }
#pragma unroll
                for (int q = 0; q < 32; ++q) row[c0 + q] = x[q];
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
                               st, colsum, wsum, rowsum, &sJ[0][0], sflag, s_first, vexp);
            }
        // ---- TMU over the lower block triangle with the checksum borders.
        // sL is free from here to the next PD: it holds the carried checksum
        // rows of the panel (c_I, w_I of block row I; c_J of block row J) and
        // the border dot products' partial sums.
        T* sCI = &sL[0][0];
        T* sWI = sCI + MAXB;
        T* sCJ = sWI + MAXB;
        T* red = sCJ + MAXB;   // [3][BT / B][MAXB] partial sums of the border products
        for (int I = k + 1; I < nt; ++I) {
            const int r0 = I * B, nr = min(B, n - r0);
            // a block with rows below it is full: kb = B from here on
#pragma unroll
            for (int e = t; e < B * B; e += BT) {
                const int i = e / B, p = e % B;
                sI[i][p] = (i < nr) ? A[(int64_t)(r0 + i) * lda + K0 + p] : (T)0;
            }
            if (check)
                for (int p = t; p < kb; p += BT) {
                    sCI[p] = S.Cc[I * MAXN + K0 + p];
                    sWI[p] = S.Cw[I * MAXN + K0 + p];
                }
            for (int J = k + 1; J <= I; ++J) {
                const int c0 = J * B, nc = min(B, n - c0);
#pragma unroll
                for (int e = t; e < B * B; e += BT) {
                    const int j = e / B, p = e % B;
                    sJ[j][p] = (j < nc) ? A[(int64_t)(c0 + j) * lda + K0 + p] : (T)0;
                }
                if (check)
                    for (int p = t; p < kb; p += BT) sCJ[p] = S.Cc[J * MAXN + K0 + p];
                __syncthreads();
                // register tile: thread (tx, ty) owns rows ty + 16 a and columns
                // tx + 16 b (a, b < B / 16); per p, B / 8 shared loads feed
                // (B / 16)^2 fused multiply-adds
                constexpr int R = B / 16;
                const int tx = t & 15, ty = t >> 4;
                T acc[R][R];
#pragma unroll
                for (int a = 0; a < R; ++a)
#pragma unroll
                    for (int b = 0; b < R; ++b) acc[a][b] = 0;
                // row / column groups of 16 beyond the tile's edge are skipped
                // (the same branch for every thread)
                const int ra = (nr + 15) / 16, rb = (nc + 15) / 16;
#pragma unroll 8
                for (int p = 0; p < B; ++p) {
                    T av[R], bv[R];
#pragma unroll
                    for (int a = 0; a < R; ++a) av[a] = sI[ty + 16 * a][p];
#pragma unroll
                    for (int b = 0; b < R; ++b) bv[b] = sJ[tx + 16 * b][p];
#pragma unroll
                    for (int a = 0; a < R; ++a)
                        if (a < ra)
#pragma unroll
                            for (int b = 0; b < R; ++b)
                                if (b < rb) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
                }
#pragma unroll
                for (int a = 0; a < R; ++a)
#pragma unroll
                    for (int b = 0; b < R; ++b) {
                        const int i = ty + 16 * a, j = tx + 16 * b;
                        if (i >= nr || j >= nc) continue;
                        T* c = A + (int64_t)(r0 + i) * lda + c0 + j;
                        T v = *c - acc[a][b];
                        if (fok && it.fstep == k && it.fkind == ABFT_FAULT_COMPUTE && it.frow == r0 + i &&
                            it.fcol == c0 + j)
                            v += (T)it.fdelta;
                        *c = v;
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
                        a1 = fma(sCI[p], sJ[j][p], a1);
                        a2 = fma(sWI[p], sJ[j][p], a2);
                        a3 = fma(sI[j][p], sCJ[p], a3);
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
                                   rowsum, &sJ[0][0], sflag, s_first, vexp);
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

// CTAs per SM: two for FP64 (the FP64 pipe is the limit), four for FP32
// (shorter arithmetic: more CTAs hide the barriers and load latencies)
template <typename T>
struct CtasPerSm { static constexpr int v = sizeof(T) == 8 ? 2 : 4; };

template <typename T>
__global__ void __launch_bounds__(BT, CtasPerSm<T>::v) k_potrf_batched(const abft_batch_item* items, int count,
                                                      int mode, double tau_scale,
                                                      abft_batch_status* status, T* scratch,
                                                      unsigned int* queue) {
    extern __shared__ __align__(16) unsigned char smb[];
    T (*sL)[MAXB + 1] = (T (*)[MAXB + 1])smb;
    T (*sI)[MAXB + 1] = sL + MAXB;
    T (*sJ)[MAXB + 1] = sI + MAXB;
    T* colsum = (T*)(sJ + MAXB);
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
            factor_one<T, 64>(it, mode, (T)tau_scale, S, st, sL, sI, sJ, colsum, wsum, rowsum,
                              rdiag, sflag, &s_first, &s_fail);
        else
            factor_one<T, 32>(it, mode, (T)tau_scale, S, st, sL, sI, sJ, colsum, wsum, rowsum,
                              rdiag, sflag, &s_first, &s_fail);
    }
}

}  // namespace

size_t batched_smem(bool f64) {
    return (size_t)(3 * MAXB * (MAXB + 1) + 4 * MAXB) * (f64 ? sizeof(double) : sizeof(float));
}

size_t batched_scratch_bytes(int grid, bool f64) {
    const size_t per = (size_t)(3 * MAXNT * MAXN + MAXN * MAXB);
    return per * (size_t)grid * (f64 ? sizeof(double) : sizeof(float));
}

int batched_grid(bool f64) {
    return (f64 ? CtasPerSm<double>::v : CtasPerSm<float>::v) * num_sms();
}

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
