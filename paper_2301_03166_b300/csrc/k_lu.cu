// k_lu.cu -- kernels of the blocked ABFT LU with partial pivoting
// (Sec. 2.1: PD  L.1 x U11 <- A.1,  PU  U12 <- L11^{-1} A12,  TMU  A22 <- A22 - L21 U12;
// Sec. 3.1.2: checksums carried through each operation).
//
// The panel factorization (getf2 on the (n - K0) x kb panel) is one
// cooperative launch: each CTA owns a contiguous block of panel rows.  Per
// column the CTAs publish their local (max |a|, first index) together with a
// copy of that candidate row (and the owner of row j a copy of row j), meet
// at one bounded grid barrier, and then every CTA picks the same pivot from
// the published values, the owners of rows j and p write the interchange
// from the copies, and every CTA scales and updates its own rows with the
// pivot row's copy.  The copies alternate between two slots by column parity:
// slot j % 2 is rewritten only at column j + 2, after the barrier of column
// j + 1, which every CTA reaches only once it has finished reading it.  (The
// earlier scheme met twice per column, the pivot chosen and the rows swapped
// by one CTA between the barriers.)  The panel (<= 32 MB at n = 16384)
// stays in L2 across the column loop.
//
// When every CTA's rows fit its shared memory (n <= 16384 at kb = 256 on
// 148 SMs), k_getf2_smem runs the same column loop with those rows held in
// shared memory from the first column to the last: the scan, the interchange,
// the scaling and the rank-1 update then make no global round trip, and only
// the published candidates and the pivot-row copies go through memory.  It
// also takes most of each rank-1 update off the chain of barriers (see the
// kernel).  Its arithmetic is that of k_getf2_coop operation for operation
// (the same division, the same fused multiply-adds), so both give identical
// panels.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "fp_bits.cuh"

namespace abft {

namespace {

constexpr int PT = 256;          // threads of the panel kernels
constexpr int MAXR = 1024;       // max rows per CTA in the cooperative panel

__device__ __forceinline__ void better(double& bv, int64_t& bi, double v, int64_t i) {
    // larger |a| wins; equal values keep the smaller index (first max)
    if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
}

__device__ void block_argmax(double& v, int64_t& idx) {
    __shared__ double sv[PT / 32];
    __shared__ int64_t si[PT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, v, o);
        int64_t oi = __shfl_xor_sync(0xffffffffu, idx, o);
        better(v, idx, ov, oi);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sv[w] = v; si[w] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) better(v, idx, sv[k], si[k]);
        sv[0] = v; si[0] = idx;
    }
    __syncthreads();
    v = sv[0]; idx = si[0];
    __syncthreads();
}

__global__ void __launch_bounds__(PT) k_getf2_coop(double* P, int64_t lda, int64_t m, int kb,
                                                   int64_t K0, int64_t* ipiv, DevStatus* st,
                                                   double* part_v, int64_t* part_i,
                                                   double* stage) {
    __shared__ double urow[512];
    __shared__ double lcol[MAXR];
    const unsigned G = gridDim.x;
    const int64_t R = (m + G - 1) / G;
    const int64_t r0 = blockIdx.x * R, r1 = (r0 + R < m) ? r0 + R : m;
    unsigned long long nbar = 0;   // grid barriers passed
    // stage: [2][G + 1][kb]: candidate row per CTA, then row j (slot G)
    for (int j = 0; j < kb; ++j) {
        const int par = j & 1;
        double* slot = stage + (size_t)par * (G + 1) * kb;
        // A: local first-max of |P[i][j]| over my rows i >= j, published with a
        // copy of the candidate row; the owner of row j publishes row j
        double bv = -1.0;
        int64_t bi = INT64_MAX;
        for (int64_t i = (r0 > j ? r0 : j) + threadIdx.x; i < r1; i += PT)
            better(bv, bi, fabs(P[i * lda + j]), i);
        block_argmax(bv, bi);
        if (threadIdx.x == 0) {
            part_v[par * G + blockIdx.x] = bv;
            part_i[par * G + blockIdx.x] = bi;
        }
        if (bi != INT64_MAX)
            for (int c = threadIdx.x; c < kb; c += PT)
                slot[(size_t)blockIdx.x * kb + c] = P[bi * lda + c];
        if (j >= r0 && j < r1)
            for (int c = threadIdx.x; c < kb; c += PT) slot[(size_t)G * kb + c] = P[(int64_t)j * lda + c];
        if (!grid_barrier(st, G, nbar)) return;
        // B: every CTA picks the pivot from the published values (same order,
        // same result); the pivot row comes from its owner's copy
        double v = -1.0;
        int64_t idx = INT64_MAX;
        unsigned win = 0;
        for (unsigned b = threadIdx.x; b < G; b += PT) {
            const double pv = part_v[par * G + b];
            const int64_t pi = part_i[par * G + b];
            if (pv > v || (pv == v && pi < idx)) { v = pv; idx = pi; }
        }
        block_argmax(v, idx);
        const int64_t p = (idx == INT64_MAX) ? j : idx;
        if (idx != INT64_MAX) win = (unsigned)(idx / R);   // the CTA that owns row p
        if (blockIdx.x == 0 && threadIdx.x == 0) ipiv[K0 + j] = K0 + p;
        for (int c = threadIdx.x; c < kb; c += PT)
            urow[c] = p == j ? slot[(size_t)G * kb + c] : slot[(size_t)win * kb + c];
        __syncthreads();
        const double piv = urow[j];
        if (piv == 0.0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&st->lu_info, 0, (int)(K0 + j + 1));
            continue;
        }
        if (p != j) {   // the interchange, written by the owners of the two rows
            if (j >= r0 && j < r1)
                for (int c = threadIdx.x; c < kb; c += PT) P[(int64_t)j * lda + c] = urow[c];
            if (p >= r0 && p < r1)
                for (int c = threadIdx.x; c < kb; c += PT) P[p * lda + c] = slot[(size_t)G * kb + c];
            __syncthreads();
        }
        // C: scale and rank-1 update of my rows below the pivot
        const int64_t ibeg = (r0 > j + 1 ? r0 : j + 1);
        for (int64_t i = ibeg + threadIdx.x; i < r1; i += PT) {
            double l = P[i * lda + j] / piv;
            P[i * lda + j] = l;
            lcol[i - r0] = l;
        }
        __syncthreads();
        // thread t: column j + 1 + t % w, row chunk t / w (with fewer columns
        // than threads the rows are split so that every thread works and the
        // dependent load rounds per thread shrink), eight rows at a time:
        // loads coalesced along the rows, eight in flight per thread
        const int w = kb - j - 1;
        const int64_t nrow = r1 - ibeg;
        int rsp = w > 0 ? PT / w : 1;
        if (rsp < 1) rsp = 1;
        if ((int64_t)rsp > (nrow + 7) / 8) rsp = (int)((nrow + 7) / 8);
        if (rsp < 1) rsp = 1;
        const int64_t rch = (nrow + rsp - 1) / rsp;
        for (int t = threadIdx.x; t < w * rsp; t += PT) {
            const int c = j + 1 + t % w;
            const int64_t ia = ibeg + (int64_t)(t / w) * rch;
            const int64_t ie = ia + rch < r1 ? ia + rch : r1;
            const double uc = urow[c];
            for (int64_t i = ia; i < ie; i += 8) {
                double av[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (i + u < ie) av[u] = P[(i + u) * lda + c];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (i + u < ie)
                        P[(i + u) * lda + c] = fma(-lcol[i + u - r0], uc, av[u]);
            }
        }
        __syncthreads();
    }
}

// Split form of grid_barrier: arrive, do work that the barrier need not wait
// for, then wait for barrier number `passed` (same counter, same bound).
__device__ __forceinline__ void grid_arrive(DevStatus* st) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&st->bar_count, 1ull);
    }
}

__device__ __forceinline__ bool grid_wait(DevStatus* st, unsigned G, unsigned long long passed,
                                          int* s_ok) {
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long target = passed * G;
        volatile unsigned long long* vc = &st->bar_count;
        if (*vc < target) {
            const unsigned long long t0 = global_ns();
            while (*vc < target) {
                if (global_ns() - t0 > kBarrierNs) {
                    atomicExch(&st->error, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

__device__ __forceinline__ void warp_argmax(double& v, int64_t& idx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int64_t oi = __shfl_xor_sync(0xffffffffu, idx, o);
        better(v, idx, ov, oi);
    }
}

// k_getf2_coop with the CTA's rows r0 .. r1 - 1 of the panel in shared memory,
// element (i, c) at sp[(i - r0) kb + (c ^ ((i - r0) & 31))] (kb a multiple of
// 32: a column read by the rows of a warp and a row read by its lanes both hit
// 32 banks), then urow[kb] (the pivot row) and uprev[kb] (the previous one).
// Rows are read once before the column loop and written once after it.
//
// The rank-1 update of step j is split: column j + 1 first, then the
// candidates of column j + 1 are published and the CTA arrives at the
// barrier, and only then are columns j + 2 .. updated, while the other CTAs
// arrive.  The published rows are therefore copies in which step j has reached
// columns <= j + 1 only; after the barrier every CTA completes the pivot row
// (and row j + 1, for the interchange) with the same fused multiply-add,
// a_c - l a_jc with the row's own multiplier l from column j, that the owner
// applies to its row, so the rows agree bit for bit with k_getf2_coop's.
__global__ void __launch_bounds__(PT) k_getf2_smem(double* P, int64_t lda, int64_t m, int kb,
                                                   int64_t K0, int64_t* ipiv, DevStatus* st,
                                                   double* part_v, int64_t* part_i,
                                                   double* stage) {
    extern __shared__ double gsm[];
    __shared__ int64_t s_i;
    __shared__ int s_ok;
    const unsigned G = gridDim.x;
    const int64_t R = (m + G - 1) / G;
    const int64_t r0 = blockIdx.x * R < m ? blockIdx.x * R : m;
    const int64_t r1 = (r0 + R < m) ? r0 + R : m;
    const int nr = (int)(r1 - r0);
    double* sp = gsm;
    double* urow = gsm + (size_t)R * kb;
    double* uprev = urow + kb;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#define SX(r, c) sp[(r) * kb + ((c) ^ ((r) & 31))]
    for (int r = warp; r < nr; r += PT / 32)
        for (int c = lane; c < kb; c += 32) SX(r, c) = P[(r0 + r) * lda + c];
    __syncthreads();
    // publish the candidates of column j: my first max of |a_ij| over my rows
    // i >= j with a copy of that row, and (owner) a copy of row j
    auto publish = [&](int j) {
        const int par = j & 1;
        double* slot = stage + (size_t)par * (G + 1) * kb;
        if (warp == 0) {
            double bv = -1.0;
            int64_t bi = INT64_MAX;
            const int rj = j - r0 > 0 ? (int)(j - r0) : 0;
            for (int r = rj + lane; r < nr; r += 32) better(bv, bi, fabs(SX(r, j)), r0 + r);
            warp_argmax(bv, bi);
            if (lane == 0) {
                s_i = bi;
                part_v[par * G + blockIdx.x] = bv;
                part_i[par * G + blockIdx.x] = bi;
            }
        }
        __syncthreads();
        const int64_t bi = s_i;
        if (bi != INT64_MAX) {
            const int r = (int)(bi - r0);
            for (int c = threadIdx.x; c < kb; c += PT) slot[(size_t)blockIdx.x * kb + c] = SX(r, c);
        }
        if (j >= r0 && j < r1) {
            const int r = (int)(j - r0);
            for (int c = threadIdx.x; c < kb; c += PT) slot[(size_t)G * kb + c] = SX(r, c);
        }
    };
    unsigned long long nbar = 0;   // grid barriers arrived at
    publish(0);
    ++nbar;
    grid_arrive(st);
    bool upd_prev = false;   // the copies of this column still lack step j - 1 beyond column j
    for (int j = 0; j < kb; ++j) {
        const int par = j & 1;
        const double* slot = stage + (size_t)par * (G + 1) * kb;
        if (!grid_wait(st, G, nbar, &s_ok)) return;
        // every CTA picks the pivot from the published values (same result)
        if (warp == 0) {
            double v = -1.0;
            int64_t idx = INT64_MAX;
            for (unsigned b = lane; b < G; b += 32) better(v, idx, part_v[par * G + b], part_i[par * G + b]);
            warp_argmax(v, idx);
            if (lane == 0) s_i = idx;
        }
        __syncthreads();
        const int64_t idx = s_i;
        const int64_t p = (idx == INT64_MAX) ? j : idx;
        const unsigned win = idx == INT64_MAX ? 0u : (unsigned)(idx / R);
        if (blockIdx.x == 0 && threadIdx.x == 0) ipiv[K0 + j] = K0 + p;
        const double* prow = p == j ? slot + (size_t)G * kb : slot + (size_t)win * kb;
        const double* jrow = slot + (size_t)G * kb;
        const double lp = upd_prev ? prow[j - 1] : 0.0;
        for (int c = threadIdx.x; c < kb; c += PT) {
            double x = prow[c];
            if (upd_prev && c > j) x = fma(-lp, uprev[c], x);
            urow[c] = x;
        }
        __syncthreads();
        const double piv = urow[j];
        const bool last = j + 1 >= kb;
        if (piv == 0.0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&st->lu_info, 0, (int)(K0 + j + 1));
            upd_prev = false;
            if (!last) {
                publish(j + 1);
                ++nbar;
                grid_arrive(st);
            }
            continue;
        }
        if (p != j) {   // the interchange, in the owners' rows (mine are complete)
            if (j >= r0 && j < r1) {
                const int r = (int)(j - r0);
                for (int c = threadIdx.x; c < kb; c += PT) SX(r, c) = urow[c];
            }
            if (p >= r0 && p < r1) {
                const int r = (int)(p - r0);
                const double lj = upd_prev ? jrow[j - 1] : 0.0;
                for (int c = threadIdx.x; c < kb; c += PT) {
                    double x = jrow[c];
                    if (upd_prev && c > j) x = fma(-lj, uprev[c], x);
                    SX(r, c) = x;
                }
            }
            __syncthreads();
        }
        // scale column j of my rows below the pivot, update column j + 1
        const int rb = j + 1 - r0 > 0 ? (int)(j + 1 - r0) : 0;
        for (int r = rb + threadIdx.x; r < nr; r += PT) {
            const double l = SX(r, j) / piv;
            SX(r, j) = l;
            if (!last) SX(r, j + 1) = fma(-l, urow[j + 1], SX(r, j + 1));
        }
        __syncthreads();
        if (last) break;
        publish(j + 1);
        ++nbar;
        grid_arrive(st);
        // the rest of step j while the other CTAs arrive
        for (int r = rb + warp; r < nr; r += PT / 32) {
            const double l = SX(r, j);
            for (int c = j + 2 + lane; c < kb; c += 32) SX(r, c) = fma(-l, urow[c], SX(r, c));
        }
        for (int c = threadIdx.x; c < kb; c += PT) uprev[c] = urow[c];
        upd_prev = true;
    }
    __syncthreads();
    for (int r = warp; r < nr; r += PT / 32)
        for (int c = lane; c < kb; c += 32) P[(r0 + r) * lda + c] = SX(r, c);
#undef SX
}

// Row interchanges of the panel applied to every column outside the panel
// (one thread per column, interchanges in order), and to the row-checksum
// columns.  For trailing columns the two tile-rows' column (and weighted)
// sums receive the row difference at the time of each interchange.
__global__ void k_laswp(double* A, int64_t lda, int64_t n, int64_t K0, int kb,
                        const int64_t* ipiv, double* CS, int64_t ldcs, int64_t nc, int64_t g,
                        double* Cr, int64_t nt, int mode) {
    const int64_t T0 = K0 + kb;
    const int64_t ndata = n - kb;
    const int64_t ncr = (mode == MODE_FULL) ? nt : 0;
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= ndata + ncr) return;
    if (v < ndata) {
        const int64_t c = v < K0 ? v : v + kb;
        const bool trail = c >= T0 && mode != MODE_NONE;
        for (int j = 0; j < kb; ++j) {
            const int64_t i = K0 + j, p = ipiv[K0 + j];
            if (p == i) continue;
            double a = A[i * lda + c], b = A[p * lda + c];
            A[i * lda + c] = b;
            A[p * lda + c] = a;
            if (trail) {
                const int64_t Ii = i / g, Ip = p / g;
                CS[(Ii * nc) * ldcs + c] += b - a;
                CS[(Ip * nc) * ldcs + c] += a - b;
                if (mode == MODE_SINGLE) {
                    const double wi = (double)(i - Ii * g + 1), wp = (double)(p - Ip * g + 1);
                    CS[(Ii * nc + 1) * ldcs + c] += wi * (b - a);
                    CS[(Ip * nc + 1) * ldcs + c] += wp * (a - b);
                }
            }
        }
    } else {
        const int64_t J = v - ndata;
        for (int j = 0; j < kb; ++j) {
            const int64_t i = K0 + j, p = ipiv[K0 + j];
            if (p == i) continue;
            double a = Cr[i * nt + J];
            Cr[i * nt + J] = Cr[p * nt + J];
            Cr[p * nt + J] = a;
        }
    }
}

// ptot[j] = sum over tile-rows I >= k of the carried column sums of panel column j.
__global__ void k_coltot(const double* CS, int64_t ldcs, int64_t nc, int64_t k, int64_t nt,
                         int64_t K0, int kb, double* ptot) {
    for (int j = threadIdx.x; j < kb; j += blockDim.x) {
        double s = 0.0;
        for (int64_t I = k; I < nt; ++I) s += CS[(I * nc) * ldcs + K0 + j];
        ptot[j] = s;
    }
}

// Column sums of L per tile-row of the panel (strictly below the unit
// diagonal in tile-row k): the border rows 1^T L_Ik (and weighted) of the
// TMU for I > k, and the per-tile parts of the PD check.
__global__ void k_lu_colsums(const double* P, int64_t lda, int64_t m, int kb, int64_t g,
                             int64_t k, int64_t K0, double* CS, int64_t ldcs, int64_t nc,
                             int mode, double* part, int64_t ldpart) {
    const int64_t I = k + blockIdx.x;
    const int64_t gr0 = I * g, gr1 = (gr0 + g < K0 + m) ? gr0 + g : K0 + m;
    for (int q = threadIdx.x; q < kb; q += blockDim.x) {
        double s = 0.0, sw = 0.0;
        for (int64_t gi = gr0; gi < gr1; ++gi) {
            const int64_t i = gi - K0;
            if (i <= q) continue;
            double l = P[i * lda + q];
            s += l;
            sw += (double)(gi - gr0 + 1) * l;
        }
        part[blockIdx.x * ldpart + q] = s;
        if (I > k && mode != MODE_NONE) {
            CS[(I * nc) * ldcs + K0 + q] = s;
            if (mode == MODE_SINGLE) CS[(I * nc + 1) * ldcs + K0 + q] = sw;
        }
    }
}

// Single CTA: running max |U| and the step's threshold, the PD check
// (total panel column sums vs (1^T L) U_kk), and z = L_kk^{-T} 1,
// zw = L_kk^{-T} (1..kb) for the column sums of U.
// The largest |u_ij| of the U11 block (j >= i), merged into st->umax (an
// atomic maximum on the bits of a non-negative double): the first half of the
// PD check, over many CTAs.
__global__ void __launch_bounds__(256) k_lu_umax(const double* P, int64_t lda, int kb,
                                                DevStatus* st) {
    double m = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)kb * kb;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / kb), j = (int)(e % kb);
        if (j >= i) m = fmax(m, fabs(P[(int64_t)i * lda + j]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg((unsigned long long*)&st->umax, m);
}

// The rest of the PD check, after k_lu_umax: the threshold from max(amax, umax)
// (every CTA forms the same value; CTA 0 stores it and the fixed-point bound),
// the check of the carried column sums 1^T [L11; L21] U11 against ptot with
// one warp per column (CTAs 0 .. nchk - 1, columns nw b + w, ...), and, on the
// last CTA, z = L^{-T} 1 and zw = L^{-T} w (unit upper L^T) for the carried
// row checksums.  Each part keeps the operations and order of the one-CTA form.
__global__ void __launch_bounds__(512) k_lu_pd_check(const double* P, int64_t lda, int kb,
                                                     const double* ptot, const double* part,
                                                     int64_t ldpart, int nparts, int step,
                                                     int64_t K0, int64_t n, int64_t g,
                                                     double tau_scale, double* z, double* zw,
                                                     int mode, DevStatus* st, int nchk) {
    __shared__ double lsum[512];
    __shared__ double tz[512], tw[512];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
    const double um = st->umax;
    const double M = st->amax > um ? st->amax : um;
    double tau = tau_scale * 8.0;
    tau *= 0x1p-53;
    tau *= (double)n;
    tau *= (double)g;
    tau *= M;
    if (blockIdx.x == 0 && t == 0) {
        st->tau = tau;
        // fixed-point bound of the verify sums: 16 max(|a|, |u| so far); a tile
        // holding an entry above it (growth beyond that, an injected error) is
        // summed in FP64
        const double bnd = 16.0 * M;
        const int ve = (int)((__double_as_longlong(bnd) >> 52) & 0x7ff);
        st->vexp = (bnd > 0.0 && bnd < 1e300 && ve >= kFixedMinExp) ? ve : 0;
    }
    if (mode == MODE_NONE) return;
    if ((int)blockIdx.x < nchk) {
        for (int q = t; q < kb; q += blockDim.x) {
            double s = 1.0;
            for (int b = 0; b < nparts; ++b) s += part[b * ldpart + q];
            lsum[q] = s;
        }
        __syncthreads();
        for (int j = (int)blockIdx.x * nw + warp; j < kb; j += nchk * nw) {
            double y = 0.0;
            for (int q = lane; q <= j; q += 32) y = fma(lsum[q], P[(int64_t)q * lda + j], y);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
            if (lane == 0) {
                double d = y - ptot[j];
                if (!(fabs(d) <= tau)) {
                    atomicAdd(&st->detected, 1ull);
                    atomicAdd(&st->uncorrectable, 1ull);
                    record_event(st, step, EV_PD, K0 + j, K0 + j, d);
                }
            }
        }
        return;
    }
    // z = L^{-T} 1, zw = L^{-T} w (unit upper L^T), chunks of 32 from the end
    for (int p = t; p < kb; p += blockDim.x) { tz[p] = 1.0; tw[p] = (double)(p + 1); }
    __syncthreads();
    for (int c1 = kb; c1 > 0; c1 -= 32) {
        const int c0 = c1 - 32 > 0 ? c1 - 32 : 0;
        // (the chunk's entries of L are loaded into registers first, so that
        // the substitution and the update wait for memory once per chunk, not
        // once per term; the terms and their order are unchanged)
        if (warp == 0) {
            const int p = c0 + lane;
            double lv[32];
#pragma unroll
            for (int u = 0; u < 32; ++u) {
                const int j = c0 + u;
                lv[u] = (j < c1 && p < j) ? P[(int64_t)j * lda + p] : 0.0;
            }
            double a = (p < c1) ? tz[p] : 0.0, b = (p < c1) ? tw[p] : 0.0;
#pragma unroll
            for (int u = 31; u >= 0; --u) {
                const int j = c0 + u;
                if (j >= c1) continue;
                double zj = __shfl_sync(0xffffffffu, a, u);
                double wj = __shfl_sync(0xffffffffu, b, u);
                if (p < j) {
                    a -= lv[u] * zj;
                    b -= lv[u] * wj;
                }
            }
            if (p < c1) { tz[p] = a; tw[p] = b; }
        }
        __syncthreads();
        for (int p = t; p < c0; p += blockDim.x) {
            double lv[32];
#pragma unroll
            for (int u = 0; u < 32; ++u)
                lv[u] = (c0 + u < c1) ? P[(int64_t)(c0 + u) * lda + p] : 0.0;
            double a = tz[p], b = tw[p];
#pragma unroll
            for (int u = 0; u < 32; ++u) {
                if (c0 + u >= c1) continue;
                a -= lv[u] * tz[c0 + u];
                b -= lv[u] * tw[c0 + u];
            }
            tz[p] = a; tw[p] = b;
        }
        __syncthreads();
    }
    for (int p = t; p < kb; p += blockDim.x) { z[p] = tz[p]; zw[p] = tw[p]; }
}

constexpr int CB = 32;    // columns per CTA of the U solve
struct TrsmLSeg {
    double* B;
    int64_t ldb;
    int64_t ncols;
};
struct TrsmLArgs {
    const double* L;
    int64_t ldl;
    int kb;
    TrsmLSeg seg[2];
    int64_t start[3];
    int nseg;
    const double* z;
    const double* zw;
    double* colchk;
    double* colchkw;
    int colchk_only;   // form colchk / colchkw from B and leave B as it is
};

// U = L^{-1} B (L unit lower kb x kb) for CB columns per CTA, in place; the
// row-checksum columns are a second segment of the same launch.  Before the
// solve, segment 0 also produces the U column sums z^T B (and zw^T B).
__global__ void __launch_bounds__(256) k_trsm_llu(TrsmLArgs a) {
    extern __shared__ double smem[];
    const int kb = a.kb;
    double* X = smem;                    // kb x (CB + 1)
    double* Ls = smem + kb * (CB + 1);   // 32 x 33
    const int64_t bid = blockIdx.x;
    const int s = (a.nseg > 1 && bid >= a.start[1]) ? 1 : 0;
    const TrsmLSeg& g = a.seg[s];
    const int64_t c0 = (bid - a.start[s]) * CB;
    const int nc = (int)((g.ncols - c0) < CB ? (g.ncols - c0) : CB);
    const int t = threadIdx.x;
    for (int e = t; e < kb * CB; e += 256) {
        int r = e / CB, c = e % CB;
        X[r * (CB + 1) + c] = (c < nc) ? g.B[(int64_t)r * g.ldb + c0 + c] : 0.0;
    }
    __syncthreads();
    if (s == 0 && a.z != nullptr) {
        const int warp = t >> 5, lane = t & 31;
        for (int c = warp; c < nc; c += 8) {
            double u = 0.0, w = 0.0;
            for (int r = lane; r < kb; r += 32) {
                double x = X[r * (CB + 1) + c];
                u = fma(a.z[r], x, u);
                w = fma(a.zw[r], x, w);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                u += __shfl_xor_sync(0xffffffffu, u, o);
                w += __shfl_xor_sync(0xffffffffu, w, o);
            }
            if (lane == 0) {
                a.colchk[c0 + c] = u;
                if (a.colchkw) a.colchkw[c0 + c] = w;
            }
        }
        __syncthreads();
    }
    if (a.colchk_only) return;
    const int gr = t >> 3, gq = (t & 7) * 4;   // row gr of the chunk, columns gq..gq+3
    for (int r0 = 0; r0 < kb; r0 += 32) {
        const int w = (kb - r0) < 32 ? (kb - r0) : 32;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int p0 = 0; p0 < r0; p0 += 32) {
            __syncthreads();
            for (int e = t; e < 32 * 32; e += 256) {
                int q = e / 32, pp = e % 32;
                Ls[q * 33 + pp] = (q < w) ? a.L[(int64_t)(r0 + q) * a.ldl + p0 + pp] : 0.0;
            }
            __syncthreads();
#pragma unroll 8
            for (int pp = 0; pp < 32; ++pp) {
                double l = Ls[gr * 33 + pp];
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u] = fma(l, X[(p0 + pp) * (CB + 1) + gq + u], acc[u]);
            }
        }
        __syncthreads();
        if (gr < w)
#pragma unroll
            for (int u = 0; u < 4; ++u) X[(r0 + gr) * (CB + 1) + gq + u] -= acc[u];
        for (int e = t; e < 32 * 32; e += 256) {
            int q = e / 32, pp = e % 32;
            Ls[q * 33 + pp] = (q < w && pp < q) ? a.L[(int64_t)(r0 + q) * a.ldl + r0 + pp] : 0.0;
        }
        __syncthreads();
        {
            // substitution inside the chunk, right-looking over all eight warps:
            // once row p is final its value updates the rows below it (lane =
            // column, warp wq owns rows q = wq mod 8); every row receives its
            // terms in the order p = 0, 1, ..., as in a row-by-row substitution
            const int lane = t & 31, wq = t >> 5;
            for (int p = 0; p < w; ++p) {
                const double xp = X[(r0 + p) * (CB + 1) + lane];
                for (int q = wq; q < w; q += 8)
                    if (q > p) {
                        double* xq = X + (r0 + q) * (CB + 1) + lane;
                        *xq = fma(-Ls[q * 33 + p], xp, *xq);
                    }
                __syncthreads();
            }
        }
        __syncthreads();
    }
    for (int e = t; e < kb * CB; e += 256) {
        int r = e / CB, c = e % CB;
        if (c < nc) g.B[(int64_t)r * g.ldb + c0 + c] = X[r * (CB + 1) + c];
    }
}

__global__ void k_absmax(const double* A, int64_t lda, int64_t rows, int64_t cols,
                         double* out) {
    __shared__ double red[32];
    double m = 0.0;
    const int64_t tot = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e / cols, j = e % cols;
        double v = fabs(A[i * lda + j]);
        if (v > m) m = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        atomic_max_nonneg((unsigned long long*)out, m);
    }
}

int g_num_sms = 0;

}  // namespace

int num_sms() {
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

size_t getf2_stage_bytes(int64_t kb) {
    return sizeof(double) * 2 * ((size_t)num_sms() + 1) * (size_t)kb;
}

// shared memory of k_getf2_smem for G CTAs (0 when the rows do not fit)
size_t getf2_smem_bytes(int64_t m, int64_t kb, int64_t G) {
    static int cap = -1;
    if (cap < 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            v = 0;
        cap = v;
    }
    const int64_t R = (m + G - 1) / G;
    const size_t bytes = sizeof(double) * ((size_t)R * (size_t)kb + 2 * (size_t)kb);
    // static shared memory of the kernel (block_argmax, grid_barrier): < 512 bytes
    return bytes + 512 <= (size_t)cap ? bytes : 0;
}

cudaError_t launch_getf2_coop(double* P, int64_t lda, int64_t m, int64_t kb, int64_t K0,
                              int64_t* ipiv, DevStatus* st, double* part_v, int64_t* part_i,
                              double* stage, cudaStream_t s) {
    {   // rows in shared memory: every SM, one CTA each
        const int64_t G = m < num_sms() ? (m > 0 ? m : 1) : num_sms();
        const size_t sm = getf2_smem_bytes(m, kb, G);
        if (sm > 0 && kb <= 512 && kb % 32 == 0) {
            static int attr = -1;
            if ((int)sm > attr) {
                cudaError_t ea = cudaFuncSetAttribute(k_getf2_smem,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)sm);
                if (ea != cudaSuccess) return ea;
                attr = (int)sm;
            }
            cudaError_t e0 = cudaMemsetAsync(&st->bar_count, 0, sizeof(st->bar_count), s);
            if (e0 != cudaSuccess) return e0;
            int kbi = (int)kb;
            void* args[] = {&P, &lda, &m, &kbi, &K0, &ipiv, &st, &part_v, &part_i, &stage};
            cudaError_t e = cudaLaunchCooperativeKernel((void*)k_getf2_smem, dim3((unsigned)G),
                                                        dim3(PT), args, sm, s);
            note_launch();
            return e;
        }
    }
    int64_t want = (m + 63) / 64;
    int64_t G = want < num_sms() ? want : num_sms();
    if (G < 1) G = 1;
    while ((m + G - 1) / G > MAXR) ++G;   // rows per CTA must fit the shared buffer
    if (G > num_sms()) return cudaErrorInvalidValue;
    int kbi = (int)kb;
    cudaError_t e0 = cudaMemsetAsync(&st->bar_count, 0, sizeof(st->bar_count), s);
    if (e0 != cudaSuccess) return e0;
    void* args[] = {&P, &lda, &m, &kbi, &K0, &ipiv, &st, &part_v, &part_i, &stage};
    cudaError_t e = cudaLaunchCooperativeKernel((void*)k_getf2_coop, dim3((unsigned)G), dim3(PT),
                                                args, 0, s);
    note_launch();
    return e;
}

cudaError_t launch_laswp(double* A, int64_t lda, int64_t n, int64_t K0, int64_t kb,
                         const int64_t* ipiv, double* CS, int64_t ldcs, int64_t nc, int64_t g,
                         double* Cr, int64_t nt, int mode, cudaStream_t s) {
    int64_t tot = (n - kb) + (mode == MODE_FULL ? nt : 0);
    if (tot <= 0) return cudaSuccess;
    k_laswp<<<(unsigned)((tot + 127) / 128), 128, 0, s>>>(A, lda, n, K0, (int)kb, ipiv, CS, ldcs,
                                                          nc, g, Cr, nt, mode);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_coltot(const double* CS, int64_t ldcs, int64_t nc, int64_t k, int64_t nt,
                          int64_t K0, int64_t kb, double* ptot, cudaStream_t s) {
    k_coltot<<<1, 512, 0, s>>>(CS, ldcs, nc, k, nt, K0, (int)kb, ptot);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_lu_colsums(const double* P, int64_t lda, int64_t m, int64_t kb, int64_t g,
                              int64_t k, int64_t nt, int64_t K0, double* CS, int64_t ldcs,
                              int64_t nc, int mode, double* part, int64_t ldpart, cudaStream_t s) {
    k_lu_colsums<<<(unsigned)(nt - k), 256, 0, s>>>(P, lda, m, (int)kb, g, k, K0, CS, ldcs, nc,
                                                     mode, part, ldpart);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_lu_pd_check(const double* P, int64_t lda, int64_t kb, const double* ptot,
                               const double* part, int64_t ldpart, int nparts, int step,
                               int64_t K0, int64_t n, int64_t g, double tau_scale, double* z,
                               double* zw, int mode, DevStatus* st, cudaStream_t s) {
    const int64_t els = kb * kb;
    k_lu_umax<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(64, (els + 255) / 256)), 256, 0,
                s>>>(P, lda, (int)kb, st);
    note_launch();
    // columns over nchk CTAs of 16 warps (one column per warp), one more CTA for z
    const int nchk = (int)std::max<int64_t>(1, (kb + 15) / 16);
    k_lu_pd_check<<<(unsigned)(nchk + 1), 512, 0, s>>>(P, lda, (int)kb, ptot, part, ldpart, nparts,
                                                       step, K0, n, g, tau_scale, z, zw, mode, st,
                                                       nchk);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_trsm_llu(const double* L, int64_t ldl, int64_t kb, double* B0, int64_t ldb0,
                            int64_t ncols0, double* B1, int64_t ldb1, int64_t ncols1,
                            const double* z, const double* zw, double* colchk, double* colchkw,
                            cudaStream_t s, bool colchk_only) {
    TrsmLArgs a{};
    a.colchk_only = colchk_only ? 1 : 0;
    a.L = L; a.ldl = ldl; a.kb = (int)kb;
    a.nseg = 0;
    int64_t total = 0;
    TrsmLSeg segs[2] = {{B0, ldb0, ncols0}, {B1, ldb1, ncols1}};
    for (int i = 0; i < 2; ++i) {
        if (segs[i].ncols <= 0 || segs[i].B == nullptr) {
            if (i == 0) z = nullptr;
            continue;
        }
        a.seg[a.nseg] = segs[i];
        a.start[a.nseg] = total;
        total += (segs[i].ncols + CB - 1) / CB;
        a.nseg++;
    }
    if (total == 0) return cudaSuccess;
    a.start[a.nseg] = total;
    a.z = z; a.zw = zw; a.colchk = colchk; a.colchkw = colchkw;
    size_t smem = (size_t)(kb * (CB + 1) + 32 * 33) * sizeof(double);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_trsm_llu, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)((512 * (CB + 1) + 32 * 33) * sizeof(double)));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_trsm_llu<<<(unsigned)total, 256, smem, s>>>(a);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_absmax(const double* A, int64_t lda, int64_t rows, int64_t cols, double* out,
                          cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    int64_t blocks = (rows * cols + 255) / 256;
    if (blocks > 4 * num_sms()) blocks = 4 * num_sms();
    k_absmax<<<(unsigned)blocks, 256, 0, s>>>(A, lda, rows, cols, out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace abft
