// k_checksum.cu -- checksum encode, verify / locate / correct, fault injection,
// diagonal-block mirroring and the detection threshold (Sec. 3.1.2 ABFT:
// encode per matrix block before the operation, verify the checksum relation
// after it, locate and correct; 0D / 1D / 2D error classes).
//
// One CTA handles one g x g checksum tile (g <= 512).  Warp w sums rows
// w, w+8, ...; lane l holds the running column sums of columns l + 32 t, so
// every global load is a coalesced 256-byte row segment and the tile is read
// from HBM exactly once.  Row sums use warp shuffles.  All reductions run in a
// fixed order, so repeated runs give identical sums.
//
// Verification sums in fixed point: B300 issues one FP64 instruction per
// sub-partition every ~64 cycles, so FP64 column / row / weighted sums bound the
// verify by the FP64 pipe.  When the factorization has a magnitude bound
// (st->vexp > 0, set by the threshold kernels: Cholesky max(max a_ii, its
// square root); QR twice the largest column norm; LU 16 times the largest
// |a_ij| and |u_ij| seen, a heuristic), each entry of biased exponent <= vexp is
// truncated to an integer multiple of 2^(vexp - 1075) (less than one unit,
// 2^-52 of the bound, per entry) and summed exactly in 64-bit integers on the
// integer pipes; the weighted sums use units 2^10 larger to stay inside 64
// bits.  A tile holding an entry above the bound (an injected error, a NaN)
// is summed again in FP64, so detection, location and correction see the
// same quantities either way.
#include <cooperative_groups.h>
#include <math.h>

#include <type_traits>

#include "common.cuh"
#include "fp_bits.cuh"

namespace abft {

namespace {

namespace cg = cooperative_groups;

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxG = 512;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void tile_coords(const TileSet& ts, int64_t idx, int64_t& I, int64_t& J) {
    if (ts.lower) {
        // (a, b), a >= b, in row-major order of the lower triangle
        int64_t a = (int64_t)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
        while (a * (a + 1) / 2 > idx) --a;
        while ((a + 1) * (a + 2) / 2 <= idx) ++a;
        I = ts.I0 + a;
        J = ts.J0 + (idx - a * (a + 1) / 2);
    } else {
        int64_t nJ = ts.J1 - ts.J0;
        I = ts.I0 + idx / nJ;
        J = ts.J0 + idx % nJ;
    }
}

// Sums of one tile into shared memory: colsum[j], and when asked wsum[j]
// (weights 1..nr) and rowsum[i].  TM = column groups of 32 per lane (g <= 32 TM);
// each warp loads 32 / TM rows per batch, so a lane has 32 loads in flight.
template <int TM, bool COLW, bool ROWS>
__device__ void tile_sums(const double* T, int64_t ldt, int nr, int nc, double* colsum,
                          double* wsum, double* rowsum, double (*part)[kMaxG]) {
    constexpr int U = 32 / TM;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nt = (nc + 31) >> 5;
    double acc[TM], wacc[TM];
#pragma unroll
    for (int t = 0; t < TM; ++t) { acc[t] = 0.0; wacc[t] = 0.0; }
    for (int i0 = warp; i0 < nr; i0 += U * kWarps) {
        double v[U][TM];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * kWarps;
            const double* row = T + (int64_t)i * ldt;
#pragma unroll
            for (int t = 0; t < TM; ++t) {
                const int j = lane + 32 * t;
                v[u][t] = (t < nt && i < nr && j < nc) ? row[j] : 0.0;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * kWarps;
            const double wi = (double)(i + 1);
            double rs = 0.0;
#pragma unroll
            for (int t = 0; t < TM; ++t) {
                acc[t] += v[u][t];
                if (COLW) wacc[t] = fma(wi, v[u][t], wacc[t]);
                rs += v[u][t];
            }
            if (ROWS) {
                rs = warp_sum(rs);
                if (lane == 0 && i < nr) rowsum[i] = rs;
            }
        }
    }
    // combine the per-warp column partial sums in warp order
#pragma unroll
    for (int t = 0; t < TM; ++t)
        if (t < nt) part[warp][lane + 32 * t] = acc[t];
    __syncthreads();
    for (int j = threadIdx.x; j < nc; j += kThreads) {
        double s = 0.0;
        for (int w = 0; w < kWarps; ++w) s += part[w][j];
        colsum[j] = s;
    }
    __syncthreads();
    if (COLW) {
#pragma unroll
        for (int t = 0; t < TM; ++t)
            if (t < nt) part[warp][lane + 32 * t] = wacc[t];
        __syncthreads();
        for (int j = threadIdx.x; j < nc; j += kThreads) {
            double s = 0.0;
            for (int w = 0; w < kWarps; ++w) s += part[w][j];
            wsum[j] = s;
        }
        __syncthreads();
    }
}

// tile_sums in exact 64-bit fixed point (same outputs, converted to double
// once per sum).  Returns false, with nothing written, when an entry of the
// tile exceeds the bound: the caller then sums in FP64.
template <int TM, bool COLW, bool ROWS>
__device__ bool tile_sums_fixed(const double* T, int64_t ldt, int nr, int nc, int vexp,
                                double* colsum, double* wsum, double* rowsum,
                                double (*part)[kMaxG]) {
    constexpr int U = 32 / TM;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nt = (nc + 31) >> 5;
    long long acc[TM], wacc[TM];
#pragma unroll
    for (int t = 0; t < TM; ++t) { acc[t] = 0; wacc[t] = 0; }
    int emax = 0;
    long long (*ipart)[kMaxG] = reinterpret_cast<long long (*)[kMaxG]>(part);
    long long* irow = reinterpret_cast<long long*>(rowsum);
    for (int i0 = warp; i0 < nr; i0 += U * kWarps) {
        double v[U][TM];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * kWarps;
            const double* row = T + (int64_t)i * ldt;
#pragma unroll
            for (int t = 0; t < TM; ++t) {
                const int j = lane + 32 * t;
                v[u][t] = (t < nt && i < nr && j < nc) ? row[j] : 0.0;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * kWarps;
            long long rs = 0;
#pragma unroll
            for (int t = 0; t < TM; ++t) {
                const long long q = to_fixed(v[u][t], vexp, emax);
                acc[t] += q;
                if (COLW) wacc[t] += (long long)(i + 1) * (q >> 10);
                rs += q;
            }
            if (ROWS) {
                rs = warp_sum_ll(rs);
                if (lane == 0 && i < nr) irow[i] = rs;
            }
        }
    }
    if (__syncthreads_or(emax > vexp ? 1 : 0)) return false;
    const double unit = ldexp(1.0, vexp - 1075), wunit = ldexp(1.0, vexp - 1065);
#pragma unroll
    for (int t = 0; t < TM; ++t)
        if (t < nt) ipart[warp][lane + 32 * t] = acc[t];
    __syncthreads();
    for (int j = threadIdx.x; j < nc; j += kThreads) {
        long long s = 0;
        for (int w = 0; w < kWarps; ++w) s += ipart[w][j];
        colsum[j] = (double)s * unit;
    }
    if (ROWS)
        for (int i = threadIdx.x; i < nr; i += kThreads) rowsum[i] = (double)irow[i] * unit;
    __syncthreads();
    if (COLW) {
#pragma unroll
        for (int t = 0; t < TM; ++t)
            if (t < nt) ipart[warp][lane + 32 * t] = wacc[t];
        __syncthreads();
        for (int j = threadIdx.x; j < nc; j += kThreads) {
            long long s = 0;
            for (int w = 0; w < kWarps; ++w) s += ipart[w][j];
            wsum[j] = (double)s * wunit;
        }
        __syncthreads();
    }
    return true;
}

__device__ __forceinline__ void tile_extent(const TileSet& ts, int64_t I, int64_t J, int& nr,
                                            int& nc) {
    int64_t r0 = I * ts.g, c0 = J * ts.g;
    int64_t a = ts.nrow_end - r0, b = ts.ncol_end - c0;
    nr = (int)(a < ts.g ? a : ts.g);
    nc = (int)(b < ts.g ? b : ts.g);
}

template <int TM, bool COLW, bool ROWS>
__global__ void __launch_bounds__(kThreads) k_encode(TileSet ts) {
    __shared__ double part[kWarps][kMaxG];
    __shared__ double colsum[kMaxG], wsum[kMaxG], rowsum[kMaxG];
    int64_t I, J;
    tile_coords(ts, blockIdx.x, I, J);
    int nr, nc;
    tile_extent(ts, I, J, nr, nc);
    if (nr <= 0 || nc <= 0) return;
    const double* T = ts.A + I * ts.g * ts.lda + J * ts.g;
    tile_sums<TM, COLW, ROWS>(T, ts.lda, nr, nc, colsum, wsum, rowsum, part);
    double* cc = ts.cc + I * ts.ccI + J * ts.g;
    for (int j = threadIdx.x; j < nc; j += kThreads) {
        cc[j] = colsum[j];
        if (COLW) ts.cw[I * ts.ccI + J * ts.g + j] = wsum[j];
    }
    if (ROWS) {
        double* cr = ts.cr + I * ts.g * ts.crs + J * ts.crJ;
        for (int i = threadIdx.x; i < nr; i += kThreads) cr[(int64_t)i * ts.crs] = rowsum[i];
    }
}

// Verify, classify and correct one tile.  Flags: |d| > tau (NaN flags).
// Full mode: 1 row + 1 col -> 0D (T[i][j] -= d^c_j when |d^c_j - d^r_i| <= tau,
// else uncorrectable); 1 row + >=2 cols -> 1D row (T[i][j] -= d^c_j);
// >=2 rows + 1 col -> 1D column (T[i][j] -= d^r_i); one side only -> the
// checksum is wrong, re-encode it; >=2 rows and >=2 cols -> 2D, uncorrectable.
// Single mode: each flagged column is located at i = rint(d^w_j / d^c_j) - 1
// (accepted within 0.05 of an integer and inside the tile) and corrected by d^c_j.
// The classification after the sums (colsum, wsum, rowsum hold the recomputed
// sums of the tile at T); part[] is scratch that aliases none of them.  sf: four
// shared ints, s_dmax: kWarps shared doubles.  Called by every thread of one CTA.
__device__ void verify_classify(const TileSet& ts, int MODE, int step, DevStatus* st, int64_t I,
                                int64_t J, int nr, int nc, double* T, double* colsum, double* wsum,
                                double* rowsum, double (*part)[kMaxG], int* sf, double* s_dmax) {
    const int64_t r0 = I * ts.g, c0 = J * ts.g;
    double* cc = ts.cc + I * ts.ccI + J * ts.g;
    double* cw = (MODE == MODE_SINGLE) ? ts.cw + I * ts.ccI + J * ts.g : nullptr;
    double* cr = (MODE == MODE_FULL) ? ts.cr + r0 * ts.crs + J * ts.crJ : nullptr;
    if (threadIdx.x == 0) { sf[0] = 0; sf[1] = 0; sf[2] = 1 << 30; sf[3] = 1 << 30; }
    __syncthreads();
    const double tau = st->tau;
    // thresholds per column and row: the scalar tau, or (mixed precision)
    // tau_coef |c|_j + tau64 from the FP32 abs-checksums, formed with one FP32
    // fused multiply-add and widened to FP64 by integer operations (the flag
    // test itself stays one FP64 comparison); part[] is free again
    const bool pc = ts.ca != nullptr;
    double* tcol = part[0];
    double* trow = part[1];
    float* tcol32 = reinterpret_cast<float*>(part[2]);
    float* trow32 = tcol32 + kMaxG;
    if (pc) {
        const float c32 = (float)st->tau_coef, t32 = (float)st->tau64;
        const float* ca = ts.ca + I * ts.caI + J * ts.g;
        float tmax = 0.0f;
        for (int j = threadIdx.x; j < nc; j += kThreads) {
            const float t = fmaf(c32, ca[j], t32);
            tcol32[j] = t;
            tcol[j] = f32_to_f64_exact(t);
            tmax = fmaxf(tmax, t);
        }
        if (MODE == MODE_FULL) {
            const float* ra = ts.ra + r0 * ts.crs + J * ts.crJ;
            for (int i = threadIdx.x; i < nr; i += kThreads) {
                const float t = fmaf(c32, ra[(int64_t)i * ts.crs], t32);
                trow32[i] = t;
                trow[i] = f32_to_f64_exact(t);
                tmax = fmaxf(tmax, t);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
        if ((threadIdx.x & 31) == 0 && tmax > 0.0f)
            atomic_max_nonneg(&st->tau_max_bits, f32_to_f64_exact(tmax));
        __syncthreads();
    }
#define TCOL(j) (pc ? tcol[j] : tau)
#define TROW(i) (pc ? trow[i] : tau)
    // largest |d| (scalar threshold) or largest |d| / threshold in FP32
    // (per-column thresholds; a diagnostic, so truncated operands suffice)
    double dmax = 0.0;
    float rmax = 0.0f;
    // d = recomputed - carried, kept in place of the sums
    for (int j = threadIdx.x; j < nc; j += kThreads) {
        double d = colsum[j] - cc[j];
        colsum[j] = d;
        if (MODE == MODE_SINGLE) wsum[j] = wsum[j] - cw[j];
        double a = fabs(d);
        if (!(a <= TCOL(j))) { atomicAdd(&sf[0], 1); atomicMin(&sf[2], j); }
        if (pc) rmax = fmaxf(rmax, __fdividef(f64_abs_to_f32_trunc(a), tcol32[j]));
        else if (a > dmax) dmax = a;
    }
    if (MODE == MODE_FULL)
        for (int i = threadIdx.x; i < nr; i += kThreads) {
            double d = rowsum[i] - cr[(int64_t)i * ts.crs];
            rowsum[i] = d;
            double a = fabs(d);
            if (!(a <= TROW(i))) { atomicAdd(&sf[1], 1); atomicMin(&sf[3], i); }
            if (pc) rmax = fmaxf(rmax, __fdividef(f64_abs_to_f32_trunc(a), trow32[i]));
            else if (a > dmax) dmax = a;
        }
    if (pc) dmax = f32_to_f64_exact(rmax);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if ((threadIdx.x & 31) == 0) s_dmax[threadIdx.x >> 5] = dmax;
    __syncthreads();
    const int nfc = sf[0], nfr = sf[1], fc = sf[2], fr = sf[3];
    if (nfc == 0 && nfr == 0) {
        if (threadIdx.x == 0) {
            double m = 0.0;
            for (int w = 0; w < kWarps; ++w) m = fmax(m, s_dmax[w]);
            if (pc) atomic_max_nonneg(&st->max_ratio_bits, m);
            else if (tau > 0.0) atomic_max_nonneg(&st->max_ratio_bits, m / tau);
        }
        return;
    }
    if (threadIdx.x == 0) atomicAdd(&st->detected, 1ull);
    if (MODE == MODE_SINGLE) {
        for (int j = threadIdx.x; j < nc; j += kThreads) {
            double dc = colsum[j];
            if (fabs(dc) <= TCOL(j)) continue;
            double rho = wsum[j] / dc;
            double ri = rint(rho);
            int64_t i = (int64_t)ri - 1;
            if (fabs(rho - ri) <= 0.05 && i >= 0 && i < nr) {
                T[i * ts.lda + j] -= dc;
                atomicAdd(&st->corrected, 1ull);
                record_event(st, step, EV_0D, r0 + i, c0 + j, dc);
            } else {
                atomicAdd(&st->uncorrectable, 1ull);
                record_event(st, step, EV_UNCORR, r0, c0 + j, dc);
            }
        }
        return;
    }
    if (nfr == 1 && nfc == 1) {
        if (threadIdx.x == 0) {
            double dc = colsum[fc], dr = rowsum[fr];
            if (fabs(dc - dr) <= (pc ? __dadd_rn(tcol[fc], trow[fr]) : tau)) {
                T[(int64_t)fr * ts.lda + fc] -= dc;
                atomicAdd(&st->corrected, 1ull);
                record_event(st, step, EV_0D, r0 + fr, c0 + fc, dc);
            } else {
                atomicAdd(&st->uncorrectable, 1ull);
                record_event(st, step, EV_UNCORR, r0, c0, dc);
            }
        }
    } else if (nfr == 1 && nfc >= 2) {
        for (int j = threadIdx.x; j < nc; j += kThreads) {
            double dc = colsum[j];
            if (fabs(dc) <= TCOL(j)) continue;
            T[(int64_t)fr * ts.lda + j] -= dc;
            atomicAdd(&st->corrected, 1ull);
            record_event(st, step, EV_ROW, r0 + fr, c0 + j, dc);
        }
    } else if (nfr >= 2 && nfc == 1) {
        for (int i = threadIdx.x; i < nr; i += kThreads) {
            double dr = rowsum[i];
            if (fabs(dr) <= TROW(i)) continue;
            T[(int64_t)i * ts.lda + fc] -= dr;
            atomicAdd(&st->corrected, 1ull);
            record_event(st, step, EV_COL, r0 + i, c0 + fc, dr);
        }
    } else if (nfr == 0 || nfc == 0) {
        // the checksum itself is wrong: re-encode it from the data
        for (int j = threadIdx.x; j < nc; j += kThreads) cc[j] += colsum[j];
        for (int i = threadIdx.x; i < nr; i += kThreads) cr[(int64_t)i * ts.crs] += rowsum[i];
        if (threadIdx.x == 0) {
            atomicAdd(&st->repaired, 1ull);
            record_event(st, step, EV_CKSUM, r0, c0, 0.0);
        }
    } else if (threadIdx.x == 0) {
        atomicAdd(&st->uncorrectable, 1ull);
        record_event(st, step, EV_UNCORR, r0, c0, 0.0);
    }
#undef TCOL
#undef TROW
}

template <int MODE, int TM>
__global__ void __launch_bounds__(kThreads) k_verify(TileSet ts, int step, DevStatus* st) {
    __shared__ double part[kWarps][kMaxG];
    __shared__ double colsum[kMaxG], wsum[kMaxG], rowsum[kMaxG];
    __shared__ int sf[4];
    __shared__ double s_dmax[kWarps];
    if (st->info != 0) return;
    int64_t I, J;
    tile_coords(ts, blockIdx.x, I, J);
    int nr, nc;
    tile_extent(ts, I, J, nr, nc);
    if (nr <= 0 || nc <= 0) return;
    double* T = ts.A + I * ts.g * ts.lda + J * ts.g;
    const int vexp = st->vexp;
    if (vexp <= 0 ||
        !tile_sums_fixed<TM, MODE == MODE_SINGLE, MODE == MODE_FULL>(T, ts.lda, nr, nc, vexp, colsum,
                                                                     wsum, rowsum, part))
        tile_sums<TM, MODE == MODE_SINGLE, MODE == MODE_FULL>(T, ts.lda, nr, nc, colsum, wsum,
                                                             rowsum, part);
    verify_classify(ts, MODE, step, st, I, J, nr, nc, T, colsum, wsum, rowsum, part, sf, s_dmax);
}

// ---- few tiles: one cluster of S CTAs per tile ----
// A launch with few tiles (the block column verified ahead of the next panel,
// the panel itself) leaves most SMs idle, and one CTA takes ~25 us for a
// 256 x 256 tile, on the critical path of the look-ahead.  Here the S CTAs of
// a cluster (S <= 8) each sum a slab of ceil(g / S) rows: the slab's row sums
// complete and its column partial sums, in its own shared memory.  After a
// cluster barrier, rank 0 adds the column partials of ranks 0 .. S-1 in rank
// order (exact in fixed point, a fixed order in FP64), gathers the row sums
// from the slabs' CTAs and classifies.  When any slab holds an entry above
// the fixed-point bound, every slab is summed again in FP64, so the ranks agree
// on the form of the sums.  The failure flag st->info is read by rank 0 alone and shared, so
// every CTA of a cluster passes the same barriers.

// Sums of rows ra .. rb - 1 of a tile (FIX: 64-bit fixed point, false when an
// entry exceeds the bound): column (weighted) partials into cpart / wpart, row
// sums into rdst (as long long when FIX).
template <int TM, bool COLW, bool ROWS, bool FIX>
__device__ bool slab_sums(const double* T, int64_t ldt, int ra, int rb, int nc, int vexp,
                          double* cpart, double* wpart, double* rdst, double (*part)[kMaxG]) {
    using Acc = typename std::conditional<FIX, long long, double>::type;
    constexpr int U = 32 / TM;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nt = (nc + 31) >> 5;
    Acc acc[TM], wacc[TM];
#pragma unroll
    for (int t = 0; t < TM; ++t) { acc[t] = 0; wacc[t] = 0; }
    int emax = 0;
    for (int i0 = ra + warp; i0 < rb; i0 += U * kWarps) {
        double v[U][TM];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * kWarps;
            const double* row = T + (int64_t)i * ldt;
#pragma unroll
            for (int t = 0; t < TM; ++t) {
                const int j = lane + 32 * t;
                v[u][t] = (t < nt && i < rb && j < nc) ? row[j] : 0.0;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * kWarps;
            Acc rs = 0;
#pragma unroll
            for (int t = 0; t < TM; ++t) {
                if constexpr (FIX) {
                    const long long q = to_fixed(v[u][t], vexp, emax);
                    acc[t] += q;
                    if (COLW) wacc[t] += (long long)(i + 1) * (q >> 10);
                    rs += q;
                } else {
                    acc[t] += v[u][t];
                    if (COLW) wacc[t] = fma((double)(i + 1), v[u][t], wacc[t]);
                    rs += v[u][t];
                }
            }
            if (ROWS) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
                if (lane == 0 && i < rb) reinterpret_cast<Acc*>(rdst)[i] = rs;
            }
        }
    }
    Acc (*ip)[kMaxG] = reinterpret_cast<Acc (*)[kMaxG]>(part);
#pragma unroll
    for (int t = 0; t < TM; ++t)
        if (t < nt) ip[warp][lane + 32 * t] = acc[t];
    const bool bad = __syncthreads_or(FIX && emax > vexp ? 1 : 0) != 0;
    for (int j = threadIdx.x; j < nc; j += kThreads) {
        Acc sm = 0;
        for (int w = 0; w < kWarps; ++w) sm += ip[w][j];
        reinterpret_cast<Acc*>(cpart)[j] = sm;
    }
    if (COLW) {
        __syncthreads();
#pragma unroll
        for (int t = 0; t < TM; ++t)
            if (t < nt) ip[warp][lane + 32 * t] = wacc[t];
        __syncthreads();
        for (int j = threadIdx.x; j < nc; j += kThreads) {
            Acc sm = 0;
            for (int w = 0; w < kWarps; ++w) sm += ip[w][j];
            reinterpret_cast<Acc*>(wpart)[j] = sm;
        }
    }
    return !bad;
}

template <int MODE, int TM, int S>
__global__ void __launch_bounds__(kThreads, 2) k_verify_cl(TileSet ts, int step, DevStatus* st) {
    __shared__ double part[kWarps][kMaxG];
    // colsum / wsum hold this slab's column partials until rank 0 adds them up
    // (each of its threads reads and then overwrites its own columns)
    __shared__ double colsum[kMaxG], wsum[kMaxG], rowsum[kMaxG];
    __shared__ int sf[4];
    __shared__ double s_dmax[kWarps];
    __shared__ int s_info, s_bad;
    constexpr bool COLW = MODE == MODE_SINGLE, ROWS = MODE == MODE_FULL;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    int64_t I, J;
    tile_coords(ts, blockIdx.x / S, I, J);
    int nr, nc;
    tile_extent(ts, I, J, nr, nc);   // the same for every CTA of the cluster
    if (nr <= 0 || nc <= 0) return;
    double* T = ts.A + I * ts.g * ts.lda + J * ts.g;
    const int slab = (int)((ts.g + S - 1) / S);
    const int ra = rank * slab < nr ? rank * slab : nr;
    const int rb = ra + slab < nr ? ra + slab : nr;
    const int vexp = st->vexp;
    if (rank == 0 && threadIdx.x == 0) s_info = st->info;
    bool fix = vexp > 0;
    int ok = 1;
    if (fix)
        ok = slab_sums<TM, COLW, ROWS, true>(T, ts.lda, ra, rb, nc, vexp, colsum, wsum, rowsum,
                                             part);
    else
        slab_sums<TM, COLW, ROWS, false>(T, ts.lda, ra, rb, nc, 0, colsum, wsum, rowsum, part);
    if (threadIdx.x == 0) s_bad = ok ? 0 : 1;
    cl.sync();
    const int info = *cl.map_shared_rank(&s_info, 0);
    int bad = 0;
    for (int r = 0; r < S; ++r) bad |= *cl.map_shared_rank(&s_bad, r);
    if (info == 0 && bad) {   // every slab again in FP64 (the flags stay as they are)
        fix = false;
        slab_sums<TM, COLW, ROWS, false>(T, ts.lda, ra, rb, nc, 0, colsum, wsum, rowsum, part);
        cl.sync();
    }
    if (info == 0 && rank == 0) {
        const double unit = fix ? ldexp(1.0, vexp - 1075) : 1.0;
        const double wunit = fix ? ldexp(1.0, vexp - 1065) : 1.0;
        for (int j = threadIdx.x; j < nc; j += kThreads) {
            if (fix) {
                long long c = 0, w = 0;
                for (int r = 0; r < S; ++r) {
                    c += reinterpret_cast<const long long*>(cl.map_shared_rank(colsum, r))[j];
                    if (COLW) w += reinterpret_cast<const long long*>(cl.map_shared_rank(wsum, r))[j];
                }
                colsum[j] = (double)c * unit;
                if (COLW) wsum[j] = (double)w * wunit;
            } else {
                double c = 0.0, w = 0.0;
                for (int r = 0; r < S; ++r) {
                    c += cl.map_shared_rank(colsum, r)[j];
                    if (COLW) w += cl.map_shared_rank(wsum, r)[j];
                }
                colsum[j] = c;
                if (COLW) wsum[j] = w;
            }
        }
        if (ROWS)
            for (int i = threadIdx.x; i < nr; i += kThreads) {
                const double* src = cl.map_shared_rank(rowsum, i / slab);
                rowsum[i] = fix ? (double)reinterpret_cast<const long long*>(src)[i] * unit : src[i];
            }
        __syncthreads();
    }
    cl.sync();   // rank 0 has read every slab's partials: no CTA leaves before
    if (info == 0 && rank == 0)
        verify_classify(ts, MODE, step, st, I, J, nr, nc, T, colsum, wsum, rowsum, part, sf,
                        s_dmax);
}

__global__ void k_inject(double* A, int64_t lda, int64_t row, int64_t col, int64_t len, int along_row,
                         double delta) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= len) return;
    if (along_row) A[row * lda + col + t] += delta;
    else A[(row + t) * lda + col] += delta;
}

// Save the strict upper triangle of every nb x nb diagonal block and mirror the
// lower triangle into it (restore = 1 puts the saved values back).
__global__ void k_mirror_diag(double* A, int64_t lda, int64_t n, int64_t nb, double* save,
                              int restore) {
    int64_t K0 = blockIdx.x * nb;
    int64_t kb = n - K0 < nb ? n - K0 : nb;
    for (int64_t e = threadIdx.x; e < kb * kb; e += blockDim.x) {
        int64_t i = e / kb, j = e % kb;
        if (j <= i) continue;
        double* up = A + (K0 + i) * lda + K0 + j;
        double* sv = save + (K0 + i) * nb + j;
        if (restore) {
            *up = *sv;
        } else {
            *sv = *up;
            *up = A[(K0 + j) * lda + K0 + i];
        }
    }
}

// tau = tau_scale * 8 * u * n * g * max_i a_ii (left to right); u = 2^-53 for the
// FP64 update, 2^-24 when the update accumulates in FP32 (mixed precision).
__global__ void k_tau_chol(const double* A, int64_t lda, int64_t n, int64_t g, double tau_scale,
                           double u, double coef, DevStatus* st) {
    __shared__ double red[32];
    double m = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double d = A[i * lda + i];
        if (d > m) m = d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        double t = tau_scale * 8.0;
        t *= u;
        t *= (double)n;
        t *= (double)g;
        t *= m;
        st->tau = t;
        if (coef > 0.0) {   // mixed precision: the FP64 term of the per-column thresholds
            double t64 = tau_scale * 8.0;
            t64 *= 0x1p-53;
            t64 *= (double)n;
            t64 *= (double)g;
            t64 *= m;
            st->tau64 = t64;
            st->tau_coef = coef;
        }
        // entries of the Schur complements are bounded by max a_ii, panel
        // entries by sqrt(max a_ii): the fixed-point verify bound
        const double bnd = fmax(m, sqrt(m));
        const int ve = (int)((__double_as_longlong(bnd) >> 52) & 0x7ff);
        st->vexp = (bnd > 0.0 && bnd < 1e300 && ve >= kFixedMinExp) ? ve : 0;
    }
}

int64_t tile_count(const TileSet& ts) {
    if (ts.lower) {
        int64_t a = ts.I1 - ts.I0;
        return a * (a + 1) / 2;
    }
    return (ts.I1 - ts.I0) * (ts.J1 - ts.J0);
}

template <int TM>
void encode_t(const TileSet& ts, int mode, int64_t nt, cudaStream_t s) {
    const bool colw = mode == MODE_SINGLE || ts.weighted;
    if (mode == MODE_FULL && colw) k_encode<TM, true, true><<<(unsigned)nt, kThreads, 0, s>>>(ts);
    else if (mode == MODE_FULL) k_encode<TM, false, true><<<(unsigned)nt, kThreads, 0, s>>>(ts);
    else k_encode<TM, true, false><<<(unsigned)nt, kThreads, 0, s>>>(ts);
}

template <int MODE, int S>
cudaError_t launch_cl(const TileSet& ts, int step, DevStatus* st, int64_t nt, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nt * S), 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = S;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_verify_cl<MODE, 8, S>, ts, step, st);
}

template <int MODE>
cudaError_t verify_cl_t(const TileSet& ts, int S, int step, DevStatus* st, int64_t nt,
                        cudaStream_t s) {
    if (S == 8) return launch_cl<MODE, 8>(ts, step, st, nt, s);
    if (S == 4) return launch_cl<MODE, 4>(ts, step, st, nt, s);
    return launch_cl<MODE, 2>(ts, step, st, nt, s);
}

template <int TM>
void verify_t(const TileSet& ts, int mode, int step, DevStatus* st, int64_t nt, cudaStream_t s) {
    if (mode == MODE_FULL) k_verify<MODE_FULL, TM><<<(unsigned)nt, kThreads, 0, s>>>(ts, step, st);
    else k_verify<MODE_SINGLE, TM><<<(unsigned)nt, kThreads, 0, s>>>(ts, step, st);
}

}  // namespace

cudaError_t launch_encode(const TileSet& ts, int mode, cudaStream_t s) {
    int64_t nt = tile_count(ts);
    if (nt <= 0 || mode == MODE_NONE) return cudaSuccess;
    if (ts.g > kMaxG) return cudaErrorInvalidValue;
    if (ts.g <= 256) encode_t<8>(ts, mode, nt, s);
    else encode_t<16>(ts, mode, nt, s);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_verify(const TileSet& ts, int mode, int step, DevStatus* st, cudaStream_t s) {
    int64_t nt = tile_count(ts);
    if (nt <= 0 || mode == MODE_NONE) return cudaSuccess;
    if (ts.g > kMaxG) return cudaErrorInvalidValue;
    // few tiles: S CTAs per tile, the largest S in {2, 4, 8} with at most two
    // CTAs per SM in all (one per tile from num_sms() tiles on)
    const int64_t slots = 2 * (int64_t)num_sms();
    const int S = nt * 8 <= slots ? 8 : nt * 4 <= slots ? 4 : nt * 2 <= slots ? 2 : 1;
    if (S > 1 && ts.g <= 256) {
        const cudaError_t e = mode == MODE_FULL ? verify_cl_t<MODE_FULL>(ts, S, step, st, nt, s)
                                                : verify_cl_t<MODE_SINGLE>(ts, S, step, st, nt, s);
        if (e != cudaSuccess) return e;
    } else if (ts.g <= 256) {
        verify_t<8>(ts, mode, step, st, nt, s);
    } else {
        verify_t<16>(ts, mode, step, st, nt, s);
    }
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_inject(double* A, int64_t lda, int64_t n, int64_t g, const abft_fault& f,
                          cudaStream_t s) {
    int64_t len = 1;
    int along_row = 1;
    if (f.kind == ABFT_FAULT_ROW1D) {
        int64_t end = (f.col / g + 1) * g;
        if (end > n) end = n;
        len = end - f.col;
    } else if (f.kind == ABFT_FAULT_COL1D) {
        int64_t end = (f.row / g + 1) * g;
        if (end > n) end = n;
        len = end - f.row;
        along_row = 0;
    }
    k_inject<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(A, lda, f.row, f.col, len, along_row,
                                                          f.delta);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_mirror_diag(double* A, int64_t lda, int64_t n, int64_t nb, double* save,
                               int restore, cudaStream_t s) {
    int64_t nblk = (n + nb - 1) / nb;
    if (nblk <= 0) return cudaSuccess;
    k_mirror_diag<<<(unsigned)nblk, 256, 0, s>>>(A, lda, n, nb, save, restore);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_tau_chol(const double* A, int64_t lda, int64_t n, int64_t g, double tau_scale,
                            DevStatus* st, cudaStream_t s, double unit_roundoff, double tau_coef) {
    k_tau_chol<<<1, 1024, 0, s>>>(A, lda, n, g, tau_scale, unit_roundoff, tau_coef, st);
    note_launch();
    return cudaGetLastError();
}

}  // namespace abft
