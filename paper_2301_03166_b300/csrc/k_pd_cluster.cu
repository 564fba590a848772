// k_pd_cluster.cu -- FP64 factorization of a diagonal block of the blocked
// Cholesky (Sec. 2.1 PD) by one thread-block cluster, with the PD checksum
// check (Sec. 3.1.2) fused.
//
// B300 runs FP64 at about two lanes per clock per SM, so a kb x kb block
// (kb <= 256: kb^3 / 6 = 2.8 M FMA) takes most of a millisecond on one SM.
// Here the block's lower triangle is held as 32 x 32 tiles spread over the
// shared memory of the CL CTAs of a cluster (tile id = q (q + 1) / 2 + r,
// home CTA id % CL, slot id / CL; rows past kb are the identity) and factored
// right-looking by tile columns p = 0 .. NT - 1:
//   A  the home CTA of tile (p, p) factors it square-root free (L D L^T, one
//      reciprocal per pivot on the dependent chain, formed while the other
//      warps apply the previous pivot; the 32 square roots and the column
//      scalings by their reciprocals at the end);
//   B  the rows of the tiles (q, p), q > p, are solved against it, one warp
//      per row (lane l holds x_l), or two rows per warp when there are more
//      rows than warps, spread over every warp of the cluster; the
//      division by L_jj is a multiplication by its reciprocal (one FP64
//      division per column instead of one per row: on B300 a dependent FP64
//      division costs hundreds of clocks; the reciprocals of the power-of-two
//      pivots of exact integer cases are exact), folded into the tile's
//      columns (L_lj / L_jj) so that each unknown costs one FMA; the home CTA
//      forms this operand when it factors the tile, the others copy it;
//   C  the trailing tiles C(q, r) -= L(q, p) L(r, p)^T, p < r <= q, in halves
//      of 16 rows (the first half of a diagonal tile in its lower 16 columns
//      only); operands are fetched from their home CTAs through
//      distributed shared memory.  Look-ahead: the home CTA of tile
//      (p + 1, p + 1) updates that tile first and factors it (A of the next
//      step) while the other CTAs share the rest of the tiles.
// The phases are separated by cluster barriers (hardware barriers, no spin).
// Then the PD checksum relation (1^T L) L^T = c^T is checked against the
// carried column checksum cc from the tiles in shared memory (per-tile
// partial sums in every CTA, added in a fixed order by CTA 0), and every CTA
// writes its tiles back to A.
#include <cooperative_groups.h>
#include <math.h>

#include "common.cuh"

namespace abft {

namespace cg = cooperative_groups;

namespace {

constexpr int PT = 32;             // tile edge
constexpr int PLD = 33;            // padded row stride (doubles)
constexpr int PMAXT = 8;           // tiles per side: kb <= 256
constexpr int PTHREADS = 256;
constexpr int PWARPS = PTHREADS / 32;
constexpr int TILE = PT * PLD;
static_assert(PT * PT == 4 * PTHREADS, "tile copies take 4 entries per thread");

template <int CL>
__host__ __device__ constexpr int pd_slots() {
    return (PMAXT * (PMAXT + 1) / 2 + CL - 1) / CL;
}

template <int CL>
constexpr size_t pd_smem() {
    return sizeof(double) * (size_t)TILE * (pd_slots<CL>() + 4);
}

__device__ __forceinline__ void tile_of(int id, int& q, int& r) {
    q = 0;
    while ((q + 1) * (q + 2) / 2 <= id) ++q;
    r = id - q * (q + 1) / 2;
}

template <int CL>
__global__ void __launch_bounds__(PTHREADS, 1) k_potrf_pd_cluster(double* A, int64_t lda, int kb,
                                                                  int64_t K0, const double* cc,
                                                                  int step, int check,
                                                                  DevStatus* st) {
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) double pd_sm[];
    double* home = pd_sm;                              // pd_slots tiles
    double* sD = pd_sm + pd_slots<CL>() * TILE;        // copy of L(p, p)
    double* sQ = sD + TILE;                            // operand copies for phase C
    double* sR = sQ + TILE;
    double* sB = sR + TILE;                            // solve operand of the last tile factored here
    __shared__ int s_fail;
    __shared__ double s_rinv[PT];                      // 1 / sqrt(d_j) (A)
    __shared__ double s_cs[PMAXT * PT];
    if (st->info != 0) return;                         // same answer in every CTA
    const int me = (int)cl.block_rank();
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int NT = (kb + PT - 1) / PT, NTILE = NT * (NT + 1) / 2;
    auto tile_ptr = [&](int q, int r) -> double* {
        const int id = q * (q + 1) / 2 + r;
        return cl.map_shared_rank(home + (id / CL) * TILE, id % CL);
    };
    // this CTA's tiles from A (the strict upper part of diagonal tiles is not
    // used; rows and columns past kb are the identity)
    for (int id = me; id < NTILE; id += CL) {
        int q, r;
        tile_of(id, q, r);
        double* T = home + (id / CL) * TILE;
        for (int e = t; e < PT * PT; e += PTHREADS) {
            const int i = e >> 5, j = e & 31, gi = q * PT + i, gj = r * PT + j;
            double v;
            if (gi < kb && gj < kb) v = (q > r || j <= i) ? A[(int64_t)gi * lda + gj] : 0.0;
            else v = gi == gj ? 1.0 : 0.0;
            T[i * PLD + j] = v;
        }
    }
    // (a, b), b <= a, of a trailing triangle in row-major order: the first
    // m (m + 1) / 2 entries are the triangle of order m
    __shared__ unsigned char s_ta[PT * (PT - 1) / 2], s_tb[PT * (PT - 1) / 2];
    __shared__ double s_sc2[2][PT];
    __shared__ double s_sq[PT];
    for (int e = t; e < PT * (PT - 1) / 2; e += PTHREADS) {
        int a = 0;
        while ((a + 1) * (a + 2) / 2 <= e) ++a;
        s_ta[e] = (unsigned char)a;
        s_tb[e] = (unsigned char)(e - a * (a + 1) / 2);
    }
    if (t == 0) s_fail = -1;
    // A: diagonal tile (p, p) in its home CTA, square-root free (L D L^T,
    // right-looking): per pivot one reciprocal of d_j on the dependent chain
    // (an FP64 square root and a division per pivot cost 675 and 431 clocks on
    // B300); the trailing entries take D[i][j] (D[l][j] / d_j), the quotient
    // formed once per row l.  Look-ahead by one pivot, one barrier per pivot:
    // while warps 1 .. 7 update the trailing entries of columns l >= j + 2 for
    // pivot j, warp 0 updates column j + 1, then forms 1 / d_(j+1) and the
    // quotients of pivot j + 1 (in the other buffer of s_sc), so that the
    // division overlaps the bulk of the update.  Every entry takes the same
    // operations in the same order as the plain recurrence.  Then
    // L = L_unit D^(1/2): column j is D[i][j] / sqrt(d_j), taken as a product
    // with 1 / sqrt(d_j).  A non-positive d_j fails at the same pivot as the
    // Cholesky recurrence (d_j is the value under its square root).
    auto factor_diag = [&](int p) {
        const int idp = p * (p + 1) / 2 + p;
        double* D = home + (idp / CL) * TILE;
        // warp 0: the quotients D[l][j] / d_j of pivot j (l > j) into s_sc2[j & 1]
        auto pivot = [&](int j) {
            const double d = D[j * PLD + j];
            if (!(d > 0.0)) {
                if (lane == 0) s_fail = j;
                return;
            }
            const double rj = 1.0 / d;
            if (lane > j) s_sc2[j & 1][lane] = D[lane * PLD + j] * rj;
        };
        if (warp == 0) pivot(0);
        __syncthreads();
        for (int j = 0; j < PT; ++j) {
            if (s_fail >= 0) return;
            if (j == PT - 1) break;
            const double* sc = s_sc2[j & 1];
            if (warp == 0) {
                if (lane > j) D[lane * PLD + j + 1] -= D[lane * PLD + j] * sc[j + 1];
                __syncwarp();
                pivot(j + 1);
            } else {
                const int m = PT - 2 - j;                    // columns j + 2 .. PT - 1
                for (int e = t - 32; e < m * (m + 1) / 2; e += PTHREADS - 32) {
                    const int i = j + 2 + s_ta[e], l = j + 2 + s_tb[e];
                    D[i * PLD + l] -= D[i * PLD + j] * sc[l];
                }
            }
            __syncthreads();
        }
        if (t < PT) {
            const double sq = sqrt(D[t * PLD + t]);
            s_sq[t] = sq;
            s_rinv[t] = 1.0 / sq;
        }
        __syncthreads();
        // and the operand of the row solves of phase B: L_ij / L_jj below the
        // diagonal, 1 / L_jj on it
        for (int e = t; e < PT * PT; e += PTHREADS) {
            const int i = e >> 5, jj = e & 31;
            if (i > jj) {
                const double v = D[i * PLD + jj] * s_rinv[jj];
                D[i * PLD + jj] = v;
                sB[i * PLD + jj] = v * s_rinv[jj];
            }
        }
        __syncthreads();
        if (t < PT) {
            D[t * PLD + t] = s_sq[t];
            sB[t * PLD + t] = s_rinv[t];
        }
        __syncthreads();
    };
    // C item w of step p: half (w & 1) of the 16-row halves of trailing tile
    // number w >> 1 (row-major over the lower triangle of the tiles below p):
    // C(q, r) -= L(q, p) L(r, p)^T with the operands from their home CTAs
    auto c_item = [&](int w, int p) {
        const int tid = w >> 1, half = w & 1;
        int a, b;
        tile_of(tid, a, b);
        const int q = p + 1 + a, r = p + 1 + b;
        // the first 16 rows of a diagonal tile: only columns 0 .. 15 hold the
        // lower triangle (the strict upper part of a diagonal tile is never read)
        const bool narrow = a == b && half == 0;
        const double* Lq = tile_ptr(q, p);
        const double* Lr = tile_ptr(r, p);
        // the remote operands into registers before the first store (stores to
        // shared memory cannot be moved past loads through cluster-mapped
        // pointers, so a load-store loop waits for each remote load in turn)
        double vq[2], vr[4];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int e = t + k * PTHREADS;
            vq[k] = Lq[(16 * half + (e >> 5)) * PLD + (e & 31)];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = t + k * PTHREADS;
            if (k < 2 || !narrow) vr[k] = Lr[(e >> 5) * PLD + (e & 31)];
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int e = t + k * PTHREADS;
            sQ[(e >> 5) * PLD + (e & 31)] = vq[k];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = t + k * PTHREADS;
            if (k < 2 || !narrow) sR[(e >> 5) * PLD + (e & 31)] = vr[k];
        }
        __syncthreads();
        double* C = tile_ptr(q, r);
        // thread: row i (16) x columns l = (t & 15) + 16 c (2; 1 when narrow)
        const int i = t >> 4, l0 = t & 15;
        const int ci = 16 * half + i;
        if (narrow) {
            double acc0 = 0.0;
#pragma unroll 8
            for (int k = 0; k < PT; ++k) acc0 = fma(sQ[i * PLD + k], sR[l0 * PLD + k], acc0);
            C[ci * PLD + l0] -= acc0;
        } else {
            double acc0 = 0.0, acc1 = 0.0;
#pragma unroll 8
            for (int k = 0; k < PT; ++k) {
                const double lq = sQ[i * PLD + k];
                acc0 = fma(lq, sR[l0 * PLD + k], acc0);
                acc1 = fma(lq, sR[(l0 + 16) * PLD + k], acc1);
            }
            C[ci * PLD + l0] -= acc0;
            C[ci * PLD + l0 + 16] -= acc1;
        }
        __syncthreads();
    };
    __syncthreads();               // tiles, tables and s_fail seen by the whole CTA
    int fail = -1;
    if (me == 0) factor_diag(0);   // tile 0 lives in CTA 0
    cl.sync();
    {
        const int f = *cl.map_shared_rank(&s_fail, 0);
        if (f >= 0) fail = f;
    }
    for (int p = 0; p < NT && fail < 0; ++p) {
        const int below = NT - 1 - p;
        if (below == 0) break;
        // B: rows of the panel tiles below, x L_pp^T = a, one warp per row
        {
            const double* Dr = cl.map_shared_rank(sB, (p * (p + 1) / 2 + p) % CL);
            double vd[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int e = t + k * PTHREADS;
                vd[k] = Dr[(e >> 5) * PLD + (e & 31)];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int e = t + k * PTHREADS;
                sD[(e >> 5) * PLD + (e & 31)] = vd[k];
            }
            __syncthreads();
            // each unknown costs one FMA in the row's recurrence, not also a
            // multiplication on one lane (the FP64 pipe charges a warp
            // instruction whatever its active lanes), and the row is scaled at
            // the end: y_l -= y_j (L_lj / L_jj), x_l = y_l / L_ll
            const int rows = below * PT;
            if (rows > CL * PWARPS) {
                // more rows than warps: two rows per warp, one per half-warp,
                // lane h holding unknowns h and 16 + h; the terms of the lower
                // half's unknowns reach the upper half as each is found (one
                // chain of 32 steps for both rows, 48 FMA instructions instead
                // of 64; every unknown takes its terms in the same order)
                const int h = lane & 15, hs = lane & 16;
                for (int pr = me * PWARPS + warp; 2 * pr < rows; pr += CL * PWARPS) {
                    const int gr = 2 * pr + (lane >> 4);       // rows is even: gr < rows
                    double* X = tile_ptr(p + 1 + gr / PT, p) + (gr % PT) * PLD;
                    double ya = X[h], yb = X[16 + h];
                    for (int j = 0; j < 16; ++j) {
                        const double yj = __shfl_sync(0xffffffffu, ya, hs | j);
                        if (h > j) ya -= yj * sD[h * PLD + j];
                        yb -= yj * sD[(16 + h) * PLD + j];
                    }
                    for (int j = 0; j < 16; ++j) {
                        const double yj = __shfl_sync(0xffffffffu, yb, hs | j);
                        if (h > j) yb -= yj * sD[(16 + h) * PLD + 16 + j];
                    }
                    X[h] = ya * sD[h * PLD + h];
                    X[16 + h] = yb * sD[(16 + h) * PLD + 16 + h];
                }
            } else {
                for (int gr = me * PWARPS + warp; gr < rows; gr += CL * PWARPS) {
                    double* X = tile_ptr(p + 1 + gr / PT, p) + (gr % PT) * PLD;
                    double x = X[lane];
                    for (int j = 0; j < PT; ++j) {
                        const double yj = __shfl_sync(0xffffffffu, x, j);
                        if (lane > j) x -= yj * sD[lane * PLD + j];
                    }
                    X[lane] = x * sD[lane * PLD + lane];
                }
            }
        }
        cl.sync();
        // C with look-ahead: the home CTA of the next diagonal tile updates it
        // first (items 0 and 1) and factors it (A of step p + 1) while the
        // other CTAs share the rest of the trailing tiles (nothing else reads
        // or writes that tile in this step)
        {
            const int idn = (p + 1) * (p + 2) / 2 + p + 1, hn = idn % CL;
            const int nitem = below * (below + 1);           // tiles x 2 halves
            if (me == hn) {
                c_item(0, p);
                c_item(1, p);
                factor_diag(p + 1);
            } else {
                const int rk = (me - hn - 1 + CL) % CL;     // 0 .. CL - 2
                for (int w = 2 + rk; w < nitem; w += CL - 1) c_item(w, p);
            }
            cl.sync();
            const int f = *cl.map_shared_rank(&s_fail, hn);
            if (f >= 0) fail = (p + 1) * PT + f;
        }
    }
    // PD check inputs while the tiles are in shared memory: every CTA adds the
    // column sums of its tiles, part[(tile id) * PT + c] (rows past kb are
    // identity rows, not part of L: skipped); CTA 0 then adds them per
    // column in tile order
    const bool do_check = fail < 0 && check;
    __shared__ double s_part[PMAXT * (PMAXT + 1) / 2 * PT];   // rank 0: per-tile partials
    if (do_check) {
        for (int id = me; id < NTILE; id += CL) {
            int q, r;
            tile_of(id, q, r);
            const double* T = home + (id / CL) * TILE;
            double* dst = cl.map_shared_rank(s_part, 0) + id * PT;
            if (t < PT) {
                double sum = 0.0;
                const int c = t;
                for (int i = (q == r ? c : 0); i < PT && q * PT + i < kb; ++i) sum += T[i * PLD + c];
                dst[c] = sum;
            }
        }
    }
    cl.sync();
    if (do_check && me == 0) {
        for (int p = t; p < kb; p += PTHREADS) {
            const int r = p / PT, c = p % PT;
            double sum = 0.0;
            for (int q = r; q < NT; ++q) sum += s_part[(q * (q + 1) / 2 + r) * PT + c];
            s_cs[p] = sum;
        }
    }
    cl.sync();
    // y_j = sum_{p <= j} s_cs[p] L[j][p]: every CTA the rows of its tiles
    // (partials per tile, reusing s_part in rank 0), CTA 0 adds them per row
    if (do_check) {
        const double* cs0 = cl.map_shared_rank(s_cs, 0);
        for (int id = me; id < NTILE; id += CL) {
            int q, r;
            tile_of(id, q, r);
            const double* T = home + (id / CL) * TILE;
            for (int i = warp; i < PT; i += PWARPS) {
                double y = 0.0;
                const int c = lane;
                if (q * PT + i < kb && (q > r || c <= i)) y = cs0[r * PT + c] * T[i * PLD + c];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
                if (lane == 0) sD[id * PT + i] = y;   // sD, sQ, sR: free; gathered below
            }
        }
    }
    cl.sync();
    if (do_check && me == 0) {
        const double tau = st->tau;
        for (int j = t; j < kb; j += PTHREADS) {
            const int q = j / PT, i = j % PT;
            double y = 0.0;
            for (int r = 0; r <= q; ++r) {
                const int id = q * (q + 1) / 2 + r;
                y += cl.map_shared_rank(sD, id % CL)[id * PT + i];
            }
            const double d = y - cc[j];
            if (!(fabs(d) <= tau)) {
                atomicAdd(&st->detected, 1ull);
                atomicAdd(&st->uncorrectable, 1ull);
                record_event(st, step, EV_PD, K0 + j, K0 + j, d);
            }
        }
    }
    // write back (the strict upper triangle of A is left as it is)
    if (fail < 0) {
        for (int id = me; id < NTILE; id += CL) {
            int q, r;
            tile_of(id, q, r);
            const double* T = home + (id / CL) * TILE;
            for (int e = t; e < PT * PT; e += PTHREADS) {
                const int i = e >> 5, j = e & 31, gi = q * PT + i, gj = r * PT + j;
                if (gi < kb && gj < kb && (q > r || j <= i)) A[(int64_t)gi * lda + gj] = T[i * PLD + j];
            }
        }
    } else if (me == 0 && t == 0) {
        atomicCAS(&st->info, 0, (int)(K0 + fail + 1));
    }
    cl.sync();   // no CTA leaves while others may still read its shared memory
}

template <int CL>
cudaError_t launch_cl(double* A, int64_t lda, int kb, int64_t K0, const double* cc, int step,
                      int check, DevStatus* st, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, 1, 1);
    cfg.blockDim = dim3(PTHREADS, 1, 1);
    cfg.dynamicSmemBytes = pd_smem<CL>();
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_potrf_pd_cluster<CL>, A, lda, kb, K0, cc, step, check, st);
}

}  // namespace

// Cluster size: 16 CTAs where the device runs such clusters, else 8.
int pd_cluster_size() {
    static int size = 0;
    if (size) return size;
    size = 8;
    if (cudaFuncSetAttribute(k_potrf_pd_cluster<16>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                             1) == cudaSuccess &&
        cudaFuncSetAttribute(k_potrf_pd_cluster<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pd_smem<16>()) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16, 1, 1);
        cfg.blockDim = dim3(PTHREADS, 1, 1);
        cfg.dynamicSmemBytes = pd_smem<16>();
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 16;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_potrf_pd_cluster<16>, &cfg) == cudaSuccess &&
            nclusters > 0)
            size = 16;
    }
    cudaGetLastError();   // a refused non-portable size is not an error of the caller
    if (size == 8)
        cudaFuncSetAttribute(k_potrf_pd_cluster<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pd_smem<8>());
    return size;
}


cudaError_t launch_potrf_pd_cluster(double* A, int64_t lda, int64_t kb, int64_t K0,
                                    const double* cc, int step, int check, DevStatus* st,
                                    cudaStream_t s) {
    if (kb <= 0) return cudaSuccess;
    if (kb > PMAXT * PT) return cudaErrorInvalidValue;
    const cudaError_t e = pd_cluster_size() == 16
                              ? launch_cl<16>(A, lda, (int)kb, K0, cc, step, check, st, s)
                              : launch_cl<8>(A, lda, (int)kb, K0, cc, step, check, st, s);
    note_launch();
    return e;
}

}  // namespace abft
