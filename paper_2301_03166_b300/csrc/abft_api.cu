// abft_api.cu -- host side of the C ABI: argument checks, workspace layout
// and the per-iteration launch sequence of the blocked ABFT factorizations
// (Sec. 2.1 PD / PU / TMU per iteration; Sec. 3.1.2 encode, carry, verify,
// locate, correct).  No host synchronization happens inside the step loop;
// the only device-to-host copy is the final status when a report is wanted.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace abft {

// ------------------------------------------------ launch and time accounting
static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {
struct Mark {
    int phase;
    cudaEvent_t a, b;
    int64_t step;
};
struct Interval {
    int phase;
    int64_t step;
    double ms;
};
std::vector<Interval> g_intervals;    // timed intervals since the last enable, in order
thread_local int64_t g_step = -1;     // iteration the next marks belong to
std::mutex g_tmu;
bool g_timing = false;
std::vector<cudaEvent_t> g_pool;      // reusable events
size_t g_pool_used = 0;
std::vector<Mark> g_marks;            // marks of the current call
double g_ms[PH_COUNT] = {};
long long g_calls[PH_COUNT] = {};
cudaEvent_t next_event() {
    if (g_pool_used == g_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        g_pool.push_back(e);
    }
    return g_pool[g_pool_used++];
}
}  // namespace

bool timing_on() { return g_timing; }

void timing_step(int64_t k) { g_step = k; }

void timing_mark(int phase, int begin, cudaStream_t s) {
    if (!g_timing) return;
    std::lock_guard<std::mutex> lk(g_tmu);
    cudaEvent_t e = next_event();
    if (!e) return;
    cudaEventRecord(e, s);
    if (begin) {
        g_marks.push_back({phase, e, nullptr, g_step});
    } else {
        for (auto it = g_marks.rbegin(); it != g_marks.rend(); ++it)
            if (it->phase == phase && it->b == nullptr) { it->b = e; break; }
    }
}

cudaError_t timing_collect(cudaStream_t s) {
    if (!g_timing) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_tmu);
    for (const Mark& m : g_marks) {
        if (!m.b) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
            g_ms[m.phase] += ms;
            g_calls[m.phase] += 1;
            g_intervals.push_back({m.phase, m.step, (double)ms});
        }
    }
    g_marks.clear();
    g_pool_used = 0;
    return cudaSuccess;
}

}  // namespace abft

using namespace abft;

namespace {


constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Byte offsets of the pieces of a Cholesky workspace.
// Diagonal blocks wider than kPdChunk are factored in chunks with a split-K
// update between them (chol_pd).
constexpr int64_t kPdChunk = 256;
constexpr int kPdSplit = 8;

size_t pd_part_bytes(int64_t nb) {
    return nb > kPdChunk ? sizeof(double) * kPdSplit * (size_t)kPdChunk * kPdChunk : 0;
}

struct CholWs {
    size_t st, cs, cr, xr, v, save, lq, sig, tq, tq32, l32, ca, ra, ta32, pdpart, eslice, eex,
        pslice, pex, total;
    int64_t nc;   // checksum rows per tile-row in CS (0, 1 or 2)
    int64_t nt;
};

CholWs chol_ws(int64_t n, int64_t nb, int mode, bool mixed = false, bool emu = false) {
    CholWs w{};
    w.nt = (n + nb - 1) / nb;
    // column sums and weighted column sums of every block row, in both modes
    // (the panel is verified with the weighted sums)
    w.nc = mode == ABFT_MODE_NONE ? 0 : 2;
    size_t off = 0;
    w.st = off; off = align_up(off + sizeof(DevStatus));
    w.cs = off; off = align_up(off + sizeof(double) * (size_t)(w.nc * w.nt) * (size_t)n);
    w.cr = off; off = align_up(off + (mode == ABFT_MODE_FULL ? sizeof(double) * (size_t)n * (size_t)w.nt : 0));
    w.xr = off;
    w.v = off;
    w.save = off; off = align_up(off + sizeof(double) * (size_t)n * (size_t)nb);
    const int64_t ncq = w.nc > 0 ? w.nc : 1;
    w.lq = off; off = align_up(off + (mixed ? sizeof(uint16_t) * (size_t)n * (size_t)nb : 0));
    w.sig = off; off = align_up(off + (mixed ? sizeof(double) * (size_t)w.nt : 0));
    w.tq = off; off = align_up(off + (mixed ? sizeof(double) * (size_t)(ncq * w.nt) * (size_t)nb : 0));
    w.tq32 = off; off = align_up(off + (mixed ? sizeof(float) * (size_t)(ncq * w.nt) * (size_t)nb : 0));
    w.l32 = off; off = align_up(off + (mixed ? sizeof(float) * (size_t)nb * (size_t)nb : 0));
    // abs-checksums of the mixed form (thresholds per column / row) and the
    // panel tiles' sums 1^T |Lq_I| that carry them
    const bool absc = mixed && mode != ABFT_MODE_NONE;
    w.ca = off; off = align_up(off + (absc ? sizeof(float) * (size_t)w.nt * (size_t)n : 0));
    w.ra = off; off = align_up(off + (absc && mode == ABFT_MODE_FULL ? sizeof(float) * (size_t)n * (size_t)w.nt : 0));
    w.ta32 = off; off = align_up(off + (absc ? sizeof(float) * (size_t)w.nt * (size_t)nb : 0));
    w.pdpart = off; off = align_up(off + pd_part_bytes(nb));
    w.eslice = off; off = align_up(off + (emu ? emu_slice_bytes(n, nb) : 0));
    w.eex = off; off = align_up(off + (emu ? sizeof(int) * (size_t)emu_rows(n, nb) : 0));
    // the blocked panel solve's own slices (it runs beside the previous step's
    // update, which still reads eslice)
    w.pslice = off; off = align_up(off + (emu ? emu_slice_bytes(n, nb) : 0));
    w.pex = off; off = align_up(off + (emu ? sizeof(int) * (size_t)emu_rows(n, nb) : 0));
    w.total = off;
    return w;
}

bool chol_fault_ok(const abft_fault& f, int64_t n, int64_t nb, int64_t N) {
    if (f.step < 0 || f.step >= N - 1) return false;
    int64_t K0 = (int64_t)f.step * nb, T0 = std::min(K0 + nb, n);
    if (f.row < 0 || f.row >= n || f.col < 0 || f.col >= n) return false;
    if (f.kind == ABFT_FAULT_PANEL) return f.row >= T0 && f.col >= K0 && f.col < T0;
    if (f.kind < ABFT_FAULT_MEMORY || f.kind > ABFT_FAULT_PANEL) return false;
    return f.row >= T0 && f.col >= T0 && f.col / nb <= f.row / nb;
}

bool event_less(const abft_fault& a, const abft_fault& b) {
    if (a.step != b.step) return a.step < b.step;
    if (a.row != b.row) return a.row < b.row;
    if (a.col != b.col) return a.col < b.col;
    return a.kind < b.kind;
}

// Copy the device status into *rep (synchronizes the stream).
int finish_report(const DevStatus* dst, abft_report* rep, cudaStream_t s, bool lu = false) {
    DevStatus h;
    ABFT_CUDA_TRY(cudaMemcpyAsync(&h, dst, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    ABFT_CUDA_TRY(cudaStreamSynchronize(s));
    std::memset(rep, 0, sizeof(*rep));
    rep->detected = (int64_t)h.detected;
    rep->corrected = (int64_t)h.corrected;
    rep->uncorrectable = (int64_t)h.uncorrectable;
    rep->checksum_repaired = (int64_t)h.repaired;
    rep->nloc = std::min(h.nloc, (int)ABFT_MAX_LOC);
    rep->info = lu ? h.lu_info : h.info;
    for (int i = 0; i < rep->nloc; ++i) rep->loc[i] = h.loc[i];
    std::sort(rep->loc, rep->loc + rep->nloc, event_less);
    double r;
    std::memcpy(&r, &h.max_ratio_bits, sizeof(r));
    rep->max_ratio = r;
    rep->tau = h.tau;
    if (h.tau_coef > 0.0 && h.tau_max_bits != 0) {   // mixed form: largest per-column threshold
        double t;
        std::memcpy(&t, &h.tau_max_bits, sizeof(t));
        rep->tau = t;
    }
    if (h.error) return ABFT_ERR_TIMEOUT;
    if (rep->info) return rep->info;
    if (h.uncorrectable) return ABFT_ERR_UNCORRECTABLE;
    return ABFT_OK;
}

// Factor the kb x kb diagonal block at A (lower) and check it against the
// carried column checksum cc (check != 0): one cluster launch for kb <= 256;
// larger blocks in 256-column chunks (cluster factorization of the chunk,
// panel solve of the rows below it, split-K update of the rest of the block)
// followed by the separate check.  part: split-K scratch (pd_part_bytes).
cudaError_t chol_pd(double* A, int64_t lda, int64_t kb, int64_t K0, const double* cc, int check,
                    int step, double* part, DevStatus* st, cudaStream_t s) {
    if (kb <= kPdChunk) return launch_potrf_pd_cluster(A, lda, kb, K0, cc, step, check, st, s);
    for (int64_t c = 0; c < kb; c += kPdChunk) {
        const int64_t w = std::min(kPdChunk, kb - c);
        double* Lc = A + c * lda + c;
        cudaError_t e = launch_potrf_pd_cluster(Lc, lda, w, K0 + c, nullptr, step, 0, st, s);
        if (e != cudaSuccess) return e;
        const int64_t r = kb - c - w;
        if (r <= 0) continue;
        TrsmSeg seg{Lc + w * lda, lda, r};
        e = launch_trsm_rlt(Lc, lda, w, &seg, 1, nullptr, nullptr, st, s);
        if (e != cudaSuccess) return e;
        GemmSeg g{};
        g.A = Lc + w * lda; g.lda = lda;
        g.B = Lc + w * lda; g.ldb = lda;
        g.C = Lc + w * lda + w; g.ldc = lda;
        g.M = r; g.N = r; g.K = w;
        g.g = 64; g.row0 = 0; g.col0 = 0;
        e = launch_gemm_f64_splitk(g, 0, 0, kPdSplit, part, st, s);
        if (e != cudaSuccess) return e;
    }
    if (check) return launch_chol_pd_check(A, lda, kb, cc, K0, step, nullptr, MODE_FULL, st, s);
    return cudaSuccess;
}

// Side stream and events of the look-ahead, per device and calling thread.
struct LookAhead {
    int dev = -1;
    cudaStream_t side = nullptr;
    cudaEvent_t ready = nullptr, rest_done = nullptr;
};

cudaError_t lookahead_streams(LookAhead*& out) {
    thread_local LookAhead la[16];   // per thread: concurrent callers never share events
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 16) return cudaErrorInvalidDevice;
    LookAhead& l = la[dev];
    if (l.dev != dev) {
        e = cudaStreamCreateWithFlags(&l.side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&l.ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&l.rest_done, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
        l.dev = dev;
    }
    out = &l;
    return cudaSuccess;
}

std::atomic<int> g_lookahead{1};

// Blocked ABFT Cholesky step loop (Sec. 2.1 PD / PU / TMU; Sec. 3.1.2).
// modes (nullable, host, one entry per step): the checksum mode of each step
// (adaptive ABFT); nullptr runs every step in `mode`.  A step in mode NONE
// neither carries nor verifies checksums; the trailing block triangle is
// encoded afresh when checking starts again or moves from SINGLE to FULL.
//
// Look-ahead (Sec. 2.1, Fig. example-lu (b), on one GPU): with a uniform mode
// and at least two trailing block columns, the update of step k is split.  The
// next block column is updated and verified first; the factorization of the
// next diagonal block (PD of step k + 1) then runs on the caller's stream
// while the rest of the update and its verification run on a side stream
// (the persistent tensor-core updates leave the PD's SMs free), and the
// caller's stream waits for both before the next panel solve.  Every kernel
// does the same arithmetic either way, so the results are identical.
int chol_steps(int64_t n, int64_t nb, int32_t mode, const int32_t* modes, double* A, int64_t lda,
               const abft_fault* faults, int32_t nfaults, double tau_scale, const CholWs& w,
               char* base, cudaStream_t s, int32_t dtype) {
    const bool mixed = dtype == ABFT_MIXED_BF16 || dtype == ABFT_MIXED_F16;
    const bool emu = dtype == ABFT_F64_EMU;
    const int bf16 = dtype == ABFT_MIXED_BF16 ? 1 : 0;
    uint16_t* Lq = (uint16_t*)(base + w.lq);
    double* sig = (double*)(base + w.sig);
    double* tq = (double*)(base + w.tq);
    float* tq32 = (float*)(base + w.tq32);
    float* Ca = (float*)(base + w.ca);
    float* Ra = (float*)(base + w.ra);
    float* ta32 = (float*)(base + w.ta32);
    DevStatus* st = (DevStatus*)(base + w.st);
    double* CS = (double*)(base + w.cs);
    double* Cr = (double*)(base + w.cr);
    double* save = (double*)(base + w.save);
    const int64_t g = nb, nt = w.nt, nc = w.nc, N = nt;
    LookAhead* la = nullptr;
    if (modes == nullptr && g_lookahead.load() && n > 2 * nb) ABFT_CUDA_TRY(lookahead_streams(la));

    timing_mark(PH_OTHER, 1, s);
    ABFT_CUDA_TRY(launch_mirror_diag(A, lda, n, nb, save, 0, s));
    // mixed form: tau_scale * 4 * gamma_g(2^-24), the factor of the per-column
    // thresholds (the same expression and order as the oracle)
    double mcoef = 0.0;
    if (mixed) {
        const double gam = ((double)g * 0x1p-24) / (1.0 - (double)g * 0x1p-24);
        mcoef = tau_scale * 4.0;
        mcoef *= gam;
    }
    ABFT_CUDA_TRY(launch_tau_chol(A, lda, n, g, tau_scale, st, s, mixed ? 0x1p-24 : 0x1p-53, mcoef));
    // checksum tile sets (Sec. 3.1.2: per matrix block)
    TileSet base_ts{};
    base_ts.A = A; base_ts.lda = lda;
    base_ts.cc = CS; base_ts.cw = CS + n; base_ts.ccI = nc * n;
    base_ts.cr = Cr; base_ts.crs = nt; base_ts.crJ = 1;
    base_ts.g = g; base_ts.nrow_end = n; base_ts.ncol_end = n;
    base_ts.weighted = 1;
    timing_mark(PH_OTHER, 0, s);
    enum { PART_ALL = 0, PART_NEXT = 1, PART_REST = 2 };
    bool pd_ahead = false;   // PD of this step already run by the previous step's look-ahead
    // The previous step's rest of the update (side stream) writes only block
    // columns >= k + 1 of this step's trailing matrix (and their checksums), so
    // this step's PD and panel solve may run beside it; the caller's stream
    // joins it before the first operation that touches what it writes or reads
    // (the panel's slices or quantized copy, or the trailing update).
    bool rest_pending = false;
    auto join_rest = [&]() -> cudaError_t {
        if (!rest_pending) return cudaSuccess;
        rest_pending = false;
        return cudaStreamWaitEvent(s, la->rest_done, 0);
    };
    for (int64_t k = 0; k < N; ++k) {
        const int64_t K0 = k * g, kb = std::min(g, n - K0), T0 = K0 + kb, m = n - T0;
        double* Akk = A + K0 * lda + K0;
        timing_step(k);
        const int32_t mk = modes ? modes[k] : mode;
        const int32_t mprev = k == 0 ? ABFT_MODE_NONE : (modes ? modes[k - 1] : mode);
        const bool full = mk == ABFT_MODE_FULL, check = mk != ABFT_MODE_NONE;
        if (check && (mprev == ABFT_MODE_NONE || (full && mprev != ABFT_MODE_FULL))) {
            // (re-)encode the trailing block triangle (Sec. 3.1.2 encode)
            timing_mark(PH_OTHER, 1, s);
            TileSet ts = base_ts;
            ts.I0 = k; ts.I1 = nt; ts.J0 = k; ts.J1 = nt; ts.lower = 1;
            ABFT_CUDA_TRY(launch_encode(ts, mk, s));
            if (mixed) {   // abs-checksums start at zero with the encoded checksums
                ABFT_CUDA_TRY(cudaMemsetAsync(Ca, 0, sizeof(float) * (size_t)nt * (size_t)n, s));
                if (full)
                    ABFT_CUDA_TRY(cudaMemsetAsync(Ra, 0, sizeof(float) * (size_t)n * (size_t)nt, s));
            }
            timing_mark(PH_OTHER, 0, s);
        }
        // PD and its checksum check
        if (!pd_ahead) {
            timing_mark(PH_PD, 1, s);
            ABFT_CUDA_TRY(chol_pd(Akk, lda, kb, K0, check ? CS + (k * nc) * n + K0 : nullptr,
                                  check ? 1 : 0, (int)k, (double*)(base + w.pdpart), st, s));
            timing_mark(PH_PD, 0, s);
        }
        pd_ahead = false;
        if (m <= 0) {
            ABFT_CUDA_TRY(join_rest());
            break;
        }
        // PU: panel rows and the carried checksum rows through X L_kk^T = B
        timing_mark(PH_PU, 1, s);
        if (emu && kb % 64 == 0 && kb >= 128) {
            // blocked by 64 columns: X_c L_cc^T = B_c - X_<c L_c,<c^T.  The 64-wide
            // diagonal solves run one thread per row (k_trsm_rows); the products
            // run FP64-accurate from BF16 slices on the tensor cores (the panel rows, the checksum rows and the
            // rows L_c,<c re-sliced with one scale per row over the columns < c)
            constexpr int64_t CW = 64;
            uint16_t* Sl = (uint16_t*)(base + w.pslice);
            int* ex = (int*)(base + w.pex);
            const int64_t mcp = check ? (nt - k - 1) * nc : 0, mrows = m + mcp;
            double* Xp = A + T0 * lda + K0;
            double* Xc = CS + ((k + 1) * nc) * n + K0;
            for (int64_t c = 0; c < kb / CW; ++c) {
                if (c > 0) {
                    const int64_t K = c * CW, Mt = mrows + CW;
                    ABFT_CUDA_TRY(launch_slice_panel(Xp, lda, m, K, Sl, Mt, 0, ex, s));
                    if (check) ABFT_CUDA_TRY(launch_slice_panel(Xc, n, mcp, K, Sl, Mt, m, ex, s));
                    ABFT_CUDA_TRY(launch_slice_panel(Akk + c * CW * lda, lda, CW, K, Sl, Mt, mrows,
                                                     ex, s));
                    EmuRectHost rc[2] = {};
                    rc[0].C = Xp + c * CW; rc[0].ldc = lda;
                    rc[0].a0 = 0; rc[0].na = m; rc[0].b0 = mrows; rc[0].nb = CW; rc[0].cdiv = 1;
                    rc[0].frow = -1;
                    rc[1].C = Xc + c * CW; rc[1].ldc = n;
                    rc[1].a0 = m; rc[1].na = mcp; rc[1].b0 = mrows; rc[1].nb = CW; rc[1].cdiv = 1;
                    rc[1].frow = -1;
                    ABFT_CUDA_TRY(launch_tmu_emu(Sl, ex, Mt, K, nullptr, 0, 0, 0, 128, rc,
                                                 check ? 2 : 1, nullptr, 0, 0, st, s));
                }
                TrsmSeg sg[2] = {{Xp + c * CW, lda, m}, {Xc + c * CW, n, mcp}};
                ABFT_CUDA_TRY(launch_trsm_rows(Akk + c * CW * lda + c * CW, lda, CW, sg,
                                               check ? 2 : 1, st, s, false));
            }
        } else {
            TrsmSeg segs[2] = {{A + T0 * lda + K0, lda, m},
                               {CS + ((k + 1) * nc) * n + K0, n, (nt - k - 1) * nc}};
            float* l32 = mixed ? (float*)(base + w.l32) : nullptr;
            if (mixed) ABFT_CUDA_TRY(launch_l_to_f32(Akk, lda, kb, l32, s));
            ABFT_CUDA_TRY(launch_trsm_rlt(Akk, lda, kb, segs, check ? 2 : 1, nullptr, nullptr, st,
                                          s, mixed, false, l32));
        }
        for (int f = 0; f < nfaults; ++f)
            if (faults[f].step == k && faults[f].kind == ABFT_FAULT_PANEL)
                ABFT_CUDA_TRY(launch_inject(A, lda, n, g, faults[f], s));
        if (check) {   // panel tiles: weighted column checksums locate 0D and row errors
            TileSet ts = base_ts;
            ts.I0 = k + 1; ts.I1 = nt; ts.J0 = k; ts.J1 = k + 1; ts.lower = 0;
            ts.ncol_end = T0;
            ABFT_CUDA_TRY(launch_verify(ts, MODE_SINGLE, (int)k, st, s));
        }
        timing_mark(PH_PU, 0, s);
        ABFT_CUDA_TRY(join_rest());

        // TMU of part p: PART_ALL the lower block triangle of the trailing
        // matrix, PART_NEXT its first block column (w columns), PART_REST the
        // triangle after it; each with its share of the checksum borders.
        const bool split = la != nullptr && m > g;
        const int64_t w1 = std::min(g, m);
        const int64_t mc = check ? (nt - k - 1) * nc : 0;
        // SMs kept from the persistent rest-of-update kernel for the caller's
        // stream: the PD cluster, and for the FP64-accurate form 16 more for
        // its blocked panel solve (measured at n = 16384: 101.8 -> 100.7 ms;
        // the 16-bit forms are fastest with the cluster alone)
        const int reserve = split ? (emu ? pd_cluster_size() + 16 : pd_cluster_size()) : 0;
        ComputeFault cfall[MAX_CF];
        int ncfall = 0;
        for (int f = 0; f < nfaults && ncfall < MAX_CF; ++f)
            if (faults[f].step == k && faults[f].kind == ABFT_FAULT_COMPUTE)
                cfall[ncfall++] = {faults[f].row - T0, faults[f].col - T0, faults[f].delta};
        if (emu) {   // the panel and checksum rows are sliced once for both parts
            timing_mark(PH_TMU, 1, s);
            ABFT_CUDA_TRY(launch_slice_panel(A + T0 * lda + K0, lda, m, kb, (uint16_t*)(base + w.eslice),
                                             m + mc, 0, (int*)(base + w.eex), s));
            if (check)
                ABFT_CUDA_TRY(launch_slice_panel(CS + ((k + 1) * nc) * n + K0, n, mc, kb,
                                                 (uint16_t*)(base + w.eslice), m + mc, m,
                                                 (int*)(base + w.eex), s));
            timing_mark(PH_TMU, 0, s);
        } else if (mixed) {
            timing_mark(PH_TMU, 1, s);
            const int64_t ncq = nc > 0 ? nc : 1;
            ABFT_CUDA_TRY(launch_quant_panel(A + K0, lda, T0, n, kb, g, k + 1, nt, bf16, Lq, sig, tq,
                                             ncq * kb, check ? 1 : 0, s, tq32,
                                             check ? ta32 : nullptr));
            timing_mark(PH_TMU, 0, s);
        }
        auto tmu = [&](int part, cudaStream_t ss) -> int {
            // columns [c0, c1) of the trailing matrix, block-column range [J0, J1)
            const int64_t c0 = part == PART_REST ? w1 : 0, c1 = part == PART_NEXT ? w1 : m;
            const int64_t J0 = k + 1 + (part == PART_REST ? 1 : 0);
            const int64_t J1 = part == PART_NEXT ? k + 2 : nt;
            const int maxg = part == PART_REST ? std::max(1, num_sms() - reserve) : 0;
            timing_mark(PH_TMU, 1, ss);
            if (emu) {
                // FP64-accurate TMU from exact BF16 slice products; the checksum
                // rows sit behind the panel rows in the slice tensor
                const uint16_t* Sl = (const uint16_t*)(base + w.eslice);
                const int* ex = (const int*)(base + w.eex);
                EmuRectHost rc[3] = {};
                int nr = 0;
                int64_t tri_m = 0, tri_o = 0;
                if (part == PART_NEXT) {
                    EmuRectHost& r = rc[nr++];
                    r.C = A + T0 * lda + T0; r.ldc = lda;
                    r.a0 = 0; r.na = m; r.b0 = 0; r.nb = w1; r.cdiv = 1; r.frow = 0; r.fcol = 0;
                } else {
                    tri_m = m;
                    tri_o = c0;
                }
                if (check) {   // border rows: c_I -= s_I L_J^T (and the weighted rows)
                    EmuRectHost& r = rc[nr++];
                    r.C = CS + ((k + 1) * nc) * n + T0 + c0; r.ldc = n;
                    r.a0 = m; r.na = mc; r.b0 = c0; r.nb = c1 - c0; r.cdiv = 1; r.frow = -1;
                }
                if (full) {    // border columns: r_I -= L_I s_J^T (plain checksum rows)
                    EmuRectHost& r = rc[nr++];
                    r.C = Cr + T0 * nt + J0; r.ldc = nt;
                    r.a0 = 0; r.na = m; r.b0 = m + (J0 - k - 1) * nc; r.nb = (J1 - J0) * nc;
                    r.cdiv = (int)nc; r.frow = -1;
                }
                ABFT_CUDA_TRY(launch_tmu_emu(Sl, ex, m + mc, kb, A + T0 * lda + T0, lda, tri_m,
                                             tri_o, g, rc, nr, cfall, ncfall, maxg, st, ss));
            } else if (mixed) {
                // TMU on the tensor cores: quantized panel, FP32 accumulation, FP64 C
                const int64_t ncq = nc > 0 ? nc : 1;
                ABFT_CUDA_TRY(launch_tmu_mixed(Lq, m, kb, bf16, A + T0 * lda + T0, lda, g, T0, sig,
                                               cfall, ncfall, st, ss, part == PART_REST ? w1 : 0,
                                               part == PART_NEXT ? 1 : 0, maxg));
                if (check) {
                    // checksum borders from the same quantized panel (one product
                    // per panel row and checksum vector, written to both borders)
                    BorderSymHost bh{};
                    bh.Lq = Lq; bh.m = m; bh.K = kb; bh.bf16 = bf16;
                    bh.tq = tq32; bh.ta = ta32; bh.nc = (int)ncq; bh.Jb = k + 1; bh.Je = nt;
                    bh.CS = CS; bh.Ca = Ca; bh.ldcs = n; bh.T0 = T0;
                    bh.Cr = full ? Cr : nullptr; bh.Ra = full ? Ra : nullptr; bh.ldr = nt;
                    bh.c0 = c0; bh.c1 = c1; bh.J0 = J0; bh.J1 = J1;
                    bh.g = g; bh.sig = sig;
                    ABFT_CUDA_TRY(launch_border_sym(bh, st, ss));
                }
            } else {
                // TMU with the checksum borders folded into the same launch
                GemmSeg gs[3] = {};
                ComputeFault cf[MAX_CF];
                int ncf = 0;
                if (part == PART_NEXT) {   // the next block column, no mask
                    gs[0].A = A + T0 * lda + K0; gs[0].lda = lda;
                    gs[0].B = A + T0 * lda + K0; gs[0].ldb = lda;
                    gs[0].C = A + T0 * lda + T0; gs[0].ldc = lda;
                    gs[0].M = m; gs[0].N = w1; gs[0].K = kb;
                } else {                   // the lower block triangle from column c0
                    gs[0].A = A + (T0 + c0) * lda + K0; gs[0].lda = lda;
                    gs[0].B = A + (T0 + c0) * lda + K0; gs[0].ldb = lda;
                    gs[0].C = A + (T0 + c0) * lda + T0 + c0; gs[0].ldc = lda;
                    gs[0].M = m - c0; gs[0].N = m - c0; gs[0].K = kb;
                    gs[0].g = g; gs[0].row0 = T0 + c0; gs[0].col0 = T0 + c0;
                }
                for (int f = 0; f < ncfall; ++f)   // faults in segment 0 coordinates
                    cf[ncf++] = {cfall[f].row - c0, cfall[f].col - c0, cfall[f].delta};
                int nseg = 1;
                if (check) {  // border rows: c_I -= s_I L_J^T (and the weighted rows)
                    GemmSeg& b = gs[nseg++];
                    b.A = CS + ((k + 1) * nc) * n + K0; b.lda = n;
                    b.B = A + (T0 + c0) * lda + K0; b.ldb = lda;
                    b.C = CS + ((k + 1) * nc) * n + T0 + c0; b.ldc = n;
                    b.M = (nt - k - 1) * nc; b.N = c1 - c0; b.K = kb;
                }
                if (full) {   // border columns: r_I -= L_I s_J^T
                    GemmSeg& b = gs[nseg++];
                    b.A = A + T0 * lda + K0; b.lda = lda;
                    b.B = CS + (J0 * nc) * n + K0; b.ldb = nc * n;
                    b.C = Cr + T0 * nt + J0; b.ldc = nt;
                    b.M = m; b.N = J1 - J0; b.K = kb;
                }
                ABFT_CUDA_TRY(launch_gemm_f64(gs, nseg, 0, 0, cf, ncf, st, ss));
            }
            timing_mark(PH_TMU, 0, ss);
            // storage errors of this step in these columns, then the verification
            timing_mark(PH_VERIFY, 1, ss);
            for (int f = 0; f < nfaults; ++f)
                if (faults[f].step == k && (faults[f].kind == ABFT_FAULT_MEMORY ||
                                            faults[f].kind == ABFT_FAULT_ROW1D ||
                                            faults[f].kind == ABFT_FAULT_COL1D) &&
                    faults[f].col - T0 >= c0 && faults[f].col - T0 < c1)
                    ABFT_CUDA_TRY(launch_inject(A, lda, n, g, faults[f], ss));
            if (check) {
                TileSet ts = base_ts;
                ts.I0 = J0; ts.I1 = nt; ts.J0 = J0; ts.J1 = J1; ts.lower = part == PART_NEXT ? 0 : 1;
                if (mixed) {   // per-column / per-row thresholds from the abs-checksums
                    ts.ca = Ca; ts.caI = n;
                    ts.ra = full ? Ra : nullptr;
                }
                ABFT_CUDA_TRY(launch_verify(ts, mk, (int)k, st, ss));
            }
            timing_mark(PH_VERIFY, 0, ss);
            return ABFT_OK;
        };
        if (!split) {
            const int rc = tmu(PART_ALL, s);
            if (rc != ABFT_OK) return rc;
        } else {
            int rc = tmu(PART_NEXT, s);
            if (rc != ABFT_OK) return rc;
            // the rest of the update on the side stream; PD of step k + 1 next on
            // the caller's stream, so that the cluster PD is dispatched first and
            // the capped persistent grid of the update fills the other SMs
            ABFT_CUDA_TRY(cudaEventRecord(la->ready, s));
            ABFT_CUDA_TRY(cudaStreamWaitEvent(la->side, la->ready, 0));
            const int64_t K1 = T0, kb1 = std::min(g, n - K1);
            timing_step(k + 1);
            timing_mark(PH_PD, 1, s);
            ABFT_CUDA_TRY(chol_pd(A + K1 * lda + K1, lda, kb1, K1,
                                  check ? CS + ((k + 1) * nc) * n + K1 : nullptr, check ? 1 : 0,
                                  (int)(k + 1), (double*)(base + w.pdpart), st, s));
            timing_mark(PH_PD, 0, s);
            timing_step(k);
            rc = tmu(PART_REST, la->side);
            if (rc != ABFT_OK) return rc;
            ABFT_CUDA_TRY(cudaEventRecord(la->rest_done, la->side));
            rest_pending = true;
            pd_ahead = true;
        }
    }
    timing_step(-1);
    timing_mark(PH_OTHER, 1, s);
    ABFT_CUDA_TRY(launch_mirror_diag(A, lda, n, nb, save, 1, s));
    timing_mark(PH_OTHER, 0, s);
    return ABFT_OK;
}

// ------------------------------------------------------------------ LU
struct LuWs {
    size_t st, cs, cr, colchk, colchkw, ptot, part, z, zw, pv, pi, stage, eslice, eex, total;
    int64_t nc, nt;
};

// rows of the LU's slice tensor: L21, the checksum panel rows, the columns of
// U12 and the row-checksum columns
int64_t lu_emu_rows(int64_t n, int64_t nt) { return 2 * n + 3 * nt; }

LuWs lu_ws(int64_t n, int64_t nb, int mode, bool emu = false) {
    LuWs w{};
    w.nt = (n + nb - 1) / nb;
    w.nc = mode == ABFT_MODE_FULL ? 1 : (mode == ABFT_MODE_SINGLE ? 2 : 0);
    const size_t d = sizeof(double);
    size_t off = 0;
    w.st = off; off = align_up(off + sizeof(DevStatus));
    w.cs = off; off = align_up(off + d * (size_t)(w.nc * w.nt) * (size_t)n);
    w.cr = off; off = align_up(off + (mode == ABFT_MODE_FULL ? d * (size_t)n * (size_t)w.nt : 0));
    w.colchk = off; off = align_up(off + d * (size_t)n);
    w.colchkw = off; off = align_up(off + d * (size_t)n);
    w.ptot = off; off = align_up(off + d * (size_t)nb);
    w.part = off; off = align_up(off + d * (size_t)w.nt * (size_t)nb);
    w.z = off; off = align_up(off + d * (size_t)nb);
    w.zw = off; off = align_up(off + d * (size_t)nb);
    w.pv = off; off = align_up(off + d * 1024);
    w.pi = off; off = align_up(off + sizeof(int64_t) * 1024);
    w.stage = off; off = align_up(off + getf2_stage_bytes(nb));
    const int64_t er = emu ? lu_emu_rows(n, w.nt) : 0;
    w.eslice = off; off = align_up(off + sizeof(uint16_t) * 8 * (size_t)er * (size_t)nb);
    w.eex = off; off = align_up(off + sizeof(int) * (size_t)er);
    w.total = off;
    return w;
}

bool lu_fault_ok(const abft_fault& f, int64_t n, int64_t nb, int64_t N) {
    if (f.step < 0 || f.step >= N - 1) return false;
    int64_t K0 = (int64_t)f.step * nb, T0 = std::min(K0 + nb, n);
    if (f.row < 0 || f.row >= n || f.col < 0 || f.col >= n) return false;
    if (f.kind == ABFT_FAULT_PANEL) return f.row >= K0 && f.row < T0 && f.col >= T0;
    if (f.kind < ABFT_FAULT_MEMORY || f.kind > ABFT_FAULT_PANEL) return false;
    return f.row >= T0 && f.col >= T0;
}

// Blocked ABFT LU step loop (Sec. 2.1 PD / PU / TMU; Sec. 3.1.2).
int lu_steps(int64_t n, int64_t nb, int32_t mode, double* A, int64_t lda, int64_t* ipiv,
             const abft_fault* faults, int32_t nfaults, double tau_scale, const LuWs& w,
             char* base, cudaStream_t s, bool emu = false) {
    DevStatus* st = (DevStatus*)(base + w.st);
    double* CS = (double*)(base + w.cs);
    double* Cr = (double*)(base + w.cr);
    double* colchk = (double*)(base + w.colchk);
    double* colchkw = (double*)(base + w.colchkw);
    double* ptot = (double*)(base + w.ptot);
    double* part = (double*)(base + w.part);
    double* z = (double*)(base + w.z);
    double* zw = (double*)(base + w.zw);
    double* pv = (double*)(base + w.pv);
    int64_t* pi = (int64_t*)(base + w.pi);
    const int64_t g = nb, nt = w.nt, nc = w.nc, N = nt;
    const bool full = mode == ABFT_MODE_FULL, check = mode != ABFT_MODE_NONE;

    TileSet base_ts{};
    base_ts.A = A; base_ts.lda = lda;
    base_ts.cc = CS; base_ts.cw = CS + n; base_ts.ccI = nc * n;
    base_ts.cr = Cr; base_ts.crs = nt; base_ts.crJ = 1;
    base_ts.g = g; base_ts.nrow_end = n; base_ts.ncol_end = n;
    timing_mark(PH_OTHER, 1, s);
    if (check) {
        ABFT_CUDA_TRY(launch_absmax(A, lda, n, n, &st->amax, s));
        TileSet ts = base_ts;
        ts.I0 = 0; ts.I1 = nt; ts.J0 = 0; ts.J1 = nt; ts.lower = 0;
        ABFT_CUDA_TRY(launch_encode(ts, mode, s));
    }
    timing_mark(PH_OTHER, 0, s);
    for (int64_t k = 0; k < N; ++k) {
        const int64_t K0 = k * g, kb = std::min(g, n - K0), T0 = K0 + kb, m = n - T0;
        double* P = A + K0 * lda + K0;
        timing_mark(PH_PD, 1, s);
        if (check) ABFT_CUDA_TRY(launch_coltot(CS, n, nc, k, nt, K0, kb, ptot, s));
        ABFT_CUDA_TRY(launch_getf2_coop(P, lda, n - K0, kb, K0, ipiv, st, pv, pi,
                                        (double*)(base + w.stage), s));
        ABFT_CUDA_TRY(launch_laswp(A, lda, n, K0, kb, ipiv, CS, n, nc, g, Cr, nt, mode, s));
        if (check) {
            ABFT_CUDA_TRY(launch_lu_colsums(P, lda, n - K0, kb, g, k, nt, K0, CS, n, nc, mode,
                                            part, nb, s));
            ABFT_CUDA_TRY(launch_lu_pd_check(P, lda, kb, ptot, part, nb, (int)(nt - k), (int)k,
                                             K0, n, g, tau_scale, z, zw, mode, st, s));
        }
        timing_mark(PH_PD, 0, s);
        if (m <= 0) break;
        // PU: U = L_kk^{-1} A_kJ with the row-checksum columns t_J = L_kk^{-1} r_kJ folded in
        timing_mark(PH_PU, 1, s);
        if (emu && kb % 64 == 0 && kb >= 128 && m >= 64) {
            // blocked by 64 rows: U_b = L_bb^{-1} (A_b - L_b,<b U_<b).  The products
            // run FP64-accurate from BF16 slices on the tensor cores (rows of
            // L_b,<b; columns of U_<b and of its row-checksum columns), the 64-wide
            // unit-lower solves in FP64; the predicted column sums z^T A_kJ are
            // formed first, from A_kJ as it stands
            constexpr int64_t RW = 64;
            uint16_t* Sl = (uint16_t*)(base + w.eslice);
            int* ex = (int*)(base + w.eex);
            double* U = A + K0 * lda + T0;
            const int64_t q = full ? nt - k - 1 : 0;
            double* Ucr = full ? Cr + K0 * nt + (k + 1) : nullptr;
            if (check)
                ABFT_CUDA_TRY(launch_trsm_llu(P, lda, kb, U, lda, m, nullptr, 0, 0, z, zw,
                                              colchk + T0,
                                              mode == ABFT_MODE_SINGLE ? colchkw + T0 : nullptr,
                                              s, true));
            for (int64_t b = 0; b < kb / RW; ++b) {
                if (b > 0) {
                    const int64_t K = b * RW, Mt = RW + m + q;
                    ABFT_CUDA_TRY(launch_slice_panel(P + b * RW * lda, lda, RW, K, Sl, Mt, 0, ex, s));
                    ABFT_CUDA_TRY(launch_slice_cols(U, lda, K, m, Sl, Mt, RW, ex, s));
                    if (full) ABFT_CUDA_TRY(launch_slice_cols(Ucr, nt, K, q, Sl, Mt, RW + m, ex, s));
                    EmuRectHost rc[2] = {};
                    rc[0].C = U + b * RW * lda; rc[0].ldc = lda;
                    rc[0].a0 = 0; rc[0].na = RW; rc[0].b0 = RW; rc[0].nb = m; rc[0].cdiv = 1;
                    rc[0].frow = -1;
                    if (full) {
                        rc[1].C = Ucr + b * RW * nt; rc[1].ldc = nt;
                        rc[1].a0 = 0; rc[1].na = RW; rc[1].b0 = RW + m; rc[1].nb = q;
                        rc[1].cdiv = 1; rc[1].frow = -1;
                    }
                    ABFT_CUDA_TRY(launch_tmu_emu(Sl, ex, Mt, K, nullptr, 0, 0, 0, 128, rc,
                                                 full && q > 0 ? 2 : 1, nullptr, 0, 0, st, s));
                }
                ABFT_CUDA_TRY(launch_trsm_llu(P + b * RW * (lda + 1), lda, RW, U + b * RW * lda,
                                              lda, m, full ? Ucr + b * RW * nt : nullptr, nt, q,
                                              nullptr, nullptr, nullptr, nullptr, s));
            }
        } else {
            ABFT_CUDA_TRY(launch_trsm_llu(P, lda, kb, A + K0 * lda + T0, lda, m,
                                          full ? Cr + K0 * nt + (k + 1) : nullptr, nt, nt - k - 1,
                                          check ? z : nullptr, zw, colchk + T0,
                                          mode == ABFT_MODE_SINGLE ? colchkw + T0 : nullptr, s));
        }
        for (int f = 0; f < nfaults; ++f)
            if (faults[f].step == k && faults[f].kind == ABFT_FAULT_PANEL)
                ABFT_CUDA_TRY(launch_inject(A, lda, n, g, faults[f], s));
        if (check) {
            TileSet ts = base_ts;
            ts.cc = colchk; ts.cw = colchkw; ts.ccI = 0;
            ts.I0 = k; ts.I1 = k + 1; ts.J0 = k + 1; ts.J1 = nt; ts.lower = 0;
            ts.nrow_end = T0;
            ABFT_CUDA_TRY(launch_verify(ts, mode, (int)k, st, s));
            ABFT_CUDA_TRY(launch_absmax(A + K0 * lda + T0, lda, kb, m, &st->umax, s));
        }
        timing_mark(PH_PU, 0, s);
        // TMU: A22 -= L21 U12 with the checksum borders
        GemmSeg gs[3] = {};
        gs[0].A = A + T0 * lda + K0; gs[0].lda = lda;
        gs[0].B = A + K0 * lda + T0; gs[0].ldb = lda;
        gs[0].C = A + T0 * lda + T0; gs[0].ldc = lda;
        gs[0].M = m; gs[0].N = m; gs[0].K = kb;
        int nseg = 1;
        if (check) {   // c_I -= (1^T L_Ik) U_kJ (and weighted)
            GemmSeg& b = gs[nseg++];
            b.A = CS + ((k + 1) * nc) * n + K0; b.lda = n;
            b.B = A + K0 * lda + T0; b.ldb = lda;
            b.C = CS + ((k + 1) * nc) * n + T0; b.ldc = n;
            b.M = (nt - k - 1) * nc; b.N = m; b.K = kb;
        }
        if (full) {    // r_I -= L_Ik t_J
            GemmSeg& b = gs[nseg++];
            b.A = A + T0 * lda + K0; b.lda = lda;
            b.B = Cr + K0 * nt + (k + 1); b.ldb = nt;
            b.C = Cr + T0 * nt + (k + 1); b.ldc = nt;
            b.M = m; b.N = nt - k - 1; b.K = kb;
        }
        ComputeFault cf[MAX_CF];
        int ncf = 0;
        for (int f = 0; f < nfaults && ncf < MAX_CF; ++f)
            if (faults[f].step == k && faults[f].kind == ABFT_FAULT_COMPUTE)
                cf[ncf++] = {faults[f].row - T0, faults[f].col - T0, faults[f].delta};
        timing_mark(PH_TMU, 1, s);
        if (emu) {
            // FP64-accurate TMU from exact BF16 slice products (as the Cholesky's):
            // slice tensor rows [L21 | checksum panel rows | columns of U12 |
            // row-checksum columns t_J], the update and both borders as rectangles
            uint16_t* Sl = (uint16_t*)(base + w.eslice);
            int* ex = (int*)(base + w.eex);
            const int64_t mc = check ? (nt - k - 1) * nc : 0, q = full ? nt - k - 1 : 0;
            const int64_t mt = 2 * m + mc + q;
            ABFT_CUDA_TRY(launch_slice_panel(A + T0 * lda + K0, lda, m, kb, Sl, mt, 0, ex, s));
            if (check)
                ABFT_CUDA_TRY(launch_slice_panel(CS + ((k + 1) * nc) * n + K0, n, mc, kb, Sl, mt, m,
                                                 ex, s));
            ABFT_CUDA_TRY(launch_slice_cols(A + K0 * lda + T0, lda, kb, m, Sl, mt, m + mc, ex, s));
            if (full)
                ABFT_CUDA_TRY(launch_slice_cols(Cr + K0 * nt + (k + 1), nt, kb, q, Sl, mt,
                                                2 * m + mc, ex, s));
            EmuRectHost rc[3] = {};
            int nr = 0;
            {
                EmuRectHost& r = rc[nr++];
                r.C = A + T0 * lda + T0; r.ldc = lda;
                r.a0 = 0; r.na = m; r.b0 = m + mc; r.nb = m; r.cdiv = 1; r.frow = 0; r.fcol = 0;
            }
            if (check) {
                EmuRectHost& r = rc[nr++];
                r.C = CS + ((k + 1) * nc) * n + T0; r.ldc = n;
                r.a0 = m; r.na = mc; r.b0 = m + mc; r.nb = m; r.cdiv = 1; r.frow = -1;
            }
            if (full) {
                EmuRectHost& r = rc[nr++];
                r.C = Cr + T0 * nt + (k + 1); r.ldc = nt;
                r.a0 = 0; r.na = m; r.b0 = 2 * m + mc; r.nb = q; r.cdiv = 1; r.frow = -1;
            }
            ABFT_CUDA_TRY(launch_tmu_emu(Sl, ex, mt, kb, nullptr, 0, 0, 0, 128, rc, nr, cf, ncf, 0,
                                         st, s));
        } else {
            ABFT_CUDA_TRY(launch_gemm_f64(gs, nseg, 0, 1, cf, ncf, st, s));
        }
        timing_mark(PH_TMU, 0, s);
        timing_mark(PH_VERIFY, 1, s);
        for (int f = 0; f < nfaults; ++f)
            if (faults[f].step == k && (faults[f].kind == ABFT_FAULT_MEMORY ||
                                        faults[f].kind == ABFT_FAULT_ROW1D ||
                                        faults[f].kind == ABFT_FAULT_COL1D))
                ABFT_CUDA_TRY(launch_inject(A, lda, n, g, faults[f], s));
        if (check) {
            TileSet ts = base_ts;
            ts.I0 = k + 1; ts.I1 = nt; ts.J0 = k + 1; ts.J1 = nt; ts.lower = 0;
            ABFT_CUDA_TRY(launch_verify(ts, mode, (int)k, st, s));
        }
        timing_mark(PH_VERIFY, 0, s);
    }
    return ABFT_OK;
}

int check_common(int64_t n, int64_t nb, int32_t dtype, int32_t mode, const void* A, int64_t lda,
                 const abft_fault* faults, int32_t nfaults, double tau_scale, const void* ws,
                 size_t* ws_bytes, bool allow_emu = false) {
    if (n < 0) return -1;
    if (nb <= 0 || nb % 32 != 0 || nb > 512) return -2;
    const bool emu_ok = allow_emu && dtype == ABFT_F64_EMU && nb <= 256;
    if (dtype != ABFT_F64 && !emu_ok) return dtype < 0 || dtype > 4 ? -3 : ABFT_ERR_UNSUPPORTED;
    if (mode < ABFT_MODE_NONE || mode > ABFT_MODE_FULL) return -4;
    if (n > 0 && A == nullptr && ws != nullptr) return -5;
    if (lda < std::max<int64_t>(1, n)) return -6;
    if (nfaults < 0) return -9;
    if (nfaults > 0 && faults == nullptr) return -8;
    if (!(tau_scale > 0.0)) return -10;
    if (ws_bytes == nullptr) return -13;
    for (int f = 0; f < nfaults; ++f) {
        int same = 0;
        for (int h = 0; h < nfaults; ++h)
            same += faults[h].kind == ABFT_FAULT_COMPUTE && faults[h].step == faults[f].step;
        if (same > MAX_CF) return -8;
    }
    return ABFT_OK;
}

}  // namespace

extern "C" {

int abft_getrf(int64_t n, int64_t nb, int32_t dtype, int32_t mode, double* A, int64_t lda,
               int64_t* ipiv, const abft_fault* faults, int32_t nfaults, double tau_scale,
               abft_report* rep, void* ws, size_t* ws_bytes, void* stream) {
    int rc = check_common(n, nb, dtype, mode, A, lda, faults, nfaults, tau_scale, ws, ws_bytes,
                          true);
    if (rc != ABFT_OK) return rc;
    if (n > 0 && ipiv == nullptr && ws != nullptr) return -7;
    const int64_t N = (n + nb - 1) / nb;
    for (int f = 0; f < nfaults; ++f)
        if (!lu_fault_ok(faults[f], n, nb, N)) return -8;
    const bool emu = dtype == ABFT_F64_EMU;
    const LuWs w = lu_ws(n, nb, mode, emu);
    if (ws == nullptr) {
        *ws_bytes = w.total;
        return ABFT_OK;
    }
    if (*ws_bytes < w.total) return -13;
    cudaStream_t s = (cudaStream_t)stream;
    char* base = (char*)ws;
    DevStatus* st = (DevStatus*)(base + w.st);
    ABFT_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(DevStatus), s));
    if (n > 0) {
        rc = lu_steps(n, nb, mode, A, lda, ipiv, faults, nfaults, tau_scale, w, base, s, emu);
        if (rc != ABFT_OK) return rc;
    }
    ABFT_CUDA_TRY(timing_collect(s));
    if (rep) return finish_report(st, rep, s, true);
    return ABFT_OK;
}

}  // extern "C"

namespace {

// ------------------------------------------------------------------ QR
struct QrWs {
    size_t st, cs, cr, nrm, part, wv, V, G, T, W, X, sw, exw, su, exu, total;
    int64_t nc, nt, ldw;
};

// FP64-accurate QR update: the reduction of V^T [C, r] over the m panel rows
// runs in QR_KC-row pieces (K of one slice product)
constexpr int64_t QR_KC = 256;

QrWs qr_ws(int64_t n, int64_t nb, int mode, bool emu = false) {
    QrWs w{};
    w.nt = (n + nb - 1) / nb;
    w.nc = mode == ABFT_MODE_FULL ? 1 : (mode == ABFT_MODE_SINGLE ? 2 : 0);
    w.ldw = n + w.nt;
    const size_t d = sizeof(double);
    size_t off = 0;
    w.st = off; off = align_up(off + sizeof(DevStatus));
    w.cs = off; off = align_up(off + d * (size_t)(w.nc * w.nt) * (size_t)n);
    w.cr = off; off = align_up(off + (mode == ABFT_MODE_FULL ? d * (size_t)n * (size_t)w.nt : 0));
    w.nrm = off; off = align_up(off + d * (size_t)nb);
    w.part = off; off = align_up(off + d * 1024 * (size_t)(nb + 1));
    w.wv = off; off = align_up(off + d * (size_t)nb);
    w.V = off; off = align_up(off + d * (size_t)n * (size_t)nb);
    w.G = off; off = align_up(off + d * (size_t)nb * (size_t)nb);
    w.T = off; off = align_up(off + d * (size_t)nb * (size_t)nb);
    w.W = off; off = align_up(off + d * (size_t)nb * (size_t)w.ldw);
    w.X = off; off = align_up(off + d * (size_t)nb * (size_t)w.ldw);
    // slices: pieces of [V | C | r] columns (first step the largest), and
    // [V rows | checksum panel rows | columns of X]
    const int64_t rw = emu ? (n + QR_KC - 1) / QR_KC * (n + w.nt) : 0;
    const int64_t ru = emu ? 2 * n + w.nt * (w.nc + 1) : 0;
    w.sw = off; off = align_up(off + sizeof(uint16_t) * 8 * (size_t)rw * (size_t)QR_KC);
    w.exw = off; off = align_up(off + sizeof(int) * (size_t)rw);
    w.su = off; off = align_up(off + sizeof(uint16_t) * 8 * (size_t)ru * (size_t)nb);
    w.exu = off; off = align_up(off + sizeof(int) * (size_t)ru);
    w.total = off;
    return w;
}

bool qr_fault_ok(const abft_fault& f, int64_t n, int64_t nb, int64_t N) {
    if (f.step < 0 || f.step >= N - 1) return false;
    int64_t K0 = (int64_t)f.step * nb, T0 = std::min(K0 + nb, n);
    if (f.row < 0 || f.row >= n || f.col < 0 || f.col >= n) return false;
    if (f.kind < ABFT_FAULT_MEMORY || f.kind > ABFT_FAULT_COL1D) return false;
    return f.row >= K0 && f.col >= T0;
}

// Blocked ABFT Householder QR step loop.
int qr_steps(int64_t n, int64_t nb, int32_t mode, double* A, int64_t lda, double* tau,
             const abft_fault* faults, int32_t nfaults, double tau_scale, const QrWs& w,
             char* base, cudaStream_t s, bool emu) {
    DevStatus* st = (DevStatus*)(base + w.st);
    double* CS = (double*)(base + w.cs);
    double* Cr = (double*)(base + w.cr);
    double* nrm = (double*)(base + w.nrm);
    double* part = (double*)(base + w.part);
    double* wv = (double*)(base + w.wv);
    double* V = (double*)(base + w.V);
    double* Gn = (double*)(base + w.G);
    double* T = (double*)(base + w.T);
    double* Wb = (double*)(base + w.W);
    double* Xb = (double*)(base + w.X);
    const int64_t g = nb, nt = w.nt, nc = w.nc, N = nt, ldw = w.ldw;
    const bool full = mode == ABFT_MODE_FULL, check = mode != ABFT_MODE_NONE;

    TileSet base_ts{};
    base_ts.A = A; base_ts.lda = lda;
    base_ts.cc = CS; base_ts.cw = CS + n; base_ts.ccI = nc * n;
    base_ts.cr = Cr; base_ts.crs = nt; base_ts.crJ = 1;
    base_ts.g = g; base_ts.nrow_end = n; base_ts.ncol_end = n;
    timing_mark(PH_OTHER, 1, s);
    ABFT_CUDA_TRY(launch_qr_tau(A, lda, n, g, tau_scale, st, s));
    if (check) {
        TileSet ts = base_ts;
        ts.I0 = 0; ts.I1 = nt; ts.J0 = 0; ts.J1 = nt; ts.lower = 0;
        ABFT_CUDA_TRY(launch_encode(ts, mode, s));
    }
    timing_mark(PH_OTHER, 0, s);
    for (int64_t k = 0; k < N; ++k) {
        const int64_t K0 = k * g, kb = std::min(g, n - K0), T0 = K0 + kb, m = n - K0;
        double* P = A + K0 * lda + K0;
        timing_mark(PH_PD, 1, s);
        ABFT_CUDA_TRY(launch_geqr2_coop(P, lda, m, kb, tau + K0, nrm, part, wv, st, s));
        if (check) ABFT_CUDA_TRY(launch_qr_pd_check(P, lda, kb, nrm, (int)k, K0, st, s));
        if (T0 >= n) { timing_mark(PH_PD, 0, s); break; }
        ABFT_CUDA_TRY(launch_qr_prep_v(P, lda, m, kb, V, s));
        if (check) ABFT_CUDA_TRY(launch_qr_vsums(V, m, kb, g, k, nt, K0, CS, n, nc, mode, s));
        timing_mark(PH_PD, 0, s);
        // TMU (larfb): W = -V^T [C, r]; X = -T^T W; [C, r] -= V X; c_I -= (1^T V_I) X.
        // Gn = -V^T V (for T) shares the operand V^T and the reduction length m with
        // W, so it is one more segment of the same launch (its 64x64 tiles alone
        // would occupy only (kb/64)^2 SMs for the whole length m).
        const int64_t ncs = full ? nt - k - 1 : 0, nd = n - T0, ncol = nd + ncs;
        timing_mark(PH_TMU, 1, s);
        ABFT_CUDA_TRY(cudaMemsetAsync(Gn, 0, sizeof(double) * kb * kb, s));
        ABFT_CUDA_TRY(cudaMemsetAsync(Wb, 0, sizeof(double) * kb * ldw, s));
        ABFT_CUDA_TRY(cudaMemsetAsync(Xb, 0, sizeof(double) * kb * ldw, s));
        ComputeFault cf[MAX_CF];
        int ncf = 0;
        for (int f = 0; f < nfaults && ncf < MAX_CF; ++f)
            if (faults[f].step == k && faults[f].kind == ABFT_FAULT_COMPUTE)
                cf[ncf++] = {faults[f].row - K0, faults[f].col - T0, faults[f].delta};
        if (emu) {
            // FP64-accurate larfb from exact BF16 slice products.  Gn and W:
            // the reduction over the m panel rows in QR_KC-row pieces, piece p
            // holding the slices of columns p of [V | C | r] (one scale per
            // column and piece); one launch per piece subtracts its exact
            // product from Gn and W in turn (fixed order, FP64 sums).
            uint16_t* Sw = (uint16_t*)(base + w.sw);
            int* exw = (int*)(base + w.exw);
            const int64_t R = kb + ncol, npc = (m + QR_KC - 1) / QR_KC, MW = npc * R;
            ABFT_CUDA_TRY(launch_slice_cols_chunked(V, kb, QR_KC, m, kb, Sw, MW, 0, R, exw, s));
            ABFT_CUDA_TRY(launch_slice_cols_chunked(A + K0 * lda + T0, lda, QR_KC, m, nd, Sw, MW,
                                                    kb, R, exw, s));
            if (ncs > 0)
                ABFT_CUDA_TRY(launch_slice_cols_chunked(Cr + K0 * nt + (k + 1), nt, QR_KC, m, ncs,
                                                        Sw, MW, kb + nd, R, exw, s));
            for (int64_t pc = 0; pc < npc; ++pc) {
                const int64_t r0 = pc * R;
                EmuRectHost rw[3] = {};
                int nr = 0;
                {   // W[:, :nd] -= V_p^T C_p
                    EmuRectHost& r = rw[nr++];
                    r.C = Wb; r.ldc = ldw; r.a0 = r0; r.na = kb; r.b0 = r0 + kb; r.nb = nd;
                    r.cdiv = 1; r.frow = -1;
                }
                if (ncs > 0) {   // W[:, nd:] -= V_p^T r_p
                    EmuRectHost& r = rw[nr++];
                    r.C = Wb + nd; r.ldc = ldw; r.a0 = r0; r.na = kb; r.b0 = r0 + kb + nd;
                    r.nb = ncs; r.cdiv = 1; r.frow = -1;
                }
                {   // Gn -= V_p^T V_p
                    EmuRectHost& r = rw[nr++];
                    r.C = Gn; r.ldc = kb; r.a0 = r0; r.na = kb; r.b0 = r0; r.nb = kb;
                    r.cdiv = 1; r.frow = -1;
                }
                ABFT_CUDA_TRY(launch_tmu_emu(Sw, exw, MW, QR_KC, nullptr, 0, 0, 0, 128, rw, nr,
                                             nullptr, 0, 0, st, s));
            }
            ABFT_CUDA_TRY(launch_larft(Gn, kb, tau + K0, T, s));
            uint16_t* Su = (uint16_t*)(base + w.su);
            int* exu = (int*)(base + w.exu);
            {   // X = -T^T W: the columns of T against the columns of W
                const int64_t MX = kb + ncol;
                ABFT_CUDA_TRY(launch_slice_cols(T, kb, kb, kb, Su, MX, 0, exu, s));
                ABFT_CUDA_TRY(launch_slice_cols(Wb, ldw, kb, ncol, Su, MX, kb, exu, s));
                EmuRectHost rx{};
                rx.C = Xb; rx.ldc = ldw; rx.a0 = 0; rx.na = kb; rx.b0 = kb; rx.nb = ncol;
                rx.cdiv = 1; rx.frow = -1;
                ABFT_CUDA_TRY(launch_tmu_emu(Su, exu, MX, kb, nullptr, 0, 0, 0, 128, &rx, 1,
                                             nullptr, 0, 0, st, s));
            }
            // [C, r] -= V X and c_I -= (1^T V_I) X: rows of V and of the
            // checksum panel against the columns of X (the slices of T and W
            // above are consumed before these overwrite them: same stream)
            const int64_t mcs = check ? (nt - k) * nc : 0, MU = m + mcs + ncol;
            ABFT_CUDA_TRY(launch_slice_panel(V, kb, m, kb, Su, MU, 0, exu, s));
            if (mcs > 0)
                ABFT_CUDA_TRY(launch_slice_panel(CS + (k * nc) * n + K0, n, mcs, kb, Su, MU, m,
                                                 exu, s));
            ABFT_CUDA_TRY(launch_slice_cols(Xb, ldw, kb, ncol, Su, MU, m + mcs, exu, s));
            EmuRectHost ru[3] = {};
            int nr = 0;
            {
                EmuRectHost& r = ru[nr++];
                r.C = A + K0 * lda + T0; r.ldc = lda; r.a0 = 0; r.na = m; r.b0 = m + mcs;
                r.nb = nd; r.cdiv = 1; r.frow = 0; r.fcol = 0;
            }
            if (check) {
                EmuRectHost& r = ru[nr++];
                r.C = CS + (k * nc) * n + T0; r.ldc = n; r.a0 = m; r.na = mcs; r.b0 = m + mcs;
                r.nb = nd; r.cdiv = 1; r.frow = -1;
            }
            if (full && ncs > 0) {
                EmuRectHost& r = ru[nr++];
                r.C = Cr + K0 * nt + (k + 1); r.ldc = nt; r.a0 = 0; r.na = m;
                r.b0 = m + mcs + nd; r.nb = ncs; r.cdiv = 1; r.frow = -1;
            }
            ABFT_CUDA_TRY(launch_tmu_emu(Su, exu, MU, kb, nullptr, 0, 0, 0, 128, ru, nr, cf, ncf,
                                         0, st, s));
            timing_mark(PH_TMU, 0, s);
        } else {
        GemmSeg g1[3] = {};
        g1[0].A = V; g1[0].lda = kb; g1[0].B = V; g1[0].ldb = kb;
        g1[0].C = Gn; g1[0].ldc = kb; g1[0].M = kb; g1[0].N = kb; g1[0].K = m;
        g1[1].A = V; g1[1].lda = kb; g1[1].B = A + K0 * lda + T0; g1[1].ldb = lda;
        g1[1].C = Wb; g1[1].ldc = ldw; g1[1].M = kb; g1[1].N = nd; g1[1].K = m;
        g1[2].A = V; g1[2].lda = kb; g1[2].B = Cr + K0 * nt + (k + 1); g1[2].ldb = nt;
        g1[2].C = Wb + nd; g1[2].ldc = ldw; g1[2].M = kb; g1[2].N = ncs; g1[2].K = m;
        ABFT_CUDA_TRY(launch_gemm_f64(g1, full ? 3 : 2, 1, 1, nullptr, 0, st, s));
        ABFT_CUDA_TRY(launch_larft(Gn, kb, tau + K0, T, s));
        GemmSeg g2{};
        g2.A = T; g2.lda = kb; g2.B = Wb; g2.ldb = ldw; g2.C = Xb; g2.ldc = ldw;
        g2.M = kb; g2.N = ncol; g2.K = kb;
        ABFT_CUDA_TRY(launch_gemm_f64(&g2, 1, 1, 1, nullptr, 0, st, s));
        GemmSeg g3[3] = {};
        g3[0].A = V; g3[0].lda = kb; g3[0].B = Xb; g3[0].ldb = ldw;
        g3[0].C = A + K0 * lda + T0; g3[0].ldc = lda; g3[0].M = m; g3[0].N = nd; g3[0].K = kb;
        int nseg = 1;
        if (check) {
            GemmSeg& b = g3[nseg++];
            b.A = CS + (k * nc) * n + K0; b.lda = n; b.B = Xb; b.ldb = ldw;
            b.C = CS + (k * nc) * n + T0; b.ldc = n; b.M = (nt - k) * nc; b.N = nd; b.K = kb;
        }
        if (full) {
            GemmSeg& b = g3[nseg++];
            b.A = V; b.lda = kb; b.B = Xb + nd; b.ldb = ldw;
            b.C = Cr + K0 * nt + (k + 1); b.ldc = nt; b.M = m; b.N = ncs; b.K = kb;
        }
        ABFT_CUDA_TRY(launch_gemm_f64(g3, nseg, 0, 1, cf, ncf, st, s));
        timing_mark(PH_TMU, 0, s);
        }
        timing_mark(PH_VERIFY, 1, s);
        for (int f = 0; f < nfaults; ++f)
            if (faults[f].step == k && (faults[f].kind == ABFT_FAULT_MEMORY ||
                                        faults[f].kind == ABFT_FAULT_ROW1D ||
                                        faults[f].kind == ABFT_FAULT_COL1D))
                ABFT_CUDA_TRY(launch_inject(A, lda, n, g, faults[f], s));
        if (check) {
            TileSet ts = base_ts;
            ts.I0 = k; ts.I1 = nt; ts.J0 = k + 1; ts.J1 = nt; ts.lower = 0;
            ABFT_CUDA_TRY(launch_verify(ts, mode, (int)k, st, s));
        }
        timing_mark(PH_VERIFY, 0, s);
    }
    return ABFT_OK;
}

}  // namespace

extern "C" {

int abft_geqrf(int64_t n, int64_t nb, int32_t dtype, int32_t mode, double* A, int64_t lda,
               double* tau, const abft_fault* faults, int32_t nfaults, double tau_scale,
               abft_report* rep, void* ws, size_t* ws_bytes, void* stream) {
    int rc = check_common(n, nb, dtype, mode, A, lda, faults, nfaults, tau_scale, ws, ws_bytes,
                          true);
    if (rc != ABFT_OK) return rc;
    if (n > 0 && tau == nullptr && ws != nullptr) return -7;
    const int64_t N = (n + nb - 1) / nb;
    for (int f = 0; f < nfaults; ++f)
        if (!qr_fault_ok(faults[f], n, nb, N)) return -8;
    const bool emu = dtype == ABFT_F64_EMU;
    const QrWs w = qr_ws(n, nb, mode, emu);
    if (ws == nullptr) {
        *ws_bytes = w.total;
        return ABFT_OK;
    }
    if (*ws_bytes < w.total) return -13;
    cudaStream_t s = (cudaStream_t)stream;
    char* base = (char*)ws;
    DevStatus* st = (DevStatus*)(base + w.st);
    ABFT_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(DevStatus), s));
    if (n > 0) {
        rc = qr_steps(n, nb, mode, A, lda, tau, faults, nfaults, tau_scale, w, base, s, emu);
        if (rc != ABFT_OK) return rc;
    }
    ABFT_CUDA_TRY(timing_collect(s));
    if (rep) return finish_report(st, rep, s);
    return ABFT_OK;
}

}  // extern "C"

namespace {

// ------------------------------------------------------------- solves / IR
constexpr int kSplit = 8;   // split-K factor of the FP64 residual

// potrs scratch: the inverses of L's diagonal blocks with the sweep's flags
// (room for either arithmetic), then, for the FP32 solve, an n x 16 FP32 copy
// of the right-hand sides and the lower triangle of L rounded to FP32 (n x n).
struct SolvePtrs {
    void* inv;
    float* Yf;
    float* L32;
};

SolvePtrs solve_ptrs(char* ws, int64_t n) {
    SolvePtrs p;
    p.inv = ws;
    size_t off = align_up(potrs_inv_bytes(n, true));
    p.Yf = (float*)(ws + off);
    off += align_up(sizeof(float) * (size_t)n * 16);
    p.L32 = (float*)(ws + off);
    return p;
}

size_t potrs_ws_bytes(int64_t n, int32_t dtype) {
    const size_t inv = align_up(potrs_inv_bytes(n, true));
    const size_t f = (dtype == ABFT_F64) ? 0
                                         : align_up(sizeof(float) * (size_t)n * 16) +
                                               align_up(sizeof(float) * (size_t)n * (size_t)n);
    return std::max<size_t>(inv + f, 256);
}

// prepared: the block inverses (and for FP32 the FP32 copy of L) of this L are
// already in ws from an earlier call.
int potrs_run(int64_t n, int64_t nrhs, int64_t nb, int32_t dtype, const double* L, int64_t ldl,
              double* B, int64_t ldb, char* ws, cudaStream_t s, bool prepared = false) {
    const SolvePtrs sp = solve_ptrs(ws, n);
    void* inv = sp.inv;
    float* Yf = sp.Yf;
    if (dtype != ABFT_F64 && !prepared && nrhs > 0)
        ABFT_CUDA_TRY(launch_tril_to_f32(L, ldl, n, sp.L32, s));
    for (int64_t r0 = 0; r0 < nrhs; r0 += 16) {
        const int nr = (int)std::min<int64_t>(16, nrhs - r0);
        const bool have_inv = prepared || r0 > 0;
        if (dtype == ABFT_F64) {
            ABFT_CUDA_TRY(launch_potrs_f64(n, nr, nb, L, ldl, B + r0, ldb, (double*)inv, s,
                                           have_inv));
        } else {
            ABFT_CUDA_TRY(launch_copy_d2f(B + r0, ldb, Yf, 16, n, nr, s));
            ABFT_CUDA_TRY(launch_potrs_f32(n, nr, nb, L, ldl, Yf, 16, (float*)inv, s, have_inv,
                                           sp.L32));
            ABFT_CUDA_TRY(launch_copy_f2d(Yf, 16, B + r0, ldb, n, nr, s));
        }
        cudaError_t ce = cudaSuccess;
        const int err = potrs_error(inv, n, dtype == ABFT_F64, s, &ce);
        ABFT_CUDA_TRY(ce);
        if (err) return ABFT_ERR_TIMEOUT;
    }
    return ABFT_OK;
}

struct IrWs {
    size_t chol, solve, R, P, rs, norms, eta, re, total;
    bool emu_resid;   // residual from BF16 slices of A on the tensor cores
};

IrWs ir_ws(int64_t n, int64_t nb, int mode, int32_t dtype) {
    IrWs w{};
    const bool mixed = dtype == ABFT_MIXED_BF16 || dtype == ABFT_MIXED_F16;
    const bool emu = dtype == ABFT_F64_EMU;
    size_t off = 0;
    w.chol = off; off = align_up(off + chol_ws(n, nb, mode, mixed, emu).total);
    w.solve = off; off = align_up(off + potrs_ws_bytes(n, ABFT_F32));
    w.R = off; off = align_up(off + sizeof(double) * (size_t)n * 16);
    w.P = off; off = align_up(off + sizeof(double) * (size_t)kSplit * (size_t)n * 16);
    w.rs = off; off = align_up(off + sizeof(double) * (size_t)n);
    w.norms = off; off = align_up(off + sizeof(unsigned long long) * 64);
    w.eta = off; off = align_up(off + sizeof(double));
    // the 16-bit and FP64-accurate factorizations refine with an FP64-accurate
    // residual from BF16 slices of A (FP64 factorizations keep the FP64 residual)
    w.emu_resid = (mixed || emu) && resid_emu_supported(n);
    w.re = off; off = align_up(off + (w.emu_resid ? resid_emu_bytes(n) : 0));
    w.total = off;
    return w;
}

constexpr int kGmresMax = 64;       // largest GMRES cycle (basis vectors)
constexpr int kGmresAttempts = 8;   // factorizations tried with growing shift

struct GmWs {
    size_t sc, V, W, part, hnew, h2, H, cs, sn, g, res, y, a32, total;
};

GmWs gm_ws(int64_t n, int m, size_t off, bool a32) {
    GmWs w{};
    const size_t d = sizeof(double);
    const size_t blk = d * (size_t)n * 16;
    w.sc = off; off = align_up(off + d * (size_t)std::max<int64_t>(n, 1));
    w.V = off; off = align_up(off + blk * (size_t)(m + 1));
    w.W = off; off = align_up(off + blk);
    w.part = off; off = align_up(off + d * 16 * (size_t)(m + 2) * (size_t)gmres_dot_blocks(n));
    w.hnew = off; off = align_up(off + d * 16 * (size_t)(m + 2));
    w.h2 = off; off = align_up(off + d * 16 * (size_t)(m + 2));
    w.H = off; off = align_up(off + d * 16 * (size_t)m * (size_t)(m + 1));
    w.cs = off; off = align_up(off + d * 16 * (size_t)m);
    w.sn = off; off = align_up(off + d * 16 * (size_t)m);
    w.g = off; off = align_up(off + d * 16 * (size_t)(m + 1));
    w.res = off; off = align_up(off + d * 16);
    w.y = off; off = align_up(off + d * 16 * (size_t)m);
    w.a32 = off; off = align_up(off + (a32 ? sizeof(float) * (size_t)n * (size_t)n : 0));
    w.total = off;
    return w;
}

}  // namespace

extern "C" {

int abft_symm_emu(int64_t n, int64_t nrhs, const double* A, int64_t lda, const double* X,
                  int64_t ldx, double* Y, int64_t ldy, void* ws, size_t* ws_bytes, void* stream) {
    if (n < 0 || (n > 0 && !resid_emu_supported(n))) return n < 0 ? -1 : ABFT_ERR_UNSUPPORTED;
    if (nrhs < 0) return -2;
    if (lda < std::max<int64_t>(1, n)) return -4;
    if (ldx < std::max<int64_t>(1, nrhs)) return -6;
    if (ldy < std::max<int64_t>(1, nrhs)) return -8;
    if (ws_bytes == nullptr) return -10;
    const size_t need = n > 0 ? align_up(resid_emu_bytes(n)) + align_up(sizeof(double) * n * 16) : 0;
    if (ws == nullptr) {
        *ws_bytes = need;
        return ABFT_OK;
    }
    if (*ws_bytes < need) return -10;
    if (n == 0 || nrhs == 0) return ABFT_OK;
    if (A == nullptr) return -3;
    if (X == nullptr) return -5;
    if (Y == nullptr) return -7;
    cudaStream_t s = (cudaStream_t)stream;
    char* base = (char*)ws;
    double* Y16 = (double*)(base + align_up(resid_emu_bytes(n)));
    timing_mark(PH_SOLVE, 1, s);
    ABFT_CUDA_TRY(launch_resid_emu_prepare(A, lda, n, base, s));
    for (int64_t r0 = 0; r0 < nrhs; r0 += 16) {
        const int nr = (int)std::min<int64_t>(16, nrhs - r0);
        ABFT_CUDA_TRY(launch_resid_emu(n, X + r0, ldx, nullptr, 0, nr, Y16, 16, base, nullptr,
                                       nullptr, s));
        ABFT_CUDA_TRY(launch_copy_d2d(Y16, 16, Y + r0, ldy, n, nr, s));
    }
    timing_mark(PH_SOLVE, 0, s);
    ABFT_CUDA_TRY(timing_collect(s));
    return ABFT_OK;
}

int abft_potrs(int64_t n, int64_t nrhs, int64_t nb, int32_t dtype, const double* L, int64_t ldl,
               double* B, int64_t ldb, void* ws, size_t* ws_bytes, void* stream) {
    if (n < 0) return -1;
    if (nrhs < 0) return -2;
    if (nb <= 0 || nb % 32 != 0 || nb > 512) return -3;
    if (dtype < 0 || dtype > 3) return -4;
    if (n > 0 && L == nullptr && ws != nullptr) return -5;
    if (ldl < std::max<int64_t>(1, n)) return -6;
    if (n > 0 && nrhs > 0 && B == nullptr && ws != nullptr) return -7;
    if (ldb < std::max<int64_t>(1, nrhs)) return -8;
    if (ws_bytes == nullptr) return -10;
    const size_t need = potrs_ws_bytes(n, dtype);
    if (ws == nullptr) {
        *ws_bytes = need;
        return ABFT_OK;
    }
    if (*ws_bytes < need) return -10;
    if (n == 0 || nrhs == 0) return ABFT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    timing_mark(PH_SOLVE, 1, s);
    int rc = potrs_run(n, nrhs, nb, dtype, L, ldl, B, ldb, (char*)ws, s);
    timing_mark(PH_SOLVE, 0, s);
    if (rc != ABFT_OK) return rc;
    ABFT_CUDA_TRY(timing_collect(s));
    return ABFT_OK;
}

int abft_posv_ir(int64_t n, int64_t nrhs, int64_t nb, int32_t dtype, int32_t mode, const double* A,
                 int64_t lda, double* L, int64_t ldl, const double* B, int64_t ldb, double* X,
                 int64_t ldx, double tol, int32_t maxit, const abft_fault* faults, int32_t nfaults,
                 double tau_scale, abft_report* rep, void* ws, size_t* ws_bytes, void* stream) {
    if (n < 0) return -1;
    if (nrhs < 0) return -2;
    if (nb <= 0 || nb % 32 != 0 || nb > 512) return -3;
    if (dtype < 0 || dtype > 4 || dtype == ABFT_F32) return dtype == ABFT_F32 ? ABFT_ERR_UNSUPPORTED : -4;
    if (mode < ABFT_MODE_NONE || mode > ABFT_MODE_FULL) return -5;
    const bool needp = ws != nullptr && n > 0;
    if (needp && A == nullptr) return -6;
    if (lda < std::max<int64_t>(1, n)) return -7;
    if (needp && L == nullptr) return -8;
    if (ldl < std::max<int64_t>(1, n)) return -9;
    if (needp && nrhs > 0 && B == nullptr) return -10;
    if (ldb < std::max<int64_t>(1, nrhs)) return -11;
    if (needp && nrhs > 0 && X == nullptr) return -12;
    if (ldx < std::max<int64_t>(1, nrhs)) return -13;
    if (!(tol >= 0.0)) return -14;
    if (maxit < 0) return -15;
    if (ws_bytes == nullptr) return -22;
    // the solves run in FP64 for the FP64 and FP64-accurate factors (their
    // accuracy would be lost in FP32 solves), in FP32 for the 16-bit ones
    const int32_t sdt = (dtype == ABFT_F64 || dtype == ABFT_F64_EMU) ? ABFT_F64 : ABFT_F32;
    const IrWs w = ir_ws(n, nb, mode, dtype);
    size_t pws = 0;
    int rc = abft_potrf(n, nb, dtype, mode, L, ldl, faults, nfaults, tau_scale, nullptr, nullptr,
                        &pws, nullptr);
    if (rc != ABFT_OK) return rc == -7 ? -16 : rc;
    if (ws == nullptr) {
        *ws_bytes = w.total;
        return ABFT_OK;
    }
    if (*ws_bytes < w.total) return -22;
    cudaStream_t s = (cudaStream_t)stream;
    char* base = (char*)ws;
    abft_report prep;
    abft_report* pr = rep ? rep : &prep;
    // factor a copy of A (lower triangle)
    ABFT_CUDA_TRY(launch_copy_d2d(A, lda, L, ldl, n, (int)n, s));
    size_t have = pws;
    rc = abft_potrf(n, nb, dtype, mode, L, ldl, faults, nfaults, tau_scale, pr, base + w.chol,
                    &have, stream);
    if (rc > 0 || rc == ABFT_ERR_CUDA || rc == ABFT_ERR_TIMEOUT) return rc;
    const int factor_rc = rc;
    if (n == 0 || nrhs == 0) return factor_rc;
    char* sws = base + w.solve;
    const SolvePtrs sp = solve_ptrs(sws, n);
    void* inv = sp.inv;
    float* Yf = sp.Yf;
    double* R = (double*)(base + w.R);
    double* P = (double*)(base + w.P);
    double* rs = (double*)(base + w.rs);
    unsigned long long* nrm = (unsigned long long*)(base + w.norms);
    unsigned long long *anorm = nrm, *bmax = nrm + 1, *rmax = nrm + 17, *xmax = nrm + 33;
    double* eta_d = (double*)(base + w.eta);
    int32_t iters_max = 0;
    double eta_max = 0.0;
    bool prepared = false;   // block inverses (and the FP32 copy of L) formed
    if (w.emu_resid) {       // slices of A, once per solve
        timing_mark(PH_SOLVE, 1, s);
        ABFT_CUDA_TRY(launch_resid_emu_prepare(A, lda, n, base + w.re, s));
        timing_mark(PH_SOLVE, 0, s);
    }
    for (int64_t r0 = 0; r0 < nrhs; r0 += 16) {
        const int nr = (int)std::min<int64_t>(16, nrhs - r0);
        ABFT_CUDA_TRY(cudaMemsetAsync(nrm, 0, sizeof(unsigned long long) * 64, s));
        ABFT_CUDA_TRY(launch_inf_norms(A, lda, n, B + r0, ldb, nr, rs, anorm, bmax, P, s));
        // X0 = L^{-T} L^{-1} B
        timing_mark(PH_SOLVE, 1, s);
        ABFT_CUDA_TRY(launch_copy_d2d(B + r0, ldb, X + r0, ldx, n, nr, s));
        rc = potrs_run(n, nr, nb, sdt, L, ldl, X + r0, ldx, sws, s, prepared);
        if (rc != ABFT_OK) return rc;
        prepared = true;
        int32_t it = 0;
        double eta = 0.0;
        for (;; ++it) {
            ABFT_CUDA_TRY(cudaMemsetAsync(rmax, 0, sizeof(unsigned long long) * 32, s));
            if (w.emu_resid)
                ABFT_CUDA_TRY(launch_resid_emu(n, X + r0, ldx, B + r0, ldb, nr, R, 16, base + w.re,
                                               rmax, xmax, s));
            else
                ABFT_CUDA_TRY(launch_residual(A, lda, n, X + r0, ldx, B + r0, ldb, nr, R, 16, P,
                                              kSplit, rmax, xmax, s));
            ABFT_CUDA_TRY(launch_eta(rmax, xmax, anorm, bmax, nr, eta_d, s));
            ABFT_CUDA_TRY(cudaMemcpyAsync(&eta, eta_d, sizeof(double), cudaMemcpyDeviceToHost, s));
            ABFT_CUDA_TRY(cudaStreamSynchronize(s));
            if (eta <= tol || it >= maxit || !(eta == eta)) break;
            // correction D = L^{-T} L^{-1} R in the solve precision, X += D
            // the inverses of L's diagonal blocks are still in inv from potrs_run
            if (sdt == ABFT_F64) {
                ABFT_CUDA_TRY(launch_potrs_f64(n, nr, nb, L, ldl, R, 16, (double*)inv, s, true));
                ABFT_CUDA_TRY(launch_add_f64(X + r0, ldx, R, 16, n, nr, s));
            } else {
                ABFT_CUDA_TRY(launch_copy_d2f(R, 16, Yf, 16, n, nr, s));
                ABFT_CUDA_TRY(launch_potrs_f32(n, nr, nb, L, ldl, Yf, 16, (float*)inv, s, true,
                                               sp.L32));
                ABFT_CUDA_TRY(launch_add_f32(X + r0, ldx, Yf, 16, n, nr, s));
            }
            cudaError_t ce = cudaSuccess;
            const int serr = potrs_error(inv, n, sdt == ABFT_F64, s, &ce);
            ABFT_CUDA_TRY(ce);
            if (serr) return ABFT_ERR_TIMEOUT;
        }
        timing_mark(PH_SOLVE, 0, s);
        iters_max = std::max(iters_max, it);
        eta_max = std::max(eta_max, eta);
    }
    ABFT_CUDA_TRY(timing_collect(s));
    pr->ir_iters = iters_max;
    pr->backward_err = eta_max;
    return factor_rc;
}


int abft_posv_gmres_ir(int64_t n, int64_t nrhs, int64_t nb, int32_t dtype, int32_t mode,
                       const double* A, int64_t lda, double* L, int64_t ldl, const double* B,
                       int64_t ldb, double* X, int64_t ldx, double tol, int32_t maxit, int32_t m,
                       double inner_tol, double shift, int32_t scale, int32_t precond_f64,
                       int32_t inner_f32, const abft_fault* faults, int32_t nfaults,
                       double tau_scale, abft_report* rep, void* ws, size_t* ws_bytes,
                       void* stream) {
    if (n < 0) return -1;
    if (nrhs < 0) return -2;
    if (nb <= 0 || nb % 32 != 0 || nb > 512) return -3;
    if (dtype < 0 || dtype > 3 || dtype == ABFT_F32) return dtype == ABFT_F32 ? ABFT_ERR_UNSUPPORTED : -4;
    if (mode < ABFT_MODE_NONE || mode > ABFT_MODE_FULL) return -5;
    const bool needp = ws != nullptr && n > 0;
    if (needp && A == nullptr) return -6;
    if (lda < std::max<int64_t>(1, n)) return -7;
    if (needp && L == nullptr) return -8;
    if (ldl < std::max<int64_t>(1, n)) return -9;
    if (needp && nrhs > 0 && B == nullptr) return -10;
    if (ldb < std::max<int64_t>(1, nrhs)) return -11;
    if (needp && nrhs > 0 && X == nullptr) return -12;
    if (ldx < std::max<int64_t>(1, nrhs)) return -13;
    if (!(tol >= 0.0)) return -14;
    if (maxit < 0) return -15;
    if (m < 1 || m > kGmresMax) return -16;
    if (!(inner_tol >= 0.0)) return -17;
    if (!(shift >= 0.0) && !(shift < 0.0)) return -18;   // NaN
    if (ws_bytes == nullptr) return -22;
    const IrWs w = ir_ws(n, nb, mode, dtype);
    const GmWs gw = gm_ws(n, m, w.total, inner_f32 != 0);
    size_t pws = 0;
    int rc = abft_potrf(n, nb, dtype, mode, L, ldl, faults, nfaults, tau_scale, nullptr, nullptr,
                        &pws, nullptr);
    if (rc != ABFT_OK) return rc == -7 ? -19 : rc;
    if (ws == nullptr) {
        *ws_bytes = gw.total;
        return ABFT_OK;
    }
    if (*ws_bytes < gw.total) return -22;
    cudaStream_t s = (cudaStream_t)stream;
    char* base = (char*)ws;
    abft_report prep;
    abft_report* pr = rep ? rep : &prep;
    double* sc = (double*)(base + gw.sc);
    // scaling (powers of two, exact) and the shifted low-precision factorization;
    // a non-positive pivot restarts it with a larger shift (automatic when shift < 0)
    const double ulow = dtype == ABFT_MIXED_F16 ? 0x1p-11 : (dtype == ABFT_F64 ? 0x1p-53 : 0x1p-8);
    double delta = shift < 0.0 ? 0.0 : shift;
    int32_t attempts = 0;
    ABFT_CUDA_TRY(launch_gm_diag_scale(A, lda, n, sc, scale ? 1 : 0, s));
    for (;;) {
        ++attempts;
        ABFT_CUDA_TRY(launch_gm_scaled_copy(A, lda, sc, delta, L, ldl, n, s));
        size_t have = pws;
        rc = abft_potrf(n, nb, dtype, mode, L, ldl, faults, nfaults, tau_scale, pr, base + w.chol,
                        &have, stream);
        if (rc > 0 && shift < 0.0 && attempts < kGmresAttempts) {
            delta = delta > 0.0 ? 4.0 * delta : ulow;
            continue;
        }
        break;
    }
    if (rc > 0 || rc == ABFT_ERR_CUDA || rc == ABFT_ERR_TIMEOUT) {
        pr->attempts = attempts;
        pr->shift = delta;
        return rc;
    }
    const int factor_rc = rc;
    pr->attempts = attempts;
    pr->shift = delta;
    if (n == 0 || nrhs == 0) return factor_rc;
    char* sws = base + w.solve;
    const SolvePtrs sp = solve_ptrs(sws, n);
    void* inv = sp.inv;
    float* Yf = sp.Yf;
    double* R = (double*)(base + w.R);
    double* P = (double*)(base + w.P);
    double* rs = (double*)(base + w.rs);
    unsigned long long* nrm = (unsigned long long*)(base + w.norms);
    unsigned long long *anorm = nrm, *bmax = nrm + 1, *rmax = nrm + 17, *xmax = nrm + 33;
    double* eta_d = (double*)(base + w.eta);
    double* V = (double*)(base + gw.V);
    const int64_t vstride = n * 16;
    double* Wb = (double*)(base + gw.W);
    double* part = (double*)(base + gw.part);
    double* hnew = (double*)(base + gw.hnew);
    double* h2 = (double*)(base + gw.h2);
    double* H = (double*)(base + gw.H);
    double* cs = (double*)(base + gw.cs);
    double* sn = (double*)(base + gw.sn);
    double* g = (double*)(base + gw.g);
    double* res = (double*)(base + gw.res);
    double* yv = (double*)(base + gw.y);
    float* A32 = (float*)(base + gw.a32);
    const bool f64 = precond_f64 != 0;
    if (inner_f32) ABFT_CUDA_TRY(launch_copy_d2f(A, lda, A32, n, n, (int)n, s));
    // z := M^{-1} z = S L^{-T} L^{-1} S z, in place on an n x 16 block; the
    // inverses of L's diagonal blocks are formed by the first application
    bool inv_ready = false;
    auto precond = [&](double* z) -> int {
        ABFT_CUDA_TRY(launch_gm_rowscale(sc, z, z, n, s));
        if (f64) {
            ABFT_CUDA_TRY(launch_potrs_f64(n, 16, nb, L, ldl, z, 16, (double*)inv, s, inv_ready));
        } else {
            if (!inv_ready) ABFT_CUDA_TRY(launch_tril_to_f32(L, ldl, n, sp.L32, s));
            ABFT_CUDA_TRY(launch_copy_d2f(z, 16, Yf, 16, n, 16, s));
            ABFT_CUDA_TRY(launch_potrs_f32(n, 16, nb, L, ldl, Yf, 16, (float*)inv, s, inv_ready,
                                           sp.L32));
            ABFT_CUDA_TRY(launch_copy_f2d(Yf, 16, z, 16, n, 16, s));
        }
        inv_ready = true;
        ABFT_CUDA_TRY(launch_gm_rowscale(sc, z, z, n, s));
        return ABFT_OK;
    };
    auto solve_err = [&]() -> int {
        cudaError_t ce = cudaSuccess;
        const int e = potrs_error(inv, n, f64, s, &ce);
        ABFT_CUDA_TRY(ce);
        return e ? ABFT_ERR_TIMEOUT : ABFT_OK;
    };
    int32_t iters_max = 0, gm_total = 0;
    double eta_max = 0.0;
    std::vector<double> hres(16), beta(16);
    if (w.emu_resid) {   // slices of A for the residuals and products, once per solve
        timing_mark(PH_SOLVE, 1, s);
        ABFT_CUDA_TRY(launch_resid_emu_prepare(A, lda, n, base + w.re, s));
        timing_mark(PH_SOLVE, 0, s);
    }
    for (int64_t r0 = 0; r0 < nrhs; r0 += 16) {
        const int nr = (int)std::min<int64_t>(16, nrhs - r0);
        ABFT_CUDA_TRY(cudaMemsetAsync(nrm, 0, sizeof(unsigned long long) * 64, s));
        ABFT_CUDA_TRY(launch_inf_norms(A, lda, n, B + r0, ldb, nr, rs, anorm, bmax, P, s));
        timing_mark(PH_SOLVE, 1, s);
        // X0 = M^{-1} B (the padding columns stay zero)
        ABFT_CUDA_TRY(cudaMemsetAsync(Wb, 0, sizeof(double) * (size_t)n * 16, s));
        ABFT_CUDA_TRY(launch_copy_d2d(B + r0, ldb, Wb, 16, n, nr, s));
        rc = precond(Wb);
        if (rc != ABFT_OK) return rc;
        ABFT_CUDA_TRY(launch_copy_d2d(Wb, 16, X + r0, ldx, n, nr, s));
        int32_t it = 0;
        double eta = 0.0;
        for (;; ++it) {
            ABFT_CUDA_TRY(cudaMemsetAsync(rmax, 0, sizeof(unsigned long long) * 32, s));
            ABFT_CUDA_TRY(cudaMemsetAsync(R, 0, sizeof(double) * (size_t)n * 16, s));
            if (w.emu_resid)
                ABFT_CUDA_TRY(launch_resid_emu(n, X + r0, ldx, B + r0, ldb, nr, R, 16, base + w.re,
                                               rmax, xmax, s));
            else
                ABFT_CUDA_TRY(launch_residual(A, lda, n, X + r0, ldx, B + r0, ldb, nr, R, 16, P, kSplit,
                                          rmax, xmax, s));
            ABFT_CUDA_TRY(launch_eta(rmax, xmax, anorm, bmax, nr, eta_d, s));
            ABFT_CUDA_TRY(cudaMemcpyAsync(&eta, eta_d, sizeof(double), cudaMemcpyDeviceToHost, s));
            rc = solve_err();
            if (rc != ABFT_OK) return rc;
            if (eta <= tol || it >= maxit || !(eta == eta)) break;
            // GMRES on M^{-1} A d = M^{-1} R from d = 0
            rc = precond(R);
            if (rc != ABFT_OK) return rc;
            ABFT_CUDA_TRY(launch_gm_dots(R, 0, 1, R, n, part, hnew, 0, s));
            ABFT_CUDA_TRY(launch_gm_init_g(hnew, g, m, res, s));
            ABFT_CUDA_TRY(launch_gm_scale(R, hnew, V, n, s));
            ABFT_CUDA_TRY(cudaMemcpyAsync(beta.data(), res, sizeof(double) * 16,
                                          cudaMemcpyDeviceToHost, s));
            ABFT_CUDA_TRY(cudaStreamSynchronize(s));
            int k = 0;
            for (int j = 0; j < m; ++j) {
                double* Vj = V + (int64_t)j * vstride;
                if (inner_f32) ABFT_CUDA_TRY(launch_symv_f32(A32, n, n, Vj, Wb, P, kSplit, s));
                else if (w.emu_resid)
                    ABFT_CUDA_TRY(launch_resid_emu(n, Vj, 16, nullptr, 0, 16, Wb, 16, base + w.re,
                                                   nullptr, nullptr, s));
                else ABFT_CUDA_TRY(launch_symv(A, lda, n, Vj, Wb, P, kSplit, s));
                rc = precond(Wb);
                if (rc != ABFT_OK) return rc;
                // classical Gram-Schmidt, twice
                ABFT_CUDA_TRY(launch_gm_dots(V, vstride, j + 1, Wb, n, part, hnew, 0, s));
                ABFT_CUDA_TRY(launch_gm_subtract(V, vstride, j + 1, hnew, Wb, n, s));
                ABFT_CUDA_TRY(launch_gm_dots(V, vstride, j + 1, Wb, n, part, h2, 0, s));
                ABFT_CUDA_TRY(launch_gm_subtract(V, vstride, j + 1, h2, Wb, n, s));
                ABFT_CUDA_TRY(launch_add_f64(hnew, 16, h2, 16, j + 1, 16, s));
                ABFT_CUDA_TRY(launch_gm_dots(Wb, 0, 1, Wb, n, part, hnew + (int64_t)(j + 1) * 16, 0, s));
                ABFT_CUDA_TRY(launch_gm_givens(H, m, hnew, cs, sn, g, j, res, s));
                ABFT_CUDA_TRY(launch_gm_scale(Wb, hnew + (int64_t)(j + 1) * 16,
                                              V + (int64_t)(j + 1) * vstride, n, s));
                ABFT_CUDA_TRY(cudaMemcpyAsync(hres.data(), res, sizeof(double) * 16,
                                              cudaMemcpyDeviceToHost, s));
                rc = solve_err();
                if (rc != ABFT_OK) return rc;
                k = j + 1;
                double worst = 0.0;
                for (int r = 0; r < nr; ++r)
                    if (beta[r] > 0.0) worst = std::max(worst, hres[r] / beta[r]);
                if (!(worst > inner_tol)) break;
            }
            ABFT_CUDA_TRY(launch_gm_update(H, m, g, k, yv, V, vstride, X + r0, ldx, nr, n, s));
            gm_total += k;
        }
        timing_mark(PH_SOLVE, 0, s);
        iters_max = std::max(iters_max, it);
        eta_max = std::max(eta_max, eta);
    }
    ABFT_CUDA_TRY(timing_collect(s));
    pr->ir_iters = iters_max;
    pr->gmres_iters = gm_total;
    pr->backward_err = eta_max;
    return factor_rc;
}
}  // extern "C"

namespace {

// -------------------------------------------------------------- adjoint
constexpr int kAdjSplit = 16;

size_t adj_base_bytes(int64_t nb) {
    const size_t d = sizeof(double);
    return align_up(d * nb * nb) * 3 + align_up(d * (size_t)kAdjSplit * nb * nb);
}

// FP64-accurate sweep: per block column J of F = Abar_L + Abar_L^T a slice
// tensor region of R = n + nb rows (F's rows, then the columns of the current
// L21 cut to block row J), 8 BF16 slices of nb columns each; one exponent per
// slice row; a status block for the tensor-core kernel; the symmetric diagonal block.
struct AdjEmu {
    size_t st, S, ex, D, PS, pex, total;
    int64_t N, R;
};
AdjEmu adj_emu_layout(int64_t n, int64_t nb) {
    AdjEmu a{};
    a.N = (n + nb - 1) / nb;
    a.R = n + nb;
    size_t off = adj_base_bytes(nb);
    a.st = off; off = align_up(off + sizeof(DevStatus));
    a.S = off; off = align_up(off + sizeof(uint16_t) * 8 * (size_t)a.N * (size_t)a.R * (size_t)nb);
    a.ex = off; off = align_up(off + sizeof(int) * (size_t)a.N * (size_t)a.R);
    a.D = off; off = align_up(off + sizeof(double) * (size_t)nb * (size_t)nb);
    // the blocked panel solve's own slices: rows of X_>c and columns of L_>c,c
    const size_t pk = nb > 64 ? (size_t)(nb - 64) : 0;
    a.PS = off; off = align_up(off + sizeof(uint16_t) * 8 * (size_t)(n + 64) * pk);
    a.pex = off; off = align_up(off + sizeof(int) * (size_t)(n + 64));
    a.total = off;
    return a;
}

size_t adj_ws_bytes(int64_t n, int64_t nb, bool emu) {
    return emu ? adj_emu_layout(n, nb).total : adj_base_bytes(nb);
}

// Blocked reverse sweep of the right-looking Cholesky (lower convention).
// emu: the dominant product Lbar21 -= F22 L21 (F = Abar_L + Abar_L^T) runs
// FP64-accurate from exact BF16 slice products on the tensor cores, one
// launch per block column J of F22 (block J's rows of L21 as the other
// operand), the launches subtracting into Lbar21 in order of J.  F's block
// column k is sliced once, when the sweep has finalized it (its rows below
// the diagonal from Abar21, the diagonal block in full, and Abar21^T as rows
// of the later block columns' tensors); F never changes afterwards.
int potrf_backward_run(int64_t n, int64_t nb, const double* L, int64_t ldl, double* Ab,
                       int64_t ldab, char* ws, cudaStream_t s, bool emu) {
    double* P = (double*)ws;
    double* Y = (double*)(ws + align_up(sizeof(double) * nb * nb));
    double* Lc = (double*)(ws + 2 * align_up(sizeof(double) * nb * nb));
    double* part = (double*)(ws + 3 * align_up(sizeof(double) * nb * nb));
    const int64_t N = (n + nb - 1) / nb;
    const AdjEmu ae = adj_emu_layout(n, nb);
    DevStatus* est = (DevStatus*)(ws + ae.st);
    uint16_t* S = (uint16_t*)(ws + ae.S);
    int* ex = (int*)(ws + ae.ex);
    double* D = (double*)(ws + ae.D);
    uint16_t* PS = (uint16_t*)(ws + ae.PS);
    int* pex = (int*)(ws + ae.pex);
    const int64_t R = ae.R, Mtot = N * R;
    if (emu) ABFT_CUDA_TRY(cudaMemsetAsync(est, 0, sizeof(DevStatus), s));
    for (int64_t k = N - 1; k >= 0; --k) {
        const int64_t K0 = k * nb, kb = std::min(nb, n - K0), T0 = K0 + kb, m = n - T0;
        const double* L11 = L + K0 * ldl + K0;
        double* A11 = Ab + K0 * ldab + K0;
        if (m > 0) {
            // trailing update A22' = A22 - L21 L21^T  =>  Lbar21 -= (Abar22 + Abar22^T) L21
            timing_mark(PH_TMU, 1, s);
            if (emu) {
                // the columns of L21, block row J's piece as rows n .. n + kb of tensor J
                ABFT_CUDA_TRY(launch_slice_cols_chunked(L + T0 * ldl + K0, ldl, nb, m, kb, S, Mtot,
                                                        (k + 1) * R + n, R, ex, s));
                for (int64_t J = k + 1; J < N; ++J) {
                    EmuRectHost rc{};
                    rc.C = Ab + T0 * ldab + K0; rc.ldc = ldab;
                    rc.a0 = J * R + T0; rc.na = m;     // F's rows T0 .. n, block column J
                    rc.b0 = J * R + n; rc.nb = kb;     // L21's columns, block row J
                    rc.cdiv = 1; rc.frow = -1; rc.fcol = -1;
                    ABFT_CUDA_TRY(launch_tmu_emu(S, ex, Mtot, nb, nullptr, 0, 0, 0, 128, &rc, 1,
                                                 nullptr, 0, 0, est, s));
                }
            } else {
                GemmSeg g1{};
                g1.A = Ab + T0 * ldab + T0; g1.lda = ldab;
                g1.B = L + T0 * ldl + K0; g1.ldb = ldl;
                g1.C = Ab + T0 * ldab + K0; g1.ldc = ldab;
                g1.M = m; g1.N = kb; g1.K = m;
                ABFT_CUDA_TRY(launch_gemm_f64(&g1, 1, 2, 1, nullptr, 0, nullptr, s));
            }
            timing_mark(PH_TMU, 0, s);
            // L21 = A21 L11^{-T}  =>  Abar21 = Lbar21 L11^{-1}, Lbar11 -= tril(Abar21^T L21)
            timing_mark(PH_PU, 1, s);
            if (emu && kb == nb && kb % 64 == 0 && kb >= 128) {
                // blocked by 64 columns from the right, X_c L_cc = B_c - X_>c L_>c,c
                // (X = Abar21, B = Lbar21): the products FP64-accurate from BF16
                // slices on the tensor cores (rows of X_>c, columns of L_>c,c), the
                // 64-wide solves in FP64
                constexpr int64_t CW = 64;
                double* X = Ab + T0 * ldab + K0;
                const int64_t ncb = kb / CW;
                for (int64_t c = ncb - 1; c >= 0; --c) {
                    if (c < ncb - 1) {
                        const int64_t K = kb - (c + 1) * CW, Mt = m + CW;
                        ABFT_CUDA_TRY(launch_slice_panel(X + (c + 1) * CW, ldab, m, K, PS, Mt, 0,
                                                         pex, s));
                        ABFT_CUDA_TRY(launch_slice_cols(L11 + (c + 1) * CW * ldl + c * CW, ldl, K,
                                                        CW, PS, Mt, m, pex, s));
                        EmuRectHost rc{};
                        rc.C = X + c * CW; rc.ldc = ldab;
                        rc.a0 = 0; rc.na = m; rc.b0 = m; rc.nb = CW; rc.cdiv = 1;
                        rc.frow = -1; rc.fcol = -1;
                        ABFT_CUDA_TRY(launch_tmu_emu(PS, pex, Mt, K, nullptr, 0, 0, 0, 128, &rc, 1,
                                                     nullptr, 0, 0, est, s));
                    }
                    TrsmSeg sg{X + c * CW, ldab, m};
                    ABFT_CUDA_TRY(launch_trsm_rows(L11 + c * CW * (ldl + 1), ldl, CW, &sg, 1,
                                                   nullptr, s, false, true));
                }
            } else {
                TrsmSeg seg{Ab + T0 * ldab + K0, ldab, m};
                ABFT_CUDA_TRY(launch_trsm_rlt(L11, ldl, kb, &seg, 1, nullptr, nullptr, nullptr, s,
                                              false, true));
            }
            if (emu) {
                // F's block column k below the diagonal is final with Abar21: slice it
                // now (its rows for the later steps' products, and Abar21^T as rows
                // of the later block columns' tensors), then Lbar11 -= tril(Abar21^T
                // L21) from those rows and L21's: one launch per block row J, each
                // subtracting its piece into P in order of J
                ABFT_CUDA_TRY(launch_slice_panel(Ab + T0 * ldab + K0, ldab, m, kb, S, Mtot,
                                                 k * R + T0, ex, s));
                ABFT_CUDA_TRY(launch_slice_cols_chunked(Ab + T0 * ldab + K0, ldab, nb, m, kb, S,
                                                        Mtot, (k + 1) * R + K0, R, ex, s));
                ABFT_CUDA_TRY(cudaMemsetAsync(P, 0, sizeof(double) * kb * kb, s));
                for (int64_t J = k + 1; J < N; ++J) {
                    EmuRectHost rc{};
                    rc.C = P; rc.ldc = kb;
                    rc.a0 = J * R + K0; rc.na = kb;    // Abar21's columns, block row J
                    rc.b0 = J * R + n; rc.nb = kb;     // L21's columns, block row J
                    rc.cdiv = 1; rc.frow = -1; rc.fcol = -1;
                    ABFT_CUDA_TRY(launch_tmu_emu(S, ex, Mtot, nb, nullptr, 0, 0, 0, 128, &rc, 1,
                                                 nullptr, 0, 0, est, s));
                }
                ABFT_CUDA_TRY(launch_add_tril(P, A11, ldab, kb, s));
            } else {
                GemmSeg g3{};
                g3.A = Ab + T0 * ldab + K0; g3.lda = ldab;
                g3.B = L + T0 * ldl + K0; g3.ldb = ldl;
                g3.C = A11; g3.ldc = ldab;
                g3.M = kb; g3.N = kb; g3.K = m;
                g3.g = 1; g3.row0 = 0; g3.col0 = 0;
                ABFT_CUDA_TRY(launch_gemm_f64_splitk(g3, 1, 1, kAdjSplit, part, nullptr, s));
            }
            timing_mark(PH_PU, 0, s);
        }
        // L11 = chol(A11)  =>  Abar11 = Phi(S + S^T), S = L11^{-T} Phi(L11^T Lbar11) L11^{-1}
        timing_mark(PH_PD, 1, s);
        ABFT_CUDA_TRY(cudaMemsetAsync(P, 0, sizeof(double) * kb * kb, s));
        ABFT_CUDA_TRY(launch_copy_lower(L11, ldl, Lc, kb, kb, s));   // L11 with zeros above
        GemmSeg g4{};
        g4.A = Lc; g4.lda = kb;
        g4.B = A11; g4.ldb = ldab;
        g4.C = P; g4.ldc = kb;
        g4.M = kb; g4.N = kb; g4.K = kb;
        ABFT_CUDA_TRY(launch_gemm_f64(&g4, 1, 1, 1, nullptr, 0, nullptr, s));
        ABFT_CUDA_TRY(launch_phi_neg(P, kb, kb, s));
        TrsmSeg sp{P, kb, kb};
        ABFT_CUDA_TRY(launch_trsm_rlt(L11, ldl, kb, &sp, 1, nullptr, nullptr, nullptr, s, false, true));
        ABFT_CUDA_TRY(launch_transpose(P, kb, Y, kb, kb, s));
        TrsmSeg sy{Y, kb, kb};
        ABFT_CUDA_TRY(launch_trsm_rlt(L11, ldl, kb, &sy, 1, nullptr, nullptr, nullptr, s, false, true));
        ABFT_CUDA_TRY(launch_assemble_diag(Y, kb, A11, ldab, kb, s));
        timing_mark(PH_PD, 0, s);
        if (emu) {   // F's diagonal block is final: slice it for the steps still to come
            timing_mark(PH_OTHER, 1, s);
            ABFT_CUDA_TRY(launch_sym_diag(A11, ldab, kb, D, s));
            ABFT_CUDA_TRY(launch_slice_panel(D, kb, kb, kb, S, Mtot, k * R + K0, ex, s));
            timing_mark(PH_OTHER, 0, s);
        }
    }
    if (emu) {
        int err = 0;
        ABFT_CUDA_TRY(cudaMemcpyAsync(&err, &est->error, sizeof(int), cudaMemcpyDeviceToHost, s));
        ABFT_CUDA_TRY(cudaStreamSynchronize(s));
        if (err) return ABFT_ERR_TIMEOUT;
    }
    return ABFT_OK;
}

}  // namespace

extern "C" {

int abft_potrf_backward(int64_t n, int64_t nb, const double* L, int64_t ldl, const double* Lbar,
                        int64_t ldlb, double* Abar, int64_t ldab, int32_t sym, void* ws,
                        size_t* ws_bytes, void* stream) {
    return abft_potrf_backward_ex(n, nb, ABFT_F64, L, ldl, Lbar, ldlb, Abar, ldab, sym, ws,
                                  ws_bytes, stream);
}

int abft_potrf_backward_ex(int64_t n, int64_t nb, int32_t dtype, const double* L, int64_t ldl,
                           const double* Lbar, int64_t ldlb, double* Abar, int64_t ldab,
                           int32_t sym, void* ws, size_t* ws_bytes, void* stream) {
    if (n < 0) return -1;
    if (nb <= 0 || nb % 32 != 0 || nb > 512) return -2;
    if (dtype != ABFT_F64 && dtype != ABFT_F64_EMU)
        return dtype < 0 || dtype > 4 ? -12 : ABFT_ERR_UNSUPPORTED;
    const bool emu = dtype == ABFT_F64_EMU;
    if (emu && ((nb != 128 && nb != 256) || n % nb != 0)) return ABFT_ERR_UNSUPPORTED;
    const bool run = ws != nullptr && n > 0;
    if (run && L == nullptr) return -3;
    if (ldl < std::max<int64_t>(1, n)) return -4;
    if (run && Lbar == nullptr) return -5;
    if (ldlb < std::max<int64_t>(1, n)) return -6;
    if (run && Abar == nullptr) return -7;
    if (ldab < std::max<int64_t>(1, n)) return -8;
    if (ws_bytes == nullptr) return -11;
    const size_t need = adj_ws_bytes(n, nb, emu);
    if (ws == nullptr) {
        *ws_bytes = need;
        return ABFT_OK;
    }
    if (*ws_bytes < need) return -11;
    if (n == 0) return ABFT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    timing_mark(PH_OTHER, 1, s);
    ABFT_CUDA_TRY(launch_copy_lower(Lbar, ldlb, Abar, ldab, n, s));
    timing_mark(PH_OTHER, 0, s);
    int rc = potrf_backward_run(n, nb, L, ldl, Abar, ldab, (char*)ws, s, emu);
    if (rc != ABFT_OK) return rc;
    if (sym) ABFT_CUDA_TRY(launch_symmetrize_half(Abar, ldab, n, s));
    ABFT_CUDA_TRY(timing_collect(s));
    return ABFT_OK;
}

int abft_potrs_backward(int64_t n, int64_t nrhs, int64_t nb, const double* L, int64_t ldl,
                        const double* X, int64_t ldx, const double* Xbar, int64_t ldxb,
                        double* Bbar, int64_t ldbb, double* Lbar, int64_t ldlb, void* ws,
                        size_t* ws_bytes, void* stream) {
    if (n < 0) return -1;
    if (nrhs < 0 || nrhs > 16) return -2;
    if (nb <= 0 || nb % 32 != 0 || nb > 512) return -3;
    const bool run = ws != nullptr && n > 0 && nrhs > 0;
    if (run && L == nullptr) return -4;
    if (ldl < std::max<int64_t>(1, n)) return -5;
    if (run && X == nullptr) return -6;
    if (ldx < std::max<int64_t>(1, nrhs)) return -7;
    if (run && Xbar == nullptr) return -8;
    if (ldxb < std::max<int64_t>(1, nrhs)) return -9;
    if (run && Bbar == nullptr) return -10;
    if (ldbb < std::max<int64_t>(1, nrhs)) return -11;
    if (run && Lbar == nullptr) return -12;
    if (ldlb < std::max<int64_t>(1, n)) return -13;
    if (ws_bytes == nullptr) return -15;
    const size_t need = align_up(sizeof(double) * (size_t)n * 16) * 4 + align_up(potrs_inv_bytes(n, true));
    if (ws == nullptr) {
        *ws_bytes = need;
        return ABFT_OK;
    }
    if (*ws_bytes < need) return -15;
    if (!run) return ABFT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t blk = align_up(sizeof(double) * (size_t)n * 16);
    double* Xc = (double*)ws;
    double* Bc = (double*)((char*)ws + blk);
    double* U = (double*)((char*)ws + 2 * blk);
    double* V = (double*)((char*)ws + 3 * blk);
    timing_mark(PH_SOLVE, 1, s);
    // Bbar = A^{-1} Xbar
    ABFT_CUDA_TRY(launch_copy_d2d(Xbar, ldxb, Bbar, ldbb, n, (int)nrhs, s));
    ABFT_CUDA_TRY(launch_potrs_f64(n, (int)nrhs, nb, L, ldl, Bbar, ldbb,
                                   (double*)((char*)ws + 4 * blk), s));
    {
        cudaError_t ce = cudaSuccess;
        const int serr = potrs_error((char*)ws + 4 * blk, n, true, s, &ce);
        ABFT_CUDA_TRY(ce);
        if (serr) return ABFT_ERR_TIMEOUT;
    }
    // Lbar -= tril((Bbar X^T + X Bbar^T) L) = tril(Bbar (L^T X)^T + X (L^T Bbar)^T)
    ABFT_CUDA_TRY(launch_copy_d2d(X, ldx, Xc, 16, n, (int)nrhs, s));
    ABFT_CUDA_TRY(launch_copy_d2d(Bbar, ldbb, Bc, 16, n, (int)nrhs, s));
    ABFT_CUDA_TRY(launch_ltx(L, ldl, n, Xc, 16, (int)nrhs, U, 16, s));
    ABFT_CUDA_TRY(launch_ltx(L, ldl, n, Bc, 16, (int)nrhs, V, 16, s));
    ABFT_CUDA_TRY(launch_syr2k_lower(Bc, Xc, U, V, 16, n, (int)nrhs, Lbar, ldlb, s));
    timing_mark(PH_SOLVE, 0, s);
    ABFT_CUDA_TRY(timing_collect(s));
    return ABFT_OK;
}

int abft_logdet(int64_t n, const double* L, int64_t ldl, double* out, void* stream) {
    if (n < 0) return -1;
    if (n > 0 && L == nullptr) return -2;
    if (ldl < std::max<int64_t>(1, n)) return -3;
    if (out == nullptr) return -4;
    cudaStream_t s = (cudaStream_t)stream;
    ABFT_CUDA_TRY(launch_logdet(L, ldl, n, out, s));
    return ABFT_OK;
}

int abft_logdet_backward(int64_t n, const double* L, int64_t ldl, double gbar, double* Lbar,
                         int64_t ldlb, void* stream) {
    if (n < 0) return -1;
    if (n > 0 && L == nullptr) return -2;
    if (ldl < std::max<int64_t>(1, n)) return -3;
    if (n > 0 && Lbar == nullptr) return -5;
    if (ldlb < std::max<int64_t>(1, n)) return -6;
    ABFT_CUDA_TRY(launch_logdet_backward(L, ldl, n, gbar, Lbar, ldlb, (cudaStream_t)stream));
    return ABFT_OK;
}

int abft_tril(int64_t n, double* A, int64_t lda, void* stream) {
    if (n < 0) return -1;
    if (n > 0 && A == nullptr) return -2;
    if (lda < std::max<int64_t>(1, n)) return -3;
    ABFT_CUDA_TRY(launch_tril_zero(A, lda, n, (cudaStream_t)stream));
    return ABFT_OK;
}

}  // extern "C"

namespace {

// -------------------------------------------------------------- batched
// A captured graph holds every kernel argument, so the key holds them all:
// the buffers, the sizes and modes, the threshold scale (as its bit pattern)
// and the device the graph was instantiated on.
struct GraphKey {
    const void* items;
    int count, dtype, mode, grid;
    uint64_t tau_bits;
    int device;
    const void* status;
    const void* ws;
    void* stream;
    bool operator<(const GraphKey& o) const {
        return std::tie(items, count, dtype, mode, grid, tau_bits, device, status, ws, stream) <
               std::tie(o.items, o.count, o.dtype, o.mode, o.grid, o.tau_bits, o.device, o.status,
                        o.ws, o.stream);
    }
};
std::mutex g_graph_mu;
std::map<GraphKey, cudaGraphExec_t> g_graphs;

}  // namespace

extern "C" {

int abft_potrf_batched(int32_t count, const abft_batch_item* items, int32_t dtype, int32_t mode,
                       double tau_scale, abft_batch_status* status, int32_t use_graph, void* ws,
                       size_t* ws_bytes, void* stream) {
    if (count < 0) return -1;
    if (count > 0 && items == nullptr && ws != nullptr) return -2;
    if (dtype != ABFT_F64 && dtype != ABFT_F32) return dtype < 0 || dtype > 3 ? -3 : ABFT_ERR_UNSUPPORTED;
    if (mode != ABFT_MODE_NONE && mode != ABFT_MODE_FULL) return mode == ABFT_MODE_SINGLE ? ABFT_ERR_UNSUPPORTED : -4;
    if (count > 0 && status == nullptr && ws != nullptr) return -6;
    if (ws_bytes == nullptr) return -9;
    const bool f64 = dtype == ABFT_F64;
    // sized for the largest grid, so that a workspace stays valid whatever
    // abft_batched_set_ctas_per_sm chooses later
    const size_t need = align_up(batched_scratch_bytes(batched_max_grid(f64), f64)) + 256;
    if (ws == nullptr) {
        *ws_bytes = need;
        return ABFT_OK;
    }
    if (*ws_bytes < need) return -9;
    if (count == 0) return ABFT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int* queue = (unsigned int*)((char*)ws + align_up(batched_scratch_bytes(batched_max_grid(f64), f64)));
    if (!use_graph) {
        ABFT_CUDA_TRY(launch_potrf_batched(items, count, f64, mode, tau_scale, status, ws, queue, s));
        ABFT_CUDA_TRY(timing_collect(s));
        return ABFT_OK;
    }
    int device = 0;
    ABFT_CUDA_TRY(cudaGetDevice(&device));
    uint64_t tau_bits = 0;
    std::memcpy(&tau_bits, &tau_scale, sizeof(tau_bits));
    GraphKey key{items, count, dtype, mode, batched_grid(f64), tau_bits, device, status, ws, stream};
    cudaGraphExec_t exec = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_graph_mu);
        auto itg = g_graphs.find(key);
        if (itg != g_graphs.end()) exec = itg->second;
    }
    if (exec == nullptr) {
        ABFT_CUDA_TRY(batched_prepare());   // kernel attributes outside the capture
        (void)batched_grid(f64);
        cudaStream_t cs;
        ABFT_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph;
        ABFT_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        cudaError_t le = launch_potrf_batched(items, count, f64, mode, tau_scale, status, ws, queue, cs);
        cudaError_t ee = cudaStreamEndCapture(cs, &graph);
        cudaStreamDestroy(cs);
        if (le != cudaSuccess || ee != cudaSuccess) return ABFT_ERR_CUDA;
        cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return ABFT_ERR_CUDA;
        std::lock_guard<std::mutex> lk(g_graph_mu);
        g_graphs[key] = exec;
    }
    ABFT_CUDA_TRY(cudaGraphLaunch(exec, s));
    note_launch();
    ABFT_CUDA_TRY(timing_collect(s));
    return ABFT_OK;
}

int abft_batched_set_ctas_per_sm(int32_t ctas) {
    if (ctas < 0) return -1;
    return batched_set_ctas_per_sm(ctas);
}

int abft_batched_graph_reset(void) {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (auto& kv : g_graphs) cudaGraphExecDestroy(kv.second);
    g_graphs.clear();
    return ABFT_OK;
}

}  // extern "C"

namespace {

}  // namespace

extern "C" {

const char* abft_version(void) { return "abft-b300 0.1 (sm_103a)"; }

int64_t abft_launch_count(void) { return (int64_t)g_launches.load(); }

int abft_set_lookahead(int32_t on) {
    return g_lookahead.exchange(on != 0 ? 1 : 0);
}

int abft_timing_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_tmu);
    g_timing = on != 0;
    for (int i = 0; i < PH_COUNT; ++i) { g_ms[i] = 0.0; g_calls[i] = 0; }
    g_marks.clear();
    g_intervals.clear();
    g_pool_used = 0;
    return ABFT_OK;
}

int abft_timing_marks(int32_t* phase, int64_t* step, double* ms, int32_t max) {
    if (max < 0 || (max > 0 && (phase == nullptr || step == nullptr || ms == nullptr))) return -1;
    std::lock_guard<std::mutex> lk(g_tmu);
    const int32_t n = (int32_t)std::min<size_t>(g_intervals.size(), (size_t)INT32_MAX);
    for (int32_t i = 0; i < n && i < max; ++i) {
        phase[i] = g_intervals[i].phase;
        step[i] = g_intervals[i].step;
        ms[i] = g_intervals[i].ms;
    }
    return n;
}

// Enhanced algorithmic slack prediction (Sec. 3.2.1): the time of an
// operation at iteration k from its profiled times at the last p = 4
// iterations, each scaled by the ratio of the operation's work between the
// two iterations and weighted 1/2, 1/4, 1/8, 1/8 (nearest first).
int abft_predict_step_times(const double* T, const double* W, int64_t nsteps, double* pred) {
    if (nsteps < 0 || (nsteps > 0 && (T == nullptr || W == nullptr || pred == nullptr))) return -1;
    static const double wt[4] = {0.5, 0.25, 0.125, 0.125};
    for (int64_t k = 0; k < nsteps; ++k) {
        double num = 0.0, wsum = 0.0;
        for (int i = 1; i <= 4 && k - i >= 0; ++i) {
            const int64_t j = k - i;
            if (!(W[j] > 0.0) || !(T[j] >= 0.0)) continue;   // no work, or not measured
            num += wt[i - 1] * (W[k] / W[j]) * T[j];
            wsum += wt[i - 1];
        }
        // fewer than four usable neighbours: their weights are renormalized
        pred[k] = wsum > 0.0 ? num / wsum : std::nan("");
    }
    return ABFT_OK;
}

// Work of one operation of iteration k of the blocked Cholesky as this
// implementation performs it (flops; elements for the verification):
// PD kb^3 / 3, PU m kb^2, TMU 2 kb E (E = elements of the lower block
// triangle of the trailing matrix, diagonal blocks full), verify E + m kb.
double abft_chol_step_work(int64_t n, int64_t nb, int32_t phase, int64_t k) {
    if (n <= 0 || nb <= 0 || k < 0) return 0.0;
    const int64_t K0 = k * nb;
    if (K0 >= n) return 0.0;
    const int64_t kb = std::min(nb, n - K0), T0 = K0 + kb, m = n - T0;
    double E = 0.0;
    for (int64_t r0 = 0; r0 < m; r0 += nb) {
        const int64_t rows = std::min(nb, m - r0);
        E += (double)rows * (double)(r0 + rows);
    }
    switch (phase) {
        case PH_PD: return (double)kb * kb * kb / 3.0;
        case PH_PU: return (double)m * kb * kb;
        case PH_TMU: return 2.0 * kb * E;
        case PH_VERIFY: return E + (double)m * kb;
        default: return 0.0;
    }
}

int abft_timing_read(double* ms, int64_t* count, int32_t nphase) {
    if (ms == nullptr || nphase < 0) return -1;
    std::lock_guard<std::mutex> lk(g_tmu);
    for (int i = 0; i < nphase && i < PH_COUNT; ++i) {
        ms[i] = g_ms[i];
        if (count) count[i] = g_calls[i];
    }
    return ABFT_OK;
}

const char* abft_strerror(int32_t code) {
    if (code == ABFT_OK) return "ok";
    if (code > 0) return "non-positive or zero pivot (info)";
    switch (code) {
        case ABFT_ERR_UNCORRECTABLE: return "uncorrectable error reported by the checksums";
        case ABFT_ERR_TIMEOUT: return "bounded device wait gave up";
        case ABFT_ERR_CUDA: return "CUDA launch or runtime error";
        case ABFT_ERR_UNSUPPORTED: return "unsupported combination of arguments";
        case ABFT_ERR_TOO_LARGE: return "problem needs more workspace than the built-in scratch array";
        default: return "invalid argument";
    }
}

int abft_potrf(int64_t n, int64_t nb, int32_t dtype, int32_t mode, double* A, int64_t lda,
               const abft_fault* faults, int32_t nfaults, double tau_scale, abft_report* rep,
               void* ws, size_t* ws_bytes, void* stream) {
    if (n < 0) return -1;
    if (nb <= 0 || nb % 32 != 0 || nb > 512) return -2;
    if (dtype < 0 || dtype > 4) return -3;
    const bool mixed = dtype == ABFT_MIXED_BF16 || dtype == ABFT_MIXED_F16;
    const bool emu = dtype == ABFT_F64_EMU;
    if (dtype == ABFT_F32 || (mixed && nb % 128 != 0) || (emu && nb != 128 && nb != 256))
        return ABFT_ERR_UNSUPPORTED;
    if (mode < ABFT_MODE_NONE || mode > ABFT_MODE_FULL) return -4;
    if (n > 0 && A == nullptr && ws != nullptr) return -5;
    if (lda < std::max<int64_t>(1, n)) return -6;
    if (nfaults < 0) return -8;
    if (nfaults > 0 && faults == nullptr) return -7;
    if (!(tau_scale > 0.0)) return -9;
    if (ws_bytes == nullptr) return -12;
    const int64_t N = (n + nb - 1) / nb;
    for (int f = 0; f < nfaults; ++f) {
        if (!chol_fault_ok(faults[f], n, nb, N)) return -7;
        int same = 0;  // compute faults are carried as TMU launch arguments
        for (int h = 0; h < nfaults; ++h)
            same += faults[h].kind == ABFT_FAULT_COMPUTE && faults[h].step == faults[f].step;
        if (same > MAX_CF) return -7;
    }
    const CholWs w = chol_ws(n, nb, mode, mixed, emu);
    if (ws == nullptr) {
        *ws_bytes = w.total;
        return ABFT_OK;
    }
    if (*ws_bytes < w.total) return -12;
    cudaStream_t s = (cudaStream_t)stream;
    char* base = (char*)ws;
    DevStatus* st = (DevStatus*)(base + w.st);
    ABFT_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(DevStatus), s));
    if (n > 0) {
        int rc = chol_steps(n, nb, mode, nullptr, A, lda, faults, nfaults, tau_scale, w, base,
                            s, dtype);
        if (rc != ABFT_OK) return rc;
    }
    ABFT_CUDA_TRY(timing_collect(s));
    if (rep) return finish_report(st, rep, s);
    return ABFT_OK;
}

int abft_syrk_mixed(int64_t m, int64_t k, int64_t g, int32_t dtype, const double* P, int64_t ldp,
                    double* C, int64_t ldc, uint16_t* Pq, double* sigma, int32_t* timed_out,
                    void* ws, size_t* ws_bytes, void* stream) {
    if (m < 0) return -1;
    if (k <= 0 || k % 64 != 0 || k > 512) return -2;
    if (g <= 0 || g % 128 != 0) return -3;
    if (dtype != ABFT_MIXED_BF16 && dtype != ABFT_MIXED_F16) return -4;
    if (m > 0 && P == nullptr && ws != nullptr) return -5;
    if (ldp < k) return -6;
    if (m > 0 && C == nullptr && ws != nullptr) return -7;
    if (ldc < std::max<int64_t>(1, m)) return -8;
    if (m > 0 && ws != nullptr && (Pq == nullptr || ((uintptr_t)Pq & 15) != 0)) return -9;
    if (m > 0 && sigma == nullptr && ws != nullptr) return -10;
    if (ws_bytes == nullptr) return -13;
    const int64_t nt = (m + g - 1) / g;
    const size_t st_off = 0, ts_off = align_up(sizeof(DevStatus));
    const size_t need = ts_off + align_up(sizeof(double) * (size_t)std::max<int64_t>(1, nt) * (size_t)k);
    if (ws == nullptr) {
        *ws_bytes = need;
        return ABFT_OK;
    }
    if (*ws_bytes < need) return -13;
    if (m == 0) return ABFT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    DevStatus* st = (DevStatus*)((char*)ws + st_off);
    double* tsum = (double*)((char*)ws + ts_off);
    const int bf16 = dtype == ABFT_MIXED_BF16 ? 1 : 0;
    ABFT_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(DevStatus), s));
    ABFT_CUDA_TRY(launch_quant_panel(P, ldp, 0, m, k, g, 0, nt, bf16, Pq, sigma, tsum, k, 0, s));
    ABFT_CUDA_TRY(launch_tmu_mixed(Pq, m, k, bf16, C, ldc, g, 0, sigma, nullptr, 0, st, s, 0, 0, 0));
    if (timed_out) {
        int err = 0;
        ABFT_CUDA_TRY(cudaMemcpyAsync(&err, &st->error, sizeof(int), cudaMemcpyDeviceToHost, s));
        ABFT_CUDA_TRY(cudaStreamSynchronize(s));
        *timed_out = err != 0;
        if (err) return ABFT_ERR_TIMEOUT;
    }
    return ABFT_OK;
}

int abft_potrf_sched(int64_t n, int64_t nb, int32_t dtype, const int32_t* modes, double* A,
                     int64_t lda, const abft_fault* faults, int32_t nfaults, double tau_scale,
                     abft_report* rep, void* ws, size_t* ws_bytes, void* stream) {
    if (n < 0) return -1;
    if (nb <= 0 || nb % 32 != 0 || nb > 512) return -2;
    const int64_t N = (n + nb - 1) / nb;
    if (N > 0 && modes == nullptr) return -4;
    int32_t top = ABFT_MODE_NONE;
    for (int64_t k = 0; k < N; ++k) {
        if (modes[k] < ABFT_MODE_NONE || modes[k] > ABFT_MODE_FULL) return -4;
        top = std::max(top, modes[k]);
    }
    // argument checks and the workspace size of the strongest mode used
    size_t need = 0;
    int rc = abft_potrf(n, nb, dtype, top, nullptr, lda, faults, nfaults, tau_scale, nullptr,
                        nullptr, &need, nullptr);
    if (rc != ABFT_OK) return rc;
    if (ws_bytes == nullptr) return -12;
    if (ws == nullptr) {
        *ws_bytes = need;
        return ABFT_OK;
    }
    if (n > 0 && A == nullptr) return -5;
    if (*ws_bytes < need) return -12;
    const bool mixed = dtype == ABFT_MIXED_BF16 || dtype == ABFT_MIXED_F16;
    const CholWs w = chol_ws(n, nb, top, mixed, dtype == ABFT_F64_EMU);
    cudaStream_t s = (cudaStream_t)stream;
    char* base = (char*)ws;
    DevStatus* st = (DevStatus*)(base + w.st);
    ABFT_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(DevStatus), s));
    if (n > 0) {
        rc = chol_steps(n, nb, top, modes, A, lda, faults, nfaults, tau_scale, w, base, s, dtype);
        if (rc != ABFT_OK) return rc;
    }
    ABFT_CUDA_TRY(timing_collect(s));
    if (rep) return finish_report(st, rep, s);
    return ABFT_OK;
}

}  // extern "C"
