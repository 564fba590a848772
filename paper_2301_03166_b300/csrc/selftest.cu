// selftest.cu -- abft_wait_selftest: runs the library's two bounded waits on
// purpose-built cases, so that their give-up path can be tested without a
// fault: the cooperative kernels' grid barrier (grid_barrier) and the
// tensor-core kernels' mbarrier wait (mbar_wait, with TMEM held).  A wait
// that cannot complete gives up after its limit, records a timeout in the
// status block, releases what the CTA holds and returns; the host reads the
// status and reports ABFT_ERR_TIMEOUT, and the context stays usable.
#include "common.cuh"
#include "tc_util.cuh"

namespace abft {
namespace {

using namespace tc;

// Two CTAs meet at one grid barrier.  absent = 1: CTA 1 returns without
// arriving, so CTA 0's wait cannot complete and gives up after limit_ns.
__global__ void k_barrier_probe(DevStatus* st, int absent, unsigned long long limit_ns) {
    if (absent && blockIdx.x == 1) return;
    unsigned long long passed = 0;
    grid_barrier(st, gridDim.x, passed, limit_ns);
}

// One CTA holding 32 TMEM columns waits for phase 0 of an mbarrier that
// expects two arrivals; missing = 1: only one arrives, the wait gives up after
// limit_ns, the CTA records the timeout, frees its TMEM and returns.
__global__ void k_mbar_probe(DevStatus* st, int missing, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 2);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(32u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
        if (!missing)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
        if (!mbar_wait(&bar, 0u, limit_ns)) atomicExch(&st->error, 2);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    __syncwarp();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32u));
    }
}

}  // namespace
}  // namespace abft

using namespace abft;

extern "C" int abft_wait_selftest(int32_t which, int64_t limit_ns, int32_t* error_out,
                                  void* ws, size_t* ws_bytes, void* stream) {
    if (which < 0 || which > 3) return -1;
    if (limit_ns <= 0 || limit_ns > 2000000000ll) return -2;
    if (ws_bytes == nullptr) return -5;
    const size_t need = sizeof(DevStatus);
    if (ws == nullptr) {
        *ws_bytes = need;
        return ABFT_OK;
    }
    if (*ws_bytes < need) return -5;
    cudaStream_t s = (cudaStream_t)stream;
    DevStatus* st = (DevStatus*)ws;
    ABFT_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(DevStatus), s));
    const int incomplete = (which == 0 || which == 1) ? 1 : 0;
    if (which == 0 || which == 2)
        k_barrier_probe<<<2, 32, 0, s>>>(st, incomplete, (unsigned long long)limit_ns);
    else
        k_mbar_probe<<<1, 128, 0, s>>>(st, incomplete, (unsigned long long)limit_ns);
    note_launch();
    ABFT_CUDA_TRY(cudaGetLastError());
    int err = 0;
    ABFT_CUDA_TRY(cudaMemcpyAsync(&err, &st->error, sizeof(int), cudaMemcpyDeviceToHost, s));
    ABFT_CUDA_TRY(cudaStreamSynchronize(s));
    if (error_out) *error_out = err;
    return err ? ABFT_ERR_TIMEOUT : ABFT_OK;
}
