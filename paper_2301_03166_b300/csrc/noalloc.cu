// noalloc.cu -- abft_potrf_noalloc: the ABFT Cholesky for callers that must not
// allocate device memory.
//
// Some host programs own every byte of device memory themselves (a framework
// whose caching allocator or fixed arena manages the whole GPU, or a plugin
// that is not allowed to grow the process's device footprint) and so can
// neither call cudaMalloc nor hand this library a workspace.  For them the
// workspace lives in one file-scope device array, sized at build time and
// created when the library's device code is loaded on a GPU; it then stays
// allocated on that GPU until the process exits.
//
// The array's name means nothing to host code (it is a host-side stand-in);
// the device address is looked up once per device with cudaGetSymbolAddress,
// with that device current, on the first call made on it.  All calls share
// the array and it keeps whatever the last call left: the status block at its
// start is cleared by every call before use (the rest is written before it
// is read), and two calls whose work overlaps on the GPU race on it.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kScratchBytes = ABFT_NOALLOC_SCRATCH_BYTES;   // 16 MiB per device
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// The library drives one GPU per process (its launchers set per-device kernel
// attributes once per process, and the look-ahead keeps state for device
// indices below 16), so the address cache covers the same 16 indices.
constexpr int kMaxDevices = 16;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device (looked up once per device).
int scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ABFT_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_addr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return ABFT_ERR_CUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return ABFT_OK;
}

}  // namespace

extern "C" {

int abft_potrf_noalloc(int64_t n, int64_t nb, int32_t dtype, int32_t mode, double* A, int64_t lda,
                       const abft_fault* faults, int32_t nfaults, double tau_scale,
                       abft_report* rep, void* stream) {
    size_t need = 0;
    int rc = abft_potrf(n, nb, dtype, mode, A, lda, faults, nfaults, tau_scale, nullptr, nullptr,
                        &need, nullptr);
    if (rc != ABFT_OK) return rc;
    if (need > kScratchBytes) return ABFT_ERR_TOO_LARGE;
    void* ws = nullptr;
    rc = scratch_address(&ws);
    if (rc != ABFT_OK) return rc;
    size_t have = kScratchBytes;
    return abft_potrf(n, nb, dtype, mode, A, lda, faults, nfaults, tau_scale, rep, ws, &have,
                      stream);
}

}  // extern "C"
