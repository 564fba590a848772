// probe_fp64.cu -- abft_fp64_pipe_probe: the microbenchmark behind the FP64
// design of this library.  B300 has two ways to run FP64 multiply-adds: the
// FP64 FMA (DFMA) on the CUDA cores and the FP64 tensor-core MMA
// (mma.sync m8n8k4 .f64).  Each kernel runs independent chains on every SM
// (so the pipe, not latency, is the limit) and reports FLOP/s from CUDA events.
#include "common.cuh"

namespace abft {
namespace {

constexpr int PT = 256;        // threads per CTA
__device__ double g_sink;      // keeps the chains' results alive
constexpr int PCH = 8;         // independent chains per thread

__global__ void __launch_bounds__(PT) k_dfma_probe(int iters) {
    double a[PCH];
    const double x = 1.0 + 1e-9 * threadIdx.x, y = 1e-12;
#pragma unroll
    for (int c = 0; c < PCH; ++c) a[c] = 1.0 + c * 1e-3 + blockIdx.x * 1e-6;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < PCH; ++c) a[c] = fma(a[c], x, y);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < PCH; ++c) s += a[c];
    if (s == 12345.678) g_sink = s;   // never true; the compiler cannot drop the chains
}

// One m8n8k4 FP64 MMA per chain and step (8 x 8 x 4 multiply-adds per warp);
// PCH / 2 independent accumulators per warp.
__global__ void __launch_bounds__(PT) k_dmma_probe(int iters) {
    constexpr int NA = PCH / 2;
    double c0[NA], c1[NA];
    const double av = 1.0 + 1e-9 * threadIdx.x, bv = 1e-3;
#pragma unroll
    for (int c = 0; c < NA; ++c) { c0[c] = c * 1e-3; c1[c] = c * 2e-3; }
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < NA; ++c)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(c0[c]), "+d"(c1[c])
                         : "d"(av), "d"(bv));
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < NA; ++c) s += c0[c] + c1[c];
    if (s == 12345.678) g_sink = s;
}

}  // namespace
}  // namespace abft

using namespace abft;

extern "C" int abft_fp64_pipe_probe(int32_t which, int64_t iters, double* tflops_out, void* stream) {
    if (which < 0 || which > 1) return -1;
    if (iters <= 0 || iters > (1 << 24)) return -2;
    if (tflops_out == nullptr) return -3;
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = 4 * num_sms();
    cudaEvent_t e0, e1;
    ABFT_CUDA_TRY(cudaEventCreate(&e0));
    ABFT_CUDA_TRY(cudaEventCreate(&e1));
    auto run = [&]() {
        if (which == 0) k_dfma_probe<<<grid, PT, 0, s>>>((int)iters);
        else k_dmma_probe<<<grid, PT, 0, s>>>((int)iters);
        note_launch();
    };
    run();   // warm-up
    ABFT_CUDA_TRY(cudaEventRecord(e0, s));
    run();
    ABFT_CUDA_TRY(cudaEventRecord(e1, s));
    ABFT_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    ABFT_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ABFT_CUDA_TRY(cudaGetLastError());
    // DFMA: 2 flops per chain step and thread; DMMA: 8 x 8 x 4 x 2 per warp MMA
    const double threads = (double)grid * PT;
    const double flops = which == 0 ? threads * PCH * 2.0 * (double)iters
                                    : threads / 32.0 * (PCH / 2) * 512.0 * (double)iters;
    *tflops_out = flops / (ms * 1e-3) / 1e12;
    return ABFT_OK;
}
