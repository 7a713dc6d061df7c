// Diagnostic entry point: a device wait that runs out.  One CTA waits on an
// mbarrier that nothing ever completes, with the same bounded polling the TMA
// kernels use for their copies; when the budget is spent it writes the
// timeout code into the state's device error word and returns, as a TMA
// kernel whose copy never landed would.  No copy is issued, so nothing is left
// in flight when the kernel exits.
#include "demag.h"
#include "tma.cuh"

namespace mm {

__global__ void diag_wait_kernel(int* err, uint32_t spins) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    bool ok = false;
    if (threadIdx.x == 0)
        for (uint32_t it = 0; it < spins && !ok; ++it) ok = mbar_try_wait(&bar, 0);
    if (__syncthreads_or(threadIdx.x == 0 && !ok)) {
        if (threadIdx.x == 0) atomicExch(err, kErrTmaTimeout);
    }
}

void launch_diag_wait(int* err, unsigned spins, cudaStream_t st) {
    diag_wait_kernel<<<1, 32, 0, st>>>(err, spins);
}

}  // namespace mm

// ------------------------------------------------------------------------
// FP64 FMA rate probe: every thread runs kFmaChains independent chains of
// dependent fused multiply-adds x <- x a + b (|a| < 1, so the values stay
// bounded), enough chains per warp that the FP64 pipe, not the dependency
// latency, sets the rate.  The sum of the chains is written only if it equals
// an impossible value, so the work is kept but nothing is stored.
namespace mm {

constexpr int kFmaChains = 8;

__global__ void __launch_bounds__(256) fp64_fma_probe_kernel(double* sink, int iters, double a, double b) {
    double x[kFmaChains];
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) x[c] = 1e-3 * (threadIdx.x + c) + 1e-7 * blockIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kFmaChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) s += x[c];
    if (s == -1.2345e300) sink[0] = s;
}

double launch_fp64_fma_probe(double* sink, int blocks, int iters, cudaStream_t st) {
    fp64_fma_probe_kernel<<<blocks, 256, 0, st>>>(sink, iters, 0.999999, 1e-6);
    return 2.0 * kFmaChains * (double)iters * 256.0 * (double)blocks;
}

}  // namespace mm
