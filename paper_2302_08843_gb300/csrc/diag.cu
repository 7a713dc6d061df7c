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
