// mm_demag_noalloc: the demag field through the same five FFT passes as
// mm_heff, with every intermediate spectrum kept in one fixed device array
// that belongs to this file, so a call performs no device (or host) memory
// allocation.
//
// Who needs it: code that may not call cudaMalloc at the moment it wants a
// field, e.g. a framework whose allocator owns all device memory and forbids
// side allocations, or a real-time loop that must not stall on the CUDA
// allocator (cudaMalloc and cudaFree can synchronise the device).  Such a
// caller still owns and passes every input and output buffer.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "demag.h"
#include "mm.h"

namespace {

// Fixed scratch for the x- and y-spectra (S1, S2).  Every GPU that loads this
// library's module keeps these bytes until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;   // 64 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
// device address of g_noalloc_scratch per device, looked up on the first call
// on that device and kept for the process (a cudaDeviceReset invalidates it)
void* g_scratch_ptr[128] = {nullptr};
thread_local char g_msg[256];

mm_status err(mm_status st, const char* what) {
    mm::set_last_error(what);
    return st;
}

mm_status err_msg(mm_status st) {
    mm::set_last_error(g_msg);
    return st;
}

}  // namespace

extern "C" mm_status mm_demag_noalloc(const mm_grid* grid, mm_precision precision, const void* m,
                                      const void* Ms_cell, double Ms, const void* spectrum, void* h_out,
                                      void* cuda_stream) {
    using namespace mm;
    if (!grid || !m || !spectrum || !h_out) return err(MM_EINVAL, "mm_demag_noalloc: null argument");
    if (precision != MM_FP64 && precision != MM_FP32_FIELDS) return err(MM_EINVAL, "mm_demag_noalloc: bad precision");
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || (double)grid->nx * grid->ny * grid->nz >= 2147483648.0)
        return err(MM_EINVAL, "mm_demag_noalloc: grid sizes must be >= 1");
    const int LX = fft_extent(grid->nx), LY = fft_extent(grid->ny), LZ = fft_extent(grid->nz);
    if (LX > kMaxFft || LY > kMaxFft || LZ > kMaxFft)
        return err(MM_EINVAL, "mm_demag_noalloc: padded FFT extent above 4096");
    const int KX = LX / 2 + 1;
    // spectra rows use stride KX here (the layout of mm_demag_spectrum_host)
    DemagDims d{grid->nx, grid->ny, grid->nz, LX, LY, LZ, KX, KX, nullptr};   // no error word: classic kernels
    const size_t csz = precision == MM_FP64 ? 2 * sizeof(double) : 2 * sizeof(float);
    const size_t s1 = 3 * csz * (size_t)grid->ny * grid->nz * KX;
    const size_t s2 = LY > 1 ? 3 * csz * (size_t)grid->nz * LY * KX : 0;
    const size_t s1a = (s1 + 255) / 256 * 256;
    if (s1a + s2 > kNoAllocScratchBytes) {
        snprintf(g_msg, sizeof(g_msg),
                 "mm_demag_noalloc: grid %d x %d x %d needs %zu bytes of spectrum scratch, above the fixed "
                 "maximum of %zu bytes", grid->nx, grid->ny, grid->nz, s1a + s2, kNoAllocScratchBytes);
        return err_msg(MM_EINVAL);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128)
        return err(MM_ECUDA, "mm_demag_noalloc: cudaGetDevice failed");
    void* base = nullptr;
    {
        // one-time set-up per device, on the device that is current
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) {
                snprintf(g_msg, sizeof(g_msg), "mm_demag_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
                return err_msg(MM_ECUDA);
            }
            g_scratch_ptr[dev] = p;
        }
        base = g_scratch_ptr[dev];
    }
    cudaError_t e = ensure_twiddles_on(dev);
    if (e != cudaSuccess) {
        snprintf(g_msg, sizeof(g_msg), "mm_demag_noalloc: twiddle upload: %s", cudaGetErrorString(e));
        return err_msg(MM_ECUDA);
    }
    KernelTimer off;   // disabled: records nothing, allocates nothing
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned char* b = static_cast<unsigned char*>(base);
    // Every scratch element a pass reads was written earlier in the same call
    // (P1 writes all of S1, P2 all of S2, P3 rewrites S2 in place, P4 all of
    // S1), so nothing needs clearing between calls.
    if (precision == MM_FP64) {
        demag_apply<double>(d, (const double*)m, (const double*)Ms_cell, Ms, (double2*)b,
                            (double2*)(b + s1a), (const double*)spectrum, (double*)h_out, st, &off);
    } else {
        demag_apply<float>(d, (const float*)m, (const float*)Ms_cell, (float)Ms, (float2*)b, (float2*)(b + s1a),
                           (const float*)spectrum, (float*)h_out, st, &off);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(g_msg, sizeof(g_msg), "mm_demag_noalloc: launch: %s", cudaGetErrorString(e));
        return err_msg(MM_ECUDA);
    }
    return MM_OK;
}
