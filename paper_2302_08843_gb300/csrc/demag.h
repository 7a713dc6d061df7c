// Internal interfaces between the C-ABI layer and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace mm {

// Lengths with a compiled mixed-radix engine (fft_engine.cuh, FftMixed); every
// other 7-smooth even length up to kMaxFft that is not a power of two runs the
// runtime-plan passes of demag_rt.cu.
bool fft_rt_length(int L);

// Padded FFT extent of an axis of n cells (Sec. 4.4 zero padding, P >= 2n):
// 1 for one cell, otherwise the smallest even 7-smooth length 2^a 3^b 5^c 7^d
// >= 2n up to kMaxRtFft, beyond that the next power of two (kMaxFft at most;
// larger values are refused by the callers).  Even lengths keep the
// two-real-rows packing of the x passes; the bound kMaxRtFft keeps the FP64
// z pass's four line buffers within shared memory.
constexpr int kMaxRtFft = 3200;
inline int fft_extent(int n) {
    if (n <= 1) return 1;
    for (int L = 2 * n; L <= kMaxRtFft; L += 2) {
        int v = L;
        for (int p : {2, 3, 5, 7})
            while (v % p == 0) v /= p;
        if (v == 1) return L;
    }
    int best = 1;       // beyond: the next power of two (above kMaxFft: refused by the callers)
    while (best < 2 * n) best <<= 1;
    return best;
}

struct DemagDims {
    int nx, ny, nz;      // cells
    int LX, LY, LZ;      // padded FFT extents
    int KX;              // LX/2 + 1 spectrum columns
    int KXS;             // row stride of S1/S2 and of the tensor spectrum (elements)
    int* err = nullptr;  // device error word for bounded-wait failures; null: no TMA kernels
    int nb = 1;          // grids of this shape stacked as a leading batch dimension
    const void* Ms_b = nullptr;   // per-grid Ms (nb values of the real type) or null
    // 2-D grids: the z-pass kernels run along y (nz' = ny, Pz' = Py); the
    // odd components' mirror signs then come from the transformed axis
    int yz_swap = 0;
    // non-equidistant layers (Sec. 4.4): no transform along z; the nz layers
    // are coupled densely at every lateral wave number (p3_layers).  lh holds
    // the nz thicknesses in the real type of the passes.
    int layers = 0;
    const void* lh = nullptr;
};

// most layers a non-equidistant stack may have (shared memory of p3_layers)
constexpr int kMaxLayers = 64;

// CUDA-event timing of kernel launches on a stream (inactive unless enabled).
struct KernelTimer {
    bool on = false;
    struct Rec { int name; cudaEvent_t a, b; };
    std::vector<std::string> names;
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    int cur = -1;
    cudaEvent_t cur_a = nullptr;
    void begin(cudaStream_t st, const char* name);
    void end(cudaStream_t st);
    void reset();
    void destroy();
};

template <typename T>
void demag_apply(const DemagDims& d, const T* m, const T* Ms_cell, T Ms, typename Cplx<T>::type* S1,
                 typename Cplx<T>::type* S2, const T* tens, T* h, cudaStream_t st, KernelTimer* tm);

// P1 (optional) .. P4: leaves the x-spectrum of h in S1
template <typename T>
void demag_front(const DemagDims& d, const T* m, const T* Ms_cell, T Ms, bool need_p1, typename Cplx<T>::type* S1,
                 typename Cplx<T>::type* S2, const T* tens, cudaStream_t st, KernelTimer* tm);

// runtime-plan passes for the lengths fft_rt_length accepts (demag_rt.cu)
template <typename T>
void launch_rt_x_fwd(const DemagDims& d, const T* m, const T* Ms_cell, T Ms, typename Cplx<T>::type* S1,
                     cudaStream_t st);
template <typename T>
void launch_rt_x_inv(const DemagDims& d, const typename Cplx<T>::type* S1, T* h, cudaStream_t st);
template <typename T, int DIR>
void launch_rt_y(const DemagDims& d, const typename Cplx<T>::type* in, typename Cplx<T>::type* out,
                 cudaStream_t st);
template <typename T>
void launch_rt_z(const DemagDims& d, typename Cplx<T>::type* S2, const T* tens, cudaStream_t st);
// copy the runtime-plan lengths' twiddle tables to the current device
cudaError_t upload_twiddles_rt();

// diagnostic: one CTA whose bounded wait on a never-completed mbarrier runs out
void launch_diag_wait(int* err, unsigned spins, cudaStream_t st);
// FP64 FMA rate probe (blocks x 256 threads, iters FMAs per chain); returns the FLOPs it enqueued
double launch_fp64_fma_probe(double* sink, int blocks, int iters, cudaStream_t st);

template <typename T> struct AdjParams;
template <typename T> void launch_adj_prep(const AdjParams<T>& p, cudaStream_t st);
template <typename T> void launch_adj_finish(const AdjParams<T>& p, cudaStream_t st);
template <typename T>
void launch_adj_renorm(const T* y, const T* lam, T* lam_y, T* lam_acc, T* u, double cb, int N, cudaStream_t st);

// number of doubles per block in the reduction partials
constexpr int kNPart = 8;
// partial / scalar slots
enum { R_TORQUE = 0, R_EDEM = 1, R_EEX = 2, R_EANI = 3, R_EZEE = 4, R_ERR = 5, R_NONFINITE = 6, R_EDMI = 7 };

template <typename T>
struct StageParams {
    int nx, ny, nz;
    long N;
    double V;                    // cell volume
    T idx2, idy2, idz2;          // 1 / d^2 per axis
    const T* m;                  // stage input (SoA)
    const T* hd;                 // demag field (SoA) or null
    const T* Ms_cell; T Ms;
    const T* A_cell; T A;
    const T* Ku_cell; T Ku;
    const T* alpha_cell; T alpha;
    const uint8_t* grain; const T* axis_tab; T ex, ey, ez;
    const T* zw; T hx0, hy0, hz0;
    T* h_out;                    // total effective field or null
    T* k_out;                    // stage derivative or null
    const T* mn;                 // m at the start of the step
    T* next;                     // mn + dt (sum_j kc_j kin_j + ck k), or null
    const T* kin[7];
    double kc[7];
    int nk;
    double ck;
    double dt;
    int renorm;
    const T* acc_in;             // acc_out = acc_in + acc_b k (acc_in may be null)
    T* acc_out;
    double acc_b;
    double eb[7];                // error e = dt (sum_j eb_j kin_j + eb_k k)
    double eb_k;
    double rtol, atol;
    int want_err, want_energy, want_torque;
    int err_on_next;             // error scale max(|mn|, |next|) instead of max(|mn|, |m|)
    int dmi;                     // DMI term on (Sec. 4.3)
    const T* D_cell; T D;        // DMI strength per cell (links averaged) or uniform
    T dmi_e[9];                  // DMI vectors e_x, e_y, e_z (each 3 components)
    T i2dx, i2dy, i2dz;          // 1 / (2 d) per axis
    int no_precession;           // drop the m x h summand of the LLG right-hand side
    // non-equidistant layers: lay[k] = h_k, lay[nz + k] = 2 / (h_k (h_k + h_{k+1})),
    // lay[2 nz + k] = 2 / (h_k (h_{k-1} + h_k)) (0 at the stack's ends), lvol[k] =
    // dx dy h_k; null: equidistant (idz2 and V)
    const T* lay;
    const double* lvol;
    double* partials;            // [number of blocks][kNPart]
    // the coefficients above in the field type (filled by launch_stage)
    T kcT[7], ckT, dtT, acc_bT;
    // the error-norm coefficients in the field type: the error norm and the
    // torque are evaluated in the state's precision (FP64 is a narrow pipe on
    // this part, and FP32 stage derivatives carry FP32 rounding anyway)
    T ebT[7], eb_kT, rtolT, atolT;
    T cex_u, cani_u, gp_u;       // 2/(mu0 Ms), 2 Ku/(mu0 Ms), -gamma/(1+alpha^2) for uniform material
};

template <typename T> void launch_stage(const StageParams<T>& p, cudaStream_t st, int* nblocks);
// fused x-inverse + stage + x-forward of the next stage input (FP32, uniform material, RK stages);
// the coefficients in the field type (kcT, ckT, dtT, acc_bT) and the uniform constants must be filled
bool fused_stage(const DemagDims& d, float2* S1, const StageParams<float>& p, cudaStream_t st, KernelTimer* tm);
bool fused_stage_supported(const DemagDims& d, const StageParams<float>& p);
// fill kcT, ckT, dtT, acc_bT and the uniform-material constants from the double fields
template <typename T> void stage_prepare(StageParams<T>& p);
template <typename T> int stage_blocks(int nx, int ny, int nz);   // blocks launch_stage will use
void launch_finalize(const double* partials, int nblocks, double* scalars, cudaStream_t st);
template <typename T> void launch_convert(const double* src, T* dst, long n, cudaStream_t st);
template <typename T> void launch_renorm_copy(const T* src, T* dst, long N, cudaStream_t st);
template <typename T> void launch_combine(const T* mn, const T* const* kin, const double* kc, int nk, double dt,
                                          T* out, long N, cudaStream_t st);
// copy the host-built twiddle table into the FFT kernels' device table (current device)
cudaError_t upload_twiddles(const double2* w64, const float2* w32, const double2* w5_64, const float2* w5_32);
// build (once, in static host storage) and upload the twiddle table to device dev, which
// must be current; a no-op after the first success on that device
cudaError_t ensure_twiddles_on(int dev);
// set the thread-local message returned by mm_last_error (fixed storage)
void set_last_error(const char* msg);

}  // namespace mm
