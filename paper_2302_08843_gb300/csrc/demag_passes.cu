// Demag field by zero-padded FFT convolution (Sec. 4.4), five passes.
//
//   P1 x-forward  : M = Ms m, real rows of nx values, zero-padded to Px, r2c
//                   -> S1[c][z][y][kx], kx <= Px/2 (two real rows per complex
//                   FFT: z = a + i b, A_k = (Z_k + conj Z_{P-k})/2,
//                   B_k = (Z_k - conj Z_{P-k})/(2i)).
//   P2 y-forward  : columns over y (ny values, zero-padded to Py)
//                   -> S2[c][z][ky][kx].
//   P3 z-conv     : per (kx, ky) column: z-forward (nz values, zero-padded to
//                   Pz), h^ = T(k) M^ with the real symmetric 3x3 spectrum T
//                   (octant-folded, sign flips of the odd components), z-inverse,
//                   keep z < nz; in place in S2.
//   P4 y-inverse  : keep y < ny -> S1.
//   P5 x-inverse  : c2r of two rows at a time, keep x < nx -> h[c][z][y][x].
//
// Strided passes (P2, P3, P4) put B consecutive kx columns in a CTA so that
// every warp access is a full 128-byte row segment; the x passes stage rows
// through shared memory with a padded stride.  The all-zero padded half of
// every forward transform is never loaded nor transformed (FftLine ZIN) and
// only the kept half of every inverse output is stored.
#include <cudaTypedefs.h>

#include <cstdio>
#include <mutex>
#include <utility>

#include "demag.h"
#include "fft_engine.cuh"
#include "fft_pair.cuh"
#include "tma.cuh"

namespace mm {

// A persistent pass lets the next kernel on the stream be launched
// (programmatic dependent launch) when each CTA enters its last tile: the
// dependent grid's CTAs then take SM room only as this grid drains.  Measured
// on the bulk RK4 stage: 383 us against 442 us with the trigger at kernel
// start (the waiting dependents delayed the running grid) and 388 us without
// programmatic launch.
__device__ __forceinline__ void pdl_trigger_late(bool last_tile) {
    if (last_tile) grid_dep_launch();
}

cudaError_t upload_twiddles(const double2* w64, const float2* w32, const double2* w5_64, const float2* w5_32) {
    cudaError_t e = cudaMemcpyToSymbol(g_tw64, w64, sizeof(double2) * kMaxFft);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tw32, w32, sizeof(float2) * kMaxFft);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tw5_64, w5_64, sizeof(double2) * kTw5);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tw5_32, w5_32, sizeof(float2) * kTw5);
    if (e == cudaSuccess) {
        static float4 twp[kTwP16];     // static host staging: the upload allocates nothing
        static bool built = false;
        if (!built) {
            build_twp16(w64, twp);
            built = true;
        }
        e = cudaMemcpyToSymbol(g_twp16, twp, sizeof(float4) * kTwP16);
    }
    return e;
}

// ------------------------------------------------------------------ P1 ----
// The x passes transform two real rows per complex FFT.  Rows are paired
// within one grid of a batch (R = 3 ny nz rows each; an odd R leaves the last
// row of every grid alone with a zero partner), so that a grid's result never
// depends on another grid's data.  Line l of block blk is pair q = blk NL + l.
template <int NL> __device__ __forceinline__ void pair_lines(const DemagDims& d, long* ra_s, long* rb_s) {
    if (threadIdx.x < NL) {
        const long R = 3L * d.ny * d.nz, ppg = (R + 1) / 2;
        const long q = (long)blockIdx.x * NL + threadIdx.x;
        const long b = q / ppg, lp = q - b * ppg;
        const bool ok = b < d.nb;
        ra_s[threadIdx.x] = ok ? b * R + 2 * lp : -1;
        rb_s[threadIdx.x] = ok && 2 * lp + 1 < R ? b * R + 2 * lp + 1 : -1;
    }
}
template <typename T, int LX, int NL>
__global__ void __launch_bounds__(NL * Fft<T, LX, -1, (LX > 1)>::TPL)
p1_x_forward(DemagDims d, const T* __restrict__ m, const T* __restrict__ Ms_cell, T Ms_const,
             typename Cplx<T>::type* __restrict__ S1) {
    using C = typename Cplx<T>::type;
    using F = Fft<T, LX, -1, (LX > 1)>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* s = reinterpret_cast<C*>(smraw);
    constexpr int LS = NL + 1;
    constexpr int NT = NL * F::TPL;
    constexpr int XH = LX > 1 ? LX / 2 : 1;     // staged input positions
    const int tid = threadIdx.x;
    const int line = tid % NL, j = tid / NL;
    const long plane = (long)d.ny * d.nz;
    const T* Ms_b = static_cast<const T*>(d.Ms_b);
    __shared__ long ra_s[NL], rb_s[NL];
    pair_lines<NL>(d, ra_s, rb_s);
    __syncthreads();

    for (int idx = tid; idx < NL * XH; idx += NT) {
        const int l = idx / XH, x = idx - l * XH;
        const long ra = ra_s[l], rb = rb_s[l];
        T a = 0, b = 0;
        if (x < d.nx) {
            if (ra >= 0) {
                const T ms = Ms_b ? Ms_b[ra / (3 * plane)] : (Ms_cell ? Ms_cell[(ra % plane) * d.nx + x] : Ms_const);
                a = m[ra * d.nx + x] * ms;
            }
            if (rb >= 0) {
                const T ms = Ms_b ? Ms_b[rb / (3 * plane)] : (Ms_cell ? Ms_cell[(rb % plane) * d.nx + x] : Ms_const);
                b = m[rb * d.nx + x] * ms;
            }
        }
        s[x * LS + l] = mk<C>(a, b);
    }
    __syncthreads();
    C v[F::NR];
#pragma unroll
    for (int r = 0; r < F::NR; ++r) {
        if (F::in_live(r)) v[r] = s[F::in_index(j, r) * LS + line];
        else v[r] = mk<C>(0, 0);
    }
    F::run(v, s + line, LS, j);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < F::NR; ++r) s[(j + r * F::TPL) * LS + line] = v[r];
    __syncthreads();
    constexpr int KXn = LX / 2 + 1;
    const T half = (T)0.5;
    for (int idx = tid; idx < NL * KXn; idx += NT) {
        const int l = idx / KXn, k = idx - l * KXn;
        const long ra = ra_s[l], rb = rb_s[l];
        const C zk = s[k * LS + l];
        const C zm = s[(k == 0 ? 0 : LX - k) * LS + l];     // mirror index, any even LX
        if (ra >= 0) S1[ra * d.KXS + k] = mk<C>(half * (zk.x + zm.x), half * (zk.y - zm.y));
        if (rb >= 0) S1[rb * d.KXS + k] = mk<C>(half * (zk.y + zm.y), half * (zm.x - zk.x));
    }
}

// ------------------------------------------------------ P1 / P5 (TMA) ----
// Persistent x passes for FP32.  A tile is 2*NL consecutive rows ([c][z][y]
// order); TMA brings the rows of the tile after next into the slot the
// current tile has just been staged out of.  Staging writes the tile into the
// engine's [x][line] work area (two real rows per complex line), which is
// then the transform's exchange scratch and the post-processing buffer.
template <int LX, int NL>
__global__ void __launch_bounds__(NL * Fft<float, LX, -1, (LX > 1)>::TPL)
p1_x_tma(DemagDims d, const __grid_constant__ CUtensorMap m_map, float Ms, float2* __restrict__ S1, int nxb,
         int nboxes, int slot_bytes) {
    using C = float2;
    using F = Fft<float, LX, -1, (LX > 1)>;
    constexpr int LS = NL + 1;
    constexpr int NT = NL * F::TPL;
    constexpr int XH = LX > 1 ? LX / 2 : 1;
    constexpr int KXn = LX / 2 + 1;
    extern __shared__ __align__(128) unsigned char smtma[];
    const int tid = threadIdx.x;
    const int line = tid % NL, j = tid / NL;
    const long rows = 3L * d.ny * d.nz;
    const int ntiles = (int)((rows + 2 * NL - 1) / (2 * NL));
    C* work = reinterpret_cast<C*>(smtma + 2 * (size_t)slot_bytes);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smtma + 2 * (size_t)slot_bytes + (size_t)LX * LS * sizeof(C));
    const int rowpitch = nboxes * nxb;       // floats per staged row (boxes side by side)
    const uint32_t tx = (uint32_t)(nboxes * nxb * 2 * NL * sizeof(float));
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int t, int sl) {
        float* dst = reinterpret_cast<float*>(smtma + (size_t)sl * slot_bytes);
        mbar_arrive_expect_tx(&bar[sl], tx);
        for (int b = 0; b < nboxes; ++b)
            tma_load_3d(dst + (size_t)b * nxb * 2 * NL, &m_map, &bar[sl], b * nxb, t * 2 * NL, 0);
    };
    const int t0 = blockIdx.x;
    if (tid == 0) {
        if (t0 < ntiles) issue(t0, 0);
        if (t0 + (int)gridDim.x < ntiles) issue(t0 + gridDim.x, 1);
    }
    int i = 0;
    for (int t = t0; t < ntiles; t += gridDim.x, ++i) {
        const int sl = i & 1;
        const float* tile = reinterpret_cast<const float*>(smtma + (size_t)sl * slot_bytes);
        const bool ok = mbar_wait_bounded(&bar[sl], (i >> 1) & 1);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(d.err, kErrTmaTimeout);
                if (t + (int)gridDim.x < ntiles) mbar_wait_bounded(&bar[sl ^ 1], ((i + 1) >> 1) & 1);
            }
            return;
        }
        // staging: box b holds rows x columns [b*nxb, (b+1)*nxb) as [row][xb]
        for (int idx = tid; idx < NL * XH; idx += NT) {
            const int l = idx / XH, x = idx - l * XH;
            float a = 0.f, b = 0.f;
            if (x < d.nx) {
                const int bx = x / nxb, xo = x - bx * nxb;
                const float* bb = tile + (size_t)bx * nxb * 2 * NL;
                a = bb[(2 * l) * nxb + xo] * Ms;
                b = bb[(2 * l + 1) * nxb + xo] * Ms;
            }
            work[x * LS + l] = mk<C>(a, b);
        }
        __syncthreads();   // slot consumed
        if (tid == 0 && t + 2 * (int)gridDim.x < ntiles) {
            fence_proxy_async_smem();
            issue(t + 2 * gridDim.x, sl);
        }
        (void)rowpitch;
        C v[F::NR];
#pragma unroll
        for (int r = 0; r < F::NR; ++r) v[r] = F::in_live(r) ? work[F::in_index(j, r) * LS + line] : mk<C>(0, 0);
        F::run(v, work + line, LS, j);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < F::NR; ++r) work[(j + r * F::TPL) * LS + line] = v[r];
        __syncthreads();
        const long row0 = (long)t * 2 * NL;
        for (int idx = tid; idx < NL * KXn; idx += NT) {
            const int l = idx / KXn, k = idx - l * KXn;
            const long ra = row0 + 2 * l, rb = ra + 1;
            const C zk = work[k * LS + l];
            const C zm = work[((LX - k) & (LX - 1)) * LS + l];
            if (ra < rows) S1[ra * d.KXS + k] = mk<C>(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
            if (rb < rows) S1[rb * d.KXS + k] = mk<C>(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
        }
        __syncthreads();   // work area free for the next tile's staging
    }
}

template <int LX, int NL>
__global__ void __launch_bounds__(NL * Fft<float, LX, +1, false>::TPL)
p5_x_tma(DemagDims d, const __grid_constant__ CUtensorMap s1_map, float* __restrict__ h, int kxb, int nboxes,
         int slot_bytes) {
    using C = float2;
    using F = Fft<float, LX, +1, false>;
    constexpr int LS = NL + 1;
    constexpr int NT = NL * F::TPL;
    constexpr int KXn = LX / 2 + 1;
    extern __shared__ __align__(128) unsigned char smtma[];
    const int tid = threadIdx.x;
    const int line = tid % NL, j = tid / NL;
    const long rows = 3L * d.ny * d.nz;
    const int ntiles = (int)((rows + 2 * NL - 1) / (2 * NL));
    C* work = reinterpret_cast<C*>(smtma + 2 * (size_t)slot_bytes);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smtma + 2 * (size_t)slot_bytes + (size_t)LX * LS * sizeof(C));
    const uint32_t tx = (uint32_t)(nboxes * kxb * 2 * NL * sizeof(C));
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int t, int sl) {
        C* dst = reinterpret_cast<C*>(smtma + (size_t)sl * slot_bytes);
        mbar_arrive_expect_tx(&bar[sl], tx);
        for (int b = 0; b < nboxes; ++b)
            tma_load_3d(dst + (size_t)b * kxb * 2 * NL, &s1_map, &bar[sl], b * kxb, t * 2 * NL, 0);
    };
    const int t0 = blockIdx.x;
    if (tid == 0) {
        if (t0 < ntiles) issue(t0, 0);
        if (t0 + (int)gridDim.x < ntiles) issue(t0 + gridDim.x, 1);
    }
    int i = 0;
    for (int t = t0; t < ntiles; t += gridDim.x, ++i) {
        const int sl = i & 1;
        const C* tile = reinterpret_cast<const C*>(smtma + (size_t)sl * slot_bytes);
        const bool ok = mbar_wait_bounded(&bar[sl], (i >> 1) & 1);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(d.err, kErrTmaTimeout);
                if (t + (int)gridDim.x < ntiles) mbar_wait_bounded(&bar[sl ^ 1], ((i + 1) >> 1) & 1);
            }
            return;
        }
        for (int idx = tid; idx < NL * KXn; idx += NT) {
            const int l = idx / KXn, k = idx - l * KXn;
            const int bk = k / kxb, ko = k - bk * kxb;
            const C* bb = tile + (size_t)bk * kxb * 2 * NL;
            C A = bb[(2 * l) * kxb + ko], Bv = bb[(2 * l + 1) * kxb + ko];
            if (k == 0 || 2 * k == LX) { A.y = 0.f; Bv.y = 0.f; }
            work[k * LS + l] = mk<C>(A.x - Bv.y, A.y + Bv.x);
            if (k > 0 && 2 * k < LX) work[(LX - k) * LS + l] = mk<C>(A.x + Bv.y, Bv.x - A.y);
        }
        __syncthreads();   // slot consumed
        if (tid == 0 && t + 2 * (int)gridDim.x < ntiles) {
            fence_proxy_async_smem();
            issue(t + 2 * gridDim.x, sl);
        }
        C v[F::NR];
#pragma unroll
        for (int r = 0; r < F::NR; ++r) v[r] = work[(j + r * F::TPL) * LS + line];
        F::run(v, work + line, LS, j);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < F::NR; ++r)
            if (LX == 1 || r < F::NR / 2) work[(j + r * F::TPL) * LS + line] = v[r];
        __syncthreads();
        const long row0 = (long)t * 2 * NL;
        for (int idx = tid; idx < NL * d.nx; idx += NT) {
            const int l = idx / d.nx, x = idx - l * d.nx;
            const long ra = row0 + 2 * l, rb = ra + 1;
            const C z = work[x * LS + l];
            if (ra < rows) h[ra * d.nx + x] = z.x;
            if (rb < rows) h[rb * d.nx + x] = z.y;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------- fused K5 ----
// x-inverse of the demag spectrum + exchange, anisotropy, Zeeman, LLG and the
// RK combination + x-forward of Ms * (next stage input), for FP32 with a
// uniform material (easy axes may vary by grain).  A tile is TY rows of y at
// one z, all three components (3*TY real rows = 3*TY/2 complex lines, pairs of
// consecutive y of one component); TMA fetches the tile after next.  After the
// inverse transform the demag field sits in the [x][line] work area; each cell
// update reads it there, writes acc/next to global memory and puts Ms * next
// back in the same place, which the forward transform then turns into the
// next stage's x-spectrum, written over this tile's rows of S1.
// NSLOT TMA slots: with one, the next tile's load is issued as soon as this
// tile is staged and has both transforms and the cell updates to land.
// skew of the fused kernel's work area (see FftLine16::at): 6 complex slots
// every 32 elements puts the exchange writes of its span-2 pass, 32 elements
// apart per thread pair, on different banks (123.7 -> 119.5 us on the bulk grid)
constexpr int kK5Skew = 6;
template <int LX, int LS> __host__ __device__ constexpr int k5_work_elems() {
    return LX * LS + (is_pow2(LX) ? (LX / 32) * kK5Skew : 0);
}
// the fused kernel's engines: radix-16 with the work-area skew for powers of
// two, the shared-memory mixed-radix engine for the compiled r 2^a lengths
// the mixed-radix lengths take the shorter radix plans (384 = 6 8 8: two
// exchanges per transform, 24 values per thread) with six rows of y per tile
// (192x192x48: 90.9 us with the radix-4 plan and two rows, 69.8 us so)
#ifndef MM_K5_ALT
#define MM_K5_ALT 1
#endif
template <int LX, int DIR, bool ZIN> struct K5Eng {
    using type = typename std::conditional<is_pow2(LX), FftLine16<float, (LX < 16 ? 16 : LX), DIR, ZIN, kK5Skew>,
                                           FftMixed<float, LX, DIR, ZIN, (MM_K5_ALT != 0)>>::type;
};

// link A of two cells (harmonic mean; zero if both are zero) and, across
// non-equidistant layers of thickness ha, hb, the two half cells in series
__device__ __forceinline__ float k5_harm(float a, float b) {
    const float s = a + b;
    return s != 0.f ? __fdividef(2.f * a * b, s) : 0.f;
}
__device__ __forceinline__ float k5_thick(float a, float b, float ha, float hb) {
    const float s = ha * b + hb * a;
    return s != 0.f ? __fdividef((ha + hb) * a * b, s) : 0.f;
}

// MAT: per-cell Ms, A and Ku1 maps (any of them may be absent) and
// non-equidistant layers (Sec. 4.4, per-layer z links); the x-forward input is
// then Ms_cell * next, and a cell with Ms = 0 carries no field.
template <int LX, int TY, int NSLOT, int PAD, int MINB, bool DMI, bool MAT>
__global__ void __launch_bounds__((3 * TY / 2) * K5Eng<LX, +1, false>::type::TPL, MINB)
k5_fused(DemagDims d, const __grid_constant__ CUtensorMap s1_map, float2* __restrict__ S1, StageParams<float> p,
         int kxb, int nboxes, int slot_bytes) {
    using C = float2;
    using FI = typename K5Eng<LX, +1, false>::type;
    using FF = typename K5Eng<LX, -1, true>::type;
    static_assert(FI::TPL == FF::TPL, "engines must agree on threads per line");
    static_assert(NSLOT == 1 || NSLOT == 2, "one or two TMA slots");
    constexpr int NL = 3 * TY / 2;
    constexpr int LS = NL + PAD;
    constexpr int NT = NL * FI::TPL;
    constexpr int KXn = LX / 2 + 1;
    constexpr int XH = LX / 2;
    extern __shared__ __align__(128) unsigned char smtma[];
    const int tid = threadIdx.x;
    const int line = tid % NL, j = tid / NL;
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    const int N = nx * ny * nz;
    const int nyt = (ny + TY - 1) / TY;
    const int ntiles = nyt * nz;
    C* work = reinterpret_cast<C*>(smtma + NSLOT * (size_t)slot_bytes);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smtma + NSLOT * (size_t)slot_bytes + (size_t)k5_work_elems<LX, LS>() * sizeof(C));
    auto wat = [](int e) { return FI::at(e, LS); };   // place of element e of line 0 in the work area
    const uint32_t tx = (uint32_t)(nboxes * kxb * TY * 3 * sizeof(C));
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    grid_dep_wait();      // the previous pass's output is complete from here on
    auto issue = [&](int t, int sl) {
        const int yt = t % nyt, z = t / nyt;
        C* dst = reinterpret_cast<C*>(smtma + (size_t)sl * slot_bytes);
        mbar_arrive_expect_tx(&bar[sl], tx);
        for (int b = 0; b < nboxes; ++b)
            tma_load_4d(dst + (size_t)b * kxb * TY * 3, &s1_map, &bar[sl], b * kxb, yt * TY, z, 0);
    };
    const int t0 = blockIdx.x;
    if (tid == 0) {
        if (t0 < ntiles) issue(t0, 0);
        if (NSLOT == 2 && t0 + (int)gridDim.x < ntiles) issue(t0 + gridDim.x, 1);
    }
    const float* m = p.m;
    int it = 0;
    for (int t = t0; t < ntiles; t += gridDim.x, ++it) {
        pdl_trigger_late(t + (int)gridDim.x >= ntiles);
        const int sl = NSLOT == 2 ? (it & 1) : 0;
        const uint32_t par = NSLOT == 2 ? ((it >> 1) & 1) : (it & 1);
        const C* tile = reinterpret_cast<const C*>(smtma + (size_t)sl * slot_bytes);   // [box][c][y][kx]
        const bool ok = mbar_wait_bounded(&bar[sl], par);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(d.err, kErrTmaTimeout);
                if (NSLOT == 2 && t + (int)gridDim.x < ntiles)
                    mbar_wait_bounded(&bar[sl ^ 1], ((it + 1) >> 1) & 1);
            }
            return;
        }
        const int yt = t % nyt, z = t / nyt;
        const int y0 = yt * TY;
        // ---- stage the c2r input: line l = (c, q) pairs rows y0+2q, y0+2q+1 of component c
        for (int idx = tid; idx < NL * KXn; idx += NT) {
            const int l = idx / KXn, k = idx - l * KXn;
            const int c = l / (TY / 2), q = l - c * (TY / 2);
            const int bk = k / kxb, ko = k - bk * kxb;
            const C* bb = tile + (size_t)bk * kxb * TY * 3;
            C A = bb[(c * TY + 2 * q) * kxb + ko], Bv = bb[(c * TY + 2 * q + 1) * kxb + ko];
            if (k == 0 || 2 * k == LX) { A.y = 0.f; Bv.y = 0.f; }
            work[wat(k) + l] = mk<C>(A.x - Bv.y, A.y + Bv.x);
            if (k > 0 && 2 * k < LX) work[wat(LX - k) + l] = mk<C>(A.x + Bv.y, Bv.x - A.y);
        }
        __syncthreads();   // slot consumed
        if (tid == 0 && t + NSLOT * (int)gridDim.x < ntiles) {
            fence_proxy_async_smem();
            issue(t + NSLOT * gridDim.x, sl);
        }
        {
            C v[FI::NR];
#pragma unroll
            for (int r = 0; r < FI::NR; ++r) v[r] = work[wat(j + r * FI::TPL) + line];
            FI::run(v, work + line, LS, j);
            __syncthreads();
#pragma unroll
            for (int r = 0; r < FI::NR / 2; ++r) work[wat(j + r * FI::TPL) + line] = v[r];
        }
        __syncthreads();
        // ---- cell updates: two consecutive x cells per item, float2 loads
        const int rows_here = (ny - y0) < TY ? (ny - y0) : TY;
        for (int idx = tid; idx < TY * (XH / 2); idx += NT) {
            const int yy = idx / (XH / 2), x0 = (idx - yy * (XH / 2)) * 2;
            const int l0 = yy >> 1, part = yy & 1;     // line of component c is c*TY/2 + l0
            float* w0 = reinterpret_cast<float*>(&work[wat(x0) + 0 * (TY / 2) + l0]) + part;
            float* w1 = reinterpret_cast<float*>(&work[wat(x0) + 1 * (TY / 2) + l0]) + part;
            float* w2 = reinterpret_cast<float*>(&work[wat(x0) + 2 * (TY / 2) + l0]) + part;
            constexpr int WS = 2 * LS;                 // floats between x and x+1 in the work area
            if (yy >= rows_here || x0 >= nx) {         // zero-padded inputs of the forward transform
                w0[0] = 0.f; w1[0] = 0.f; w2[0] = 0.f;
                w0[WS] = 0.f; w1[WS] = 0.f; w2[WS] = 0.f;
                continue;
            }
            const int y = y0 + yy;
            const int i = x0 + nx * (y + ny * z);      // even: float2 aligned (nx even)
            if constexpr (MAT) {
                const float2* m2 = reinterpret_cast<const float2*>(m);
                const int i2 = i >> 1, N2 = N >> 1;
                const float2 mx = m2[i2], my = m2[N2 + i2], mz = m2[2 * N2 + i2];
                const float2 Ms = p.Ms_cell ? reinterpret_cast<const float2*>(p.Ms_cell)[i2] : f2s(p.Ms);
                const float2* A2 = reinterpret_cast<const float2*>(p.A_cell);
                const float2 A = A2 ? A2[i2] : f2s(p.A);
                float2 sx, sy, sz;
                {   // x links: the inner link, then the outer neighbours (absent ones weigh nothing)
                    const float wi = p.idx2 * (A2 ? k5_harm(A.x, A.y) : p.A);
                    sx = f2mul(f2s(wi), f2sub(make_float2(mx.y, mx.x), mx));
                    sy = f2mul(f2s(wi), f2sub(make_float2(my.y, my.x), my));
                    sz = f2mul(f2s(wi), f2sub(make_float2(mz.y, mz.x), mz));
                    const bool hl = x0 > 0, hr = x0 + 2 < nx;
                    const float wl = hl ? p.idx2 * (A2 ? k5_harm(A.x, p.A_cell[i - 1]) : p.A) : 0.f;
                    const float wr = hr ? p.idx2 * (A2 ? k5_harm(A.y, p.A_cell[i + 2]) : p.A) : 0.f;
                    const float2 wo = make_float2(wl, wr);
                    const float2 ox = make_float2(hl ? m[i - 1] : mx.x, hr ? m[i + 2] : mx.y);
                    const float2 oy = make_float2(hl ? m[N + i - 1] : my.x, hr ? m[N + i + 2] : my.y);
                    const float2 oz = make_float2(hl ? m[2 * N + i - 1] : mz.x, hr ? m[2 * N + i + 2] : mz.y);
                    sx = f2fma(wo, f2sub(ox, mx), sx);
                    sy = f2fma(wo, f2sub(oy, my), sy);
                    sz = f2fma(wo, f2sub(oz, mz), sz);
                }
                // y and z links; across non-equidistant layers the z link is
                // 2 A_link / (h_k (h_k + h_nb)) with the two half cells in series
                auto link = [&](bool cond, int off2, float c, bool thick, float hk, float hn) {
                    if (cond) {
                        float2 w;
                        if (A2) {
                            const float2 An = A2[i2 + off2];
                            w = thick ? make_float2(c * k5_thick(A.x, An.x, hk, hn), c * k5_thick(A.y, An.y, hk, hn))
                                      : make_float2(c * k5_harm(A.x, An.x), c * k5_harm(A.y, An.y));
                        } else {
                            w = f2s(c * p.A);
                        }
                        const float2 a = m2[i2 + off2], b = m2[N2 + i2 + off2], cc = m2[2 * N2 + i2 + off2];
                        sx = f2fma(w, f2sub(a, mx), sx);
                        sy = f2fma(w, f2sub(b, my), sy);
                        sz = f2fma(w, f2sub(cc, mz), sz);
                    }
                };
                link(y > 0, -(nx >> 1), p.idy2, false, 0.f, 0.f);
                link(y < ny - 1, nx >> 1, p.idy2, false, 0.f, 0.f);
                if (!p.lay) {
                    link(z > 0, -((nx * ny) >> 1), p.idz2, false, 0.f, 0.f);
                    link(z < nz - 1, (nx * ny) >> 1, p.idz2, false, 0.f, 0.f);
                } else {
                    const float hk = p.lay[z];
                    link(z > 0, -((nx * ny) >> 1), p.lay[2 * nz + z], true, hk, p.lay[z > 0 ? z - 1 : z]);
                    link(z < nz - 1, (nx * ny) >> 1, p.lay[nz + z], true, hk, p.lay[z < nz - 1 ? z + 1 : z]);
                }
                const float2* mn2 = reinterpret_cast<const float2*>(p.mn);
                const float2 nX = mn2[i2], nY = mn2[N2 + i2], nZ = mn2[2 * N2 + i2];
                float2 aX = f2s(0.f), aY = f2s(0.f), aZ = f2s(0.f);
                const float* accsrc = p.acc_in ? p.acc_in : (p.nk > 0 ? p.kin[0] : nullptr);
                if (accsrc) {
                    const float2* a2 = reinterpret_cast<const float2*>(accsrc);
                    aX = a2[i2]; aY = a2[N2 + i2]; aZ = a2[2 * N2 + i2];
                }
                // 2 / (mu0 Ms) per cell; a cell with Ms = 0 carries no field
                const float c2 = (float)(2.0 / kMu0);
                const float2 inv = make_float2(Ms.x != 0.f ? 1.f / Ms.x : 0.f, Ms.y != 0.f ? 1.f / Ms.y : 0.f);
                const float2 on = make_float2(Ms.x != 0.f ? 1.f : 0.f, Ms.y != 0.f ? 1.f : 0.f);
                const float2 cex = f2mul(f2s(c2), inv);
                float2 hx = f2mul(cex, sx), hy = f2mul(cex, sy), hz = f2mul(cex, sz);
                const float2 Ku = p.Ku_cell ? reinterpret_cast<const float2*>(p.Ku_cell)[i2] : f2s(p.Ku);
                if (Ku.x != 0.f || Ku.y != 0.f) {
                    float2 ex = f2s(p.ex), ey = f2s(p.ey), ez = f2s(p.ez);
                    if (p.grain) {
                        const int g0 = p.grain[i], g1 = p.grain[i + 1];
                        ex = make_float2(p.axis_tab[3 * g0], p.axis_tab[3 * g1]);
                        ey = make_float2(p.axis_tab[3 * g0 + 1], p.axis_tab[3 * g1 + 1]);
                        ez = make_float2(p.axis_tab[3 * g0 + 2], p.axis_tab[3 * g1 + 2]);
                    }
                    const float2 ck = f2mul(f2mul(f2s(c2), Ku), inv);
                    const float2 c = f2mul(ck, f2fma(ex, mx, f2fma(ey, my, f2mul(ez, mz))));
                    hx = f2fma(c, ex, hx);
                    hy = f2fma(c, ey, hy);
                    hz = f2fma(c, ez, hz);
                }
                constexpr int WSP = 2 * LS;
                float* w0 = reinterpret_cast<float*>(&work[wat(x0) + 0 * (TY / 2) + (yy >> 1)]) + (yy & 1);
                float* w1 = reinterpret_cast<float*>(&work[wat(x0) + 1 * (TY / 2) + (yy >> 1)]) + (yy & 1);
                float* w2 = reinterpret_cast<float*>(&work[wat(x0) + 2 * (TY / 2) + (yy >> 1)]) + (yy & 1);
                hx = f2mul(on, f2add(hx, f2add(make_float2(w0[0], w0[WSP]), f2s(p.hx0))));
                hy = f2mul(on, f2add(hy, f2add(make_float2(w1[0], w1[WSP]), f2s(p.hy0))));
                hz = f2mul(on, f2add(hz, f2add(make_float2(w2[0], w2[WSP]), f2s(p.hz0))));
                const float2 cx = f2sub(f2mul(my, hz), f2mul(mz, hy));
                const float2 cy = f2sub(f2mul(mz, hx), f2mul(mx, hz));
                const float2 cz = f2sub(f2mul(mx, hy), f2mul(my, hx));
                const float2 dx_ = f2sub(f2mul(my, cz), f2mul(mz, cy));
                const float2 dy_ = f2sub(f2mul(mz, cx), f2mul(mx, cz));
                const float2 dz_ = f2sub(f2mul(mx, cy), f2mul(my, cx));
                const float2 al = f2s(p.alpha), gp = f2s(p.gp_u), pc = f2s(p.no_precession ? 0.f : 1.f);
                const float2 kx = f2mul(gp, f2fma(al, dx_, f2mul(pc, cx)));
                const float2 ky = f2mul(gp, f2fma(al, dy_, f2mul(pc, cy)));
                const float2 kz = f2mul(gp, f2fma(al, dz_, f2mul(pc, cz)));
                if (p.acc_out) {
                    const float2 ab = f2s(p.acc_bT);
                    float2* ao = reinterpret_cast<float2*>(p.acc_out);
                    ao[i2] = p.acc_in ? f2fma(ab, kx, aX) : f2mul(ab, kx);
                    ao[N2 + i2] = p.acc_in ? f2fma(ab, ky, aY) : f2mul(ab, ky);
                    ao[2 * N2 + i2] = p.acc_in ? f2fma(ab, kz, aZ) : f2mul(ab, kz);
                }
                const float2 c0 = f2s(p.nk > 0 ? p.kcT[0] : 0.f), ckk = f2s(p.ckT), dtv = f2s(p.dtT);
                float2 a = f2fma(dtv, f2fma(ckk, kx, f2mul(c0, aX)), nX);
                float2 b = f2fma(dtv, f2fma(ckk, ky, f2mul(c0, aY)), nY);
                float2 c = f2fma(dtv, f2fma(ckk, kz, f2mul(c0, aZ)), nZ);
                if (p.renorm) {
                    const float2 nn = f2fma(a, a, f2fma(b, b, f2mul(c, c)));
                    const float2 sc = make_float2(nn.x > 0.f ? 1.f / sqrtf(nn.x) : 1.f,
                                                  nn.y > 0.f ? 1.f / sqrtf(nn.y) : 1.f);
                    a = f2mul(a, sc); b = f2mul(b, sc); c = f2mul(c, sc);
                }
                float2* no = reinterpret_cast<float2*>(p.next);
                no[i2] = a;
                no[N2 + i2] = b;
                no[2 * N2 + i2] = c;
                const float2 ma = f2mul(Ms, a), mb = f2mul(Ms, b), mc = f2mul(Ms, c);
                w0[0] = ma.x; w0[WSP] = ma.y;
                w1[0] = mb.x; w1[WSP] = mb.y;
                w2[0] = mc.x; w2[WSP] = mc.y;
                continue;
            }
            if constexpr (!DMI) {
                // the two cells of the item are the two lanes of every paired
                // FP32 instruction (add/sub/mul/fma .f32x2)
                const float2* m2 = reinterpret_cast<const float2*>(m);
                const int i2 = i >> 1, N2 = N >> 1;
                const float2 mx = m2[i2], my = m2[N2 + i2], mz = m2[2 * N2 + i2];
                float2 sx, sy, sz;
                {   // x links: the inner link, then the outer neighbours (a missing
                    // neighbour stands in as the cell itself and adds nothing)
                    const float2 wx = f2s(p.A * p.idx2);
                    sx = f2mul(wx, f2sub(make_float2(mx.y, mx.x), mx));
                    sy = f2mul(wx, f2sub(make_float2(my.y, my.x), my));
                    sz = f2mul(wx, f2sub(make_float2(mz.y, mz.x), mz));
                    const bool hl = x0 > 0, hr = x0 + 2 < nx;
                    const float2 ox = make_float2(hl ? m[i - 1] : mx.x, hr ? m[i + 2] : mx.y);
                    const float2 oy = make_float2(hl ? m[N + i - 1] : my.x, hr ? m[N + i + 2] : my.y);
                    const float2 oz = make_float2(hl ? m[2 * N + i - 1] : mz.x, hr ? m[2 * N + i + 2] : mz.y);
                    sx = f2fma(wx, f2sub(ox, mx), sx);
                    sy = f2fma(wx, f2sub(oy, my), sy);
                    sz = f2fma(wx, f2sub(oz, mz), sz);
                }
                auto link = [&](bool cond, int off2, float id2) {
                    if (cond) {
                        const float2 w = f2s(p.A * id2);
                        const float2 a = m2[i2 + off2], b = m2[N2 + i2 + off2], c = m2[2 * N2 + i2 + off2];
                        sx = f2fma(w, f2sub(a, mx), sx);
                        sy = f2fma(w, f2sub(b, my), sy);
                        sz = f2fma(w, f2sub(c, mz), sz);
                    }
                };
                link(y > 0, -(nx >> 1), p.idy2);
                link(y < ny - 1, nx >> 1, p.idy2);
                link(z > 0, -((nx * ny) >> 1), p.idz2);
                link(z < nz - 1, (nx * ny) >> 1, p.idz2);
                const float2* mn2 = reinterpret_cast<const float2*>(p.mn);
                const float2 nX = mn2[i2], nY = mn2[N2 + i2], nZ = mn2[2 * N2 + i2];
                float2 aX = f2s(0.f), aY = f2s(0.f), aZ = f2s(0.f);
                const float* accsrc = p.acc_in ? p.acc_in : (p.nk > 0 ? p.kin[0] : nullptr);
                if (accsrc) {
                    const float2* a2 = reinterpret_cast<const float2*>(accsrc);
                    aX = a2[i2]; aY = a2[N2 + i2]; aZ = a2[2 * N2 + i2];
                }
                const float2 cex = f2s(p.cex_u);
                float2 hx = f2mul(cex, sx), hy = f2mul(cex, sy), hz = f2mul(cex, sz);
                if (p.Ku != 0.f) {
                    float2 ex = f2s(p.ex), ey = f2s(p.ey), ez = f2s(p.ez);
                    if (p.grain) {
                        const int g0 = p.grain[i], g1 = p.grain[i + 1];
                        ex = make_float2(p.axis_tab[3 * g0], p.axis_tab[3 * g1]);
                        ey = make_float2(p.axis_tab[3 * g0 + 1], p.axis_tab[3 * g1 + 1]);
                        ez = make_float2(p.axis_tab[3 * g0 + 2], p.axis_tab[3 * g1 + 2]);
                    }
                    const float2 c = f2mul(f2s(p.cani_u), f2fma(ex, mx, f2fma(ey, my, f2mul(ez, mz))));
                    hx = f2fma(c, ex, hx);
                    hy = f2fma(c, ey, hy);
                    hz = f2fma(c, ez, hz);
                }
                constexpr int WSP = 2 * LS;            // floats between x and x+1 in the work area
                float* w0 = reinterpret_cast<float*>(&work[wat(x0) + 0 * (TY / 2) + (yy >> 1)]) + (yy & 1);
                float* w1 = reinterpret_cast<float*>(&work[wat(x0) + 1 * (TY / 2) + (yy >> 1)]) + (yy & 1);
                float* w2 = reinterpret_cast<float*>(&work[wat(x0) + 2 * (TY / 2) + (yy >> 1)]) + (yy & 1);
                hx = f2add(hx, f2add(make_float2(w0[0], w0[WSP]), f2s(p.hx0)));
                hy = f2add(hy, f2add(make_float2(w1[0], w1[WSP]), f2s(p.hy0)));
                hz = f2add(hz, f2add(make_float2(w2[0], w2[WSP]), f2s(p.hz0)));
                // Eq. llg: k = gp (pc m x h + alpha m x (m x h))
                const float2 cx = f2sub(f2mul(my, hz), f2mul(mz, hy));
                const float2 cy = f2sub(f2mul(mz, hx), f2mul(mx, hz));
                const float2 cz = f2sub(f2mul(mx, hy), f2mul(my, hx));
                const float2 dx_ = f2sub(f2mul(my, cz), f2mul(mz, cy));
                const float2 dy_ = f2sub(f2mul(mz, cx), f2mul(mx, cz));
                const float2 dz_ = f2sub(f2mul(mx, cy), f2mul(my, cx));
                const float2 al = f2s(p.alpha), gp = f2s(p.gp_u), pc = f2s(p.no_precession ? 0.f : 1.f);
                const float2 kx = f2mul(gp, f2fma(al, dx_, f2mul(pc, cx)));
                const float2 ky = f2mul(gp, f2fma(al, dy_, f2mul(pc, cy)));
                const float2 kz = f2mul(gp, f2fma(al, dz_, f2mul(pc, cz)));
                // RK combination: acc_out = acc_in + acc_b k;  next = mn + dt (kc0 kin0 + ck k)
                if (p.acc_out) {
                    const float2 ab = f2s(p.acc_bT);
                    float2* ao = reinterpret_cast<float2*>(p.acc_out);
                    ao[i2] = p.acc_in ? f2fma(ab, kx, aX) : f2mul(ab, kx);
                    ao[N2 + i2] = p.acc_in ? f2fma(ab, ky, aY) : f2mul(ab, ky);
                    ao[2 * N2 + i2] = p.acc_in ? f2fma(ab, kz, aZ) : f2mul(ab, kz);
                }
                const float2 c0 = f2s(p.nk > 0 ? p.kcT[0] : 0.f), ck = f2s(p.ckT), dtv = f2s(p.dtT);
                float2 a = f2fma(dtv, f2fma(ck, kx, f2mul(c0, aX)), nX);
                float2 b = f2fma(dtv, f2fma(ck, ky, f2mul(c0, aY)), nY);
                float2 c = f2fma(dtv, f2fma(ck, kz, f2mul(c0, aZ)), nZ);
                if (p.renorm) {
                    const float2 nn = f2fma(a, a, f2fma(b, b, f2mul(c, c)));
                    const float2 sc = make_float2(nn.x > 0.f ? 1.f / sqrtf(nn.x) : 1.f,
                                                  nn.y > 0.f ? 1.f / sqrtf(nn.y) : 1.f);
                    a = f2mul(a, sc); b = f2mul(b, sc); c = f2mul(c, sc);
                }
                float2* no = reinterpret_cast<float2*>(p.next);
                no[i2] = a;
                no[N2 + i2] = b;
                no[2 * N2 + i2] = c;
                // Ms * next for the forward transform (the demag values at this place are consumed)
                const float2 msv = f2s(p.Ms);
                const float2 ma = f2mul(msv, a), mb = f2mul(msv, b), mc = f2mul(msv, c);
                w0[0] = ma.x; w0[WSP] = ma.y;
                w1[0] = mb.x; w1[WSP] = mb.y;
                w2[0] = mc.x; w2[WSP] = mc.y;
                continue;
            }
            const float2* m2 = reinterpret_cast<const float2*>(m);
            const int i2 = i >> 1, N2 = N >> 1;
            const float2 cx2 = m2[i2], cy2 = m2[N2 + i2], cz2 = m2[2 * N2 + i2];
            const float mxv[2] = {cx2.x, cx2.y}, myv[2] = {cy2.x, cy2.y}, mzv[2] = {cz2.x, cz2.y};
            float sx[2] = {0.f, 0.f}, sy[2] = {0.f, 0.f}, sz[2] = {0.f, 0.f};
            // DMI sums (uniform D, Sec. 4.3): per cell, sum over axes of e_a x (m_{+a} - m_{-a}) D / (2 d_a)
            float qx[2] = {0.f, 0.f}, qy[2] = {0.f, 0.f}, qz[2] = {0.f, 0.f};
            {   // x links
                const float wx = p.A * p.idx2;
                // inner link between the two cells
                sx[0] += wx * (mxv[1] - mxv[0]); sy[0] += wx * (myv[1] - myv[0]); sz[0] += wx * (mzv[1] - mzv[0]);
                sx[1] += wx * (mxv[0] - mxv[1]); sy[1] += wx * (myv[0] - myv[1]); sz[1] += wx * (mzv[0] - mzv[1]);
                float dl[3] = {0.f, 0.f, 0.f}, dr[3] = {0.f, 0.f, 0.f};   // DMI: m_{+x} - m_{-x} per cell
                if constexpr (DMI) {
                    dl[0] = mxv[1]; dl[1] = myv[1]; dl[2] = mzv[1];
                    dr[0] = -mxv[0]; dr[1] = -myv[0]; dr[2] = -mzv[0];
                }
                if (x0 > 0) {
                    const float ax = m[i - 1], ay = m[N + i - 1], az = m[2 * N + i - 1];
                    sx[0] += wx * (ax - mxv[0]); sy[0] += wx * (ay - myv[0]); sz[0] += wx * (az - mzv[0]);
                    if constexpr (DMI) { dl[0] -= ax; dl[1] -= ay; dl[2] -= az; }
                }
                if (x0 + 2 < nx) {
                    const float ax = m[i + 2], ay = m[N + i + 2], az = m[2 * N + i + 2];
                    sx[1] += wx * (ax - mxv[1]); sy[1] += wx * (ay - myv[1]); sz[1] += wx * (az - mzv[1]);
                    if constexpr (DMI) { dr[0] += ax; dr[1] += ay; dr[2] += az; }
                }
                if constexpr (DMI) {
                    const float c = p.D * p.i2dx;
                    const float* e = &p.dmi_e[0];
                    qx[0] += c * (e[1] * dl[2] - e[2] * dl[1]); qy[0] += c * (e[2] * dl[0] - e[0] * dl[2]);
                    qz[0] += c * (e[0] * dl[1] - e[1] * dl[0]);
                    qx[1] += c * (e[1] * dr[2] - e[2] * dr[1]); qy[1] += c * (e[2] * dr[0] - e[0] * dr[2]);
                    qz[1] += c * (e[0] * dr[1] - e[1] * dr[0]);
                }
            }
#define MM_F2LINK(COND, OFF2, ID2, SIGN, EOFF, I2D)                                            \
            if (COND) {                                                                        \
                const float w = p.A * (ID2);                                                   \
                const float2 a = m2[i2 + (OFF2)], b = m2[N2 + i2 + (OFF2)], c = m2[2 * N2 + i2 + (OFF2)]; \
                sx[0] += w * (a.x - mxv[0]); sy[0] += w * (b.x - myv[0]); sz[0] += w * (c.x - mzv[0]); \
                sx[1] += w * (a.y - mxv[1]); sy[1] += w * (b.y - myv[1]); sz[1] += w * (c.y - mzv[1]); \
                if constexpr (DMI) {                                                           \
                    const float g = (SIGN) * p.D * (I2D);                                      \
                    const float* e = &p.dmi_e[EOFF];                                           \
                    qx[0] += g * (e[1] * c.x - e[2] * b.x); qy[0] += g * (e[2] * a.x - e[0] * c.x); \
                    qz[0] += g * (e[0] * b.x - e[1] * a.x);                                    \
                    qx[1] += g * (e[1] * c.y - e[2] * b.y); qy[1] += g * (e[2] * a.y - e[0] * c.y); \
                    qz[1] += g * (e[0] * b.y - e[1] * a.y);                                    \
                }                                                                              \
            }
            MM_F2LINK(y > 0, -(nx >> 1), p.idy2, -1.f, 3, p.i2dy)
            MM_F2LINK(y < ny - 1, (nx >> 1), p.idy2, 1.f, 3, p.i2dy)
            MM_F2LINK(z > 0, -((nx * ny) >> 1), p.idz2, -1.f, 6, p.i2dz)
            MM_F2LINK(z < nz - 1, ((nx * ny) >> 1), p.idz2, 1.f, 6, p.i2dz)
#undef MM_F2LINK
            const float2 n0 = reinterpret_cast<const float2*>(p.mn)[i2];
            const float2 n1 = reinterpret_cast<const float2*>(p.mn)[N2 + i2];
            const float2 n2 = reinterpret_cast<const float2*>(p.mn)[2 * N2 + i2];
            const float mnx[2] = {n0.x, n0.y}, mny[2] = {n1.x, n1.y}, mnz[2] = {n2.x, n2.y};
            float ax_[2] = {0.f, 0.f}, ay_[2] = {0.f, 0.f}, az_[2] = {0.f, 0.f};
            const float* accsrc = p.acc_in ? p.acc_in : (p.nk > 0 ? p.kin[0] : nullptr);
            if (accsrc) {
                const float2 a0 = reinterpret_cast<const float2*>(accsrc)[i2];
                const float2 a1 = reinterpret_cast<const float2*>(accsrc)[N2 + i2];
                const float2 a2 = reinterpret_cast<const float2*>(accsrc)[2 * N2 + i2];
                ax_[0] = a0.x; ax_[1] = a0.y; ay_[0] = a1.x; ay_[1] = a1.y; az_[0] = a2.x; az_[1] = a2.y;
            }
            float ox[2], oy[2], oz[2], accx[2], accy[2], accz[2];
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const float mx = mxv[v], my = myv[v], mz = mzv[v];
                float hx = p.cex_u * sx[v], hy = p.cex_u * sy[v], hz = p.cex_u * sz[v];
                if constexpr (DMI) { hx += p.cex_u * qx[v]; hy += p.cex_u * qy[v]; hz += p.cex_u * qz[v]; }
                if (p.Ku != 0.f) {
                    float ex = p.ex, ey = p.ey, ez = p.ez;
                    if (p.grain) {
                        const int gi = p.grain[i + v];
                        ex = p.axis_tab[3 * gi]; ey = p.axis_tab[3 * gi + 1]; ez = p.axis_tab[3 * gi + 2];
                    }
                    const float c = p.cani_u * (ex * mx + ey * my + ez * mz);
                    hx += c * ex; hy += c * ey; hz += c * ez;
                }
                hx += w0[v * WS] + p.hx0;
                hy += w1[v * WS] + p.hy0;
                hz += w2[v * WS] + p.hz0;
                const float al = p.alpha, gp = p.gp_u;
                const float cx = my * hz - mz * hy, cy = mz * hx - mx * hz, cz = mx * hy - my * hx;
                const float dx_ = my * cz - mz * cy, dy_ = mz * cx - mx * cz, dz_ = mx * cy - my * cx;
                const float pc = p.no_precession ? 0.f : 1.f;
                const float kx = gp * (pc * cx + al * dx_), ky = gp * (pc * cy + al * dy_),
                            kz = gp * (pc * cz + al * dz_);
                // RK combination: acc_out = acc_in + acc_b k;  next = mn + dt (kc0 kin0 + ck k)
                accx[v] = p.acc_bT * kx + (p.acc_in ? ax_[v] : 0.f);
                accy[v] = p.acc_bT * ky + (p.acc_in ? ay_[v] : 0.f);
                accz[v] = p.acc_bT * kz + (p.acc_in ? az_[v] : 0.f);
                const float c0 = p.nk > 0 ? p.kcT[0] : 0.f;
                float a = mnx[v] + p.dtT * (p.ckT * kx + c0 * ax_[v]);
                float b = mny[v] + p.dtT * (p.ckT * ky + c0 * ay_[v]);
                float c = mnz[v] + p.dtT * (p.ckT * kz + c0 * az_[v]);
                if (p.renorm) {
                    const float nn = a * a + b * b + c * c;
                    if (nn > 0.f) {
                        const float sc = 1.f / sqrtf(nn);
                        a *= sc; b *= sc; c *= sc;
                    }
                }
                ox[v] = a; oy[v] = b; oz[v] = c;
                // Ms * next for the forward transform (the demag values at this place are consumed)
                w0[v * WS] = p.Ms * a; w1[v * WS] = p.Ms * b; w2[v * WS] = p.Ms * c;
            }
            if (p.acc_out) {
                float2* ao = reinterpret_cast<float2*>(p.acc_out);
                ao[i2] = make_float2(accx[0], accx[1]);
                ao[N2 + i2] = make_float2(accy[0], accy[1]);
                ao[2 * N2 + i2] = make_float2(accz[0], accz[1]);
            }
            float2* no = reinterpret_cast<float2*>(p.next);
            no[i2] = make_float2(ox[0], ox[1]);
            no[N2 + i2] = make_float2(oy[0], oy[1]);
            no[2 * N2 + i2] = make_float2(oz[0], oz[1]);
        }
        __syncthreads();
        // ---- forward transform of Ms * next and the real-pair post-processing
        {
            C v[FF::NR];
#pragma unroll
            for (int r = 0; r < FF::NR; ++r) v[r] = FF::in_live(r) ? work[wat(FF::in_index(j, r)) + line] : mk<C>(0, 0);
            FF::run(v, work + line, LS, j);
            __syncthreads();
#pragma unroll
            for (int r = 0; r < FF::NR; ++r) work[wat(j + r * FF::TPL) + line] = v[r];
        }
        __syncthreads();
        for (int idx = tid; idx < NL * KXn; idx += NT) {
            const int l = idx / KXn, k = idx - l * KXn;
            const int c = l / (TY / 2), q = l - c * (TY / 2);
            const int ya = y0 + 2 * q, yb = ya + 1;
            const C zk = work[wat(k) + l];
            const C zm = work[wat(k == 0 ? 0 : LX - k) + l];   // mirror index, any even LX
            if (ya < ny) S1[((long)(c * nz + z) * ny + ya) * d.KXS + k] = mk<C>(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
            if (yb < ny) S1[((long)(c * nz + z) * ny + yb) * d.KXS + k] = mk<C>(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
        }
        __syncthreads();   // work area free for the next tile
    }
}

// ------------------------------------------------------------- P2 / P4 ----
// DIR = -1: S1 (ny rows) -> S2 (Py rows), forward, zero upper half.
// DIR = +1: S2 (Py rows) -> S1 (ny rows), inverse, keep the lower half.
template <typename T, int LY, int B, int G, int DIR>
__global__ void __launch_bounds__(B * G * Fft<T, LY, DIR, (DIR < 0 && LY > 1)>::TPL)
p_y_pass(DemagDims d, const typename Cplx<T>::type* __restrict__ in,
         typename Cplx<T>::type* __restrict__ out) {
    using C = typename Cplx<T>::type;
    constexpr bool ZIN = DIR < 0 && LY > 1;
    using F = Fft<T, LY, DIR, ZIN>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* s = reinterpret_cast<C*>(smraw);
    constexpr int NL = B * G;
    const int tid = threadIdx.x;
    const int line = tid % NL, j = tid / NL;
    const int kl = line % B, g = line / B;
    const int kx = blockIdx.x * B + kl;
    const int cz = blockIdx.y * G + g;
    const bool valid = kx < d.KX && cz < d.nb * 3 * d.nz;
    const int rows_in = DIR < 0 ? d.ny : LY;
    const int rows_out = DIR < 0 ? LY : d.ny;
    const C* src = in + ((long)cz * rows_in) * d.KXS + kx;
    C* dst = out + ((long)cz * rows_out) * d.KXS + kx;
    C v[F::NR];
#pragma unroll
    for (int r = 0; r < F::NR; ++r) {
        const int e = F::in_index(j, r);
        v[r] = mk<C>(0, 0);
        if (valid && F::in_live(r) && e < rows_in) v[r] = src[(long)e * d.KXS];
    }
    F::run(v, s + line, NL, j);
    if (valid) {
#pragma unroll
        for (int r = 0; r < F::NR; ++r) {
            const int e = j + r * F::TPL;
            if (e < rows_out) dst[(long)e * d.KXS] = v[r];
        }
    }
}

// ------------------------------------------------------- P2 / P4 (TMA) ----
// Persistent, double-buffered y pass for FP32: each CTA walks tiles of B kx
// columns x all rows of one (component, z) plane; the tile after next is
// fetched by the tensor-memory accelerator into the shared-memory slot the
// finished tile frees, so HBM traffic overlaps the transforms.  Each thread
// transforms two adjacent columns at once on the paired engine (FftPair16):
// every butterfly instruction serves both columns and the twiddles, which
// both share, are read once.  B / 2 column pairs x L / 16 threads per CTA; the
// tile's slot is the exchange scratch (row e of pair p at P2 index e B/2 + p:
// the same bytes as the tile's row e, columns 2p and 2p + 1).  Every mbarrier
// wait is bounded; on timeout the CTA records kErrTmaTimeout, waits (bounded)
// for its other copy in flight and leaves.
template <int L, int B, int DIR>
__global__ void __launch_bounds__((B / 2) * FftPair16<L, DIR, (DIR < 0)>::TPL, 3)
p_y_tma(DemagDims d, const __grid_constant__ CUtensorMap in_map, float2* __restrict__ out, int box_rows,
         int nboxes) {
    constexpr bool ZIN = DIR < 0;
    using F = FftPair16<L, DIR, ZIN>;
    constexpr int NP = B / 2, TPL = F::TPL, NR = F::NR;
    static_assert(B % 2 == 0, "columns are taken in pairs");
    extern __shared__ __align__(128) unsigned char smtma[];
    float2* slot0 = reinterpret_cast<float2*>(smtma);
    float2* slot1 = slot0 + L * B;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smtma + 2 * (size_t)L * B * sizeof(float2));
    const int tid = threadIdx.x;
    const int pr = tid % NP, j = tid / NP;
    const int rows_in = DIR < 0 ? d.ny : L;
    const int rows_out = DIR < 0 ? L : d.ny;
    const int nkt = (d.KX + B - 1) / B;
    const int ntiles = nkt * 3 * d.nz * d.nb;      // (grid, component, z) planes of a batch, grid-major
    const uint32_t tile_bytes = (uint32_t)(nboxes * box_rows * B * sizeof(float2));
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    grid_dep_wait();      // the previous pass's output is complete from here on
    auto issue = [&](int t, int sl) {
        const int kt = t % nkt, cz = t / nkt;
        float2* dst = sl ? slot1 : slot0;
        mbar_arrive_expect_tx(&bar[sl], tile_bytes);
        for (int b = 0; b < nboxes; ++b)
            tma_load_3d(dst + (size_t)b * box_rows * B, &in_map, &bar[sl], kt * B, b * box_rows, cz);
    };
    const int t0 = blockIdx.x;
    if (tid == 0) {
        if (t0 < ntiles) issue(t0, 0);
        if (t0 + (int)gridDim.x < ntiles) issue(t0 + gridDim.x, 1);
    }
    int i = 0;
    for (int t = t0; t < ntiles; t += gridDim.x, ++i) {
        pdl_trigger_late(t + (int)gridDim.x >= ntiles);
        const int sl = i & 1;
        float2* cur = sl ? slot1 : slot0;
        const bool ok = mbar_wait_bounded(&bar[sl], (i >> 1) & 1);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(d.err, kErrTmaTimeout);
                if (t + (int)gridDim.x < ntiles) mbar_wait_bounded(&bar[sl ^ 1], ((i + 1) >> 1) & 1);
            }
            return;
        }
        P2 v[NR];
        const float4* cur4 = reinterpret_cast<const float4*>(cur);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int e = F::in_index(j, r);
            if (F::in_live(r) && e < rows_in) {
                const float4 q = cur4[e * NP + pr];
                v[r].re = make_float2(q.x, q.z);
                v[r].im = make_float2(q.y, q.w);
            } else {
                v[r].re = make_float2(0.f, 0.f);
                v[r].im = make_float2(0.f, 0.f);
            }
        }
        F::run(v, reinterpret_cast<P2*>(cur) + pr, NP, j);
        const int kt = t % nkt, cz = t / nkt;
        const int kx = kt * B + 2 * pr;
        if (kx < d.KX) {
            float2* dst = out + ((long)cz * rows_out) * d.KXS + kx;
            const bool both = kx + 1 < d.KX;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int e = j + r * TPL;
                if (e < rows_out) {
                    if (both)
                        *reinterpret_cast<float4*>(dst + (long)e * d.KXS) =
                            make_float4(v[r].re.x, v[r].im.x, v[r].re.y, v[r].im.y);
                    else
                        dst[(long)e * d.KXS] = make_float2(v[r].re.x, v[r].im.x);
                }
            }
        }
        __syncthreads();   // every thread is done with this slot
        if (tid == 0 && t + 2 * (int)gridDim.x < ntiles) {
            fence_proxy_async_smem();
            issue(t + 2 * gridDim.x, sl);
        }
    }
}

// ------------------------------------------------------------------ P3 ----
// resident CTAs asked of the register allocator: 1024 (FP32) or 512 (FP64) threads per SM
// (mixed-radix lines: one, their three parked components fill shared memory anyway)
template <typename T, int L = 2> constexpr int p3_min_blocks(int threads) {
    return !is_pow2(L) ? 1
           : (sizeof(T) == 4 ? 1024 : 512) / threads > 1 ? (sizeof(T) == 4 ? 1024 : 512) / threads : 1;
}

// Three shared-memory areas, one per component, each the FFT scratch of its
// component: every global load of the column tile is issued first and parked
// in its area, then each component is transformed in place, the 3x3 multiply
// reads and rewrites the areas, and each inverse transform streams its kept
// half straight to global memory.  Only one component's registers are live at
// a time, which keeps the kernel at four CTAs per SM.
template <typename T, int LZ, int B, int G>
__global__ void __launch_bounds__(B * G * Fft<T, LZ, -1, (LZ > 1)>::TPL,
                                  p3_min_blocks<T, LZ>(B * G * Fft<T, LZ, -1, (LZ > 1)>::TPL))
p3_z_conv(DemagDims d, typename Cplx<T>::type* __restrict__ S2, const T* __restrict__ tens) {
    using C = typename Cplx<T>::type;
    using FF = Fft<T, LZ, -1, (LZ > 1)>;
    using FI = Fft<T, LZ, +1, false>;
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int NL = B * G;
    constexpr int NR = FF::NR, TPL = FF::TPL;
    constexpr int NIN = LZ == 1 ? 1 : NR / 2;     // registers holding input / kept output
    C* area[3];
    area[0] = reinterpret_cast<C*>(smraw);
    area[1] = area[0] + LZ * NL;
    area[2] = area[1] + LZ * NL;
    const int tid = threadIdx.x;
    const int line = tid % NL, j = tid / NL;
    const int kl = line % B, g = line / B;
    const int kx = blockIdx.x * B + kl;
    const int kyi = blockIdx.y * G + g;           // (folded ky, side) pairs, side fastest
    const int p = kyi >> 1, side = kyi & 1;
    const int LY = d.LY;
    const int KY2 = LY / 2 + 1;
    const bool valid = kx < d.KX && p < KY2 && (side == 0 || (p > 0 && 2 * p < LY));
    const int ky = side ? LY - p : p;
    const long cstride = (long)d.nz * LY * d.KXS;   // component stride in S2
    C* col = S2 + (long)blockIdx.z * 3 * cstride + (long)ky * d.KXS + kx;   // (c, z) at col[c*cstride + z*LY*KXS]
    const long zs = (long)LY * d.KXS;

    if constexpr (NR <= 16) {   // all loads in flight together, parked at this thread's own (pattern) positions
        C in[3][NR];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int z = FF::in_index(j, r);
                in[c][r] = (FF::in_live(r) && valid && z < d.nz) ? col[c * cstride + z * zs] : mk<C>(0, 0);
            }
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < NR; ++r)
                if (FF::in_live(r)) area[c][(j + r * TPL) * NL + line] = in[c][r];
    } else {                    // long mixed-radix lines: straight to shared memory, one component at a time
#pragma unroll 1
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int z = FF::in_index(j, r);
                if (FF::in_live(r))
                    area[c][(j + r * TPL) * NL + line] = (valid && z < d.nz) ? col[c * cstride + z * zs] : mk<C>(0, 0);
            }
    }
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        C v[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) v[r] = FF::in_live(r) ? area[c][(j + r * TPL) * NL + line] : mk<C>(0, 0);
        FF::run(v, area[c] + line, NL, j);
#pragma unroll
        for (int r = 0; r < NR; ++r) area[c][(j + r * TPL) * NL + line] = v[r];
    }
    // h^ = T M^ at this thread's wave numbers (its own positions in the three areas)
    const int KZ2 = LZ / 2 + 1;
    const long tcomp = (long)KZ2 * KY2 * d.KXS;
    const T sy = side ? (T)-1 : (T)1;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int kz = j + r * TPL;
        const int kzf = (2 * kz <= LZ) ? kz : LZ - kz;
        const T sz = (2 * kz <= LZ) ? (T)1 : (T)-1;
        T txx = 0, txy = 0, txz = 0, tyy = 0, tyz = 0, tzz = 0;
        if (valid) {
            const T* tp = tens + ((long)kzf * KY2 + p) * d.KXS + kx;
            txx = __ldg(tp);
            txy = (d.yz_swap ? sz : sy) * __ldg(tp + tcomp);
            txz = (d.yz_swap ? sy : sz) * __ldg(tp + 2 * tcomp);
            tyy = __ldg(tp + 3 * tcomp);
            tyz = sy * sz * __ldg(tp + 4 * tcomp);
            tzz = __ldg(tp + 5 * tcomp);
        }
        const int o = (j + r * TPL) * NL + line;
        const C mx = area[0][o], my = area[1][o], mz = area[2][o];
        area[0][o] = mk<C>(txx * mx.x + txy * my.x + txz * mz.x, txx * mx.y + txy * my.y + txz * mz.y);
        area[1][o] = mk<C>(txy * mx.x + tyy * my.x + tyz * mz.x, txy * mx.y + tyy * my.y + tyz * mz.y);
        area[2][o] = mk<C>(txz * mx.x + tyz * my.x + tzz * mz.x, txz * mx.y + tyz * my.y + tzz * mz.y);
    }
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        C v[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) v[r] = area[c][(j + r * TPL) * NL + line];
        FI::run(v, area[c] + line, NL, j);
        if (valid) {
#pragma unroll
            for (int r = 0; r < NIN; ++r) {
                const int z = j + r * TPL;
                if (z < d.nz) col[c * cstride + z * zs] = v[r];
            }
        }
    }
}

// Register-resident variant (FP32): each thread keeps its 16 values of all
// three components from the first load to the last store; shared memory only
// carries the exchanges inside each transform (one per 128-point transform).
template <typename T, int LZ, int B, int G>
__global__ void __launch_bounds__(B * G * Fft<T, LZ, -1, (LZ > 1)>::TPL,
                                  (384 / (B * G * Fft<T, LZ, -1, (LZ > 1)>::TPL)) > 1
                                      ? 384 / (B * G * Fft<T, LZ, -1, (LZ > 1)>::TPL) : 1)
p3_z_conv_reg(DemagDims d, typename Cplx<T>::type* __restrict__ S2, const T* __restrict__ tens) {
    using C = typename Cplx<T>::type;
    using FF = Fft<T, LZ, -1, (LZ > 1)>;
    using FI = Fft<T, LZ, +1, false>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* s = reinterpret_cast<C*>(smraw);
    constexpr int NL = B * G;
    constexpr int NR = FF::NR, TPL = FF::TPL;
    constexpr int NOUT = LZ == 1 ? 1 : NR / 2;
    const int tid = threadIdx.x;
    const int line = tid % NL, j = tid / NL;
    const int kl = line % B, g = line / B;
    const int kx = blockIdx.x * B + kl;
    const int kyi = blockIdx.y * G + g;           // (folded ky, side) pairs, side fastest
    const int p = kyi >> 1, side = kyi & 1;
    const int LY = d.LY;
    const int KY2 = LY / 2 + 1;
    const bool valid = kx < d.KX && p < KY2 && (side == 0 || (p > 0 && 2 * p < LY));
    const int ky = side ? LY - p : p;
    const long cstride = (long)d.nz * LY * d.KXS;
    C* col = S2 + (long)blockIdx.z * 3 * cstride + (long)ky * d.KXS + kx;
    const long zs = (long)LY * d.KXS;

    C vx[NR], vy[NR], vz[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int z = FF::in_index(j, r);
        vx[r] = vy[r] = vz[r] = mk<C>(0, 0);
        if (valid && FF::in_live(r) && z < d.nz) {
            vx[r] = col[z * zs];
            vy[r] = col[cstride + z * zs];
            vz[r] = col[2 * cstride + z * zs];
        }
    }
    FF::run(vx, s + line, NL, j);
    FF::run(vy, s + line, NL, j);
    FF::run(vz, s + line, NL, j);
    const int KZ2 = LZ / 2 + 1;
    const long tcomp = (long)KZ2 * KY2 * d.KXS;
    const T sy = side ? (T)-1 : (T)1;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int kz = j + r * TPL;
        const int kzf = (2 * kz <= LZ) ? kz : LZ - kz;
        const T sz = (2 * kz <= LZ) ? (T)1 : (T)-1;
        T txx = 0, txy = 0, txz = 0, tyy = 0, tyz = 0, tzz = 0;
        if (valid) {
            const T* tp = tens + ((long)kzf * KY2 + p) * d.KXS + kx;
            txx = __ldg(tp);
            txy = (d.yz_swap ? sz : sy) * __ldg(tp + tcomp);
            txz = (d.yz_swap ? sy : sz) * __ldg(tp + 2 * tcomp);
            tyy = __ldg(tp + 3 * tcomp);
            tyz = sy * sz * __ldg(tp + 4 * tcomp);
            tzz = __ldg(tp + 5 * tcomp);
        }
        const C mx = vx[r], my = vy[r], mz = vz[r];
        vx[r] = mk<C>(txx * mx.x + txy * my.x + txz * mz.x, txx * mx.y + txy * my.y + txz * mz.y);
        vy[r] = mk<C>(txy * mx.x + tyy * my.x + tyz * mz.x, txy * mx.y + tyy * my.y + tyz * mz.y);
        vz[r] = mk<C>(txz * mx.x + tyz * my.x + tzz * mz.x, txz * mx.y + tyz * my.y + tzz * mz.y);
    }
    FI::run(vx, s + line, NL, j);
    FI::run(vy, s + line, NL, j);
    FI::run(vz, s + line, NL, j);
    if (valid) {
#pragma unroll
        for (int r = 0; r < NOUT; ++r) {
            const int z = j + r * TPL;
            if (z < d.nz) {
                col[z * zs] = vx[r];
                col[cstride + z * zs] = vy[r];
                col[2 * cstride + z * zs] = vz[r];
            }
        }
    }
}

// ----------------------------------------------------------- P3 layers ----
// Non-equidistant layers (Sec. 4.4): no transform along z; at every lateral
// wave number (kx, ky) the nz layers are coupled densely,
//   h^_i = sum_j K_ij(kx, ky) M^_j,
// with K_ij the 2-D spectrum of the layer-pair tensor (scaled by -1/(Px Py)).
// Only pairs i <= j are stored, for ky <= Py/2.  Two sign identities fold
// the rest into the operands:
//   * the mirrored row ky = Py - p flips the components odd in y (xy, yz):
//     K(Py - p) = E K(p) E with E = diag(1, -1, 1);
//   * h_i N_ij(r) = h_j N_ji(-r) gives K_ij(k) = (h_j / h_i) K_ji(-k), and -k
//     flips the single-odd components (xz, yz): K(-k) = D K(k) D with
//     D = diag(1, 1, -1).
// So with P_j = E M^_j and Q_j = h_j D P_j (both parked in shared memory),
//   h^_i = E [ sum_{j >= i} K_ij P_j + (1 / h_i) D sum_{j < i} K_ji Q_j ],
// and the inner loops are plain multiply-adds of stored entries.
// A CTA takes 32 kx columns of one ky (the mirrored ky = Py - p next to it, so
// both read the tensor row p while it is in L2); each thread row computes
// whole layers and writes them back in place once every input is parked.
constexpr int kLayCols = 32, kLayRows = 8;

__host__ __device__ constexpr int layer_pair(int i, int j, int nz) { return i * nz - i * (i - 1) / 2 + (j - i); }

// acc += K v for one stored pair: xx, xy, yy, zz real; xz, yz are -i t.
// GLOBAL: tp points into the tensor in global memory (read-only path),
// otherwise into the shared-memory copy of the CTA's tensor slice.
template <typename T, typename C, bool GLOBAL>
__device__ __forceinline__ void layer_mac(const T* __restrict__ tp, long tc, const C& vx, const C& vy, const C& vz,
                                          T& axr, T& axi, T& ayr, T& ayi, T& azr, T& azi) {
    T txx, txy, txz, tyy, tyz, tzz;
    if constexpr (GLOBAL) {
        txx = __ldg(tp); txy = __ldg(tp + tc); txz = __ldg(tp + 2 * tc);
        tyy = __ldg(tp + 3 * tc); tyz = __ldg(tp + 4 * tc); tzz = __ldg(tp + 5 * tc);
    } else {
        txx = tp[0]; txy = tp[tc]; txz = tp[2 * tc]; tyy = tp[3 * tc]; tyz = tp[4 * tc]; tzz = tp[5 * tc];
    }
    // (-i t)(a + i b) = t b - i t a
    axr += txx * vx.x + txy * vy.x + txz * vz.y;
    axi += txx * vx.y + txy * vy.y - txz * vz.x;
    ayr += txy * vx.x + tyy * vy.x + tyz * vz.y;
    ayi += txy * vx.y + tyy * vy.y - tyz * vz.x;
    azr += txz * vx.y + tyz * vy.y + tzz * vz.x;
    azi += tzz * vz.y - txz * vx.x - tyz * vy.x;
}

template <typename T>
__global__ void __launch_bounds__(kLayCols * kLayRows)
p3_layers(DemagDims d, typename Cplx<T>::type* __restrict__ S, const T* __restrict__ tens) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nz = d.nz, LY = d.LY, KY2 = LY / 2 + 1;
    C* sP = reinterpret_cast<C*>(smraw);          // [nz][3][kLayCols]: P_j
    C* sQ = sP + 3 * nz * kLayCols;               // [nz][3][kLayCols]: Q_j
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int kx = blockIdx.x * kLayCols + tx;
    const int p = blockIdx.y >> 1, side = blockIdx.y & 1;
    const bool row_ok = p < KY2 && (side == 0 || (p > 0 && 2 * p < LY));
    const bool valid = row_ok && kx < d.KX;
    const int ky = side ? LY - p : p;
    const long zs = (long)LY * d.KXS;                       // one (component, layer) plane
    C* col = S + (long)blockIdx.z * 3 * nz * zs + (long)ky * d.KXS + kx;
    const T* lh = static_cast<const T*>(d.lh);
    const T e = side ? (T)-1 : (T)1;
    for (int q = ty; q < 3 * nz; q += kLayRows) {
        const int c = q / nz, j = q - c * nz;
        C v = valid ? col[q * zs] : mk<C>(0, 0);
        if (c == 1) { v.x *= e; v.y *= e; }
        const T w = (c == 2 ? -lh[j] : lh[j]);
        sP[(j * 3 + c) * kLayCols + tx] = v;
        sQ[(j * 3 + c) * kLayCols + tx] = mk<C>(w * v.x, w * v.y);
    }
    __syncthreads();
    if (!valid) return;
    const long prow = (long)KY2 * d.KXS;                    // one pair
    const long tc = (long)(nz * (nz + 1) / 2) * prow;       // one component
    const T* t0 = tens + (long)p * d.KXS + kx;
    for (int i = ty; i < nz; i += kLayRows) {
        T axr = 0, axi = 0, ayr = 0, ayi = 0, azr = 0, azi = 0;
        {   // j >= i: pairs q(i, i) .. q(i, nz - 1) are consecutive
            const T* tp = t0 + (long)layer_pair(i, i, nz) * prow;
#pragma unroll 1
            for (int j = i; j < nz; ++j, tp += prow) {
                const C* v = sP + j * 3 * kLayCols + tx;
                layer_mac<T, C, true>(tp, tc, v[0], v[kLayCols], v[2 * kLayCols], axr, axi, ayr, ayi, azr, azi);
            }
        }
        T bxr = 0, bxi = 0, byr = 0, byi = 0, bzr = 0, bzi = 0;
        {   // j < i: pair q(j, i); q(j + 1, i) - q(j, i) = nz - j - 1
            const T* tp = t0 + (long)i * prow;              // q(0, i) = i
#pragma unroll 1
            for (int j = 0; j < i; ++j) {
                const C* v = sQ + j * 3 * kLayCols + tx;
                layer_mac<T, C, true>(tp, tc, v[0], v[kLayCols], v[2 * kLayCols], bxr, bxi, byr, byi, bzr, bzi);
                tp += (long)(nz - j - 1) * prow;
            }
        }
        const T ih = (T)1 / lh[i];
        const T cz = -ih;                                   // D on the lower-triangle sum
        col[(long)i * zs] = mk<C>(axr + ih * bxr, axi + ih * bxi);
        col[(long)(nz + i) * zs] = mk<C>(e * (ayr + ih * byr), e * (ayi + ih * byi));
        col[(long)(2 * nz + i) * zs] = mk<C>(azr + cz * bzr, azi + cz * bzi);
    }
}

// The same coupling with everything a CTA reads staged in shared memory by
// TMA in one round trip: the tensor slice of row p (6 components x all stored
// pairs x 32 columns) and the 3 nz input planes of the 32 columns for both
// rows that share the slice, ky = p and its mirror ky = Py - p.  Every staged
// tensor entry is read once and applied to both rows.  For stacks whose slice
// fits (npair <= 256 and 3 nz <= 256 per box dimension, shared memory
// permitting).  The wait is bounded: on timeout the CTA records
// kErrTmaTimeout, waits (bounded) once more for its copies and leaves.
template <typename T, typename C>
__device__ __forceinline__ void layer_fma(const T (&t)[6], const C* v, int ps, T (&a)[6]) {
    const C vx = v[0], vy = v[ps], vz = v[2 * ps];
    // xx, xy, yy, zz real; xz, yz are -i t: (-i t)(a + i b) = t b - i t a
    a[0] += t[0] * vx.x + t[1] * vy.x + t[2] * vz.y;
    a[1] += t[0] * vx.y + t[1] * vy.y - t[2] * vz.x;
    a[2] += t[1] * vx.x + t[3] * vy.x + t[4] * vz.y;
    a[3] += t[1] * vx.y + t[3] * vy.y - t[4] * vz.x;
    a[4] += t[2] * vx.y + t[4] * vy.y + t[5] * vz.x;
    a[5] += t[5] * vz.y - t[2] * vx.x - t[4] * vy.x;
}

// h^_i = E [A + (1 / h_i) D B] written to the column's three planes of layer i
template <typename T, typename C>
__device__ __forceinline__ void layer_store(C* col, long zs, int nz, int i, T ih, T e, const T (&a)[6],
                                            const T (&b)[6]) {
    col[(long)i * zs] = mk<C>(a[0] + ih * b[0], a[1] + ih * b[1]);
    col[(long)(nz + i) * zs] = mk<C>(e * (a[2] + ih * b[2]), e * (a[3] + ih * b[3]));
    col[(long)(2 * nz + i) * zs] = mk<C>(a[4] - ih * b[4], a[5] - ih * b[5]);
}

template <typename T>
__global__ void __launch_bounds__(kLayCols * kLayRows)
p3_layers_tma(DemagDims d, const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap smap,
              typename Cplx<T>::type* __restrict__ S) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(128) unsigned char smtma[];
    const int nz = d.nz, LY = d.LY;
    const int npair = nz * (nz + 1) / 2;
    const int pl = 3 * nz * kLayCols;                                      // one row's planes
    T* sT = reinterpret_cast<T*>(smtma);                                   // [6][npair][kLayCols]
    C* sP = reinterpret_cast<C*>(sT + 6 * npair * kLayCols);              // [row][c nz + j][kLayCols]
    C* sQ = sP + 2 * pl;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sQ + 2 * pl);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kLayCols + tx;
    const int p = blockIdx.y;
    const bool two = p > 0 && 2 * p < LY;                                  // a distinct mirrored row
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        const uint32_t tb = (uint32_t)(6 * npair * kLayCols * sizeof(T)), mb = (uint32_t)(pl * sizeof(C));
        mbar_arrive_expect_tx(bar, tb + (two ? 2 : 1) * mb);
        tma_load_4d(sT, &tmap, bar, blockIdx.x * kLayCols, p, 0, 0);
        const int xw = blockIdx.x * kLayCols * (int)(sizeof(C) / 8);       // 8-byte elements
        tma_load_3d(sP, &smap, bar, xw, p, 0);
        if (two) tma_load_3d(sP + pl, &smap, bar, xw, LY - p, 0);
    }
    __syncthreads();                        // the barrier's init is visible to every waiting thread
    const bool ok = mbar_wait_bounded(bar, 0);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) {
            atomicExch(d.err, kErrTmaTimeout);
            mbar_wait_bounded(bar, 0);
        }
        return;
    }
    // P = E M (E on the mirrored row), Q = h_j D P, each thread on its own column
    const T* lh = static_cast<const T*>(d.lh);
    for (int side = 0; side < (two ? 2 : 1); ++side)
        for (int q = ty; q < 3 * nz; q += kLayRows) {
            const int c = q >= 2 * nz ? 2 : (q >= nz ? 1 : 0), j = q - c * nz;
            C v = sP[side * pl + q * kLayCols + tx];
            if (side && c == 1) { v.x = -v.x; v.y = -v.y; sP[side * pl + q * kLayCols + tx] = v; }
            const T w = c == 2 ? -lh[j] : lh[j];
            sQ[side * pl + q * kLayCols + tx] = mk<C>(w * v.x, w * v.y);
        }
    __syncthreads();
    const int kx = blockIdx.x * kLayCols + tx;
    if (kx >= d.KX) return;
    const long zs = (long)LY * d.KXS;
    const long tc = (long)npair * kLayCols;
    const int ps = nz * kLayCols;
    for (int i = ty; i < nz; i += kLayRows) {
        T a0[6] = {0, 0, 0, 0, 0, 0}, a1[6] = {0, 0, 0, 0, 0, 0};
        T b0[6] = {0, 0, 0, 0, 0, 0}, b1[6] = {0, 0, 0, 0, 0, 0};
        const T* tp = sT + (long)layer_pair(i, i, nz) * kLayCols + tx;    // j >= i: consecutive pairs
        for (int j = i; j < nz; ++j, tp += kLayCols) {
            const T t[6] = {tp[0], tp[tc], tp[2 * tc], tp[3 * tc], tp[4 * tc], tp[5 * tc]};
            layer_fma<T, C>(t, sP + j * kLayCols + tx, ps, a0);
            if (two) layer_fma<T, C>(t, sP + pl + j * kLayCols + tx, ps, a1);
        }
        tp = sT + (long)i * kLayCols + tx;                                // j < i: pair q(j, i)
        for (int j = 0; j < i; ++j) {
            const T t[6] = {tp[0], tp[tc], tp[2 * tc], tp[3 * tc], tp[4 * tc], tp[5 * tc]};
            layer_fma<T, C>(t, sQ + j * kLayCols + tx, ps, b0);
            if (two) layer_fma<T, C>(t, sQ + pl + j * kLayCols + tx, ps, b1);
            tp += (long)(nz - j - 1) * kLayCols;
        }
        const T ih = (T)1 / lh[i];
        layer_store<T, C>(S + (long)p * d.KXS + kx, zs, nz, i, ih, (T)1, a0, b0);
        if (two) layer_store<T, C>(S + (long)(LY - p) * d.KXS + kx, zs, nz, i, ih, (T)-1, a1, b1);
    }
}

// Persistent TMA variant of the register-resident z pass (FP32, Pz <= 256):
// tile = (16 kx columns, one ky); tiles run ky = 0, 1, Py-1, 2, Py-2, ... so
// that the two wave numbers sharing a tensor slice are neighbours in time.
// Shared memory holds one tile's three z-columns (TMA box 16 x 1 x nz x 3 of
// S2), one tensor slice (box 16 x 1 x (Pz/2+1) x 6) and the transforms'
// exchange scratch.  The two loads complete on separate barriers and are
// single-buffered: the next tile's columns are requested as soon as this
// tile's are in registers, its tensor slice once the multiply has read this
// one, so each load has a whole transform to land in while three CTAs share
// an SM.
// z pass: the twiddles of its one radix-16 pass come from a per-CTA
// shared-memory table instead of being derived in every transform
// (141.5 -> 136.3 us on the bulk grid)
constexpr bool kZTwTab = true;
// the 96-point z line (8 x 12) on the two-factor engine
constexpr bool kZTwo = true;
// the radix-16 engine's plan for a z line: one radix-16 pass after the first, and its first radix
template <int L> __host__ __device__ constexpr bool z_one_pass16() {
    if constexpr (is_pow2(L) && L >= 16) return FftLine16<float, L, -1, true>::NPASS == 2;
    else return false;
}
template <int L> __host__ __device__ constexpr int z_r0() {
    if constexpr (is_pow2(L) && L >= 16) return FftLine16<float, L, -1, true>::R0;
    else return 1;
}

template <int LZ, int B> constexpr int p3_min_blocks_tma() {
    return (384 / (B * Fft<float, LZ, -1, (LZ > 1)>::TPL)) < 1 ? 1
           : (384 / (B * Fft<float, LZ, -1, (LZ > 1)>::TPL)) > 8 ? 8
           : 384 / (B * Fft<float, LZ, -1, (LZ > 1)>::TPL);
}

template <int LZ, int B>
__global__ void __launch_bounds__(B * Fft<float, LZ, -1, (LZ > 1)>::TPL, (p3_min_blocks_tma<LZ, B>()))
p3_z_tma(DemagDims d, const __grid_constant__ CUtensorMap s2_map, const __grid_constant__ CUtensorMap t_map,
         float2* __restrict__ S2, int s2_bytes, int t_bytes) {
    using C = float2;
    using FF = Fft<float, LZ, -1, (LZ > 1)>;
    using FI = Fft<float, LZ, +1, false>;
    constexpr int NR = FF::NR, TPL = FF::TPL;
    constexpr int NOUT = LZ == 1 ? 1 : NR / 2;
    constexpr int KZ2 = LZ / 2 + 1;
    extern __shared__ __align__(128) unsigned char smtma[];
    C* cs = reinterpret_cast<C*>(smtma);                                        // [c][z][kx]
    const float* ts = reinterpret_cast<const float*>(smtma + s2_bytes);         // [comp][kz'][kx]
    C* scr = reinterpret_cast<C*>(smtma + s2_bytes + t_bytes);                  // [LZ][kx]
    uint64_t* bar = reinterpret_cast<uint64_t*>(smtma + s2_bytes + t_bytes + (size_t)LZ * B * sizeof(C));
    const int tid = threadIdx.x;
    const int line = tid % B, j = tid / B;
    const int nz = d.nz, LY = d.LY;
    const int nkt = (d.KX + B - 1) / B;
    const int ntiles = nkt * LY;
    const uint32_t s2_tx = (uint32_t)(3 * nz * B * sizeof(C));
    const uint32_t t_tx = (uint32_t)(6 * KZ2 * B * sizeof(float));
    // the single radix-16 pass's twiddles of every butterfly k < R0 (one per
    // thread row j): read from shared memory instead of derived per transform
    constexpr bool TWT = kZTwTab && z_one_pass16<LZ>();
    __shared__ C twt[TWT ? 16 * 16 : 1];
    if constexpr (TWT) {
        constexpr int R0 = z_r0<LZ>();
        for (int e = tid; e < R0 * 16; e += blockDim.x) {
            const int k = e >> 4, q = e & 15;
            twt[e] = twiddle<float, LZ, -1>((k * q * (LZ / (16 * R0))) & (LZ - 1));
        }
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);     // S2 columns
        mbar_init(&bar[1], 1);     // tensor slice
        fence_mbar_init();
    }
    __syncthreads();
    const C* twk = TWT ? twt + 16 * (j & (z_r0<LZ>() - 1)) : nullptr;
    grid_dep_wait();      // the previous pass's output is complete from here on
    auto ky_of = [&](int kyo, int& p, int& side) {
        p = (kyo + 1) >> 1;
        side = (kyo > 0 && (kyo & 1) == 0) ? 1 : 0;
        return side ? LY - p : p;
    };
    auto issue_s2 = [&](int t) {
        const int kt = t % nkt, kyo = t / nkt;
        int p, side;
        const int ky = ky_of(kyo, p, side);
        mbar_arrive_expect_tx(&bar[0], s2_tx);
        tma_load_4d(smtma, &s2_map, &bar[0], kt * B, ky, 0, 0);
    };
    auto issue_t = [&](int t) {
        const int kt = t % nkt, kyo = t / nkt;
        int p, side;
        ky_of(kyo, p, side);
        mbar_arrive_expect_tx(&bar[1], t_tx);
        tma_load_4d(smtma + s2_bytes, &t_map, &bar[1], kt * B, p, 0, 0);
    };
    const int t0 = blockIdx.x;
    if (tid == 0 && t0 < ntiles) {
        issue_s2(t0);
        issue_t(t0);
    }
    int i = 0;
    for (int t = t0; t < ntiles; t += gridDim.x, ++i) {
        pdl_trigger_late(t + (int)gridDim.x >= ntiles);
        const uint32_t par = i & 1;
        const bool more = t + (int)gridDim.x < ntiles;
        bool ok = mbar_wait_bounded(&bar[0], par);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(d.err, kErrTmaTimeout);
                mbar_wait_bounded(&bar[0], par);                 // the late columns
                mbar_wait_bounded(&bar[1], par);                 // this tile's tensor slice is in flight
            }
            return;
        }
        const int kt = t % nkt, kyo = t / nkt;
        int p, side;
        const int ky = ky_of(kyo, p, side);
        C vx[NR], vy[NR], vz[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int z = FF::in_index(j, r);
            const bool live = FF::in_live(r) && z < nz;
            vx[r] = live ? cs[(0 * nz + z) * B + line] : mk<C>(0, 0);
            vy[r] = live ? cs[(1 * nz + z) * B + line] : mk<C>(0, 0);
            vz[r] = live ? cs[(2 * nz + z) * B + line] : mk<C>(0, 0);
        }
        __syncthreads();   // the columns are in registers: the buffer takes the next tile's
        if (tid == 0 && more) {
            fence_proxy_async_smem();
            issue_s2(t + gridDim.x);
        }
        FF::run(vx, scr + line, B, j, twk);
        FF::run(vy, scr + line, B, j, twk);
        FF::run(vz, scr + line, B, j, twk);
        ok = mbar_wait_bounded(&bar[1], par);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(d.err, kErrTmaTimeout);
                mbar_wait_bounded(&bar[1], par);                  // the late slice
                if (more) mbar_wait_bounded(&bar[0], par ^ 1u);   // the next tile's columns are in flight
            }
            return;
        }
        const float sy = side ? -1.f : 1.f;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int kz = j + r * TPL;
            const int kzf = (2 * kz <= LZ) ? kz : LZ - kz;
            const float sz = (2 * kz <= LZ) ? 1.f : -1.f;
            const float txx = ts[(0 * KZ2 + kzf) * B + line];
            const float txy = (d.yz_swap ? sz : sy) * ts[(1 * KZ2 + kzf) * B + line];
            const float txz = (d.yz_swap ? sy : sz) * ts[(2 * KZ2 + kzf) * B + line];
            const float tyy = ts[(3 * KZ2 + kzf) * B + line];
            const float tyz = sy * sz * ts[(4 * KZ2 + kzf) * B + line];
            const float tzz = ts[(5 * KZ2 + kzf) * B + line];
            const C mx = vx[r], my = vy[r], mz = vz[r];
            vx[r] = mk<C>(txx * mx.x + txy * my.x + txz * mz.x, txx * mx.y + txy * my.y + txz * mz.y);
            vy[r] = mk<C>(txy * mx.x + tyy * my.x + tyz * mz.x, txy * mx.y + tyy * my.y + tyz * mz.y);
            vz[r] = mk<C>(txz * mx.x + tyz * my.x + tzz * mz.x, txz * mx.y + tyz * my.y + tzz * mz.y);
        }
        __syncthreads();   // the slice has been read: the buffer takes the next tile's
        if (tid == 0 && more) {
            fence_proxy_async_smem();
            issue_t(t + gridDim.x);
        }
        FI::run(vx, scr + line, B, j, twk);
        FI::run(vy, scr + line, B, j, twk);
        FI::run(vz, scr + line, B, j, twk);
        const int kx = kt * B + line;
        if (kx < d.KX) {
            const long cstride = (long)nz * LY * d.KXS, zs = (long)LY * d.KXS;
            C* col = S2 + (long)ky * d.KXS + kx;
#pragma unroll
            for (int r = 0; r < NOUT; ++r) {
                const int z = j + r * TPL;
                if (z < nz) {
                    col[z * zs] = vx[r];
                    col[cstride + z * zs] = vy[r];
                    col[2 * cstride + z * zs] = vz[r];
                }
            }
        }
    }
}

// TMA z pass on the two-factor engine (FP32; L = R1 R2, e.g. 96 = 8 x 12):
// the tiles, loads, barriers and tensor product are those of p3_z_tma; each
// transform makes one exchange through the scratch area instead of one per
// radix pass, and the spectra stay in the forward's order (fr_index), which
// the tensor product and the inverse take as they are.
template <int R1, int R2> struct ZTwoTpl { static constexpr int value = 4; };
template <int R1, int R2, int B>
__global__ void __launch_bounds__(B * ZTwoTpl<R1, R2>::value, 4)
p3_z_two(DemagDims d, const __grid_constant__ CUtensorMap s2_map, const __grid_constant__ CUtensorMap t_map,
         float2* __restrict__ S2, int s2_bytes, int t_bytes) {
    using C = float2;
    constexpr int TPL = ZTwoTpl<R1, R2>::value;
    using FF = FftTwo<float, R1, R2, TPL, -1, true>;
    using FI = FftTwo<float, R1, R2, TPL, +1, false>;
    constexpr int LZ = R1 * R2, NR = FF::NR;
    constexpr int KZ2 = LZ / 2 + 1;
    extern __shared__ __align__(128) unsigned char smtma[];
    C* cs = reinterpret_cast<C*>(smtma);                                        // [c][z][kx]
    const float* ts = reinterpret_cast<const float*>(smtma + s2_bytes);         // [comp][kz'][kx]
    C* scr = reinterpret_cast<C*>(smtma + s2_bytes + t_bytes);                  // [LZ][kx]
    uint64_t* bar = reinterpret_cast<uint64_t*>(smtma + s2_bytes + t_bytes + (size_t)LZ * B * sizeof(C));
    __shared__ C tw[LZ];                                                        // W_L^m, forward sign
    const int tid = threadIdx.x;
    const int line = tid % B, j = tid / B;
    const int nz = d.nz, LY = d.LY;
    const int nkt = (d.KX + B - 1) / B;
    const int ntiles = nkt * LY;
    const uint32_t s2_tx = (uint32_t)(3 * nz * B * sizeof(C));
    const uint32_t t_tx = (uint32_t)(6 * KZ2 * B * sizeof(float));
    for (int e = tid; e < LZ; e += blockDim.x) tw[e] = twiddle5<float, -1>(e * (kTw5 / LZ));
    if (tid == 0) {
        mbar_init(&bar[0], 1);     // S2 columns
        mbar_init(&bar[1], 1);     // tensor slice
        fence_mbar_init();
    }
    __syncthreads();
    grid_dep_wait();      // the previous pass's output is complete from here on
    auto ky_of = [&](int kyo, int& p, int& side) {
        p = (kyo + 1) >> 1;
        side = (kyo > 0 && (kyo & 1) == 0) ? 1 : 0;
        return side ? LY - p : p;
    };
    auto issue_s2 = [&](int t) {
        const int kt = t % nkt, kyo = t / nkt;
        int p, side;
        const int ky = ky_of(kyo, p, side);
        mbar_arrive_expect_tx(&bar[0], s2_tx);
        tma_load_4d(smtma, &s2_map, &bar[0], kt * B, ky, 0, 0);
    };
    auto issue_t = [&](int t) {
        const int kt = t % nkt, kyo = t / nkt;
        int p, side;
        ky_of(kyo, p, side);
        mbar_arrive_expect_tx(&bar[1], t_tx);
        tma_load_4d(smtma + s2_bytes, &t_map, &bar[1], kt * B, p, 0, 0);
    };
    const int t0 = blockIdx.x;
    if (tid == 0 && t0 < ntiles) {
        issue_s2(t0);
        issue_t(t0);
    }
    int i = 0;
    for (int t = t0; t < ntiles; t += gridDim.x, ++i) {
        pdl_trigger_late(t + (int)gridDim.x >= ntiles);
        const uint32_t par = i & 1;
        const bool more = t + (int)gridDim.x < ntiles;
        bool ok = mbar_wait_bounded(&bar[0], par);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(d.err, kErrTmaTimeout);
                mbar_wait_bounded(&bar[0], par);                 // the late columns
                mbar_wait_bounded(&bar[1], par);                 // this tile's tensor slice is in flight
            }
            return;
        }
        const int kt = t % nkt, kyo = t / nkt;
        int p, side;
        const int ky = ky_of(kyo, p, side);
        C vx[NR], vy[NR], vz[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int z = FF::sp_index(j, r);
            const bool live = FF::sp_half(r) && z < nz;
            vx[r] = live ? cs[(0 * nz + z) * B + line] : mk<C>(0, 0);
            vy[r] = live ? cs[(1 * nz + z) * B + line] : mk<C>(0, 0);
            vz[r] = live ? cs[(2 * nz + z) * B + line] : mk<C>(0, 0);
        }
        __syncthreads();   // the columns are in registers: the buffer takes the next tile's
        if (tid == 0 && more) {
            fence_proxy_async_smem();
            issue_s2(t + gridDim.x);
        }
        FF::run(vx, scr + line, B, j, tw);
        FF::run(vy, scr + line, B, j, tw);
        FF::run(vz, scr + line, B, j, tw);
        ok = mbar_wait_bounded(&bar[1], par);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(d.err, kErrTmaTimeout);
                mbar_wait_bounded(&bar[1], par);                  // the late slice
                if (more) mbar_wait_bounded(&bar[0], par ^ 1u);   // the next tile's columns are in flight
            }
            return;
        }
        const float sy = side ? -1.f : 1.f;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int kz = FF::fr_index(j, r);
            const int kzf = (2 * kz <= LZ) ? kz : LZ - kz;
            const float sz = (2 * kz <= LZ) ? 1.f : -1.f;
            const float txx = ts[(0 * KZ2 + kzf) * B + line];
            const float txy = (d.yz_swap ? sz : sy) * ts[(1 * KZ2 + kzf) * B + line];
            const float txz = (d.yz_swap ? sy : sz) * ts[(2 * KZ2 + kzf) * B + line];
            const float tyy = ts[(3 * KZ2 + kzf) * B + line];
            const float tyz = sy * sz * ts[(4 * KZ2 + kzf) * B + line];
            const float tzz = ts[(5 * KZ2 + kzf) * B + line];
            const C mx = vx[r], my = vy[r], mz = vz[r];
            vx[r] = mk<C>(txx * mx.x + txy * my.x + txz * mz.x, txx * mx.y + txy * my.y + txz * mz.y);
            vy[r] = mk<C>(txy * mx.x + tyy * my.x + tyz * mz.x, txy * mx.y + tyy * my.y + tyz * mz.y);
            vz[r] = mk<C>(txz * mx.x + tyz * my.x + tzz * mz.x, txz * mx.y + tyz * my.y + tzz * mz.y);
        }
        __syncthreads();   // the slice has been read: the buffer takes the next tile's
        if (tid == 0 && more) {
            fence_proxy_async_smem();
            issue_t(t + gridDim.x);
        }
        FI::run(vx, scr + line, B, j, tw);
        FI::run(vy, scr + line, B, j, tw);
        FI::run(vz, scr + line, B, j, tw);
        const int kx = kt * B + line;
        if (kx < d.KX) {
            const long cstride = (long)nz * LY * d.KXS, zs = (long)LY * d.KXS;
            C* col = S2 + (long)ky * d.KXS + kx;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int z = FI::sp_index(j, r);
                if (FI::sp_half(r) && z < nz) {
                    col[z * zs] = vx[r];
                    col[cstride + z * zs] = vy[r];
                    col[2 * cstride + z * zs] = vz[r];
                }
            }
        }
    }
}

// ------------------------------------------------------------------ P5 ----
template <typename T, int LX, int NL>
__global__ void __launch_bounds__(NL * Fft<T, LX, +1, false>::TPL)
p5_x_inverse(DemagDims d, const typename Cplx<T>::type* __restrict__ S1, T* __restrict__ h) {
    using C = typename Cplx<T>::type;
    using F = Fft<T, LX, +1, false>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* s = reinterpret_cast<C*>(smraw);
    constexpr int LS = NL + 1;
    constexpr int NT = NL * F::TPL;
    constexpr int KXn = LX / 2 + 1;
    const int tid = threadIdx.x;
    const int line = tid % NL, j = tid / NL;
    __shared__ long ra_s[NL], rb_s[NL];
    pair_lines<NL>(d, ra_s, rb_s);
    __syncthreads();
    for (int idx = tid; idx < NL * KXn; idx += NT) {
        const int l = idx / KXn, k = idx - l * KXn;
        const long ra = ra_s[l], rb = rb_s[l];
        C A = mk<C>(0, 0), Bv = mk<C>(0, 0);
        if (ra >= 0) A = S1[ra * d.KXS + k];
        if (rb >= 0) Bv = S1[rb * d.KXS + k];
        if (k == 0 || 2 * k == LX) { A.y = 0; Bv.y = 0; }   // a real row has real DC and Nyquist
        s[k * LS + l] = mk<C>(A.x - Bv.y, A.y + Bv.x);
        if (k > 0 && 2 * k < LX) s[(LX - k) * LS + l] = mk<C>(A.x + Bv.y, Bv.x - A.y);
    }
    __syncthreads();
    C v[F::NR];
#pragma unroll
    for (int r = 0; r < F::NR; ++r) v[r] = s[(j + r * F::TPL) * LS + line];
    F::run(v, s + line, LS, j);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < F::NR; ++r)
        if (LX == 1 || r < F::NR / 2) s[(j + r * F::TPL) * LS + line] = v[r];
    __syncthreads();
    for (int idx = tid; idx < NL * d.nx; idx += NT) {
        const int l = idx / d.nx, x = idx - l * d.nx;
        const long ra = ra_s[l], rb = rb_s[l];
        const C z = s[x * LS + l];
        if (ra >= 0) h[ra * d.nx + x] = z.x;
        if (rb >= 0) h[rb * d.nx + x] = z.y;
    }
}

// ------------------------------------------------------------ launchers ----
template <typename T> struct Geo;
template <> struct Geo<float> { static constexpr int BS = 16; };   // 16 x 8 B = 128 B rows
template <> struct Geo<double> { static constexpr int BS = 8; };   // 8 x 16 B = 128 B rows

// threads per line of the engine a pass uses (forward and inverse engines of
// one precision and length have the same thread count)
template <typename T, int L> constexpr int tpl_of() { return Fft<T, L, +1, false>::TPL; }
// lines per CTA for the x passes: about 256 threads
template <typename T, int L> constexpr int nl_x() { return tpl_of<T, L>() >= 256 ? 1 : 256 / tpl_of<T, L>(); }
// kx columns per CTA for strided passes: 128-byte rows, at most 512 threads per group
template <typename T, int L> constexpr int b_of() {
    return (Geo<T>::BS * tpl_of<T, L>() <= 512) ? Geo<T>::BS
                                                : ((512 / tpl_of<T, L>()) < 2 ? 2 : 512 / tpl_of<T, L>());
}
template <typename T, int L> constexpr int g_of() {
    return (b_of<T, L>() * tpl_of<T, L>() >= 256) ? 1 : 256 / (b_of<T, L>() * tpl_of<T, L>());
}
// the shared-memory z pass parks three components of every line: keep its
// B x G lines within 200 KB (long FP64 lines take fewer columns per CTA)
constexpr size_t kP3Smem = 200 * 1024;
template <typename T, int L> constexpr int b_p3() {
    return (size_t)3 * L * b_of<T, L>() * sizeof(typename Cplx<T>::type) <= kP3Smem
               ? b_of<T, L>()
               : ((int)(kP3Smem / ((size_t)3 * L * sizeof(typename Cplx<T>::type))) < 1
                      ? 1 : (int)(kP3Smem / ((size_t)3 * L * sizeof(typename Cplx<T>::type))));
}
template <typename T, int L> constexpr int g_p3() {
    return (size_t)3 * L * b_p3<T, L>() * g_of<T, L>() * sizeof(typename Cplx<T>::type) <= kP3Smem
               ? g_of<T, L>()
               : ((int)(kP3Smem / ((size_t)3 * L * b_p3<T, L>() * sizeof(typename Cplx<T>::type))) < 1
                      ? 1 : (int)(kP3Smem / ((size_t)3 * L * b_p3<T, L>() * sizeof(typename Cplx<T>::type))));
}

// raise a kernel's dynamic shared-memory limit when the request comes near the
// 48 KB default (kernels may also hold a little static shared memory)
template <typename K> static void set_smem(K kernel, size_t bytes) {
    if (bytes > 40 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int L> static void launch_p1(const DemagDims& d, const T* m, const T* Ms_cell, T Ms,
                                                   typename Cplx<T>::type* S1, cudaStream_t st) {
    constexpr int NL = nl_x<T, L>();
    using C = typename Cplx<T>::type;
    const size_t sm = (size_t)L * (NL + 1) * sizeof(C);
    const long pairs = (long)d.nb * ((3L * d.ny * d.nz + 1) / 2);
    const unsigned grid = (unsigned)((pairs + NL - 1) / NL);
    auto k = p1_x_forward<T, L, NL>;
    set_smem(k, sm);
    k<<<grid, NL * tpl_of<T, L>(), sm, st>>>(d, m, Ms_cell, Ms, S1);
}

template <typename T, int L> static void launch_p5(const DemagDims& d, const typename Cplx<T>::type* S1, T* h,
                                                   cudaStream_t st) {
    constexpr int NL = nl_x<T, L>();
    using C = typename Cplx<T>::type;
    const size_t sm = (size_t)L * (NL + 1) * sizeof(C);
    const long pairs = (long)d.nb * ((3L * d.ny * d.nz + 1) / 2);
    const unsigned grid = (unsigned)((pairs + NL - 1) / NL);
    auto k = p5_x_inverse<T, L, NL>;
    set_smem(k, sm);
    k<<<grid, NL * tpl_of<T, L>(), sm, st>>>(d, S1, h);
}

template <typename T, int L, int DIR> static void launch_py(const DemagDims& d, const typename Cplx<T>::type* in,
                                                            typename Cplx<T>::type* out, cudaStream_t st) {
    constexpr int B = b_of<T, L>(), G = g_of<T, L>();
    using C = typename Cplx<T>::type;
    const size_t sm = (size_t)L * B * G * sizeof(C);
    dim3 grid((d.KX + B - 1) / B, (d.nb * 3 * d.nz + G - 1) / G);
    auto k = p_y_pass<T, L, B, G, DIR>;
    set_smem(k, sm);
    k<<<grid, B * G * tpl_of<T, L>(), sm, st>>>(d, in, out);
}

// ---- tensor maps (driver entry point looked up once through the runtime) ----
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 3-D map over 8-byte elements (one float complex), dims innermost first
static bool encode_3d(CUtensorMap* map, const void* base, const cuuint64_t dims[3], const cuuint64_t strides[2],
                      const cuuint32_t box[3]) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename K> static int persistent_grid(K kernel, int threads, size_t smem, int work) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem);
    const int g = sms * (occ > 0 ? occ : 1);
    return work < g ? work : g;
}

// launch with programmatic stream serialization (the kernel calls
// grid_dep_wait before it reads what the previous kernel wrote)
template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kernel)(KArgs...), int grid, int threads, size_t smem, cudaStream_t st,
                       Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// TMA y pass (FP32 only): returns false if it could not be used (caller falls back)
// kx columns per TMA tile: two slots of L x B complex floats stay within 128 KB
// kx columns per tile of the TMA y passes: about 4096 points per slot, and
// even, so that every tile's first column (x coordinate) is 16-byte aligned
template <int L> constexpr int b_tma() { return (4096 / L) >= 8 ? 8 : ((4096 / L) < 2 ? 2 : (4096 / L) & ~1); }
// lines the TMA z pass takes: powers of two and the mixed-radix 3 x 2^a lines
// (12 values per thread, no spills; measured 130 us against 162 us for the
// register-resident pass on 192x192x48).  The TMA y passes stay on powers of
// two: on the 384-point line they measured slower than the classic pass.
template <int L> constexpr bool tma_len() {
    return is_pow2(L) || Fft<float, L, -1, true>::NR <= 12;
}

template <int L, int DIR>
static bool launch_py_tma(const DemagDims& d, const float2* in, float2* out, cudaStream_t st) {
    constexpr int B = b_tma<L>();
    const int rows_in = DIR < 0 ? d.ny : L;
    static_assert(B % 2 == 0, "tile x coordinates must be 16-byte aligned");
    if (!d.err || d.nb != 1 || (d.KXS * 8) % 16 != 0 || (reinterpret_cast<uintptr_t>(in) & 15) != 0) return false;
    // the fewest boxes of at most 256 rows, rows split evenly; with several boxes
    // rounded up to 16 rows (each box then starts 128-byte aligned in the slot);
    // the slot holds L rows
    const int nboxes = (rows_in + 255) / 256;
    const int box_rows = nboxes == 1 ? rows_in : ((rows_in + nboxes - 1) / nboxes + 15) / 16 * 16;
    if (box_rows > 256 || (size_t)nboxes * box_rows > (size_t)L) return false;
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)d.KX, (cuuint64_t)rows_in, (cuuint64_t)(3 * d.nz * d.nb)};
    const cuuint64_t strides[2] = {(cuuint64_t)d.KXS * 8, (cuuint64_t)rows_in * d.KXS * 8};
    const cuuint32_t box[3] = {(cuuint32_t)B, (cuuint32_t)box_rows, 1};
    if (!encode_3d(&map, in, dims, strides, box)) return false;
    const size_t sm = 2 * (size_t)L * B * sizeof(float2) + 16;
    const int nkt = (d.KX + B - 1) / B;
    const int threads = (B / 2) * FftPair16<L, DIR, (DIR < 0)>::TPL;
    auto k = p_y_tma<L, B, DIR>;
    set_smem(k, sm);
    const int grid = persistent_grid(k, threads, sm, nkt * 3 * d.nz * d.nb);
    launch_pdl(k, grid, threads, sm, st, d, map, out, box_rows, nboxes);
    return true;
}

static bool encode_4d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, const cuuint64_t dims[4],
                      const cuuint64_t strides[3], const cuuint32_t box[4]) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return fn(map, dt, 4, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// TMA z pass (FP32, Pz <= 256, nz <= 256): false if it cannot be used
template <int L>
static bool launch_p3_tma(const DemagDims& d, float2* S2, const float* tens, cudaStream_t st) {
    constexpr int B = 16;
    if (!d.err || (d.KXS * 8) % 16 != 0 || (d.KXS * 4) % 16 != 0 || d.nz > 256 || L / 2 + 1 > 256) return false;
    if ((reinterpret_cast<uintptr_t>(S2) & 15) != 0 || (reinterpret_cast<uintptr_t>(tens) & 15) != 0) return false;
    const int KY2 = d.LY / 2 + 1, KZ2 = L / 2 + 1;
    CUtensorMap s2m, tm;
    const cuuint64_t sd[4] = {(cuuint64_t)d.KX, (cuuint64_t)d.LY, (cuuint64_t)d.nz, 3};
    const cuuint64_t ss[3] = {(cuuint64_t)d.KXS * 8, (cuuint64_t)d.LY * d.KXS * 8, (cuuint64_t)d.nz * d.LY * d.KXS * 8};
    const cuuint32_t sb[4] = {(cuuint32_t)B, 1, (cuuint32_t)d.nz, 3};
    const cuuint64_t td[4] = {(cuuint64_t)d.KX, (cuuint64_t)KY2, (cuuint64_t)KZ2, 6};
    const cuuint64_t ts[3] = {(cuuint64_t)d.KXS * 4, (cuuint64_t)KY2 * d.KXS * 4, (cuuint64_t)KZ2 * KY2 * d.KXS * 4};
    const cuuint32_t tb[4] = {(cuuint32_t)B, 1, (cuuint32_t)KZ2, 6};
    if (!encode_4d(&s2m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, S2, sd, ss, sb)) return false;
    if (!encode_4d(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, tens, td, ts, tb)) return false;
    const int s2_bytes = (int)((3 * (size_t)d.nz * B * sizeof(float2) + 127) / 128 * 128);
    const int t_bytes = (int)((6 * (size_t)KZ2 * B * sizeof(float) + 127) / 128 * 128);
    const int nkt = (d.KX + B - 1) / B;
    const size_t sm = (size_t)s2_bytes + t_bytes + (size_t)L * B * sizeof(float2) + 16;
    if (sm > 220 * 1024) return false;
    auto k = p3_z_tma<L, B>;
    set_smem(k, sm);
    const int threads = B * Fft<float, L, -1, (L > 1)>::TPL;
    const int grid = persistent_grid(k, threads, sm, nkt * d.LY);
    launch_pdl(k, grid, threads, sm, st, d, s2m, tm, S2, s2_bytes, t_bytes);
    return true;
}

// factors of the z lines that run the two-factor TMA z pass (0: none)
template <int L> constexpr int z_two_r1() { return L == 96 ? 8 : 0; }
template <int L> constexpr int z_two_r2() { return L == 96 ? 12 : 0; }

// TMA z pass on the two-factor engine: false if it cannot be used
template <int L>
static bool launch_p3_two(const DemagDims& d, float2* S2, const float* tens, cudaStream_t st) {
    constexpr int B = 16, R1 = z_two_r1<L>(), R2 = z_two_r2<L>();
    static_assert(R1 * R2 == L, "two-factor z line");
    if (!d.err || (d.KXS * 8) % 16 != 0 || (d.KXS * 4) % 16 != 0 || d.nz > L / 2) return false;
    if ((reinterpret_cast<uintptr_t>(S2) & 15) != 0 || (reinterpret_cast<uintptr_t>(tens) & 15) != 0) return false;
    const int KY2 = d.LY / 2 + 1, KZ2 = L / 2 + 1;
    CUtensorMap s2m, tm;
    const cuuint64_t sd[4] = {(cuuint64_t)d.KX, (cuuint64_t)d.LY, (cuuint64_t)d.nz, 3};
    const cuuint64_t ss[3] = {(cuuint64_t)d.KXS * 8, (cuuint64_t)d.LY * d.KXS * 8, (cuuint64_t)d.nz * d.LY * d.KXS * 8};
    const cuuint32_t sb[4] = {(cuuint32_t)B, 1, (cuuint32_t)d.nz, 3};
    const cuuint64_t td[4] = {(cuuint64_t)d.KX, (cuuint64_t)KY2, (cuuint64_t)KZ2, 6};
    const cuuint64_t ts[3] = {(cuuint64_t)d.KXS * 4, (cuuint64_t)KY2 * d.KXS * 4, (cuuint64_t)KZ2 * KY2 * d.KXS * 4};
    const cuuint32_t tb[4] = {(cuuint32_t)B, 1, (cuuint32_t)KZ2, 6};
    if (!encode_4d(&s2m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, S2, sd, ss, sb)) return false;
    if (!encode_4d(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, tens, td, ts, tb)) return false;
    const int s2_bytes = (int)((3 * (size_t)d.nz * B * sizeof(float2) + 127) / 128 * 128);
    const int t_bytes = (int)((6 * (size_t)KZ2 * B * sizeof(float) + 127) / 128 * 128);
    const int nkt = (d.KX + B - 1) / B;
    const size_t sm = (size_t)s2_bytes + t_bytes + (size_t)L * B * sizeof(float2) + 16;
    if (sm > 200 * 1024) return false;
    auto k = p3_z_two<R1, R2, B>;
    set_smem(k, sm);
    const int threads = B * ZTwoTpl<R1, R2>::value;
    const int grid = persistent_grid(k, threads, sm, nkt * d.LY);
    launch_pdl(k, grid, threads, sm, st, d, s2m, tm, S2, s2_bytes, t_bytes);
    return true;
}

// widest multiple of 8 elements <= 256 that covers n in the fewest boxes
static int box_width(int n, int* nboxes) {
    const int nb = (n + 255) / 256;
    int w = (n + nb - 1) / nb;
    w = (w + 7) / 8 * 8;
    *nboxes = (n + w - 1) / w;
    return w;
}

template <int L> static bool launch_p1_tma(const DemagDims& d, const float* m, const float* Ms_cell, float Ms,
                                           float2* S1, cudaStream_t st) {
    constexpr int NL = nl_x<float, L>();
    if (!d.err || d.nb != 1 || d.Ms_b || Ms_cell || L < 16 || (d.nx * 4) % 16 != 0 ||
        (reinterpret_cast<uintptr_t>(m) & 15) != 0)
        return false;
    if (2 * NL > 256) return false;
    int nb = 0;
    const int w = box_width(d.nx, &nb);
    const long rows = 3L * d.ny * d.nz;
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)d.nx, (cuuint64_t)rows, 1};
    const cuuint64_t strides[2] = {(cuuint64_t)d.nx * 4, (cuuint64_t)rows * d.nx * 4};
    const cuuint32_t box[3] = {(cuuint32_t)w, (cuuint32_t)(2 * NL), 1};
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint32_t es[3] = {1, 1, 1};
    if (fn(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(m), dims, strides, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const int slot_bytes = (int)(((size_t)nb * w * 2 * NL * sizeof(float) + 127) / 128 * 128);
    const size_t sm = 2 * (size_t)slot_bytes + (size_t)L * (NL + 1) * sizeof(float2) + 16;
    if (sm > 200 * 1024) return false;
    auto k = p1_x_tma<L, NL>;
    set_smem(k, sm);
    const int threads = NL * Fft<float, L, -1, (L > 1)>::TPL;
    const int ntiles = (int)((rows + 2 * NL - 1) / (2 * NL));
    const int grid = persistent_grid(k, threads, sm, ntiles);
    k<<<grid, threads, sm, st>>>(d, map, Ms, S1, w, nb, slot_bytes);
    return true;
}

template <int L> static bool launch_p5_tma(const DemagDims& d, const float2* S1, float* h, cudaStream_t st) {
    constexpr int NL = nl_x<float, L>();
    if (!d.err || d.nb != 1 || L < 16 || (d.KXS * 8) % 16 != 0 || (reinterpret_cast<uintptr_t>(S1) & 15) != 0)
        return false;
    if (2 * NL > 256) return false;
    int nb = 0;
    const int w = box_width(d.KX, &nb);
    const long rows = 3L * d.ny * d.nz;
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)d.KX, (cuuint64_t)rows, 1};
    const cuuint64_t strides[2] = {(cuuint64_t)d.KXS * 8, (cuuint64_t)rows * d.KXS * 8};
    const cuuint32_t box[3] = {(cuuint32_t)w, (cuuint32_t)(2 * NL), 1};
    if (!encode_3d(&map, S1, dims, strides, box)) return false;
    const int slot_bytes = (int)(((size_t)nb * w * 2 * NL * sizeof(float2) + 127) / 128 * 128);
    const size_t sm = 2 * (size_t)slot_bytes + (size_t)L * (NL + 1) * sizeof(float2) + 16;
    if (sm > 200 * 1024) return false;
    auto k = p5_x_tma<L, NL>;
    set_smem(k, sm);
    const int threads = NL * Fft<float, L, +1, false>::TPL;
    const int ntiles = (int)((rows + 2 * NL - 1) / (2 * NL));
    const int grid = persistent_grid(k, threads, sm, ntiles);
    k<<<grid, threads, sm, st>>>(d, map, h, w, nb, slot_bytes);
    return true;
}

template <typename T, int L> static void launch_p3(const DemagDims& d, typename Cplx<T>::type* S2, const T* tens,
                                                   cudaStream_t st) {
    constexpr int B = b_p3<T, L>(), G = g_p3<T, L>();
    using C = typename Cplx<T>::type;
    const int kyi = 2 * (d.LY / 2 + 1);
    dim3 grid((d.KX + B - 1) / B, (kyi + G - 1) / G, d.nb);
    // the register-resident variant holds 3 NR values per thread: up to 20
    if constexpr (sizeof(T) == 4 && L <= 256 && Fft<T, L, -1, (L > 1)>::NR <= 20) {
        if constexpr (z_two_r1<L>() > 0) {
            if (kZTwo && d.nb == 1 && launch_p3_two<L>(d, S2, tens, st)) return;
        }
        if constexpr (tma_len<L>()) {
            if (d.nb == 1 && launch_p3_tma<L>(d, S2, tens, st)) return;
        }
        // 128-thread CTAs: three fit per SM at up to 170 registers per thread
        constexpr int G3 = (B * tpl_of<T, L>() >= 128) ? 1 : 128 / (B * tpl_of<T, L>());
        dim3 grid3((d.KX + B - 1) / B, (kyi + G3 - 1) / G3, d.nb);
        const size_t sm = (size_t)L * B * G3 * sizeof(C);
        auto k = p3_z_conv_reg<T, L, B, G3>;
        set_smem(k, sm);
        k<<<grid3, B * G3 * tpl_of<T, L>(), sm, st>>>(d, S2, tens);
    } else {
        const size_t sm = 3 * (size_t)L * B * G * sizeof(C);
        auto k = p3_z_conv<T, L, B, G>;
        set_smem(k, sm);
        k<<<grid, B * G * tpl_of<T, L>(), sm, st>>>(d, S2, tens);
    }
}

template <typename T, int L, int DIR> static void launch_y(const DemagDims& d, const typename Cplx<T>::type* in,
                                                           typename Cplx<T>::type* out, cudaStream_t st) {
    if constexpr (sizeof(T) == 4 && L >= 16 && is_pow2(L)) {
        if (launch_py_tma<L, DIR>(d, in, out, st)) return;
    }
    launch_py<T, L, DIR>(d, in, out, st);
}

template <typename T, int L> static void launch_x_fwd(const DemagDims& d, const T* m, const T* Ms_cell, T Ms,
                                                      typename Cplx<T>::type* S1, cudaStream_t st) {
    if constexpr (sizeof(T) == 4 && L >= 16 && is_pow2(L)) {
        if (launch_p1_tma<L>(d, m, Ms_cell, Ms, S1, st)) return;
    }
    launch_p1<T, L>(d, m, Ms_cell, Ms, S1, st);
}

template <typename T, int L> static void launch_x_inv(const DemagDims& d, const typename Cplx<T>::type* S1, T* h,
                                                      cudaStream_t st) {
    if constexpr (sizeof(T) == 4 && L >= 16 && is_pow2(L)) {
        if (launch_p5_tma<L>(d, S1, h, st)) return;
    }
    launch_p5<T, L>(d, S1, h, st);
}

// fused K5 launcher (see k5_fused): false if the shape or material does not qualify
// k5_fused configuration: TMA slots, work-area row padding, resident CTAs per SM
constexpr int kK5Rows = 2, kK5Slots = 1, kK5Pad = 0, kK5MinBlocks = 8;
#ifndef MM_K5_MIXED_MINB
#define MM_K5_MIXED_MINB 4
#endif
#ifndef MM_K5_MIXED_ROWS
#define MM_K5_MIXED_ROWS 6
#endif
// rows of y per tile (the mixed lines above 448 points keep two: their
// 32-thread lines would not fit six rows without spills)
template <int L> constexpr int k5_rows() { return is_pow2(L) ? kK5Rows : (L <= 448 ? MM_K5_MIXED_ROWS : 2); }
template <int L> constexpr int k5_threads() { return (3 * k5_rows<L>() / 2) * K5Eng<L, +1, false>::type::TPL; }
// resident CTAs asked of the register allocator, capped so that a thread keeps
// at least 85 (radix-16) or 113 (mixed-radix) registers: the long lines' larger
// CTAs would spill otherwise (1024-point lines spilled at eight CTAs)
template <int L> constexpr int k5_minb() {
    return is_pow2(L) ? (768 / k5_threads<L>() < 1 ? 1 : (768 / k5_threads<L>() > kK5MinBlocks ? kK5MinBlocks : 768 / k5_threads<L>()))
                      : (576 / k5_threads<L>() < 1 ? 1
                         : (576 / k5_threads<L>() > MM_K5_MIXED_MINB ? MM_K5_MIXED_MINB : 576 / k5_threads<L>()));
}

template <int L> static bool launch_k5(const DemagDims& d, float2* S1, const StageParams<float>& p, cudaStream_t st) {
    constexpr int TY = k5_rows<L>();
    if constexpr (L < 16 || !(is_pow2(L) || kTw5 % L == 0)) {
        return false;
    } else {
        if (!d.err || (d.KXS * 8) % 16 != 0 || (reinterpret_cast<uintptr_t>(S1) & 15) != 0) return false;
        const bool mat = p.Ms_cell || p.A_cell || p.Ku_cell || p.lay;
        if (p.alpha_cell || p.zw || p.D_cell || (!p.Ms_cell && p.Ms == 0.f) || p.hd || p.k_out || p.h_out ||
            p.want_err || p.want_energy || p.want_torque || !p.next || p.nk > 1 || (mat && p.dmi))
            return false;
        if (d.nx % 2 != 0) return false;
        int nb = 0;
        const int w = box_width(d.KX, &nb);
        CUtensorMap map;
        const cuuint64_t dims[4] = {(cuuint64_t)d.KX, (cuuint64_t)d.ny, (cuuint64_t)d.nz, 3};
        const cuuint64_t strides[3] = {(cuuint64_t)d.KXS * 8, (cuuint64_t)d.ny * d.KXS * 8,
                                       (cuuint64_t)d.nz * d.ny * d.KXS * 8};
        const cuuint32_t box[4] = {(cuuint32_t)w, (cuuint32_t)TY, 1, 3};
        if (!encode_4d(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, S1, dims, strides, box)) return false;
        constexpr int NL = 3 * TY / 2;
        const int slot_bytes = (int)(((size_t)nb * w * TY * 3 * sizeof(float2) + 127) / 128 * 128);
        const size_t sm = kK5Slots * (size_t)slot_bytes + (size_t)k5_work_elems<L, NL + kK5Pad>() * sizeof(float2) + 16;
        if (sm > 220 * 1024) return false;
        auto k = mat ? k5_fused<L, TY, kK5Slots, kK5Pad, k5_minb<L>(), false, true>
                 : p.dmi ? k5_fused<L, TY, kK5Slots, kK5Pad, k5_minb<L>(), true, false>
                         : k5_fused<L, TY, kK5Slots, kK5Pad, k5_minb<L>(), false, false>;
        set_smem(k, sm);
        const int threads = NL * K5Eng<L, +1, false>::type::TPL;
        if (threads > 1024) return false;
        const int ntiles = ((d.ny + TY - 1) / TY) * d.nz;
        const int grid = persistent_grid(k, threads, sm, ntiles);
        launch_pdl(k, grid, threads, sm, st, d, map, S1, p, w, nb, slot_bytes);
        return true;
    }
}

#define MM_DISPATCH_L(Lv, CALL)             \
    switch (Lv) {                           \
        case 1: { constexpr int L_ = 1; CALL; } break;       \
        case 2: { constexpr int L_ = 2; CALL; } break;       \
        case 4: { constexpr int L_ = 4; CALL; } break;       \
        case 8: { constexpr int L_ = 8; CALL; } break;       \
        case 16: { constexpr int L_ = 16; CALL; } break;     \
        case 32: { constexpr int L_ = 32; CALL; } break;     \
        case 64: { constexpr int L_ = 64; CALL; } break;     \
        case 128: { constexpr int L_ = 128; CALL; } break;   \
        case 256: { constexpr int L_ = 256; CALL; } break;   \
        case 512: { constexpr int L_ = 512; CALL; } break;   \
        case 1024: { constexpr int L_ = 1024; CALL; } break; \
        case 2048: { constexpr int L_ = 2048; CALL; } break; \
        case 4096: { constexpr int L_ = 4096; CALL; } break; \
        case 96: { constexpr int L_ = 96; CALL; } break;     \
        case 100: { constexpr int L_ = 100; CALL; } break;   \
        case 112: { constexpr int L_ = 112; CALL; } break;   \
        case 192: { constexpr int L_ = 192; CALL; } break;   \
        case 200: { constexpr int L_ = 200; CALL; } break;   \
        case 224: { constexpr int L_ = 224; CALL; } break;   \
        case 384: { constexpr int L_ = 384; CALL; } break;   \
        case 400: { constexpr int L_ = 400; CALL; } break;   \
        case 448: { constexpr int L_ = 448; CALL; } break;   \
        case 768: { constexpr int L_ = 768; CALL; } break;   \
        case 800: { constexpr int L_ = 800; CALL; } break;   \
        case 896: { constexpr int L_ = 896; CALL; } break;   \
        default: break;                     \
    }

// the compiled passes for the lengths MM_DISPATCH_L lists, the runtime-plan
// passes (demag_rt.cu) for every other 7-smooth length
#define MM_DISPATCH_RT(Lv, CALL, RTCALL) \
    if (fft_rt_length(Lv)) {             \
        RTCALL;                          \
    } else {                             \
        MM_DISPATCH_L(Lv, CALL);         \
    }

// P2 .. P4: S1 -> S1 through the tensor multiply.  A 2-D grid (nz = 1, Py <= 256)
// runs the z-pass kernel along y in place on S1 instead (one pass, no S2).
template <typename T>
static bool launch_p3_layers_tma(const DemagDims& d, typename Cplx<T>::type* S2, const T* tens, cudaStream_t st) {
    using C = typename Cplx<T>::type;
    const int npair = d.nz * (d.nz + 1) / 2;
    if (!d.err || d.nb != 1 || npair > 256 || 3 * d.nz > 256 || (d.KXS * sizeof(T)) % 16 != 0 ||
        (reinterpret_cast<uintptr_t>(tens) & 15) != 0 || (reinterpret_cast<uintptr_t>(S2) & 15) != 0)
        return false;
    const size_t sm = (size_t)6 * npair * kLayCols * sizeof(T) + (size_t)4 * 3 * d.nz * kLayCols * sizeof(C) + 16;
    if (sm > 200 * 1024) return false;
    const int KY2 = d.LY / 2 + 1;
    CUtensorMap tmap, smap;
    const cuuint64_t tdims[4] = {(cuuint64_t)d.KX, (cuuint64_t)KY2, (cuuint64_t)npair, 6};
    const cuuint64_t tstrides[3] = {(cuuint64_t)d.KXS * sizeof(T), (cuuint64_t)KY2 * d.KXS * sizeof(T),
                                    (cuuint64_t)npair * KY2 * d.KXS * sizeof(T)};
    const cuuint32_t tbox[4] = {(cuuint32_t)kLayCols, 1, (cuuint32_t)npair, 6};
    const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    if (!encode_4d(&tmap, dt, tens, tdims, tstrides, tbox)) return false;
    // the spectrum as 8-byte elements: (KX complex columns, Py rows, 3 nz planes)
    constexpr int W8 = (int)(sizeof(C) / 8);
    const cuuint64_t sdims[3] = {(cuuint64_t)d.KX * W8, (cuuint64_t)d.LY, (cuuint64_t)(3 * d.nz)};
    const cuuint64_t sstrides[2] = {(cuuint64_t)d.KXS * sizeof(C), (cuuint64_t)d.LY * d.KXS * sizeof(C)};
    const cuuint32_t sbox[3] = {(cuuint32_t)(kLayCols * W8), 1, (cuuint32_t)(3 * d.nz)};
    if (!encode_3d(&smap, S2, sdims, sstrides, sbox)) return false;
    auto k = p3_layers_tma<T>;
    set_smem(k, sm);
    dim3 grid((d.KX + kLayCols - 1) / kLayCols, KY2, 1);
    k<<<grid, dim3(kLayCols, kLayRows), sm, st>>>(d, tmap, smap, S2);
    return true;
}

template <typename T>
static void launch_p3_layers(const DemagDims& d, typename Cplx<T>::type* S2, const T* tens, cudaStream_t st) {
    using C = typename Cplx<T>::type;
    if (launch_p3_layers_tma<T>(d, S2, tens, st)) return;
    const size_t sm = (size_t)2 * 3 * d.nz * kLayCols * sizeof(C);
    auto k = p3_layers<T>;
    set_smem(k, sm);
    dim3 grid((d.KX + kLayCols - 1) / kLayCols, 2 * (d.LY / 2 + 1), d.nb);
    k<<<grid, dim3(kLayCols, kLayRows), sm, st>>>(d, S2, tens);
}

// largest padded y extent of a 2-D grid (nz = 1) whose y transforms and tensor
// multiply run as one pass of the z-pass kernel along y (above it the
// shared-memory kernel along y measured slower than the y passes: 32 served
// 256x256x1 grids, 2.36 ms against 2.07 ms per Dormand-Prince attempt)
constexpr int k2dMaxPy = 256;

template <typename T>
static void yzy(const DemagDims& d, typename Cplx<T>::type* S1, typename Cplx<T>::type* S2, const T* tens,
                cudaStream_t st, KernelTimer* tm) {
    using C = typename Cplx<T>::type;
    if (d.layers) {
        C* S2l = d.LY == 1 ? S1 : S2;
        if (d.LY > 1) {
            tm->begin(st, "p2_y_forward");
            MM_DISPATCH_RT(d.LY, (launch_y<T, L_, -1>(d, S1, S2, st)), (launch_rt_y<T, -1>(d, S1, S2, st)));
            tm->end(st);
        }
        tm->begin(st, "p3_layers");
        launch_p3_layers<T>(d, S2l, tens, st);
        tm->end(st);
        if (d.LY > 1) {
            tm->begin(st, "p4_y_inverse");
            MM_DISPATCH_RT(d.LY, (launch_y<T, L_, +1>(d, S2, S1, st)), (launch_rt_y<T, +1>(d, S2, S1, st)));
            tm->end(st);
        }
        return;
    }
    if (d.nz == 1 && d.LY > 1 && d.LY <= k2dMaxPy) {
        DemagDims d2 = d;
        d2.ny = 1; d2.nz = d.ny; d2.LY = 1; d2.LZ = d.LY; d2.yz_swap = 1;
        tm->begin(st, "p3_z_conv");
        MM_DISPATCH_RT(d2.LZ, (launch_p3<T, L_>(d2, S1, tens, st)), (launch_rt_z<T>(d2, S1, tens, st)));
        tm->end(st);
        return;
    }
    C* S2e = d.LY == 1 ? S1 : S2;
    if (d.LY > 1) {
        tm->begin(st, "p2_y_forward");
        MM_DISPATCH_RT(d.LY, (launch_y<T, L_, -1>(d, S1, S2, st)), (launch_rt_y<T, -1>(d, S1, S2, st)));
        tm->end(st);
    }
    tm->begin(st, "p3_z_conv");
    MM_DISPATCH_RT(d.LZ, (launch_p3<T, L_>(d, S2e, tens, st)), (launch_rt_z<T>(d, S2e, tens, st)));
    tm->end(st);
    if (d.LY > 1) {
        tm->begin(st, "p4_y_inverse");
        MM_DISPATCH_RT(d.LY, (launch_y<T, L_, +1>(d, S2, S1, st)), (launch_rt_y<T, +1>(d, S2, S1, st)));
        tm->end(st);
    }
}

template <typename T>
void demag_apply(const DemagDims& d, const T* m, const T* Ms_cell, T Ms, typename Cplx<T>::type* S1,
                 typename Cplx<T>::type* S2, const T* tens, T* h, cudaStream_t st, KernelTimer* tm) {
    // With ny == 1 the y passes are the identity and S2 aliases S1.
    tm->begin(st, "p1_x_forward");
    MM_DISPATCH_RT(d.LX, (launch_x_fwd<T, L_>(d, m, Ms_cell, Ms, S1, st)), (launch_rt_x_fwd<T>(d, m, Ms_cell, Ms, S1, st)));
    tm->end(st);
    yzy<T>(d, S1, S2, tens, st, tm);
    tm->begin(st, "p5_x_inverse");
    MM_DISPATCH_RT(d.LX, (launch_x_inv<T, L_>(d, S1, h, st)), (launch_rt_x_inv<T>(d, S1, h, st)));
    tm->end(st);
}

template <typename T>
void demag_front(const DemagDims& d, const T* m, const T* Ms_cell, T Ms, bool need_p1, typename Cplx<T>::type* S1,
                 typename Cplx<T>::type* S2, const T* tens, cudaStream_t st, KernelTimer* tm) {
    if (need_p1) {
        tm->begin(st, "p1_x_forward");
        MM_DISPATCH_RT(d.LX, (launch_x_fwd<T, L_>(d, m, Ms_cell, Ms, S1, st)), (launch_rt_x_fwd<T>(d, m, Ms_cell, Ms, S1, st)));
        tm->end(st);
    }
    yzy<T>(d, S1, S2, tens, st, tm);
}

bool fused_stage(const DemagDims& d, float2* S1, const StageParams<float>& p, cudaStream_t st, KernelTimer* tm) {
    bool ok = false;
    tm->begin(st, "k5_fused");
    MM_DISPATCH_L(d.LX, (ok = launch_k5<L_>(d, S1, p, st)));
    tm->end(st);
    return ok;
}

bool fused_stage_supported(const DemagDims& d, const StageParams<float>& p) {
    if (!d.err || d.LX < 16 || d.LX > 4096 || d.nx % 2 != 0) return false;
    if (fft_rt_length(d.LX)) return false;        // compiled engines only (powers of two, r 2^a)
    if (p.alpha_cell || p.zw || p.D_cell || (!p.Ms_cell && p.Ms == 0.f)) return false;
    if ((p.Ms_cell || p.A_cell || p.Ku_cell || p.lay) && p.dmi) return false;
    const int threads = (3 * kK5Rows / 2) * (d.LX / 16);
    return threads <= 1024;
}

template void demag_front<float>(const DemagDims&, const float*, const float*, float, bool, float2*, float2*,
                                 const float*, cudaStream_t, KernelTimer*);
template void demag_front<double>(const DemagDims&, const double*, const double*, double, bool, double2*, double2*,
                                  const double*, cudaStream_t, KernelTimer*);

template void demag_apply<float>(const DemagDims&, const float*, const float*, float, float2*, float2*,
                                 const float*, float*, cudaStream_t, KernelTimer*);
template void demag_apply<double>(const DemagDims&, const double*, const double*, double, double2*, double2*,
                                  const double*, double*, cudaStream_t, KernelTimer*);

}  // namespace mm
