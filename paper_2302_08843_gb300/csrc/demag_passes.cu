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
#include <cstdio>

#include "demag.h"
#include "fft_engine.cuh"

namespace mm {

cudaError_t upload_twiddles(const double2* w64, const float2* w32) {
    cudaError_t e = cudaMemcpyToSymbol(g_tw64, w64, sizeof(double2) * kMaxFft);
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(g_tw32, w32, sizeof(float2) * kMaxFft);
}

// ------------------------------------------------------------------ P1 ----
template <typename T, int LX, int NL>
__global__ void __launch_bounds__(NL * FftLine<T, LX, -1, (LX > 1)>::TPL)
p1_x_forward(DemagDims d, const T* __restrict__ m, const T* __restrict__ Ms_cell, T Ms_const,
             typename Cplx<T>::type* __restrict__ S1) {
    using C = typename Cplx<T>::type;
    using F = FftLine<T, LX, -1, (LX > 1)>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* s = reinterpret_cast<C*>(smraw);
    constexpr int LS = NL + 1;
    constexpr int NT = NL * F::TPL;
    constexpr int XH = LX > 1 ? LX / 2 : 1;     // staged input positions
    const int tid = threadIdx.x;
    const int line = tid % NL, j = tid / NL;
    const long plane = (long)d.ny * d.nz;
    const long rows = 3 * plane;
    const long row0 = (long)blockIdx.x * (2 * NL);

    for (int idx = tid; idx < NL * XH; idx += NT) {
        const int l = idx / XH, x = idx - l * XH;
        const long ra = row0 + 2 * l, rb = ra + 1;
        T a = 0, b = 0;
        if (x < d.nx) {
            if (ra < rows) {
                const T ms = Ms_cell ? Ms_cell[(ra % plane) * d.nx + x] : Ms_const;
                a = m[ra * d.nx + x] * ms;
            }
            if (rb < rows) {
                const T ms = Ms_cell ? Ms_cell[(rb % plane) * d.nx + x] : Ms_const;
                b = m[rb * d.nx + x] * ms;
            }
        }
        s[x * LS + l] = mk<C>(a, b);
    }
    __syncthreads();
    C v[F::NR];
#pragma unroll
    for (int r = 0; r < F::NR; ++r) {
        if (LX == 1 || r < F::NR / 2) v[r] = s[(j + r * F::TPL) * LS + line];
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
        const long ra = row0 + 2 * l, rb = ra + 1;
        const C zk = s[k * LS + l];
        const C zm = s[((LX - k) & (LX - 1)) * LS + l];
        if (ra < rows) S1[ra * d.KXS + k] = mk<C>(half * (zk.x + zm.x), half * (zk.y - zm.y));
        if (rb < rows) S1[rb * d.KXS + k] = mk<C>(half * (zk.y + zm.y), half * (zm.x - zk.x));
    }
}

// ------------------------------------------------------------- P2 / P4 ----
// DIR = -1: S1 (ny rows) -> S2 (Py rows), forward, zero upper half.
// DIR = +1: S2 (Py rows) -> S1 (ny rows), inverse, keep the lower half.
template <typename T, int LY, int B, int G, int DIR>
__global__ void __launch_bounds__(B * G * FftLine<T, LY, DIR, (DIR < 0 && LY > 1)>::TPL)
p_y_pass(DemagDims d, const typename Cplx<T>::type* __restrict__ in,
         typename Cplx<T>::type* __restrict__ out) {
    using C = typename Cplx<T>::type;
    constexpr bool ZIN = DIR < 0 && LY > 1;
    using F = FftLine<T, LY, DIR, ZIN>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* s = reinterpret_cast<C*>(smraw);
    constexpr int NL = B * G;
    const int tid = threadIdx.x;
    const int line = tid % NL, j = tid / NL;
    const int kl = line % B, g = line / B;
    const int kx = blockIdx.x * B + kl;
    const int cz = blockIdx.y * G + g;
    const bool valid = kx < d.KX && cz < 3 * d.nz;
    const int rows_in = DIR < 0 ? d.ny : LY;
    const int rows_out = DIR < 0 ? LY : d.ny;
    const C* src = in + ((long)cz * rows_in) * d.KXS + kx;
    C* dst = out + ((long)cz * rows_out) * d.KXS + kx;
    C v[F::NR];
#pragma unroll
    for (int r = 0; r < F::NR; ++r) {
        const int e = j + r * F::TPL;
        v[r] = mk<C>(0, 0);
        if (valid && (!ZIN || r < F::NR / 2) && e < rows_in) v[r] = src[(long)e * d.KXS];
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

// ------------------------------------------------------------------ P3 ----
// resident CTAs asked of the register allocator: 1024 (FP32) or 512 (FP64) threads per SM
template <typename T> constexpr int p3_min_blocks(int threads) {
    return (sizeof(T) == 4 ? 1024 : 512) / threads > 1 ? (sizeof(T) == 4 ? 1024 : 512) / threads : 1;
}

// Three shared-memory areas, one per component, each the FFT scratch of its
// component: every global load of the column tile is issued first and parked
// in its area, then each component is transformed in place, the 3x3 multiply
// reads and rewrites the areas, and each inverse transform streams its kept
// half straight to global memory.  Only one component's registers are live at
// a time, which keeps the kernel at four CTAs per SM.
template <typename T, int LZ, int B, int G>
__global__ void __launch_bounds__(B * G * FftLine<T, LZ, -1, (LZ > 1)>::TPL,
                                  p3_min_blocks<T>(B * G * FftLine<T, LZ, -1, (LZ > 1)>::TPL))
p3_z_conv(DemagDims d, typename Cplx<T>::type* __restrict__ S2, const T* __restrict__ tens) {
    using C = typename Cplx<T>::type;
    using FF = FftLine<T, LZ, -1, (LZ > 1)>;
    using FI = FftLine<T, LZ, +1, false>;
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
    C* col = S2 + (long)ky * d.KXS + kx;            // element (c, z) at col[c*cstride + z*LY*KXS]
    const long zs = (long)LY * d.KXS;

    {   // all loads in flight together, parked at this thread's own positions
        C in[3][NIN];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < NIN; ++r) {
                const int z = j + r * TPL;
                in[c][r] = (valid && z < d.nz) ? col[c * cstride + z * zs] : mk<C>(0, 0);
            }
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < NIN; ++r) area[c][(j + r * TPL) * NL + line] = in[c][r];
    }
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        C v[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) v[r] = r < NIN ? area[c][(j + r * TPL) * NL + line] : mk<C>(0, 0);
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
            txy = sy * __ldg(tp + tcomp);
            txz = sz * __ldg(tp + 2 * tcomp);
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

// ------------------------------------------------------------------ P5 ----
template <typename T, int LX, int NL>
__global__ void __launch_bounds__(NL * FftLine<T, LX, +1, false>::TPL)
p5_x_inverse(DemagDims d, const typename Cplx<T>::type* __restrict__ S1, T* __restrict__ h) {
    using C = typename Cplx<T>::type;
    using F = FftLine<T, LX, +1, false>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* s = reinterpret_cast<C*>(smraw);
    constexpr int LS = NL + 1;
    constexpr int NT = NL * F::TPL;
    constexpr int KXn = LX / 2 + 1;
    const int tid = threadIdx.x;
    const int line = tid % NL, j = tid / NL;
    const long rows = 3L * d.ny * d.nz;
    const long row0 = (long)blockIdx.x * (2 * NL);
    for (int idx = tid; idx < NL * KXn; idx += NT) {
        const int l = idx / KXn, k = idx - l * KXn;
        const long ra = row0 + 2 * l, rb = ra + 1;
        C A = mk<C>(0, 0), Bv = mk<C>(0, 0);
        if (ra < rows) A = S1[ra * d.KXS + k];
        if (rb < rows) Bv = S1[rb * d.KXS + k];
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
        const long ra = row0 + 2 * l, rb = ra + 1;
        const C z = s[x * LS + l];
        if (ra < rows) h[ra * d.nx + x] = z.x;
        if (rb < rows) h[rb * d.nx + x] = z.y;
    }
}

// ------------------------------------------------------------ launchers ----
template <typename T> struct Geo;
template <> struct Geo<float> { static constexpr int BS = 16; };   // 16 x 8 B = 128 B rows
template <> struct Geo<double> { static constexpr int BS = 8; };   // 8 x 16 B = 128 B rows

template <int L> constexpr int tpl_of() { return L >= 8 ? L / 8 : 1; }
// lines per CTA for the x passes: about 256 threads
template <int L> constexpr int nl_x() { return tpl_of<L>() >= 256 ? 1 : 256 / tpl_of<L>(); }
// kx columns per CTA for strided passes: 128-byte rows, at most 512 threads per group
template <typename T, int L> constexpr int b_of() {
    return (Geo<T>::BS * tpl_of<L>() <= 512) ? Geo<T>::BS : ((512 / tpl_of<L>()) < 2 ? 2 : 512 / tpl_of<L>());
}
template <typename T, int L> constexpr int g_of() {
    return (b_of<T, L>() * tpl_of<L>() >= 256) ? 1 : 256 / (b_of<T, L>() * tpl_of<L>());
}

template <typename K> static void set_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int L> static void launch_p1(const DemagDims& d, const T* m, const T* Ms_cell, T Ms,
                                                   typename Cplx<T>::type* S1, cudaStream_t st) {
    constexpr int NL = nl_x<L>();
    using C = typename Cplx<T>::type;
    const size_t sm = (size_t)L * (NL + 1) * sizeof(C);
    const long rows = 3L * d.ny * d.nz;
    const unsigned grid = (unsigned)((rows + 2 * NL - 1) / (2 * NL));
    auto k = p1_x_forward<T, L, NL>;
    set_smem(k, sm);
    k<<<grid, NL * tpl_of<L>(), sm, st>>>(d, m, Ms_cell, Ms, S1);
}

template <typename T, int L> static void launch_p5(const DemagDims& d, const typename Cplx<T>::type* S1, T* h,
                                                   cudaStream_t st) {
    constexpr int NL = nl_x<L>();
    using C = typename Cplx<T>::type;
    const size_t sm = (size_t)L * (NL + 1) * sizeof(C);
    const long rows = 3L * d.ny * d.nz;
    const unsigned grid = (unsigned)((rows + 2 * NL - 1) / (2 * NL));
    auto k = p5_x_inverse<T, L, NL>;
    set_smem(k, sm);
    k<<<grid, NL * tpl_of<L>(), sm, st>>>(d, S1, h);
}

template <typename T, int L, int DIR> static void launch_py(const DemagDims& d, const typename Cplx<T>::type* in,
                                                            typename Cplx<T>::type* out, cudaStream_t st) {
    constexpr int B = b_of<T, L>(), G = g_of<T, L>();
    using C = typename Cplx<T>::type;
    const size_t sm = (size_t)L * B * G * sizeof(C);
    dim3 grid((d.KX + B - 1) / B, (3 * d.nz + G - 1) / G);
    auto k = p_y_pass<T, L, B, G, DIR>;
    set_smem(k, sm);
    k<<<grid, B * G * tpl_of<L>(), sm, st>>>(d, in, out);
}

template <typename T, int L> static void launch_p3(const DemagDims& d, typename Cplx<T>::type* S2, const T* tens,
                                                   cudaStream_t st) {
    constexpr int B = b_of<T, L>(), G = g_of<T, L>();
    using C = typename Cplx<T>::type;
    const size_t sm = 3 * (size_t)L * B * G * sizeof(C);
    const int kyi = 2 * (d.LY / 2 + 1);
    dim3 grid((d.KX + B - 1) / B, (kyi + G - 1) / G);
    auto k = p3_z_conv<T, L, B, G>;
    set_smem(k, sm);
    k<<<grid, B * G * tpl_of<L>(), sm, st>>>(d, S2, tens);
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
        default: break;                     \
    }

template <typename T>
void demag_apply(const DemagDims& d, const T* m, const T* Ms_cell, T Ms, typename Cplx<T>::type* S1,
                 typename Cplx<T>::type* S2, const T* tens, T* h, cudaStream_t st, KernelTimer* tm) {
    using C = typename Cplx<T>::type;
    // With ny == 1 the y passes are the identity and S2 aliases S1.
    C* S2e = d.LY == 1 ? S1 : S2;
    tm->begin(st, "p1_x_forward");
    MM_DISPATCH_L(d.LX, (launch_p1<T, L_>(d, m, Ms_cell, Ms, S1, st)));
    tm->end(st);
    if (d.LY > 1) {
        tm->begin(st, "p2_y_forward");
        MM_DISPATCH_L(d.LY, (launch_py<T, L_, -1>(d, S1, S2, st)));
        tm->end(st);
    }
    tm->begin(st, "p3_z_conv");
    MM_DISPATCH_L(d.LZ, (launch_p3<T, L_>(d, S2e, tens, st)));
    tm->end(st);
    if (d.LY > 1) {
        tm->begin(st, "p4_y_inverse");
        MM_DISPATCH_L(d.LY, (launch_py<T, L_, +1>(d, S2, S1, st)));
        tm->end(st);
    }
    tm->begin(st, "p5_x_inverse");
    MM_DISPATCH_L(d.LX, (launch_p5<T, L_>(d, S1, h, st)));
    tm->end(st);
}

template void demag_apply<float>(const DemagDims&, const float*, const float*, float, float2*, float2*,
                                 const float*, float*, cudaStream_t, KernelTimer*);
template void demag_apply<double>(const DemagDims&, const double*, const double*, double, double2*, double2*,
                                  const double*, double*, cudaStream_t, KernelTimer*);

}  // namespace mm
