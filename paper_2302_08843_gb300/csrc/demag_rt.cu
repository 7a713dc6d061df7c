// Demag FFT passes for every 7-smooth padded length 2^a 3^b 5^c 7^d (even,
// <= 4096) that has no compiled engine: the same five passes as
// demag_passes.cu (x-forward r2c, y-forward, z-forward + 3x3 tensor multiply
// + z-inverse, y-inverse, x-inverse c2r; Sec. 4.4), with the line length and
// its radix plan known only at run time.
//
// Engine: a self-sorting Stockham FFT over a batch of lines held in shared
// memory (element e of line l at s[e NLc + l]), all threads of the CTA
// sharing the butterflies of every pass: a pass of radix R and span Ns reads
// butterfly b's inputs at b + q L/R, multiplies input q by W_{Ns R}^(q k)
// (k = b mod Ns), transforms them and writes output q to
// (b - k) R + k + q Ns, ping-ponging between two buffers.  Plan: every radix 7,
// then 5, then 3, then radix-4 passes and at most one radix-2 pass.
// Twiddles W_L^m (m < L) come from one double-precision table per length,
// all lengths concatenated (g_twrt64 / g_twrt32), built on the host with the
// octant-exact evaluation of the other tables and uploaded once per device.
#include <cmath>
#include <mutex>
#include <vector>

#include "demag.h"
#include "tensor_host.h"

namespace mm {

namespace {

constexpr int kRtMaxPass = 16;
constexpr int kRtThreads = 256;
constexpr int kRtMaxLines = 16;

struct RtPlan {
    int L;
    int np;
    int R[kRtMaxPass];
    int tw;          // offset of this length's table W_L^m in g_twrt
};

// the lengths this file serves, their twiddle offsets and the table size
struct RtTable {
    std::vector<int> lengths;
    std::vector<int> offsets;
    int total = 0;
};

const RtTable& rt_table() {
    static RtTable t;
    static std::once_flag once;
    std::call_once(once, [] {
        for (int L = 2; L <= kMaxRtFft; L += 2)
            if (fft_rt_length(L)) {
                t.lengths.push_back(L);
                t.offsets.push_back(t.total);
                t.total += L;
            }
    });
    return t;
}

}  // namespace

// total entries of the concatenated runtime twiddle tables (a compile-time
// bound for the device arrays; checked against the host table at upload)
constexpr int kTwRt = 161076;
static __device__ double2 g_twrt64[kTwRt];
static __device__ float2 g_twrt32[kTwRt];

template <typename T> struct TwRt;
template <> struct TwRt<float> {
    static __device__ __forceinline__ float2 get(int m) { return __ldg(&g_twrt32[m]); }
};
template <> struct TwRt<double> {
    static __device__ __forceinline__ double2 get(int m) { return __ldg(&g_twrt64[m]); }
};

bool fft_rt_length(int L) {
    if (L < 2 || L > kMaxRtFft || (L & 1)) return false;
    if (is_pow2(L)) return false;
    static const int compiled[12] = {96, 100, 112, 192, 200, 224, 384, 400, 448, 768, 800, 896};
    for (int c : compiled)
        if (c == L) return false;
    int v = L;
    for (int p : {2, 3, 5, 7})
        while (v % p == 0) v /= p;
    return v == 1;
}

static RtPlan make_plan(int L) {
    RtPlan pl{};
    pl.L = L;
    int v = L;
    for (int r : {7, 5, 3})
        while (v % r == 0) {
            pl.R[pl.np++] = r;
            v /= r;
        }
    while (v % 4 == 0) {
        pl.R[pl.np++] = 4;
        v /= 4;
    }
    if (v == 2) pl.R[pl.np++] = 2;
    const RtTable& t = rt_table();
    pl.tw = -1;
    for (size_t i = 0; i < t.lengths.size(); ++i)
        if (t.lengths[i] == L) pl.tw = t.offsets[i];
    return pl;
}

cudaError_t upload_twiddles_rt() {
    const RtTable& t = rt_table();
    if (t.total != kTwRt) return cudaErrorInvalidValue;
    static std::vector<double2> h64;
    static std::vector<float2> h32;
    if (h64.empty()) {
        h64.resize(kTwRt);
        h32.resize(kTwRt);
        for (size_t i = 0; i < t.lengths.size(); ++i) {
            const int L = t.lengths[i];
            for (int m = 0; m < L; ++m) {
                double c, sn;
                twiddle_entry(L, m, &c, &sn);
                h64[t.offsets[i] + m] = make_double2(c, sn);
                h32[t.offsets[i] + m] = make_float2((float)c, (float)sn);
            }
        }
    }
    cudaError_t e = cudaMemcpyToSymbol(g_twrt64, h64.data(), sizeof(double2) * kTwRt);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_twrt32, h32.data(), sizeof(float2) * kTwRt);
    return e;
}

// One radix-R Stockham pass of span Ns over NLc lines of length L.
template <typename T, int DIR, int R>
__device__ __forceinline__ void rt_pass(const typename Cplx<T>::type* __restrict__ src,
                                        typename Cplx<T>::type* __restrict__ dst, int NLc, int L, int Ns, int tw) {
    using C = typename Cplx<T>::type;
    const int M = L / R, step = L / (Ns * R);
    for (int idx = threadIdx.x; idx < M * NLc; idx += blockDim.x) {
        const int l = idx % NLc, b = idx / NLc;
        const int k = b % Ns;
        C x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            C v = src[(b + q * M) * NLc + l];
            if (q > 0 && k > 0) {
                C w = TwRt<T>::get(tw + q * k * step);
                if (DIR > 0) w.y = -w.y;
                v = cmul(v, w);
            }
            x[q] = v;
        }
        if constexpr (R == 2) dft2<DIR>(x[0], x[1]);
        else if constexpr (R == 3) dft3<DIR>(x[0], x[1], x[2]);
        else if constexpr (R == 4) dft4<DIR>(x[0], x[1], x[2], x[3]);
        else if constexpr (R == 5) dft5<DIR>(x[0], x[1], x[2], x[3], x[4]);
        else dft7<DIR>(x);
        const int base = (b - k) * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) dst[(base + q * Ns) * NLc + l] = x[q];
    }
}

// One Stockham transform of NLc lines of length pl.L in shared memory (src,
// with dst as the other buffer of the ping-pong); returns the buffer holding
// the result.  Every thread of the CTA must call it.  DIR = -1 forward,
// +1 inverse (unnormalised).
template <typename T, int DIR>
__device__ typename Cplx<T>::type* rt_fft(typename Cplx<T>::type* src, typename Cplx<T>::type* dst, int NLc,
                                         const RtPlan& pl) {
    using C = typename Cplx<T>::type;
    int Ns = 1;
    for (int p = 0; p < pl.np; ++p) {
        const int R = pl.R[p];
        switch (R) {
            case 2: rt_pass<T, DIR, 2>(src, dst, NLc, pl.L, Ns, pl.tw); break;
            case 3: rt_pass<T, DIR, 3>(src, dst, NLc, pl.L, Ns, pl.tw); break;
            case 4: rt_pass<T, DIR, 4>(src, dst, NLc, pl.L, Ns, pl.tw); break;
            case 5: rt_pass<T, DIR, 5>(src, dst, NLc, pl.L, Ns, pl.tw); break;
            default: rt_pass<T, DIR, 7>(src, dst, NLc, pl.L, Ns, pl.tw); break;
        }
        __syncthreads();
        C* t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}

// ------------------------------------------------------------- x passes ----
// Two real rows per complex line, paired within one grid of a batch as in the
// compiled x passes (an odd row count leaves the last row with a zero partner).
__device__ __forceinline__ void rt_pair(const DemagDims& d, int NLc, long* ra_s, long* rb_s) {
    if (threadIdx.x < NLc) {
        const long R = 3L * d.ny * d.nz, ppg = (R + 1) / 2;
        const long q = (long)blockIdx.x * NLc + threadIdx.x;
        const long b = q / ppg, lp = q - b * ppg;
        const bool ok = b < d.nb;
        ra_s[threadIdx.x] = ok ? b * R + 2 * lp : -1;
        rb_s[threadIdx.x] = ok && 2 * lp + 1 < R ? b * R + 2 * lp + 1 : -1;
    }
}

template <typename T>
__global__ void __launch_bounds__(kRtThreads)
rt_x_forward(DemagDims d, const T* __restrict__ m, const T* __restrict__ Ms_cell, T Ms_const,
             typename Cplx<T>::type* __restrict__ S1, RtPlan pl, int NLc) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = pl.L;
    C* a = reinterpret_cast<C*>(smraw);
    C* b = a + (size_t)L * NLc;
    __shared__ long ra_s[kRtMaxLines], rb_s[kRtMaxLines];
    rt_pair(d, NLc, ra_s, rb_s);
    __syncthreads();
    const long plane = (long)d.ny * d.nz;
    const T* Ms_b = static_cast<const T*>(d.Ms_b);
    for (int idx = threadIdx.x; idx < L * NLc; idx += blockDim.x) {
        const int l = idx % NLc, x = idx / NLc;
        const long ra = ra_s[l], rb = rb_s[l];
        T va = 0, vb = 0;
        if (x < d.nx) {
            if (ra >= 0) {
                const T ms = Ms_b ? Ms_b[ra / (3 * plane)] : (Ms_cell ? Ms_cell[(ra % plane) * d.nx + x] : Ms_const);
                va = m[ra * d.nx + x] * ms;
            }
            if (rb >= 0) {
                const T ms = Ms_b ? Ms_b[rb / (3 * plane)] : (Ms_cell ? Ms_cell[(rb % plane) * d.nx + x] : Ms_const);
                vb = m[rb * d.nx + x] * ms;
            }
        }
        a[x * NLc + l] = mk<C>(va, vb);
    }
    __syncthreads();
    const C* z = rt_fft<T, -1>(a, b, NLc, pl);
    const int KX = L / 2 + 1;
    const T half = (T)0.5;
    for (int idx = threadIdx.x; idx < KX * NLc; idx += blockDim.x) {
        const int l = idx % NLc, k = idx / NLc;
        const long ra = ra_s[l], rb = rb_s[l];
        const C zk = z[k * NLc + l];
        const C zm = z[(k == 0 ? 0 : L - k) * NLc + l];
        if (ra >= 0) S1[ra * d.KXS + k] = mk<C>(half * (zk.x + zm.x), half * (zk.y - zm.y));
        if (rb >= 0) S1[rb * d.KXS + k] = mk<C>(half * (zk.y + zm.y), half * (zm.x - zk.x));
    }
}

template <typename T>
__global__ void __launch_bounds__(kRtThreads)
rt_x_inverse(DemagDims d, const typename Cplx<T>::type* __restrict__ S1, T* __restrict__ h, RtPlan pl, int NLc) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = pl.L;
    C* a = reinterpret_cast<C*>(smraw);
    C* b = a + (size_t)L * NLc;
    __shared__ long ra_s[kRtMaxLines], rb_s[kRtMaxLines];
    rt_pair(d, NLc, ra_s, rb_s);
    __syncthreads();
    const int KX = L / 2 + 1;
    for (int idx = threadIdx.x; idx < KX * NLc; idx += blockDim.x) {
        const int l = idx % NLc, k = idx / NLc;
        const long ra = ra_s[l], rb = rb_s[l];
        C A = mk<C>(0, 0), Bv = mk<C>(0, 0);
        if (ra >= 0) A = S1[ra * d.KXS + k];
        if (rb >= 0) Bv = S1[rb * d.KXS + k];
        if (k == 0 || 2 * k == L) { A.y = 0; Bv.y = 0; }   // a real row has real DC and Nyquist
        a[k * NLc + l] = mk<C>(A.x - Bv.y, A.y + Bv.x);
        if (k > 0 && 2 * k < L) a[(L - k) * NLc + l] = mk<C>(A.x + Bv.y, Bv.x - A.y);
    }
    __syncthreads();
    const C* z = rt_fft<T, +1>(a, b, NLc, pl);
    for (int idx = threadIdx.x; idx < d.nx * NLc; idx += blockDim.x) {
        const int l = idx % NLc, x = idx / NLc;
        const long ra = ra_s[l], rb = rb_s[l];
        const C v = z[x * NLc + l];
        if (ra >= 0) h[ra * d.nx + x] = v.x;
        if (rb >= 0) h[rb * d.nx + x] = v.y;
    }
}

// ------------------------------------------------------------- y passes ----
// DIR = -1: S1 (ny rows) -> S2 (Py rows), forward.  DIR = +1: S2 -> S1, keep y < ny.
// A CTA takes B kx columns of one (grid, component, z) plane.
template <typename T, int DIR>
__global__ void __launch_bounds__(kRtThreads)
rt_y_pass(DemagDims d, const typename Cplx<T>::type* __restrict__ in, typename Cplx<T>::type* __restrict__ out,
          RtPlan pl, int B) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = pl.L;
    C* a = reinterpret_cast<C*>(smraw);
    C* b = a + (size_t)L * B;
    const int kx0 = blockIdx.x * B;
    const long cz = blockIdx.y;
    const int rows_in = DIR < 0 ? d.ny : L;
    const int rows_out = DIR < 0 ? L : d.ny;
    const C* src = in + (cz * rows_in) * d.KXS;
    C* dst = out + (cz * rows_out) * d.KXS;
    for (int idx = threadIdx.x; idx < L * B; idx += blockDim.x) {
        const int l = idx % B, e = idx / B;
        const int kx = kx0 + l;
        a[e * B + l] = (e < rows_in && kx < d.KX) ? src[(long)e * d.KXS + kx] : mk<C>(0, 0);
    }
    __syncthreads();
    const C* z = rt_fft<T, DIR>(a, b, B, pl);
    for (int idx = threadIdx.x; idx < rows_out * B; idx += blockDim.x) {
        const int l = idx % B, e = idx / B;
        const int kx = kx0 + l;
        if (kx < d.KX) dst[(long)e * d.KXS + kx] = z[e * B + l];
    }
}

// -------------------------------------------------------------- z pass ----
// Per (kx, ky) column: z-forward of the three components, h^ = T M^ with the
// octant-folded real tensor (sign flips of the odd components from the
// parity of ky and kz, or of the transformed axis on 2-D grids), z-inverse,
// keep z < nz; in place in S2.  A CTA takes B kx columns of one ky; blockIdx.z
// is the grid of a batch.
template <typename T>
__global__ void __launch_bounds__(kRtThreads)
rt_z_conv(DemagDims d, typename Cplx<T>::type* __restrict__ S2, const T* __restrict__ tens, RtPlan pl, int B) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int LZ = pl.L;
    C* buf[4];
    buf[0] = reinterpret_cast<C*>(smraw);
    for (int q = 1; q < 4; ++q) buf[q] = buf[q - 1] + (size_t)LZ * B;
    const int LY = d.LY;
    const int KY2 = LY / 2 + 1;
    const int p = blockIdx.y >> 1, side = blockIdx.y & 1;
    if (!(p < KY2 && (side == 0 || (p > 0 && 2 * p < LY)))) return;      // uniform over the CTA
    const int ky = side ? LY - p : p;
    const int kx0 = blockIdx.x * B;
    const long cstride = (long)d.nz * LY * d.KXS;
    const long zs = (long)LY * d.KXS;
    C* col = S2 + (long)blockIdx.z * 3 * cstride + (long)ky * d.KXS + kx0;
    C* area[3] = {buf[0], buf[1], buf[2]};
    C* scratch = buf[3];
    for (int c = 0; c < 3; ++c)
        for (int idx = threadIdx.x; idx < LZ * B; idx += blockDim.x) {
            const int l = idx % B, z = idx / B;
            area[c][z * B + l] = (z < d.nz && kx0 + l < d.KX) ? col[c * cstride + z * zs + l] : mk<C>(0, 0);
        }
    __syncthreads();
    for (int c = 0; c < 3; ++c) {
        C* r = rt_fft<T, -1>(area[c], scratch, B, pl);
        if (r != area[c]) { scratch = area[c]; area[c] = r; }
    }
    const int KZ2 = LZ / 2 + 1;
    const long tcomp = (long)KZ2 * KY2 * d.KXS;
    const T sy = side ? (T)-1 : (T)1;
    for (int idx = threadIdx.x; idx < LZ * B; idx += blockDim.x) {
        const int l = idx % B, kz = idx / B;
        const int kx = kx0 + l;
        if (kx >= d.KX) continue;
        const int kzf = (2 * kz <= LZ) ? kz : LZ - kz;
        const T sz = (2 * kz <= LZ) ? (T)1 : (T)-1;
        const T* tp = tens + ((long)kzf * KY2 + p) * d.KXS + kx;
        const T txx = __ldg(tp);
        const T txy = (d.yz_swap ? sz : sy) * __ldg(tp + tcomp);
        const T txz = (d.yz_swap ? sy : sz) * __ldg(tp + 2 * tcomp);
        const T tyy = __ldg(tp + 3 * tcomp);
        const T tyz = sy * sz * __ldg(tp + 4 * tcomp);
        const T tzz = __ldg(tp + 5 * tcomp);
        const int o = kz * B + l;
        const C mx = area[0][o], my = area[1][o], mz = area[2][o];
        area[0][o] = mk<C>(txx * mx.x + txy * my.x + txz * mz.x, txx * mx.y + txy * my.y + txz * mz.y);
        area[1][o] = mk<C>(txy * mx.x + tyy * my.x + tyz * mz.x, txy * mx.y + tyy * my.y + tyz * mz.y);
        area[2][o] = mk<C>(txz * mx.x + tyz * my.x + tzz * mz.x, txz * mx.y + tyz * my.y + tzz * mz.y);
    }
    __syncthreads();
    for (int c = 0; c < 3; ++c) {
        C* r = rt_fft<T, +1>(area[c], scratch, B, pl);
        if (r != area[c]) { scratch = area[c]; area[c] = r; }
    }
    for (int c = 0; c < 3; ++c)
        for (int idx = threadIdx.x; idx < d.nz * B; idx += blockDim.x) {
            const int l = idx % B, z = idx / B;
            if (kx0 + l < d.KX) col[c * cstride + z * zs + l] = area[c][z * B + l];
        }
}

// ------------------------------------------------------------- launchers ----
namespace {
template <typename K> void rt_smem(K kernel, size_t bytes) {
    if (bytes > 40 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
constexpr size_t kRtSmem = 200 * 1024;
// lines (or columns) per CTA: up to `cap`, as many as two (or four) buffers of L complex values allow
int rt_lines(int L, size_t csz, int nbuf, int cap) {
    int n = cap;
    while (n > 1 && (size_t)nbuf * L * n * csz > kRtSmem) --n;
    return n;
}
}  // namespace

template <typename T>
void launch_rt_x_fwd(const DemagDims& d, const T* m, const T* Ms_cell, T Ms, typename Cplx<T>::type* S1,
                     cudaStream_t st) {
    using C = typename Cplx<T>::type;
    const RtPlan pl = make_plan(d.LX);
    const int NL = rt_lines(d.LX, sizeof(C), 2, kRtMaxLines);
    const size_t sm = 2 * (size_t)d.LX * NL * sizeof(C);
    const long pairs = (long)d.nb * ((3L * d.ny * d.nz + 1) / 2);
    auto k = rt_x_forward<T>;
    rt_smem(k, sm);
    k<<<(unsigned)((pairs + NL - 1) / NL), kRtThreads, sm, st>>>(d, m, Ms_cell, Ms, S1, pl, NL);
}

template <typename T>
void launch_rt_x_inv(const DemagDims& d, const typename Cplx<T>::type* S1, T* h, cudaStream_t st) {
    using C = typename Cplx<T>::type;
    const RtPlan pl = make_plan(d.LX);
    const int NL = rt_lines(d.LX, sizeof(C), 2, kRtMaxLines);
    const size_t sm = 2 * (size_t)d.LX * NL * sizeof(C);
    const long pairs = (long)d.nb * ((3L * d.ny * d.nz + 1) / 2);
    auto k = rt_x_inverse<T>;
    rt_smem(k, sm);
    k<<<(unsigned)((pairs + NL - 1) / NL), kRtThreads, sm, st>>>(d, S1, h, pl, NL);
}

template <typename T, int DIR>
void launch_rt_y(const DemagDims& d, const typename Cplx<T>::type* in, typename Cplx<T>::type* out,
                 cudaStream_t st) {
    using C = typename Cplx<T>::type;
    const RtPlan pl = make_plan(d.LY);
    const int B = rt_lines(d.LY, sizeof(C), 2, (int)(128 / sizeof(C)));
    const size_t sm = 2 * (size_t)d.LY * B * sizeof(C);
    dim3 grid((d.KX + B - 1) / B, (unsigned)(d.nb * 3 * d.nz));
    auto k = rt_y_pass<T, DIR>;
    rt_smem(k, sm);
    k<<<grid, kRtThreads, sm, st>>>(d, in, out, pl, B);
}

template <typename T>
void launch_rt_z(const DemagDims& d, typename Cplx<T>::type* S2, const T* tens, cudaStream_t st) {
    using C = typename Cplx<T>::type;
    const RtPlan pl = make_plan(d.LZ);
    const int B = rt_lines(d.LZ, sizeof(C), 4, (int)(128 / sizeof(C)));
    const size_t sm = 4 * (size_t)d.LZ * B * sizeof(C);
    dim3 grid((d.KX + B - 1) / B, 2 * (d.LY / 2 + 1), d.nb);
    auto k = rt_z_conv<T>;
    rt_smem(k, sm);
    k<<<grid, kRtThreads, sm, st>>>(d, S2, tens, pl, B);
}

template void launch_rt_x_fwd<float>(const DemagDims&, const float*, const float*, float, float2*, cudaStream_t);
template void launch_rt_x_fwd<double>(const DemagDims&, const double*, const double*, double, double2*,
                                      cudaStream_t);
template void launch_rt_x_inv<float>(const DemagDims&, const float2*, float*, cudaStream_t);
template void launch_rt_x_inv<double>(const DemagDims&, const double2*, double*, cudaStream_t);
template void launch_rt_y<float, -1>(const DemagDims&, const float2*, float2*, cudaStream_t);
template void launch_rt_y<float, +1>(const DemagDims&, const float2*, float2*, cudaStream_t);
template void launch_rt_y<double, -1>(const DemagDims&, const double2*, double2*, cudaStream_t);
template void launch_rt_y<double, +1>(const DemagDims&, const double2*, double2*, cudaStream_t);
template void launch_rt_z<float>(const DemagDims&, float2*, const float*, cudaStream_t);
template void launch_rt_z<double>(const DemagDims&, double2*, const double*, cudaStream_t);

}  // namespace mm
