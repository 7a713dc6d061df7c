// Shared device helpers: complex arithmetic, twiddle tables, small DFTs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mm {

constexpr int kMaxFft = 4096;          // largest padded extent per axis
constexpr double kMu0 = 4.0e-7 * 3.14159265358979323846;
constexpr double kGamma = 2.21e5;      // reduced gyromagnetic ratio (Eq. llg)

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

template <typename C> __host__ __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) {
    C r; r.x = a; r.y = b; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
// multiply by -i (DIR = -1, forward) or +i (DIR = +1, inverse)
template <int DIR, typename C> __device__ __forceinline__ C mul_i(C a) {
    return DIR < 0 ? mk<C>(a.y, -a.x) : mk<C>(-a.y, a.x);
}

// W[m] = exp(-2 pi i m / kMaxFft), built on the host in double precision with
// exact octant symmetry and copied to the device once per device (each
// translation unit that runs FFTs owns a copy and an upload function).
static __device__ double2 g_tw64[kMaxFft];
static __device__ float2 g_tw32[kMaxFft];

template <typename T> struct Tw;
template <> struct Tw<float> {
    static __device__ __forceinline__ float2 get(int m) { return __ldg(&g_tw32[m]); }
};
template <> struct Tw<double> {
    static __device__ __forceinline__ double2 get(int m) { return __ldg(&g_tw64[m]); }
};

// exp(DIR * 2 pi i k / L) for 0 <= k < L (L a power of two <= kMaxFft)
template <typename T, int L, int DIR> __device__ __forceinline__ typename Cplx<T>::type twiddle(int k) {
    typename Cplx<T>::type w = Tw<T>::get(k * (kMaxFft / L));
    if (DIR > 0) w.y = -w.y;
    return w;
}

// ---- small DFTs, in place; X_q = sum_r a_r exp(DIR 2 pi i r q / R) ----
template <int DIR, typename C> __device__ __forceinline__ void dft2(C& a0, C& a1) {
    C t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

template <int DIR, typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
    C t0 = cadd(a0, a2), t1 = csub(a0, a2);
    C t2 = cadd(a1, a3), t3 = mul_i<DIR>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

template <int DIR, typename C> __device__ __forceinline__ C mul_w8_1(C a) {
    // a * exp(DIR i pi / 4)
    using T = decltype(C::x);
    const T s = (T)0.70710678118654752440;
    return DIR < 0 ? mk<C>(s * (a.x + a.y), s * (a.y - a.x)) : mk<C>(s * (a.x - a.y), s * (a.x + a.y));
}
template <int DIR, typename C> __device__ __forceinline__ C mul_w8_3(C a) {
    // a * exp(DIR 3 i pi / 4)
    using T = decltype(C::x);
    const T s = (T)0.70710678118654752440;
    return DIR < 0 ? mk<C>(s * (a.y - a.x), -s * (a.x + a.y)) : mk<C>(-s * (a.x + a.y), s * (a.x - a.y));
}

template <int DIR, typename C> __device__ __forceinline__ void dft8(C* a) {
    C e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
    C o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
    dft4<DIR>(e0, e1, e2, e3);
    dft4<DIR>(o0, o1, o2, o3);
    o1 = mul_w8_1<DIR>(o1);
    o2 = mul_i<DIR>(o2);
    o3 = mul_w8_3<DIR>(o3);
    a[0] = cadd(e0, o0); a[4] = csub(e0, o0);
    a[1] = cadd(e1, o1); a[5] = csub(e1, o1);
    a[2] = cadd(e2, o2); a[6] = csub(e2, o2);
    a[3] = cadd(e3, o3); a[7] = csub(e3, o3);
}

// DFT8 of (a0..a3, 0, 0, 0, 0): the zero-padded upper half is never touched.
template <int DIR, typename C> __device__ __forceinline__ void dft8_half(C* a) {
    // even part DFT4(a0, a2, 0, 0), odd part DFT4(a1, a3, 0, 0)
    C e0 = cadd(a[0], a[2]), e2 = csub(a[0], a[2]);
    C e1 = cadd(a[0], mul_i<DIR>(a[2])), e3 = csub(a[0], mul_i<DIR>(a[2]));
    C o0 = cadd(a[1], a[3]), o2 = csub(a[1], a[3]);
    C o1 = cadd(a[1], mul_i<DIR>(a[3])), o3 = csub(a[1], mul_i<DIR>(a[3]));
    o1 = mul_w8_1<DIR>(o1);
    o2 = mul_i<DIR>(o2);
    o3 = mul_w8_3<DIR>(o3);
    a[0] = cadd(e0, o0); a[4] = csub(e0, o0);
    a[1] = cadd(e1, o1); a[5] = csub(e1, o1);
    a[2] = cadd(e2, o2); a[6] = csub(e2, o2);
    a[3] = cadd(e3, o3); a[7] = csub(e3, o3);
}

__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }

}  // namespace mm
