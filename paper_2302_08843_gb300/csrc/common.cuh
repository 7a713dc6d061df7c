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
// W5[m] = exp(-2 pi i m / kTw5): twiddles of the mixed-radix lengths r 2^k
// (r = 3, 7 or 25), all of which divide kTw5 = 2^8 3 5^2 7
constexpr int kTw5 = 134400;
static __device__ double2 g_tw5_64[kTw5];
static __device__ float2 g_tw5_32[kTw5];

__host__ __device__ constexpr bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

template <typename T> struct Tw;
template <> struct Tw<float> {
    static __device__ __forceinline__ float2 get(int m) { return __ldg(&g_tw32[m]); }
};
template <> struct Tw<double> {
    static __device__ __forceinline__ double2 get(int m) { return __ldg(&g_tw64[m]); }
};

template <typename T> struct Tw5;
template <> struct Tw5<float> {
    static __device__ __forceinline__ float2 get(int m) { return __ldg(&g_tw5_32[m]); }
};
template <> struct Tw5<double> {
    static __device__ __forceinline__ double2 get(int m) { return __ldg(&g_tw5_64[m]); }
};
// exp(DIR * 2 pi i m / kTw5), 0 <= m < kTw5
template <typename T, int DIR> __device__ __forceinline__ typename Cplx<T>::type twiddle5(int m) {
    typename Cplx<T>::type w = Tw5<T>::get(m);
    if (DIR > 0) w.y = -w.y;
    return w;
}

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

// DFT5 in place, X_q = sum_r a_r exp(DIR 2 pi i r q / 5), from the pairs
// a1 +- a4, a2 +- a3 and the cosines and sines of 2 pi / 5 and 4 pi / 5
template <int DIR, typename C> __device__ __forceinline__ void dft5(C& a0, C& a1, C& a2, C& a3, C& a4) {
    using T = decltype(C::x);
    constexpr T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;
    constexpr T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;
    const C p1 = cadd(a1, a4), m1 = csub(a1, a4), p2 = cadd(a2, a3), m2 = csub(a2, a3);
    const C t1 = mk<C>(a0.x + c1 * p1.x + c2 * p2.x, a0.y + c1 * p1.y + c2 * p2.y);
    const C t2 = mk<C>(a0.x + c2 * p1.x + c1 * p2.x, a0.y + c2 * p1.y + c1 * p2.y);
    // u = s1 m1 + s2 m2, w = s2 m1 - s1 m2: X1 = t1 + DIR i u, X4 = t1 - DIR i u,
    // X2 = t2 + DIR i w, X3 = t2 - DIR i w
    const C u = mk<C>(s1 * m1.x + s2 * m2.x, s1 * m1.y + s2 * m2.y);
    const C w = mk<C>(s2 * m1.x - s1 * m2.x, s2 * m1.y - s1 * m2.y);
    const C iu = DIR < 0 ? mk<C>(u.y, -u.x) : mk<C>(-u.y, u.x);     // DIR i u
    const C iw = DIR < 0 ? mk<C>(w.y, -w.x) : mk<C>(-w.y, w.x);
    a0 = mk<C>(a0.x + p1.x + p2.x, a0.y + p1.y + p2.y);
    a1 = cadd(t1, iu);
    a4 = csub(t1, iu);
    a2 = cadd(t2, iw);
    a3 = csub(t2, iw);
}

// DFT3 in place, X_q = sum_r a_r exp(DIR 2 pi i r q / 3):
// X0 = a0 + (a1 + a2), X1,2 = a0 - (a1 + a2) / 2 +- DIR i (sqrt 3 / 2)(a1 - a2)
template <int DIR, typename C> __device__ __forceinline__ void dft3(C& a0, C& a1, C& a2) {
    using T = decltype(C::x);
    constexpr T h = (T)0.86602540378443864676;      // sin(2 pi / 3)
    const C sm = cadd(a1, a2), df = csub(a1, a2);
    const C t = mk<C>(a0.x - (T)0.5 * sm.x, a0.y - (T)0.5 * sm.y);
    const C u = DIR < 0 ? mk<C>(h * df.y, -h * df.x) : mk<C>(-h * df.y, h * df.x);    // DIR i h df
    a0 = cadd(a0, sm);
    a1 = cadd(t, u);
    a2 = csub(t, u);
}

// DFT6 in place, X_q = sum_r a_r exp(DIR 2 pi i r q / 6), as two DFT3 of the
// even and odd inputs: X_k = E_k + W6^k O_k, X_{k+3} = E_k - W6^k O_k (k < 3),
// W6 = exp(DIR i pi / 3) = (1/2, DIR sqrt(3)/2), W6^2 = (-1/2, DIR sqrt(3)/2)
template <int DIR, typename C> __device__ __forceinline__ void dft6(C (&a)[6]) {
    using T = decltype(C::x);
    constexpr T h = (T)0.86602540378443864676;      // sin(pi / 3)
    C e0 = a[0], e1 = a[2], e2 = a[4], o0 = a[1], o1 = a[3], o2 = a[5];
    dft3<DIR>(e0, e1, e2);
    dft3<DIR>(o0, o1, o2);
    const T sh = DIR * h;
    const C w1 = mk<C>((T)0.5 * o1.x - sh * o1.y, (T)0.5 * o1.y + sh * o1.x);     // W6 o1
    const C w2 = mk<C>((T)-0.5 * o2.x - sh * o2.y, (T)-0.5 * o2.y + sh * o2.x);   // W6^2 o2
    a[0] = cadd(e0, o0); a[3] = csub(e0, o0);
    a[1] = cadd(e1, w1); a[4] = csub(e1, w1);
    a[2] = cadd(e2, w2); a[5] = csub(e2, w2);
}

// DFT12 in place by the prime-factor (Good-Thomas) split 12 = 4 x 3, which
// needs no twiddles: input n = (3 n1 + 4 n2) mod 12 enters DFT4 number n2 at
// place n1, then DFT3 number k1 runs over n2, and its output k2 is X at
// k = (9 k1 + 4 k2) mod 12 (k = k1 mod 4, k = k2 mod 3)
template <int DIR, typename C> __device__ __forceinline__ void dft12(C* a) {
    C t[4][3];
#pragma unroll
    for (int n2 = 0; n2 < 3; ++n2)
#pragma unroll
        for (int n1 = 0; n1 < 4; ++n1) t[n1][n2] = a[(3 * n1 + 4 * n2) % 12];
#pragma unroll
    for (int n2 = 0; n2 < 3; ++n2) dft4<DIR>(t[0][n2], t[1][n2], t[2][n2], t[3][n2]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft3<DIR>(t[k1][0], t[k1][1], t[k1][2]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 3; ++k2) a[(9 * k1 + 4 * k2) % 12] = t[k1][k2];
}

// DFT7 in place, X_q = sum_r a_r exp(DIR 2 pi i r q / 7), from the pairs
// p_k = a_k + a_{7-k}, m_k = a_k - a_{7-k} (k = 1, 2, 3):
// X_q, X_{7-q} = a0 + sum_k p_k cos(2 pi k q / 7) +- DIR i sum_k m_k sin(2 pi k q / 7)
template <int DIR, typename C> __device__ __forceinline__ void dft7(C (&a)[7]) {
    using T = decltype(C::x);
    constexpr T c1 = (T)0.62348980185873353053, c2 = (T)-0.22252093395631440429, c3 = (T)-0.90096886790241912624;
    constexpr T s1 = (T)0.78183148246802980871, s2 = (T)0.97492791218182360702, s3 = (T)0.43388373911755812048;
    const C p1 = cadd(a[1], a[6]), m1 = csub(a[1], a[6]);
    const C p2 = cadd(a[2], a[5]), m2 = csub(a[2], a[5]);
    const C p3 = cadd(a[3], a[4]), m3 = csub(a[3], a[4]);
    const C a0 = a[0];
    // cosine parts (kq mod 7 -> cos of the nearer of r, 7 - r)
    const C t1 = mk<C>(a0.x + c1 * p1.x + c2 * p2.x + c3 * p3.x, a0.y + c1 * p1.y + c2 * p2.y + c3 * p3.y);
    const C t2 = mk<C>(a0.x + c2 * p1.x + c3 * p2.x + c1 * p3.x, a0.y + c2 * p1.y + c3 * p2.y + c1 * p3.y);
    const C t3 = mk<C>(a0.x + c3 * p1.x + c1 * p2.x + c2 * p3.x, a0.y + c3 * p1.y + c1 * p2.y + c2 * p3.y);
    // sine parts (sin of 7 - r is -sin r)
    const C u1 = mk<C>(s1 * m1.x + s2 * m2.x + s3 * m3.x, s1 * m1.y + s2 * m2.y + s3 * m3.y);
    const C u2 = mk<C>(s2 * m1.x - s3 * m2.x - s1 * m3.x, s2 * m1.y - s3 * m2.y - s1 * m3.y);
    const C u3 = mk<C>(s3 * m1.x - s1 * m2.x + s2 * m3.x, s3 * m1.y - s1 * m2.y + s2 * m3.y);
    const C i1 = DIR < 0 ? mk<C>(u1.y, -u1.x) : mk<C>(-u1.y, u1.x);      // DIR i u
    const C i2 = DIR < 0 ? mk<C>(u2.y, -u2.x) : mk<C>(-u2.y, u2.x);
    const C i3 = DIR < 0 ? mk<C>(u3.y, -u3.x) : mk<C>(-u3.y, u3.x);
    a[0] = mk<C>(a0.x + p1.x + p2.x + p3.x, a0.y + p1.y + p2.y + p3.y);
    a[1] = cadd(t1, i1); a[6] = csub(t1, i1);
    a[2] = cadd(t2, i2); a[5] = csub(t2, i2);
    a[3] = cadd(t3, i3); a[4] = csub(t3, i3);
}

// cos and sin of pi k / 8, k = 0..15
__host__ __device__ constexpr double c16(int k) {
    return k == 0 ? 1.0 : k == 1 ? 0.92387953251128675613 : k == 2 ? 0.70710678118654752440
         : k == 3 ? 0.38268343236508977173 : k == 4 ? 0.0 : k == 5 ? -0.38268343236508977173
         : k == 6 ? -0.70710678118654752440 : k == 7 ? -0.92387953251128675613 : k == 8 ? -1.0
         : k == 9 ? -0.92387953251128675613 : k == 10 ? -0.70710678118654752440
         : k == 11 ? -0.38268343236508977173 : k == 12 ? 0.0 : k == 13 ? 0.38268343236508977173
         : k == 14 ? 0.70710678118654752440 : 0.92387953251128675613;
}
__host__ __device__ constexpr double s16(int k) { return c16((k + 12) & 15); }   // sin(x) = cos(x - pi/2)

// a * exp(DIR 2 pi i K / 16)
template <int DIR, int K, typename C> __device__ __forceinline__ C mul_w16(C a) {
    using T = decltype(C::x);
    constexpr int k = K & 15;
    if constexpr (k == 0) {
        return a;
    } else if constexpr (k == 4) {
        return mul_i<DIR>(a);
    } else if constexpr (k == 8) {
        return mk<C>(-a.x, -a.y);
    } else if constexpr (k == 12) {
        return mul_i<-DIR>(a);
    } else {
        constexpr T c = (T)c16(k), sn = (T)(DIR * s16(k));
        return mk<C>(a.x * c - a.y * sn, a.x * sn + a.y * c);
    }
}

// DFT16 in place (radix 4 x 4); HALF: inputs 8..15 are known zeros
template <int DIR, bool HALF, typename C> __device__ __forceinline__ void dft16(C* a) {
    C y0[4], y1[4], y2[4], y3[4];
    C* y[4] = {y0, y1, y2, y3};
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        C b0 = a[n2], b1 = a[4 + n2];
        if (HALF) {
            y[n2][0] = cadd(b0, b1);
            y[n2][2] = csub(b0, b1);
            y[n2][1] = cadd(b0, mul_i<DIR>(b1));
            y[n2][3] = csub(b0, mul_i<DIR>(b1));
        } else {
            C b2 = a[8 + n2], b3 = a[12 + n2];
            dft4<DIR>(b0, b1, b2, b3);
            y[n2][0] = b0; y[n2][1] = b1; y[n2][2] = b2; y[n2][3] = b3;
        }
    }
    // twiddles W16^(n2 k1)
    y1[1] = mul_w16<DIR, 1>(y1[1]); y1[2] = mul_w16<DIR, 2>(y1[2]); y1[3] = mul_w16<DIR, 3>(y1[3]);
    y2[1] = mul_w16<DIR, 2>(y2[1]); y2[2] = mul_w16<DIR, 4>(y2[2]); y2[3] = mul_w16<DIR, 6>(y2[3]);
    y3[1] = mul_w16<DIR, 3>(y3[1]); y3[2] = mul_w16<DIR, 6>(y3[2]); y3[3] = mul_w16<DIR, 9>(y3[3]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        C b0 = y0[k1], b1 = y1[k1], b2 = y2[k1], b3 = y3[k1];
        dft4<DIR>(b0, b1, b2, b3);
        a[k1] = b0; a[k1 + 4] = b1; a[k1 + 8] = b2; a[k1 + 12] = b3;
    }
}

}  // namespace mm
