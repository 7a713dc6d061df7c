// Packed two-line radix-16 Stockham FFT (FP32): one thread transforms the
// same element positions of TWO lines at once.  The two lines' values are
// kept as planar pairs -- P2.re = (re of line A, re of line B), P2.im
// likewise -- so every butterfly add, subtract and multiply of both lines is
// one paired FP32 instruction (add/sub/mul/fma .f32x2), and the twiddles,
// which both lines share, are read once for both.
//
// Layout and calling convention are those of FftLine16 (fft_engine.cuh):
// L = R0 * 16^m, TPL = L / 16 threads per line pair, register r of thread j
// holds element j + r TPL ("pattern" layout) at entry and exit; with ZIN the
// upper half of the input is known zero, and with ZIN and R0 = 2 the first
// radix-2 pass is folded into the load (register r then holds input element
// (j + r TPL) / 2).  The exchange between passes goes through shared memory
// as whole P2 values (16 bytes): element e of the pair at s[e LS].
//
// Twiddles: a radix-16 pass of span Ns multiplies element q of butterfly k
// by W_{16 Ns}^(k q) (W_N = exp(-2 pi i / N); conjugated for the inverse),
// which depends on (Ns, k, q) only.  g_twp16 holds them for every span
// Ns = 1, 2, 4, ..., 256 as (cos, cos, sin, sin) -- already broadcast to
// both lanes -- at index 16 (Ns - 1) + 16 k + q.
#pragma once

#include "common.cuh"

namespace mm {

struct __align__(16) P2 {
    float2 re, im;
};

constexpr int kTwP16 = 16 * 511;     // spans 1 .. 256: 16 * (1 + 2 + ... + 256)
static __device__ float4 g_twp16[kTwP16];

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
    unsigned long long ra = *reinterpret_cast<unsigned long long*>(&a);
    unsigned long long rb = *reinterpret_cast<unsigned long long*>(&b);
    unsigned long long rd;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    return *reinterpret_cast<float2*>(&rd);
}
__device__ __forceinline__ float2 f2s(float v) { return make_float2(v, v); }

__device__ __forceinline__ P2 padd(P2 a, P2 b) { return {f2add(a.re, b.re), f2add(a.im, b.im)}; }
__device__ __forceinline__ P2 psub(P2 a, P2 b) { return {f2sub(a.re, b.re), f2sub(a.im, b.im)}; }
// a + DIR i b and a - DIR i b
template <int DIR> __device__ __forceinline__ P2 paddi(P2 a, P2 b) {
    return DIR > 0 ? P2{f2sub(a.re, b.im), f2add(a.im, b.re)} : P2{f2add(a.re, b.im), f2sub(a.im, b.re)};
}
template <int DIR> __device__ __forceinline__ P2 psubi(P2 a, P2 b) { return paddi<-DIR>(a, b); }

// a * (c + i s) with c, s the same for both lanes
__device__ __forceinline__ P2 pmul_cs(P2 a, float2 c, float2 s) {
    return {f2sub(f2mul(a.re, c), f2mul(a.im, s)), f2fma(a.re, s, f2mul(a.im, c))};
}
// a * W from a table entry t = (cos, cos, sin, sin) of W_N^m = exp(-2 pi i m / N):
// the forward transform multiplies by W, the inverse by its conjugate
template <int DIR> __device__ __forceinline__ P2 ptw(P2 a, float4 t) {
    const float2 c = make_float2(t.x, t.y), s = make_float2(t.z, t.w);
    if (DIR < 0) return {f2sub(f2mul(a.re, c), f2mul(a.im, s)), f2fma(a.re, s, f2mul(a.im, c))};
    return {f2fma(a.im, s, f2mul(a.re, c)), f2sub(f2mul(a.im, c), f2mul(a.re, s))};
}

// product of two broadcast table entries (cos, cos, sin, sin)
__device__ __forceinline__ float4 bmul(float4 a, float4 b) {
    const float2 ac = make_float2(a.x, a.y), as = make_float2(a.z, a.w);
    const float2 bc = make_float2(b.x, b.y), bs = make_float2(b.z, b.w);
    const float2 c = f2sub(f2mul(ac, bc), f2mul(as, bs)), sn = f2fma(ac, bs, f2mul(as, bc));
    return make_float4(c.x, c.y, sn.x, sn.y);
}

// DFT4 in place, X_q = sum_r a_r exp(DIR 2 pi i r q / 4)
template <int DIR> __device__ __forceinline__ void pdft4(P2& a0, P2& a1, P2& a2, P2& a3) {
    const P2 t0 = padd(a0, a2), t1 = psub(a0, a2), t2 = padd(a1, a3), d = psub(a1, a3);
    a0 = padd(t0, t2);
    a2 = psub(t0, t2);
    a1 = paddi<DIR>(t1, d);
    a3 = psubi<DIR>(t1, d);
}

// a * exp(DIR 2 pi i K / 16), K = 1..15 (K = 4, 8, 12 are handled by callers)
template <int DIR, int K> __device__ __forceinline__ P2 pmul_w16(P2 a) {
    constexpr float c = (float)c16(K & 15), sn = (float)(DIR * s16(K & 15));
    if constexpr ((K & 3) == 2) {
        // +-45 degree multiples: c = +-sn in magnitude, two adds and two multiplies
        constexpr float m = c;    // |c| = |sn| = sqrt(1/2)
        if constexpr (c * sn > 0) {   // (re - im, re + im) * c
            return {f2mul(f2sub(a.re, a.im), f2s(m)), f2mul(f2add(a.re, a.im), f2s(m))};
        } else {                      // (re + im, im - re) * c
            return {f2mul(f2add(a.re, a.im), f2s(m)), f2mul(f2sub(a.im, a.re), f2s(m))};
        }
    } else {
        return pmul_cs(a, f2s(c), f2s(sn));
    }
}

// DFT16 in place (radix 4 x 4); HALF: inputs 8..15 are known zeros
template <int DIR, bool HALF> __device__ __forceinline__ void pdft16(P2* a) {
    P2 y0[4], y1[4], y2[4], y3[4];
    P2* y[4] = {y0, y1, y2, y3};
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        P2 b0 = a[n2], b1 = a[4 + n2];
        if (HALF) {
            y[n2][0] = padd(b0, b1);
            y[n2][2] = psub(b0, b1);
            y[n2][1] = paddi<DIR>(b0, b1);
            y[n2][3] = psubi<DIR>(b0, b1);
        } else {
            P2 b2 = a[8 + n2], b3 = a[12 + n2];
            pdft4<DIR>(b0, b1, b2, b3);
            y[n2][0] = b0; y[n2][1] = b1; y[n2][2] = b2; y[n2][3] = b3;
        }
    }
    // twiddles W16^(n2 k1); y2[2] takes W16^4 = DIR i, folded into the k1 = 2 butterfly below
    y1[1] = pmul_w16<DIR, 1>(y1[1]); y1[2] = pmul_w16<DIR, 2>(y1[2]); y1[3] = pmul_w16<DIR, 3>(y1[3]);
    y2[1] = pmul_w16<DIR, 2>(y2[1]); y2[3] = pmul_w16<DIR, 6>(y2[3]);
    y3[1] = pmul_w16<DIR, 3>(y3[1]); y3[2] = pmul_w16<DIR, 6>(y3[2]); y3[3] = pmul_w16<DIR, 9>(y3[3]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        P2 b0 = y0[k1], b1 = y1[k1], b2 = y2[k1], b3 = y3[k1];
        if (k1 == 2) {
            // b2 stands for DIR i b2: t0 = b0 + DIR i b2, t1 = b0 - DIR i b2
            const P2 t0 = paddi<DIR>(b0, b2), t1 = psubi<DIR>(b0, b2), t2 = padd(b1, b3), d = psub(b1, b3);
            b0 = padd(t0, t2);
            b2 = psub(t0, t2);
            b1 = paddi<DIR>(t1, d);
            b3 = psubi<DIR>(t1, d);
        } else {
            pdft4<DIR>(b0, b1, b2, b3);
        }
        a[k1] = b0; a[k1 + 4] = b1; a[k1 + 8] = b2; a[k1 + 12] = b3;
    }
}

// DFT8 in place; HALF: inputs 4..7 are known zeros
template <int DIR, bool HALF> __device__ __forceinline__ void pdft8(P2* a) {
    P2 e0, e1, e2, e3, o0, o1, o2, o3;
    if (HALF) {
        e0 = padd(a[0], a[2]); e2 = psub(a[0], a[2]);
        e1 = paddi<DIR>(a[0], a[2]); e3 = psubi<DIR>(a[0], a[2]);
        o0 = padd(a[1], a[3]); o2 = psub(a[1], a[3]);
        o1 = paddi<DIR>(a[1], a[3]); o3 = psubi<DIR>(a[1], a[3]);
    } else {
        e0 = a[0]; e1 = a[2]; e2 = a[4]; e3 = a[6];
        o0 = a[1]; o1 = a[3]; o2 = a[5]; o3 = a[7];
        pdft4<DIR>(e0, e1, e2, e3);
        pdft4<DIR>(o0, o1, o2, o3);
    }
    o1 = pmul_w16<DIR, 2>(o1);     // W8^1
    o3 = pmul_w16<DIR, 6>(o3);     // W8^3
    // o2 takes W8^2 = DIR i
    a[0] = padd(e0, o0); a[4] = psub(e0, o0);
    a[1] = padd(e1, o1); a[5] = psub(e1, o1);
    a[2] = paddi<DIR>(e2, o2); a[6] = psubi<DIR>(e2, o2);
    a[3] = padd(e3, o3); a[7] = psub(e3, o3);
}

template <int L, int DIR, bool ZIN>
struct FftPair16 {
    static_assert(L >= 16 && is_pow2(L) && L <= kMaxFft, "FftPair16: power-of-two lines of 16..4096 points");
    static constexpr int K = ilog2(L);
    static constexpr int NR = 16;
    static constexpr int TPL = L / 16;
    static constexpr int R0 = (K % 4) ? (1 << (K % 4)) : 16;
    static constexpr int NPASS = (K % 4) ? (K / 4 + 1) : (K / 4);
    static constexpr bool FOLD2 = ZIN && R0 == 2;

    static __device__ __forceinline__ int in_index(int j, int r) { return FOLD2 ? ((j + r * TPL) >> 1) : (j + r * TPL); }
    static __host__ __device__ constexpr bool in_live(int r) { return FOLD2 || !ZIN || r < 8; }

    static __device__ __forceinline__ void run(P2* v, P2* s, int LS, int j) {
        if constexpr (NPASS == 1) {
            pdft16<DIR, ZIN>(v);
            return;
        } else {
            if constexpr (!FOLD2) {
                if constexpr (R0 == 16) {
                    pdft16<DIR, ZIN>(v);
                    __syncthreads();
#pragma unroll
                    for (int q = 0; q < 16; ++q) s[(16 * j + q) * LS] = v[q];
                } else if constexpr (R0 == 8) {
                    __syncthreads();
#pragma unroll
                    for (int rr = 0; rr < 2; ++rr) {
                        P2 a[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) a[q] = v[rr + 2 * q];
                        pdft8<DIR, ZIN>(a);
                        const int b = j + rr * TPL;
#pragma unroll
                        for (int q = 0; q < 8; ++q) s[(8 * b + q) * LS] = a[q];
                    }
                } else if constexpr (R0 == 4) {
                    __syncthreads();
#pragma unroll
                    for (int rr = 0; rr < 4; ++rr) {
                        P2 a0 = v[rr], a1 = v[rr + 4], a2, a3;
                        if (ZIN) {
                            a2 = psub(a0, a1);
                            a3 = psubi<DIR>(a0, a1);
                            const P2 b1 = paddi<DIR>(a0, a1);
                            a0 = padd(a0, a1);
                            a1 = b1;
                        } else {
                            a2 = v[rr + 8];
                            a3 = v[rr + 12];
                            pdft4<DIR>(a0, a1, a2, a3);
                        }
                        const int b = j + rr * TPL;
                        s[(4 * b + 0) * LS] = a0;
                        s[(4 * b + 1) * LS] = a1;
                        s[(4 * b + 2) * LS] = a2;
                        s[(4 * b + 3) * LS] = a3;
                    }
                } else {  // R0 == 2, not zero-padded
                    __syncthreads();
#pragma unroll
                    for (int rr = 0; rr < 8; ++rr) {
                        const P2 a0 = v[rr], a1 = v[rr + 8];
                        const int b = j + rr * TPL;
                        s[(2 * b + 0) * LS] = padd(a0, a1);
                        s[(2 * b + 1) * LS] = psub(a0, a1);
                    }
                }
            }
#pragma unroll
            for (int p = 1; p < NPASS; ++p) {
                const int Ns = R0 << (4 * (p - 1));
                if (!(FOLD2 && p == 1)) {
                    __syncthreads();
#pragma unroll
                    for (int r = 0; r < 16; ++r) v[r] = s[(j + r * TPL) * LS];
                }
                const int k = j & (Ns - 1);
                const float4* tw = g_twp16 + 16 * (Ns - 1) + 16 * k;
                // four table loads (q = 1, 2, 4, 8), the other powers by products
                const float4 w1 = __ldg(tw + 1), w2 = __ldg(tw + 2), w4 = __ldg(tw + 4), w8 = __ldg(tw + 8);
                const float4 w3 = bmul(w1, w2), w5 = bmul(w1, w4), w6 = bmul(w2, w4), w7 = bmul(w3, w4);
                v[1] = ptw<DIR>(v[1], w1); v[2] = ptw<DIR>(v[2], w2); v[3] = ptw<DIR>(v[3], w3);
                v[4] = ptw<DIR>(v[4], w4); v[5] = ptw<DIR>(v[5], w5); v[6] = ptw<DIR>(v[6], w6);
                v[7] = ptw<DIR>(v[7], w7); v[8] = ptw<DIR>(v[8], w8);
                v[9] = ptw<DIR>(v[9], bmul(w1, w8)); v[10] = ptw<DIR>(v[10], bmul(w2, w8));
                v[11] = ptw<DIR>(v[11], bmul(w3, w8)); v[12] = ptw<DIR>(v[12], bmul(w4, w8));
                v[13] = ptw<DIR>(v[13], bmul(w5, w8)); v[14] = ptw<DIR>(v[14], bmul(w6, w8));
                v[15] = ptw<DIR>(v[15], bmul(w7, w8));
                pdft16<DIR, false>(v);
                if (p < NPASS - 1) {
                    __syncthreads();
                    const int idxD = (j / Ns) * Ns * 16 + k;
#pragma unroll
                    for (int q = 0; q < 16; ++q) s[(idxD + q * Ns) * LS] = v[q];
                }
            }
        }
    }
};

// host: fill the broadcast twiddle table from a table W[m] = exp(-2 pi i m / kMaxFft)
// (kMaxFft = 16 * 256, so W_{16 Ns}^(k q) = W[k q (256 / Ns) mod kMaxFft])
inline void build_twp16(const double2* w, float4* out) {
    for (int Ns = 1; Ns <= 256; Ns <<= 1)
        for (int k = 0; k < Ns; ++k)
            for (int q = 0; q < 16; ++q) {
                const double2 v = w[(k * q * (256 / Ns)) % kMaxFft];
                out[16 * (Ns - 1) + 16 * k + q] = make_float4((float)v.x, (float)v.x, (float)v.y, (float)v.y);
            }
}

}  // namespace mm
