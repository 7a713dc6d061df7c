// Shared-memory, register-blocked Stockham FFT over a batch of lines.
//
// One FFT of length L (a power of two, 1..kMaxFft) per "line"; a CTA holds
// several lines.  Each line is served by TPL = max(1, L/8) threads; thread j
// of a line keeps NR = min(8, L) complex values in registers, element
// e = j + r*TPL in register r ("pattern" layout).  The caller loads its input
// in that pattern (from global memory or shared memory), calls run(), and
// finds the output in the same pattern.  Between radix passes the line is
// exchanged through shared memory: element e of the line lives at s[e*LS].
//
// Radix plan: L = R0 * 8^m with R0 in {2, 4, 8}; the first pass (radix R0,
// span 1) may take the zero-padded upper half of the input as known zeros
// (ZIN), which is how the padded demag convolution skips the all-zero half
// of every forward transform.  Later passes are radix 8 with twiddles
// exp(DIR 2 pi i (b mod Ns) q / (8 Ns)) from a double-precision table
// (self-sorting Stockham: input b + q L/8, output
// (b div Ns) 8 Ns + (b mod Ns) + q Ns).  DIR = -1 forward, +1 inverse
// (unnormalised).  Every thread of the CTA must call run() (it contains
// __syncthreads()).
#pragma once

#include "common.cuh"

namespace mm {

template <typename T, int L, int DIR, bool ZIN>
struct FftLine {
    using C = typename Cplx<T>::type;
    static constexpr int K = ilog2(L);
    static constexpr int NR = L >= 8 ? 8 : L;
    static constexpr int TPL = L >= 8 ? L / 8 : 1;
    static constexpr int R0 = (K <= 3) ? L : ((K % 3) ? (1 << (K % 3)) : 8);
    static constexpr int NPASS = (K <= 3) ? 1 : (K / 3 + ((K % 3) ? 1 : 0));

    static __device__ __forceinline__ void run(C* v, C* s, int LS, int j) {
        if constexpr (L == 1) {
            return;
        } else if constexpr (L == 2) {
            if (ZIN) { v[1] = v[0]; } else { dft2<DIR>(v[0], v[1]); }
        } else if constexpr (L == 4) {
            if (ZIN) {
                C a0 = v[0], a1 = v[1];
                v[0] = cadd(a0, a1);
                v[2] = csub(a0, a1);
                v[1] = cadd(a0, mul_i<DIR>(a1));
                v[3] = csub(a0, mul_i<DIR>(a1));
            } else {
                dft4<DIR>(v[0], v[1], v[2], v[3]);
            }
        } else if constexpr (L == 8) {
            if (ZIN) dft8_half<DIR>(v); else dft8<DIR>(v);
        } else {
            // ---- first pass: radix R0, span 1, no twiddles ----
            __syncthreads();                       // the caller may still read s
            if constexpr (R0 == 8) {
                if (ZIN) dft8_half<DIR>(v); else dft8<DIR>(v);
#pragma unroll
                for (int q = 0; q < 8; ++q) s[(8 * j + q) * LS] = v[q];
            } else if constexpr (R0 == 4) {
#pragma unroll
                for (int rr = 0; rr < 2; ++rr) {
                    const int b = j + rr * TPL;
                    C a0 = v[rr], a1 = v[rr + 2], a2, a3;
                    if (ZIN) {
                        a2 = csub(a0, a1);
                        a3 = csub(a0, mul_i<DIR>(a1));
                        C b1 = cadd(a0, mul_i<DIR>(a1));
                        a0 = cadd(a0, a1);
                        a1 = b1;
                    } else {
                        a2 = v[rr + 4];
                        a3 = v[rr + 6];
                        dft4<DIR>(a0, a1, a2, a3);
                    }
                    s[(4 * b + 0) * LS] = a0;
                    s[(4 * b + 1) * LS] = a1;
                    s[(4 * b + 2) * LS] = a2;
                    s[(4 * b + 3) * LS] = a3;
                }
            } else {  // R0 == 2
#pragma unroll
                for (int rr = 0; rr < 4; ++rr) {
                    const int b = j + rr * TPL;
                    C a0 = v[rr], a1;
                    if (ZIN) {
                        a1 = a0;
                    } else {
                        a1 = v[rr + 4];
                        dft2<DIR>(a0, a1);
                    }
                    s[(2 * b + 0) * LS] = a0;
                    s[(2 * b + 1) * LS] = a1;
                }
            }
            // ---- radix-8 passes ----
#pragma unroll
            for (int p = 1; p < NPASS; ++p) {
                const int Ns = R0 << (3 * (p - 1));
                __syncthreads();
#pragma unroll
                for (int r = 0; r < 8; ++r) v[r] = s[(j + r * TPL) * LS];
                const int k = j & (Ns - 1);
                const int step = L / (Ns * 8);
#pragma unroll
                for (int r = 1; r < 8; ++r) v[r] = cmul(v[r], twiddle<T, L, DIR>(k * r * step));
                dft8<DIR>(v);
                if (p < NPASS - 1) {
                    __syncthreads();
                    const int idxD = (j / Ns) * Ns * 8 + k;
#pragma unroll
                    for (int q = 0; q < 8; ++q) s[(idxD + q * Ns) * LS] = v[q];
                }
            }
        }
    }
};

}  // namespace mm
