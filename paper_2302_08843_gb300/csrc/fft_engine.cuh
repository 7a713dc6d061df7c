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

#include <type_traits>

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

    // element of the input that register r of thread j holds, and whether it can be nonzero
    static __device__ __forceinline__ int in_index(int j, int r) { return j + r * TPL; }
    static __host__ __device__ constexpr bool in_live(int r) { return !ZIN || L == 1 || r < NR / 2; }

    static __device__ __forceinline__ void run(C* v, C* s, int LS, int j, const C* = nullptr) {
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

// Radix-16 variant (L >= 16): NR = 16 registers, TPL = L/16 threads per line,
// plan R0 x 16^m with R0 = 2^(log2 L mod 4) (or 16).  The pattern layout and
// the calling convention are those of FftLine, except that with ZIN and
// R0 = 2 the first radix-2 pass (which only duplicates each input) is folded
// into the load: register r then holds input element in_index(j, r) =
// (j + r TPL) / 2 and one shared-memory exchange is saved.  Twiddles of a
// radix-16 pass come from four table loads (w, w^2, w^4, w^8); the other
// powers are at most three products away.
template <typename T, int L, int DIR, bool ZIN, int SKW = 0>
struct FftLine16 {
    using C = typename Cplx<T>::type;
    static_assert(L >= 16, "FftLine16 needs L >= 16");
    static constexpr int K = ilog2(L);
    static constexpr int NR = 16;
    static constexpr int TPL = L / 16;
    static constexpr int R0 = (K % 4) ? (1 << (K % 4)) : 16;
    static constexpr int NPASS = (K % 4) ? (K / 4 + 1) : (K / 4);
    static constexpr bool FOLD2 = ZIN && R0 == 2;

    // shared-memory place of element e: e LS, plus SKW more every 32 elements
    // (a skew that spreads the strided exchange writes over the banks)
    static __device__ __forceinline__ int at(int e, int LS) { return e * LS + (SKW ? (e >> 5) * SKW : 0); }

    static __device__ __forceinline__ int in_index(int j, int r) { return FOLD2 ? ((j + r * TPL) >> 1) : (j + r * TPL); }
    static __host__ __device__ constexpr bool in_live(int r) { return FOLD2 || !ZIN || r < 8; }

    static __device__ __forceinline__ void twiddle16(C* v, int kidx) {
        // v[r] *= W_L^(kidx r), r = 1..15
        const C w1 = twiddle<T, L, DIR>(kidx & (L - 1));
        const C w2 = twiddle<T, L, DIR>((2 * kidx) & (L - 1));
        const C w4 = twiddle<T, L, DIR>((4 * kidx) & (L - 1));
        const C w8 = twiddle<T, L, DIR>((8 * kidx) & (L - 1));
        const C w3 = cmul(w1, w2), w5 = cmul(w1, w4), w6 = cmul(w2, w4), w7 = cmul(w3, w4);
        v[1] = cmul(v[1], w1); v[2] = cmul(v[2], w2); v[3] = cmul(v[3], w3); v[4] = cmul(v[4], w4);
        v[5] = cmul(v[5], w5); v[6] = cmul(v[6], w6); v[7] = cmul(v[7], w7); v[8] = cmul(v[8], w8);
        v[9] = cmul(v[9], cmul(w1, w8)); v[10] = cmul(v[10], cmul(w2, w8)); v[11] = cmul(v[11], cmul(w3, w8));
        v[12] = cmul(v[12], cmul(w4, w8)); v[13] = cmul(v[13], cmul(w5, w8)); v[14] = cmul(v[14], cmul(w6, w8));
        v[15] = cmul(v[15], cmul(w7, w8));
    }

    // twk (optional, for plans with one radix-16 pass): the 16 forward twiddles
    // W_L^(k q L / (16 R0)), q = 0..15, of this thread's butterfly k = j mod R0,
    // read instead of derived (conjugated for the inverse)
    static __device__ __forceinline__ void run(C* v, C* s, int LS, int j, const C* twk = nullptr) {
        if constexpr (NPASS == 1) {
            dft16<DIR, ZIN>(v);
            return;
        } else {
            // ---- first pass (radix R0, span 1), unless folded into the load ----
            if constexpr (!FOLD2) {
                if constexpr (R0 == 16) {
                    dft16<DIR, ZIN>(v);
                    __syncthreads();
#pragma unroll
                    for (int q = 0; q < 16; ++q) s[at(16 * j + q, LS)] = v[q];
                } else if constexpr (R0 == 8) {
                    __syncthreads();
#pragma unroll
                    for (int rr = 0; rr < 2; ++rr) {
                        C a[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) a[q] = v[rr + 2 * q];
                        if (ZIN) dft8_half<DIR>(a); else dft8<DIR>(a);
                        const int b = j + rr * TPL;
#pragma unroll
                        for (int q = 0; q < 8; ++q) s[at(8 * b + q, LS)] = a[q];
                    }
                } else if constexpr (R0 == 4) {
                    __syncthreads();
#pragma unroll
                    for (int rr = 0; rr < 4; ++rr) {
                        C a0 = v[rr], a1 = v[rr + 4], a2, a3;
                        if (ZIN) {
                            a2 = csub(a0, a1);
                            a3 = csub(a0, mul_i<DIR>(a1));
                            C b1 = cadd(a0, mul_i<DIR>(a1));
                            a0 = cadd(a0, a1);
                            a1 = b1;
                        } else {
                            a2 = v[rr + 8];
                            a3 = v[rr + 12];
                            dft4<DIR>(a0, a1, a2, a3);
                        }
                        const int b = j + rr * TPL;
                        s[at(4 * b + 0, LS)] = a0;
                        s[at(4 * b + 1, LS)] = a1;
                        s[at(4 * b + 2, LS)] = a2;
                        s[at(4 * b + 3, LS)] = a3;
                    }
                } else {  // R0 == 2, not zero-padded
                    __syncthreads();
#pragma unroll
                    for (int rr = 0; rr < 8; ++rr) {
                        C a0 = v[rr], a1 = v[rr + 8];
                        dft2<DIR>(a0, a1);
                        const int b = j + rr * TPL;
                        s[at(2 * b + 0, LS)] = a0;
                        s[at(2 * b + 1, LS)] = a1;
                    }
                }
            }
            // ---- radix-16 passes ----
#pragma unroll
            for (int p = 1; p < NPASS; ++p) {
                const int Ns = R0 << (4 * (p - 1));
                if (!(FOLD2 && p == 1)) {
                    __syncthreads();
#pragma unroll
                    for (int r = 0; r < 16; ++r) v[r] = s[at(j + r * TPL, LS)];
                }
                const int k = j & (Ns - 1);
                if (NPASS == 2 && twk) {
#pragma unroll
                    for (int r = 1; r < 16; ++r) {
                        C w = twk[r];
                        if (DIR > 0) w.y = -w.y;
                        v[r] = cmul(v[r], w);
                    }
                } else {
                    twiddle16(v, k * (L / (Ns * 16)));
                }
                dft16<DIR, false>(v);
                if (p < NPASS - 1) {
                    __syncthreads();
                    const int idxD = (j / Ns) * Ns * 16 + k;
#pragma unroll
                    for (int q = 0; q < 16; ++q) s[at(idxD + q * Ns, LS)] = v[q];
                }
            }
        }
    }
};

// ------------------------------------------------------------------------
// Mixed-radix engine for the lengths L = r 2^a with r = 3, 7 or 25 (L
// divides kTw5): passes of the odd radix (3, 7, or 5 twice), then radix-4
// passes and at most one radix-2 pass, Stockham ordering.  Every pass keeps
// the line in shared memory: a thread reads its butterflies' inputs (stride
// L/R), applies the twiddles W_{Ns R}^(q k), transforms them and writes the
// outputs to their autosorted places.  The register layout at entry and exit
// and the calling convention are those of FftLine (register r of thread j
// holds element j + r TPL), so the same kernels drive it; TPL is the largest
// thread count that divides L/R for every radix R of the plan.
__host__ __device__ constexpr int m5_oddr(int L) { return L % 3 == 0 ? 3 : (L % 7 == 0 ? 7 : 5); }
__host__ __device__ constexpr int m5_fives(int L, int r = 0) {
    return L % (r ? r : m5_oddr(L)) ? 0 : 1 + m5_fives(L / (r ? r : m5_oddr(L)), r ? r : m5_oddr(L));
}
__host__ __device__ constexpr int m5_powr(int r, int b) { return b == 0 ? 1 : r * m5_powr(r, b - 1); }
__host__ __device__ constexpr int m5_twos(int L) { return ilog2(L / m5_powr(m5_oddr(L), m5_fives(L))); }
// Shorter plans where the registers allow them (fewer shared-memory round
// trips): 96 = 6 4 4 (12 values per thread, as before), 384 = 6 8 8 and
// 768 = 3 8 8 4 (24 values per thread instead of 12).
__host__ __device__ constexpr int m5_alt_np(int L) { return L == 96 ? 3 : (L == 384 ? 3 : (L == 768 ? 4 : 0)); }
__host__ __device__ constexpr int m5_alt_r(int L, int p) {
    return L == 96 ? (p == 0 ? 6 : 4) : (L == 384 ? (p == 0 ? 6 : 8) : (p == 0 ? 3 : (p < 3 ? 8 : 4)));
}
// (ALT = false keeps the radix 4/2 plan, whose 12 values per thread suit the
// fused stage kernel's small CTAs better.)
__host__ __device__ constexpr int m5_npass(int L, bool alt = true) {
    return (alt && m5_alt_np(L)) ? m5_alt_np(L) : m5_fives(L) + m5_twos(L) / 2 + m5_twos(L) % 2;
}
__host__ __device__ constexpr int m5_radix(int L, int p, bool alt = true) {
    return (alt && m5_alt_np(L)) ? m5_alt_r(L, p)
                                 : (p < m5_fives(L) ? m5_oddr(L) : (p < m5_fives(L) + m5_twos(L) / 2 ? 4 : 2));
}
__host__ __device__ constexpr int m5_gcd(int a, int b) { return b == 0 ? a : m5_gcd(b, a % b); }
__host__ __device__ constexpr int m5_tpl(int L, int p = 0, bool alt = true) {
    return p == m5_npass(L, alt) - 1 ? L / m5_radix(L, p, alt)
                                     : m5_gcd(L / m5_radix(L, p, alt), m5_tpl(L, p + 1, alt));
}

template <typename T, int L, int DIR, bool ZIN, bool ALT = true>
struct FftMixed {
    using C = typename Cplx<T>::type;
    static_assert(kTw5 % L == 0, "mixed-radix lengths must divide the twiddle table");
    static constexpr int NP = m5_npass(L, ALT);
    static constexpr int TPL = m5_tpl(L, 0, ALT);
    static constexpr int NR = L / TPL;
    static constexpr int NTW = 0;
    static_assert(NR % 2 == 0, "the zero-padded half must be whole registers");

    static __device__ __forceinline__ int in_index(int j, int r) { return j + r * TPL; }
    static __host__ __device__ constexpr bool in_live(int r) { return !ZIN || r < NR / 2; }
    static __device__ __forceinline__ int at(int e, int LS) { return e * LS; }   // shared-memory place of element e
    static __device__ void tw_build(C*, int, int) {}

    // Pass P (NS = product of the earlier radices).  The first pass takes its
    // butterflies' inputs from the registers (element b + q L/R of butterfly b
    // = j + t TPL is register t + q NB of the same thread) and the last pass
    // leaves its outputs there (its autosorted places are b + q L/R again), so
    // a transform makes NP - 1 shared-memory exchanges.
    template <int P, int NS>
    static __device__ __forceinline__ void pass(C* v, C* s, int LS, int j) {
        constexpr int R = m5_radix(L, P, ALT);
        constexpr int NB = L / (R * TPL);    // butterflies per thread
        C a[NB][R];
#pragma unroll
        for (int t = 0; t < NB; ++t) {
            const int b = j + t * TPL;
            const int k = b % NS;
#pragma unroll
            for (int q = 0; q < R; ++q) a[t][q] = P == 0 ? v[t + q * NB] : s[(b + q * (L / R)) * LS];
            if (NS > 1) {
#pragma unroll
                for (int q = 1; q < R; ++q) a[t][q] = cmul(a[t][q], twiddle5<T, DIR>(q * k * (kTw5 / (NS * R))));
            }
            if constexpr (R == 8) dft8<DIR>(a[t]);
            else if constexpr (R == 7) dft7<DIR>(a[t]);
            else if constexpr (R == 6) dft6<DIR>(a[t]);
            else if constexpr (R == 5) dft5<DIR>(a[t][0], a[t][1], a[t][2], a[t][3], a[t][4]);
            else if constexpr (R == 4) dft4<DIR>(a[t][0], a[t][1], a[t][2], a[t][3]);
            else if constexpr (R == 3) dft3<DIR>(a[t][0], a[t][1], a[t][2]);
            else dft2<DIR>(a[t][0], a[t][1]);
        }
        if constexpr (P + 1 == NP) {
#pragma unroll
            for (int t = 0; t < NB; ++t)
#pragma unroll
                for (int q = 0; q < R; ++q) v[t + q * NB] = a[t][q];
        } else {
            __syncthreads();   // every read of the scratch (this pass's, or an earlier user's) is done
#pragma unroll
            for (int t = 0; t < NB; ++t) {
                const int b = j + t * TPL;
                const int k = b % NS;
                const int base = (b - k) * R + k;
#pragma unroll
                for (int q = 0; q < R; ++q) s[(base + q * NS) * LS] = a[t][q];
            }
            __syncthreads();
            pass<P + 1, NS * R>(v, s, LS, j);
        }
    }

    static __device__ __forceinline__ void run(C* v, C* s, int LS, int j, const C* = nullptr) {
        pass<0, 1>(v, s, LS, j);
    }
};

// ------------------------------------------------------------------------
// Two-factor engine L = R1 R2 (Cooley-Tukey with one shared-memory exchange
// per transform), TPL threads per line, TPL dividing R1 and R2.
//   forward: x at n = R2 n1 + n2; DFT_R1 over n1 for each n2, times
//            W_L^(n2 k1), exchange, DFT_R2 over n2 for each k1 -> X at k1 + R1 k2
//   inverse: X at k1 + R1 k2; DFT_R2 over k2 for each k1, times W_L^(-na k1),
//            exchange, DFT_R1 over k1 for each na -> x at na + R2 nb
// Register r of thread j holds the spatial element sp_index(j, r) (the
// forward's input, the inverse's output) or the spectral element
// fr_index(j, r) (the forward's output, the inverse's input): the spectrum
// stays in the forward's order, so a pointwise product between the two
// transforms needs no exchange.  Spatial place n < L/2 is register r with
// r mod R1 < R1/2 (the zero-padded input half, the kept output half).  The
// twiddles W_L^m (m < L, forward sign) come from a table tw.
template <typename T, int R1, int R2, int TPL, int DIR, bool ZIN>
struct FftTwo {
    using C = typename Cplx<T>::type;
    static_assert(R1 % TPL == 0 && R2 % TPL == 0, "threads per line must divide both factors");
    static_assert(R1 % 2 == 0, "the zero-padded half must be whole DFT_R1 inputs");
    static constexpr int L = R1 * R2, NR = L / TPL, NA = R2 / TPL, NB = R1 / TPL;
    static __device__ __forceinline__ int sp_index(int j, int r) { return j + (r / R1) * TPL + R2 * (r % R1); }
    static __device__ __forceinline__ int fr_index(int j, int r) { return j + (r / R2) * TPL + R1 * (r % R2); }
    static __host__ __device__ constexpr bool sp_half(int r) { return r % R1 < R1 / 2; }

    template <int R, bool HALF> static __device__ __forceinline__ void dftr(C* a) {
        if constexpr (R == 8) {
            if constexpr (HALF) dft8_half<DIR>(a); else dft8<DIR>(a);
        } else if constexpr (R == 12) {
            dft12<DIR>(a);
        } else if constexpr (R == 4) {
            dft4<DIR>(a[0], a[1], a[2], a[3]);
        } else {
            static_assert(R == 4 || R == 8 || R == 12, "factor without a register DFT");
        }
    }
    static __device__ __forceinline__ C tws(const C* tw, int m) {
        const C w = tw[m];
        return DIR < 0 ? w : mk<C>(w.x, -w.y);
    }
    // s: the line's exchange scratch (element e at s[e LS]); every thread of
    // the block calls run (it synchronises the block)
    static __device__ __forceinline__ void run(C (&v)[NR], C* s, int LS, int j, const C* tw) {
        if constexpr (DIR < 0) {
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                dftr<R1, ZIN>(v + a * R1);
                const int n2 = j + a * TPL;
#pragma unroll
                for (int k1 = 1; k1 < R1; ++k1) v[a * R1 + k1] = cmul(v[a * R1 + k1], tws(tw, n2 * k1));
            }
            __syncthreads();
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int k1 = 0; k1 < R1; ++k1) s[(k1 * R2 + j + a * TPL) * LS] = v[a * R1 + k1];
            __syncthreads();
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
                for (int n2 = 0; n2 < R2; ++n2) v[b * R2 + n2] = s[((j + b * TPL) * R2 + n2) * LS];
#pragma unroll
            for (int b = 0; b < NB; ++b) dftr<R2, false>(v + b * R2);
        } else {
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                dftr<R2, false>(v + b * R2);
                const int k1 = j + b * TPL;
#pragma unroll
                for (int na = 1; na < R2; ++na) v[b * R2 + na] = cmul(v[b * R2 + na], tws(tw, na * k1));
            }
            __syncthreads();
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
                for (int na = 0; na < R2; ++na) s[((j + b * TPL) * R2 + na) * LS] = v[b * R2 + na];
            __syncthreads();
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int k1 = 0; k1 < R1; ++k1) v[a * R1 + k1] = s[(k1 * R2 + j + a * TPL) * LS];
#pragma unroll
            for (int a = 0; a < NA; ++a) dftr<R1, false>(v + a * R1);
        }
    }
};

// engine choice: the mixed-radix engine for the r 2^a lengths, radix 16 for
// FP32 power-of-two lines of 16+ points, radix 8 otherwise
template <typename T, int L, int DIR, bool ZIN>
using Fft = typename std::conditional<
    !is_pow2(L), FftMixed<T, L, DIR, ZIN>,
    typename std::conditional<(sizeof(T) == 4 && L >= 16), FftLine16<T, L, DIR, ZIN>,
                              FftLine<T, L, DIR, ZIN>>::type>::type;

}  // namespace mm
