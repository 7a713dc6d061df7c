// Local field terms, LLG right-hand side and Runge-Kutta stage combination,
// one thread per cell, with block-level reductions.
//
// Per cell i (Ms_i != 0; a cell with Ms_i = 0 has h = 0):
//   exchange   (Sec. 4.2): h_ex = 2/(mu0 Ms_i) sum_k (2 A_i A_k/(A_i+A_k)) / d_k^2 (m_k - m_i),
//              links only to cells inside the grid (Neumann boundary);
//   anisotropy (Sec. 4.1): h_u = 2 Ku1/(mu0 Ms_i) e (e.m);
//   Zeeman:                h_z = w_i h(t);
//   demag      (Sec. 4.4): read from the FFT passes;
//   LLG        (Eq. llg):  k = -gamma/(1+alpha^2) [m x h + alpha m x (m x h)].
// Then, depending on the stage:
//   acc_out = acc_in + acc_b k                          (RK4 weight accumulator)
//   next    = mn + dt (sum_j kc_j kin_j + ck k)          (next stage input / new m)
//   e       = dt (sum_j eb_j kin_j + eb_k k)             (DP45 error estimate)
// and per-block partials: max |m x h|/Ms, the four energies
// (Eq. linear_energy_discrete), max |e| / (atol + rtol max(|mn|, |m|)), and a
// non-finite flag.  Partials are reduced by a single-block kernel in a fixed
// order, so every scalar is deterministic.
#include "demag.h"

namespace mm {

constexpr int kStageThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

template <typename T>
__device__ __forceinline__ T harmonic(T a, T b) {
    const T s = a + b;
    return s != (T)0 ? (T)2 * a * b / s : (T)0;
}

// A of a link between cells of thickness ha, hb in series (non-equidistant
// layers): (ha + hb) a b / (ha b + hb a), the harmonic mean when ha = hb
template <typename T>
__device__ __forceinline__ T thick_harmonic(T a, T b, T ha, T hb) {
    const T s = ha * b + hb * a;
    return s != (T)0 ? (ha + hb) * a * b / s : (T)0;
}

// VEC consecutive cells along x per thread (float2 / double2 loads).
template <typename T, int VEC> struct Vec;
template <> struct Vec<float, 2> {
    static __device__ __forceinline__ void ld(const float* p, float* v) {
        const float2 q = *reinterpret_cast<const float2*>(p);
        v[0] = q.x; v[1] = q.y;
    }
    static __device__ __forceinline__ void st(float* p, const float* v) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    }
};
template <> struct Vec<double, 2> {
    static __device__ __forceinline__ void ld(const double* p, double* v) {
        const double2 q = *reinterpret_cast<const double2*>(p);
        v[0] = q.x; v[1] = q.y;
    }
    static __device__ __forceinline__ void st(double* p, const double* v) {
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    }
};
template <typename T> struct Vec<T, 1> {
    static __device__ __forceinline__ void ld(const T* p, T* v) { v[0] = *p; }
    static __device__ __forceinline__ void st(T* p, const T* v) { *p = v[0]; }
};

constexpr int kBX = 64, kBY = 4;   // threads per block: 64 along x, 4 rows of y

// 3-D launch: blockIdx.z = z, blockIdx.y * kBY + threadIdx.y = y,
// (blockIdx.x * kBX + threadIdx.x) * VEC = first x of the thread's cells.
// Requires nx % VEC == 0 (all of a thread's cells in one row).
// UNI: Ms, A, Ku and alpha are uniform scalars (easy axes may still vary by
// grain); the per-cell branches for material maps then compile away.
// Eq. D_avg as read: harmonic mean for equal signs, otherwise the geometric mean
// of the geometric and the arithmetic mean with the sign of the sum
template <typename T> __device__ __forceinline__ T dmi_avg(T a, T b) {
    const T prod = a * b, s = a + b;
    if (prod >= (T)0) return s != (T)0 ? (T)2 * prod / s : (T)0;
    return copysign(sqrt(sqrt(-prod) * fabs(s) * (T)0.5), s);
}

// out += e x w
template <typename T> __device__ __forceinline__ void cross_add(const T* e, T wx, T wy, T wz, T& ox, T& oy, T& oz) {
    ox += e[1] * wz - e[2] * wy;
    oy += e[2] * wx - e[0] * wz;
    oz += e[0] * wy - e[1] * wx;
}

// resident CTAs asked of the register allocator: three for FP32 without DMI
// (a latency-bound kernel; measured 13 % faster than two at 128 registers on
// a 256x256x8 grid), two otherwise (FP64 is ALU-bound, the DMI variant would spill)
template <typename T, bool DMI> constexpr int stage_min_blocks() { return (sizeof(T) == 4 && !DMI) ? 3 : 2; }

template <typename T, int VEC, bool UNI, bool DMI>
__global__ void __launch_bounds__(kStageThreads, stage_min_blocks<T, DMI>()) stage_kernel(StageParams<T> p) {
    using LV = Vec<T, VEC>;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int N = (int)p.N;
    const int x0 = (blockIdx.x * kBX + threadIdx.x) * VEC;
    const int y = blockIdx.y * kBY + threadIdx.y;
    const int z = blockIdx.z;
    double red_e0 = 0.0, red_e1 = 0.0, red_e2 = 0.0, red_e3 = 0.0, red_e4 = 0.0;
    int red_nf = 0;
    // the torque |m x h| / Ms and the error ratio |dt e| / sc, in the state's
    // precision; the error's maximum kept as a fraction en / ed (cross-multiplied
    // comparisons, one division per thread)
    T red_tq = 0, en = 0, ed = 1;
    if (x0 < nx && y < ny) {
        const int i = x0 + nx * (y + ny * z);
        const int sy = nx, sz = nx * ny;
        const T* m = p.m;
        T mx[VEC], my[VEC], mz[VEC];
        LV::ld(m + i, mx); LV::ld(m + N + i, my); LV::ld(m + 2 * N + i, mz);
        T Ms[VEC], A[VEC];
        if (!UNI && p.Ms_cell) LV::ld(p.Ms_cell + i, Ms); else { for (int v = 0; v < VEC; ++v) Ms[v] = p.Ms; }
        if (!UNI && p.A_cell) LV::ld(p.A_cell + i, A); else { for (int v = 0; v < VEC; ++v) A[v] = p.A; }
        const bool a_cell = !UNI && p.A_cell;
        // exchange sums s = sum_links w_link / d^2 (m_nb - m_i), w_link the harmonic mean of A
        T sx[VEC], sy_[VEC], sz_[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) { sx[v] = 0; sy_[v] = 0; sz_[v] = 0; }
        // x links inside the vector and to the scalar neighbours at both ends
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const int x = x0 + v;
            if (x > 0) {
                T nbx, nby, nbz, Anb;
                if (v > 0) { nbx = mx[v - 1]; nby = my[v - 1]; nbz = mz[v - 1]; Anb = A[v - 1]; }
                else { nbx = m[i - 1]; nby = m[N + i - 1]; nbz = m[2 * N + i - 1]; Anb = a_cell ? p.A_cell[i - 1] : p.A; }
                const T w = (a_cell ? harmonic(A[v], Anb) : p.A) * p.idx2;
                sx[v] += w * (nbx - mx[v]); sy_[v] += w * (nby - my[v]); sz_[v] += w * (nbz - mz[v]);
            }
            if (x < nx - 1) {
                T nbx, nby, nbz, Anb;
                if (v < VEC - 1) { nbx = mx[v + 1]; nby = my[v + 1]; nbz = mz[v + 1]; Anb = A[v + 1]; }
                else { nbx = m[i + VEC]; nby = m[N + i + VEC]; nbz = m[2 * N + i + VEC]; Anb = a_cell ? p.A_cell[i + VEC] : p.A; }
                const T w = (a_cell ? harmonic(A[v], Anb) : p.A) * p.idx2;
                sx[v] += w * (nbx - mx[v]); sy_[v] += w * (nby - my[v]); sz_[v] += w * (nbz - mz[v]);
            }
        }
        // y and z links: whole vectors of neighbours
#define MM_VLINK(COND, OFF, ID2)                                                          \
        if (COND) {                                                                       \
            T nbx[VEC], nby[VEC], nbz[VEC], Anb[VEC];                                     \
            LV::ld(m + i + (OFF), nbx); LV::ld(m + N + i + (OFF), nby); LV::ld(m + 2 * N + i + (OFF), nbz); \
            if (a_cell) LV::ld(p.A_cell + i + (OFF), Anb);                                \
            _Pragma("unroll") for (int v = 0; v < VEC; ++v) {                              \
                const T w = (a_cell ? harmonic(A[v], Anb[v]) : p.A) * (ID2);              \
                sx[v] += w * (nbx[v] - mx[v]); sy_[v] += w * (nby[v] - my[v]); sz_[v] += w * (nbz[v] - mz[v]); \
            }                                                                             \
        }
        MM_VLINK(y > 0, -sy, p.idy2)
        MM_VLINK(y < ny - 1, sy, p.idy2)
        if (!p.lay) {
            MM_VLINK(z > 0, -sz, p.idz2)
            MM_VLINK(z < nz - 1, sz, p.idz2)
        } else {
            // non-equidistant layers: 2 A_link / (h_k (h_k + h_nb)) per z link, A_link in series
            const T hk = p.lay[z];
#define MM_LLINK(COND, OFF, COEF, HNB)                                                    \
            if (COND) {                                                                   \
                const T c = (COEF), hn = (HNB);                                           \
                T nbx[VEC], nby[VEC], nbz[VEC], Anb[VEC];                                 \
                LV::ld(m + i + (OFF), nbx); LV::ld(m + N + i + (OFF), nby); LV::ld(m + 2 * N + i + (OFF), nbz); \
                if (a_cell) LV::ld(p.A_cell + i + (OFF), Anb);                            \
                _Pragma("unroll") for (int v = 0; v < VEC; ++v) {                          \
                    const T w = (a_cell ? thick_harmonic(A[v], Anb[v], hk, hn) : p.A) * c; \
                    sx[v] += w * (nbx[v] - mx[v]); sy_[v] += w * (nby[v] - my[v]); sz_[v] += w * (nbz[v] - mz[v]); \
                }                                                                         \
            }
            MM_LLINK(z > 0, -sz, p.lay[2 * nz + z], p.lay[z > 0 ? z - 1 : z])
            MM_LLINK(z < nz - 1, sz, p.lay[nz + z], p.lay[z < nz - 1 ? z + 1 : z])
#undef MM_LLINK
        }
#undef MM_VLINK
        // DMI (Sec. 4.3): dm_i = sum_axes e_a x (Dt_+ m_{i+a} - Dt_- m_{i-a}) / (2 d_a); a neighbour
        // outside the grid is left out; Dt the link average of D (D itself when uniform)
        T dmx[VEC], dmy[VEC], dmz[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) { dmx[v] = 0; dmy[v] = 0; dmz[v] = 0; }
        if constexpr (DMI) {
            const bool d_cell = p.D_cell != nullptr;
            T Dc[VEC];
            if (d_cell) LV::ld(p.D_cell + i, Dc); else { for (int v = 0; v < VEC; ++v) Dc[v] = p.D; }
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                const int x = x0 + v;
                T wx = 0, wy = 0, wz = 0;
                if (x < nx - 1) {
                    T nbx, nby, nbz, Dn;
                    if (v < VEC - 1) { nbx = mx[v + 1]; nby = my[v + 1]; nbz = mz[v + 1]; Dn = Dc[v + 1]; }
                    else { nbx = m[i + VEC]; nby = m[N + i + VEC]; nbz = m[2 * N + i + VEC]; Dn = d_cell ? p.D_cell[i + VEC] : p.D; }
                    const T Dt = d_cell ? dmi_avg(Dc[v], Dn) : p.D;
                    wx += Dt * nbx; wy += Dt * nby; wz += Dt * nbz;
                }
                if (x > 0) {
                    T nbx, nby, nbz, Dn;
                    if (v > 0) { nbx = mx[v - 1]; nby = my[v - 1]; nbz = mz[v - 1]; Dn = Dc[v - 1]; }
                    else { nbx = m[i - 1]; nby = m[N + i - 1]; nbz = m[2 * N + i - 1]; Dn = d_cell ? p.D_cell[i - 1] : p.D; }
                    const T Dt = d_cell ? dmi_avg(Dc[v], Dn) : p.D;
                    wx -= Dt * nbx; wy -= Dt * nby; wz -= Dt * nbz;
                }
                cross_add(&p.dmi_e[0], wx * p.i2dx, wy * p.i2dx, wz * p.i2dx, dmx[v], dmy[v], dmz[v]);
            }
#define MM_DLINK(COND, OFF, SIGN, E, I2D)                                                  \
            if (COND) {                                                                    \
                T nbx[VEC], nby[VEC], nbz[VEC], Dn[VEC];                                   \
                LV::ld(m + i + (OFF), nbx); LV::ld(m + N + i + (OFF), nby); LV::ld(m + 2 * N + i + (OFF), nbz); \
                if (d_cell) LV::ld(p.D_cell + i + (OFF), Dn);                              \
                _Pragma("unroll") for (int v = 0; v < VEC; ++v) {                           \
                    const T Dt = (SIGN) * (d_cell ? dmi_avg(Dc[v], Dn[v]) : p.D) * (I2D);  \
                    cross_add(E, Dt * nbx[v], Dt * nby[v], Dt * nbz[v], dmx[v], dmy[v], dmz[v]); \
                }                                                                          \
            }
            MM_DLINK(y > 0, -sy, (T)-1, &p.dmi_e[3], p.i2dy)
            MM_DLINK(y < ny - 1, sy, (T)1, &p.dmi_e[3], p.i2dy)
            MM_DLINK(z > 0, -sz, (T)-1, &p.dmi_e[6], p.i2dz)
            MM_DLINK(z < nz - 1, sz, (T)1, &p.dmi_e[6], p.i2dz)
#undef MM_DLINK
        }
        T Ku[VEC], al[VEC], zw[VEC], hdx[VEC], hdy[VEC], hdz[VEC];
        if (!UNI && p.Ku_cell) LV::ld(p.Ku_cell + i, Ku); else { for (int v = 0; v < VEC; ++v) Ku[v] = p.Ku; }
        if (!UNI && p.alpha_cell) LV::ld(p.alpha_cell + i, al); else { for (int v = 0; v < VEC; ++v) al[v] = p.alpha; }
        if (!UNI && p.zw) LV::ld(p.zw + i, zw); else { for (int v = 0; v < VEC; ++v) zw[v] = (T)1; }
        if (p.hd) { LV::ld(p.hd + i, hdx); LV::ld(p.hd + N + i, hdy); LV::ld(p.hd + 2 * N + i, hdz); }
        else { for (int v = 0; v < VEC; ++v) { hdx[v] = 0; hdy[v] = 0; hdz[v] = 0; } }
        T kx[VEC], ky[VEC], kz[VEC];
        T hxo[VEC], hyo[VEC], hzo[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            T hx = 0, hy = 0, hz = 0, hex = 0, hey = 0, hez = 0, hax = 0, hay = 0, haz = 0, hzx = 0, hzy = 0, hzz = 0;
            T hdxv = 0, hdyv = 0, hdzv = 0, hmx = 0, hmy = 0, hmz = 0;
            if (UNI || Ms[v] != (T)0) {
                const bool uni = UNI || !p.Ms_cell;
                const T inv = uni ? (T)0 : (T)1 / Ms[v];
                const T cex = uni ? p.cex_u : (T)(2.0 / kMu0) * inv;
                hex = cex * sx[v]; hey = cex * sy_[v]; hez = cex * sz_[v];
                if constexpr (DMI) { hmx = cex * dmx[v]; hmy = cex * dmy[v]; hmz = cex * dmz[v]; }
                if (UNI ? (p.Ku != (T)0) : (Ku[v] != (T)0)) {
                    T ex = p.ex, ey = p.ey, ez = p.ez;
                    if (p.grain) {
                        const int gi = p.grain[i + v];
                        ex = p.axis_tab[3 * gi]; ey = p.axis_tab[3 * gi + 1]; ez = p.axis_tab[3 * gi + 2];
                    }
                    const T ck = (UNI || (uni && !p.Ku_cell)) ? p.cani_u : (T)(2.0 / kMu0) * Ku[v] * (uni ? (T)1 / Ms[v] : inv);
                    const T c = ck * (ex * mx[v] + ey * my[v] + ez * mz[v]);
                    hax = c * ex; hay = c * ey; haz = c * ez;
                }
                hzx = zw[v] * p.hx0; hzy = zw[v] * p.hy0; hzz = zw[v] * p.hz0;
                hdxv = hdx[v]; hdyv = hdy[v]; hdzv = hdz[v];
                hx = hdxv + hex + hax + hzx + hmx;
                hy = hdyv + hey + hay + hzy + hmy;
                hz = hdzv + hez + haz + hzz + hmz;
            }
            hxo[v] = hx; hyo[v] = hy; hzo[v] = hz;
            const T gp = (!UNI && p.alpha_cell) ? (T)(-kGamma) / ((T)1 + al[v] * al[v]) : p.gp_u;
            const T cx = my[v] * hz - mz[v] * hy, cy = mz[v] * hx - mx[v] * hz, cz = mx[v] * hy - my[v] * hx;
            const T dx_ = my[v] * cz - mz[v] * cy, dy_ = mz[v] * cx - mx[v] * cz, dz_ = mx[v] * cy - my[v] * cx;
            const T pc = p.no_precession ? (T)0 : (T)1;
            kx[v] = gp * (pc * cx + al[v] * dx_); ky[v] = gp * (pc * cy + al[v] * dy_);
            kz[v] = gp * (pc * cz + al[v] * dz_);
            if (!(isfinite(kx[v]) && isfinite(ky[v]) && isfinite(kz[v]))) red_nf = 1;
            if (p.want_torque && Ms[v] != (T)0) red_tq = fmax(red_tq, sqrt(cx * cx + cy * cy + cz * cz) / Ms[v]);
            if (p.want_energy && Ms[v] != (T)0) {
                const double f = -0.5 * kMu0 * (p.lvol ? p.lvol[z] : p.V) * (double)Ms[v];
                red_e0 += f * ((double)mx[v] * hdxv + (double)my[v] * hdyv + (double)mz[v] * hdzv);
                red_e1 += f * ((double)mx[v] * hex + (double)my[v] * hey + (double)mz[v] * hez);
                red_e2 += f * ((double)mx[v] * hax + (double)my[v] * hay + (double)mz[v] * haz);
                red_e3 += 2.0 * f * ((double)mx[v] * hzx + (double)my[v] * hzy + (double)mz[v] * hzz);
                if constexpr (DMI) red_e4 += f * ((double)mx[v] * hmx + (double)my[v] * hmy + (double)mz[v] * hmz);
            }
        }
        if (p.h_out) { LV::st(p.h_out + i, hxo); LV::st(p.h_out + N + i, hyo); LV::st(p.h_out + 2 * N + i, hzo); }
        if (p.k_out) { LV::st(p.k_out + i, kx); LV::st(p.k_out + N + i, ky); LV::st(p.k_out + 2 * N + i, kz); }
        if (p.acc_out) {
            T ax[VEC], ay[VEC], az[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) { ax[v] = p.acc_bT * kx[v]; ay[v] = p.acc_bT * ky[v]; az[v] = p.acc_bT * kz[v]; }
            if (p.acc_in) {
                T bx[VEC], by[VEC], bz[VEC];
                LV::ld(p.acc_in + i, bx); LV::ld(p.acc_in + N + i, by); LV::ld(p.acc_in + 2 * N + i, bz);
#pragma unroll
                for (int v = 0; v < VEC; ++v) { ax[v] += bx[v]; ay[v] += by[v]; az[v] += bz[v]; }
            }
            LV::st(p.acc_out + i, ax); LV::st(p.acc_out + N + i, ay); LV::st(p.acc_out + 2 * N + i, az);
        }
        if (p.next || p.want_err) {
            T snx[VEC], sny[VEC], snz[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) { snx[v] = p.ckT * kx[v]; sny[v] = p.ckT * ky[v]; snz[v] = p.ckT * kz[v]; }
            T ex_[VEC], ey_[VEC], ez_[VEC];
            if (p.want_err) {
#pragma unroll
                for (int v = 0; v < VEC; ++v) { ex_[v] = p.eb_kT * kx[v]; ey_[v] = p.eb_kT * ky[v]; ez_[v] = p.eb_kT * kz[v]; }
            }
            for (int q = 0; q < p.nk; ++q) {
                const T* kq = p.kin[q];
                T ax[VEC], ay[VEC], az[VEC];
                LV::ld(kq + i, ax); LV::ld(kq + N + i, ay); LV::ld(kq + 2 * N + i, az);
                const T c = p.kcT[q];
#pragma unroll
                for (int v = 0; v < VEC; ++v) { snx[v] += c * ax[v]; sny[v] += c * ay[v]; snz[v] += c * az[v]; }
                if (p.want_err) {
                    const T e = p.ebT[q];
#pragma unroll
                    for (int v = 0; v < VEC; ++v) { ex_[v] += e * ax[v]; ey_[v] += e * ay[v]; ez_[v] += e * az[v]; }
                }
            }
            T m0x[VEC], m0y[VEC], m0z[VEC];
            LV::ld(p.mn + i, m0x); LV::ld(p.mn + N + i, m0y); LV::ld(p.mn + 2 * N + i, m0z);
            if (p.want_err) {
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    // the solution the error is measured against: the stage input, or
                    // the combination this stage writes (before renormalisation)
                    const T ux = p.err_on_next ? m0x[v] + p.dtT * snx[v] : mx[v];
                    const T uy = p.err_on_next ? m0y[v] + p.dtT * sny[v] : my[v];
                    const T uz = p.err_on_next ? m0z[v] + p.dtT * snz[v] : mz[v];
                    const T scx = p.atolT + p.rtolT * fmax(fabs(m0x[v]), fabs(ux));
                    const T scy = p.atolT + p.rtolT * fmax(fabs(m0y[v]), fabs(uy));
                    const T scz = p.atolT + p.rtolT * fmax(fabs(m0z[v]), fabs(uz));
                    const T nx = fabs(p.dtT * ex_[v]), ny = fabs(p.dtT * ey_[v]), nz = fabs(p.dtT * ez_[v]);
                    if (!(isfinite(nx) && isfinite(ny) && isfinite(nz))) red_nf = 1;
                    if (nx * ed > en * scx) { en = nx; ed = scx; }
                    if (ny * ed > en * scy) { en = ny; ed = scy; }
                    if (nz * ed > en * scz) { en = nz; ed = scz; }
                }
            }
            if (p.next) {
                const T dt = p.dtT;
                T ox[VEC], oy[VEC], oz[VEC];
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    T a = m0x[v] + dt * snx[v], b = m0y[v] + dt * sny[v], c = m0z[v] + dt * snz[v];
                    if (p.renorm) {
                        const T n2 = a * a + b * b + c * c;
                        if (n2 > (T)0) {
                            const T s = (T)1 / sqrt(n2);
                            a *= s; b *= s; c *= s;
                        }
                    }
                    ox[v] = a; oy[v] = b; oz[v] = c;
                }
                LV::st(p.next + i, ox); LV::st(p.next + N + i, oy); LV::st(p.next + 2 * N + i, oz);
            }
        }
    }
    // ---- block reduction (all threads participate) ----
    if (p.partials) {
        // energies: FP64 sums; torque, error and the non-finite flag: maxima in
        // the state's precision, the error as a fraction divided once per block
        constexpr int NW = kStageThreads / 32;
        __shared__ double red[NW][kNPart];
        __shared__ T redt[NW][3];
        const int tid = threadIdx.y * kBX + threadIdx.x;
        const int lane = tid & 31, wid = tid >> 5;
        double vals[kNPart] = {0.0, red_e0, red_e1, red_e2, red_e3, 0.0, 0.0, red_e4};
        if (p.want_energy) {
#pragma unroll
            for (int q = R_EDEM; q <= R_EZEE; ++q) vals[q] = warp_sum(vals[q]);
            vals[R_EDMI] = warp_sum(vals[R_EDMI]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T n2 = __shfl_down_sync(0xffffffffu, en, o), d2 = __shfl_down_sync(0xffffffffu, ed, o);
            if (n2 * ed > en * d2) { en = n2; ed = d2; }
            red_tq = fmax(red_tq, __shfl_down_sync(0xffffffffu, red_tq, o));
        }
        const bool nf = __any_sync(0xffffffffu, red_nf);
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < kNPart; ++q) red[wid][q] = vals[q];
            red[wid][R_NONFINITE] = nf ? 1.0 : 0.0;
            redt[wid][0] = red_tq; redt[wid][1] = en; redt[wid][2] = ed;
        }
        __syncthreads();
        if (tid < kNPart) {
            const int q = tid;
            double acc = red[0][q];
            if (q == R_TORQUE || q == R_ERR) {
                T t = redt[0][0], n = redt[0][1], d = redt[0][2];
                for (int w = 1; w < NW; ++w) {
                    t = fmax(t, redt[w][0]);
                    if (redt[w][1] * d > n * redt[w][2]) { n = redt[w][1]; d = redt[w][2]; }
                }
                acc = q == R_TORQUE ? (double)t : (double)(n / d);
            } else {
                for (int w = 1; w < NW; ++w) acc = q == R_NONFINITE ? fmax(acc, red[w][q]) : acc + red[w][q];
            }
            const long b = ((long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
            p.partials[b * kNPart + q] = acc;
        }
    }
}

__global__ void __launch_bounds__(256) finalize_kernel(const double* __restrict__ partials, int nblocks,
                                                       double* __restrict__ scalars) {
    __shared__ double sm[256];
    for (int q = 0; q < kNPart; ++q) {
        const bool ismax = (q == R_TORQUE || q == R_ERR || q == R_NONFINITE);
        double acc = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += 256) {
            const double v = partials[(long)b * kNPart + q];
            acc = ismax ? fmax(acc, v) : acc + v;
        }
        sm[threadIdx.x] = acc;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                const double a = sm[threadIdx.x], b = sm[threadIdx.x + s];
                sm[threadIdx.x] = ismax ? fmax(a, b) : a + b;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) scalars[q] = sm[0];
        __syncthreads();
    }
}

template <typename T> __global__ void convert_kernel(const double* __restrict__ src, T* __restrict__ dst, long n) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (T)src[i];
}

template <typename T> __global__ void renorm_copy_kernel(const T* src, T* dst, long N) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        T a = src[i], b = src[N + i], c = src[2 * N + i];
        const T n2 = a * a + b * b + c * c;
        if (n2 > (T)0) {
            const T s = (T)1 / sqrt(n2);
            a *= s; b *= s; c *= s;
        }
        dst[i] = a; dst[N + i] = b; dst[2 * N + i] = c;
    }
}

template <typename T> struct CombineParams {
    const T* mn;
    const T* kin[7];
    double kc[7];
    int nk;
    double dt;
    T* out;
    long N;
};

// out = mn + dt sum_j kc_j kin_j  (a Runge-Kutta stage input without a field evaluation)
template <typename T> __global__ void combine_kernel(CombineParams<T> p) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * p.N) return;
    T acc = 0;
    for (int q = 0; q < p.nk; ++q) acc += (T)p.kc[q] * p.kin[q][i];
    p.out[i] = p.mn[i] + (T)p.dt * acc;
}

template <typename T> void launch_combine(const T* mn, const T* const* kin, const double* kc, int nk, double dt,
                                          T* out, long N, cudaStream_t st) {
    CombineParams<T> p;
    p.mn = mn;
    for (int q = 0; q < 7; ++q) { p.kin[q] = q < nk ? kin[q] : nullptr; p.kc[q] = q < nk ? kc[q] : 0.0; }
    p.nk = nk; p.dt = dt; p.out = out; p.N = N;
    combine_kernel<T><<<(unsigned)((3 * N + 255) / 256), 256, 0, st>>>(p);
}

template <typename T> int stage_vec(int nx);
template <> int stage_vec<float>(int nx) { return nx % 2 == 0 ? 2 : 1; }
template <> int stage_vec<double>(int nx) { return nx % 2 == 0 ? 2 : 1; }

// an upper bound on the blocks launch_stage uses (the scalar path has the most)
template <typename T> int stage_blocks(int nx, int ny, int nz) {
    const int gx = (nx + kBX - 1) / kBX;
    const int gy = (ny + kBY - 1) / kBY;
    return gx * gy * nz;
}

static bool al16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; }

// the vector path needs every per-cell array 16-byte aligned (caller buffers may be views)
template <typename T> static bool all_aligned(const StageParams<T>& p) {
    const void* ptrs[] = {p.m, p.hd, p.Ms_cell, p.A_cell, p.Ku_cell, p.alpha_cell, p.zw, p.h_out, p.k_out,
                          p.mn, p.next, p.acc_in, p.acc_out};
    for (const void* q : ptrs)
        if (!al16(q)) return false;
    for (int q = 0; q < p.nk; ++q)
        if (!al16(p.kin[q])) return false;
    return true;
}

template <typename T> void stage_prepare(StageParams<T>& p) {
    for (int q = 0; q < 7; ++q) p.kcT[q] = (T)p.kc[q];
    p.ckT = (T)p.ck;
    p.dtT = (T)p.dt;
    p.acc_bT = (T)p.acc_b;
    for (int q = 0; q < 7; ++q) p.ebT[q] = (T)p.eb[q];
    p.eb_kT = (T)p.eb_k;
    p.rtolT = (T)p.rtol;
    p.atolT = (T)p.atol;
    // uniform-material constants, computed once in double
    p.cex_u = p.Ms != (T)0 ? (T)(2.0 / kMu0 / (double)p.Ms) : (T)0;
    p.cani_u = p.Ms != (T)0 ? (T)(2.0 / kMu0 * (double)p.Ku / (double)p.Ms) : (T)0;
    p.gp_u = (T)(-kGamma / (1.0 + (double)p.alpha * (double)p.alpha));
}
template void stage_prepare<float>(StageParams<float>&);
template void stage_prepare<double>(StageParams<double>&);

template <typename T> void launch_stage(const StageParams<T>& p0, cudaStream_t st, int* nblocks) {
    StageParams<T> p = p0;
    stage_prepare(p);
    const int vec = all_aligned(p) ? stage_vec<T>(p.nx) : 1;
    dim3 block(kBX, kBY);
    dim3 grid((p.nx / vec + kBX - 1) / kBX, (p.ny + kBY - 1) / kBY, p.nz);
    *nblocks = (int)(grid.x * grid.y * grid.z);
    // uniform material needs Ms != 0 too (the Ms = 0 test is compiled away)
    const bool uni = !p.Ms_cell && !p.A_cell && !p.Ku_cell && !p.alpha_cell && !p.zw && p.Ms != (T)0;
    if (p.dmi) {
        // DMI runs the general (non-uniform) variant
        if (vec == 1) stage_kernel<T, 1, false, true><<<grid, block, 0, st>>>(p);
        else stage_kernel<T, 2, false, true><<<grid, block, 0, st>>>(p);
    } else if (vec == 1) {
        if (uni) stage_kernel<T, 1, true, false><<<grid, block, 0, st>>>(p);
        else stage_kernel<T, 1, false, false><<<grid, block, 0, st>>>(p);
    } else {
        if (uni) stage_kernel<T, 2, true, false><<<grid, block, 0, st>>>(p);
        else stage_kernel<T, 2, false, false><<<grid, block, 0, st>>>(p);
    }
}

void launch_finalize(const double* partials, int nblocks, double* scalars, cudaStream_t st) {
    finalize_kernel<<<1, 256, 0, st>>>(partials, nblocks, scalars);
}

template <typename T> void launch_convert(const double* src, T* dst, long n, cudaStream_t st) {
    if (n <= 0) return;
    convert_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, n);
}

template <typename T> void launch_renorm_copy(const T* src, T* dst, long N, cudaStream_t st) {
    renorm_copy_kernel<T><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(src, dst, N);
}

template int stage_blocks<float>(int, int, int);
template int stage_blocks<double>(int, int, int);
template void launch_stage<float>(const StageParams<float>&, cudaStream_t, int*);
template void launch_stage<double>(const StageParams<double>&, cudaStream_t, int*);
template void launch_convert<float>(const double*, float*, long, cudaStream_t);
template void launch_convert<double>(const double*, double*, long, cudaStream_t);
template void launch_combine<float>(const float*, const float* const*, const double*, int, double, float*, long,
                                    cudaStream_t);
template void launch_combine<double>(const double*, const double* const*, const double*, int, double, double*,
                                     long, cudaStream_t);
template void launch_renorm_copy<float>(const float*, float*, long, cudaStream_t);
template void launch_renorm_copy<double>(const double*, double*, long, cudaStream_t);

}  // namespace mm
