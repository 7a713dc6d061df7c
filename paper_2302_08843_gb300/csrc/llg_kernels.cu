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
__device__ __forceinline__ T link_weight(const T* A_cell, T A, T Ai, long nb) {
    if (!A_cell) return A;
    const T Aj = A_cell[nb];
    const T s = Ai + Aj;
    return s != (T)0 ? (T)2 * Ai * Aj / s : (T)0;
}

template <typename T>
__global__ void __launch_bounds__(kStageThreads) stage_kernel(StageParams<T> p) {
    const long N = p.N;
    const long i = (long)blockIdx.x * kStageThreads + threadIdx.x;
    double red_torque = 0.0, red_e[4] = {0.0, 0.0, 0.0, 0.0}, red_err = 0.0, red_nf = 0.0;
    if (i < N) {
        const int x = (int)(i % p.nx);
        const long yz = i / p.nx;
        const int y = (int)(yz % p.ny);
        const int z = (int)(yz / p.ny);
        const T* m = p.m;
        const T mx = m[i], my = m[N + i], mz = m[2 * N + i];
        const T Ms = p.Ms_cell ? p.Ms_cell[i] : p.Ms;
        T hx = 0, hy = 0, hz = 0;
        T hdx = 0, hdy = 0, hdz = 0, hex = 0, hey = 0, hez = 0, hax = 0, hay = 0, haz = 0;
        T hzx = 0, hzy = 0, hzz = 0;
        if (Ms != (T)0) {
            const T inv = (T)1 / Ms;
            const T Ai = p.A_cell ? p.A_cell[i] : p.A;
            T sx = 0, sy = 0, sz = 0;
            const long sxs = 1, sys = p.nx, szs = (long)p.nx * p.ny;
#define MM_LINK(COND, OFF, ID2)                                            \
            if (COND) {                                                    \
                const long nb = i + (OFF);                                 \
                const T w = link_weight<T>(p.A_cell, p.A, Ai, nb) * (ID2); \
                sx += w * (m[nb] - mx);                                    \
                sy += w * (m[N + nb] - my);                                \
                sz += w * (m[2 * N + nb] - mz);                            \
            }
            MM_LINK(x > 0, -sxs, p.idx2)
            MM_LINK(x < p.nx - 1, sxs, p.idx2)
            MM_LINK(y > 0, -sys, p.idy2)
            MM_LINK(y < p.ny - 1, sys, p.idy2)
            MM_LINK(z > 0, -szs, p.idz2)
            MM_LINK(z < p.nz - 1, szs, p.idz2)
#undef MM_LINK
            const T cex = (T)(2.0 / kMu0) * inv;
            hex = cex * sx; hey = cex * sy; hez = cex * sz;
            const T Ku = p.Ku_cell ? p.Ku_cell[i] : p.Ku;
            if (Ku != (T)0) {
                T ex = p.ex, ey = p.ey, ez = p.ez;
                if (p.grain) {
                    const int gi = p.grain[i];
                    ex = p.axis_tab[3 * gi]; ey = p.axis_tab[3 * gi + 1]; ez = p.axis_tab[3 * gi + 2];
                }
                const T c = (T)(2.0 / kMu0) * Ku * inv * (ex * mx + ey * my + ez * mz);
                hax = c * ex; hay = c * ey; haz = c * ez;
            }
            const T w = p.zw ? p.zw[i] : (T)1;
            hzx = w * p.hx0; hzy = w * p.hy0; hzz = w * p.hz0;
            if (p.hd) { hdx = p.hd[i]; hdy = p.hd[N + i]; hdz = p.hd[2 * N + i]; }
            hx = hdx + hex + hax + hzx;
            hy = hdy + hey + hay + hzy;
            hz = hdz + hez + haz + hzz;
        }
        if (p.h_out) { p.h_out[i] = hx; p.h_out[N + i] = hy; p.h_out[2 * N + i] = hz; }
        const T al = p.alpha_cell ? p.alpha_cell[i] : p.alpha;
        const T gp = (T)(-kGamma) / ((T)1 + al * al);
        const T cx = my * hz - mz * hy, cy = mz * hx - mx * hz, cz = mx * hy - my * hx;
        const T dx_ = my * cz - mz * cy, dy_ = mz * cx - mx * cz, dz_ = mx * cy - my * cx;
        const T kx = gp * (cx + al * dx_), ky = gp * (cy + al * dy_), kz = gp * (cz + al * dz_);
        if (!(isfinite(kx) && isfinite(ky) && isfinite(kz))) red_nf = 1.0;
        if (p.want_torque && Ms != (T)0)
            red_torque = sqrt((double)cx * cx + (double)cy * cy + (double)cz * cz) / (double)Ms;
        if (p.want_energy && Ms != (T)0) {
            const double f = -0.5 * kMu0 * p.V * (double)Ms;
            red_e[0] = f * ((double)mx * hdx + (double)my * hdy + (double)mz * hdz);
            red_e[1] = f * ((double)mx * hex + (double)my * hey + (double)mz * hez);
            red_e[2] = f * ((double)mx * hax + (double)my * hay + (double)mz * haz);
            red_e[3] = 2.0 * f * ((double)mx * hzx + (double)my * hzy + (double)mz * hzz);
        }
        if (p.k_out) { p.k_out[i] = kx; p.k_out[N + i] = ky; p.k_out[2 * N + i] = kz; }
        if (p.acc_out) {
            T ax = (T)p.acc_b * kx, ay = (T)p.acc_b * ky, az = (T)p.acc_b * kz;
            if (p.acc_in) { ax += p.acc_in[i]; ay += p.acc_in[N + i]; az += p.acc_in[2 * N + i]; }
            p.acc_out[i] = ax; p.acc_out[N + i] = ay; p.acc_out[2 * N + i] = az;
        }
        if (p.next || p.want_err) {
            T sxn = (T)p.ck * kx, syn = (T)p.ck * ky, szn = (T)p.ck * kz;
            double ex_ = p.eb_k * kx, ey_ = p.eb_k * ky, ez_ = p.eb_k * kz;
            for (int q = 0; q < p.nk; ++q) {
                const T* kq = p.kin[q];
                const T ax = kq[i], ay = kq[N + i], az = kq[2 * N + i];
                sxn += (T)p.kc[q] * ax; syn += (T)p.kc[q] * ay; szn += (T)p.kc[q] * az;
                if (p.want_err) { ex_ += p.eb[q] * ax; ey_ += p.eb[q] * ay; ez_ += p.eb[q] * az; }
            }
            const T m0x = p.mn[i], m0y = p.mn[N + i], m0z = p.mn[2 * N + i];
            if (p.want_err) {
                const double sc_x = p.atol + p.rtol * fmax(fabs((double)m0x), fabs((double)mx));
                const double sc_y = p.atol + p.rtol * fmax(fabs((double)m0y), fabs((double)my));
                const double sc_z = p.atol + p.rtol * fmax(fabs((double)m0z), fabs((double)mz));
                red_err = fmax(fmax(fabs(p.dt * ex_) / sc_x, fabs(p.dt * ey_) / sc_y), fabs(p.dt * ez_) / sc_z);
                if (!isfinite(red_err)) red_nf = 1.0;
            }
            if (p.next) {
                const T dt = (T)p.dt;
                T nx_ = m0x + dt * sxn, ny_ = m0y + dt * syn, nz_ = m0z + dt * szn;
                if (p.renorm) {
                    const T n2 = nx_ * nx_ + ny_ * ny_ + nz_ * nz_;
                    if (n2 > (T)0) {
                        const T s = (T)1 / sqrt(n2);
                        nx_ *= s; ny_ *= s; nz_ *= s;
                    }
                }
                p.next[i] = nx_; p.next[N + i] = ny_; p.next[2 * N + i] = nz_;
            }
        }
    }
    // ---- block reduction (all threads participate) ----
    if (p.partials) {
        __shared__ double red[kStageThreads / 32][kNPart];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        double vals[kNPart] = {red_torque, red_e[0], red_e[1], red_e[2], red_e[3], red_err, red_nf, 0.0};
        vals[R_TORQUE] = warp_max(vals[R_TORQUE]);
        vals[R_ERR] = warp_max(vals[R_ERR]);
        vals[R_NONFINITE] = warp_max(vals[R_NONFINITE]);
#pragma unroll
        for (int q = R_EDEM; q <= R_EZEE; ++q) vals[q] = warp_sum(vals[q]);
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < kNPart; ++q) red[wid][q] = vals[q];
        }
        __syncthreads();
        if (threadIdx.x < kNPart) {
            const int q = threadIdx.x;
            double acc = red[0][q];
            for (int w = 1; w < kStageThreads / 32; ++w) {
                const double v = red[w][q];
                acc = (q == R_TORQUE || q == R_ERR || q == R_NONFINITE) ? fmax(acc, v) : acc + v;
            }
            p.partials[(long)blockIdx.x * kNPart + q] = acc;
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

template <typename T> void launch_stage(const StageParams<T>& p, cudaStream_t st, int* nblocks) {
    const int nb = (int)((p.N + kStageThreads - 1) / kStageThreads);
    *nblocks = nb;
    stage_kernel<T><<<nb, kStageThreads, 0, st>>>(p);
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
