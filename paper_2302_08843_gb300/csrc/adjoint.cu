// Hand-written discrete adjoint of one RK4 step (the gradient Sec. 5.2 gets
// from autograd), per cell, for the LLG right-hand side of Eq. llg:
//
//   f(m) = -g' [p m x h + a m x (m x h)],  h = H m + h_ext,  g' = gamma/(1+a^2),
//   p = 1 with the precession term, 0 without it (Sec. 3)
//   for a cotangent u of f:  v = p u + a (u x m),  w = v x m,  G = m x h
//   (df/dm)^T u  = -g' [h x v + a G x u + H^T w]
//   (df/dMs)^T u = -g' [m . hw - w . (h_ex + h_dmi + h_u) / Ms]      (per cell)
//
// with hw = -N * w (the demag convolution is symmetric and even, so its
// transpose is itself), H^T w = Ms hw + (2/mu0) (S + Q)(w/Ms) + h_u(w), S the
// exchange link sum (the exchange operator is diag(2/(mu0 Ms)) times a
// symmetric graph Laplacian), Q the DMI link sum (Sec. 4.3: cell i gets
// Dt e_k x m_{i+k} / (2 d) from each neighbour, with e_{-k} = -e_k, which
// makes Q symmetric too), h_u symmetric per cell.
#include "adjoint.h"

namespace mm {

template <typename T> __device__ __forceinline__ T hmean(T a, T b) {
    const T s = a + b;
    return s != (T)0 ? (T)2 * a * b / s : (T)0;
}

// Eq. D_avg as read (the forward field's link average): harmonic mean for
// equal signs, otherwise the geometric mean of the geometric and the
// arithmetic mean with the sign of the sum
template <typename T> __device__ __forceinline__ T adj_dmi_avg(T a, T b) {
    const T prod = a * b, s = a + b;
    if (prod >= (T)0) return s != (T)0 ? (T)2 * prod / s : (T)0;
    return copysign(sqrt(sqrt(-prod) * fabs(s) * (T)0.5), s);
}

// out += c e x (a, b, d)
template <typename T> __device__ __forceinline__ void adj_cross_add(const T* e, T c, T a, T b, T d, T& ox, T& oy,
                                                                    T& oz) {
    ox += c * (e[1] * d - e[2] * b);
    oy += c * (e[2] * a - e[0] * d);
    oz += c * (e[0] * b - e[1] * a);
}

template <typename T> __device__ __forceinline__ void axis_of(const AdjParams<T>& p, int i, T& ex, T& ey, T& ez) {
    ex = p.ex; ey = p.ey; ez = p.ez;
    if (p.grain) {
        const int g = p.grain[i];
        ex = p.axis_tab[3 * g]; ey = p.axis_tab[3 * g + 1]; ez = p.axis_tab[3 * g + 2];
    }
}

template <typename T> __global__ void adj_prep_kernel(AdjParams<T> p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    const int N = p.N;
    const T mx = p.m[i], my = p.m[N + i], mz = p.m[2 * N + i];
    const T hx = p.h[i], hy = p.h[N + i], hz = p.h[2 * N + i];
    const T ux = p.u[i], uy = p.u[N + i], uz = p.u[2 * N + i];
    const T Ms = p.Ms_cell ? p.Ms_cell[i] : p.Ms;
    const T al = p.alpha_cell ? p.alpha_cell[i] : p.alpha;
    const T gp = (T)kGamma / ((T)1 + al * al);
    // v = p u + a u x m ; w = v x m ; G = m x h
    const T vx = p.pc * ux + al * (uy * mz - uz * my), vy = p.pc * uy + al * (uz * mx - ux * mz),
            vz = p.pc * uz + al * (ux * my - uy * mx);
    const T wx = vy * mz - vz * my, wy = vz * mx - vx * mz, wz = vx * my - vy * mx;
    const T Gx = my * hz - mz * hy, Gy = mz * hx - mx * hz, Gz = mx * hy - my * hx;
    // h x v + a G x u
    const T px = (hy * vz - hz * vy) + al * (Gy * uz - Gz * uy);
    const T py = (hz * vx - hx * vz) + al * (Gz * ux - Gx * uz);
    const T pz = (hx * vy - hy * vx) + al * (Gx * uy - Gy * ux);
    const bool on = Ms != (T)0;
    p.w[i] = on ? wx : (T)0; p.w[N + i] = on ? wy : (T)0; p.w[2 * N + i] = on ? wz : (T)0;
    const T inv = on ? (T)1 / Ms : (T)0;
    p.q[i] = wx * inv; p.q[N + i] = wy * inv; p.q[2 * N + i] = wz * inv;
    p.part[i] = on ? -gp * px : (T)0;
    p.part[N + i] = on ? -gp * py : (T)0;
    p.part[2 * N + i] = on ? -gp * pz : (T)0;
}

template <typename T> __global__ void adj_finish_kernel(AdjParams<T> p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    const int N = p.N;
    const int x = i % p.nx, yz = i / p.nx, y = yz % p.ny, z = yz / p.ny;
    const T Ms = p.Ms_cell ? p.Ms_cell[i] : p.Ms;
    T lx = p.part[i], ly = p.part[N + i], lz = p.part[2 * N + i];
    if (Ms != (T)0) {
        const T inv = (T)1 / Ms;
        const T al = p.alpha_cell ? p.alpha_cell[i] : p.alpha;
        const T gp = (T)kGamma / ((T)1 + al * al);
        const T Ai = p.A_cell ? p.A_cell[i] : p.A;
        const T mx = p.m[i], my = p.m[N + i], mz = p.m[2 * N + i];
        const T qx = p.q[i], qy = p.q[N + i], qz = p.q[2 * N + i];
        T Sqx = 0, Sqy = 0, Sqz = 0, Smx = 0, Smy = 0, Smz = 0;
#define MM_ALINK(COND, OFF, ID2)                                                   \
        if (COND) {                                                                \
            const int k = i + (OFF);                                               \
            const T wl = (p.A_cell ? hmean(Ai, p.A_cell[k]) : p.A) * (ID2);        \
            Sqx += wl * (p.q[k] - qx); Sqy += wl * (p.q[N + k] - qy); Sqz += wl * (p.q[2 * N + k] - qz); \
            Smx += wl * (p.m[k] - mx); Smy += wl * (p.m[N + k] - my); Smz += wl * (p.m[2 * N + k] - mz); \
        }
        MM_ALINK(x > 0, -1, p.idx2)
        MM_ALINK(x < p.nx - 1, 1, p.idx2)
        MM_ALINK(y > 0, -p.nx, p.idy2)
        MM_ALINK(y < p.ny - 1, p.nx, p.idy2)
        MM_ALINK(z > 0, -p.nx * p.ny, p.idz2)
        MM_ALINK(z < p.nz - 1, p.nx * p.ny, p.idz2)
#undef MM_ALINK
        // DMI link sums Q q and Q m (the neighbour k's term is Dt e_k x v_k / (2 d), e_{-k} = -e_k)
        T Dqx = 0, Dqy = 0, Dqz = 0, Dmx = 0, Dmy = 0, Dmz = 0;
        if (p.dmi) {
            const T Di = p.D_cell ? p.D_cell[i] : p.D;
            auto dlink = [&](bool cond, int off, T sgn, const T* e, T i2d) {
                if (!cond) return;
                const int k = i + off;
                const T c = sgn * (p.D_cell ? adj_dmi_avg(Di, p.D_cell[k]) : p.D) * i2d;
                adj_cross_add(e, c, p.q[k], p.q[N + k], p.q[2 * N + k], Dqx, Dqy, Dqz);
                adj_cross_add(e, c, p.m[k], p.m[N + k], p.m[2 * N + k], Dmx, Dmy, Dmz);
            };
            dlink(x > 0, -1, (T)-1, &p.dmi_e[0], p.i2dx);
            dlink(x < p.nx - 1, 1, (T)1, &p.dmi_e[0], p.i2dx);
            dlink(y > 0, -p.nx, (T)-1, &p.dmi_e[3], p.i2dy);
            dlink(y < p.ny - 1, p.nx, (T)1, &p.dmi_e[3], p.i2dy);
            dlink(z > 0, -p.nx * p.ny, (T)-1, &p.dmi_e[6], p.i2dz);
            dlink(z < p.nz - 1, p.nx * p.ny, (T)1, &p.dmi_e[6], p.i2dz);
        }
        const T wx = p.w[i], wy = p.w[N + i], wz = p.w[2 * N + i];
        const T hwx = p.hw ? p.hw[i] : (T)0, hwy = p.hw ? p.hw[N + i] : (T)0, hwz = p.hw ? p.hw[2 * N + i] : (T)0;
        T ex, ey, ez;
        axis_of(p, i, ex, ey, ez);
        const T Ku = p.Ku_cell ? p.Ku_cell[i] : p.Ku;
        const T cu = (T)(2.0 / kMu0) * Ku * inv;
        const T ew = ex * wx + ey * wy + ez * wz, em = ex * mx + ey * my + ez * mz;
        const T c2 = (T)(2.0 / kMu0);
        // H^T w
        const T tx = Ms * hwx + c2 * (Sqx + Dqx) + cu * ew * ex;
        const T ty = Ms * hwy + c2 * (Sqy + Dqy) + cu * ew * ey;
        const T tz = Ms * hwz + c2 * (Sqz + Dqz) + cu * ew * ez;
        lx -= gp * tx; ly -= gp * ty; lz -= gp * tz;
        // d<w,h>/dMs = m.hw - w.(h_ex + h_dmi + h_u)/Ms
        const T hex = c2 * inv, hu = cu * em;
        const T wh = wx * (hex * (Smx + Dmx) + hu * ex) + wy * (hex * (Smy + Dmy) + hu * ey) +
                     wz * (hex * (Smz + Dmz) + hu * ez);
        const T dMs = (mx * hwx + my * hwy + mz * hwz) - wh * inv;
        if (p.gMs) p.gMs[i] += -gp * dMs;
    }
    p.part[i] = lx; p.part[N + i] = ly; p.part[2 * N + i] = lz;
    p.lam_acc[i] += lx; p.lam_acc[N + i] += ly; p.lam_acc[2 * N + i] += lz;
    if (p.u_prev) {
        p.u_prev[i] = p.cb * p.lam_y[i] + p.cc * lx;
        p.u_prev[N + i] = p.cb * p.lam_y[N + i] + p.cc * ly;
        p.u_prev[2 * N + i] = p.cb * p.lam_y[2 * N + i] + p.cc * lz;
    }
}

// lambda_y = (lambda - r (r . lambda)) / |y|, r = y/|y|; also lam_acc = lambda_y and
// u = dt b_last lambda_y (cotangent of the last stage derivative)
template <typename T> __global__ void adj_renorm_kernel(const T* __restrict__ y, const T* __restrict__ lam,
                                                        T* __restrict__ lam_y, T* __restrict__ lam_acc,
                                                        T* __restrict__ u, T cb, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const T a = y[i], b = y[N + i], c = y[2 * N + i];
    const T n2 = a * a + b * b + c * c;
    T lx = lam[i], ly = lam[N + i], lz = lam[2 * N + i];
    if (n2 > (T)0) {
        const T inv = (T)1 / sqrt(n2);
        const T rx = a * inv, ry = b * inv, rz = c * inv;
        const T d = rx * lx + ry * ly + rz * lz;
        lx = (lx - rx * d) * inv; ly = (ly - ry * d) * inv; lz = (lz - rz * d) * inv;
    }
    lam_y[i] = lx; lam_y[N + i] = ly; lam_y[2 * N + i] = lz;
    lam_acc[i] = lx; lam_acc[N + i] = ly; lam_acc[2 * N + i] = lz;
    u[i] = cb * lx; u[N + i] = cb * ly; u[2 * N + i] = cb * lz;
}

template <typename T>
void launch_adj_prep(const AdjParams<T>& p, cudaStream_t st) {
    adj_prep_kernel<T><<<(p.N + 255) / 256, 256, 0, st>>>(p);
}
template <typename T>
void launch_adj_finish(const AdjParams<T>& p, cudaStream_t st) {
    adj_finish_kernel<T><<<(p.N + 255) / 256, 256, 0, st>>>(p);
}
template <typename T>
void launch_adj_renorm(const T* y, const T* lam, T* lam_y, T* lam_acc, T* u, double cb, int N, cudaStream_t st) {
    adj_renorm_kernel<T><<<(N + 255) / 256, 256, 0, st>>>(y, lam, lam_y, lam_acc, u, (T)cb, N);
}

template void launch_adj_prep<float>(const AdjParams<float>&, cudaStream_t);
template void launch_adj_prep<double>(const AdjParams<double>&, cudaStream_t);
template void launch_adj_finish<float>(const AdjParams<float>&, cudaStream_t);
template void launch_adj_finish<double>(const AdjParams<double>&, cudaStream_t);
template void launch_adj_renorm<float>(const float*, const float*, float*, float*, float*, double, int, cudaStream_t);
template void launch_adj_renorm<double>(const double*, const double*, double*, double*, double*, double, int,
                                        cudaStream_t);

}  // namespace mm
