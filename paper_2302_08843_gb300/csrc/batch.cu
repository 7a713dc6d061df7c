// Kernels of the batched (served) relax path: nb grids of one shape stacked as
// a leading batch dimension ([b][3][nz][ny][nx]), each with its own uniform
// Ms, A, alpha and its own Dormand-Prince step size.  A request's arithmetic
// never mixes with another's (per-grid reductions in a fixed order), so its
// result does not depend on which other requests share the batch.
#include "batch.h"

namespace mm {

// out += e x w
template <typename T> __device__ __forceinline__ void bcross_add(const T* e, T wx, T wy, T wz, T& ox, T& oy, T& oz) {
    ox += e[1] * wz - e[2] * wy;
    oy += e[2] * wx - e[0] * wz;
    oz += e[0] * wy - e[1] * wx;
}

// one thread per cell, grid (ceil(N/256), nb); a masked-off grid does nothing
template <typename T> __global__ void __launch_bounds__(256) batch_stage_kernel(BatchStageParams<T> p) {
    const int b = blockIdx.y;
    if (!p.mask[b]) return;                       // uniform per block
    const int N = p.N;
    const int i = blockIdx.x * 256 + threadIdx.x;
    const long off = (long)b * 3 * N;
    // per thread: the largest |m x h|^2 (the torque's square; sqrt and 1/Ms are
    // monotone, so they are applied once per warp) and the largest error ratio
    // |dt e_c| / sc_c, kept as a fraction en / ed (cross-multiplied comparisons,
    // one division per warp)
    T tq2 = 0, en = 0, ed = 1;
    int nf = 0;
    if (i < N) {
        const int x = i % p.nx, yz = i / p.nx, y = yz % p.ny, z = yz / p.ny;
        const T* m = p.m + off;
        const T mx = m[i], my = m[N + i], mz = m[2 * N + i];
        const T Ms = p.Ms[b], A = p.A[b], al = p.alpha[b];
        T hx = 0, hy = 0, hz = 0, cx = 0, cy = 0, cz = 0;
        if (Ms != (T)0) {
            T sx = 0, sy = 0, sz = 0;
#define MM_BLINK(COND, OFF, ID2)                                              \
            if (COND) {                                                       \
                const int k = i + (OFF);                                      \
                const T w = A * (ID2);                                        \
                sx += w * (m[k] - mx); sy += w * (m[N + k] - my); sz += w * (m[2 * N + k] - mz); \
            }
            MM_BLINK(x > 0, -1, p.idx2)
            MM_BLINK(x < p.nx - 1, 1, p.idx2)
            MM_BLINK(y > 0, -p.nx, p.idy2)
            MM_BLINK(y < p.ny - 1, p.nx, p.idy2)
            MM_BLINK(z > 0, -p.nx * p.ny, p.idz2)
            MM_BLINK(z < p.nz - 1, p.nx * p.ny, p.idz2)
#undef MM_BLINK
            // DMI (Sec. 4.3), uniform D: sum over the axes of e_a x D (m_{i+a} - m_{i-a}) / (2 d_a),
            // a neighbour outside the grid left out; it enters h with the exchange sum's 2 / (mu0 Ms)
            const int kind = p.dmi_kind[b];
            if (kind) {
                const T* e = p.dmi_e[kind];
#define MM_BDMI(LO, HI, OFF, EA, I2D)                                                 \
                {                                                                     \
                    T wx = 0, wy = 0, wz = 0;                                         \
                    if (HI) { const int k = i + (OFF); wx += m[k]; wy += m[N + k]; wz += m[2 * N + k]; } \
                    if (LO) { const int k = i - (OFF); wx -= m[k]; wy -= m[N + k]; wz -= m[2 * N + k]; } \
                    const T c = p.D[b] * (I2D);                                       \
                    bcross_add(EA, c * wx, c * wy, c * wz, sx, sy, sz);               \
                }
                MM_BDMI(x > 0, x < p.nx - 1, 1, e, p.i2dx)
                MM_BDMI(y > 0, y < p.ny - 1, p.nx, e + 3, p.i2dy)
                MM_BDMI(z > 0, z < p.nz - 1, p.nx * p.ny, e + 6, p.i2dz)
#undef MM_BDMI
            }
            const T cex = (T)(2.0 / kMu0) / Ms;
            const T* hd = p.hd + off;
            hx = hd[i] + cex * sx + p.hx0;
            hy = hd[N + i] + cex * sy + p.hy0;
            hz = hd[2 * N + i] + cex * sz + p.hz0;
        }
        const T gp = (T)(-kGamma) / ((T)1 + al * al);
        cx = my * hz - mz * hy; cy = mz * hx - mx * hz; cz = mx * hy - my * hx;
        const T dx_ = my * cz - mz * cy, dy_ = mz * cx - mx * cz, dz_ = mx * cy - my * cx;
        const T pcf = p.pc[b];
        const T kx = gp * (pcf * cx + al * dx_), ky = gp * (pcf * cy + al * dy_), kz = gp * (pcf * cz + al * dz_);
        if (!(isfinite(kx) && isfinite(ky) && isfinite(kz))) nf = 1;
        if (p.want_torque && Ms != (T)0) tq2 = cx * cx + cy * cy + cz * cz;
        if (p.k_out) { T* ko = p.k_out + off; ko[i] = kx; ko[N + i] = ky; ko[2 * N + i] = kz; }
        if (p.next || p.want_err) {
            const T dt = (T)p.dt[b];
            T sxn = p.ck * kx, syn = p.ck * ky, szn = p.ck * kz;
            T ex_ = 0, ey_ = 0, ez_ = 0;
            if (p.want_err) { ex_ = p.eb_k * kx; ey_ = p.eb_k * ky; ez_ = p.eb_k * kz; }
            for (int q = 0; q < p.nk; ++q) {
                const T* kq = p.kin[q] + off;
                const T ax = kq[i], ay = kq[N + i], az = kq[2 * N + i];
                sxn += p.kc[q] * ax; syn += p.kc[q] * ay; szn += p.kc[q] * az;
                if (p.want_err) { ex_ += p.eb[q] * ax; ey_ += p.eb[q] * ay; ez_ += p.eb[q] * az; }
            }
            const T* mn = p.mn + off;
            const T m0x = mn[i], m0y = mn[N + i], m0z = mn[2 * N + i];
            if (p.want_err) {
                const T scx = p.rtol + p.rtol * fmax(fabs(m0x), fabs(mx));
                const T scy = p.rtol + p.rtol * fmax(fabs(m0y), fabs(my));
                const T scz = p.rtol + p.rtol * fmax(fabs(m0z), fabs(mz));
                const T nx = fabs(dt * ex_), ny = fabs(dt * ey_), nz = fabs(dt * ez_);
                if (!(isfinite(nx) && isfinite(ny) && isfinite(nz))) nf = 1;
                en = nx; ed = scx;
                if (ny * ed > en * scy) { en = ny; ed = scy; }
                if (nz * ed > en * scz) { en = nz; ed = scz; }
            }
            if (p.next) {
                T* nx_ = p.next + off;
                nx_[i] = m0x + dt * sxn; nx_[N + i] = m0y + dt * syn; nx_[2 * N + i] = m0z + dt * szn;
            }
        }
    }
    if (p.partials) {
        // maxima in the state's precision; the torque's sqrt and 1/Ms and the
        // error's division once per block
        __shared__ T red[8][3];
        __shared__ int rednf[8];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T n2 = __shfl_down_sync(0xffffffffu, en, o), d2 = __shfl_down_sync(0xffffffffu, ed, o);
            if (n2 * ed > en * d2) { en = n2; ed = d2; }
            tq2 = fmax(tq2, __shfl_down_sync(0xffffffffu, tq2, o));
        }
        const int anynf = __any_sync(0xffffffffu, nf);
        if (lane == 0) { red[wid][0] = tq2; red[wid][1] = en; red[wid][2] = ed; rednf[wid] = anynf; }
        __syncthreads();
        if (threadIdx.x == 0) {
            T t2 = red[0][0], n = red[0][1], d = red[0][2];
            int f = rednf[0];
            for (int w = 1; w < 8; ++w) {
                t2 = fmax(t2, red[w][0]);
                if (red[w][1] * d > n * red[w][2]) { n = red[w][1]; d = red[w][2]; }
                f |= rednf[w];
            }
            const T Ms = p.Ms[b];
            double* o = p.partials + ((long)b * gridDim.x + blockIdx.x) * 3;
            o[0] = Ms != (T)0 ? (double)(sqrt(t2) / Ms) : 0.0;
            o[1] = (double)(n / d);
            o[2] = f ? 1.0 : 0.0;
        }
    }
}

// per-grid maxima of the block partials: scalars[b][0..2] = (torque, err, nonfinite)
__global__ void batch_finalize_kernel(const double* __restrict__ partials, int nblk, double* __restrict__ scalars) {
    const int b = blockIdx.x;
    __shared__ double sm[3][128];
    for (int q = 0; q < 3; ++q) {
        double a = 0.0;
        for (int k = threadIdx.x; k < nblk; k += 128) a = fmax(a, partials[((long)b * nblk + k) * 3 + q]);
        sm[q][threadIdx.x] = a;
    }
    __syncthreads();
    for (int s = 64; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int q = 0; q < 3; ++q) sm[q][threadIdx.x] = fmax(sm[q][threadIdx.x], sm[q][threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x < 3) scalars[b * 3 + threadIdx.x] = sm[threadIdx.x][0];
}

// out[b] = m[b] + dt[b] a k[b] for masked grids
template <typename T> __global__ void batch_combine_kernel(const T* __restrict__ m, const T* __restrict__ k,
                                                           const double* __restrict__ dt, double a,
                                                           const int* __restrict__ mask, T* __restrict__ out, int n3) {
    const int b = blockIdx.y;
    if (!mask[b]) return;
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= n3) return;
    const long o = (long)b * n3 + i;
    out[o] = m[o] + (T)(dt[b] * a) * k[o];
}

// accepted grids: m[b] = y5[b] / |y5[b]|, k1[b] = k7[b]
template <typename T> __global__ void batch_accept_kernel(const T* __restrict__ y5, const T* __restrict__ k7,
                                                          const int* __restrict__ acc, T* __restrict__ m,
                                                          T* __restrict__ k1, int N) {
    const int b = blockIdx.y;
    if (!acc[b]) return;
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= N) return;
    const long o = (long)b * 3 * N;
    T a = y5[o + i], c = y5[o + N + i], e = y5[o + 2 * N + i];
    const T n2 = a * a + c * c + e * e;
    if (n2 > (T)0) {
        const T s = (T)1 / sqrt(n2);
        a *= s; c *= s; e *= s;
    }
    m[o + i] = a; m[o + N + i] = c; m[o + 2 * N + i] = e;
    k1[o + i] = k7[o + i]; k1[o + N + i] = k7[o + N + i]; k1[o + 2 * N + i] = k7[o + 2 * N + i];
}

// ---- device-side Dormand-Prince controller (one thread per slot) ----------
// Slot status: 0 empty, 1 running, 2 converged, 3 max steps, 4 failed.

// mask[0..cap): running and not yet evaluated; mask[cap..2cap): running
__global__ void batch_masks_kernel(const int* __restrict__ status, const int* __restrict__ fresh,
                                   int* __restrict__ mask, int cap) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) {
        const int run = status[i] == 1;
        mask[i] = run && fresh[i];
        mask[cap + i] = run;
    }
}

// after the first-stage evaluation of fresh slots: their initial torque (a
// slot already below tol converges without a step) or failure
__global__ void batch_first_kernel(const double* __restrict__ scal, const int* __restrict__ fmask,
                                   int* __restrict__ status, int* __restrict__ fresh, double* __restrict__ torque,
                                   double tol, int cap) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) {
        if (!fmask[i]) continue;
        fresh[i] = 0;
        const double tq = scal[3 * i], nf = scal[3 * i + 2];
        if (nf != 0.0 || !isfinite(tq)) { status[i] = 4; continue; }
        torque[i] = tq;
        if (tq < tol) status[i] = 2;
    }
}

// one attempt's outcome per running slot: accept (err <= 1) or reject, the
// next step size dt * min(5, max(0.2, 0.9 err^-1/5)), the time, the step count
// and the status; acc[i] selects the slots whose solution is taken, and the
// running mask is updated for the next attempt
__global__ void batch_control_kernel(const double* __restrict__ scal, int* __restrict__ run,
                                     int* __restrict__ status, int* __restrict__ steps, double* __restrict__ dt,
                                     double* __restrict__ t, double* __restrict__ torque, int* __restrict__ acc,
                                     double tol, int max_steps, int cap) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) {
        acc[i] = 0;
        if (!run[i]) continue;
        const double tq = scal[3 * i], err = scal[3 * i + 1], nf = scal[3 * i + 2];
        if (nf != 0.0 || !isfinite(err)) { status[i] = 4; run[i] = 0; continue; }
        const double f = err == 0.0 ? 5.0 : fmin(5.0, fmax(0.2, 0.9 * pow(err, -0.2)));
        if (err <= 1.0) {
            acc[i] = 1;
            t[i] += dt[i];
            steps[i] += 1;
            torque[i] = tq;
            dt[i] *= f;
            if (tq < tol) status[i] = 2;
            else if (steps[i] >= max_steps) status[i] = 3;
        } else {
            dt[i] *= f;
            if (!(dt[i] >= 1e-22)) status[i] = 4;
        }
        run[i] = status[i] == 1;
    }
}

void launch_batch_masks(const int* status, const int* fresh, int* mask, int cap, cudaStream_t st) {
    batch_masks_kernel<<<(cap + 127) / 128, 128, 0, st>>>(status, fresh, mask, cap);
}
void launch_batch_first(const double* scal, const int* fmask, int* status, int* fresh, double* torque, double tol,
                        int cap, cudaStream_t st) {
    batch_first_kernel<<<(cap + 127) / 128, 128, 0, st>>>(scal, fmask, status, fresh, torque, tol, cap);
}
void launch_batch_control(const double* scal, int* run, int* status, int* steps, double* dt, double* t,
                          double* torque, int* acc, double tol, int max_steps, int cap, cudaStream_t st) {
    batch_control_kernel<<<(cap + 127) / 128, 128, 0, st>>>(scal, run, status, steps, dt, t, torque, acc, tol,
                                                            max_steps, cap);
}

template <typename T> void launch_batch_stage(const BatchStageParams<T>& p, cudaStream_t st) {
    dim3 grid((p.N + 255) / 256, p.nb);
    batch_stage_kernel<T><<<grid, 256, 0, st>>>(p);
}
void launch_batch_finalize(const double* partials, int nblk, int nb, double* scalars, cudaStream_t st) {
    batch_finalize_kernel<<<nb, 128, 0, st>>>(partials, nblk, scalars);
}
template <typename T> void launch_batch_combine(const T* m, const T* k, const double* dt, double a, const int* mask,
                                                T* out, int N, int nb, cudaStream_t st) {
    dim3 grid((3 * N + 255) / 256, nb);
    batch_combine_kernel<T><<<grid, 256, 0, st>>>(m, k, dt, a, mask, out, 3 * N);
}
template <typename T> void launch_batch_accept(const T* y5, const T* k7, const int* acc, T* m, T* k1, int N, int nb,
                                               cudaStream_t st) {
    dim3 grid((N + 255) / 256, nb);
    batch_accept_kernel<T><<<grid, 256, 0, st>>>(y5, k7, acc, m, k1, N);
}

template void launch_batch_stage<float>(const BatchStageParams<float>&, cudaStream_t);
template void launch_batch_stage<double>(const BatchStageParams<double>&, cudaStream_t);
template void launch_batch_combine<float>(const float*, const float*, const double*, double, const int*, float*, int,
                                          int, cudaStream_t);
template void launch_batch_combine<double>(const double*, const double*, const double*, double, const int*, double*,
                                           int, int, cudaStream_t);
template void launch_batch_accept<float>(const float*, const float*, const int*, float*, float*, int, int,
                                         cudaStream_t);
template void launch_batch_accept<double>(const double*, const double*, const int*, double*, double*, int, int,
                                          cudaStream_t);

}  // namespace mm
