// Batched (served) relax path: parameters and launchers of csrc/batch.cu.
#pragma once

#include "demag.h"

namespace mm {

template <typename T> struct BatchStageParams {
    int nx, ny, nz, N, nb;
    T idx2, idy2, idz2;
    const T* Ms;              // [nb] per-grid material (device)
    const T* A;
    const T* alpha;
    // per grid (Sec. 4.3, Sec. 3): DMI kind (0 none, 1 interface, 2 bulk, 3 D2d)
    // with a uniform D, and the precession factor (1, or 0 without the m x h term)
    const int* dmi_kind;
    const T* D;
    const T* pc;
    T dmi_e[4][9];            // DMI vectors e_x, e_y, e_z of each kind
    T i2dx, i2dy, i2dz;       // 1 / (2 d) per axis
    const double* dt;         // [nb] per-grid step
    const int* mask;          // [nb] grids this launch works on
    T hx0, hy0, hz0;          // uniform external field
    const T* m;               // stage input [nb][3][N]
    const T* hd;              // demag field [nb][3][N]
    const T* mn;              // m at the start of the step
    T* k_out;
    T* next;                  // mn + dt (sum_j kc_j kin_j + ck k)
    const T* kin[7];
    // the stage and error coefficients in the state's precision: the error
    // norm and the torque are evaluated in it (FP64 is a narrow pipe on this
    // part, and an FP32 state's stage derivatives carry FP32 rounding anyway)
    T kc[7];
    int nk;
    T ck;
    int want_err, want_torque;
    T eb[7];
    T eb_k;
    T rtol;                   // atol = rtol
    double* partials;         // [nb][blocks per grid][3]
};

template <typename T> void launch_batch_stage(const BatchStageParams<T>& p, cudaStream_t st);
void launch_batch_finalize(const double* partials, int nblk, int nb, double* scalars, cudaStream_t st);
template <typename T> void launch_batch_combine(const T* m, const T* k, const double* dt, double a, const int* mask,
                                                T* out, int N, int nb, cudaStream_t st);
void launch_batch_masks(const int* status, const int* fresh, int* mask, int cap, cudaStream_t st);
void launch_batch_first(const double* scal, const int* fmask, int* status, int* fresh, double* torque, double tol,
                        int cap, cudaStream_t st);
void launch_batch_control(const double* scal, int* run, int* status, int* steps, double* dt, double* t,
                          double* torque, int* acc, double tol, int max_steps, int cap, cudaStream_t st);
template <typename T> void launch_batch_accept(const T* y5, const T* k7, const int* acc, T* m, T* k1, int N, int nb,
                                               cudaStream_t st);

}  // namespace mm
