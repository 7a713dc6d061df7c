// Parameters of the adjoint kernels (csrc/adjoint.cu).
#pragma once

#include "demag.h"

namespace mm {

template <typename T> struct AdjParams {
    int nx, ny, nz;
    int N;
    T idx2, idy2, idz2;
    const T* Ms_cell; T Ms;
    const T* A_cell; T A;
    const T* Ku_cell; T Ku;
    const T* alpha_cell; T alpha;
    const uint8_t* grain; const T* axis_tab; T ex, ey, ez;
    const T* m;      // stage input m_s
    const T* h;      // total field at m_s
    const T* u;      // cotangent of k_s
    T* w;            // v x m
    T* q;            // w / Ms
    T* part;         // -g' [h x v + a G x u], then the full lambda_s
    const T* hw;     // -N * w
    T* lam_acc;      // += lambda_s
    T* gMs;          // += (df/dMs)^T u
    T* u_prev;       // dt b_{s-1} lambda_y + dt c_s lambda_s (null for the first stage)
    const T* lam_y;
    T cb, cc;        // dt b_{s-1}, dt c_s
    T pc;            // 1 with the precession term of Eq. llg, 0 without it
    // DMI (Sec. 4.3): on, uniform D or per-cell D_cell (links averaged as in
    // the forward field), the DMI vectors e_x, e_y, e_z and 1 / (2 d) per axis
    int dmi;
    const T* D_cell; T D;
    T dmi_e[9];
    T i2dx, i2dy, i2dz;
};

}  // namespace mm
