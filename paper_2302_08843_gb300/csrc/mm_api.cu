// C ABI of libmm.so (declarations and contracts in include/mm.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <map>
#include <vector>

#include "adjoint.h"
#include "batch.h"
#include "demag.h"
#include "mm.h"
#include "tensor_host.h"

using namespace mm;

namespace {

thread_local char g_err[512] = "no error";   // fixed storage: reporting an error allocates nothing

mm_status fail(mm_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

#define MM_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? MM_ENOMEM : MM_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);               \
    } while (0)

#define MM_LAUNCHED()                                                                     \
    do {                                                                                  \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess)                                                            \
            return fail(MM_ECUDA, "kernel launch: %s (%s:%d)", cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define MM_TRY(expr)                     \
    do {                                 \
        mm_status s_ = (expr);           \
        if (s_ != MM_OK) return s_;      \
    } while (0)


std::mutex g_tw_mu;
bool g_tw_done[128] = {false};
double2 g_tw_host64[kMaxFft];    // static host staging: the upload allocates nothing
float2 g_tw_host32[kMaxFft];
double2 g_tw5_host64[kTw5];
float2 g_tw5_host32[kTw5];

}  // namespace

namespace mm {
void set_last_error(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

// Upload the FFT twiddle table to the current device once (no allocation).
cudaError_t ensure_twiddles_on(int dev) {
    std::lock_guard<std::mutex> lk(g_tw_mu);
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    if (g_tw_done[dev]) return cudaSuccess;
    static bool built = false;
    if (!built) {
        for (int i = 0; i < kMaxFft; ++i) {
            double c, sn;
            twiddle_entry(kMaxFft, i, &c, &sn);
            g_tw_host64[i] = make_double2(c, sn);
            g_tw_host32[i] = make_float2((float)c, (float)sn);
        }
        for (int i = 0; i < kTw5; ++i) {
            double c, sn;
            twiddle_entry(kTw5, i, &c, &sn);
            g_tw5_host64[i] = make_double2(c, sn);
            g_tw5_host32[i] = make_float2((float)c, (float)sn);
        }
        built = true;
    }
    cudaError_t e = upload_twiddles(g_tw_host64, g_tw_host32, g_tw5_host64, g_tw5_host32);
    if (e == cudaSuccess) e = upload_twiddles_rt();
    if (e == cudaSuccess) g_tw_done[dev] = true;
    return e;
}
}  // namespace mm

namespace {

mm_status ensure_twiddles(int dev) {
    cudaError_t e = ensure_twiddles_on(dev);
    if (e != cudaSuccess) return fail(MM_ECUDA, "twiddle upload: %s", cudaGetErrorString(e));
    return MM_OK;
}

}  // namespace

// --------------------------------------------------------------- timer ----
namespace mm {
void KernelTimer::begin(cudaStream_t st, const char* name) {
    if (!on) return;
    int id = -1;
    for (size_t i = 0; i < names.size(); ++i)
        if (names[i] == name) { id = (int)i; break; }
    if (id < 0) { names.emplace_back(name); id = (int)names.size() - 1; }
    while (pool.size() < used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { on = false; return; }
        pool.push_back(e);
    }
    cur = id;
    cur_a = pool[used++];
    cudaEventRecord(cur_a, st);
}
void KernelTimer::end(cudaStream_t st) {
    if (!on || cur < 0) return;
    cudaEvent_t b = pool[used++];
    cudaEventRecord(b, st);
    recs.push_back({cur, cur_a, b});
    cur = -1;
}
void KernelTimer::reset() {
    recs.clear();
    used = 0;
    cur = -1;
}
void KernelTimer::destroy() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
    recs.clear();
    used = 0;
}
}  // namespace mm

// --------------------------------------------------------------- state ----
struct mm_state {
    mm_grid g{};
    mm_precision prec = MM_FP64;
    cudaStream_t st = nullptr;
    int device = 0;
    DemagDims d{};
    long N = 0;
    size_t rsz = 8;          // sizeof(real)
    size_t csz = 16;         // sizeof(complex)
    // device buffers
    void* m = nullptr;       // 3N, the state's magnetisation
    void* mA = nullptr;      // 3N stage inputs (ping)
    void* mB = nullptr;      // 3N stage inputs (pong)
    void* acc = nullptr;     // 3N RK4 weighted sum
    void* hd = nullptr;      // 3N demag field
    void* S1 = nullptr;      // 3 ny nz KXS complex
    void* S2 = nullptr;      // 3 nz Py KXS complex (Py > 1)
    void* tens = nullptr;    // 6 KZ2 KY2 KXS real
    void* K[7] = {nullptr};  // DP45 stage derivatives
    void* adj[19] = {nullptr};  // adjoint: 3 stage inputs, 4 fields, 4 derivatives, y, lambda_y, 2 u, w, q, hw, part
    void* Ms_cell = nullptr;
    void* A_cell = nullptr;
    void* Ku_cell = nullptr;
    void* alpha_cell = nullptr;
    void* axis_tab = nullptr;
    uint8_t* grain = nullptr;
    void* zw = nullptr;
    double* partials = nullptr;
    int part_cap = 0;
    double* scalars = nullptr;     // device kNPart
    int* dev_err = nullptr;        // device error word written by bounded waits
    double* h_scalars = nullptr;   // pinned host kNPart
    // material and field
    double Ms = 0, A = 0, Ku = 0, alpha = 0, axis[3] = {1, 0, 0};
    double h0[3] = {0, 0, 0};
    mm_field_fn fn = nullptr;
    void* user = nullptr;
    bool have_m = false, have_mat = false, demag_ready = false, demag_off = false;
    bool fsal = false;             // K[0] holds the DP45 first stage of the next step
    bool k1_exact = false;         // K[0] = f(m, t) at the current m (RKF45 needs exactly that)
    int precession = 1;            // 0: LLG without the m x h term
    int dmi_kind = 0;              // mm_dmi_kind
    double D = 0.0;                // uniform DMI strength (J/m^2), used when D_cell is null
    void* D_cell = nullptr;        // per-cell DMI strength (real type)
    mm_method relax_method = MM_DP45;
    bool s1_fresh = false;   // S1 holds the x-spectrum of Ms m for the current m (left by the fused RK4 path)
    bool use_fused = true;   // RK4 in FP32 may take the fused stage kernel
    // non-equidistant layers: thicknesses (host), per-layer coefficients
    // (3 nz of the real type, StageParams::lay) and cell volumes (nz doubles)
    std::vector<double> lay_h;
    void* lay_t = nullptr;
    double* lay_v = nullptr;
    KernelTimer timer;
};

namespace {

mm_status dev_alloc(void** p, size_t bytes) {
    if (bytes == 0) { *p = nullptr; return MM_OK; }
    MM_CUDA(cudaMalloc(p, bytes));
    return MM_OK;
}

void dev_free(void*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

mm_status check_state(const mm_state* s) {
    if (!s) return fail(MM_EINVAL, "null state");
    return MM_OK;
}

mm_status set_device(const mm_state* s) {
    MM_CUDA(cudaSetDevice(s->device));
    return MM_OK;
}

mm_status ensure_partials(mm_state* s, int nblocks) {
    if (nblocks <= s->part_cap) return MM_OK;
    dev_free(reinterpret_cast<void*&>(s->partials));
    MM_TRY(dev_alloc(reinterpret_cast<void**>(&s->partials), sizeof(double) * kNPart * (size_t)nblocks));
    s->part_cap = nblocks;
    return MM_OK;
}

// upload a per-cell (or small) double array into a device buffer of the state's real type
mm_status upload_real(mm_state* s, const double* src, long n, int on_device, void** dst) {
    dev_free(*dst);
    if (!src) return MM_OK;
    MM_TRY(dev_alloc(dst, s->rsz * (size_t)n));
    if (on_device) {
        if (s->prec == MM_FP64) {
            MM_CUDA(cudaMemcpyAsync(*dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->st));
        } else {
            launch_convert<float>(src, (float*)*dst, n, s->st);
            MM_LAUNCHED();
        }
    } else {
        if (s->prec == MM_FP64) {
            MM_CUDA(cudaMemcpyAsync(*dst, src, sizeof(double) * n, cudaMemcpyHostToDevice, s->st));
            MM_CUDA(cudaStreamSynchronize(s->st));
        } else {
            std::vector<float> tmp(n);
            for (long i = 0; i < n; ++i) tmp[i] = (float)src[i];
            MM_CUDA(cudaMemcpyAsync(*dst, tmp.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s->st));
            MM_CUDA(cudaStreamSynchronize(s->st));
        }
    }
    return MM_OK;
}

mm_status ready_for_fields(const mm_state* s) {
    if (!s->have_mat) return fail(MM_ENOTSETUP, "mm_set_material has not been called");
    if (!s->demag_ready && !s->demag_off) return fail(MM_ENOTSETUP, "mm_demag_setup has not been called");
    return MM_OK;
}

void zeeman_at(const mm_state* s, double t, double h[3]) {
    if (s->fn) {
        s->fn(t, h, s->user);
    } else {
        h[0] = s->h0[0]; h[1] = s->h0[1]; h[2] = s->h0[2];
    }
}

// DMI vectors e_x, e_y, e_z of the paper's table per mm_dmi_kind (e_{-k} = -e_k; Sec. 4.3)
const double kDmiVectors[4][9] = {{0, 0, 0, 0, 0, 0, 0, 0, 0},
                                  {0, 1, 0, -1, 0, 0, 0, 0, 0},     // interface
                                  {1, 0, 0, 0, 1, 0, 0, 0, 1},      // bulk
                                  {-1, 0, 0, 0, 1, 0, 0, 0, 0}};    // D2d

template <typename T> void fill_common(const mm_state* s, StageParams<T>& p, const void* m, double t) {
    std::memset(&p, 0, sizeof(p));
    p.nx = s->g.nx; p.ny = s->g.ny; p.nz = s->g.nz;
    p.N = s->N;
    p.V = s->g.dx * s->g.dy * s->g.dz;
    p.idx2 = (T)(1.0 / (s->g.dx * s->g.dx));
    p.idy2 = (T)(1.0 / (s->g.dy * s->g.dy));
    p.idz2 = (T)(1.0 / (s->g.dz * s->g.dz));
    p.m = (const T*)m;
    p.hd = s->demag_off ? nullptr : (const T*)s->hd;
    p.Ms_cell = (const T*)s->Ms_cell; p.Ms = (T)s->Ms;
    p.A_cell = (const T*)s->A_cell; p.A = (T)s->A;
    p.Ku_cell = (const T*)s->Ku_cell; p.Ku = (T)s->Ku;
    p.alpha_cell = (const T*)s->alpha_cell; p.alpha = (T)s->alpha;
    p.grain = s->grain; p.axis_tab = (const T*)s->axis_tab;
    p.ex = (T)s->axis[0]; p.ey = (T)s->axis[1]; p.ez = (T)s->axis[2];
    p.zw = (const T*)s->zw;
    double h[3];
    zeeman_at(s, t, h);
    p.hx0 = (T)h[0]; p.hy0 = (T)h[1]; p.hz0 = (T)h[2];
    p.mn = (const T*)s->m;
    p.no_precession = s->precession ? 0 : 1;
    p.i2dx = (T)(0.5 / s->g.dx); p.i2dy = (T)(0.5 / s->g.dy); p.i2dz = (T)(0.5 / s->g.dz);
    if (!s->lay_h.empty()) {
        p.lay = (const T*)s->lay_t;
        p.lvol = s->lay_v;
    }
    if (s->dmi_kind != MM_DMI_NONE && (s->D != 0.0 || s->D_cell)) {
        p.dmi = 1;
        p.D = (T)s->D;
        p.D_cell = (const T*)s->D_cell;
        for (int q = 0; q < 9; ++q) p.dmi_e[q] = (T)kDmiVectors[s->dmi_kind][q];
    }
}

// demag field of m into s->hd
template <typename T> mm_status run_demag(mm_state* s, const void* m) {
    s->s1_fresh = false;
    if (s->demag_off) return MM_OK;
    using C = typename Cplx<T>::type;
    demag_apply<T>(s->d, (const T*)m, (const T*)s->Ms_cell, (T)s->Ms, (C*)s->S1, (C*)s->S2, (const T*)s->tens,
                   (T*)s->hd, s->st, &s->timer);
    MM_LAUNCHED();
    return MM_OK;
}

template <typename T> mm_status run_stage(mm_state* s, StageParams<T>& p, bool reduce) {
    const int nb = stage_blocks<T>(s->g.nx, s->g.ny, s->g.nz);
    if (reduce) {
        MM_TRY(ensure_partials(s, nb));
        p.partials = s->partials;
    } else {
        p.partials = nullptr;
    }
    int nblocks = 0;
    s->timer.begin(s->st, "stage_llg");
    launch_stage<T>(p, s->st, &nblocks);
    s->timer.end(s->st);
    MM_LAUNCHED();
    if (reduce) {
        s->timer.begin(s->st, "finalize_reduce");
        launch_finalize(s->partials, nblocks, s->scalars, s->st);
        s->timer.end(s->st);
        MM_LAUNCHED();
    }
    return MM_OK;
}

mm_status read_scalars(mm_state* s) {
    MM_CUDA(cudaMemcpyAsync(s->h_scalars, s->scalars, sizeof(double) * kNPart, cudaMemcpyDeviceToHost, s->st));
    int derr = 0;
    MM_CUDA(cudaMemcpyAsync(&derr, s->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s->st));
    MM_CUDA(cudaStreamSynchronize(s->st));
    if (derr != 0) return fail(MM_ETIMEOUT, "a bounded device-side wait gave up (code %d)", derr);
    return MM_OK;
}

template <typename T>
mm_status heff_impl(mm_state* s, const void* m, void* h_out, double* E_out, double t, double* torque_out) {
    MM_TRY(ready_for_fields(s));
    if (!m && !s->have_m) return fail(MM_ENOTSETUP, "no magnetisation: call mm_set_m or pass m");
    const void* mm_ = m ? m : s->m;
    MM_TRY(run_demag<T>(s, mm_));
    StageParams<T> p;
    fill_common<T>(s, p, mm_, t);
    p.h_out = (T*)h_out;
    p.want_energy = E_out != nullptr;
    p.want_torque = torque_out != nullptr;
    const bool reduce = E_out || torque_out;
    MM_TRY(run_stage<T>(s, p, reduce));
    if (reduce) {
        MM_TRY(read_scalars(s));
        if (E_out) {
            for (int q = 0; q < 4; ++q) E_out[q] = s->h_scalars[R_EDEM + q];
            E_out[4] = s->h_scalars[R_EDMI];
        }
        if (torque_out) *torque_out = s->h_scalars[R_TORQUE];
        if (s->h_scalars[R_NONFINITE] != 0.0) return fail(MM_ENONFINITE, "non-finite field or torque");
    }
    return MM_OK;
}

// k = f(m, t) (Eq. llg with the field of Sec. 4) into k_out.  FP32 states whose
// RK4 steps take the fused kernel take it here too (x-forward, y/z/y passes,
// fused x-inverse + local terms + LLG with the stage derivative as its
// accumulator output), so the derivative is the one those steps use.
template <typename T> mm_status rhs_impl(mm_state* s, const void* m, void* k_out, double t) {
    MM_TRY(ready_for_fields(s));
    if (!m && !s->have_m) return fail(MM_ENOTSETUP, "no magnetisation: call mm_set_m or pass m");
    const void* mm_ = m ? m : s->m;
    if constexpr (sizeof(T) == 4) {
        StageParams<float> p;
        fill_common<float>(s, p, mm_, t);
        if (s->use_fused && !s->demag_off && s->demag_ready && fused_stage_supported(s->d, p)) {
            demag_front<float>(s->d, (const float*)mm_, (const float*)s->Ms_cell, (float)s->Ms, true,
                               (float2*)s->S1, (float2*)s->S2, (const float*)s->tens, s->st, &s->timer);
            MM_LAUNCHED();
            p.hd = nullptr;
            p.dt = 0.0;
            p.next = (float*)s->mB;       // a stage buffer, free between steps
            p.acc_in = nullptr;
            p.acc_out = (float*)k_out;
            p.acc_b = 1.0;
            p.ck = 0.0;
            stage_prepare(p);
            if (!fused_stage(s->d, (float2*)s->S1, p, s->st, &s->timer))
                return fail(MM_ECUDA, "fused stage kernel could not be launched for this grid");
            MM_LAUNCHED();
            s->s1_fresh = false;
            return MM_OK;
        }
    }
    MM_TRY(run_demag<T>(s, mm_));
    StageParams<T> p;
    fill_common<T>(s, p, mm_, t);
    p.k_out = (T*)k_out;
    return run_stage<T>(s, p, false);
}

const double kRK4_C[4] = {0.0, 0.5, 0.5, 1.0};

// RK4 through the fused x-inverse + stage + x-forward kernel (FP32, uniform material)
mm_status rk4_fused(mm_state* s, double dt, double t, bool* used) {
    *used = false;
    const double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    const double anext[3] = {0.5, 0.5, 1.0};
    void* in[4] = {s->m, s->mA, s->mB, s->mA};
    void* out[4] = {s->m, s->mA, s->mB, s->mA};
    out[0] = s->mA; out[1] = s->mB; out[2] = s->mA; out[3] = s->m;
    StageParams<float> probe;
    fill_common<float>(s, probe, s->m, t);
    if (s->demag_off || !s->demag_ready || !fused_stage_supported(s->d, probe)) return MM_OK;
    for (int st = 0; st < 4; ++st) {
        demag_front<float>(s->d, (const float*)in[st], (const float*)s->Ms_cell, (float)s->Ms,
                           st == 0 && !s->s1_fresh, (float2*)s->S1, (float2*)s->S2, (const float*)s->tens, s->st,
                           &s->timer);
        MM_LAUNCHED();
        StageParams<float> p;
        fill_common<float>(s, p, in[st], t + kRK4_C[st] * dt);
        p.hd = nullptr;
        p.dt = dt;
        p.next = (float*)out[st];
        if (st < 3) {
            p.acc_in = st == 0 ? nullptr : (const float*)s->acc;
            p.acc_out = (float*)s->acc;
            p.acc_b = b[st];
            p.ck = anext[st];
        } else {
            p.kin[0] = (const float*)s->acc;
            p.kc[0] = 1.0;
            p.nk = 1;
            p.ck = b[3];
            p.renorm = 1;
        }
        stage_prepare(p);
        if (!fused_stage(s->d, (float2*)s->S1, p, s->st, &s->timer))
            return fail(MM_ECUDA, "fused stage kernel could not be launched for this grid");
        MM_LAUNCHED();
    }
    s->s1_fresh = true;
    s->fsal = s->k1_exact = false;
    *used = true;
    return MM_OK;
}

template <typename T> mm_status rk4_impl(mm_state* s, double dt, double t) {
    if constexpr (sizeof(T) == 4) {
        if (s->use_fused) {
            bool used = false;
            MM_TRY(rk4_fused(s, dt, t, &used));
            if (used) return MM_OK;
        }
    }
    const double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    const double anext[3] = {0.5, 0.5, 1.0};
    void* in[4] = {s->m, s->mA, s->mB, s->mA};
    void* out[4] = {s->mA, s->mB, s->mA, s->m};
    for (int st = 0; st < 4; ++st) {
        MM_TRY(run_demag<T>(s, in[st]));
        StageParams<T> p;
        fill_common<T>(s, p, in[st], t + kRK4_C[st] * dt);
        p.dt = dt;
        p.next = (T*)out[st];
        if (st < 3) {
            p.acc_in = st == 0 ? nullptr : (const T*)s->acc;
            p.acc_out = (T*)s->acc;
            p.acc_b = b[st];
            p.ck = anext[st];
        } else {
            p.kin[0] = (const T*)s->acc;
            p.kc[0] = 1.0;
            p.nk = 1;
            p.ck = b[3];
            p.renorm = 1;
        }
        MM_TRY(run_stage<T>(s, p, false));
    }
    s->fsal = s->k1_exact = false;
    return MM_OK;
}

// Dormand-Prince 5(4) tableau (Dormand & Prince 1980)
const double kDP_C[7] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0};
const double kDP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0},
    {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0}};
const double kDP_B5[7] = {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0, 0.0};
const double kDP_B4[7] = {5179.0 / 57600.0, 0.0, 7571.0 / 16695.0, 393.0 / 640.0, -92097.0 / 339200.0,
                          187.0 / 2100.0, 1.0 / 40.0};

mm_status ensure_dp_buffers(mm_state* s) {
    for (int q = 0; q < 7; ++q)
        if (!s->K[q]) MM_TRY(dev_alloc(&s->K[q], 3 * s->rsz * (size_t)s->N));
    return MM_OK;
}

// k1 = f(m, t) into K[0]; optional torque readback
template <typename T> mm_status dp_first_stage(mm_state* s, double t, double* torque) {
    MM_TRY(run_demag<T>(s, s->m));
    StageParams<T> p;
    fill_common<T>(s, p, s->m, t);
    p.k_out = (T*)s->K[0];
    p.want_torque = torque != nullptr;
    MM_TRY(run_stage<T>(s, p, torque != nullptr));
    if (torque) {
        MM_TRY(read_scalars(s));
        *torque = s->h_scalars[R_TORQUE];
        if (s->h_scalars[R_NONFINITE] != 0.0) return fail(MM_ENONFINITE, "non-finite field or torque");
    }
    s->fsal = true;
    s->k1_exact = true;
    return MM_OK;
}

// one DP45 attempt with step dt; fills err, torque (at y5) and leaves y5 in *y5buf
template <typename T>
mm_status dp_attempt(mm_state* s, double t, double dt, double rtol, double* err, double* torque, void** y5buf) {
    // y2 = m + dt a21 k1
    const T* k0 = (const T*)s->K[0];
    launch_combine<T>((const T*)s->m, &k0, &kDP_A[1][0], 1, dt, (T*)s->mA, s->N, s->st);
    MM_LAUNCHED();
    void* ybuf[2] = {s->mA, s->mB};
    int cur = 0;
    for (int st = 1; st <= 6; ++st) {     // stage st computes K[st] from y_{st+1} (0-based K)
        void* yin = ybuf[cur];
        MM_TRY(run_demag<T>(s, yin));
        StageParams<T> p;
        fill_common<T>(s, p, yin, t + kDP_C[st] * dt);
        p.dt = dt;
        p.k_out = (T*)s->K[st];
        if (st < 6) {
            p.next = (T*)ybuf[1 - cur];
            for (int q = 0; q < st; ++q) { p.kin[q] = (const T*)s->K[q]; p.kc[q] = kDP_A[st + 1][q]; }
            p.nk = st;
            p.ck = kDP_A[st + 1][st];
            MM_TRY(run_stage<T>(s, p, false));
            cur = 1 - cur;
        } else {
            // last stage: k7 = f(y7), error estimate, torque at y7
            for (int q = 0; q < 6; ++q) { p.kin[q] = (const T*)s->K[q]; p.eb[q] = kDP_B5[q] - kDP_B4[q]; }
            p.nk = 6;
            p.eb_k = kDP_B5[6] - kDP_B4[6];
            p.want_err = 1;
            p.rtol = rtol;
            p.atol = rtol;
            p.want_torque = 1;
            MM_TRY(run_stage<T>(s, p, true));
            *y5buf = yin;
        }
    }
    MM_TRY(read_scalars(s));
    *err = s->h_scalars[R_ERR];
    *torque = s->h_scalars[R_TORQUE];
    if (s->h_scalars[R_NONFINITE] != 0.0 || !std::isfinite(*err))
        return fail(MM_ENONFINITE, "non-finite values in a DP45 stage");
    return MM_OK;
}

template <typename T>
mm_status adjoint_impl(mm_state* s, const void* m_n, const void* lam_np1, void* lam_n, void* gMs, double dt,
                       double t) {
    const double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    for (int q = 0; q < 19; ++q)
        if (!s->adj[q]) MM_TRY(dev_alloc(&s->adj[q], 3 * s->rsz * (size_t)s->N));
    T** A = reinterpret_cast<T**>(s->adj);
    T* const* Am = A;          // stage inputs m_2..m_4
    T* const* Ah = A + 3;      // fields at the four stage inputs
    T* const* Ak = A + 7;      // stage derivatives
    T* Ay = A[11];
    T* Aly = A[12];
    T* Au[2] = {A[13], A[14]};
    T* Aw = A[15];
    T* Aq = A[16];
    T* Ahw = A[17];
    T* Apart = A[18];
    const T* ms[4] = {(const T*)m_n, Am[0], Am[1], Am[2]};
    // forward recompute of the stage inputs, fields and derivatives
    for (int st = 0; st < 4; ++st) {
        MM_TRY(run_demag<T>(s, ms[st]));
        StageParams<T> p;
        fill_common<T>(s, p, ms[st], t + kRK4_C[st] * dt);
        p.mn = (const T*)m_n;
        p.h_out = Ah[st];
        p.k_out = Ak[st];
        p.dt = dt;
        if (st < 3) {
            p.next = Am[st];
            p.ck = kRK4_C[st + 1];
        }
        MM_TRY(run_stage<T>(s, p, false));
    }
    const T* kin[4] = {Ak[0], Ak[1], Ak[2], Ak[3]};
    launch_combine<T>((const T*)m_n, kin, b, 4, dt, Ay, s->N, s->st);
    MM_LAUNCHED();
    launch_adj_renorm<T>(Ay, (const T*)lam_np1, Aly, (T*)lam_n, Au[0], dt * b[3], (int)s->N, s->st);
    MM_LAUNCHED();
    int cur = 0;
    for (int st = 3; st >= 0; --st) {
        AdjParams<T> p;
        std::memset(&p, 0, sizeof(p));
        p.nx = s->g.nx; p.ny = s->g.ny; p.nz = s->g.nz; p.N = (int)s->N;
        p.idx2 = (T)(1.0 / (s->g.dx * s->g.dx));
        p.idy2 = (T)(1.0 / (s->g.dy * s->g.dy));
        p.idz2 = (T)(1.0 / (s->g.dz * s->g.dz));
        p.Ms_cell = (const T*)s->Ms_cell; p.Ms = (T)s->Ms;
        p.A_cell = (const T*)s->A_cell; p.A = (T)s->A;
        p.Ku_cell = (const T*)s->Ku_cell; p.Ku = (T)s->Ku;
        p.alpha_cell = (const T*)s->alpha_cell; p.alpha = (T)s->alpha;
        p.grain = s->grain; p.axis_tab = (const T*)s->axis_tab;
        p.ex = (T)s->axis[0]; p.ey = (T)s->axis[1]; p.ez = (T)s->axis[2];
        p.m = ms[st];
        p.h = Ah[st];
        p.u = Au[cur];
        p.w = Aw; p.q = Aq; p.part = Apart;
        p.hw = s->demag_off ? nullptr : Ahw;
        p.lam_acc = (T*)lam_n;
        p.gMs = (T*)gMs;
        p.u_prev = st > 0 ? Au[1 - cur] : nullptr;
        p.lam_y = Aly;
        p.cb = st > 0 ? (T)(dt * b[st - 1]) : (T)0;
        p.cc = (T)(dt * kRK4_C[st]);
        p.pc = s->precession ? (T)1 : (T)0;
        {
            StageParams<T> fp;     // the forward field's DMI settings
            fill_common<T>(s, fp, ms[st], t);
            p.dmi = fp.dmi;
            p.D_cell = fp.D_cell; p.D = fp.D;
            for (int q = 0; q < 9; ++q) p.dmi_e[q] = fp.dmi_e[q];
            p.i2dx = fp.i2dx; p.i2dy = fp.i2dy; p.i2dz = fp.i2dz;
        }
        launch_adj_prep<T>(p, s->st);
        MM_LAUNCHED();
        if (!s->demag_off) {
            // transpose of the demag map applied to w: the same convolution with Ms = 1
            s->s1_fresh = false;
            demag_apply<T>(s->d, Aw, nullptr, (T)1, (typename Cplx<T>::type*)s->S1,
                           (typename Cplx<T>::type*)s->S2, (const T*)s->tens, Ahw, s->st, &s->timer);
            MM_LAUNCHED();
        }
        launch_adj_finish<T>(p, s->st);
        MM_LAUNCHED();
        cur = 1 - cur;
    }
    return MM_OK;
}

double dp_factor(double err) {
    if (err == 0.0) return 5.0;
    return std::min(5.0, std::max(0.2, 0.9 * std::pow(err, -0.2)));
}

template <typename T>
mm_status dp_step(mm_state* s, double* dt_inout, double rtol, double* t_inout, double* torque_out) {
    MM_TRY(ensure_dp_buffers(s));
    if (!s->fsal) MM_TRY(dp_first_stage<T>(s, *t_inout, nullptr));
    double dt = *dt_inout;
    for (;;) {
        if (!(dt >= 1e-22)) return fail(MM_ESTEP, "DP45 step size underflow (dt = %g s)", dt);
        double err = 0, tq = 0;
        void* y5 = nullptr;
        MM_TRY(dp_attempt<T>(s, *t_inout, dt, rtol, &err, &tq, &y5));
        const double f = dp_factor(err);
        if (err <= 1.0) {
            launch_renorm_copy<T>((const T*)y5, (T*)s->m, s->N, s->st);
            MM_LAUNCHED();
            std::swap(s->K[0], s->K[6]);    // first same as last
            s->fsal = true;
            s->k1_exact = false;            // f(y5) before renormalisation
            *t_inout += dt;
            *dt_inout = dt * f;
            if (torque_out) *torque_out = tq;
            return MM_OK;
        }
        dt *= f;
    }
}

// Runge-Kutta-Fehlberg 4(5) (E. Fehlberg, NASA TR R-315, 1969): six stages,
// the fourth-order solution propagated, the fifth-order one for the error
const double kRKF_C[6] = {0.0, 1.0 / 4.0, 3.0 / 8.0, 12.0 / 13.0, 1.0, 1.0 / 2.0};
const double kRKF_A[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0 / 4.0, 0, 0, 0, 0},
    {3.0 / 32.0, 9.0 / 32.0, 0, 0, 0},
    {1932.0 / 2197.0, -7200.0 / 2197.0, 7296.0 / 2197.0, 0, 0},
    {439.0 / 216.0, -8.0, 3680.0 / 513.0, -845.0 / 4104.0, 0},
    {-8.0 / 27.0, 2.0, -3544.0 / 2565.0, 1859.0 / 4104.0, -11.0 / 40.0}};
const double kRKF_B4[6] = {25.0 / 216.0, 0.0, 1408.0 / 2565.0, 2197.0 / 4104.0, -1.0 / 5.0, 0.0};
const double kRKF_B5[6] = {16.0 / 135.0, 0.0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0, 2.0 / 55.0};

// one attempt from (m, t) with K[0] = f(m, t): K[1..5], the fourth-order y4
// (returned in *y4buf, not renormalised) and the error norm against it
template <typename T>
mm_status rkf_attempt(mm_state* s, double t, double dt, double rtol, double* err, void** y4buf) {
    const T* k0 = (const T*)s->K[0];
    launch_combine<T>((const T*)s->m, &k0, &kRKF_A[1][0], 1, dt, (T*)s->mA, s->N, s->st);
    MM_LAUNCHED();
    void* ybuf[2] = {s->mA, s->mB};
    int cur = 0;
    for (int st = 1; st <= 5; ++st) {     // stage st computes K[st] from y_{st+1}
        void* yin = ybuf[cur];
        MM_TRY(run_demag<T>(s, yin));
        StageParams<T> p;
        fill_common<T>(s, p, yin, t + kRKF_C[st] * dt);
        p.dt = dt;
        p.k_out = (T*)s->K[st];
        p.next = (T*)ybuf[1 - cur];
        if (st < 5) {
            for (int q = 0; q < st; ++q) { p.kin[q] = (const T*)s->K[q]; p.kc[q] = kRKF_A[st + 1][q]; }
            p.nk = st;
            p.ck = kRKF_A[st + 1][st];
            MM_TRY(run_stage<T>(s, p, false));
        } else {
            // last stage: k6, y4 = m + dt sum b4 k, error sum (b5 - b4) k against y4
            for (int q = 0; q < 5; ++q) {
                p.kin[q] = (const T*)s->K[q];
                p.kc[q] = kRKF_B4[q];
                p.eb[q] = kRKF_B5[q] - kRKF_B4[q];
            }
            p.nk = 5;
            p.ck = kRKF_B4[5];
            p.eb_k = kRKF_B5[5] - kRKF_B4[5];
            p.want_err = 1;
            p.err_on_next = 1;
            p.rtol = rtol;
            p.atol = rtol;
            MM_TRY(run_stage<T>(s, p, true));
            *y4buf = ybuf[1 - cur];
        }
        cur = 1 - cur;
    }
    MM_TRY(read_scalars(s));
    *err = s->h_scalars[R_ERR];
    if (s->h_scalars[R_NONFINITE] != 0.0 || !std::isfinite(*err))
        return fail(MM_ENONFINITE, "non-finite values in an RKF45 stage");
    return MM_OK;
}

// attempts until one is accepted (same accept rule and step-size factor as DP45)
template <typename T>
mm_status rkf_step(mm_state* s, double* dt_inout, double rtol, double* t_inout) {
    MM_TRY(ensure_dp_buffers(s));
    if (!s->k1_exact) MM_TRY(dp_first_stage<T>(s, *t_inout, nullptr));
    double dt = *dt_inout;
    for (;;) {
        if (!(dt >= 1e-22)) return fail(MM_ESTEP, "RKF45 step size underflow (dt = %g s)", dt);
        double err = 0;
        void* y4 = nullptr;
        MM_TRY(rkf_attempt<T>(s, *t_inout, dt, rtol, &err, &y4));
        const double f = dp_factor(err);
        if (err <= 1.0) {
            launch_renorm_copy<T>((const T*)y4, (T*)s->m, s->N, s->st);
            MM_LAUNCHED();
            s->fsal = s->k1_exact = false;
            *t_inout += dt;
            *dt_inout = dt * f;
            return MM_OK;
        }
        dt *= f;
    }
}

}  // namespace

// ================================================================ batch ====
struct mm_batch {
    mm_grid g{};
    mm_precision prec = MM_FP32_FIELDS;
    cudaStream_t st = nullptr;
    int device = 0;
    int cap = 0;
    long N = 0;
    size_t rsz = 4, csz = 8;
    DemagDims d{};
    void* m = nullptr;
    void* K[7] = {nullptr};
    void* Y[2] = {nullptr};
    void* hd = nullptr;
    void* S1 = nullptr;
    void* S2 = nullptr;
    void* tens = nullptr;
    void* Ms_d = nullptr;
    void* A_d = nullptr;
    void* alpha_d = nullptr;
    // per-slot field terms (mm_batch_set_slot_terms): DMI D, precession factor, DMI kind
    void* D_d = nullptr;
    void* pc_d = nullptr;
    int* kind_d = nullptr;
    std::vector<char> unstarted;   // loaded and not yet in an mm_batch_begin
    // per-slot controller state, on the device: status, steps, fresh, dt, t, torque
    int* ctl_i = nullptr;        // [3][cap] ints
    double* ctl_d = nullptr;     // [3][cap] doubles
    int* mask_d = nullptr;       // [2][cap]: first-stage mask, running mask
    int* acc_d = nullptr;
    double* partials = nullptr;
    int nblk = 0;
    double* scal_d = nullptr;    // [2][cap][3]: first stage, attempt
    int* rep_i = nullptr;        // pinned report: status, steps
    double* rep_d = nullptr;     // pinned report: torque
    cudaEvent_t done = nullptr;  // recorded after the report copy of mm_batch_begin
    int y5 = 0;                  // which Y buffer holds an attempt's fifth-order solution
    int nact = 0;                // slots [0, nact) are launched (highest running slot + 1)
    bool pending = false;
    bool fresh_any = false;
    std::vector<int> status;     // host mirror of the last report
    // cached CUDA graphs of `attempts` consecutive attempts, per (nact, attempts)
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
    double g_rtol = -1, g_tol = -1;
    int g_max_steps = -1;

    int* status_d() { return ctl_i; }
    int* steps_d() { return ctl_i + cap; }
    int* fresh_d() { return ctl_i + 2 * cap; }
    double* dt_d() { return ctl_d; }
    double* t_d() { return ctl_d + cap; }
    double* torque_d() { return ctl_d + 2 * cap; }
};

namespace {

size_t batch_bytes(const mm_grid* g, mm_precision prec, int cap, int* LXo, int* LYo, int* LZo, int* KXSo) {
    const int LX = fft_extent(g->nx), LY = fft_extent(g->ny), LZ = fft_extent(g->nz);
    const size_t rsz = prec == MM_FP64 ? 8 : 4, csz = 2 * rsz;
    const int align = (int)(128 / csz);
    const int KX = LX / 2 + 1, KXS = (KX + align - 1) / align * align;
    const size_t N = (size_t)g->nx * g->ny * g->nz;
    size_t bytes = (size_t)cap * 3 * N * rsz * (1 + 7 + 2 + 1);               // m, K, Y, hd
    bytes += (size_t)cap * 3 * csz * g->ny * g->nz * KXS;                       // S1
    if (LY > 1) bytes += (size_t)cap * 3 * csz * g->nz * LY * KXS;              // S2
    bytes += 6 * rsz * (size_t)(LZ / 2 + 1) * (LY / 2 + 1) * KXS;               // tensor
    const size_t nblk = (N + 255) / 256;
    bytes += (size_t)cap * (2 * nblk * 3 * 8 + 5 * rsz + 4 + 3 * 4 + 3 * 8 + 2 * 4 + 4 + 2 * 3 * 8);
    if (LXo) { *LXo = LX; *LYo = LY; *LZo = LZ; *KXSo = KXS; }
    return bytes;
}

template <typename T> mm_status batch_stage(mm_batch* b, const void* m, const void* mn, void* k_out, void* next,
                                            const int* mask, int st, bool err, bool torque, double* partials,
                                            double rtol) {
    BatchStageParams<T> p;
    std::memset(&p, 0, sizeof(p));
    p.nx = b->g.nx; p.ny = b->g.ny; p.nz = b->g.nz; p.N = (int)b->N; p.nb = b->nact;
    p.idx2 = (T)(1.0 / (b->g.dx * b->g.dx));
    p.idy2 = (T)(1.0 / (b->g.dy * b->g.dy));
    p.idz2 = (T)(1.0 / (b->g.dz * b->g.dz));
    p.Ms = (const T*)b->Ms_d; p.A = (const T*)b->A_d; p.alpha = (const T*)b->alpha_d;
    p.dmi_kind = b->kind_d; p.D = (const T*)b->D_d; p.pc = (const T*)b->pc_d;
    for (int k = 0; k < 4; ++k)
        for (int q = 0; q < 9; ++q) p.dmi_e[k][q] = (T)kDmiVectors[k][q];
    p.i2dx = (T)(0.5 / b->g.dx); p.i2dy = (T)(0.5 / b->g.dy); p.i2dz = (T)(0.5 / b->g.dz);
    p.dt = b->dt_d();
    p.mask = mask;
    p.m = (const T*)m; p.hd = (const T*)b->hd; p.mn = (const T*)mn;
    p.k_out = (T*)k_out; p.next = (T*)next;
    if (st >= 1 && st <= 6) {
        if (st < 6) {
            for (int q = 0; q < st; ++q) { p.kin[q] = (const T*)b->K[q]; p.kc[q] = kDP_A[st + 1][q]; }
            p.nk = st;
            p.ck = kDP_A[st + 1][st];
        } else {
            for (int q = 0; q < 6; ++q) { p.kin[q] = (const T*)b->K[q]; p.eb[q] = kDP_B5[q] - kDP_B4[q]; }
            p.nk = 6;
            p.eb_k = kDP_B5[6] - kDP_B4[6];
        }
    }
    p.want_err = err;
    p.want_torque = torque;
    p.partials = partials;
    p.rtol = rtol;
    launch_batch_stage<T>(p, b->st);
    MM_LAUNCHED();
    return MM_OK;
}

template <typename T> mm_status batch_demag(mm_batch* b, const void* m) {
    using C = typename Cplx<T>::type;
    KernelTimer off;
    demag_apply<T>(b->d, (const T*)m, nullptr, (T)0, (C*)b->S1, (C*)b->S2, (const T*)b->tens, (T*)b->hd, b->st, &off);
    MM_LAUNCHED();
    return MM_OK;
}

// first-stage derivative k1 = f(m) and initial torque of newly loaded slots
template <typename T> mm_status batch_first(mm_batch* b, double rtol, double tol) {
    const int cap = b->cap;
    launch_batch_masks(b->status_d(), b->fresh_d(), b->mask_d, cap, b->st);
    MM_LAUNCHED();
    MM_TRY(batch_demag<T>(b, b->m));
    MM_TRY(batch_stage<T>(b, b->m, b->m, b->K[0], nullptr, b->mask_d, 0, false, true, b->partials, rtol));
    launch_batch_finalize(b->partials, b->nblk, b->nact, b->scal_d, b->st);
    MM_LAUNCHED();
    launch_batch_first(b->scal_d, b->mask_d, b->status_d(), b->fresh_d(), b->torque_d(), tol, cap, b->st);
    MM_LAUNCHED();
    return MM_OK;
}

// `attempts` DP45 attempts of every running slot, all decisions on the device
template <typename T> mm_status batch_attempts(mm_batch* b, int attempts, double rtol, double tol, int max_steps) {
    const int cap = b->cap;
    int* run = b->mask_d + cap;
    double* p1 = b->partials + (size_t)cap * b->nblk * 3;
    launch_batch_masks(b->status_d(), b->fresh_d(), b->mask_d, cap, b->st);
    MM_LAUNCHED();
    for (int a = 0; a < attempts; ++a) {
        launch_batch_combine<T>((const T*)b->m, (const T*)b->K[0], b->dt_d(), kDP_A[1][0], run, (T*)b->Y[0],
                                (int)b->N, b->nact, b->st);
        MM_LAUNCHED();
        int cur = 0;
        for (int st = 1; st <= 6; ++st) {
            MM_TRY(batch_demag<T>(b, b->Y[cur]));
            if (st < 6) {
                MM_TRY(batch_stage<T>(b, b->Y[cur], b->m, b->K[st], b->Y[1 - cur], run, st, false, false, nullptr,
                                      rtol));
                cur = 1 - cur;
            } else {
                MM_TRY(batch_stage<T>(b, b->Y[cur], b->m, b->K[6], nullptr, run, 6, true, true, p1, rtol));
                b->y5 = cur;
            }
        }
        launch_batch_finalize(p1, b->nblk, b->nact, b->scal_d + 3 * cap, b->st);
        MM_LAUNCHED();
        launch_batch_control(b->scal_d + 3 * cap, run, b->status_d(), b->steps_d(), b->dt_d(), b->t_d(),
                             b->torque_d(), b->acc_d, tol, max_steps, cap, b->st);
        MM_LAUNCHED();
        launch_batch_accept<T>((const T*)b->Y[b->y5], (const T*)b->K[6], b->acc_d, (T*)b->m, (T*)b->K[0],
                               (int)b->N, b->nact, b->st);
        MM_LAUNCHED();
    }
    return MM_OK;
}

void batch_drop_graphs(mm_batch* b) {
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

template <typename T>
mm_status batch_begin_impl(mm_batch* b, int attempts, double rtol, double tol, int max_steps) {
    const int cap = b->cap;
    int nrun = 0, hi = 0;
    for (int i = 0; i < cap; ++i)
        if (b->status[i] == 1) { ++nrun; hi = i + 1; }
    b->pending = true;                         // the report copy below is always enqueued
    if (nrun) {
        // grids past the highest running slot are not launched at all; the
        // masked ones below it cost one early-exiting block per tile
        b->nact = hi;
        b->d.nb = hi;
        if (b->fresh_any) {
            MM_TRY(batch_first<T>(b, rtol, tol));
            b->fresh_any = false;
        }
        if (rtol != b->g_rtol || tol != b->g_tol || max_steps != b->g_max_steps) {
            batch_drop_graphs(b);
            b->g_rtol = rtol; b->g_tol = tol; b->g_max_steps = max_steps;
        }
        const auto key = std::make_pair(hi, attempts);
        auto it = b->graphs.find(key);
        cudaGraphExec_t exec = it == b->graphs.end() ? nullptr : it->second;
        if (!exec) {
            // capture once; a stream that cannot be captured (the legacy
            // default stream) gets the same launches directly
            cudaGraph_t graph = nullptr;
            if (b->st && cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                const mm_status cs = batch_attempts<T>(b, attempts, rtol, tol, max_steps);
                const cudaError_t ce = cudaStreamEndCapture(b->st, &graph);
                if (cs != MM_OK || ce != cudaSuccess) {
                    if (graph) cudaGraphDestroy(graph);
                    cudaGetLastError();
                    return cs != MM_OK ? cs : fail(MM_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
                }
                const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
                cudaGraphDestroy(graph);
                if (ie != cudaSuccess) return fail(MM_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
                b->graphs[key] = exec;
            } else {
                cudaGetLastError();
                MM_TRY(batch_attempts<T>(b, attempts, rtol, tol, max_steps));
            }
        }
        if (exec) MM_CUDA(cudaGraphLaunch(exec, b->st));
    }
    MM_CUDA(cudaMemcpyAsync(b->rep_i, b->ctl_i, sizeof(int) * 2 * cap, cudaMemcpyDeviceToHost, b->st));
    MM_CUDA(cudaMemcpyAsync(b->rep_d, b->torque_d(), sizeof(double) * cap, cudaMemcpyDeviceToHost, b->st));
    MM_CUDA(cudaEventRecord(b->done, b->st));
    return MM_OK;
}

}  // namespace

// ================================================================= ABI ====
extern "C" {

const char* mm_last_error(void) { return g_err; }

const char* mm_version(void) { return "libmm 0.1 (sm_103a)"; }

mm_status mm_state_create(const mm_grid* grid, mm_precision precision, void* cuda_stream, mm_state** out) {
    if (!grid || !out) return fail(MM_EINVAL, "null argument");
    *out = nullptr;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return fail(MM_EINVAL, "grid sizes must be >= 1");
    if (!(grid->dx > 0) || !(grid->dy > 0) || !(grid->dz > 0)) return fail(MM_EINVAL, "cell sizes must be > 0");
    if ((double)grid->nx * grid->ny * grid->nz >= 2147483648.0) return fail(MM_EINVAL, "too many cells");
    if (precision != MM_FP64 && precision != MM_FP32_FIELDS) return fail(MM_EINVAL, "bad precision");
    const int LX = fft_extent(grid->nx), LY = fft_extent(grid->ny), LZ = fft_extent(grid->nz);
    if (LX > kMaxFft || LY > kMaxFft || LZ > kMaxFft)
        return fail(MM_EINVAL, "padded FFT extent above %d (grid %d x %d x %d)", kMaxFft, grid->nx, grid->ny,
                    grid->nz);
    mm_state* s = new (std::nothrow) mm_state();
    if (!s) return fail(MM_ENOMEM, "host allocation");
    s->g = *grid;
    s->prec = precision;
    s->st = (cudaStream_t)cuda_stream;
    s->rsz = precision == MM_FP64 ? sizeof(double) : sizeof(float);
    s->csz = 2 * s->rsz;
    s->N = (long)grid->nx * grid->ny * grid->nz;
    const int align = (int)(128 / s->csz);      // 128-byte rows
    const int KX = LX / 2 + 1;
    s->d = DemagDims{grid->nx, grid->ny, grid->nz, LX, LY, LZ, KX, (KX + align - 1) / align * align};
    auto bail = [&](mm_status st) { mm_state_destroy(s); return st; };
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) return bail(fail(MM_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e)));
    mm_status st = ensure_twiddles(s->device);
    if (st != MM_OK) return bail(st);
    const size_t v3 = 3 * s->rsz * (size_t)s->N;
    const size_t s1 = 3 * s->csz * (size_t)grid->ny * grid->nz * s->d.KXS;
    const size_t s2 = LY > 1 ? 3 * s->csz * (size_t)grid->nz * LY * s->d.KXS : 0;
    void** bufs[5] = {&s->m, &s->mA, &s->mB, &s->acc, &s->hd};
    for (void** b : bufs)
        if ((st = dev_alloc(b, v3)) != MM_OK) return bail(st);
    if ((st = dev_alloc(&s->S1, s1)) != MM_OK) return bail(st);
    if ((st = dev_alloc(&s->S2, s2)) != MM_OK) return bail(st);
    if ((st = dev_alloc(reinterpret_cast<void**>(&s->scalars), sizeof(double) * kNPart)) != MM_OK) return bail(st);
    if ((st = dev_alloc(reinterpret_cast<void**>(&s->dev_err), sizeof(int))) != MM_OK) return bail(st);
    s->d.err = s->dev_err;
    e = cudaMallocHost(reinterpret_cast<void**>(&s->h_scalars), sizeof(double) * kNPart);
    if (e != cudaSuccess) return bail(fail(MM_ENOMEM, "cudaMallocHost: %s", cudaGetErrorString(e)));
    // spectrum padding columns are never written by the passes; keep them defined
    e = cudaMemsetAsync(s->S1, 0, s1, s->st);
    if (e == cudaSuccess && s2) e = cudaMemsetAsync(s->S2, 0, s2, s->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->hd, 0, v3, s->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->dev_err, 0, sizeof(int), s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return bail(fail(MM_ECUDA, "initialising buffers: %s", cudaGetErrorString(e)));
    *out = s;
    return MM_OK;
}

void mm_state_destroy(mm_state* s) {
    if (!s) return;
    cudaSetDevice(s->device);
    cudaStreamSynchronize(s->st);
    void** bufs[] = {&s->m, &s->mA, &s->mB, &s->acc, &s->hd, &s->S1, &s->S2, &s->tens, &s->D_cell, &s->Ms_cell,
                     &s->A_cell, &s->Ku_cell, &s->alpha_cell, &s->axis_tab, reinterpret_cast<void**>(&s->grain),
                     &s->zw, reinterpret_cast<void**>(&s->partials), reinterpret_cast<void**>(&s->scalars),
                     reinterpret_cast<void**>(&s->dev_err), &s->lay_t, reinterpret_cast<void**>(&s->lay_v)};
    for (void** b : bufs) dev_free(*b);
    for (int q = 0; q < 7; ++q) dev_free(s->K[q]);
    for (int q = 0; q < 19; ++q) dev_free(s->adj[q]);
    if (s->h_scalars) cudaFreeHost(s->h_scalars);
    s->timer.destroy();
    delete s;
}

mm_status mm_set_material(mm_state* s, const mm_material* mat, int ptrs_on_device) {
    MM_TRY(check_state(s));
    if (!mat) return fail(MM_EINVAL, "null material");
    if (!(mat->Ms >= 0) || !(mat->A >= 0) || !(mat->alpha >= 0) || !std::isfinite(mat->Ku1))
        return fail(MM_EINVAL, "material scalars must satisfy Ms >= 0, A >= 0, alpha >= 0, finite Ku1");
    if (mat->grain_id && (mat->ngrains < 1 || mat->ngrains > 256 || !mat->ku_axis_table))
        return fail(MM_EINVAL, "grain_id needs ku_axis_table and 1 <= ngrains <= 256");
    MM_TRY(set_device(s));
    s->Ms = mat->Ms; s->A = mat->A; s->Ku = mat->Ku1; s->alpha = mat->alpha;
    for (int q = 0; q < 3; ++q) s->axis[q] = mat->ku_axis[q];
    MM_TRY(upload_real(s, mat->Ms_cell, s->N, ptrs_on_device, &s->Ms_cell));
    MM_TRY(upload_real(s, mat->A_cell, s->N, ptrs_on_device, &s->A_cell));
    MM_TRY(upload_real(s, mat->Ku1_cell, s->N, ptrs_on_device, &s->Ku_cell));
    MM_TRY(upload_real(s, mat->alpha_cell, s->N, ptrs_on_device, &s->alpha_cell));
    MM_TRY(upload_real(s, mat->grain_id ? mat->ku_axis_table : nullptr, 3L * mat->ngrains, ptrs_on_device,
                       &s->axis_tab));
    dev_free(reinterpret_cast<void*&>(s->grain));
    if (mat->grain_id) {
        MM_TRY(dev_alloc(reinterpret_cast<void**>(&s->grain), (size_t)s->N));
        MM_CUDA(cudaMemcpyAsync(s->grain, mat->grain_id, (size_t)s->N,
                                ptrs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->st));
        MM_CUDA(cudaStreamSynchronize(s->st));
    }
    s->have_mat = true;
    s->fsal = s->k1_exact = false;
    s->s1_fresh = false;
    return MM_OK;
}

mm_status mm_set_m(mm_state* s, const void* m, int on_device) {
    MM_TRY(check_state(s));
    if (!m) return fail(MM_EINVAL, "null m");
    MM_TRY(set_device(s));
    MM_CUDA(cudaMemcpyAsync(s->m, m, 3 * s->rsz * (size_t)s->N,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->st));
    s->have_m = true;
    s->fsal = s->k1_exact = false;
    s->s1_fresh = false;
    return MM_OK;
}

mm_status mm_get_m(const mm_state* s, void* m_out, int on_device) {
    MM_TRY(check_state(s));
    if (!m_out) return fail(MM_EINVAL, "null m_out");
    MM_TRY(set_device(s));
    MM_CUDA(cudaMemcpyAsync(m_out, s->m, 3 * s->rsz * (size_t)s->N,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->st));
    if (!on_device) MM_CUDA(cudaStreamSynchronize(s->st));
    return MM_OK;
}

mm_status mm_set_zeeman(mm_state* s, const double h_const[3], mm_field_fn fn, void* user, const double* weight,
                        int on_device) {
    MM_TRY(check_state(s));
    MM_TRY(set_device(s));
    for (int q = 0; q < 3; ++q) s->h0[q] = h_const ? h_const[q] : 0.0;
    s->fn = fn;
    s->user = user;
    MM_TRY(upload_real(s, weight, s->N, on_device, &s->zw));
    s->fsal = s->k1_exact = false;
    return MM_OK;
}

mm_status mm_demag_setup(mm_state* s, int p_newell) {
    MM_TRY(check_state(s));
    MM_TRY(set_device(s));
    const int n[3] = {s->g.nx, s->g.ny, s->g.nz};
    const double dd[3] = {s->g.dx, s->g.dy, s->g.dz};
    const int P[3] = {s->d.LX, s->d.LY, s->d.LZ};
    std::vector<double> spec;
    if (!s->lay_h.empty())
        tensor_layers_spectrum(n[0], n[1], n[2], dd[0], dd[1], s->lay_h.data(), p_newell, P[0], P[1], s->d.KXS, spec);
    else
        tensor_spectrum(n, dd, p_newell, P, s->d.KXS, spec);
    const long cnt = (long)spec.size();
    dev_free(s->tens);
    MM_TRY(dev_alloc(&s->tens, s->rsz * (size_t)cnt));
    if (s->prec == MM_FP64) {
        MM_CUDA(cudaMemcpyAsync(s->tens, spec.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice, s->st));
    } else {
        std::vector<float> f(cnt);
        for (long i = 0; i < cnt; ++i) f[i] = (float)spec[i];
        MM_CUDA(cudaMemcpyAsync(s->tens, f.data(), sizeof(float) * cnt, cudaMemcpyHostToDevice, s->st));
        MM_CUDA(cudaStreamSynchronize(s->st));
    }
    MM_CUDA(cudaStreamSynchronize(s->st));
    s->demag_ready = true;
    s->demag_off = false;
    s->fsal = s->k1_exact = false;
    return MM_OK;
}

mm_status mm_demag_disable(mm_state* s) {
    MM_TRY(check_state(s));
    s->demag_off = true;
    s->fsal = s->k1_exact = false;
    return MM_OK;
}

mm_status mm_heff(mm_state* s, const void* m, void* h_out, double E_out[4], double t, double* torque_out) {
    MM_TRY(check_state(s));
    MM_TRY(set_device(s));
    return s->prec == MM_FP64 ? heff_impl<double>(s, m, h_out, E_out, t, torque_out)
                              : heff_impl<float>(s, m, h_out, E_out, t, torque_out);
}

mm_status mm_llg_rhs(mm_state* s, const void* m, void* k_out, double t) {
    MM_TRY(check_state(s));
    if (!k_out) return fail(MM_EINVAL, "null k_out");
    MM_TRY(set_device(s));
    return s->prec == MM_FP64 ? rhs_impl<double>(s, m, k_out, t) : rhs_impl<float>(s, m, k_out, t);
}

mm_status mm_llg_step(mm_state* s, mm_method method, double* dt_inout, double rtol, double* t_inout) {
    MM_TRY(check_state(s));
    if (!dt_inout || !t_inout) return fail(MM_EINVAL, "null dt or t");
    if (!(*dt_inout > 0) || !std::isfinite(*dt_inout)) return fail(MM_EINVAL, "dt must be > 0");
    MM_TRY(ready_for_fields(s));
    if (!s->have_m) return fail(MM_ENOTSETUP, "mm_set_m has not been called");
    MM_TRY(set_device(s));
    if (method == MM_RK4) {
        MM_TRY(s->prec == MM_FP64 ? rk4_impl<double>(s, *dt_inout, *t_inout) : rk4_impl<float>(s, *dt_inout, *t_inout));
        *t_inout += *dt_inout;
        return MM_OK;
    }
    if (method == MM_DP45) {
        if (!(rtol > 0)) return fail(MM_EINVAL, "rtol must be > 0");
        return s->prec == MM_FP64 ? dp_step<double>(s, dt_inout, rtol, t_inout, nullptr)
                                  : dp_step<float>(s, dt_inout, rtol, t_inout, nullptr);
    }
    if (method == MM_RKF45) {
        if (!(rtol > 0)) return fail(MM_EINVAL, "rtol must be > 0");
        return s->prec == MM_FP64 ? rkf_step<double>(s, dt_inout, rtol, t_inout)
                                  : rkf_step<float>(s, dt_inout, rtol, t_inout);
    }
    return fail(MM_EINVAL, "unknown method %d", (int)method);
}

mm_status mm_relax(mm_state* s, double tol, int max_steps, double rtol, double* dt_inout, double* t_inout,
                   int* steps_out, double* torque_out) {
    MM_TRY(check_state(s));
    if (!(tol > 0) || max_steps < 0 || !(rtol > 0)) return fail(MM_EINVAL, "bad tol, rtol or max_steps");
    MM_TRY(ready_for_fields(s));
    if (!s->have_m) return fail(MM_ENOTSETUP, "mm_set_m has not been called");
    MM_TRY(set_device(s));
    double dt = (dt_inout && *dt_inout > 0) ? *dt_inout : 1e-13;
    double t = t_inout ? *t_inout : 0.0;
    double tq = 0.0;
    MM_TRY(ensure_dp_buffers(s));
    int steps = 0;
    mm_status st = MM_OK;
    if (s->relax_method == MM_RKF45) {
        // the torque at each new m comes with the first stage of the next step
        for (;;) {
            st = s->prec == MM_FP64 ? dp_first_stage<double>(s, t, &tq) : dp_first_stage<float>(s, t, &tq);
            if (st != MM_OK || tq < tol || steps >= max_steps) break;
            st = s->prec == MM_FP64 ? rkf_step<double>(s, &dt, rtol, &t) : rkf_step<float>(s, &dt, rtol, &t);
            if (st != MM_OK) break;
            ++steps;
        }
    } else {
        MM_TRY(s->prec == MM_FP64 ? dp_first_stage<double>(s, t, &tq) : dp_first_stage<float>(s, t, &tq));
        while (tq >= tol && steps < max_steps) {
            st = s->prec == MM_FP64 ? dp_step<double>(s, &dt, rtol, &t, &tq)
                                    : dp_step<float>(s, &dt, rtol, &t, &tq);
            if (st != MM_OK) break;
            ++steps;
        }
    }
    if (dt_inout) *dt_inout = dt;
    if (t_inout) *t_inout = t;
    if (steps_out) *steps_out = steps;
    if (torque_out) *torque_out = tq;
    if (st != MM_OK) return st;
    if (tq >= tol) return fail(MM_ENOTCONVERGED, "relax: torque %g >= %g after %d steps", tq, tol, steps);
    return MM_OK;
}

mm_status mm_llg_step_adjoint(mm_state* s, const void* m_n, const void* lambda_np1, void* lambda_n,
                              void* grad_Ms_accum, double dt, double t) {
    MM_TRY(check_state(s));
    if (!m_n || !lambda_np1 || !lambda_n) return fail(MM_EINVAL, "null m_n, lambda_np1 or lambda_n");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(MM_EINVAL, "dt must be > 0");
    if (lambda_n == lambda_np1 || lambda_n == m_n) return fail(MM_EINVAL, "lambda_n must not alias the inputs");
    if (!s->lay_h.empty()) return fail(MM_EINVAL, "the adjoint does not cover non-equidistant layers");
    MM_TRY(ready_for_fields(s));
    MM_TRY(set_device(s));
    return s->prec == MM_FP64 ? adjoint_impl<double>(s, m_n, lambda_np1, lambda_n, grad_Ms_accum, dt, t)
                              : adjoint_impl<float>(s, m_n, lambda_np1, lambda_n, grad_Ms_accum, dt, t);
}

mm_status mm_set_dmi(mm_state* s, mm_dmi_kind kind, double D, const double* D_cell, int on_device) {
    MM_TRY(check_state(s));
    if (kind < MM_DMI_NONE || kind > MM_DMI_D2D) return fail(MM_EINVAL, "unknown DMI kind %d", (int)kind);
    if (!std::isfinite(D)) return fail(MM_EINVAL, "D must be finite");
    if (kind != MM_DMI_NONE && !s->lay_h.empty())
        return fail(MM_EINVAL, "DMI is not defined with non-equidistant layers");
    MM_TRY(set_device(s));
    MM_TRY(upload_real(s, kind == MM_DMI_NONE ? nullptr : D_cell, s->N, on_device, &s->D_cell));
    s->dmi_kind = kind;
    s->D = D;
    s->fsal = s->k1_exact = false;
    return MM_OK;
}

mm_status mm_set_llg_options(mm_state* s, mm_method relax_method, int precession) {
    MM_TRY(check_state(s));
    if (relax_method != MM_DP45 && relax_method != MM_RKF45)
        return fail(MM_EINVAL, "relax method must be MM_DP45 or MM_RKF45");
    if (precession != 0 && precession != 1) return fail(MM_EINVAL, "precession must be 0 or 1");
    s->relax_method = relax_method;
    if (s->precession != precession) s->fsal = s->k1_exact = false;
    s->precession = precession;
    return MM_OK;
}

mm_status mm_selftest_wait_timeout(mm_state* s, unsigned spins) {
    MM_TRY(check_state(s));
    MM_TRY(set_device(s));
    if (spins < 1) return fail(MM_EINVAL, "spins must be >= 1");
    launch_diag_wait(s->dev_err, spins, s->st);
    MM_LAUNCHED();
    return MM_OK;
}

mm_status mm_probe_fp64_fma(void* cuda_stream, double* sink, int blocks, int iters, double* flops_out) {
    if (!sink || !flops_out) return fail(MM_EINVAL, "null argument");
    if (blocks < 1 || blocks > (1 << 20) || iters < 1) return fail(MM_EINVAL, "blocks must be 1..2^20, iters >= 1");
    cudaGetLastError();
    *flops_out = launch_fp64_fma_probe(sink, blocks, iters, (cudaStream_t)cuda_stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(MM_ECUDA, "FP64 probe launch: %s", cudaGetErrorString(e));
    return MM_OK;
}

mm_status mm_set_layers(mm_state* s, const double* h, int nz) {
    MM_TRY(check_state(s));
    if (!h) {
        if (s->lay_h.empty()) return MM_OK;
    } else {
        if (nz != s->g.nz) return fail(MM_EINVAL, "need one thickness per layer (%d), got %d", s->g.nz, nz);
        if (nz < 2 || nz > kMaxLayers) return fail(MM_EINVAL, "a layer stack has 2 to %d layers", kMaxLayers);
        for (int k = 0; k < nz; ++k)
            if (!(h[k] > 0.0) || !std::isfinite(h[k])) return fail(MM_EINVAL, "layer %d thickness must be > 0", k);
        if (s->dmi_kind != MM_DMI_NONE) return fail(MM_EINVAL, "DMI is not defined with non-equidistant layers");
    }
    MM_TRY(set_device(s));
    MM_CUDA(cudaStreamSynchronize(s->st));
    dev_free(s->lay_t);
    dev_free(reinterpret_cast<void*&>(s->lay_v));
    s->lay_t = nullptr;
    s->lay_v = nullptr;
    s->lay_h.clear();
    s->d.layers = 0;
    s->d.lh = nullptr;
    // the tensor of the old geometry no longer applies
    s->demag_ready = false;
    s->fsal = s->k1_exact = s->s1_fresh = false;
    if (!h) return MM_OK;
    std::vector<double> t(3 * (size_t)nz, 0.0), v(nz);
    for (int k = 0; k < nz; ++k) {
        t[k] = h[k];
        if (k < nz - 1) t[nz + k] = 2.0 / (h[k] * (h[k] + h[k + 1]));
        if (k > 0) t[2 * nz + k] = 2.0 / (h[k] * (h[k - 1] + h[k]));
        v[k] = s->g.dx * s->g.dy * h[k];
    }
    MM_TRY(dev_alloc(&s->lay_t, s->rsz * t.size()));
    MM_TRY(dev_alloc(reinterpret_cast<void**>(&s->lay_v), sizeof(double) * nz));
    if (s->prec == MM_FP64) {
        MM_CUDA(cudaMemcpy(s->lay_t, t.data(), sizeof(double) * t.size(), cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f(t.begin(), t.end());
        MM_CUDA(cudaMemcpy(s->lay_t, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice));
    }
    MM_CUDA(cudaMemcpy(s->lay_v, v.data(), sizeof(double) * nz, cudaMemcpyHostToDevice));
    s->lay_h.assign(h, h + nz);
    s->d.layers = 1;
    s->d.lh = s->lay_t;
    return MM_OK;
}

int mm_fft_extent(int n) { return n < 1 ? 0 : fft_extent(n); }

size_t mm_batch_footprint(const mm_grid* grid, mm_precision precision, int capacity) {
    if (!grid || capacity < 1) return 0;
    return batch_bytes(grid, precision, capacity, nullptr, nullptr, nullptr, nullptr);
}

void mm_batch_destroy(mm_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->st);
    batch_drop_graphs(b);
    void** bufs[] = {&b->m, &b->Y[0], &b->Y[1], &b->hd, &b->S1, &b->S2, &b->tens, &b->Ms_d, &b->A_d, &b->alpha_d,
                     &b->D_d, &b->pc_d, reinterpret_cast<void**>(&b->kind_d), reinterpret_cast<void**>(&b->ctl_i), reinterpret_cast<void**>(&b->ctl_d),
                     reinterpret_cast<void**>(&b->mask_d), reinterpret_cast<void**>(&b->acc_d),
                     reinterpret_cast<void**>(&b->partials), reinterpret_cast<void**>(&b->scal_d)};
    for (void** q : bufs) dev_free(*q);
    for (int q = 0; q < 7; ++q) dev_free(b->K[q]);
    if (b->rep_i) cudaFreeHost(b->rep_i);
    if (b->rep_d) cudaFreeHost(b->rep_d);
    if (b->done) cudaEventDestroy(b->done);
    delete b;
}

mm_status mm_batch_create(const mm_grid* grid, mm_precision precision, int capacity, int p_newell, void* cuda_stream,
                          mm_batch** out) {
    if (!grid || !out) return fail(MM_EINVAL, "null argument");
    *out = nullptr;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->dx > 0) || !(grid->dy > 0) || !(grid->dz > 0))
        return fail(MM_EINVAL, "bad grid");
    if (capacity < 1 || capacity > 4096) return fail(MM_EINVAL, "capacity must be in 1..4096");
    if (precision != MM_FP64 && precision != MM_FP32_FIELDS) return fail(MM_EINVAL, "bad precision");
    if ((double)grid->nx * grid->ny * grid->nz * capacity * 3 >= 2147483648.0) return fail(MM_EINVAL, "batch too large");
    int LX, LY, LZ, KXS;
    batch_bytes(grid, precision, capacity, &LX, &LY, &LZ, &KXS);
    if (LX > kMaxFft || LY > kMaxFft || LZ > kMaxFft) return fail(MM_EINVAL, "padded FFT extent above %d", kMaxFft);
    mm_batch* b = new (std::nothrow) mm_batch();
    if (!b) return fail(MM_ENOMEM, "host allocation");
    auto bail = [&](mm_status st) { mm_batch_destroy(b); return st; };
    b->g = *grid;
    b->prec = precision;
    b->st = (cudaStream_t)cuda_stream;
    b->cap = capacity;
    b->N = (long)grid->nx * grid->ny * grid->nz;
    b->rsz = precision == MM_FP64 ? 8 : 4;
    b->csz = 2 * b->rsz;
    b->d = DemagDims{grid->nx, grid->ny, grid->nz, LX, LY, LZ, LX / 2 + 1, KXS};
    b->d.nb = capacity;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e != cudaSuccess) return bail(fail(MM_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e)));
    mm_status st = ensure_twiddles(b->device);
    if (st != MM_OK) return bail(st);
    const size_t v3 = (size_t)capacity * 3 * b->rsz * b->N;
    void** bufs[] = {&b->m, &b->Y[0], &b->Y[1], &b->hd};
    for (void** q : bufs)
        if ((st = dev_alloc(q, v3)) != MM_OK) return bail(st);
    for (int q = 0; q < 7; ++q)
        if ((st = dev_alloc(&b->K[q], v3)) != MM_OK) return bail(st);
    const size_t s1 = (size_t)capacity * 3 * b->csz * grid->ny * grid->nz * KXS;
    const size_t s2 = LY > 1 ? (size_t)capacity * 3 * b->csz * grid->nz * LY * KXS : 0;
    if ((st = dev_alloc(&b->S1, s1)) != MM_OK) return bail(st);
    if ((st = dev_alloc(&b->S2, s2)) != MM_OK) return bail(st);
    if ((st = dev_alloc(&b->Ms_d, b->rsz * capacity)) != MM_OK) return bail(st);
    if ((st = dev_alloc(&b->A_d, b->rsz * capacity)) != MM_OK) return bail(st);
    if ((st = dev_alloc(&b->alpha_d, b->rsz * capacity)) != MM_OK) return bail(st);
    if ((st = dev_alloc(&b->D_d, b->rsz * capacity)) != MM_OK) return bail(st);
    if ((st = dev_alloc(&b->pc_d, b->rsz * capacity)) != MM_OK) return bail(st);
    if ((st = dev_alloc(reinterpret_cast<void**>(&b->kind_d), sizeof(int) * capacity)) != MM_OK) return bail(st);
    if ((st = dev_alloc(reinterpret_cast<void**>(&b->ctl_i), sizeof(int) * 3 * capacity)) != MM_OK) return bail(st);
    if ((st = dev_alloc(reinterpret_cast<void**>(&b->ctl_d), sizeof(double) * 3 * capacity)) != MM_OK)
        return bail(st);
    if ((st = dev_alloc(reinterpret_cast<void**>(&b->mask_d), sizeof(int) * 2 * capacity)) != MM_OK) return bail(st);
    if ((st = dev_alloc(reinterpret_cast<void**>(&b->acc_d), sizeof(int) * capacity)) != MM_OK) return bail(st);
    b->nblk = (int)((b->N + 255) / 256);
    if ((st = dev_alloc(reinterpret_cast<void**>(&b->partials), sizeof(double) * 2 * 3 * (size_t)capacity * b->nblk)) !=
        MM_OK)
        return bail(st);
    if ((st = dev_alloc(reinterpret_cast<void**>(&b->scal_d), sizeof(double) * 6 * capacity)) != MM_OK) return bail(st);
    if (cudaMallocHost(reinterpret_cast<void**>(&b->rep_i), sizeof(int) * 2 * capacity) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&b->rep_d), sizeof(double) * capacity) != cudaSuccess)
        return bail(fail(MM_ENOMEM, "cudaMallocHost"));
    if ((e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming)) != cudaSuccess)
        return bail(fail(MM_ECUDA, "cudaEventCreate: %s", cudaGetErrorString(e)));
    b->d.Ms_b = b->Ms_d;
    // the size bucket's plan: tensor spectrum of this shape, shared by every slot
    const int n[3] = {grid->nx, grid->ny, grid->nz};
    const double dd[3] = {grid->dx, grid->dy, grid->dz};
    const int P[3] = {LX, LY, LZ};
    std::vector<double> spec;
    tensor_spectrum(n, dd, p_newell, P, KXS, spec);
    if ((st = dev_alloc(&b->tens, b->rsz * spec.size())) != MM_OK) return bail(st);
    if (precision == MM_FP64) {
        e = cudaMemcpy(b->tens, spec.data(), sizeof(double) * spec.size(), cudaMemcpyHostToDevice);
    } else {
        std::vector<float> f(spec.size());
        for (size_t i = 0; i < spec.size(); ++i) f[i] = (float)spec[i];
        e = cudaMemcpy(b->tens, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(b->S1, 0, s1, b->st);
    if (e == cudaSuccess && s2) e = cudaMemsetAsync(b->S2, 0, s2, b->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->m, 0, v3, b->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->Ms_d, 0, b->rsz * capacity, b->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->D_d, 0, b->rsz * capacity, b->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->pc_d, 0, b->rsz * capacity, b->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->kind_d, 0, sizeof(int) * capacity, b->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ctl_i, 0, sizeof(int) * 3 * capacity, b->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ctl_d, 0, sizeof(double) * 3 * capacity, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return bail(fail(MM_ECUDA, "batch set-up: %s", cudaGetErrorString(e)));
    b->status.assign(capacity, 0);
    b->unstarted.assign(capacity, 0);
    *out = b;
    return MM_OK;
}

mm_status mm_batch_set_slot(mm_batch* b, int slot, double Ms, double A, double alpha, const void* m0, int on_device,
                            double dt0) {
    if (!b || !m0) return fail(MM_EINVAL, "null argument");
    if (slot < 0 || slot >= b->cap) return fail(MM_EINVAL, "slot %d out of range", slot);
    if (b->pending) return fail(MM_EINVAL, "attempts are in flight: call mm_batch_end first");
    if (b->status[slot] != 0) return fail(MM_EINVAL, "slot %d is busy", slot);
    if (!(Ms >= 0) || !(A >= 0) || !(alpha >= 0)) return fail(MM_EINVAL, "bad material");
    MM_CUDA(cudaSetDevice(b->device));
    const size_t v = 3 * b->rsz * (size_t)b->N;
    MM_CUDA(cudaMemcpyAsync(static_cast<char*>(b->m) + slot * v, m0, v,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->st));
    // the slot's material; no DMI and the precession term on until mm_batch_set_slot_terms
    const double mat[5] = {Ms, A, alpha, 0.0, 1.0};
    void* dst[5] = {b->Ms_d, b->A_d, b->alpha_d, b->D_d, b->pc_d};
    MM_CUDA(cudaMemsetAsync(b->kind_d + slot, 0, sizeof(int), b->st));
    for (int q = 0; q < 5; ++q) {
        if (b->prec == MM_FP64) {
            MM_CUDA(cudaMemcpyAsync(static_cast<double*>(dst[q]) + slot, &mat[q], 8, cudaMemcpyHostToDevice, b->st));
        } else {
            const float f = (float)mat[q];
            MM_CUDA(cudaMemcpyAsync(static_cast<float*>(dst[q]) + slot, &f, 4, cudaMemcpyHostToDevice, b->st));
        }
    }
    const int one = 1, zero = 0;
    const double dt = dt0 > 0 ? dt0 : 1e-13, dz = 0.0;
    MM_CUDA(cudaMemcpyAsync(b->status_d() + slot, &one, sizeof(int), cudaMemcpyHostToDevice, b->st));
    MM_CUDA(cudaMemcpyAsync(b->steps_d() + slot, &zero, sizeof(int), cudaMemcpyHostToDevice, b->st));
    MM_CUDA(cudaMemcpyAsync(b->fresh_d() + slot, &one, sizeof(int), cudaMemcpyHostToDevice, b->st));
    MM_CUDA(cudaMemcpyAsync(b->dt_d() + slot, &dt, sizeof(double), cudaMemcpyHostToDevice, b->st));
    MM_CUDA(cudaMemcpyAsync(b->t_d() + slot, &dz, sizeof(double), cudaMemcpyHostToDevice, b->st));
    MM_CUDA(cudaMemcpyAsync(b->torque_d() + slot, &dz, sizeof(double), cudaMemcpyHostToDevice, b->st));
    MM_CUDA(cudaStreamSynchronize(b->st));   // the host values above are stack copies
    b->status[slot] = 1;
    b->unstarted[slot] = 1;
    b->fresh_any = true;
    return MM_OK;
}

mm_status mm_batch_set_slot_terms(mm_batch* b, int slot, int dmi_kind, double D, int precession) {
    if (!b) return fail(MM_EINVAL, "null batch");
    if (slot < 0 || slot >= b->cap) return fail(MM_EINVAL, "slot %d out of range", slot);
    if (b->pending) return fail(MM_EINVAL, "attempts are in flight: call mm_batch_end first");
    if (!b->unstarted[slot]) return fail(MM_EINVAL, "slot %d is not freshly loaded", slot);
    if (dmi_kind < MM_DMI_NONE || dmi_kind > MM_DMI_D2D || !std::isfinite(D))
        return fail(MM_EINVAL, "bad DMI kind or strength");
    MM_CUDA(cudaSetDevice(b->device));
    const int kind = D != 0.0 ? dmi_kind : MM_DMI_NONE;
    const double v[2] = {D, precession ? 1.0 : 0.0};
    void* dst[2] = {b->D_d, b->pc_d};
    for (int q = 0; q < 2; ++q) {
        if (b->prec == MM_FP64) {
            MM_CUDA(cudaMemcpyAsync(static_cast<double*>(dst[q]) + slot, &v[q], 8, cudaMemcpyHostToDevice, b->st));
        } else {
            const float f = (float)v[q];
            MM_CUDA(cudaMemcpyAsync(static_cast<float*>(dst[q]) + slot, &f, 4, cudaMemcpyHostToDevice, b->st));
        }
    }
    MM_CUDA(cudaMemcpyAsync(b->kind_d + slot, &kind, sizeof(int), cudaMemcpyHostToDevice, b->st));
    MM_CUDA(cudaStreamSynchronize(b->st));   // the host values above are stack copies
    return MM_OK;
}

mm_status mm_batch_clear_slot(mm_batch* b, int slot) {
    if (!b) return fail(MM_EINVAL, "null batch");
    if (slot < 0 || slot >= b->cap) return fail(MM_EINVAL, "slot %d out of range", slot);
    if (b->pending) return fail(MM_EINVAL, "attempts are in flight: call mm_batch_end first");
    MM_CUDA(cudaSetDevice(b->device));
    const int zero = 0;
    MM_CUDA(cudaMemcpyAsync(b->status_d() + slot, &zero, sizeof(int), cudaMemcpyHostToDevice, b->st));
    MM_CUDA(cudaMemcpyAsync(b->fresh_d() + slot, &zero, sizeof(int), cudaMemcpyHostToDevice, b->st));
    MM_CUDA(cudaStreamSynchronize(b->st));
    b->status[slot] = 0;
    b->unstarted[slot] = 0;
    return MM_OK;
}

mm_status mm_batch_begin(mm_batch* b, int attempts, double rtol, double tol, int max_steps) {
    if (!b) return fail(MM_EINVAL, "null batch");
    if (attempts < 1 || attempts > 1024) return fail(MM_EINVAL, "attempts must be in 1..1024");
    if (!(rtol > 0) || !(tol >= 0) || max_steps < 1) return fail(MM_EINVAL, "bad rtol, tol or max_steps");
    if (b->pending) return fail(MM_EINVAL, "attempts are already in flight");
    MM_CUDA(cudaSetDevice(b->device));
    std::fill(b->unstarted.begin(), b->unstarted.end(), 0);
    return b->prec == MM_FP64 ? batch_begin_impl<double>(b, attempts, rtol, tol, max_steps)
                              : batch_begin_impl<float>(b, attempts, rtol, tol, max_steps);
}

mm_status mm_batch_query(mm_batch* b, int* ready) {
    if (!b || !ready) return fail(MM_EINVAL, "null argument");
    if (!b->pending) return fail(MM_EINVAL, "nothing in flight: call mm_batch_begin first");
    MM_CUDA(cudaSetDevice(b->device));
    const cudaError_t e = cudaEventQuery(b->done);
    if (e == cudaErrorNotReady) {
        *ready = 0;
        return MM_OK;
    }
    MM_CUDA(e);
    *ready = 1;
    return MM_OK;
}

mm_status mm_batch_end(mm_batch* b, int* status, int* steps, double* torque) {
    if (!b) return fail(MM_EINVAL, "null batch");
    if (!b->pending) return fail(MM_EINVAL, "nothing in flight: call mm_batch_begin first");
    MM_CUDA(cudaSetDevice(b->device));
    b->pending = false;
    MM_CUDA(cudaStreamSynchronize(b->st));
    for (int i = 0; i < b->cap; ++i) {
        b->status[i] = b->rep_i[i];
        if (status) status[i] = b->rep_i[i];
        if (steps) steps[i] = b->rep_i[b->cap + i];
        if (torque) torque[i] = b->rep_d[i];
    }
    return MM_OK;
}

mm_status mm_batch_get_m(mm_batch* b, int slot, void* m_out, int on_device) {
    if (!b || !m_out) return fail(MM_EINVAL, "null argument");
    if (slot < 0 || slot >= b->cap) return fail(MM_EINVAL, "slot %d out of range", slot);
    if (b->pending) return fail(MM_EINVAL, "attempts are in flight: call mm_batch_end first");
    MM_CUDA(cudaSetDevice(b->device));
    const size_t v = 3 * b->rsz * (size_t)b->N;
    MM_CUDA(cudaMemcpyAsync(m_out, static_cast<char*>(b->m) + slot * v, v,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->st));
    if (!on_device) MM_CUDA(cudaStreamSynchronize(b->st));
    return MM_OK;
}

mm_status mm_demag_tensor_host(const mm_grid* grid, int p_newell, double* out) {
    if (!grid || !out) return fail(MM_EINVAL, "null argument");
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->dx > 0) || !(grid->dy > 0) || !(grid->dz > 0))
        return fail(MM_EINVAL, "bad grid");
    const int n[3] = {grid->nx, grid->ny, grid->nz};
    const double dd[3] = {grid->dx, grid->dy, grid->dz};
    tensor_full_offsets(n, dd, p_newell, out);
    return MM_OK;
}

mm_status mm_demag_spectrum_host(const mm_grid* grid, int p_newell, double* out) {
    if (!grid || !out) return fail(MM_EINVAL, "null argument");
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->dx > 0) || !(grid->dy > 0) || !(grid->dz > 0))
        return fail(MM_EINVAL, "bad grid");
    const int n[3] = {grid->nx, grid->ny, grid->nz};
    const double dd[3] = {grid->dx, grid->dy, grid->dz};
    const int P[3] = {fft_extent(grid->nx), fft_extent(grid->ny), fft_extent(grid->nz)};
    if (P[0] > kMaxFft || P[1] > kMaxFft || P[2] > kMaxFft) return fail(MM_EINVAL, "padded extent too large");
    std::vector<double> spec;
    tensor_spectrum(n, dd, p_newell, P, P[0] / 2 + 1, spec);
    std::memcpy(out, spec.data(), sizeof(double) * spec.size());
    return MM_OK;
}

mm_status mm_layers_spectrum_host(const mm_grid* grid, const double* h, int p_newell, double* out) {
    if (!grid || !h || !out) return fail(MM_EINVAL, "null argument");
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->dx > 0) || !(grid->dy > 0))
        return fail(MM_EINVAL, "bad grid");
    for (int k = 0; k < grid->nz; ++k)
        if (!(h[k] > 0.0) || !std::isfinite(h[k])) return fail(MM_EINVAL, "layer %d thickness must be > 0", k);
    const int Px = fft_extent(grid->nx), Py = fft_extent(grid->ny);
    if (Px > kMaxFft || Py > kMaxFft) return fail(MM_EINVAL, "padded extent too large");
    std::vector<double> spec;
    tensor_layers_spectrum(grid->nx, grid->ny, grid->nz, grid->dx, grid->dy, h, p_newell, Px, Py, Px / 2 + 1, spec);
    std::memcpy(out, spec.data(), sizeof(double) * spec.size());
    return MM_OK;
}

mm_status mm_state_info(const mm_state* s, int out[5]) {
    MM_TRY(check_state(s));
    if (!out) return fail(MM_EINVAL, "null out");
    out[0] = s->d.LX; out[1] = s->d.LY; out[2] = s->d.LZ; out[3] = s->d.KX; out[4] = s->d.KXS;
    return MM_OK;
}

mm_status mm_profile_enable(mm_state* s, int on) {
    MM_TRY(check_state(s));
    if (on) {
        cudaStreamSynchronize(s->st);
        s->timer.reset();
    }
    s->timer.on = on != 0;
    return MM_OK;
}

int mm_profile_read(mm_state* s, const char** names, int* counts, double* ms, int max) {
    if (!s) return -1;
    if (cudaStreamSynchronize(s->st) != cudaSuccess) return -1;
    const int nn = (int)s->timer.names.size();
    std::vector<double> tot(nn, 0.0);
    std::vector<int> cnt(nn, 0);
    for (const auto& r : s->timer.recs) {
        float f = 0.f;
        if (cudaEventElapsedTime(&f, r.a, r.b) == cudaSuccess) {
            tot[r.name] += f;
            cnt[r.name] += 1;
        }
    }
    const int k = std::min(nn, max);
    for (int i = 0; i < k; ++i) {
        if (names) names[i] = s->timer.names[i].c_str();
        if (counts) counts[i] = cnt[i];
        if (ms) ms[i] = tot[i];
    }
    return nn;
}

}  // extern "C"
