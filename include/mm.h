/*
 * mm.h -- C ABI of libmm.so, a GB300 (sm_103a) implementation of the hot path
 * of the finite-difference micromagnetic method of arXiv 2302.08843
 * (magnum.np): one effective-field evaluation (demag, exchange, uniaxial
 * anisotropy, Zeeman), the LLG right-hand side and the Runge-Kutta stage
 * update on a regular cell grid.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid (Sec. 2): nx x ny x nz cells of size dx x dy x dz metres, cell centre
 *   (i dx, j dy, k dz).  Cell index c = i + nx * (j + ny * k) (x fastest).
 * Vector fields (m, h): structure of arrays, three planes of nx*ny*nz values,
 *   [3][nz][ny][nx].  Their element type is the state's "real": double for
 *   MM_FP64, float for MM_FP32_FIELDS.  Fields are in A/m, m is unit length.
 * Scalar material maps: nx*ny*nz doubles in the same cell order.
 * Pointers: caller memory is borrowed for the duration of the call only; a
 *   flag says whether it is host or device memory (device memory must be on the
 *   state's device).  The state owns all of its device buffers.
 * Streams: all GPU work of a state is enqueued on the CUDA stream given at
 *   creation (NULL = the legacy default stream).  Functions return after
 *   enqueueing, except those that return host scalars (E_out, DP45 step
 *   acceptance, mm_relax, mm_get_m to host), which synchronise that stream.
 * Errors: every function returns an mm_status; mm_last_error() gives a
 *   thread-local message for the last failure.  Nothing aborts or throws.
 * Devices: per-device constant tables (FFT twiddles) are uploaded on a
 *   device's first use and kept for the process; after cudaDeviceReset on a
 *   device, do not use the library on that device again.
 * Cells with Ms = 0 carry no effective field (the nan_to_num of the
 *   anisotropy listing in Sec. 4.1, applied to every term).
 */
#ifndef MM_H
#define MM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mm_state mm_state;   /* opaque, library-owned */

typedef enum {
    MM_OK = 0,
    MM_EINVAL = 1,          /* bad argument (null pointer, size, enum)          */
    MM_ENOMEM = 2,          /* device or host allocation failed                 */
    MM_ECUDA = 3,           /* a CUDA call failed (message says which)           */
    MM_ENONFINITE = 4,      /* a NaN or Inf appeared in m or in a reduction      */
    MM_ESTEP = 5,           /* DP45 step size underflow (dt < 1e-22 s)           */
    MM_ENOTCONVERGED = 6,   /* mm_relax reached max_steps                        */
    MM_ETIMEOUT = 7,        /* reserved: a bounded device-side wait gave up      */
    MM_ENOTSETUP = 8        /* mm_demag_setup / mm_set_m / mm_set_material missing */
} mm_status;

typedef enum {
    MM_FP64 = 0,            /* every array and all arithmetic in double          */
    MM_FP32_FIELDS = 1      /* m, fields, FFT and stencil in float; the Newell
                               tensor is built in double, reductions, the DP45
                               error norm and time are accumulated in double     */
} mm_precision;

/* Explicit Runge-Kutta methods (Sec. 3): classic RK4 (fixed step), Dormand-
 * Prince 5(4) with first-same-as-last, and Runge-Kutta-Fehlberg 4(5) -- the
 * paper's default solver, which propagates the fourth-order solution and uses
 * the fifth-order one only for the error.  The adaptive two share the error
 * norm max |y_hi - y_lo| / (rtol + rtol max(|y_n|, |y_prop|)), accept if
 * <= 1, and the step factor min(5, max(0.2, 0.9 err^-1/5)). */
typedef enum { MM_RK4 = 0, MM_DP45 = 1, MM_RKF45 = 2 } mm_method;

/* DMI types of the paper's table (Sec. 4.3), by their DMI vectors
 * (e_x, e_y, e_z): interface (e_y, -e_x, 0), bulk (e_x, e_y, e_z),
 * D2d (-e_x, e_y, 0). */
typedef enum { MM_DMI_NONE = 0, MM_DMI_INTERFACE = 1, MM_DMI_BULK = 2, MM_DMI_D2D = 3 } mm_dmi_kind;

typedef struct {
    int nx, ny, nz;          /* cells per axis, each >= 1, nx*ny*nz < 2^31       */
    double dx, dy, dz;       /* cell size in metres, > 0                         */
} mm_grid;

/* Material (Sec. 2 material dict; Sec. 4.1, 4.2, Eq. llg).  Each scalar is
 * used for every cell unless the matching per-cell pointer is non-NULL.
 * Easy axis: ku_axis for every cell, or, if grain_id is non-NULL, row
 * grain_id[c] of ku_axis_table (ngrains x 3 doubles, unit vectors).
 * All pointers are host or device memory according to the flag passed to
 * mm_set_material; the data is copied into the state. */
typedef struct {
    double Ms;               /* saturation magnetisation, A/m                    */
    double A;                /* exchange constant, J/m                            */
    double Ku1;              /* first-order uniaxial anisotropy constant, J/m^3  */
    double alpha;            /* Gilbert damping                                  */
    double ku_axis[3];       /* unit easy axis                                   */
    const double* Ms_cell;   /* nx*ny*nz or NULL                                 */
    const double* A_cell;
    const double* Ku1_cell;
    const double* alpha_cell;
    const double* ku_axis_table;  /* ngrains x 3 or NULL                         */
    const uint8_t* grain_id;      /* nx*ny*nz or NULL                            */
    int ngrains;                  /* 1..256 when grain_id is given               */
} mm_material;

/* Uniform time-dependent external field h(t) in A/m, evaluated on the host at
 * every stage time t (seconds). */
typedef void (*mm_field_fn)(double t, double h_out[3], void* user);

/* Create a state for one grid.  cuda_stream is a cudaStream_t (NULL allowed).
 * Allocates the state's device buffers on the current device.  Padded FFT
 * extents are the next power of two >= 2 n per axis (1 for an axis with one
 * cell); each padded extent must be <= 4096.  Fails with MM_EINVAL for bad
 * sizes, MM_ENOMEM if the buffers do not fit. */
mm_status mm_state_create(const mm_grid* grid, mm_precision precision, void* cuda_stream,
                          mm_state** out);

/* Release every buffer of the state (NULL is a no-op).  Synchronises its stream. */
void mm_state_destroy(mm_state* s);

/* Copy the material into the state (Sec. 2 material dict; Sec. 4.1, 4.2).
 * ptrs_on_device: 0 = host pointers, 1 = device pointers.  Checks Ms >= 0,
 * A >= 0, alpha >= 0 for the scalar values and ngrains in 1..256. */
mm_status mm_set_material(mm_state* s, const mm_material* mat, int ptrs_on_device);

/* Copy m (SoA [3][nz][ny][nx], the state's real type) into the state.  The
 * values are taken as given (no normalisation).  Resets the DP45 first stage. */
mm_status mm_set_m(mm_state* s, const void* m, int on_device);

/* Copy the state's m out (same layout and type).  A host copy synchronises. */
mm_status mm_get_m(const mm_state* s, void* m_out, int on_device);

/* External field (Zeeman): h_i(t) = w_i * h(t), with h(t) = fn(t) if fn is
 * non-NULL, else h_const (A/m).  weight: nx*ny*nz doubles or NULL (w = 1),
 * host or device according to on_device. */
mm_status mm_set_zeeman(mm_state* s, const double h_const[3], mm_field_fn fn, void* user,
                        const double* weight, int on_device);

/* Build the demag tensor (Sec. 4.4): Newell's cell-averaged tensor where the
 * Chebyshev cell distance is <= p_newell, the point dipole of Eq. dipole
 * beyond (p_newell < 0: Newell everywhere), in double precision on the host,
 * then its real, six-component Fourier spectrum over the padded grid, scaled
 * by -1/(Px Py Pz) and stored on the device in the state's real type.
 * A state without this call has no demag term (MM_ENOTSETUP from mm_heff and
 * the integrators unless mm_demag_disable was called). */
mm_status mm_demag_setup(mm_state* s, int p_newell);

/* Run without a demag term (tests and macrospin problems). */
mm_status mm_demag_disable(mm_state* s);

/* One effective-field evaluation (Sec. 4) at time t on m (device pointer in
 * the state's layout and type, or NULL for the state's m).  h_out: device
 * buffer for the total field or NULL.  E_out: host array of 5 doubles or NULL,
 * receives (E_demag, E_exchange, E_anisotropy, E_zeeman, E_dmi) in joules
 * (Eq. linear_energy_discrete for the linear terms, -mu0 V sum Ms m.h for
 * Zeeman); asking for E_out synchronises the stream.  torque_out: host double
 * or NULL, receives max over cells of |m x h| / Ms (synchronises).  When
 * E_out or torque_out is asked for and a cell's field or torque is not
 * finite, the call returns MM_ENONFINITE (h_out and the scalars are still
 * written). */
mm_status mm_heff(mm_state* s, const void* m, void* h_out, double E_out[5], double t,
                  double* torque_out);

/* Right-hand side of the LLG equation (Eq. llg) at time t for m (device
 * pointer in the state's layout and type, or NULL for the state's m):
 * k = -gamma/(1+alpha^2) [m x h + alpha m x (m x h)] with h the field of
 * mm_heff (without the precession term if mm_set_llg_options switched it
 * off), written to k_out (device, [3][nz][ny][nx] real).  For an FP32 state
 * whose RK4 steps run the fused stage kernel (uniform material) this takes
 * the same kernels, so k is the stage derivative those steps use.  The state's
 * m and its integrator history are left unchanged; enqueue only.  Cells with
 * Ms = 0 get k = 0.  MM_EINVAL for a null k_out, MM_ENOTSETUP as mm_heff. */
mm_status mm_llg_rhs(mm_state* s, const void* m, void* k_out, double t);

/* Advance the state by one step of the LLG equation (Eq. llg).
 * MM_RK4: one classic RK4 step of size *dt_inout from *t_inout (four field
 *   evaluations; enqueue only, no synchronisation).
 * MM_DP45: Dormand-Prince 5(4) with first-same-as-last; tries *dt_inout,
 *   shrinks it until the error norm max |y5 - y4| / (rtol + rtol max(|y_n|,|y5|))
 *   is <= 1, returns with the step accepted, *dt_inout set to the proposed next
 *   step (dt * min(5, max(0.2, 0.9 err^-1/5))).  Synchronises once per attempt
 *   to read the error norm.  MM_ESTEP if dt falls below 1e-22 s.
 * MM_RKF45: Runge-Kutta-Fehlberg 4(5), same contract as MM_DP45; the
 *   fourth-order solution is propagated and the error is measured against it
 *   (no first-same-as-last stage: the first stage is evaluated at the new m).
 * On return *t_inout is advanced by the step taken.  m is renormalised to
 * unit length after each step.  MM_ENONFINITE if the step produced NaN/Inf
 * (adaptive methods only; RK4 checks nothing to stay asynchronous). */
mm_status mm_llg_step(mm_state* s, mm_method method, double* dt_inout, double rtol,
                      double* t_inout);

/* Relax (Sec. 3): DP45 (or RKF45, see mm_set_llg_options) steps with the
 * material's damping until max_i |m_i x h_i| / Ms_i < tol (DP45: the field of
 * the last stage of the accepted step; RKF45: the field at the new m, which is
 * the next step's first stage), or max_steps accepted steps (then
 * MM_ENOTCONVERGED).  Starts from
 * dt = *dt_inout (1e-13 s if *dt_inout <= 0) and time *t_inout; both are
 * updated.  steps_out, torque_out: host outputs or NULL. */
mm_status mm_relax(mm_state* s, double tol, int max_steps, double rtol, double* dt_inout,
                   double* t_inout, int* steps_out, double* torque_out);

/* Discrete adjoint of one RK4 step of mm_llg_step (Eq. llg, Sec. 3; the
 * gradient Sec. 5.2 obtains with autograd), written by hand.  For the step
 * m_{n+1} = Phi(m_n) of size dt from time t with the state's material, field
 * and demag settings (renormalisation included):
 *   lambda_n       = (dPhi/dm_n)^T lambda_np1
 *   grad_Ms_accum += (dPhi/dMs)^T lambda_np1   (per cell; NULL to skip)
 * The demag part uses that the convolution is its own transpose, the exchange
 * and DMI parts that their link sums are symmetric; the precession switch of
 * mm_set_llg_options is honoured.  All four arrays are device memory in the
 * state's layout and real type (grad_Ms_accum has nx*ny*nz values); lambda_n
 * must not alias the inputs.  The step's stage inputs and fields are
 * recomputed from m_n (no forward state is kept).  MM_EINVAL for
 * non-equidistant layers (not covered).  Enqueues only. */
mm_status mm_llg_step_adjoint(mm_state* s, const void* m_n, const void* lambda_np1, void* lambda_n,
                              void* grad_Ms_accum, double dt, double t);

/* ---- Batched relaxation (served requests) ----
 * A batch holds up to `capacity` grids of one shape (nx, ny, nz, cell size),
 * each a "slot" with its own uniform Ms, A, alpha, optional uniform DMI and
 * precession switch (mm_batch_set_slot_terms), magnetisation and
 * Dormand-Prince step, relaxed as in mm_relax (Sec. 3: integrate with the
 * material's damping until max |m x h| / Ms < tol).  The demag tensor
 * spectrum is built once per batch (the size bucket's plan) and shared by
 * all slots; the stacked grids go through the same FFT passes as one larger
 * problem, and every slot's arithmetic is private (its own reductions in a
 * fixed order), so a slot's result does not depend on the other slots.
 * Device buffers are allocated at creation: mm_batch_footprint gives their
 * size for admission control.  All work of a batch runs on its stream. */
typedef struct mm_batch mm_batch;

/* Bytes of device memory mm_batch_create allocates for this shape and capacity. */
size_t mm_batch_footprint(const mm_grid* grid, mm_precision precision, int capacity);

/* Create a batch (builds the Newell/dipole tensor spectrum with radius p_newell). */
mm_status mm_batch_create(const mm_grid* grid, mm_precision precision, int capacity, int p_newell,
                          void* cuda_stream, mm_batch** out);
void mm_batch_destroy(mm_batch* b);

/* Load a request into a free slot: uniform material, m0 ([3][nz][ny][nx], the
 * batch's real type, host or device), first step dt0 (<= 0: 1e-13 s).
 * MM_EINVAL if the slot is out of range or busy. */
mm_status mm_batch_set_slot(mm_batch* b, int slot, double Ms, double A, double alpha, const void* m0,
                            int on_device, double dt0);

/* Field terms of a freshly loaded slot (after mm_batch_set_slot, before the
 * next mm_batch_begin): the DMI term of Sec. 4.3 with `dmi_kind`
 * (mm_dmi_kind) and a uniform D in J/m^2, as mm_set_dmi defines it (D = 0
 * or MM_DMI_NONE: no DMI), and the precession switch of Sec. 3 (0: the m x h
 * summand is left out, as mm_set_llg_options does).  mm_batch_set_slot
 * resets both (no DMI, precession on).  Synchronises the batch's stream.
 * MM_EINVAL for a slot that is not freshly loaded, a bad kind or a
 * non-finite D. */
mm_status mm_batch_set_slot_terms(mm_batch* b, int slot, int dmi_kind, double D, int precession);

/* Free a slot (any state); its next request may be loaded at once. */
mm_status mm_batch_clear_slot(mm_batch* b, int slot);

/* Enqueue `attempts` (1..1024) consecutive DP45 attempts for every running
 * slot, asynchronously on the batch's stream, preceded by the first-stage
 * evaluation of newly loaded slots.  Every decision is taken on the device,
 * per slot, with mm_llg_step's DP45 rule (error norm with atol = rtol, accept
 * if err <= 1, dt <- dt min(5, max(0.2, 0.9 err^-1/5))): a slot whose torque
 * max |m x h| / Ms falls below tol becomes 2 (converged) and takes no further
 * steps, 3 = max_steps accepted steps reached, 4 = failed (non-finite values
 * or step underflow).  The attempts are captured once per (number of launched
 * slots, attempts, rtol, tol, max_steps) into a CUDA graph and replayed; a
 * stream that cannot be captured (the legacy default stream) gets the same
 * launches directly.  Slots may not be loaded, cleared or read until
 * mm_batch_end. */
mm_status mm_batch_begin(mm_batch* b, int attempts, double rtol, double tol, int max_steps);

/* Non-blocking: *ready = 1 once the work of mm_batch_begin has finished on
 * the device (mm_batch_end will not wait), else 0.  MM_EINVAL if nothing is in
 * flight. */
mm_status mm_batch_query(mm_batch* b, int* ready);

/* Wait for the work of mm_batch_begin and report every slot: status (0 empty,
 * 1 running, 2/3/4 as above), accepted steps and last torque; host arrays of
 * `capacity` entries or NULL.  MM_EINVAL if nothing is in flight. */
mm_status mm_batch_end(mm_batch* b, int* status, int* steps, double* torque);

/* Copy a slot's magnetisation out (host copies synchronise). */
mm_status mm_batch_get_m(mm_batch* b, int slot, void* m_out, int on_device);

/* DMI field (Sec. 4.3): h_i = 2/(mu0 Ms_i) sum_{k=+-x,+-y,+-z} Dt_{i,k}
 * e_k x m_{i+k} / (2 d_k), e_{-k} = -e_k, with the DMI vectors of `kind`; a
 * neighbour outside the grid is left out.  D in J/m^2 for every cell, or
 * D_cell (nx*ny*nz doubles, [nz][ny][nx], host or device per on_device,
 * copied) per cell, each link then taking the average Dt of Eq. D_avg (the
 * harmonic mean for equal signs; for opposite signs the geometric mean of the
 * geometric and the arithmetic mean, with the sign of the sum).  Its energy
 * is the fifth entry of mm_heff's E_out.  MM_DMI_NONE switches the term off.
 * mm_llg_step_adjoint differentiates through it.  MM_EINVAL for an unknown
 * kind or a non-finite D. */
mm_status mm_set_dmi(mm_state* s, mm_dmi_kind kind, double D, const double* D_cell, int on_device);

/* Non-equidistant layers (Sec. 4.4): the grid's nz cells along z become
 * layers of thickness h[0..nz-1] (metres, host array of nz doubles, copied),
 * stacked without gaps from the bottom; the grid's dz is then unused.  Demag
 * keeps the zero-padded FFT along x and y and couples the layers densely at
 * every lateral wave number, with Newell's cell average for boxes of
 * different thickness (the z stencil F(Z0) - F(Z0+h_i) - F(Z0-h_j) +
 * F(Z0+h_i-h_j), divided by the target volume) within a Chebyshev distance p
 * of (lateral offset, layer offset) and the source cell's point dipole
 * beyond.  Exchange between layers k and k+1 is
 * 2 A_link (m_{k+1} - m_k) / (mu0 Ms_k h_k (h_k + h_{k+1}) / 2) with the A of
 * the two half cells in series, A_link = (h_k + h_{k+1}) A_k A_{k+1} /
 * (h_k A_{k+1} + h_{k+1} A_k); energies use each cell's volume dx dy h_k.
 * The demag tensor must be built again (mm_demag_setup) after this call; h =
 * NULL returns to the equidistant grid.  Not with DMI (mm_set_dmi refuses
 * either order), not in the adjoint, always through the unfused stage path.
 * MM_EINVAL unless nz equals the grid's nz, 2 <= nz <= 64 and every h is
 * finite and > 0. */
mm_status mm_set_layers(mm_state* s, const double* h, int nz);

/* Integrator options (Sec. 3): relax_method is the adaptive method mm_relax
 * uses (MM_DP45, the default, or MM_RKF45); precession = 0 drops the m x h
 * term of Eq. llg for every integrator of this state (the damping term keeps
 * its factor gamma alpha / (1 + alpha^2)), as for ground-state searches;
 * 1 (the default) restores it; mm_llg_step_adjoint follows the setting.
 * MM_EINVAL for other values. */
mm_status mm_set_llg_options(mm_state* s, mm_method relax_method, int precession);

/* Diagnostic (the paper has no counterpart): enqueue on the state's stream
 * one CTA that waits on an mbarrier nothing ever completes, polling it at most
 * `spins` times the way the TMA kernels wait for their copies.  When the
 * budget runs out the kernel writes the timeout code into the state's device
 * error word and returns, as a kernel whose copy never landed would; the next
 * call that reads results from this state (mm_heff with energies or torque,
 * a DP45 step, mm_relax) then returns MM_ETIMEOUT, and so does every later
 * one: destroy the state.  The GPU context stays usable.  MM_EINVAL if
 * spins < 1. */
mm_status mm_selftest_wait_timeout(mm_state* s, unsigned spins);

/* Measurement helper (the paper has no counterpart): enqueue on cuda_stream
 * (NULL = legacy default stream) a kernel of `blocks` CTAs x 256 threads in
 * which every thread runs 8 independent chains of `iters` dependent FP64
 * fused multiply-adds, and return in *flops_out the FLOPs it performs
 * (2 per FMA).  Timed by the caller with CUDA events on that stream, it gives
 * the FP64 FMA rate the plain-FP64 path is compared with.  sink: device
 * pointer to one double, never written in practice (it keeps the work
 * alive).  Changes no GPU setting.  MM_EINVAL for a null pointer,
 * blocks outside 1..2^20 or iters < 1; MM_ECUDA if the launch fails. */
mm_status mm_probe_fp64_fma(void* cuda_stream, double* sink, int blocks, int iters, double* flops_out);

/* Host-only helper (no GPU): the padded FFT extent the library uses along an
 * axis of n cells (Sec. 4.4 zero padding, P >= 2n): 1 for n = 1, otherwise the
 * smallest even 7-smooth length 2^a 3^b 5^c 7^d >= 2n up to 3200, and above
 * that the next power of two (grids needing more than 4096 are refused by
 * mm_state_create).  Powers of two and the lengths r 2^a with r = 3, 7, 25
 * run compiled FFT engines; every other such length runs the runtime-plan
 * passes.  0 for n < 1. */
int mm_fft_extent(int n);

/* Host-only helper (no GPU): the real-space demag tensor this library builds
 * (Sec. 4.4, same rule as mm_demag_setup) for every cell offset, as
 * 6 x (2nx-1) x (2ny-1) x (2nz-1) doubles, components (xx, xy, xz, yy, yz, zz),
 * offset (i, j, k) at [c][i+nx-1][j+ny-1][k+nz-1].  out must hold that many. */
mm_status mm_demag_tensor_host(const mm_grid* grid, int p_newell, double* out);

/* Host-only helper (no GPU): the real Fourier spectrum mm_demag_setup builds,
 * over the padded grid Px x Py x Pz of mm_state_create, for the octant
 * kz <= Pz/2, ky <= Py/2, kx <= Px/2, as 6 x (Pz/2+1) x (Py/2+1) x (Px/2+1)
 * doubles (kx fastest), already multiplied by -1/(Px Py Pz). */
mm_status mm_demag_spectrum_host(const mm_grid* grid, int p_newell, double* out);

/* Host-only helper (no GPU): the layer-pair spectrum mm_demag_setup builds
 * after mm_set_layers (Sec. 4.4, non-equidistant layers) for a grid whose nz
 * layers have thicknesses h[0..nz-1] (grid->dz unused), over the padded
 * lateral grid Px x Py of mm_state_create.  Pairs i <= j only, pair index
 * q(i, j) = i nz - i (i - 1) / 2 + j - i, as 6 x npair x (Py/2+1) x (Px/2+1)
 * doubles (kx fastest, npair = nz (nz + 1) / 2), multiplied by -1/(Px Py):
 * xx, xy, yy, zz are the real spectra, xz and yz the value t of the spectrum
 * -i t.  out must hold that many.  MM_EINVAL for a bad grid or thickness. */
mm_status mm_layers_spectrum_host(const mm_grid* grid, const double* h, int p_newell, double* out);

/* Demag field without any memory allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory when
 * they need a field -- frameworks whose allocator owns all device memory and
 * forbids side allocations, or loops that must not stall on the CUDA
 * allocator (cudaMalloc and cudaFree can synchronise the device).
 * It runs the same five FFT passes as mm_heff's demag term on caller buffers:
 *   m        device, [3][nz][ny][nx] in the precision's real type;
 *   Ms_cell  device, nx*ny*nz real values, or NULL to use Ms for every cell;
 *   spectrum device, the layout and values of mm_demag_spectrum_host for this
 *            grid, converted by the caller to the real type;
 *   h_out    device, [3][nz][ny][nx] real: the demag field h = -N * (Ms m) in
 *            every cell (cells with Ms = 0 included, unlike mm_heff).
 * The intermediate spectra live in one fixed 64 MiB device array inside the
 * library (held by every GPU that loads it until the process exits); grids
 * whose spectra need more (about 128x128x32 cells in FP32, half that in FP64)
 * are rejected with MM_EINVAL and a message giving the size needed.  The first
 * call on a device looks up that array's address and uploads the FFT twiddle
 * table (no allocation either); make that first call before any stream
 * capture.  That address is cached per device for the life of the process:
 * do not call this entry point on a device after cudaDeviceReset there.
 * All calls share the one array and it keeps the last call's data:
 * calls whose kernels may overlap on the GPU (different streams without
 * ordering, or several host threads) race on it and must be serialised by the
 * caller.  Enqueues on cuda_stream (NULL = legacy default stream) and returns
 * without synchronising. */
mm_status mm_demag_noalloc(const mm_grid* grid, mm_precision precision, const void* m, const void* Ms_cell,
                           double Ms, const void* spectrum, void* h_out, void* cuda_stream);

/* Padded FFT extents and the row stride of the x-spectrum of a state
 * (out: Px, Py, Pz, Kx = Px/2+1, Kx_stride). */
mm_status mm_state_info(const mm_state* s, int out[5]);

/* Per-kernel timing with CUDA events recorded on the state's stream.
 * mm_profile_enable(s, 1) starts recording (clears totals); 0 stops.
 * mm_profile_read synchronises and returns, for up to max kernels, the name,
 * the launch count and the summed device time in milliseconds. */
mm_status mm_profile_enable(mm_state* s, int on);
int       mm_profile_read(mm_state* s, const char** names, int* counts, double* ms, int max);

/* Thread-local description of the last error (never NULL). */
const char* mm_last_error(void);

/* Library version string. */
const char* mm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MM_H */
