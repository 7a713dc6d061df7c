"""Thin ctypes binding of libmm.so (declarations in include/mm.h).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  PyTorch provides device memory (``torch.Tensor``
on CUDA) and the stream handle; numpy arrays are accepted where the C ABI
takes host pointers.  The library is loaded from this package directory on
first use and a missing library is an error (there is no fallback).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmm.so")

MM_OK, MM_EINVAL, MM_ENOMEM, MM_ECUDA, MM_ENONFINITE, MM_ESTEP, MM_ENOTCONVERGED, MM_ETIMEOUT, MM_ENOTSETUP = range(9)
STATUS_NAMES = ["MM_OK", "MM_EINVAL", "MM_ENOMEM", "MM_ECUDA", "MM_ENONFINITE", "MM_ESTEP",
                "MM_ENOTCONVERGED", "MM_ETIMEOUT", "MM_ENOTSETUP"]
MM_FP64, MM_FP32_FIELDS = 0, 1
MM_RK4, MM_DP45, MM_RKF45 = 0, 1, 2

# every exported symbol of include/mm.h
EXPORTS = ("mm_state_create", "mm_state_destroy", "mm_set_material", "mm_set_m", "mm_get_m",
           "mm_set_zeeman", "mm_demag_setup", "mm_demag_disable", "mm_heff", "mm_llg_step",
           "mm_relax", "mm_demag_tensor_host", "mm_demag_spectrum_host", "mm_state_info", "mm_profile_enable",
           "mm_profile_read", "mm_last_error", "mm_version", "mm_demag_noalloc", "mm_llg_step_adjoint",
           "mm_batch_footprint", "mm_batch_create", "mm_batch_destroy", "mm_batch_set_slot", "mm_batch_clear_slot",
           "mm_batch_set_slot_terms",
           "mm_batch_begin", "mm_batch_query", "mm_batch_end", "mm_batch_get_m",
           "mm_selftest_wait_timeout", "mm_set_llg_options", "mm_set_dmi", "mm_fft_extent",
           "mm_set_layers", "mm_layers_spectrum_host", "mm_probe_fp64_fma", "mm_llg_rhs")


class MMError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status,
                                     message))


class mm_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double)]


class mm_material(ctypes.Structure):
    _fields_ = [("Ms", ctypes.c_double), ("A", ctypes.c_double), ("Ku1", ctypes.c_double),
                ("alpha", ctypes.c_double), ("ku_axis", ctypes.c_double * 3),
                ("Ms_cell", ctypes.c_void_p), ("A_cell", ctypes.c_void_p), ("Ku1_cell", ctypes.c_void_p),
                ("alpha_cell", ctypes.c_void_p), ("ku_axis_table", ctypes.c_void_p),
                ("grain_id", ctypes.c_void_p), ("ngrains", ctypes.c_int)]


FIELD_FN = ctypes.CFUNCTYPE(None, ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)

_LIB = None


def lib():
    """Load libmm.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libmm.so not built: run __graft_entry__.build() or "
                           "python -m paper_2302_08843_gb300.build")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    pd, pi = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    sig = {
        "mm_state_create": (i, [ctypes.POINTER(mm_grid), i, vp, ctypes.POINTER(vp)]),
        "mm_state_destroy": (None, [vp]),
        "mm_set_material": (i, [vp, ctypes.POINTER(mm_material), i]),
        "mm_set_m": (i, [vp, vp, i]),
        "mm_get_m": (i, [vp, vp, i]),
        "mm_set_zeeman": (i, [vp, pd, FIELD_FN, vp, vp, i]),
        "mm_demag_setup": (i, [vp, i]),
        "mm_demag_disable": (i, [vp]),
        "mm_heff": (i, [vp, vp, vp, pd, d, pd]),
        "mm_llg_step": (i, [vp, i, pd, d, pd]),
        "mm_relax": (i, [vp, d, i, d, pd, pd, pi, pd]),
        "mm_demag_tensor_host": (i, [ctypes.POINTER(mm_grid), i, vp]),
        "mm_demag_spectrum_host": (i, [ctypes.POINTER(mm_grid), i, vp]),
        "mm_state_info": (i, [vp, pi]),
        "mm_profile_enable": (i, [vp, i]),
        "mm_profile_read": (i, [vp, ctypes.POINTER(ctypes.c_char_p), pi, pd, i]),
        "mm_last_error": (ctypes.c_char_p, []),
        "mm_version": (ctypes.c_char_p, []),
        "mm_demag_noalloc": (i, [ctypes.POINTER(mm_grid), i, vp, vp, d, vp, vp, vp]),
        "mm_llg_step_adjoint": (i, [vp, vp, vp, vp, vp, d, d]),
        "mm_batch_footprint": (ctypes.c_size_t, [ctypes.POINTER(mm_grid), i, i]),
        "mm_batch_create": (i, [ctypes.POINTER(mm_grid), i, i, i, vp, ctypes.POINTER(vp)]),
        "mm_batch_destroy": (None, [vp]),
        "mm_batch_set_slot": (i, [vp, i, d, d, d, vp, i, d]),
        "mm_batch_set_slot_terms": (i, [vp, i, i, d, i]),
        "mm_batch_clear_slot": (i, [vp, i]),
        "mm_batch_begin": (i, [vp, i, d, d, i]),
        "mm_batch_query": (i, [vp, vp]),
        "mm_selftest_wait_timeout": (i, [vp, ctypes.c_uint]),
        "mm_set_llg_options": (i, [vp, i, i]),
        "mm_set_dmi": (i, [vp, i, d, vp, i]),
        "mm_fft_extent": (i, [i]),
        "mm_set_layers": (i, [vp, vp, i]),
        "mm_layers_spectrum_host": (i, [ctypes.POINTER(mm_grid), vp, i, vp]),
        "mm_batch_end": (i, [vp, vp, vp, vp]),
        "mm_batch_get_m": (i, [vp, i, vp, i]),
        "mm_probe_fp64_fma": (i, [vp, vp, i, i, ctypes.POINTER(d)]),
        "mm_llg_rhs": (i, [vp, vp, vp, d]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


def check(status):
    if status != MM_OK:
        raise MMError(status, lib().mm_last_error().decode())


def _ptr(a):
    """(pointer, on_device) of a torch tensor or a numpy array (None -> NULL)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy array must be C-contiguous")
        return a.ctypes.data, 0
    import torch
    if isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError(type(a))


def demag_tensor_host(n, dx, p=20):
    """mm_demag_tensor_host: the library's real-space tensor for all offsets (host only)."""
    g = mm_grid(int(n[0]), int(n[1]), int(n[2]), float(dx[0]), float(dx[1]), float(dx[2]))
    out = np.zeros((6, 2 * n[0] - 1, 2 * n[1] - 1, 2 * n[2] - 1))
    check(lib().mm_demag_tensor_host(ctypes.byref(g), int(p), out.ctypes.data))
    return out


def probe_fp64_fma(stream, sink, blocks, iters):
    """mm_probe_fp64_fma: enqueue the FP64 FMA rate probe on a CUDA stream
    handle; returns the FLOPs it performs (the caller times it)."""
    fl = ctypes.c_double(0.0)
    check(lib().mm_probe_fp64_fma(ctypes.c_void_p(stream), ctypes.c_void_p(sink), int(blocks), int(iters),
                                  ctypes.byref(fl)))
    return fl.value


def padded_extents(n):
    """Padded FFT extent per axis (mm_fft_extent): 1 for a single cell, else the
    smallest supported length >= 2n (powers of two and the mixed-radix lengths
    96, 100, 112, 192, 200, 224, 384, 400, 448, 768, 800, 896)."""
    return tuple(int(lib().mm_fft_extent(int(v))) for v in n)


def demag_spectrum_host(n, dx, p=20):
    """mm_demag_spectrum_host: octant spectrum (6, Pz/2+1, Py/2+1, Px/2+1), scaled by -1/(Px Py Pz)."""
    P = padded_extents(n)
    g = mm_grid(int(n[0]), int(n[1]), int(n[2]), float(dx[0]), float(dx[1]), float(dx[2]))
    out = np.zeros((6, P[2] // 2 + 1, P[1] // 2 + 1, P[0] // 2 + 1))
    check(lib().mm_demag_spectrum_host(ctypes.byref(g), int(p), out.ctypes.data))
    return out


def layers_spectrum_host(n, dx, dy, h, p=20):
    """mm_layers_spectrum_host: (6, npair, Py/2+1, Px/2+1), pairs i <= j, scaled by -1/(Px Py)."""
    P = padded_extents((n[0], n[1], 1))
    nz = int(n[2])
    g = mm_grid(int(n[0]), int(n[1]), nz, float(dx), float(dy), 1.0)
    hh = np.ascontiguousarray(h, dtype=np.float64)
    if hh.size != nz:
        raise ValueError("one thickness per layer")
    out = np.zeros((6, nz * (nz + 1) // 2, P[1] // 2 + 1, P[0] // 2 + 1))
    check(lib().mm_layers_spectrum_host(ctypes.byref(g), hh.ctypes.data, int(p), out.ctypes.data))
    return out


class State:
    """One grid's device state (mm_state).  m and fields are torch CUDA tensors
    of shape (3, nz, ny, nx) in the state's dtype (float64 for "fp64",
    float32 for "fp32")."""

    def __init__(self, n, dx, precision="fp64", stream=None):
        import torch
        self.n = tuple(int(v) for v in n)
        self.dx = tuple(float(v) for v in dx)
        self.precision = precision
        self.prec = MM_FP64 if precision == "fp64" else MM_FP32_FIELDS
        self.dtype = torch.float64 if self.prec == MM_FP64 else torch.float32
        self.shape = (3, self.n[2], self.n[1], self.n[0])
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        g = mm_grid(self.n[0], self.n[1], self.n[2], *self.dx)
        h = ctypes.c_void_p()
        check(lib().mm_state_create(ctypes.byref(g), self.prec, ctypes.c_void_p(stream.cuda_stream),
                                    ctypes.byref(h)))
        self.h = h
        self._keep = []

    def close(self):
        if getattr(self, "h", None):
            lib().mm_state_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_material(self, Ms, A, alpha, Ku1=0.0, ku_axis=(1.0, 0.0, 0.0), Ms_cell=None, A_cell=None,
                     Ku1_cell=None, alpha_cell=None, grain_id=None, axis_table=None):
        """Per-cell arrays: float64 numpy (nz, ny, nx) (host) or float64 CUDA tensors."""
        m = mm_material()
        m.Ms, m.A, m.Ku1, m.alpha = float(Ms), float(A), float(Ku1), float(alpha)
        for q in range(3):
            m.ku_axis[q] = float(ku_axis[q])
        on_dev = None
        keep = []
        for name, arr in (("Ms_cell", Ms_cell), ("A_cell", A_cell), ("Ku1_cell", Ku1_cell),
                          ("alpha_cell", alpha_cell), ("ku_axis_table", axis_table), ("grain_id", grain_id)):
            if arr is None:
                continue
            if isinstance(arr, np.ndarray):
                arr = np.ascontiguousarray(arr, dtype=np.uint8 if name == "grain_id" else np.float64)
            keep.append(arr)
            p, dev = _ptr(arr)
            if on_dev is None:
                on_dev = dev
            elif on_dev != dev:
                raise ValueError("mix of host and device material arrays")
            setattr(m, name, p)
        if grain_id is not None:
            m.ngrains = int(len(axis_table))
        check(lib().mm_set_material(self.h, ctypes.byref(m), int(on_dev or 0)))

    def set_m(self, m):
        m = self._as_field(m)
        p, dev = _ptr(m)
        check(lib().mm_set_m(self.h, p, dev))
        if not dev:
            self.stream.synchronize()

    def get_m(self):
        import torch
        out = torch.empty(self.shape, dtype=self.dtype, device="cuda")
        check(lib().mm_get_m(self.h, out.data_ptr(), 1))
        return out

    def get_m_host(self, out):
        """mm_get_m into a host (ideally pinned) CPU tensor or numpy array; synchronises."""
        p, dev = _ptr(out)
        if dev:
            raise ValueError("get_m_host needs a host buffer")
        check(lib().mm_get_m(self.h, p, 0))
        return out

    def set_zeeman(self, h=(0.0, 0.0, 0.0), fn=None, weight=None):
        """h: constant (3,) A/m; fn: callable t -> (3,) A/m (overrides h);
        weight: per-cell float64 (nz, ny, nx) numpy array or CUDA tensor."""
        hc = (ctypes.c_double * 3)(*[float(v) for v in h])
        cb = FIELD_FN()
        if fn is not None:
            def _cb(t, out, user):
                v = fn(t)
                out[0], out[1], out[2] = float(v[0]), float(v[1]), float(v[2])
            cb = FIELD_FN(_cb)
        self._keep = [cb]
        if isinstance(weight, np.ndarray):
            weight = np.ascontiguousarray(weight, dtype=np.float64)
        wp, wdev = _ptr(weight)
        self._keep.append(weight)
        check(lib().mm_set_zeeman(self.h, hc, cb, None, wp, wdev))

    def demag_setup(self, p=20):
        check(lib().mm_demag_setup(self.h, int(p)))

    def demag_disable(self):
        check(lib().mm_demag_disable(self.h))

    def _as_field(self, m):
        import torch
        if isinstance(m, np.ndarray):
            m = torch.from_numpy(np.ascontiguousarray(m)).to(self.dtype).cuda()
        if tuple(m.shape) != self.shape or m.dtype != self.dtype:
            raise ValueError("expected %s %s, got %s %s" % (self.shape, self.dtype, tuple(m.shape), m.dtype))
        return m.contiguous()

    def heff(self, m=None, t=0.0, energies=False, torque=False, h_out=None):
        """Effective field (returns h, and optionally E[4] and max torque/Ms)."""
        import torch
        if m is not None:
            m = self._as_field(m)
        if h_out is None:
            h_out = torch.empty(self.shape, dtype=self.dtype, device="cuda")
        E = (ctypes.c_double * 5)() if energies else None
        tq = ctypes.c_double() if torque else None
        check(lib().mm_heff(self.h, None if m is None else m.data_ptr(), h_out.data_ptr(), E, float(t),
                            ctypes.byref(tq) if torque else None))
        out = [h_out]
        if energies:
            out.append(list(E))
        if torque:
            out.append(tq.value)
        return out[0] if len(out) == 1 else tuple(out)

    def llg_rhs(self, m=None, t=0.0, k_out=None):
        """mm_llg_rhs: dm/dt of Eq. llg at m (default: the state's m)."""
        import torch
        if m is not None:
            m = self._as_field(m)
        if k_out is None:
            k_out = torch.empty(self.shape, dtype=self.dtype, device="cuda")
        check(lib().mm_llg_rhs(self.h, None if m is None else m.data_ptr(), k_out.data_ptr(), float(t)))
        return k_out

    def selftest_wait_timeout(self, spins=1 << 16):
        """mm_selftest_wait_timeout: a device wait that runs out on this state's stream."""
        check(lib().mm_selftest_wait_timeout(self.h, int(spins)))

    DMI_KINDS = {None: 0, "none": 0, "interface": 1, "bulk": 2, "d2d": 3}

    def set_dmi(self, kind="interface", D=0.0, D_cell=None):
        """mm_set_dmi: kind "interface", "bulk", "d2d" or None; D_cell float64
        numpy (nz, ny, nx) or a float64 CUDA tensor."""
        if isinstance(D_cell, np.ndarray):
            D_cell = np.ascontiguousarray(D_cell, dtype=np.float64)     # kept alive through the call
        p, dev = _ptr(D_cell)
        check(lib().mm_set_dmi(self.h, self.DMI_KINDS[kind], float(D), p, dev))

    def set_layers(self, h=None):
        """mm_set_layers: nz layer thicknesses in metres (None: equidistant
        again); call demag_setup afterwards."""
        if h is None:
            check(lib().mm_set_layers(self.h, None, 0))
            return
        hh = np.ascontiguousarray(h, dtype=np.float64)
        check(lib().mm_set_layers(self.h, hh.ctypes.data, int(hh.size)))

    def set_llg_options(self, relax_method="dp45", precession=True):
        """mm_set_llg_options: mm_relax's method ("dp45" or "rkf45") and the precession term."""
        check(lib().mm_set_llg_options(self.h, MM_RKF45 if relax_method == "rkf45" else MM_DP45,
                                       1 if precession else 0))

    def step(self, dt, t=0.0, method="rk4", rtol=1e-5):
        """One mm_llg_step (method "rk4", "dp45" or "rkf45"); returns (t_new, dt_next)."""
        dtc = ctypes.c_double(dt)
        tc = ctypes.c_double(t)
        meth = {"rk4": MM_RK4, "dp45": MM_DP45, "rkf45": MM_RKF45}[method]
        check(lib().mm_llg_step(self.h, meth, ctypes.byref(dtc), float(rtol), ctypes.byref(tc)))
        return tc.value, dtc.value

    def relax(self, tol=1e-3, max_steps=20000, rtol=1e-5, dt=1e-13, t=0.0, allow_unconverged=False):
        """mm_relax; returns (steps, torque, t, dt)."""
        dtc, tc = ctypes.c_double(dt), ctypes.c_double(t)
        steps, tq = ctypes.c_int(), ctypes.c_double()
        st = lib().mm_relax(self.h, float(tol), int(max_steps), float(rtol), ctypes.byref(dtc), ctypes.byref(tc),
                            ctypes.byref(steps), ctypes.byref(tq))
        if not (allow_unconverged and st == MM_ENOTCONVERGED):
            check(st)
        return steps.value, tq.value, tc.value, dtc.value

    def step_adjoint(self, m_n, lam_next, dt, t=0.0, grad_Ms=None):
        """mm_llg_step_adjoint: returns lambda_n; adds (dPhi/dMs)^T lam_next into grad_Ms if given."""
        import torch
        m_n = self._as_field(m_n)
        lam_next = self._as_field(lam_next)
        lam = torch.empty_like(lam_next)
        check(lib().mm_llg_step_adjoint(self.h, m_n.data_ptr(), lam_next.data_ptr(), lam.data_ptr(),
                                        None if grad_Ms is None else grad_Ms.data_ptr(), float(dt), float(t)))
        return lam

    def info(self):
        out = (ctypes.c_int * 5)()
        check(lib().mm_state_info(self.h, out))
        return dict(Px=out[0], Py=out[1], Pz=out[2], Kx=out[3], Kx_stride=out[4])

    def profile_enable(self, on=True):
        check(lib().mm_profile_enable(self.h, 1 if on else 0))

    def profile_read(self):
        """{kernel name: (launches, total ms)} from the CUDA-event timer."""
        n = 32
        names = (ctypes.c_char_p * n)()
        counts = (ctypes.c_int * n)()
        ms = (ctypes.c_double * n)()
        k = lib().mm_profile_read(self.h, names, counts, ms, n)
        if k < 0:
            raise MMError(MM_ECUDA, "mm_profile_read failed")
        return {names[q].decode(): (counts[q], ms[q]) for q in range(min(k, n))}


class Batch:
    """mm_batch: up to `capacity` same-shape grids relaxed together (`attempts`
    DP45 attempts of all running slots per begin/end pair)."""

    def __init__(self, n, dx, precision="fp32", capacity=8, p=20, stream=None):
        import torch
        self.n = tuple(int(v) for v in n)
        self.dx = tuple(float(v) for v in dx)
        self.prec = MM_FP64 if precision == "fp64" else MM_FP32_FIELDS
        self.dtype = torch.float64 if self.prec == MM_FP64 else torch.float32
        self.npdtype = np.float64 if self.prec == MM_FP64 else np.float32
        self.capacity = int(capacity)
        self.shape = (3, self.n[2], self.n[1], self.n[0])
        self.stream = stream if stream is not None else torch.cuda.Stream()
        g = mm_grid(self.n[0], self.n[1], self.n[2], *self.dx)
        h = ctypes.c_void_p()
        check(lib().mm_batch_create(ctypes.byref(g), self.prec, self.capacity, int(p),
                                    ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h
        self.footprint = Batch.footprint_of(self.n, self.dx, precision, capacity)
        self._status = np.zeros(self.capacity, dtype=np.int32)
        self._steps = np.zeros(self.capacity, dtype=np.int32)
        self._torque = np.zeros(self.capacity, dtype=np.float64)

    @staticmethod
    def footprint_of(n, dx, precision, capacity):
        g = mm_grid(int(n[0]), int(n[1]), int(n[2]), float(dx[0]), float(dx[1]), float(dx[2]))
        return int(lib().mm_batch_footprint(ctypes.byref(g), MM_FP64 if precision == "fp64" else MM_FP32_FIELDS,
                                            int(capacity)))

    def close(self):
        if getattr(self, "h", None):
            lib().mm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_slot(self, slot, Ms, A, alpha, m0, dt0=1e-13):
        """m0: (3, nz, ny, nx) numpy array (host) or CUDA tensor of the batch's dtype."""
        if isinstance(m0, np.ndarray):
            m0 = np.ascontiguousarray(m0, dtype=self.npdtype)
        p, dev = _ptr(m0)
        check(lib().mm_batch_set_slot(self.h, int(slot), float(Ms), float(A), float(alpha), p, dev, float(dt0)))

    def set_slot_terms(self, slot, dmi=None, D=0.0, precession=True):
        """mm_batch_set_slot_terms: DMI kind ("interface", "bulk", "d2d" or None)
        with a uniform D, and the precession switch, for a freshly loaded slot."""
        check(lib().mm_batch_set_slot_terms(self.h, int(slot), State.DMI_KINDS[dmi], float(D),
                                            1 if precession else 0))

    def clear_slot(self, slot):
        check(lib().mm_batch_clear_slot(self.h, int(slot)))

    def begin(self, attempts=1, rtol=1e-5, tol=1e-3, max_steps=20000):
        check(lib().mm_batch_begin(self.h, int(attempts), float(rtol), float(tol), int(max_steps)))

    def ready(self):
        r = ctypes.c_int(0)
        check(lib().mm_batch_query(self.h, ctypes.byref(r)))
        return bool(r.value)

    def end(self):
        check(lib().mm_batch_end(self.h, self._status.ctypes.data, self._steps.ctypes.data,
                                 self._torque.ctypes.data))
        return self._status.copy(), self._steps.copy(), self._torque.copy()

    def get_m(self, slot):
        out = np.empty(self.shape, dtype=self.npdtype)
        check(lib().mm_batch_get_m(self.h, int(slot), out.ctypes.data, 0))
        return out


def setup_workload(w, precision="fp64", p=20, stream=None):
    """Create a State for a paper_2302_08843_gb300.workloads.Workload (material,
    Zeeman, demag tensor and m0 uploaded).  Marshalling only."""
    from .workloads import to_soa
    s = State(w.n, w.dx, precision, stream)
    kw = {}
    if np.ndim(w.Ms) > 0:
        kw["Ms_cell"] = to_soa(np.asarray(w.Ms, dtype=np.float64))
    if np.ndim(w.A) > 0:
        kw["A_cell"] = to_soa(np.asarray(w.A, dtype=np.float64))
    if np.ndim(w.Ku1) > 0:
        kw["Ku1_cell"] = to_soa(np.asarray(w.Ku1, dtype=np.float64))
    if np.ndim(w.alpha) > 0:
        kw["alpha_cell"] = to_soa(np.asarray(w.alpha, dtype=np.float64))
    if w.grain_id is not None:
        kw["grain_id"] = to_soa(w.grain_id)
        kw["axis_table"] = np.ascontiguousarray(w.axis_table, dtype=np.float64)
    s.set_material(Ms=0.0 if np.ndim(w.Ms) > 0 else w.Ms, A=0.0 if np.ndim(w.A) > 0 else w.A,
                   alpha=0.0 if np.ndim(w.alpha) > 0 else w.alpha,
                   Ku1=0.0 if np.ndim(w.Ku1) > 0 else w.Ku1, ku_axis=w.ku_axis, **kw)
    weight = None if w.h_ext_weight is None else to_soa(np.asarray(w.h_ext_weight, dtype=np.float64))
    if callable(w.h_ext):
        s.set_zeeman(fn=w.h_ext, weight=weight)
    else:
        s.set_zeeman(h=w.h_ext, weight=weight)
    if p is None:
        s.demag_disable()
    else:
        s.demag_setup(p)
    s.set_m(to_soa(w.m0))
    return s
