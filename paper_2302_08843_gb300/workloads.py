"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generation only (grids, material maps, initial
states, request streams) and none of the method's arithmetic; the oracle and
the CUDA path both consume what it produces.  Every array is float64 in the
paper's layout: (nx, ny, nz) for scalars, (nx, ny, nz, 3) for vectors
(Sec. 2).  ``to_soa`` / ``from_soa`` convert to and from the library's
structure-of-arrays layout [3][nz][ny][nx] (x fastest).

Workloads (sizes and materials as used for the benchmark and parity tests):

* ``plain_fp64``  : 32x32x4 cells of 2.5x2.5x3 nm, Ms 8e5 A/m, A 1.3e-11 J/m,
                    alpha 0.5, 10 mT along x, random unit m0 (seed 1),
                    RK4 dt 1e-13 s, 200 steps.
* ``thin_film``   : 512x128x1 cells of 3.90625x3.90625x3 nm, Ms 8e5, A 1.3e-11,
                    Ku1 5e3 along x, alpha 0.02, m0 (1,1,1)/sqrt3 + 1% Gaussian
                    tilt (seed 2), 25 mT at 170 deg in-plane, DP45 rtol 1e-5 to 1 ns.
* ``bulk``        : 256x256x64 cells of 2 nm, Ms 1e6, A 1.5e-11, alpha 0.1,
                    Ku1 4e5 with easy axes from 64 Voronoi grains (seed 3),
                    random m0 (seed 3); RK4 dt 5e-14 s.  ``crop`` selects a
                    sub-box of the same maps (e.g. 64x64x16).
* ``inverse_design``: 128x128x1 cells of 5 nm, Ms = sigmoid(w) 8e5 with
                    w ~ N(0, 0.1) (seed 5), A 1.3e-11, alpha 0.05, 5 mT sinc
                    excitation along y in the strip x < 10 cells, m0 = +x.
* ``multilayer``  : 256x256x8 cells of 2x2 nm laterally in 8 layers of
                    unequal thickness (1.0, 0.6, 2.4, 0.8, 1.5, 0.6, 3.0, 1.1 nm,
                    repeated / cut for other nz), alternating materials per
                    layer: thick layers Ms 1.1e6, A 1.6e-11, Ku1 3e5 along z;
                    0.6 nm layers Ms 4e5, A 0.4e-11; the rest Ms 8e5, A 1.3e-11;
                    alpha 0.1, 20 mT along x, random unit m0 (seed 6), RK4 dt 2e-14 s.
* ``serving_stream``: 512 relax requests, Poisson arrivals (mean 2 ms, seed 4),
                    grids from {64x64x1, 128x32x4, 100x100x8, 200x50x2, 256x256x1},
                    3 nm cubes, Ms ~ U[6e5, 1.2e6], A ~ U[1e-11, 2e-11], alpha 1.
"""
import math
from dataclasses import dataclass, field
from typing import Callable, Optional, Tuple, Union

import numpy as np

MU0_FOR_INPUTS = 4.0e-7 * math.pi   # only to express the mT inputs in A/m


@dataclass
class Workload:
    name: str
    n: Tuple[int, int, int]
    dx: Tuple[float, float, float]
    Ms: Union[float, np.ndarray]
    A: Union[float, np.ndarray]
    alpha: Union[float, np.ndarray]
    m0: np.ndarray
    Ku1: Union[float, np.ndarray] = 0.0
    ku_axis: Union[Tuple[float, float, float], np.ndarray] = (1.0, 0.0, 0.0)
    grain_id: Optional[np.ndarray] = None          # (nx, ny, nz) uint8
    axis_table: Optional[np.ndarray] = None        # (ngrains, 3)
    h_ext: Union[Tuple[float, float, float], Callable[[float], np.ndarray]] = (0.0, 0.0, 0.0)
    h_ext_weight: Optional[np.ndarray] = None
    dt: float = 1e-13
    steps: int = 1
    method: str = "rk4"
    extra: dict = field(default_factory=dict)

    @property
    def ncells(self):
        return int(self.n[0] * self.n[1] * self.n[2])

    def ku_axis_cells(self):
        """Easy axis per cell, (nx, ny, nz, 3), expanded from the grain table."""
        if self.grain_id is not None:
            return self.axis_table[self.grain_id]
        return np.broadcast_to(np.asarray(self.ku_axis, dtype=np.float64), tuple(self.n) + (3,))


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def to_soa(v):
    """(nx, ny, nz, 3) -> contiguous (3, nz, ny, nx); (nx, ny, nz) -> (nz, ny, nx)."""
    v = np.asarray(v)
    if v.ndim == 4:
        return np.ascontiguousarray(v.transpose(3, 2, 1, 0))
    return np.ascontiguousarray(v.transpose(2, 1, 0))


def from_soa(v):
    """(3, nz, ny, nx) -> (nx, ny, nz, 3); (nz, ny, nx) -> (nx, ny, nz)."""
    v = np.asarray(v)
    if v.ndim == 4:
        return np.ascontiguousarray(v.transpose(3, 2, 1, 0))
    return np.ascontiguousarray(v.transpose(2, 1, 0))


def plain_fp64(seed=1):
    n = (32, 32, 4)
    rng = np.random.default_rng(seed)
    m0 = _unit(rng.normal(size=n + (3,)))
    return Workload("plain_fp64 32x32x4", n, (2.5e-9, 2.5e-9, 3e-9), Ms=8e5, A=1.3e-11,
                    alpha=0.5, m0=m0, h_ext=(0.010 / MU0_FOR_INPUTS, 0.0, 0.0),
                    dt=1e-13, steps=200, method="rk4")


def thin_film(seed=2, n=(512, 128, 1)):
    rng = np.random.default_rng(seed)
    m0 = _unit(np.ones(tuple(n) + (3,)) / math.sqrt(3.0) + 0.01 * rng.normal(size=tuple(n) + (3,)))
    B = 0.025
    ang = math.radians(170.0)
    return Workload("thin_film %dx%dx%d" % tuple(n), tuple(n), (3.90625e-9, 3.90625e-9, 3e-9),
                    Ms=8e5, A=1.3e-11, alpha=0.02, m0=m0, Ku1=5e3, ku_axis=(1.0, 0.0, 0.0),
                    h_ext=(B / MU0_FOR_INPUTS * math.cos(ang), B / MU0_FOR_INPUTS * math.sin(ang), 0.0),
                    dt=1e-13, steps=0, method="dp45", extra={"t_end": 1e-9, "rtol": 1e-5})


def voronoi_grains(n, dx, ngrains, rng, crop=None):
    """Nearest-seed grain id per cell (Euclidean, non-periodic, ties -> lowest
    index) for seeds uniform in the box, and a uniform random unit axis per
    grain.  ``crop`` = ((x0, x1), (y0, y1), (z0, z1)) evaluates only that sub-box."""
    L = np.array([n[0] * dx[0], n[1] * dx[1], n[2] * dx[2]])
    seeds = rng.uniform(size=(ngrains, 3)) * L
    axes = _unit(rng.normal(size=(ngrains, 3)))
    if crop is None:
        crop = ((0, n[0]), (0, n[1]), (0, n[2]))
    xs = (np.arange(crop[0][0], crop[0][1]) + 0.5) * dx[0]
    ys = (np.arange(crop[1][0], crop[1][1]) + 0.5) * dx[1]
    zs = (np.arange(crop[2][0], crop[2][1]) + 0.5) * dx[2]
    gid = np.empty((len(xs), len(ys), len(zs)), dtype=np.uint8)
    for i, x in enumerate(xs):
        X, Y, Z = np.meshgrid([x], ys, zs, indexing="ij")
        d2 = ((X[..., None] - seeds[:, 0]) ** 2 + (Y[..., None] - seeds[:, 1]) ** 2
              + (Z[..., None] - seeds[:, 2]) ** 2)
        gid[i] = np.argmin(d2, axis=-1)[0].astype(np.uint8)
    return gid, axes


def bulk(seed=3, crop=None, n=(256, 256, 64)):
    """Bulk grains workload; ``crop`` = ((x0,x1),(y0,y1),(z0,z1)) gives the same
    construction restricted to a sub-box (its own, smaller, problem)."""
    dx = (2e-9, 2e-9, 2e-9)
    rng = np.random.default_rng(seed)
    gid, axes = voronoi_grains(n, dx, 64, rng, crop=crop)
    if crop is None:
        m0 = _unit(rng.normal(size=tuple(n) + (3,)))
        nn = tuple(n)
    else:
        # draw the full-size state so the crop sees the same values
        full = rng.normal(size=tuple(n) + (3,))
        m0 = _unit(full[crop[0][0]:crop[0][1], crop[1][0]:crop[1][1], crop[2][0]:crop[2][1]])
        nn = tuple(int(c[1] - c[0]) for c in crop)
    return Workload("bulk %dx%dx%d" % nn, nn, dx, Ms=1e6, A=1.5e-11, alpha=0.1, m0=m0,
                    Ku1=4e5, grain_id=gid, axis_table=axes, dt=5e-14, steps=25, method="rk4")


def sinc_pulse(B0=0.005, fc=20e9, t0=50e-12):
    """Scalar excitation B(t) = B0 sinc(2 pi fc (t - t0)) in tesla, sinc(x) = sin(x)/x."""
    def B(t):
        x = 2.0 * math.pi * fc * (t - t0)
        return B0 if x == 0.0 else B0 * math.sin(x) / x
    return B


def inverse_design(seed=5, n=(128, 128, 1), strip=10, out_box=((108, 118), (59, 69))):
    rng = np.random.default_rng(seed)
    w = rng.normal(0.0, 0.1, size=n)
    theta = 1.0 / (1.0 + np.exp(-w))
    m0 = np.zeros(tuple(n) + (3,))
    m0[..., 0] = 1.0
    weight = np.zeros(n)
    weight[:strip] = 1.0
    B = sinc_pulse()
    def h_ext(t):
        return np.array([0.0, B(t) / MU0_FOR_INPUTS, 0.0])
    return Workload("inverse_design %dx%dx%d" % tuple(n), tuple(n), (5e-9, 5e-9, 5e-9),
                    Ms=theta * 8e5, A=1.3e-11, alpha=0.05, m0=m0, h_ext=h_ext,
                    h_ext_weight=weight, dt=5e-14, steps=2000, method="rk4",
                    extra={"w": w, "Ms0": 8e5, "out_box": out_box})


SERVING_GRIDS = ((64, 64, 1), (128, 32, 4), (100, 100, 8), (200, 50, 2), (256, 256, 1))


MULTILAYER_THICKNESS_NM = (1.0, 0.6, 2.4, 0.8, 1.5, 0.6, 3.0, 1.1)


def multilayer(seed=6, n=(256, 256, 8)):
    """Non-equidistant stack; the thicknesses are in ``extra["layers"]``."""
    n = tuple(int(v) for v in n)
    nz = n[2]
    h = np.array([MULTILAYER_THICKNESS_NM[k % len(MULTILAYER_THICKNESS_NM)] for k in range(nz)]) * 1e-9
    Ms_l, A_l, Ku_l = np.empty(nz), np.empty(nz), np.empty(nz)
    for k in range(nz):
        if h[k] >= 1.5e-9:
            Ms_l[k], A_l[k], Ku_l[k] = 1.1e6, 1.6e-11, 3e5
        elif h[k] <= 0.6e-9:
            Ms_l[k], A_l[k], Ku_l[k] = 4e5, 0.4e-11, 0.0
        else:
            Ms_l[k], A_l[k], Ku_l[k] = 8e5, 1.3e-11, 0.0
    shape = n
    rng = np.random.default_rng(seed)
    m0 = _unit(rng.normal(size=n + (3,)))
    return Workload("multilayer %dx%dx%d" % n, n, (2e-9, 2e-9, float(h.mean())),
                    Ms=np.broadcast_to(Ms_l, shape).copy(), A=np.broadcast_to(A_l, shape).copy(),
                    alpha=0.1, m0=m0, Ku1=np.broadcast_to(Ku_l, shape).copy(), ku_axis=(0.0, 0.0, 1.0),
                    h_ext=(0.020 / MU0_FOR_INPUTS, 0.0, 0.0), dt=2e-14, steps=1, method="rk4",
                    extra={"layers": h})


def serving_stream(seed=4, count=512, mean_gap=2e-3):
    """List of (arrival_time_s, Workload) relax requests."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(mean_gap, size=count)
    arrivals = np.cumsum(gaps) - gaps[0]
    reqs = []
    for i in range(count):
        n = SERVING_GRIDS[int(rng.integers(len(SERVING_GRIDS)))]
        Ms = float(rng.uniform(6e5, 1.2e6))
        A = float(rng.uniform(1e-11, 2e-11))
        m0 = _unit(rng.normal(size=n + (3,)))
        reqs.append((float(arrivals[i]), Workload("request %d %dx%dx%d" % ((i,) + n), n,
                                                   (3e-9, 3e-9, 3e-9), Ms=Ms, A=A, alpha=1.0,
                                                   m0=m0, method="relax",
                                                   extra={"tol": 1e-3, "max_steps": 20000})))
    return reqs
