"""Python access to the plain FP64 CPU oracle (cartogram_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of
the benchmark may use this module; the library's product path never does.
The oracle is compiled with gcc (no FMA contraction, OpenMP when available) into
oracle/_build/liboracle.so by build().
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cartogram_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (seconds). Returns the path of the shared library."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int), ("Ly", ctypes.c_int), ("blur", ctypes.c_double),
                ("dt0", ctypes.c_double), ("atol", ctypes.c_double), ("grow", ctypes.c_double),
                ("shrink", ctypes.c_double), ("cfl", ctypes.c_double), ("rho_tol", ctypes.c_double),
                ("area_tol", ctypes.c_double), ("max_steps", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("blur_decay", ctypes.c_double), ("flow", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("status", ctypes.c_int),
                ("steps_accepted", ctypes.c_longlong), ("steps_rejected", ctypes.c_longlong),
                ("max_area_error", ctypes.c_double), ("t_end_last", ctypes.c_double)]


# Step-control constants of the method as read from the paper (predictor-corrector
# with adaptive steps; stop when the density has equalised). They are stated here
# independently of the CUDA library's defaults; the parity tests pass the same
# values to both sides explicitly.
DEFAULTS = dict(dt0=1e-2, atol=1e-2, grow=1.2, shrink=0.5, cfl=1.0, rho_tol=1e-4,
                area_tol=0.01, max_steps=4000, max_iter=50, blur_decay=0.5, flow=0)


def params(Lx, Ly, blur, **kw) -> Params:
    d = dict(DEFAULTS)
    d.update(kw)
    return Params(Lx, Ly, blur, d["dt0"], d["atol"], d["grow"], d["shrink"], d["cfl"],
                  d["rho_tol"], d["area_tol"], d["max_steps"], d["max_iter"], d["blur_decay"], d["flow"])


_D = ctypes.POINTER(ctypes.c_double)
_LL = ctypes.POINTER(ctypes.c_longlong)
_I = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        L.orc_forward.argtypes = [ctypes.c_int, ctypes.c_int, _D, ctypes.c_double, _D]
        L.orc_fields.argtypes = [ctypes.c_int, ctypes.c_int, _D, ctypes.c_double, _D, _D, _D]
        L.orc_velocity.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, _D]
        L.orc_velocity.restype = ctypes.c_double
        L.orc_interp.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_double, _D, _D]
        L.orc_heun_step.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, ctypes.c_longlong,
                                    _D, _D, ctypes.c_double, _D, _D, _D, _D]
        L.orc_heun_step.restype = ctypes.c_double
        L.orc_integrate.argtypes = [ctypes.POINTER(Params), _D, _D, _D, _LL, _LL, _D, _D, _I, ctypes.c_int]
        L.orc_region_areas.argtypes = [ctypes.c_int, ctypes.c_longlong, _LL, _I, _D, _D]
        L.orc_area_errors.argtypes = [ctypes.c_int, _D, _D, _D]
        L.orc_area_errors.restype = ctypes.c_double
        L.orc_rasterize.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_longlong,
                                    _LL, _I, _D, _D]
        L.orc_map_points.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_longlong, _D, _D]
        L.orc_cartogram.argtypes = [ctypes.POINTER(Params), ctypes.c_int, _D, ctypes.c_longlong, _LL, _I,
                                    ctypes.c_longlong, _D, _D, _D, ctypes.POINTER(Stats)]
        L.orc_flux_linear.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D]
        L.orc_integrate_linear.argtypes = [ctypes.POINTER(Params), _D, _D, _D, _LL, _LL, _D]
        L.orc_distortion.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]
        L.orc_integrate_replay.argtypes = [ctypes.POINTER(Params), _D, _D, ctypes.c_int, _D, _D]
        L.orc_coverage.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_longlong, _LL, _I, _D, _D]
        L.orc_inverse_points.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, ctypes.c_longlong, _D, _D]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def forward(rho: np.ndarray, blur: float) -> np.ndarray:
    rho = _f64(rho)
    Ly, Lx = rho.shape
    out = np.empty_like(rho)
    lib().orc_forward(Lx, Ly, _d(rho), blur, _d(out))
    return out


def fields(spec: np.ndarray, t: float):
    spec = _f64(spec)
    Ly, Lx = spec.shape
    rho = np.empty_like(spec)
    gx = np.empty_like(spec)
    gy = np.empty_like(spec)
    lib().orc_fields(Lx, Ly, _d(spec), float(t), _d(rho), _d(gx), _d(gy))
    return rho, gx, gy


def velocity(rho, gx, gy):
    rho, gx, gy = _f64(rho), _f64(gx), _f64(gy)
    Ly, Lx = rho.shape
    vx = np.empty_like(rho)
    vy = np.empty_like(rho)
    vmax = lib().orc_velocity(Lx, Ly, _d(rho), _d(gx), _d(gy), _d(vx), _d(vy))
    return vx, vy, vmax


def interp(vx, vy, x: float, y: float):
    vx, vy = _f64(vx), _f64(vy)
    Ly, Lx = vx.shape
    ux = ctypes.c_double()
    uy = ctypes.c_double()
    lib().orc_interp(Lx, Ly, _d(vx), _d(vy), float(x), float(y), ctypes.byref(ux), ctypes.byref(uy))
    return ux.value, uy.value


def heun_step(v0x, v0y, v1x, v1y, x, y, h):
    v0x, v0y, v1x, v1y = map(_f64, (v0x, v0y, v1x, v1y))
    x, y = _f64(x), _f64(y)
    Ly, Lx = v0x.shape
    n = x.size
    xp, yp, xc, yc = (np.empty(n) for _ in range(4))
    err = lib().orc_heun_step(Lx, Ly, _d(v0x), _d(v0y), _d(v1x), _d(v1y), n, _d(x), _d(y), float(h),
                              _d(xp), _d(yp), _d(xc), _d(yc))
    return xp, yp, xc, yc, err


@dataclass
class IntegrateResult:
    X: np.ndarray
    Y: np.ndarray
    accepted: int
    rejected: int
    t_end: float
    status: int
    sched_h: np.ndarray
    sched_acc: np.ndarray


def integrate(spec: np.ndarray, blur: float = 0.0, sched_cap: int = 20000, **kw) -> IntegrateResult:
    spec = _f64(spec)
    Ly, Lx = spec.shape
    P = params(Lx, Ly, blur, **kw)
    X = np.empty((Ly, Lx))
    Y = np.empty((Ly, Lx))
    a = ctypes.c_longlong()
    r = ctypes.c_longlong()
    t = ctypes.c_double()
    sh = np.zeros(sched_cap)
    sa = np.zeros(sched_cap, dtype=np.int32)
    st = lib().orc_integrate(ctypes.byref(P), _d(spec), _d(X), _d(Y), ctypes.byref(a), ctypes.byref(r),
                             ctypes.byref(t), _d(sh), sa.ctypes.data_as(_I), sched_cap)
    n = min(a.value + r.value, sched_cap)
    return IntegrateResult(X, Y, a.value, r.value, t.value, st, sh[:n], sa[:n])


def integrate_replay(spec: np.ndarray, steps, **kw):
    """Integration with the fixed accepted step sizes `steps` (no acceptance test)."""
    spec = _f64(spec)
    Ly, Lx = spec.shape
    P = params(Lx, Ly, 0.0, **kw)
    X = np.empty((Ly, Lx))
    Y = np.empty((Ly, Lx))
    h = _f64(np.asarray(steps, dtype=np.float64))
    lib().orc_integrate_replay(ctypes.byref(P), _d(spec), _d(h), int(h.size), _d(X), _d(Y))
    return X, Y


def flux_linear(spec: np.ndarray):
    """Flux (Jx, Jy) of the linear-equalisation flow at the cell centres."""
    spec = _f64(spec)
    Ly, Lx = spec.shape
    jx = np.empty_like(spec)
    jy = np.empty_like(spec)
    lib().orc_flux_linear(Lx, Ly, _d(spec), _d(jx), _d(jy))
    return jx, jy


def integrate_linear(spec: np.ndarray, blur: float = 0.0, **kw) -> IntegrateResult:
    spec = _f64(spec)
    Ly, Lx = spec.shape
    P = params(Lx, Ly, blur, **kw)
    X = np.empty((Ly, Lx))
    Y = np.empty((Ly, Lx))
    a, r, t = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_double()
    st = lib().orc_integrate_linear(ctypes.byref(P), _d(spec), _d(X), _d(Y), ctypes.byref(a), ctypes.byref(r),
                                    ctypes.byref(t))
    return IntegrateResult(X, Y, a.value, r.value, t.value, st, np.zeros(0), np.zeros(0, dtype=np.int32))


def region_areas(n_regions, ring_offsets, ring_region, xy) -> np.ndarray:
    ro = np.ascontiguousarray(ring_offsets, dtype=np.int64)
    rr = np.ascontiguousarray(ring_region, dtype=np.int32)
    xy = _f64(xy)
    out = np.empty(n_regions)
    lib().orc_region_areas(n_regions, rr.size, ro.ctypes.data_as(_LL), rr.ctypes.data_as(_I), _d(xy), _d(out))
    return out


def area_errors(values, areas):
    values, areas = _f64(values), _f64(areas)
    err = np.empty_like(values)
    mx = lib().orc_area_errors(values.size, _d(values), _d(areas), _d(err))
    return err, mx


def rasterize(Lx, Ly, values, areas, ring_offsets, ring_region, xy) -> np.ndarray:
    values, areas, xy = _f64(values), _f64(areas), _f64(xy)
    ro = np.ascontiguousarray(ring_offsets, dtype=np.int64)
    rr = np.ascontiguousarray(ring_region, dtype=np.int32)
    rho = np.empty((Ly, Lx))
    lib().orc_rasterize(Lx, Ly, values.size, _d(values), _d(areas), rr.size, ro.ctypes.data_as(_LL),
                        rr.ctypes.data_as(_I), _d(xy), _d(rho))
    return rho


def map_points(X, Y, pts) -> np.ndarray:
    X, Y, pts = _f64(X), _f64(Y), _f64(pts)
    Ly, Lx = X.shape
    out = np.empty_like(pts)
    lib().orc_map_points(Lx, Ly, _d(X), _d(Y), pts.shape[0], _d(pts), _d(out))
    return out


def coverage(m) -> np.ndarray:
    """Area of every cell covered by every region, [n_regions][Ly][Lx]."""
    ro = np.ascontiguousarray(m.ring_offsets, dtype=np.int64)
    rr = np.ascontiguousarray(m.ring_region, dtype=np.int32)
    xy = _f64(m.xy)
    out = np.empty((m.n_regions, m.Ly, m.Lx))
    lib().orc_coverage(m.Lx, m.Ly, m.n_regions, rr.size, ro.ctypes.data_as(_LL), rr.ctypes.data_as(_I), _d(xy),
                       _d(out))
    return out


def distortion(grids) -> np.ndarray:
    """e_a, e_inf, e~_a, e~_inf of the composed projection given its grids [K][2][Ly][Lx]
    (projected X, Y at the cell centres) -- SI section 3."""
    g = _f64(grids)
    K, _, Ly, Lx = g.shape
    out = np.empty(4)
    lib().orc_distortion(Lx, Ly, K, _d(g), _d(out))
    return out


def inverse_points(grids, q) -> np.ndarray:
    """Preimages of points q [n][2] under the composed projection (NaN where none)."""
    g = _f64(grids)
    q = _f64(q)
    K, _, Ly, Lx = g.shape
    out = np.empty_like(q)
    lib().orc_inverse_points(Lx, Ly, K, _d(g), q.shape[0], _d(q), _d(out))
    return out


@dataclass
class CartogramResult:
    xy: np.ndarray
    grids: np.ndarray
    err: np.ndarray
    iterations: int
    converged: bool
    status: int
    steps_accepted: int
    steps_rejected: int
    max_area_error: float


def cartogram(m, blur: float, keep_grids: bool = True, **kw) -> CartogramResult:
    """Run the whole method on a synth.RegionMap-like object (Lx, Ly, values, rings, xy)."""
    P = params(m.Lx, m.Ly, blur, **kw)
    xy = _f64(m.xy).copy()
    ro = np.ascontiguousarray(m.ring_offsets, dtype=np.int64)
    rr = np.ascontiguousarray(m.ring_region, dtype=np.int32)
    vals = _f64(m.values)
    grids = np.zeros((P.max_iter, 2, m.Ly, m.Lx)) if keep_grids else None
    err = np.empty(vals.size)
    st = Stats()
    lib().orc_cartogram(ctypes.byref(P), vals.size, _d(vals), rr.size, ro.ctypes.data_as(_LL),
                        rr.ctypes.data_as(_I), xy.shape[0], _d(xy),
                        _d(grids) if keep_grids else None, _d(err), ctypes.byref(st))
    return CartogramResult(xy, grids[:st.iterations] if keep_grids else None, err, st.iterations,
                           bool(st.converged), st.status, st.steps_accepted, st.steps_rejected,
                           st.max_area_error)
