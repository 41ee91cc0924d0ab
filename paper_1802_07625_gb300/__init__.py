"""GB300 (sm_103a) diffusion-flow cartogram library: Python binding of the C-ABI.

Every function here marshals arguments for the call of the same name in
include/cartogram.h and nothing else: all computation runs in the CUDA library
(_build/libcartogram.so). Arrays may be numpy arrays (host) or torch tensors on the
host or on the context's GPU; outputs are written into caller-provided arrays or
freshly allocated numpy arrays. There is no CPU fallback: if the library is not
built or CUDA is unusable, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

__all__ = [
    "CG_OK", "CG_EINVAL", "CG_ENOMEM", "CG_ECUDA", "CG_ENOCONVERGE", "CG_EFOLD", "CG_ESTEPFAIL", "CG_ETIMEOUT",
    "CG_ESTATE", "CG_PRECISION_FP64", "CG_PRECISION_MIXED", "CG_PRECISION_MIXED_FF", "CG_FLOW_DIFFUSION",
    "CG_FLOW_LINEAR", "CartogramError", "Options", "Stats",
    "library_path", "load", "cartogram_default_options", "cartogram_init", "cartogram_set_stream",
    "cartogram_set_regions", "cartogram_integrate", "cartogram_project", "cartogram_area_errors",
    "cartogram_get_vertices", "cartogram_reset", "cartogram_set_values", "cartogram_polygon_measures", "cartogram_autotune", "cartogram_read_bandwidth", "cartogram_profile", "cartogram_history_length", "cartogram_iteration_record", "cartogram_fold_count", "cartogram_get_grid", "cartogram_density",
    "cartogram_spectrum", "cartogram_velocity", "cartogram_heun_step", "cartogram_integrate_once",
    "cartogram_velocity_noalloc", "cartogram_inverse_project", "cartogram_distortion",
    "cartogram_iteration_gradient", "cartogram_iteration_vjp", "cartogram_last_error",
    "cartogram_destroy", "cartogram_batch_create",
    "cartogram_batch_integrate", "cartogram_batch_last_error", "cartogram_batch_destroy", "Cartogram", "Batch",
    "iteration_loss", "mapped_iterations",
]

CG_OK, CG_EINVAL, CG_ENOMEM, CG_ECUDA, CG_ENOCONVERGE, CG_EFOLD, CG_ESTEPFAIL = 0, -1, -2, -3, -4, -5, -6
CG_ETIMEOUT, CG_ESTATE = -7, -8
CG_PRECISION_FP64, CG_PRECISION_MIXED, CG_PRECISION_MIXED_FF = 0, 1, 2
CG_FLOW_DIFFUSION, CG_FLOW_LINEAR = 0, 1

_ERRNAMES = {0: "CG_OK", -1: "CG_EINVAL", -2: "CG_ENOMEM", -3: "CG_ECUDA", -4: "CG_ENOCONVERGE",
             -5: "CG_EFOLD", -6: "CG_ESTEPFAIL", -7: "CG_ETIMEOUT", -8: "CG_ESTATE"}


class CartogramError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_ERRNAMES.get(code, code), msg))
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("dt0", ctypes.c_double), ("atol", ctypes.c_double),
                ("grow", ctypes.c_double), ("shrink", ctypes.c_double), ("cfl", ctypes.c_double),
                ("rho_tol", ctypes.c_double), ("area_tol", ctypes.c_double), ("max_steps", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("use_graph", ctypes.c_int), ("blur_decay", ctypes.c_double),
                ("autotune", ctypes.c_int), ("flow", ctypes.c_int), ("time_limit", ctypes.c_double),
                ("barrier_spins", ctypes.c_longlong)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("steps_accepted", ctypes.c_longlong), ("steps_rejected", ctypes.c_longlong),
                ("max_area_error", ctypes.c_double), ("t_end", ctypes.c_double),
                ("seconds", ctypes.c_double), ("step_loop_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_P = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("CUDA library not built: %s (run __graft_entry__.build())" % path)
    L = ctypes.CDLL(path)
    i, d, ll = ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "cartogram_default_options": (i, [ctypes.POINTER(Options)]),
        "cartogram_init": (i, [i, i, d, ctypes.POINTER(Options), ctypes.POINTER(_P)]),
        "cartogram_set_stream": (i, [_P, _P]),
        "cartogram_set_regions": (i, [_P, i, _P, ll, _P, _P, _P]),
        "cartogram_integrate": (i, [_P, ctypes.POINTER(Stats)]),
        "cartogram_project": (i, [_P, ll, _P, _P]),
        "cartogram_area_errors": (i, [_P, _P]),
        "cartogram_get_vertices": (i, [_P, _P]),
        "cartogram_history_length": (i, [_P]),
        "cartogram_iteration_record": (i, [_P, i, _P]),
        "cartogram_fold_count": (i, [_P, i, ctypes.POINTER(ll), ctypes.POINTER(d)]),
        "cartogram_reset": (i, [_P]),
        "cartogram_set_values": (i, [_P, _P]),
        "cartogram_polygon_measures": (i, [_P, _P]),
        "cartogram_autotune": (i, [_P, i, _P, _P]),
        "cartogram_read_bandwidth": (i, [ll, i, ctypes.POINTER(d)]),
        "cartogram_profile": (i, [_P, i, _P]),
        "cartogram_get_grid": (i, [_P, i, _P]),
        "cartogram_density": (i, [_P, _P]),
        "cartogram_spectrum": (i, [_P, _P]),
        "cartogram_velocity": (i, [_P, d, _P, _P]),
        "cartogram_heun_step": (i, [_P, d, d, _P, _P, _P]),
        "cartogram_integrate_once": (i, [_P, _P, ctypes.POINTER(ll), ctypes.POINTER(ll), ctypes.POINTER(d)]),
        "cartogram_velocity_noalloc": (i, [i, i, _P, d, _P, _P]),
        "cartogram_inverse_project": (i, [_P, ll, _P, _P]),
        "cartogram_distortion": (i, [_P, _P]),
        "cartogram_iteration_gradient": (i, [_P, _P, d, d, i, i, i, _P, _P, _P]),
        "cartogram_iteration_vjp": (i, [_P, _P, d, i, i, i, _P, _P, _P, _P, _P, _P]),
        "cartogram_last_error": (ctypes.c_char_p, [_P]),
        "cartogram_destroy": (None, [_P]),
        "cartogram_batch_create": (i, [ctypes.POINTER(_P), i, ctypes.POINTER(_P)]),
        "cartogram_batch_integrate": (i, [_P, _P, _P]),
        "cartogram_batch_last_error": (ctypes.c_char_p, [_P]),
        "cartogram_batch_destroy": (None, [_P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(ctx, rc):
    if rc != CG_OK:
        msg = load().cartogram_last_error(ctx) if ctx else b""
        raise CartogramError(rc, (msg or b"").decode())
    return rc


def _ptr(a, dtype, writable=False):
    """Address of a contiguous numpy array or torch tensor of the given numpy dtype."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr") and hasattr(a, "is_contiguous"):  # torch tensor
        import torch
        want = {np.float64: torch.float64, np.int64: torch.int64, np.int32: torch.int32}[dtype]
        if a.dtype != want or not a.is_contiguous():
            if writable:
                raise ValueError("output tensor must be contiguous %s" % want)
            a = a.to(want).contiguous()
        if a.is_cuda:
            # the library's stream does not wait on torch's: make the data ready first
            torch.cuda.current_stream(a.device).synchronize()
        return a.data_ptr(), a
    arr = np.asarray(a)
    if arr.dtype != dtype or not arr.flags["C_CONTIGUOUS"]:
        if writable:
            raise ValueError("output array must be C-contiguous %s" % np.dtype(dtype))
        arr = np.ascontiguousarray(arr, dtype=dtype)
    return arr.ctypes.data, arr


# ---------------------------------------------------------------------------
# one function per C entry point
# ---------------------------------------------------------------------------

def cartogram_default_options() -> Options:
    o = Options()
    _check(None, load().cartogram_default_options(ctypes.byref(o)))
    return o


def cartogram_init(Lx: int, Ly: int, blur_width: float, opt: Options | None = None) -> int:
    ctx = _P()
    rc = load().cartogram_init(int(Lx), int(Ly), float(blur_width),
                               ctypes.byref(opt) if opt is not None else None, ctypes.byref(ctx))
    if rc != CG_OK:
        raise CartogramError(rc, "cartogram_init(%d, %d, %g) failed" % (Lx, Ly, blur_width))
    return ctx.value


def cartogram_set_stream(ctx, stream) -> None:
    """`stream`: a torch.cuda.Stream, a raw cudaStream_t integer, or None (own stream)."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(ctx, load().cartogram_set_stream(ctx, stream))


def cartogram_set_regions(ctx, target_values, ring_offsets, ring_region, xy) -> None:
    pv, v = _ptr(target_values, np.float64)
    po, o = _ptr(ring_offsets, np.int64)
    pr, r = _ptr(ring_region, np.int32)
    px, x = _ptr(xy, np.float64)
    n_regions = int(v.shape[0]) if hasattr(v, "shape") else len(v)
    n_rings = int(r.shape[0]) if hasattr(r, "shape") else len(r)
    _check(ctx, load().cartogram_set_regions(ctx, n_regions, pv, n_rings, po, pr, px))


def cartogram_integrate(ctx) -> Stats:
    s = Stats()
    rc = load().cartogram_integrate(ctx, ctypes.byref(s))
    if rc not in (CG_OK,):
        err = CartogramError(rc, (load().cartogram_last_error(ctx) or b"").decode())
        err.stats = s
        raise err
    return s


def cartogram_project(ctx, xy_in, xy_out=None):
    pi_, a = _ptr(xy_in, np.float64)
    n = int(a.shape[0])
    if xy_out is None:
        xy_out = np.empty((n, 2), dtype=np.float64)
    po, _ = _ptr(xy_out, np.float64, writable=True)
    _check(ctx, load().cartogram_project(ctx, n, pi_, po))
    return xy_out


def cartogram_area_errors(ctx, out):
    po, _ = _ptr(out, np.float64, writable=True)
    _check(ctx, load().cartogram_area_errors(ctx, po))
    return out


def cartogram_get_vertices(ctx, out):
    po, _ = _ptr(out, np.float64, writable=True)
    _check(ctx, load().cartogram_get_vertices(ctx, po))
    return out


def cartogram_reset(ctx) -> None:
    _check(ctx, load().cartogram_reset(ctx))


def cartogram_polygon_measures(ctx) -> dict:
    out = np.zeros(3)
    po, _ = _ptr(out, np.float64, writable=True)
    _check(ctx, load().cartogram_polygon_measures(ctx, po))
    return {"alpha": float(out[0]), "theta": float(out[1]), "alpha_input": float(out[2])}


def cartogram_set_values(ctx, target_values) -> None:
    pv, _ = _ptr(target_values, np.float64)
    _check(ctx, load().cartogram_set_values(ctx, pv))


PROFILE_CLASSES = ("inverse_rows", "inverse_cols_velocity", "heun_step", "rasterise", "forward",
                   "map_and_areas")


def cartogram_profile(ctx, reps: int = 20) -> dict:
    out = np.zeros(len(PROFILE_CLASSES))
    _check(ctx, load().cartogram_profile(ctx, int(reps), out.ctypes.data))
    return dict(zip(PROFILE_CLASSES, out.tolist()))


def cartogram_autotune(ctx, reps: int = 10) -> dict:
    shapes = np.zeros(3, dtype=np.int32)
    ms = np.zeros(3)
    _check(ctx, load().cartogram_autotune(ctx, int(reps), shapes.ctypes.data, ms.ctypes.data))
    return {"rows_per_block": int(shapes[0]), "cols_per_block": int(shapes[1]),
            "heun_blocks_per_sm": int(shapes[2]), "ms": ms.tolist()}


def cartogram_read_bandwidth(nbytes: int, passes: int = 20) -> float:
    """Read bandwidth (GB/s) of the current GPU over a resident buffer of nbytes."""
    g = ctypes.c_double()
    rc = load().cartogram_read_bandwidth(int(nbytes), int(passes), ctypes.byref(g))
    if rc != CG_OK:
        raise CartogramError(rc, "cartogram_read_bandwidth(%d, %d) failed" % (nbytes, passes))
    return g.value


def cartogram_history_length(ctx) -> int:
    return load().cartogram_history_length(ctx)


ITERATION_RECORD = ("max_area_error", "t_end", "steps_accepted", "steps_rejected", "step_loop_ms", "blur")


def cartogram_iteration_record(ctx, k) -> dict:
    out = np.zeros(len(ITERATION_RECORD))
    _check(ctx, load().cartogram_iteration_record(ctx, int(k), out.ctypes.data))
    d = dict(zip(ITERATION_RECORD, out.tolist()))
    d["steps_accepted"] = int(d["steps_accepted"])
    d["steps_rejected"] = int(d["steps_rejected"])
    return d


def cartogram_fold_count(ctx, k):
    n, a = ctypes.c_longlong(), ctypes.c_double()
    _check(ctx, load().cartogram_fold_count(ctx, int(k), ctypes.byref(n), ctypes.byref(a)))
    return n.value, a.value


def cartogram_get_grid(ctx, k, out):
    po, _ = _ptr(out, np.float64, writable=True)
    _check(ctx, load().cartogram_get_grid(ctx, int(k), po))
    return out


def cartogram_density(ctx, out):
    po, _ = _ptr(out, np.float64, writable=True)
    _check(ctx, load().cartogram_density(ctx, po))
    return out


def cartogram_spectrum(ctx, out=None):
    po = None
    if out is not None:
        po, _ = _ptr(out, np.float64, writable=True)
    _check(ctx, load().cartogram_spectrum(ctx, po))
    return out


def cartogram_velocity(ctx, t, rho_out=None, v_out=None):
    pr = _ptr(rho_out, np.float64, writable=True)[0] if rho_out is not None else None
    pv = _ptr(v_out, np.float64, writable=True)[0] if v_out is not None else None
    _check(ctx, load().cartogram_velocity(ctx, float(t), pr, pv))
    return rho_out, v_out


def cartogram_heun_step(ctx, t, h, disp_in, disp_out):
    pi_, _a = _ptr(disp_in, np.float64)
    po, _ = _ptr(disp_out, np.float64, writable=True)
    e = ctypes.c_double()
    _check(ctx, load().cartogram_heun_step(ctx, float(t), float(h), pi_, po, ctypes.byref(e)))
    return e.value


def cartogram_integrate_once(ctx, grid_out=None):
    pg = _ptr(grid_out, np.float64, writable=True)[0] if grid_out is not None else None
    a, r, t = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_double()
    _check(ctx, load().cartogram_integrate_once(ctx, pg, ctypes.byref(a), ctypes.byref(r), ctypes.byref(t)))
    return a.value, r.value, t.value


def cartogram_velocity_noalloc(Lx, Ly, spec, t, v_out, stream=None) -> None:
    """Field from a device FP32 spectrum into a device FP32 [Ly, Lx, 2] buffer, with no
    device allocation (torch CUDA tensors on one device; queued on `stream`, default
    torch's current stream of that device)."""
    import torch
    if not (spec.is_cuda and v_out.is_cuda and spec.dtype == torch.float32 and v_out.dtype == torch.float32
            and spec.is_contiguous() and v_out.is_contiguous()):
        raise ValueError("spec and v_out must be contiguous float32 CUDA tensors")
    if spec.device != v_out.device:
        raise ValueError("spec and v_out must be on the same device")
    if spec.numel() < int(Lx) * int(Ly) or v_out.numel() < 2 * int(Lx) * int(Ly):
        raise ValueError("spec needs Lx*Ly and v_out 2*Lx*Ly elements")
    with torch.cuda.device(spec.device):
        if stream is None:
            stream = torch.cuda.current_stream(spec.device)
        if hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        rc = load().cartogram_velocity_noalloc(int(Lx), int(Ly), spec.data_ptr(), float(t), v_out.data_ptr(),
                                               stream)
    if rc != CG_OK:
        raise CartogramError(rc, "cartogram_velocity_noalloc(%d, %d) failed" % (Lx, Ly))


def cartogram_inverse_project(ctx, xy_in, xy_out):
    pi_, _a = _ptr(xy_in, np.float64)
    po, _ = _ptr(xy_out, np.float64, writable=True)
    n = xy_in.shape[0] if hasattr(xy_in, "shape") else len(xy_in)
    _check(ctx, load().cartogram_inverse_project(ctx, int(n), pi_, po))
    return xy_out


def cartogram_distortion(ctx) -> dict:
    out = np.zeros(4)
    _check(ctx, load().cartogram_distortion(ctx, out.ctypes.data))
    return {"e_a": out[0], "e_inf": out[1], "et_a": out[2], "et_inf": out[3]}


def cartogram_iteration_gradient(ctx, values, blur, lam=1e-3, replay=False, checkpoint=8, grad=True, iterations=1):
    """Loss of `iterations` outer iterations and (grad=True) its gradient w.r.t. values and blur."""
    v = np.ascontiguousarray(values, dtype=np.float64)
    loss = ctypes.c_double()
    gv = np.zeros_like(v) if grad else None
    gb = ctypes.c_double()
    _check(ctx, load().cartogram_iteration_gradient(ctx, v.ctypes.data, float(blur), float(lam), int(iterations),
                                                   int(bool(replay)),
                                                   int(checkpoint), ctypes.byref(loss),
                                                   gv.ctypes.data if grad else None,
                                                   ctypes.byref(gb) if grad else None))
    return (loss.value, gv, gb.value) if grad else loss.value


def cartogram_iteration_vjp(ctx, values, blur, n_vertices, iterations=1, replay=False, checkpoint=8,
                            grad_xy=None, grad_area=None, grad=True):
    """Mapped vertices X' [n_vertices, 2] and areas A' of `iterations` outer iterations and
    (grad=True) the vector-Jacobian product of the adjoints grad_xy = dL/dX', grad_area =
    dL/dA' (None: zero) with respect to the values and the blur width."""
    v = np.ascontiguousarray(values, dtype=np.float64)
    xy = np.empty((int(n_vertices), 2))
    area = np.empty(v.shape[0])
    gx = None if grad_xy is None else np.ascontiguousarray(grad_xy, dtype=np.float64)
    ga = None if grad_area is None else np.ascontiguousarray(grad_area, dtype=np.float64)
    if gx is not None and gx.shape != xy.shape:
        raise ValueError("grad_xy must have shape %s" % (xy.shape,))
    if ga is not None and ga.shape != area.shape:
        raise ValueError("grad_area must have shape %s" % (area.shape,))
    gv = np.zeros_like(v) if grad else None
    gb = ctypes.c_double()
    _check(ctx, load().cartogram_iteration_vjp(ctx, v.ctypes.data, float(blur), int(iterations), int(bool(replay)),
                                              int(checkpoint), xy.ctypes.data, area.ctypes.data,
                                              gx.ctypes.data if gx is not None else None,
                                              ga.ctypes.data if ga is not None else None,
                                              gv.ctypes.data if grad else None,
                                              ctypes.byref(gb) if grad else None))
    return (xy, area, gv, gb.value) if grad else (xy, area)


def cartogram_last_error(ctx) -> str:
    return (load().cartogram_last_error(ctx) or b"").decode()


def cartogram_destroy(ctx) -> None:
    if ctx:
        load().cartogram_destroy(ctx)


def cartogram_batch_create(ctxs):
    """Batch of contexts (handles) whose outer iterations run in one graph launch."""
    arr = (_P * len(ctxs))(*ctxs)
    out = _P()
    rc = load().cartogram_batch_create(arr, len(ctxs), ctypes.byref(out))
    if rc != CG_OK:
        raise CartogramError(rc, "cartogram_batch_create failed")
    return out.value


def cartogram_batch_integrate(batch, n: int, check: bool = True):
    """Run the batch; returns (list of Stats, list of per-context status codes)."""
    stats = (Stats * n)()
    status = np.zeros(n, dtype=np.int32)
    rc = load().cartogram_batch_integrate(batch, ctypes.cast(stats, _P), status.ctypes.data)
    if check and rc != CG_OK:
        raise CartogramError(rc, cartogram_batch_last_error(batch))
    return list(stats), status.tolist()


def cartogram_batch_last_error(batch) -> str:
    return (load().cartogram_batch_last_error(batch) or b"").decode()


def cartogram_batch_destroy(batch) -> None:
    if batch:
        load().cartogram_batch_destroy(batch)


# ---------------------------------------------------------------------------
# convenience object owning a context
# ---------------------------------------------------------------------------

@dataclass
class _Map:
    n_regions: int
    n_vertices: int


class Cartogram:
    """Owns one context; methods call the entry points above."""

    def __init__(self, Lx, Ly, blur_width=0.0, precision="fp64", flow="diffusion", **options):
        o = cartogram_default_options()
        precisions = {"fp64": CG_PRECISION_FP64, "mixed": CG_PRECISION_MIXED, "mixed_ff": CG_PRECISION_MIXED_FF}
        if precision not in precisions:
            raise ValueError("precision must be one of %s" % sorted(precisions))
        o.precision = precisions[precision]
        if flow not in ("diffusion", "linear"):
            raise ValueError("flow must be 'diffusion' or 'linear'")
        o.flow = CG_FLOW_LINEAR if flow == "linear" else CG_FLOW_DIFFUSION
        for k, v in options.items():
            if not hasattr(o, k):
                raise TypeError("unknown option %s" % k)
            setattr(o, k, v)
        self.Lx, self.Ly = int(Lx), int(Ly)
        self.options = o
        self.ctx = cartogram_init(Lx, Ly, blur_width, o)
        self._map = None

    def close(self):
        if self.ctx:
            cartogram_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream):
        cartogram_set_stream(self.ctx, stream)

    def set_regions(self, values, ring_offsets, ring_region, xy):
        cartogram_set_regions(self.ctx, values, ring_offsets, ring_region, xy)
        self._map = _Map(len(values), int(np.asarray(ring_offsets)[-1]) if not hasattr(ring_offsets, "data_ptr")
                         else int(ring_offsets[-1]))

    def set_map(self, m):
        self.set_regions(m.values, m.ring_offsets, m.ring_region, m.xy)

    def integrate(self) -> Stats:
        return cartogram_integrate(self.ctx)

    def project(self, xy, out=None):
        return cartogram_project(self.ctx, xy, out)

    def inverse_project(self, xy, out=None):
        xy = np.ascontiguousarray(xy, dtype=np.float64) if not hasattr(xy, "data_ptr") else xy
        if out is None:
            out = np.empty_like(xy)
        return cartogram_inverse_project(self.ctx, xy, out)

    def distortion(self):
        return cartogram_distortion(self.ctx)

    def iteration_gradient(self, values, blur, lam=1e-3, replay=False, checkpoint=8, grad=True, iterations=1):
        return cartogram_iteration_gradient(self.ctx, values, blur, lam, replay, checkpoint, grad, iterations)

    def iteration_vjp(self, values, blur, iterations=1, replay=False, checkpoint=8, grad_xy=None, grad_area=None,
                      grad=True):
        return cartogram_iteration_vjp(self.ctx, values, blur, self._map.n_vertices, iterations, replay, checkpoint,
                                       grad_xy, grad_area, grad)

    def area_errors(self):
        return cartogram_area_errors(self.ctx, np.empty(self._map.n_regions))

    def vertices(self):
        return cartogram_get_vertices(self.ctx, np.empty((self._map.n_vertices, 2)))

    def polygon_measures(self):
        return cartogram_polygon_measures(self.ctx)

    def set_values(self, values):
        cartogram_set_values(self.ctx, values)

    def reset(self):
        cartogram_reset(self.ctx)

    def autotune(self, reps=10):
        return cartogram_autotune(self.ctx, reps)

    def profile(self, reps=20):
        return cartogram_profile(self.ctx, reps)

    def history_length(self):
        return cartogram_history_length(self.ctx)

    def iteration_record(self, k):
        return cartogram_iteration_record(self.ctx, k)

    def iteration_history(self):
        return [cartogram_iteration_record(self.ctx, k) for k in range(self.history_length())]

    def fold_count(self, k):
        return cartogram_fold_count(self.ctx, k)

    def grid(self, k):
        return cartogram_get_grid(self.ctx, k, np.empty((self.Ly, self.Lx, 2)))

    def density(self):
        return cartogram_density(self.ctx, np.empty((self.Ly, self.Lx)))

    def spectrum(self):
        return cartogram_spectrum(self.ctx, np.empty((self.Ly, self.Lx)))

    def velocity(self, t):
        rho = np.empty((self.Ly, self.Lx))
        v = np.empty((self.Ly, self.Lx, 2))
        cartogram_velocity(self.ctx, t, rho, v)
        return rho, v

    def heun_step(self, t, h, disp):
        out = np.empty((self.Ly, self.Lx, 2))
        err = cartogram_heun_step(self.ctx, t, h, disp, out)
        return out, err

    def integrate_once(self):
        g = np.empty((self.Ly, self.Lx, 2))
        a, r, t = cartogram_integrate_once(self.ctx, g)
        return g, a, r, t


class Batch:
    """Owns a batch over Cartogram objects (which must outlive it)."""

    def __init__(self, carts):
        self.carts = list(carts)
        self.handle = cartogram_batch_create([c.ctx for c in self.carts])

    def integrate(self, check: bool = True):
        return cartogram_batch_integrate(self.handle, len(self.carts), check)

    def close(self):
        if self.handle:
            cartogram_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



def iteration_loss(values, blur, cartogram, lam=1e-3, checkpoint=8, iterations=1):
    """The one-iteration loss of `cartogram` (see cartogram_iteration_gradient) as a
    differentiable torch function of the target values (1-D float64 tensor) and the blur
    width (0-D tensor or float). The forward records the step schedule; the backward asks
    the library for the gradient of that same function (replaying the schedule). The
    context must not run anything else between the two."""
    import torch

    class _IterationLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, v, b):
            loss = cartogram.iteration_gradient(v.detach().cpu().double().numpy(), float(b), lam, replay=False,
                                                checkpoint=checkpoint, grad=False, iterations=iterations)
            ctx.args = (v.detach().cpu().double().numpy(), float(b), v.device, v.dtype)
            return torch.tensor(loss, dtype=torch.float64, device=v.device)

        @staticmethod
        def backward(ctx, g):
            vals, b, dev, dt = ctx.args
            _, gv, gb = cartogram.iteration_gradient(vals, b, lam, replay=True, checkpoint=checkpoint,
                                                     iterations=iterations)
            gvt = torch.as_tensor(gv, device=dev).to(dt) * g
            gbt = torch.tensor(gb, dtype=torch.float64, device=dev) * g
            return gvt, gbt

    b = blur if isinstance(blur, torch.Tensor) else torch.tensor(float(blur), dtype=torch.float64)
    return _IterationLoss.apply(values, b)


def mapped_iterations(values, blur, cartogram, iterations=1, checkpoint=8):
    """The mapped vertices X' [n_vertices, 2] and region areas A' [n_regions] after
    `iterations` outer iterations from the cartogram's current vertices, as a
    differentiable torch function of the target values (1-D float64 tensor) and the blur
    width (0-D tensor or float). Any loss written in torch on (X', A') -- and on the values
    directly -- can be differentiated: the backward hands dL/dX' and dL/dA' to the library's
    vector-Jacobian product (cartogram_iteration_vjp), which replays the step schedules the
    forward recorded. The context must not run anything else between the two."""
    import torch

    class _MappedIterations(torch.autograd.Function):
        @staticmethod
        def forward(ctx, v, b):
            vals = v.detach().cpu().double().numpy()
            xy, area = cartogram.iteration_vjp(vals, float(b), iterations=iterations, replay=False,
                                               checkpoint=checkpoint, grad=False)
            ctx.args = (vals, float(b), v.device, v.dtype)
            return (torch.as_tensor(xy, dtype=torch.float64, device=v.device),
                    torch.as_tensor(area, dtype=torch.float64, device=v.device))

        @staticmethod
        def backward(ctx, g_xy, g_area):
            vals, b, dev, dt = ctx.args
            gx = None if g_xy is None else g_xy.detach().cpu().double().numpy()
            ga = None if g_area is None else g_area.detach().cpu().double().numpy()
            _, _, gv, gb = cartogram.iteration_vjp(vals, b, iterations=iterations, replay=True,
                                                   checkpoint=checkpoint, grad_xy=gx, grad_area=ga)
            return (torch.as_tensor(gv, device=dev).to(dt),
                    torch.tensor(gb, dtype=torch.float64, device=dev))

    b = blur if isinstance(blur, torch.Tensor) else torch.tensor(float(blur), dtype=torch.float64)
    return _MappedIterations.apply(values, b)
