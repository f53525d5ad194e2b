"""ctypes binding of the C ABI declared in ``include/fslbm.h``.

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``libfslbm.so``.  There is no CPU fallback; ``load()`` raises when the
library cannot be built or loaded.  Function names mirror the C entry points
(``fslbm_create``, ``fslbm_init``, ``fslbm_step``, ...); ``Context`` is a thin
convenience wrapper that owns one ``fslbm_ctx``.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfslbm.so")

OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ETIMEOUT, ESTATE, ECAPACITY = range(8)
STATUS = {0: "FSLBM_OK", 1: "FSLBM_EINVAL", 2: "FSLBM_ENOMEM", 3: "FSLBM_ECUDA",
          4: "FSLBM_EUNSTABLE", 5: "FSLBM_ETIMEOUT", 6: "FSLBM_ESTATE", 7: "FSLBM_ECAPACITY"}
LATTICE = {19: 19, 27: 27, "D3Q19": 19, "D3Q27": 27}
COLLISION = {"SRT": 0, "TRT": 1}
VARIANT = {"NBRC": 1, "NBKC": 2, "OM": 3, "OM3": 4}
PRECISION = {"FP64": 0, "FP32": 1, "FP16S": 2, "BF16S": 3, "FP32MC": 4, "FP16SMC": 5}


class fslbm_domain(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("periodic", C.c_int * 3)]


class fslbm_params(C.Structure):
    _fields_ = [("omega", C.c_double), ("trt_magic", C.c_double), ("g", C.c_double * 3),
                ("sigma", C.c_double), ("eps_phi", C.c_double), ("p_v0", C.c_double),
                ("precision", C.c_int), ("om3_fallback", C.c_int), ("bubble_model", C.c_int),
                ("stream", C.c_void_p), ("smagorinsky_cs", C.c_double), ("bubble_relabel_every", C.c_int)]


class fslbm_tuning(C.Structure):
    _fields_ = [("bulk_blocks_per_sm", C.c_int), ("band_blocks_per_sm", C.c_int),
                ("ms_per_step", C.c_double)]


class fslbm_front_stats(C.Structure):
    _fields_ = [("count", C.c_int64), ("r_min", C.c_double), ("r_max", C.c_double), ("r_mean", C.c_double)]


class fslbm_obs(C.Structure):
    _fields_ = [("step", C.c_int64), ("total_mass", C.c_double), ("n_liquid", C.c_int64),
                ("n_interface", C.c_int64), ("n_gas", C.c_int64), ("n_obstacle", C.c_int64),
                ("max_u", C.c_double), ("nan_seen", C.c_int), ("n_bubbles", C.c_int),
                ("liquid_volume", C.c_double)]


class fslbm_server_config(C.Structure):
    _fields_ = [("lattice", C.c_int), ("collision", C.c_int), ("precision", C.c_int),
                ("max_active", C.c_int), ("chunk_steps", C.c_int), ("memory_budget", C.c_int64),
                ("stream", C.c_void_p)]


class fslbm_request(C.Structure):
    _fields_ = [("domain", fslbm_domain), ("bc_variant", C.c_int), ("params", fslbm_params),
                ("fill", C.c_void_p), ("flags", C.c_void_p), ("velocity", C.c_void_p),
                ("density", C.c_void_p), ("steps", C.c_int)]


class fslbm_result(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int), ("steps", C.c_int64), ("cells", C.c_int64),
                ("obs", fslbm_obs), ("t_queue", C.c_double), ("t_result", C.c_double)]


class fslbm_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("queued", C.c_int), ("active", C.c_int), ("max_active_seen", C.c_int),
                ("batch_rebuilds", C.c_int64), ("batch_steps", C.c_int64), ("cell_updates", C.c_double),
                ("memory_used", C.c_int64), ("memory_budget", C.c_int64)]


_lib = None
_lock = threading.Lock()

# Exported symbols (kept in sync with include/fslbm.h by a CPU test).
SYMBOLS = ["fslbm_params_default", "fslbm_create", "fslbm_init", "fslbm_step", "fslbm_sync",
           "fslbm_observables", "fslbm_front", "fslbm_read_fields", "fslbm_bubbles", "fslbm_set_timing",
           "fslbm_stage_times", "fslbm_save", "fslbm_load", "fslbm_interface_count", "fslbm_work_counts",
           "fslbm_observables_noalloc", "fslbm_set_axis_order", "fslbm_get_axis_order", "fslbm_destroy", "fslbm_last_error", "fslbm_version",
           "fslbm_batch_create", "fslbm_batch_step", "fslbm_batch_sync", "fslbm_batch_autotune",
           "fslbm_batch_set_tuning", "fslbm_batch_get_tuning", "fslbm_batch_launches",
           "fslbm_batch_destroy", "fslbm_batch_last_error", "fslbm_memory_estimate",
           "fslbm_server_create", "fslbm_server_submit", "fslbm_server_poll", "fslbm_server_result",
           "fslbm_server_stats_get", "fslbm_server_destroy", "fslbm_server_last_error"]


def load(build_if_missing: bool = True):
    """Load libfslbm.so (building it with nvcc when missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            from . import build as _build
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library missing: {LIB_PATH}")
        lib = C.CDLL(LIB_PATH)
        p, i, d = C.c_void_p, C.c_int, C.c_double
        lib.fslbm_params_default.argtypes = [C.POINTER(fslbm_params)]
        lib.fslbm_params_default.restype = None
        lib.fslbm_create.argtypes = [C.POINTER(fslbm_domain), i, i, i, C.POINTER(fslbm_params),
                                     C.POINTER(p)]
        lib.fslbm_create.restype = i
        lib.fslbm_init.argtypes = [p, p, p, p, p]
        lib.fslbm_init.restype = i
        lib.fslbm_step.argtypes = [p, i]
        lib.fslbm_step.restype = i
        lib.fslbm_sync.argtypes = [p]
        lib.fslbm_sync.restype = i
        lib.fslbm_observables.argtypes = [p, C.POINTER(fslbm_obs)]
        lib.fslbm_observables.restype = i
        lib.fslbm_front.argtypes = [p, i, d, d, C.POINTER(fslbm_front_stats), p]
        lib.fslbm_front.restype = i
        lib.fslbm_read_fields.argtypes = [p, p, p, p, p]
        lib.fslbm_read_fields.restype = i
        lib.fslbm_bubbles.argtypes = [p, p, p, i, C.POINTER(i)]
        lib.fslbm_bubbles.restype = i
        lib.fslbm_set_timing.argtypes = [p, i]
        lib.fslbm_set_timing.restype = i
        lib.fslbm_stage_times.argtypes = [p, p, i, C.POINTER(i)]
        lib.fslbm_stage_times.restype = i
        lib.fslbm_save.argtypes = [p, p, C.POINTER(C.c_size_t)]
        lib.fslbm_save.restype = i
        lib.fslbm_load.argtypes = [p, p, C.c_size_t]
        lib.fslbm_load.restype = i
        lib.fslbm_interface_count.argtypes = [p, C.POINTER(C.c_int64)]
        lib.fslbm_interface_count.restype = i
        lib.fslbm_work_counts.argtypes = [p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        lib.fslbm_work_counts.restype = i
        lib.fslbm_observables_noalloc.argtypes = [C.POINTER(fslbm_domain), i, p, p, p, p, p,
                                                  C.POINTER(fslbm_obs), p]
        lib.fslbm_observables_noalloc.restype = i
        lib.fslbm_set_axis_order.argtypes = [p, p]
        lib.fslbm_set_axis_order.restype = i
        lib.fslbm_get_axis_order.argtypes = [p, p]
        lib.fslbm_get_axis_order.restype = i
        lib.fslbm_destroy.argtypes = [p]
        lib.fslbm_destroy.restype = None
        lib.fslbm_last_error.argtypes = [p]
        lib.fslbm_last_error.restype = C.c_char_p
        lib.fslbm_version.argtypes = []
        lib.fslbm_version.restype = C.c_char_p
        lib.fslbm_batch_create.argtypes = [C.POINTER(p), i, p, C.POINTER(p)]
        lib.fslbm_batch_create.restype = i
        lib.fslbm_batch_step.argtypes = [p, i]
        lib.fslbm_batch_step.restype = i
        lib.fslbm_batch_sync.argtypes = [p, C.POINTER(C.c_int)]
        lib.fslbm_batch_sync.restype = i
        lib.fslbm_batch_autotune.argtypes = [p, i, C.POINTER(fslbm_tuning)]
        lib.fslbm_batch_autotune.restype = i
        lib.fslbm_batch_set_tuning.argtypes = [p, C.POINTER(fslbm_tuning)]
        lib.fslbm_batch_set_tuning.restype = i
        lib.fslbm_batch_get_tuning.argtypes = [p, C.POINTER(fslbm_tuning)]
        lib.fslbm_batch_get_tuning.restype = i
        lib.fslbm_batch_launches.argtypes = [p, C.POINTER(C.c_int64)]
        lib.fslbm_batch_launches.restype = i
        lib.fslbm_batch_destroy.argtypes = [p]
        lib.fslbm_batch_destroy.restype = None
        lib.fslbm_batch_last_error.argtypes = [p]
        lib.fslbm_batch_last_error.restype = C.c_char_p
        lib.fslbm_memory_estimate.argtypes = [C.POINTER(fslbm_domain), i, i, i, C.POINTER(C.c_size_t)]
        lib.fslbm_memory_estimate.restype = i
        lib.fslbm_server_create.argtypes = [C.POINTER(fslbm_server_config), C.POINTER(p)]
        lib.fslbm_server_create.restype = i
        lib.fslbm_server_submit.argtypes = [p, C.POINTER(fslbm_request), C.POINTER(C.c_int64)]
        lib.fslbm_server_submit.restype = i
        lib.fslbm_server_poll.argtypes = [p, C.POINTER(i)]
        lib.fslbm_server_poll.restype = i
        lib.fslbm_server_result.argtypes = [p, C.c_int64, C.POINTER(fslbm_result), p, p]
        lib.fslbm_server_result.restype = i
        lib.fslbm_server_stats_get.argtypes = [p, C.POINTER(fslbm_server_stats)]
        lib.fslbm_server_stats_get.restype = i
        lib.fslbm_server_destroy.argtypes = [p]
        lib.fslbm_server_destroy.restype = None
        lib.fslbm_server_last_error.argtypes = [p]
        lib.fslbm_server_last_error.restype = C.c_char_p
        _lib = lib
        return lib


class FslbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


class Context:
    """One FSLBM domain on the current CUDA device (wraps ``fslbm_ctx``).

    ``stream`` is a raw ``cudaStream_t`` handle (int) or None for the default
    stream; e.g. ``torch.cuda.current_stream().cuda_stream``.
    """

    def __init__(self, shape, periodic=(False, False, False), q=19, collision="TRT", variant="OM",
                 precision="FP32", omega=1.0, trt_magic=3.0 / 16.0, g=(0.0, 0.0, 0.0), sigma=0.0,
                 eps_phi=1e-2, p_v0=1.0 / 3.0, om3_fallback="NBKC", bubble_model=False,
                 stream=None, axis_order=None, smagorinsky_cs=0.0, bubble_relabel_every=0):
        self.lib = load()
        self.shape = tuple(int(s) for s in shape)
        self.N = int(np.prod(self.shape))
        self.q = LATTICE[q]
        # boundary of each axis: 0 / False no-slip, 1 / True periodic, 2 free-slip
        dom = fslbm_domain(self.shape[0], self.shape[1], self.shape[2],
                           (C.c_int * 3)(*[int(x) for x in periodic]))
        prm = fslbm_params()
        self.lib.fslbm_params_default(C.byref(prm))
        prm.omega = float(omega)
        prm.trt_magic = float(trt_magic)
        prm.g = (C.c_double * 3)(*[float(x) for x in g])
        prm.sigma = float(sigma)
        prm.eps_phi = float(eps_phi)
        prm.p_v0 = float(p_v0)
        prm.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        prm.om3_fallback = VARIANT[om3_fallback] if isinstance(om3_fallback, str) else int(om3_fallback)
        prm.bubble_model = int(bool(bubble_model))
        prm.stream = C.c_void_p(int(stream)) if stream else None
        prm.smagorinsky_cs = float(smagorinsky_cs)
        prm.bubble_relabel_every = int(bubble_relabel_every)
        self.precision = prm.precision
        h = C.c_void_p()
        col = COLLISION[collision] if isinstance(collision, str) else int(collision)
        var = VARIANT[variant] if isinstance(variant, str) else int(variant)
        st = self.lib.fslbm_create(C.byref(dom), self.q, col, var, C.byref(prm), C.byref(h))
        if st != OK:
            raise FslbmError(st, "fslbm_create failed")
        self.h = h
        if axis_order is not None:
            self.set_axis_order(axis_order)

    def _check(self, st):
        if st != OK:
            raise FslbmError(st, self.lib.fslbm_last_error(self.h).decode())
        return st

    def set_axis_order(self, order):
        """Storage order for the next init: (contiguous axis, ..., slowest
        axis) as axis numbers 0..2, or None to let init choose."""
        arr = None if order is None else (C.c_int * 3)(*[int(a) for a in order])
        self._check(self.lib.fslbm_set_axis_order(self.h, arr))

    def axis_order(self):
        arr = (C.c_int * 3)()
        self._check(self.lib.fslbm_get_axis_order(self.h, arr))
        return tuple(arr)

    def close(self):
        if getattr(self, "h", None):
            self.lib.fslbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, fill, flags, velocity=None, density=None):
        fill = np.ascontiguousarray(fill, np.float64).reshape(-1)
        flags = np.ascontiguousarray(flags, np.uint8).reshape(-1)
        vel = None if velocity is None else np.ascontiguousarray(velocity, np.float64).reshape(-1)
        den = None if density is None else np.ascontiguousarray(density, np.float64).reshape(-1)
        if fill.size != self.N or flags.size != self.N:
            raise ValueError("fill/flags size mismatch")
        self._check(self.lib.fslbm_init(self.h, _ptr(fill), _ptr(flags), _ptr(vel), _ptr(den)))

    def init_raw(self, fill_ptr, flags_ptr, vel_ptr=None, den_ptr=None):
        """Initialise from raw host pointers (e.g. pinned torch tensors)."""
        return self.lib.fslbm_init(self.h, C.c_void_p(fill_ptr), C.c_void_p(flags_ptr),
                                   C.c_void_p(vel_ptr) if vel_ptr else None,
                                   C.c_void_p(den_ptr) if den_ptr else None)

    def step(self, n=1):
        self._check(self.lib.fslbm_step(self.h, int(n)))

    def sync(self):
        return self.lib.fslbm_sync(self.h)

    def observables(self, check=True):
        o = fslbm_obs()
        st = self.lib.fslbm_observables(self.h, C.byref(o))
        if check and st not in (OK, EUNSTABLE):
            self._check(st)
        return {k: getattr(o, k) for k, _ in fslbm_obs._fields_} | {"status": st}

    def front(self, layer, center, mask=False):
        """Seed-fill front of the z-layer ``layer`` (fslbm_front): a dict with
        count, r_min, r_max, r_mean about ``center`` = (xc, yc), plus the front
        mask [ny, nx] of bools when ``mask``."""
        st = fslbm_front_stats()
        nx, ny = self.shape[0], self.shape[1]
        m = np.zeros(nx * ny, np.uint8) if mask else None
        self._check(self.lib.fslbm_front(self.h, int(layer), float(center[0]), float(center[1]), C.byref(st),
                                         _ptr(m)))
        out = {k: getattr(st, k) for k, _ in fslbm_front_stats._fields_}
        if mask:
            out["mask"] = m.reshape(ny, nx).astype(bool)
        return out

    def read(self, pdf=True):
        out = {"fill": np.zeros(self.N, np.float64), "flags": np.zeros(self.N, np.uint8),
               "mass": np.zeros(self.N, np.float64)}
        if pdf:
            out["pdf"] = np.zeros(self.q * self.N, np.float64)
        self._check(self.lib.fslbm_read_fields(self.h, _ptr(out.get("pdf")), _ptr(out["fill"]),
                                               _ptr(out["flags"]), _ptr(out["mass"])))
        if pdf:
            out["pdf"] = out["pdf"].reshape(self.q, self.N)
        return out

    def bubbles(self, cap=4096):
        V = np.zeros(cap, np.float64)
        P = np.zeros(cap, np.float64)
        n = C.c_int(0)
        self._check(self.lib.fslbm_bubbles(self.h, _ptr(V), _ptr(P), cap, C.byref(n)))
        return V[: n.value].copy(), P[: n.value].copy()

    def set_timing(self, on):
        self._check(self.lib.fslbm_set_timing(self.h, int(bool(on))))

    STAGES = ["geometry", "bulk", "interface", "resolve", "count", "apply", "finalize", "bubbles"]

    def stage_times(self):
        ms = np.zeros(len(self.STAGES), np.float64)
        n = C.c_int(0)
        self._check(self.lib.fslbm_stage_times(self.h, _ptr(ms), len(self.STAGES), C.byref(n)))
        return dict(zip(self.STAGES, ms.tolist())), n.value

    def interface_count(self):
        n = C.c_int64(0)
        self._check(self.lib.fslbm_interface_count(self.h, C.byref(n)))
        return n.value

    def work_counts(self):
        a, b, t = C.c_int64(0), C.c_int64(0), C.c_int64(0)
        self._check(self.lib.fslbm_work_counts(self.h, C.byref(a), C.byref(b), C.byref(t)))
        return {"interface_cells": a.value, "liquid_segments": b.value, "geometry_tiles": t.value}

    def save(self):
        size = C.c_size_t(0)
        self._check(self.lib.fslbm_save(self.h, None, C.byref(size)))
        buf = np.zeros(size.value, np.uint8)
        self._check(self.lib.fslbm_save(self.h, _ptr(buf), C.byref(size)))
        return buf

    def load(self, buf):
        buf = np.ascontiguousarray(buf, np.uint8)
        self._check(self.lib.fslbm_load(self.h, _ptr(buf), buf.size))


class Batch:
    """Several initialized contexts advanced together (wraps ``fslbm_batch``):
    one launch per phase of the step over all member domains.  The members
    stay usable on their own (``read``, ``observables``, ``step``)."""

    def __init__(self, members, stream=None):
        self.lib = load()
        self.members = list(members)
        arr = (C.c_void_p * len(self.members))(*[m.h.value for m in self.members])
        h = C.c_void_p()
        st = self.lib.fslbm_batch_create(arr, len(self.members), C.c_void_p(int(stream)) if stream else None,
                                         C.byref(h))
        if st != OK:
            raise FslbmError(st, "fslbm_batch_create failed")
        self.h = h

    def _check(self, st):
        if st != OK:
            raise FslbmError(st, self.lib.fslbm_batch_last_error(self.h).decode())
        return st

    def step(self, n=1):
        self._check(self.lib.fslbm_batch_step(self.h, int(n)))

    def sync(self):
        out = (C.c_int * len(self.members))()
        st = self.lib.fslbm_batch_sync(self.h, out)
        return st, list(out)

    def autotune(self, steps=3):
        t = fslbm_tuning()
        self._check(self.lib.fslbm_batch_autotune(self.h, int(steps), C.byref(t)))
        return {"bulk_blocks_per_sm": t.bulk_blocks_per_sm, "band_blocks_per_sm": t.band_blocks_per_sm,
                "ms_per_step": t.ms_per_step}

    def set_tuning(self, bulk_blocks_per_sm, band_blocks_per_sm):
        t = fslbm_tuning(int(bulk_blocks_per_sm), int(band_blocks_per_sm), 0.0)
        self._check(self.lib.fslbm_batch_set_tuning(self.h, C.byref(t)))

    def tuning(self):
        t = fslbm_tuning()
        self._check(self.lib.fslbm_batch_get_tuning(self.h, C.byref(t)))
        return {"bulk_blocks_per_sm": t.bulk_blocks_per_sm, "band_blocks_per_sm": t.band_blocks_per_sm,
                "ms_per_step": t.ms_per_step}

    def launches(self):
        n = C.c_int64(0)
        self._check(self.lib.fslbm_batch_launches(self.h, C.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.fslbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _params_for(sc, precision, **over):
    """fslbm_params of a scenario (keywords as for Context)."""
    lib = load()
    kw = dict(omega=sc.omega, g=sc.g, sigma=sc.sigma, bubble_model=sc.bubble_model)
    kw.update({k: v for k, v in over.items() if k in ("omega", "g", "sigma", "bubble_model", "trt_magic",
                                                      "eps_phi", "p_v0", "om3_fallback", "smagorinsky_cs",
                                                      "bubble_relabel_every")})
    prm = fslbm_params()
    lib.fslbm_params_default(C.byref(prm))
    prm.omega = float(kw["omega"])
    prm.g = (C.c_double * 3)(*[float(x) for x in kw["g"]])
    prm.sigma = float(kw["sigma"])
    prm.bubble_model = int(bool(kw["bubble_model"]))
    for k in ("trt_magic", "eps_phi", "p_v0"):
        if k in kw:
            setattr(prm, k, float(kw[k]))
    if "om3_fallback" in kw:
        prm.om3_fallback = VARIANT[kw["om3_fallback"]]
    if "smagorinsky_cs" in kw:
        prm.smagorinsky_cs = float(kw["smagorinsky_cs"])
    if "bubble_relabel_every" in kw:
        prm.bubble_relabel_every = int(kw["bubble_relabel_every"])
    prm.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    return prm


class Server:
    """Continuous-batching request loop (wraps ``fslbm_server``)."""

    def __init__(self, q=19, collision="TRT", precision="FP32", max_active=16, chunk_steps=100,
                 memory_budget=0, stream=None):
        self.lib = load()
        cfg = fslbm_server_config(LATTICE[q], COLLISION[collision], PRECISION[precision], int(max_active),
                                  int(chunk_steps), int(memory_budget), C.c_void_p(int(stream)) if stream else None)
        self.precision = precision
        h = C.c_void_p()
        st = self.lib.fslbm_server_create(C.byref(cfg), C.byref(h))
        if st != OK:
            raise FslbmError(st, "fslbm_server_create failed")
        self.h = h
        self.shapes = {}

    def _check(self, st):
        if st != OK:
            raise FslbmError(st, self.lib.fslbm_server_last_error(self.h).decode())
        return st

    def submit(self, sc, steps, **over):
        """Queue scenario ``sc`` for ``steps`` steps; returns the request id."""
        fill = np.ascontiguousarray(sc.fill, np.float64)
        flags = np.ascontiguousarray(sc.flags, np.uint8)
        vel = None if sc.velocity is None else np.ascontiguousarray(sc.velocity, np.float64)
        den = None if sc.density is None else np.ascontiguousarray(sc.density, np.float64)
        rq = fslbm_request()
        rq.domain = fslbm_domain(*sc.shape, (C.c_int * 3)(*[int(x) for x in sc.periodic]))
        rq.bc_variant = VARIANT[over.get("variant", sc.variant)]
        rq.params = _params_for(sc, self.precision, **over)
        rq.fill, rq.flags = fill.ctypes.data, flags.ctypes.data
        rq.velocity = None if vel is None else vel.ctypes.data
        rq.density = None if den is None else den.ctypes.data
        rq.steps = int(steps)
        rid = C.c_int64(0)
        self._check(self.lib.fslbm_server_submit(self.h, C.byref(rq), C.byref(rid)))
        self.shapes[rid.value] = sc.N
        return rid.value

    def poll(self):
        n = C.c_int(0)
        self._check(self.lib.fslbm_server_poll(self.h, C.byref(n)))
        return n.value

    def result(self, rid):
        """Final fields and timing of a finished run, or None while it runs."""
        N = self.shapes[rid]
        res = fslbm_result()
        fill = np.zeros(N, np.float64)
        flags = np.zeros(N, np.uint8)
        st = self.lib.fslbm_server_result(self.h, rid, C.byref(res), fill.ctypes.data, flags.ctypes.data)
        if st == ESTATE:
            return None
        self._check(st)
        obs = {k: getattr(res.obs, k) for k, _ in fslbm_obs._fields_}
        return {"id": res.id, "status": res.status, "steps": res.steps, "cells": res.cells, "obs": obs,
                "t_queue": res.t_queue, "t_result": res.t_result, "fill": fill, "flags": flags}

    def stats(self):
        st = fslbm_server_stats()
        self._check(self.lib.fslbm_server_stats_get(self.h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in fslbm_server_stats._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.lib.fslbm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def memory_estimate(shape, q=19, precision="FP32", with_velocity=False):
    lib = load()
    b = C.c_size_t(0)
    dom = fslbm_domain(*shape, (C.c_int * 3)(0, 0, 0))
    st = lib.fslbm_memory_estimate(C.byref(dom), LATTICE[q], PRECISION[precision], int(bool(with_velocity)),
                                   C.byref(b))
    if st != OK:
        raise FslbmError(st, "fslbm_memory_estimate failed")
    return b.value


def context_for(sc, precision="FP64", stream=None, **over):
    """Context configured from a ``scenarios.Scenario`` (same keywords as the
    oracle) and initialised with its arrays."""
    kw = dict(periodic=sc.periodic, q=sc.q, collision=sc.collision, variant=sc.variant,
              omega=sc.omega, g=sc.g, sigma=sc.sigma, bubble_model=sc.bubble_model)
    kw.update(over)
    ctx = Context(sc.shape, precision=precision, stream=stream, **kw)
    ctx.init(sc.fill, sc.flags, sc.velocity, sc.density)
    return ctx
