"""ctypes wrapper of the plain C oracle (``fslbm_oracle.c``).

Test infrastructure only.  The C source is compiled with gcc, single-threaded
and without floating-point contraction, into ``oracle/_build/liboracle.so``.
All arrays are numpy float64 / uint8 / int32 in the cell order
``x + nx * (y + ny * z)``; PDFs and velocities are direction- or
component-major (``pdf[i * N + cell]``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fslbm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

VARIANTS = {"NBRC": 1, "NBKC": 2, "OM": 3, "OM3": 4}


def build_oracle(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2,
    -ffp-contract=off so that no multiply-add is fused).  ``openmp`` builds
    ``liboracle_omp.so`` from the same source with -fopenmp: its
    stream-collide cell loop runs on all host threads, for the CPU-baseline
    timing only (the tests use the sequential library)."""
    lib_path = _LIB_OMP if openmp else _LIB
    os.makedirs(os.path.dirname(lib_path), exist_ok=True)
    if (not force and os.path.exists(lib_path)
            and os.path.getmtime(lib_path) >= os.path.getmtime(_SRC)
            and os.path.getmtime(lib_path) >= os.path.getmtime(os.path.join(_HERE, "fslbm_oracle.h"))):
        return lib_path
    tmp = lib_path + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=gnu99", "-fPIC"]
    cmd += ["-fopenmp"] if openmp else []
    cmd += ["-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib_path)
    return lib_path


def _load(openmp: bool = False):
    global _lib, _lib_omp
    with _lock:
        if openmp and _lib_omp is not None:
            return _lib_omp
        if not openmp and _lib is not None:
            return _lib
        lib = C.CDLL(build_oracle(openmp=openmp))
        d, i, p = C.c_double, C.c_int, C.c_void_p
        lib.orc_create.restype = p
        lib.orc_create.argtypes = [i, i, i, i, i, i, i, i, i, i, i, d, d, d, d, d, d, d, d, d]
        lib.orc_destroy.argtypes = [p]
        lib.orc_init.restype = i
        lib.orc_init.argtypes = [p, p, p, p, p]
        lib.orc_step.argtypes = [p, i]
        lib.orc_steps_done.restype = C.c_long
        lib.orc_steps_done.argtypes = [p]
        lib.orc_read.argtypes = [p, p, p, p, p]
        lib.orc_read_moments.argtypes = [p, p, p]
        lib.orc_geometry.argtypes = [p, p, p, p]
        lib.orc_bubbles.restype = i
        lib.orc_bubbles.argtypes = [p, p, p, p, i]
        lib.orc_total_mass.restype = d
        lib.orc_total_mass.argtypes = [p]
        lib.orc_lattice.restype = i
        lib.orc_lattice.argtypes = [i, p, p, p]
        lib.orc_feq.argtypes = [i, d, p, p]
        lib.orc_collide.argtypes = [i, i, d, d, d, p, p, p, p]
        lib.orc_select.argtypes = [i, i, i, p, p, p]
        lib.orc_reconstruct.argtypes = [i, p, d, p, p, p]
        lib.orc_k8_smooth.restype = d
        lib.orc_k8_smooth.argtypes = [p]
        lib.orc_py_gradient.argtypes = [p, p]
        lib.orc_seed_fill_front.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, p, C.c_int,
                                            C.c_double, C.c_double, p, p]
        lib.orc_seed_fill_front.restype = C.c_int
        lib.orc_set_bubble_relabel.argtypes = [p, C.c_int]
        lib.orc_set_bubble_relabel.restype = None
        lib.orc_relabel_bubbles.argtypes = [p]
        lib.orc_relabel_bubbles.restype = None
        if openmp:
            _lib_omp = lib
        else:
            _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def lattice(q: int):
    """Direction table (c[q,3] int, w[q], opp[q]) of D2Q9 / D3Q19 / D3Q27."""
    lib = _load()
    c = np.zeros((q, 3), np.int32)
    w = np.zeros(q, np.float64)
    o = np.zeros(q, np.int32)
    if lib.orc_lattice(q, _ptr(c), _ptr(w), _ptr(o)):
        raise ValueError(f"unsupported q={q}")
    return c, w, o


def feq(q: int, rho: float, u) -> np.ndarray:
    lib = _load()
    u = np.ascontiguousarray(u, np.float64)
    out = np.zeros(q, np.float64)
    lib.orc_feq(q, float(rho), _ptr(u), _ptr(out))
    return out


def collide(q: int, collision: int, omega: float, trt_magic: float, g, fin, cs: float = 0.0):
    """One cell collision (Smagorinsky constant cs, 0: no LES); returns
    (f_out[q], rho, u[3])."""
    lib = _load()
    g = np.ascontiguousarray(g, np.float64)
    fin = np.ascontiguousarray(fin, np.float64)
    out = np.zeros(q, np.float64)
    ru = np.zeros(4, np.float64)
    lib.orc_collide(q, collision, float(omega), float(trt_magic), float(cs), _ptr(g), _ptr(fin), _ptr(out),
                    _ptr(ru))
    return out, ru[0], ru[1:].copy()


def select(q: int, variant: int, om3_fallback: int, nhat, miss) -> np.ndarray:
    """Reconstruction set R (bool[q]) of one interface cell."""
    lib = _load()
    nhat = np.ascontiguousarray(nhat, np.float64)
    miss = np.ascontiguousarray(miss, np.int32)
    rec = np.zeros(q, np.int32)
    lib.orc_select(q, int(variant), int(om3_fallback), _ptr(nhat), _ptr(miss), _ptr(rec))
    return rec.astype(bool)


def reconstruct(q: int, recon, rho_g: float, u, fstar_x, fin) -> np.ndarray:
    """Apply the free-surface BC to the entries of ``fin`` marked in ``recon``."""
    lib = _load()
    recon = np.ascontiguousarray(recon, np.int32)
    u = np.ascontiguousarray(u, np.float64)
    fstar_x = np.ascontiguousarray(fstar_x, np.float64)
    out = np.array(fin, np.float64, copy=True)
    lib.orc_reconstruct(q, _ptr(recon), float(rho_g), _ptr(u), _ptr(fstar_x), _ptr(out))
    return out


def k8_smooth(block) -> float:
    """K8-smoothed value at the centre of a 3x3x3 block (indexed [dz, dy, dx])."""
    lib = _load()
    b = np.ascontiguousarray(block, np.float64).reshape(27)
    return float(lib.orc_k8_smooth(_ptr(b)))


def py_gradient(block) -> np.ndarray:
    """Raw Parker-Youngs gradient at the centre of a 3x3x3 block ([dz, dy, dx])."""
    lib = _load()
    b = np.ascontiguousarray(block, np.float64).reshape(27)
    out = np.zeros(3, np.float64)
    lib.orc_py_gradient(_ptr(b), _ptr(out))
    return out


def seed_fill_front(flags, shape, layer, center, periodic=(False, False)):
    """Seed-fill front of the z-layer ``layer`` of a flags array in caller
    order (reading R23): returns (front mask [ny, nx] of bools, dict with
    count, r_min, r_max, r_mean about ``center`` = (xc, yc))."""
    lib = _load()
    nx, ny, nz = shape
    fl = np.ascontiguousarray(flags, np.uint8).reshape(-1)
    assert fl.size == nx * ny * nz
    front = np.zeros(nx * ny, np.uint8)
    st = np.zeros(4, np.float64)
    rc = lib.orc_seed_fill_front(nx, ny, nz, int(bool(periodic[0])), int(bool(periodic[1])), _ptr(fl),
                                 int(layer), float(center[0]), float(center[1]), _ptr(front), _ptr(st))
    if rc != 0:
        raise ValueError("bad arguments")
    return front.reshape(ny, nx).astype(bool), {"count": int(st[0]), "r_min": st[1], "r_max": st[2],
                                                "r_mean": st[3]}


class Oracle:
    """Whole-domain FP64 FSLBM run on one CPU thread.

    Parameters mirror the GPU library's create call: domain (nx, ny, nz),
    boundary of each axis (``periodic``: 0 / False no-slip walls, 1 / True
    periodic, 2 free-slip walls), q (19/27), collision ('SRT'/'TRT'), variant
    ('NBRC'/'NBKC'/'OM'/'OM3'), OM3 fallback, bubble model, omega, TRT magic
    parameter, gravity g[3], surface tension sigma, eps_phi, p_v0, the
    Smagorinsky constant and the steps between bubble relabellings (reading
    R24; 0 keeps the initial labels).  ``openmp`` runs the stream-collide cell loop on all host threads (the
    OpenMP build of the same source; same results).
    """

    def __init__(self, nx, ny, nz, periodic=(False, False, False), q=19, collision="TRT",
                 variant="OM", om3_fallback="NBKC", bubble_model=False, omega=1.0,
                 trt_magic=3.0 / 16.0, g=(0.0, 0.0, 0.0), sigma=0.0, eps_phi=1e-2,
                 p_v0=1.0 / 3.0, smagorinsky_cs=0.0, bubble_relabel_every=0, openmp=False):
        self._lib = _load(openmp)
        self.shape = (int(nx), int(ny), int(nz))
        self.N = int(nx) * int(ny) * int(nz)
        self.q = int(q)
        col = {"SRT": 0, "TRT": 1}[collision] if isinstance(collision, str) else int(collision)
        var = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        fb = VARIANTS[om3_fallback] if isinstance(om3_fallback, str) else int(om3_fallback)
        h = self._lib.orc_create(int(nx), int(ny), int(nz), int(periodic[0]),
                                 int(periodic[1]), int(periodic[2]), self.q, col, var, fb,
                                 int(bool(bubble_model)), float(omega), float(trt_magic),
                                 float(g[0]), float(g[1]), float(g[2]), float(sigma), float(eps_phi),
                                 float(p_v0), float(smagorinsky_cs))
        if not h:
            raise ValueError("oracle: invalid parameters")
        self._h = h
        self._lib.orc_set_bubble_relabel(h, int(bubble_relabel_every))

    def relabel_bubbles(self):
        """Bubble coalescence and segmentation now (reading R24)."""
        self._lib.orc_relabel_bubbles(self._h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    def init(self, fill, flags, velocity=None, density=None):
        fill = np.ascontiguousarray(fill, np.float64).reshape(-1)
        flags = np.ascontiguousarray(flags, np.uint8).reshape(-1)
        vel = None if velocity is None else np.ascontiguousarray(velocity, np.float64).reshape(-1)
        den = None if density is None else np.ascontiguousarray(density, np.float64).reshape(-1)
        assert fill.size == self.N and flags.size == self.N
        rc = self._lib.orc_init(self._h, _ptr(fill), _ptr(flags), _ptr(vel), _ptr(den))
        if rc:
            raise ValueError("oracle: invalid initial state (bad flag or liquid cell next to gas)")

    def step(self, n=1):
        self._lib.orc_step(self._h, int(n))

    @property
    def steps_done(self):
        return int(self._lib.orc_steps_done(self._h))

    def read(self):
        """Returns dict(pdf[q,N], fill[N], flags[N], mass[N])."""
        pdf = np.zeros(self.q * self.N, np.float64)
        fill = np.zeros(self.N, np.float64)
        flags = np.zeros(self.N, np.uint8)
        mass = np.zeros(self.N, np.float64)
        self._lib.orc_read(self._h, _ptr(pdf), _ptr(fill), _ptr(flags), _ptr(mass))
        return {"pdf": pdf.reshape(self.q, self.N), "fill": fill, "flags": flags, "mass": mass}

    def moments(self):
        rho = np.zeros(self.N, np.float64)
        u = np.zeros(3 * self.N, np.float64)
        self._lib.orc_read_moments(self._h, _ptr(rho), _ptr(u))
        return rho, u.reshape(3, self.N)

    def geometry(self):
        nhat = np.zeros(3 * self.N, np.float64)
        kappa = np.zeros(self.N, np.float64)
        phis = np.zeros(self.N, np.float64)
        self._lib.orc_geometry(self._h, _ptr(nhat), _ptr(kappa), _ptr(phis))
        return nhat.reshape(3, self.N), kappa, phis

    def bubbles(self, cap=4096):
        V = np.zeros(cap, np.float64)
        P = np.zeros(cap, np.float64)
        ids = np.zeros(self.N, np.int32)
        nb = self._lib.orc_bubbles(self._h, _ptr(V), _ptr(P), _ptr(ids), cap)
        return V[:nb].copy(), P[:nb].copy(), ids

    def total_mass(self):
        return float(self._lib.orc_total_mass(self._h))
