"""Seeded synthetic initial states for the FSLBM runs.

This module holds no arithmetic of the method itself: it only lays out cell
types, fill levels, initial velocities and hydrostatic initial densities of
the paper's workloads (Sec. 4: gravity wave, rectangular and cylindrical dam
break, Taylor bubble, drop impact) and of the pin cases.  Both the CUDA path
and the CPU oracle consume exactly these arrays.

Conventions
-----------
* Cell (i, j, k) covers [i, i+1) x [j, j+1) x [k, k+1); linear index
  ``i + nx * (j + ny * k)``; arrays are returned flattened in that order.
* Flags: 0 gas, 1 interface, 2 liquid, 3 obstacle.  Cells outside a
  non-periodic boundary act as no-slip walls, so walls need no cells.
* Fill levels come from the exact column height (height-profile interfaces)
  or from 8 x 8 x 8 sub-sampling (spheres, cylinders).
* Closure of the interface layer: a liquid cell that has a gas cell in its
  lattice neighbourhood becomes an interface cell with fill level 1.
* Hydrostatic density rho = 1 + 3 |g| (h_ref - height of the cell centre) in
  liquid and interface cells, so that the pressure equals p0 = 1/3 at h_ref.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

GAS, IFACE, LIQ, OBST = 0, 1, 2, 3


def neighbour_offsets(q: int):
    """Lattice neighbourhood (without the rest direction) of D3Q19 or D3Q27."""
    offs = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                n2 = dx * dx + dy * dy + dz * dz
                if n2 == 0:
                    continue
                if q == 19 and n2 > 2:
                    continue
                offs.append((dx, dy, dz))
    return offs


@dataclass
class Scenario:
    name: str
    shape: tuple                       # (nx, ny, nz)
    periodic: tuple                    # (px, py, pz)
    fill: np.ndarray                   # float64[N]
    flags: np.ndarray                  # uint8[N]
    velocity: np.ndarray | None        # float64[3N] component-major or None
    density: np.ndarray | None         # float64[N] or None
    q: int = 19
    collision: str = "TRT"
    variant: str = "OM"
    omega: float = 1.0
    g: tuple = (0.0, 0.0, 0.0)
    sigma: float = 0.0
    bubble_model: bool = False
    steps: int = 1000
    meta: dict = field(default_factory=dict)

    @property
    def N(self):
        return int(np.prod(self.shape))

    def params(self):
        return dict(q=self.q, collision=self.collision, variant=self.variant, omega=self.omega,
                    g=self.g, sigma=self.sigma, bubble_model=self.bubble_model)


def omega_from_nu(nu: float) -> float:
    """Relaxation rate for a kinematic viscosity (Eq. nm-lbm-viscosity)."""
    return 1.0 / (3.0 * nu + 0.5)


def _shift(a, d, axis, periodic, fillval):
    """b[x] = a[x + d] along axis; outside a non-periodic boundary -> fillval."""
    if periodic:
        return np.roll(a, -d, axis=axis)
    b = np.full_like(a, fillval)
    n = a.shape[axis]
    src = [slice(None)] * a.ndim
    dst = [slice(None)] * a.ndim
    if d > 0:
        src[axis] = slice(d, n)
        dst[axis] = slice(0, n - d)
    elif d < 0:
        src[axis] = slice(0, n + d)
        dst[axis] = slice(-d, n)
    else:
        return a.copy()
    b[tuple(dst)] = a[tuple(src)]
    return b


def classify(phi_zyx: np.ndarray, obstacle_zyx: np.ndarray | None, periodic, q: int):
    """Cell types from fill levels + closure of the interface layer.

    phi_zyx: float array indexed [k, j, i].  Returns (fill, flags) flattened.
    """
    phi = np.clip(phi_zyx, 0.0, 1.0)
    flags = np.where(phi >= 1.0, LIQ, np.where(phi <= 0.0, GAS, IFACE)).astype(np.uint8)
    if obstacle_zyx is not None:
        flags[obstacle_zyx] = OBST
        phi = np.where(obstacle_zyx, 0.0, phi)
    gas = flags == GAS
    near_gas = np.zeros_like(gas)
    for dx, dy, dz in neighbour_offsets(q):
        s = gas
        s = _shift(s, dz, 0, periodic[2], False)
        s = _shift(s, dy, 1, periodic[1], False)
        s = _shift(s, dx, 2, periodic[0], False)
        near_gas |= s
    fix = (flags == LIQ) & near_gas
    flags[fix] = IFACE
    phi = np.where(flags == GAS, 0.0, np.where(flags == LIQ, 1.0, phi))
    phi = np.where(flags == OBST, 0.0, phi)
    return phi.reshape(-1).astype(np.float64), flags.reshape(-1)


def hydrostatic(shape, axis: int, g_abs: float, h_ref: float, flags):
    """rho = 1 + 3 |g| (h_ref - centre height) on liquid/interface cells."""
    nx, ny, nz = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    h = (i, j, k)[axis].astype(np.float64) + 0.5
    rho = 1.0 + 3.0 * g_abs * (h_ref - h)
    rho = rho.reshape(-1)
    return np.where((flags == LIQ) | (flags == IFACE), rho, 1.0)


def _subsample_fraction(inside, shape, origin=(0.0, 0.0, 0.0), s=8):
    """Volume fraction of each cell inside a region given as a vectorised
    predicate inside(x, y, z) of physical coordinates.  Cells whose 8 corners
    agree are taken as fully inside or outside (the regions used here are
    unions of convex bodies much larger than a cell); the others are
    sub-sampled with s^3 points."""
    nx, ny, nz = shape
    zc, yc, xc = np.meshgrid(np.arange(nz + 1) + origin[2], np.arange(ny + 1) + origin[1],
                             np.arange(nx + 1) + origin[0], indexing="ij")
    corner = inside(xc, yc, zc).astype(np.int8)
    tot = np.zeros((nz, ny, nx), np.int8)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                tot += corner[dz:dz + nz, dy:dy + ny, dx:dx + nx]
    frac = (tot == 8).astype(np.float64)
    mixed = np.nonzero((tot > 0) & (tot < 8))
    if mixed[0].size:
        k, j, i = mixed
        off = (np.arange(s) + 0.5) / s
        acc = np.zeros(k.size, np.float64)
        for oz in off:
            for oy in off:
                for ox in off:
                    acc += inside(i + ox + origin[0], j + oy + origin[1], k + oz + origin[2])
        frac[mixed] = acc / float(s ** 3)
    return frac


# ------------------------------------------------------------------ workloads

def gravity_wave(L=32, H=64, depth=32.0, amp_frac=0.01, g=1e-5, nu=0.01, variant="OM",
                 q=19, collision="TRT", steps=1000):
    """Standing gravity wave (Sec. 4.1): L x H x 1, periodic x and z, no-slip
    walls in y, interface y_s(i) = d + a0 cos(2 pi i / L) with a0 = amp_frac*L,
    hydrostatic pressure equal to p0 at y = d."""
    nx, ny, nz = L, H, 1
    a0 = amp_frac * L
    i = np.arange(nx, dtype=np.float64)
    ys = depth + a0 * np.cos(2.0 * np.pi * i / L)
    j = np.arange(ny, dtype=np.float64)
    phi = np.clip(ys[None, None, :] - j[None, :, None], 0.0, 1.0)
    phi = np.broadcast_to(phi, (nz, ny, nx)).copy()
    periodic = (True, False, True)
    fill, flags = classify(phi, None, periodic, q)
    rho = hydrostatic((nx, ny, nz), 1, g, depth, flags)
    return Scenario("gravity_wave", (nx, ny, nz), periodic, fill, flags, None, rho, q=q,
                    collision=collision, variant=variant, omega=omega_from_nu(nu),
                    g=(0.0, -g, 0.0), steps=steps,
                    meta=dict(depth=depth, a0=a0, wavelength=L, g_abs=g, nu=nu))


def dam_break(nx=256, ny=128, nz=64, W=64, H=64, D=None, g=1e-5, nu=1e-3, variant="OM", q=19,
              collision="TRT", steps=20000):
    """Rectangular dam break: closed box with no-slip walls, liquid column
    x < W, y < H, z < D (D = nz: full depth) at rest with hydrostatic pressure,
    gravity along -y."""
    D = nz if D is None else D
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    phi = ((i < W) & (j < H) & (k < D)).astype(np.float64)
    periodic = (False, False, False)
    fill, flags = classify(phi, None, periodic, q)
    rho = hydrostatic((nx, ny, nz), 1, g, float(H), flags)
    return Scenario("dam_break", (nx, ny, nz), periodic, fill, flags, None, rho, q=q,
                    collision=collision, variant=variant, omega=omega_from_nu(nu),
                    g=(0.0, -g, 0.0), steps=steps, meta=dict(W=W, H=H, D=D, g_abs=g, nu=nu))


def cylinder_dam_break(L=96, r_frac=0.3, h_frac=0.3, g=1e-5, nu=1e-3, variant="OM", q=27,
                       collision="TRT", steps=5000):
    """Cylindrical dam break in an L^3 box with no-slip walls: liquid cylinder
    (axis z, centred, radius r_frac*L, height h_frac*L) on the floor."""
    nx = ny = nz = int(L)
    R = r_frac * L
    Hh = h_frac * L
    cx = cy = L / 2.0

    def inside(x, y, z):
        return (((x - cx) ** 2 + (y - cy) ** 2) < R * R) & (z < Hh)

    phi = _subsample_fraction(inside, (nx, ny, nz))
    periodic = (False, False, False)
    fill, flags = classify(phi, None, periodic, q)
    rho = hydrostatic((nx, ny, nz), 2, g, Hh, flags)
    return Scenario("cylinder_dam_break", (nx, ny, nz), periodic, fill, flags, None, rho, q=q,
                    collision=collision, variant=variant, omega=omega_from_nu(nu),
                    g=(0.0, 0.0, -g), steps=steps, meta=dict(L=L, R=R, H=Hh, g_abs=g, nu=nu))


def cylinder_batch_params(n=64, seed=2207, lo=64, hi=160):
    """Seeded parameters of a batch of cylindrical dam breaks: cube sides
    U{lo..hi}, radius and height fractions U(0.2, 0.4)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n):
        L = int(rng.integers(lo, hi + 1))
        rf = float(rng.uniform(0.2, 0.4))
        hf = float(rng.uniform(0.2, 0.4))
        out.append(dict(L=L, r_frac=rf, h_frac=hf))
    return out


def cylinder_batch(n=64, seed=2207, lo=64, hi=160, **kw):
    """Batch of cylindrical dam breaks (see cylinder_batch_params)."""
    return [cylinder_dam_break(**prm, **kw) for prm in cylinder_batch_params(n, seed, lo, hi)]


def taylor_bubble(nx=160, ny=160, nz=1024, D=128, bubble_d=96, bubble_len=256, z0=128,
                  z_ref=512.0, g=1e-6, sigma=1e-4, nu=5e-3, variant="OM", q=19,
                  collision="TRT", steps=1000):
    """Rising Taylor bubble: cells outside a circular tube of diameter D (axis z)
    are obstacles; a gas cylinder of diameter bubble_d and length bubble_len
    with its bottom at z0; liquid elsewhere in the tube; gravity along -z;
    the bubble's pressure follows the bubble model."""
    cx, cy = nx / 2.0, ny / 2.0
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    obst = ((i + 0.5 - cx) ** 2 + (j + 0.5 - cy) ** 2) >= (D / 2.0) ** 2
    rb = bubble_d / 2.0

    def in_bubble(x, y, z):
        return (((x - cx) ** 2 + (y - cy) ** 2) < rb * rb) & (z >= z0) & (z < z0 + bubble_len)

    # sub-sample only the slab that holds the bubble
    zlo, zhi = max(0, int(z0) - 1), min(nz, int(z0 + bubble_len) + 2)
    frac = np.zeros((nz, ny, nx), np.float64)
    frac[zlo:zhi] = _subsample_fraction(in_bubble, (nx, ny, zhi - zlo), origin=(0.0, 0.0, float(zlo)))
    phi = 1.0 - frac
    periodic = (False, False, False)
    fill, flags = classify(phi, obst, periodic, q)
    rho = hydrostatic((nx, ny, nz), 2, g, z_ref, flags)
    return Scenario("taylor_bubble", (nx, ny, nz), periodic, fill, flags, None, rho, q=q,
                    collision=collision, variant=variant, omega=omega_from_nu(nu),
                    g=(0.0, 0.0, -g), sigma=sigma, bubble_model=True, steps=steps,
                    meta=dict(D=D, bubble_d=bubble_d, bubble_len=bubble_len, g_abs=g, nu=nu))


def _drop_geometry(L, R_frac, depth_frac, q):
    """Fill levels and cell types of a drop above a thin pool in an L^3 cube."""
    nx = ny = nz = int(L)
    depth = depth_frac * L
    R = R_frac * L
    zc = depth + R + 1.0
    c = L / 2.0

    def inside(x, y, z):
        return (((x - c) ** 2 + (y - c) ** 2 + (z - zc) ** 2) < R * R) | (z < depth)

    phi = _subsample_fraction(inside, (nx, ny, nz))
    return classify(phi, None, (True, True, False), q)


def _drop_state(fill, flags, L, R_frac, depth_frac, U, g, sigma, nu, variant, q, collision, steps):
    """Scenario of a drop impact from its fill levels and cell types: the pool
    hydrostatic below depth + 1 (rho = 1 + 3 g (depth - z)), the drop at
    rho = 1 moving with -U along z."""
    nx = ny = nz = int(L)
    depth = depth_frac * L
    R = R_frac * L
    fluid = (flags == LIQ) | (flags == IFACE)
    zc = np.arange(nz, dtype=np.float64) + 0.5
    above = np.repeat(zc > depth + 1.0, nx * ny)
    rho_layer = np.repeat(1.0 + 3.0 * g * (depth - zc), nx * ny)
    rho = np.where(fluid & ~above, rho_layer, 1.0)
    vel = np.zeros(3 * nx * ny * nz, np.float64)
    vel[2 * nx * ny * nz:][above & fluid] = -U
    return Scenario("drop_impact", (nx, ny, nz), (True, True, False), fill, flags, vel, rho, q=q,
                    collision=collision, variant=variant, omega=omega_from_nu(nu),
                    g=(0.0, 0.0, -g), sigma=sigma, steps=steps,
                    meta=dict(L=L, R=R, depth=depth, U=U, g_abs=g, nu=nu))


def drop_impact(L=96, R_frac=0.12, depth_frac=0.1, U=0.03, g=1e-5, sigma=1e-4, nu=1e-3,
                variant="OM", q=19, collision="TRT", steps=5000):
    """Drop onto a thin pool: L^3 cube, periodic x/y, no-slip z; pool depth
    depth_frac*L; sphere of radius R_frac*L centred at height pool + R + 1
    moving with velocity -U along z."""
    fill, flags = _drop_geometry(L, R_frac, depth_frac, q)
    return _drop_state(fill, flags, L, R_frac, depth_frac, U, g, sigma, nu, variant, q, collision, steps)


@dataclass
class CompactDrop:
    """A drop-impact initial state held as its cell types and the fill levels
    of its interface cells (about one byte per cell, against ~80 for the full
    host arrays); expand() rebuilds exactly the arrays of drop_impact()."""
    kw: dict
    flags: np.ndarray
    iface_fill: np.ndarray

    @property
    def shape(self):
        return (int(self.kw["L"]),) * 3

    @property
    def N(self):
        return int(self.flags.size)

    @property
    def depth(self):
        return self.kw["depth_frac"] * self.kw["L"]

    def expand(self) -> Scenario:
        fill = (self.flags == LIQ).astype(np.float64)
        fill[self.flags == IFACE] = self.iface_fill
        return _drop_state(fill, self.flags, **self.kw)


def drop_impact_compact(L=96, R_frac=0.12, depth_frac=0.1, U=0.03, g=1e-5, sigma=1e-4, nu=1e-3,
                        variant="OM", q=19, collision="TRT", steps=5000) -> CompactDrop:
    """drop_impact() in compact form (for request streams held on the host)."""
    fill, flags = _drop_geometry(L, R_frac, depth_frac, q)
    kw = dict(L=L, R_frac=R_frac, depth_frac=depth_frac, U=U, g=g, sigma=sigma, nu=nu, variant=variant, q=q,
              collision=collision, steps=steps)
    return CompactDrop(kw, flags, fill[flags == IFACE].copy())


def bubble_pair(shape=(24, 16, 16), r=3.5, gap=0.3, U=0.05, sigma=1e-3, nu=0.02, q=19, variant="OM"):
    """Two gas spheres of radius r in liquid (periodic box), their surfaces a
    distance ``gap`` apart along x, pushed together by a liquid velocity
    +-U along x (a Gaussian profile around their axis): the film between them
    drains and the gas regions connect and part again (bubble coalescence and
    segmentation), with the bubble model on."""
    nx, ny, nz = shape
    c1 = (nx / 2 - r - gap / 2, ny / 2, nz / 2)
    c2 = (nx / 2 + r + gap / 2, ny / 2, nz / 2)

    def inside(x, y, z):
        d1 = (x - c1[0]) ** 2 + (y - c1[1]) ** 2 + (z - c1[2]) ** 2
        d2 = (x - c2[0]) ** 2 + (y - c2[1]) ** 2 + (z - c2[2]) ** 2
        return ~((d1 < r * r) | (d2 < r * r))

    phi = _subsample_fraction(inside, (nx, ny, nz))
    per = (True, True, True)
    fill, flags = classify(phi, None, per, q)
    N = nx * ny * nz
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    prof = np.exp(-((j + 0.5 - ny / 2) ** 2 + (k + 0.5 - nz / 2) ** 2) / 18.0)
    ux = np.where(i + 0.5 < nx / 2, U, -U) * prof
    vel = np.zeros(3 * N, np.float64)
    live = (flags == LIQ) | (flags == IFACE)
    vel[:N] = np.where(live, ux.reshape(-1), 0.0)
    return Scenario("bubble_pair", (nx, ny, nz), per, fill, flags, vel, None, q=q, collision="TRT",
                    variant=variant, omega=omega_from_nu(nu), sigma=sigma, bubble_model=True,
                    meta=dict(r=r, gap=gap, U=U))


def drop_requests(n=200, seed=13962, rate=20.0, lo=96, hi=256, **kw):
    """Poisson-arrival stream of drop-impact requests: list of
    (arrival_time_s, scenario kwargs) with seeded sizes and parameters."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for _ in range(n):
        t += float(rng.exponential(1.0 / rate))
        L = int(rng.integers(lo, hi + 1))
        out.append((t, dict(L=L, R_frac=float(rng.uniform(0.08, 0.15)),
                            U=float(rng.uniform(0.02, 0.05)), **kw)))
    return out


# ------------------------------------------------------------------ pin cases

def flat_interface(nx=16, ny=32, nz=4, depth=16.5, g=0.0, nu=0.05, variant="OM", q=19,
                   collision="TRT", sigma=0.0):
    """Flat interface at y = depth, periodic x and z, walls in y, hydrostatic."""
    j = np.arange(ny, dtype=np.float64)
    phi = np.clip(depth - j, 0.0, 1.0)[None, :, None]
    phi = np.broadcast_to(phi, (nz, ny, nx)).copy()
    periodic = (True, False, True)
    fill, flags = classify(phi, None, periodic, q)
    rho = hydrostatic((nx, ny, nz), 1, g, depth, flags) if g else None
    return Scenario("flat_interface", (nx, ny, nz), periodic, fill, flags, None, rho, q=q,
                    collision=collision, variant=variant, omega=omega_from_nu(nu),
                    g=(0.0, -g, 0.0), sigma=sigma, meta=dict(depth=depth))


def static_drop(n=48, nz=1, R=12.0, sigma=0.01, nu=0.1, variant="OM", q=19, collision="TRT"):
    """Static drop (nz > 1: sphere) or cylinder (nz == 1: quasi-2-D) of radius R
    in a fully periodic box, no gravity."""
    nx = ny = int(n)
    c = n / 2.0
    if nz == 1:
        def inside(x, y, z):
            return ((x - c) ** 2 + (y - c) ** 2) < R * R
        phi = _subsample_fraction(inside, (nx, ny, 1), s=16)
    else:
        cz = nz / 2.0

        def inside(x, y, z):
            return ((x - c) ** 2 + (y - c) ** 2 + (z - cz) ** 2) < R * R
        phi = _subsample_fraction(inside, (nx, ny, nz))
    periodic = (True, True, True)
    fill, flags = classify(phi, None, periodic, q)
    return Scenario("static_drop", (nx, ny, nz), periodic, fill, flags, None, None, q=q,
                    collision=collision, variant=variant, omega=omega_from_nu(nu), sigma=sigma,
                    meta=dict(R=R))


def random_interface(shape=(37, 21, 11), seed=0, q=19, variant="OM", periodic=(True, False, True),
                     g=1e-4, sigma=1e-3, nu=0.02, collision="TRT", amp=3.0, obstacles=True,
                     velocity=0.02):
    """Rough, randomly perturbed free surface with random velocities and a few
    obstacle blocks: a stress case that exercises conversions in both
    directions, all mass-flux classes and the wall rules."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nx, ny, nz = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    kx, kz = rng.uniform(0.5, 2.0, 2)
    ph = rng.uniform(0, 2 * np.pi, 2)
    surf = ny / 2.0 + amp * np.sin(2 * np.pi * kx * i / nx + ph[0]) * np.cos(2 * np.pi * kz * k / max(nz, 1) + ph[1])
    surf = surf + rng.uniform(-0.7, 0.7, surf.shape)
    phi = np.clip(surf - j, 0.0, 1.0)
    # a droplet above the surface
    c = (nx * 0.3, ny * 0.8, nz * 0.5)
    d2 = (i + 0.5 - c[0]) ** 2 + (j + 0.5 - c[1]) ** 2 + (k + 0.5 - c[2]) ** 2
    phi = np.maximum(phi, np.clip(2.5 - np.sqrt(d2), 0.0, 1.0))
    obst = None
    if obstacles:
        obst = np.zeros((nz, ny, nx), bool)
        obst[:, : max(2, ny // 6), nx // 2: nx // 2 + 3] = True
        obst[:, ny // 3: ny // 3 + 2, : 3] = True
    fill, flags = classify(phi, obst, periodic, q)
    rho = np.where((flags == LIQ) | (flags == IFACE), 1.0 + rng.uniform(-2e-3, 2e-3, flags.size), 1.0)
    N = flags.size
    vel = rng.uniform(-velocity, velocity, 3 * N)
    fl3 = np.concatenate([flags, flags, flags])
    vel = np.where((fl3 == LIQ) | (fl3 == IFACE), vel, 0.0)
    return Scenario("random_interface", shape, periodic, fill, flags, vel, rho, q=q,
                    collision=collision, variant=variant, omega=omega_from_nu(nu),
                    g=(0.0, -g, 0.0), sigma=sigma, meta=dict(seed=seed))


def z_slab(sc: Scenario, zlo: int, zhi: int) -> Scenario:
    """The layers zlo <= k < zhi of a scenario's initial state as a domain of
    their own.  The cut faces become non-periodic (walls), and liquid cells
    that a cut exposes to a gas cell become interface cells (closure).  Cells
    far enough from the cuts evolve exactly as in the full domain for the
    first few steps, which lets a slab stand in for a domain too large for
    the CPU oracle."""
    nx, ny, nz = sc.shape
    zlo, zhi = max(0, zlo), min(nz, zhi)
    sl = slice(zlo * nx * ny, zhi * nx * ny)
    fill = sc.fill[sl].copy()
    flags = sc.flags[sl].copy()
    den = None if sc.density is None else sc.density[sl].copy()
    vel = None
    if sc.velocity is not None:
        N = sc.N
        vel = np.concatenate([sc.velocity[a * N:(a + 1) * N][sl] for a in range(3)])
    shape = (nx, ny, zhi - zlo)
    per = (sc.periodic[0], sc.periodic[1], False)
    f3 = flags.reshape(shape[2], ny, nx)
    p3 = fill.reshape(shape[2], ny, nx)
    gas = f3 == GAS
    for dx, dy, dz in neighbour_offsets(sc.q):
        sh = _shift(_shift(_shift(gas, dz, 0, per[2], False), dy, 1, per[1], False), dx, 2, per[0], False)
        fix = sh & (f3 == LIQ)
        f3[fix] = IFACE
        p3[fix] = 1.0
    return Scenario(f"{sc.name}[z={zlo}:{zhi}]", shape, per, fill, flags, vel, den, q=sc.q,
                    collision=sc.collision, variant=sc.variant, omega=sc.omega, g=sc.g,
                    sigma=sc.sigma, bubble_model=sc.bubble_model, meta=dict(sc.meta, zlo=zlo))


def make_oracle_kwargs(sc: Scenario, **over):
    """Keyword arguments shared by the GPU context and the oracle."""
    kw = dict(periodic=sc.periodic, q=sc.q, collision=sc.collision, variant=sc.variant,
              omega=sc.omega, g=sc.g, sigma=sc.sigma, bubble_model=sc.bubble_model)
    kw.update(over)
    return kw
