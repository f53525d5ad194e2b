"""Host-side logic that needs no GPU.

* the multiply-high division by invariant integers used to decode cell
  coordinates (Granlund & Montgomery 1994), emulated exactly in Python for
  the magic numbers the library computes;
* the seeded scenario generators (closure of the interface layer, mass of the
  initial state, seeds of the batched and served workloads).
"""
import numpy as np
import pytest

from paper_2207_13962_gb300 import scenarios as S


def _magic(d):
    l = 0
    while (1 << l) < d:
        l += 1
    m = ((((1 << l) - d) << 32) // d + 1) & 0xFFFFFFFF
    return m, l


def _div(n, m, l):
    return (((n * m) >> 32) + n) >> l


@pytest.mark.parametrize("d", [1, 2, 3, 5, 7, 32, 37, 64, 96, 100, 128, 160, 255, 256, 1000, 1024,
                               4099, 65535, 1 << 20, (1 << 31) - 1])
def test_fastdiv_matches_integer_division(d):
    m, l = _magic(d)
    rng = np.random.default_rng(d)
    ns = list(rng.integers(0, 2 ** 31, 20000)) + [0, 1, d - 1, d, d + 1, 2 ** 31 - 1,
                                                  (2 ** 31 - 1) // d * d, (2 ** 31 - 1) // d * d - 1]
    for n in ns:
        n = int(n)
        if n < 0:
            continue
        assert _div(n, m, l) == n // d, (n, d)
        assert ((n * m) >> 32) + n < 2 ** 32  # the 32-bit sum cannot overflow


@pytest.mark.parametrize("maker", [lambda: S.gravity_wave(), lambda: S.dam_break(nx=64, ny=32, nz=16, W=16, H=16),
                                   lambda: S.cylinder_dam_break(L=40, q=27), lambda: S.drop_impact(L=48),
                                   lambda: S.taylor_bubble(nx=24, ny=24, nz=64, D=20, bubble_d=12,
                                                           bubble_len=20, z0=12, z_ref=40.0),
                                   lambda: S.random_interface(seed=9)])
def test_generators_close_the_interface_layer(maker):
    sc = maker()
    nx, ny, nz = sc.shape
    f = sc.flags.reshape(nz, ny, nx)
    gas = f == S.GAS
    for dx, dy, dz in S.neighbour_offsets(sc.q):
        sh = S._shift(S._shift(S._shift(gas, dz, 0, sc.periodic[2], False), dy, 1, sc.periodic[1], False),
                      dx, 2, sc.periodic[0], False)
        assert not np.any(sh & (f == S.LIQ))
    assert np.all((sc.fill >= 0) & (sc.fill <= 1))
    assert np.all(sc.fill[sc.flags == S.LIQ] == 1.0) and np.all(sc.fill[sc.flags == S.GAS] == 0.0)


def test_gravity_wave_initial_amplitude():
    sc = S.gravity_wave()
    a0 = sc.fill.reshape(64, 32)[:, 0].sum() - 32.0
    assert abs(a0 - 0.32) < 1e-12


def test_dam_break_column_volume():
    sc = S.dam_break()
    assert sc.fill.sum() == 64 * 64 * 64
    assert sc.N == 256 * 128 * 64


def test_batch_and_request_seeds_are_reproducible():
    a = S.cylinder_batch_params(n=64)
    b = S.cylinder_batch_params(n=64)
    assert a == b and all(64 <= p["L"] <= 160 and 0.2 <= p["r_frac"] <= 0.4 for p in a)
    r1 = S.drop_requests(n=10)
    r2 = S.drop_requests(n=10)
    assert [t for t, _ in r1] == [t for t, _ in r2]
    assert all(96 <= kw["L"] <= 256 and 0.08 <= kw["R_frac"] <= 0.15 for _, kw in r1)


def test_sector_census_bounds():
    """The bulk sweep's sector census (bench.py --sector-census) on the dam
    break: every count lies between the algorithmic bytes and the whole-line
    bound, in the order the memory hierarchy implies."""
    import bench
    c = bench.sector_census("dam_break")
    assert c["liquid_cells"] > 0 and 0.0 < c["lane_occupancy"] <= 1.0
    assert c["segments"] >= c["liquid_cells"] / 32
    distinct = c["distinct_read_sectors"]
    # 19 FP32 pulls per liquid cell can never fit in fewer sectors than bytes / 32
    assert distinct * 32 >= c["algorithmic_read_MB"] * 1e6 - 1
    assert distinct <= c["warp_sector_requests"]
    assert distinct <= c["read_sectors_64B_chunks"] <= c["read_sectors_128B_lines"]
    assert c["partial_write_sectors"] >= 0 and c["reflected_write_sectors"] >= 0


def test_compact_drop_expands_to_the_full_arrays():
    """The request stream holds drop impacts as cell types plus interface
    fill levels; expanding them must give exactly the generator's arrays."""
    for kw in (dict(L=33, R_frac=0.14, U=0.045), dict(L=48, R_frac=0.08, U=0.02)):
        full = S.drop_impact(**kw)
        comp = S.drop_impact_compact(**kw)
        assert comp.flags.nbytes + comp.iface_fill.nbytes < 2 * comp.N
        back = comp.expand()
        for a, b in ((full.fill, back.fill), (full.flags, back.flags), (full.velocity, back.velocity),
                     (full.density, back.density)):
            np.testing.assert_array_equal(a, b)
        assert back.meta == full.meta and back.shape == full.shape


def test_request_replay_and_expander():
    """The serving benchmark's replay: requests start no earlier than their
    arrival, every one finishes once, time-to-result is measured from the
    arrival, and the worker-thread expansion gives the generator's arrays."""
    import sys
    import os
    import time
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    trace = S.drop_requests(n=5, rate=50.0, lo=20, hi=28)
    comp = [S.drop_impact_compact(**kw) for _, kw in trace]
    arrivals = [t for t, _ in trace]
    exp = bench._Expander(comp, 2)
    started = {}
    t0 = [None]

    def step(ready):
        if t0[0] is None:
            t0[0] = time.perf_counter()
        exp.prefetch(ready)
        if not ready:
            return [], False
        k = ready.pop(0)
        started[k] = time.perf_counter() - t0[0]
        sc = exp.take(k)
        full = S.drop_impact(**trace[k][1])
        np.testing.assert_array_equal(sc.velocity, full.velocity)
        return [(k, {"k": k})], True

    res, makespan = bench._replay(arrivals, step)
    exp.close()
    assert sorted(res) == list(range(5))
    for k in range(5):
        assert started[k] >= arrivals[k] - 0.05
        assert res[k]["ttr"] >= 0.0
    assert makespan >= arrivals[-1] - 0.05


def test_openmp_oracle_equals_single_thread():
    """The all-core CPU baseline times the oracle built with OpenMP over its
    stream-collide cell loop; it must compute exactly what the single-thread
    oracle computes (each cell's arithmetic is independent of the others)."""
    from oracle import Oracle
    sc = S.random_interface(shape=(14, 12, 9), seed=5)
    runs = []
    for omp in (False, True):
        o = Oracle(*sc.shape, **S.make_oracle_kwargs(sc), openmp=omp)
        o.init(sc.fill, sc.flags, sc.velocity, sc.density)
        o.step(12)
        runs.append(o.read())
    for key in ("pdf", "fill", "flags", "mass"):
        np.testing.assert_array_equal(runs[0][key], runs[1][key], err_msg=key)
