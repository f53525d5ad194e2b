"""Pins of the oracle's bubble coalescence and segmentation (reading R24;
Sec. 2.2 cites a bubble model that follows them without giving it).

Each relabelling is checked against what physics and the reading fix, with
arithmetic of the test's own (fixed-point volumes summed from the fields):
  * with no change of the gas regions it changes nothing, bit for bit;
  * the new labels are the connected gas components of the current flags
    (scipy.ndimage.label with the lattice neighbourhood, periodic);
  * the gas amount sum_b p_b V_b of the bubbles that hand cells on to new ones
    is conserved, plus p^V(0) times the volume of gas and interface cells that
    carried no id (they hold gas at p^V(0));
  * a bubble formed by merging old bubbles A and B only has Boyle's pressure
    (p_A V_A + p_B V_B) / (V_A + V_B); a part of a split bubble keeps its
    pressure.
The two-bubble case pushes the bubbles together until the film between them
drains: within 80 steps they merge and part again several times."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2207_13962_gb300 import scenarios as S

GAS, IFACE = 0, 1
FIX = 4294967296.0


def _vol(flags, fill, mask):
    """Fixed-point volume (gas 1, interface 1 - phi, 2^-32 steps) of the cells in mask."""
    g = (flags == GAS) & mask
    i = (flags == IFACE) & mask
    v = int(g.sum()) * (1 << 32) + int(np.rint((1.0 - fill[i]) * FIX).astype(np.int64).sum())
    return v / FIX


def _components(flags, shape, q):
    ndimage = pytest.importorskip("scipy.ndimage")
    nx, ny, nz = shape
    gas = (flags == GAS).reshape(nz, ny, nx)
    st = np.zeros((3, 3, 3), bool)
    for dx, dy, dz in S.neighbour_offsets(q):
        st[dz + 1, dy + 1, dx + 1] = True
    st[1, 1, 1] = True
    big = np.tile(gas, (3, 3, 3))
    lab, _ = ndimage.label(big, structure=st)
    return lab[nz:2 * nz, ny:2 * ny, nx:2 * nx].reshape(-1)


def test_relabel_without_change_is_the_identity():
    sc = S.bubble_pair()
    o = Oracle(*sc.shape, **S.make_oracle_kwargs(sc))
    o.init(sc.fill, sc.flags, sc.velocity, sc.density)
    o.step(2)
    V0, P0, ids0 = o.bubbles()
    o.relabel_bubbles()
    V1, P1, ids1 = o.bubbles()
    np.testing.assert_array_equal(ids0, ids1)
    np.testing.assert_array_equal(V0, V1)
    np.testing.assert_array_equal(P0, P1)


def test_merges_and_splits_conserve_gas():
    sc = S.bubble_pair(gap=0.3, U=0.05)
    pv0 = 1.0 / 3.0
    o = Oracle(*sc.shape, **S.make_oracle_kwargs(sc))
    o.init(sc.fill, sc.flags, sc.velocity, sc.density)
    merges = splits = 0
    for step in range(80):
        o.step(1)
        V0, P0, ids0 = o.bubbles()
        r = o.read()
        flags, fill = r["flags"], r["fill"]
        o.relabel_bubbles()
        V1, P1, ids1 = o.bubbles()
        # labels: the connected gas components, numbered by lowest index
        comp = _components(flags, sc.shape, sc.q)
        gas = flags == GAS
        for b in range(len(V1)):
            members = np.unique(comp[gas & (ids1 == b)])
            assert members.size == 1
        assert len(V1) == len(np.unique(comp[gas]))
        firsts = [np.nonzero(gas & (ids1 == b))[0].min() for b in range(len(V1))]
        assert firsts == sorted(firsts)
        # volumes follow the fields
        for b in range(len(V1)):
            assert V1[b] == _vol(flags, fill, ids1 == b)
        # gas amount: sum p V of the old bubbles that hand cells on, plus the
        # cells without an id at p^V(0)
        free = (ids0 < 0) & (ids1 >= 0)
        kept = [A for A in range(len(V0)) if ((ids0 == A) & (ids1 >= 0)).any()]
        before = float(sum(P0[A] * V0[A] for A in kept)) + pv0 * _vol(flags, fill, free)
        after = float(np.dot(P1, V1))
        assert after == pytest.approx(before, rel=1e-13)
        # Boyle for pure merges, unchanged pressure for pure split parts
        # (old bubbles that hand every cell on, new bubbles without free cells)
        held = (flags == GAS) | (flags == IFACE)
        for C in range(len(V1)):
            cells = ids1 == C
            olds = set(np.unique(ids0[cells]).tolist())
            if -1 in olds or any(((ids0 == A) & (ids1 < 0) & held).any() for A in olds):
                continue
            parts_elsewhere = any(((ids0 == A) & (ids1 != C) & held).any() for A in olds)
            if len(olds) > 1 and not parts_elsewhere:
                merges += 1
                A = sorted(olds)
                expect = sum(P0[a] * V0[a] for a in A) / sum(V0[a] for a in A)
                assert P1[C] == pytest.approx(expect, rel=1e-13)
            if len(olds) == 1 and len(V1) > len(V0):
                (A,) = olds
                splits += 1
                assert P1[C] == pytest.approx(P0[A], rel=1e-13)
    assert merges > 0 and splits > 0, (merges, splits)


def test_relabel_every_k_steps_in_the_step():
    """relabel_every = K runs the same relabelling after every K-th step."""
    sc = S.bubble_pair(gap=0.3, U=0.05)
    a = Oracle(*sc.shape, **S.make_oracle_kwargs(sc), bubble_relabel_every=4)
    b = Oracle(*sc.shape, **S.make_oracle_kwargs(sc))
    for o in (a, b):
        o.init(sc.fill, sc.flags, sc.velocity, sc.density)
    for s in range(1, 25):
        a.step(1)
        b.step(1)
        if s % 4 == 0:
            b.relabel_bubbles()
    ra, rb = a.read(), b.read()
    np.testing.assert_array_equal(ra["pdf"], rb["pdf"])
    np.testing.assert_array_equal(a.bubbles()[1], b.bubbles()[1])
