"""Bubble coalescence and segmentation on the device (fslbm_params.
bubble_relabel_every; reading R24) against the oracle with the same
relabelling interval: two bubbles pushed together merge and part again
several times within the run, and the FP64 engine follows the oracle's
trajectory (flags identical, fill levels and PDFs within relative 1e-12,
bubble volumes and pressures within relative 1e-12) through every
relabelling.  The batch and the server reject contexts that relabel."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2207_13962_gb300 import scenarios as S

pytestmark = pytest.mark.gpu


def _close(a, b, rel=1e-12):
    return np.all(np.abs(a - b) <= rel * np.abs(b))


@pytest.mark.parametrize("every", [1, 5])
def test_relabelling_matches_oracle(every, gpu_lib):
    from paper_2207_13962_gb300 import fslbm
    sc = S.bubble_pair(gap=0.3, U=0.05)
    o = Oracle(*sc.shape, **S.make_oracle_kwargs(sc), bubble_relabel_every=every)
    o.init(sc.fill, sc.flags, sc.velocity, sc.density)
    g = fslbm.context_for(sc, precision="FP64", bubble_relabel_every=every)
    counts = set()
    for s in range(1, 81):
        o.step(1)
        g.step(1)
        Vo, Po, ido = o.bubbles()
        Vg, Pg = g.bubbles()
        counts.add(len(Vo))
        assert len(Vg) == len(Vo), s
        assert _close(Vg, Vo) and _close(Pg, Po), s
        if s % 10 == 0:
            ro, rg = o.read(), g.read()
            np.testing.assert_array_equal(rg["flags"], ro["flags"])
            fl = ro["flags"]
            fluid = (fl == S.LIQ) | (fl == S.IFACE)
            assert _close(rg["fill"], ro["fill"])
            assert _close(rg["pdf"][:, fluid], ro["pdf"][:, fluid])
    # the run saw both one and two bubbles
    assert {1, 2} <= counts, counts
    g.close()


def test_relabelling_fp32_and_checkpoint(gpu_lib):
    """The FP32 engine relabels too; a checkpoint taken while the bubble count
    differs from the initial one loads into a fresh context, which then
    continues bit for bit like the run it was taken from."""
    from paper_2207_13962_gb300 import fslbm
    sc = S.bubble_pair(gap=0.3, U=0.05)
    g = fslbm.context_for(sc, precision="FP32", bubble_relabel_every=1)
    n0 = len(g.bubbles()[0])
    blob = None
    seen = {n0}
    for s in range(1, 81):
        g.step(1)
        n = len(g.bubbles()[0])
        seen.add(n)
        if n != n0:
            blob = g.save()
            break
    assert blob is not None, seen
    h = fslbm.context_for(sc, precision="FP32", bubble_relabel_every=1)
    assert len(h.bubbles()[0]) == n0
    h.load(blob)
    assert len(h.bubbles()[0]) == n
    g.step(7)
    h.step(7)
    np.testing.assert_array_equal(h.read()["pdf"], g.read()["pdf"])
    np.testing.assert_array_equal(h.bubbles()[1], g.bubbles()[1])
    for c in (g, h):
        c.close()


def test_batch_and_server_reject_relabelling(gpu_lib):
    from paper_2207_13962_gb300 import fslbm
    sc = S.bubble_pair()
    c = fslbm.context_for(sc, precision="FP32", bubble_relabel_every=3)
    with pytest.raises(fslbm.FslbmError) as e:
        fslbm.Batch([c])
    assert e.value.status == fslbm.EINVAL
    c.close()
    srv = fslbm.Server(q=19, precision="FP32", max_active=2, chunk_steps=2)
    with pytest.raises(fslbm.FslbmError) as e:
        srv.submit(sc, 4, bubble_relabel_every=3)
    assert e.value.status == fslbm.EINVAL
    srv.close()
