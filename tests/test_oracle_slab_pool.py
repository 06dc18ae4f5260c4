"""The slab-parallel driver of the oracle reproduces the oracle's whole-grid steps.

Each slab is ``advance_window`` with a two-plane margin, which equals ``advance``
on the whole grid cell by cell, so the driver's states must equal ``oracle.run``
bit for bit (periodic and outflow grids, slabs that do not divide the grid, one
and several workers).
"""
import numpy as np
import pytest

import oracle as O
from oracle.slab_pool import SlabPool, host_cores
from paper_1311_0861_gb300 import inputs as I


@pytest.mark.parametrize("boundary,poisson,slab,workers", [("periodic", "periodic", 5, 2),
                                                            ("outflow", "isolated", 3, 3),
                                                            ("periodic", "periodic", 16, 1)])
def test_slab_pool_equals_whole_grid(boundary, poisson, slab, workers):
    s = I.random_state((16, 16, 16), seed=11, rough=True)
    prm = O.Params(h=s.h, gamma=s.gamma, poisson=poisson, boundary=boundary)
    ref, rrec = O.run(s.state, prm, 2)
    with SlabPool((16, 16, 16), workers=workers, slab=slab) as pool:
        out, recs = pool.run(s.state, prm, 2)
    for f in O.FIELDS:
        assert np.array_equal(out[f], ref[f]), f
    for a, b in zip(recs, rrec):
        assert a["dt"] == b["dt"] and a["vmax"] == b["vmax"]


def test_slab_pool_kappa_and_fixed_dt():
    s = I.random_state((12, 12, 12), seed=12)
    prm = O.Params(h=s.h, gamma=s.gamma)
    ref, rrec = O.step(s.state, prm, dt=1e-3)
    with SlabPool((12, 12, 12), workers=2, slab=4) as pool:
        pool.load(s.state)
        rec = pool.step(prm, dt=1e-3, with_kappa=True)
        out = pool.state()
    assert rec["dt"] == 1e-3
    for f in O.FIELDS:
        assert np.array_equal(out[f], ref[f]), f
    for k in ("kappa_gas", "kappa_bme"):
        assert abs(rec[k] - rrec[k]) <= 1e-13 * abs(rrec[k])


def test_host_cores_positive():
    assert host_cores() >= 1
