"""Batched ensembles of independent runs (uneven sizes) through the C ABI.

Every run of an ensemble must evolve exactly as the same run stepped alone:
the per-cell arithmetic does not depend on how cells are grouped into launches
(a cell's update and the max signal speed are independent of tiling; only the
per-block diagnostic partial sums regroup).  FP64 runs are also checked against
the oracle.
"""
import numpy as np
import pytest

import oracle as O
from paper_1311_0861_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def flic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    from paper_1311_0861_gb300 import flic as F
    if not os.path.exists(F.LIB_PATH):
        from paper_1311_0861_gb300 import build
        build.build()
    F.load()
    return F


def _states(sizes, seed0):
    return [I.random_state((n, n, n), seed=seed0 + i, box=2.0) for i, n in enumerate(sizes)]


@pytest.mark.parametrize("precision,poisson", [("fp64", "periodic"), ("mixed", "periodic"), ("fp64", "isolated")])
def test_ensemble_runs_equal_single_runs(flic, precision, poisson):
    sizes = [16, 24, 16, 32, 12, 24]
    sts = _states(sizes, 100)
    with flic.Ensemble(sizes, precision=precision, poisson=poisson) as ens:
        for r, s in enumerate(sts):
            ens.set_state(r, s.state)
        ens.step(3)
        outs = [ens.get_state(r) for r in range(len(sizes))]
        recs = [ens.diagnostics(r) for r in range(len(sizes))]
    for r, (n, s) in enumerate(zip(sizes, sts)):
        with flic.Grid(n, precision=precision, poisson=poisson) as g:
            g.set_state(s.state)
            g.run(3)
            ref = g.get_state()
            d = g.step_diagnostics()
        for f in flic.FIELDS:
            assert np.array_equal(outs[r][f], ref[f]), (r, f)
        assert recs[r]["dt"] == d["dt"] and recs[r]["step"] == 3
        # the per-block partial sums regroup with the launch geometry: float64
        # sums agree to rounding, float32 compensated sums (mixed) to ~1e-10
        tol = 1e-12 if precision == "fp64" else 1e-8
        for k in ("mass_gas", "mass_bme", "ekin_gas", "epot", "kappa_bme"):
            assert abs(recs[r][k] - d[k]) <= tol * max(1e-30, abs(d[k])), (r, k)


def test_ensemble_fp64_matches_oracle(flic):
    sizes = [16, 24]
    sts = _states(sizes, 200)
    with flic.Ensemble(sizes, precision="fp64") as ens:
        for r, s in enumerate(sts):
            ens.set_state(r, s.state)
        ens.step(2)
        outs = [ens.get_state(r) for r in range(len(sizes))]
    for r, s in enumerate(sts):
        ref, _ = O.run(s.state, O.Params(h=s.h, gamma=s.gamma), 2)
        for f in flic.FIELDS:
            err = np.sum(np.abs(outs[r][f] - ref[f])) / max(1e-300, np.sum(np.abs(ref[f])))
            assert err <= 1e-10, (r, f, err)


def test_ensemble_collision_members(flic):
    """The 64-run collision ensemble recipe, first members, mixed precision."""
    members = [I.ensemble_member(r) for r in range(4)]
    sizes = [m.shape[0] for m in members]
    with flic.Ensemble(sizes, precision="mixed") as ens:
        for r, m in enumerate(members):
            ens.set_state(r, m.state)
        ens.step(5)
        for r in range(len(sizes)):
            d = ens.diagnostics(r)
            assert d["step"] == 5 and not d["nonphysical"]


def test_ensemble_rejects_mixed_constants(flic):
    import ctypes
    lib = flic.load()
    descs = (flic.GridDesc * 2)(flic.GridDesc(16, -1, 1, 5 / 3, 1, 0.2, 1e-3, 0, 0),
                                flic.GridDesc(16, -1, 1, 1.4, 1, 0.2, 1e-3, 0, 0))
    out = ctypes.c_void_p()
    assert lib.flic_ensemble_create(descs, 2, None, ctypes.byref(out)) == flic.ERR_INVALID_ARG


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ensemble_outflow_and_cooling(flic, precision):
    """Outflow boundaries with isolated gravity, and the cooling placeholder: every
    run of the ensemble equals the same run stepped alone."""
    sizes = [16, 24, 12]
    sts = _states(sizes, 300)
    for opts in ({"boundary": "outflow", "poisson": "isolated"}, {"cooling": 0.6}):
        with flic.Ensemble(sizes, precision=precision, **opts) as ens:
            for r, s in enumerate(sts):
                ens.set_state(r, s.state)
            ens.step(3)
            outs = [ens.get_state(r) for r in range(len(sizes))]
        for r, (n, s) in enumerate(zip(sizes, sts)):
            with flic.Grid(n, precision=precision, **opts) as g:
                g.set_state(s.state)
                g.run(3)
                ref = g.get_state()
            for f in flic.FIELDS:
                assert np.array_equal(outs[r][f], ref[f]), (opts, r, f)
