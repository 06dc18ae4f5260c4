"""Accuracy gates at the benchmark's full size: the 256^3 head-on two-galaxy
collision advanced 10 CFL steps on the GPU and by the oracle over the whole grid.

The oracle steps all 256^3 cells (``oracle.slab_pool``: the oracle's own step,
evaluated slab by slab on the host cores), so errors that grow over the steps are
seen at the size the benchmark times.
  * FP64 path: relative L1 (sum |a - b| / sum |b|) at most 1e-10 on every one of
    the 22 fields after 10 steps, and every step's CFL step size within 1e-13
    (relative) of the oracle's.
  * Mixed path (float32 bulk): relative L1 at most 1e-4 in the gas and
    collisionless densities after 10 steps, relative mass drift at most 1e-6;
    the other 20 fields are held to the bounds in MIXED_L1, each set about 10x
    above the error measured on GB300.
Set FLIC_GATE_REPORT to a file path to have the per-field errors written there
as JSON.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from oracle.slab_pool import SlabPool, host_cores
from paper_1311_0861_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N = 256
STEPS = 10
FIELDS = O.FIELDS

# per-field bounds of the mixed path after 10 steps: the 1e-4 gate for the
# densities, about ten times the error measured on GB300 for the rest (measured:
# rho 2.2e-7, n 9.9e-8, momenta 1e-7..1.1e-6, E 3.8e-7, e 2.4e-6, energy tensor
# 9e-8..2e-6, dispersion tensor 1e-7..8e-6)
MIXED_L1 = {"rho": 1e-4, "n": 1e-4,
            "mx": 5e-6, "my": 5e-6, "mz": 5e-6, "E": 5e-6, "e": 3e-5,
            "qx": 2e-6, "qy": 2e-5, "qz": 2e-5,
            "nExx": 2e-6, "nEyy": 2e-6, "nEzz": 2e-6, "nExy": 2e-5, "nExz": 2e-5, "nEyz": 2e-5,
            "Pxx": 5e-6, "Pyy": 2e-6, "Pzz": 2e-6, "Pxy": 1e-4, "Pxz": 1e-4, "Pyz": 2e-5}


def rel_l1(a, b):
    return float(np.sum(np.abs(a - b)) / max(1e-300, np.sum(np.abs(b))))


@pytest.fixture(scope="module")
def gate():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_0861_gb300 import flic
    if not os.path.exists(flic.LIB_PATH):
        from paper_1311_0861_gb300 import build
        build.build()
    flic.load()
    s = I.head_on(N)
    prm = O.Params(h=s.h, gamma=s.gamma)
    with SlabPool((N, N, N), workers=host_cores()) as pool:
        ref, recs = pool.run(s.state, prm, STEPS)
    report = {"n": N, "steps": STEPS, "oracle_dt": [r["dt"] for r in recs]}
    yield flic, s, ref, recs, report
    path = os.environ.get("FLIC_GATE_REPORT")
    if path:
        with open(path, "w") as f:
            json.dump(report, f, indent=1)


def test_fp64_ten_steps_all_fields(gate):
    flic, s, ref, recs, report = gate
    dts = []
    with flic.Grid(N, precision="fp64", gamma=s.gamma) as g:
        g.set_state(s.state)
        for _ in range(STEPS):
            dts.append(g.step())
        out = g.get_state()
    dt_err = [abs(a - r["dt"]) / r["dt"] for a, r in zip(dts, recs)]
    err = {f: rel_l1(out[f], ref[f]) for f in FIELDS}
    report["fp64_rel_l1"] = err
    report["fp64_dt_rel_err"] = dt_err
    assert max(dt_err) <= 1e-13, dt_err
    assert max(err.values()) <= 1e-10, err


def test_mixed_ten_steps_all_fields(gate):
    flic, s, ref, recs, report = gate
    with flic.Grid(N, precision="mixed", gamma=s.gamma) as g:
        g.set_state(s.state)
        d0 = g.diagnostics()
        dts = []
        for _ in range(STEPS):
            dts.append(g.step())
        d1 = g.diagnostics()
        out = g.get_state()
    err = {f: rel_l1(out[f], ref[f]) for f in FIELDS}
    drift = {k: abs(d1[k] - d0[k]) / d0[k] for k in ("mass_gas", "mass_bme")}
    report["mixed_rel_l1"] = err
    report["mixed_mass_drift"] = drift
    report["mixed_dt_rel_err"] = [abs(a - r["dt"]) / r["dt"] for a, r in zip(dts, recs)]
    assert err["rho"] <= 1e-4 and err["n"] <= 1e-4, err
    assert max(drift.values()) <= 1e-6, drift
    bad = {f: e for f, e in err.items() if e > MIXED_L1[f]}
    assert not bad, bad
