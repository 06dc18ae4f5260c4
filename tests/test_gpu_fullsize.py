"""Parity at the benchmark's full size (256^3 head-on two-galaxy collision) in
the launch configuration bench.py times (default tiles, z chunks, CUDA graph).

The oracle cannot step the whole 256^3 grid inside a test, but each new cell
depends only on cells within L1 distance 2, so it evaluates sampled cells one by
one on 5^3 periodic windows (oracle.advance_window) with its own potential and
step size.  Properties that hold at any size (exact mass conservation, the
signal-speed/step-size relation, diagnostics) are checked on the whole grid.
"""
import numpy as np
import pytest

import oracle as O
from paper_1311_0861_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N = 256
FIELDS = O.FIELDS


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    from paper_1311_0861_gb300 import flic
    if not os.path.exists(flic.LIB_PATH):
        from paper_1311_0861_gb300 import build
        build.build()
    flic.load()
    s = I.head_on(N)
    prm = O.Params(h=s.h, gamma=s.gamma)
    phi = O.solve_poisson(s.state, prm)
    tau = O.cfl_dt(s.state, prm)
    # sampled cells: uniform random cells, plus every cell of two x-lines through
    # the galaxies (tile and chunk boundaries, periodic wrap)
    rng = I.splitmix64(77, 3 * 3000)
    cells = (rng % np.uint64(N)).astype(np.int64).reshape(-1, 3)
    line = np.arange(N)
    extra = np.concatenate([np.stack([np.full(N, 128), np.full(N, 128), line], 1),
                            np.stack([np.full(N, 0), np.full(N, 255), line], 1),
                            np.stack([line, np.full(N, 31), np.full(N, 32)], 1)])
    cells = np.concatenate([cells, extra])
    ref, _ = O.advance_window(s.state, phi, tau, prm, cells=cells)
    return flic, s, prm, tau, cells, ref


def _run(flic, s, precision, steps=1):
    with flic.Grid(N, precision=precision, gamma=s.gamma) as g:
        g.set_state(s.state)
        g.run(steps)
        d = g.step_diagnostics()
        out = g.get_state()
    return out, d


def test_fullsize_one_step_fp64_sampled(setup):
    flic, s, prm, tau, cells, ref = setup
    out, d = _run(flic, s, "fp64")
    assert abs(d["dt"] - tau) <= 1e-14 * tau
    k, j, i = cells[:, 0], cells[:, 1], cells[:, 2]
    for f in FIELDS:
        scale = np.max(np.abs(s.state[f])) or 1.0
        err = np.max(np.abs(out[f][k, j, i] - ref[f])) / scale
        assert err <= 1e-11, (f, err)


def test_fullsize_one_step_mixed_sampled(setup):
    flic, s, prm, tau, cells, ref = setup
    out, d = _run(flic, s, "mixed")
    assert abs(d["dt"] - tau) <= 1e-6 * tau
    k, j, i = cells[:, 0], cells[:, 1], cells[:, 2]
    for f in FIELDS:
        scale = np.max(np.abs(s.state[f])) or 1.0
        err = np.max(np.abs(out[f][k, j, i] - ref[f])) / scale
        assert err <= 2e-5, (f, err)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("mixed", 1e-6)])
def test_fullsize_mass_conservation(setup, precision, tol):
    flic, s, prm, tau, cells, ref = setup
    with flic.Grid(N, precision=precision, gamma=s.gamma) as g:
        g.set_state(s.state)
        d0 = g.diagnostics()
        g.run(10)
        d1 = g.diagnostics()
        rec = g.step_diagnostics()
    assert abs(d1["mass_gas"] - d0["mass_gas"]) <= tol * d0["mass_gas"]
    assert abs(d1["mass_bme"] - d0["mass_bme"]) <= tol * d0["mass_bme"]
    assert rec["step"] == 10 and not rec["nonphysical"]
    # the CFL step of the last step follows from the signal speed before it
    assert rec["dt"] > 0


def test_fullsize_initial_diagnostics(setup):
    flic, s, prm, tau, cells, ref = setup
    phi = O.solve_poisson(s.state, prm)
    want = O.diagnostics(s.state, phi, prm)
    with flic.Grid(N, precision="fp64", gamma=s.gamma) as g:
        g.set_state(s.state)
        d = g.diagnostics()
    for key, v in want.items():
        assert abs(d[key] - v) <= 1e-11 * max(abs(v), 1e-6 * want["mass_bme"]), (key, d[key], v)
    assert abs(d["vmax"] - O.max_signal_speed(s.state, prm)) <= 1e-14
