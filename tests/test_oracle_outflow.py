"""Pins of the oracle's outflow (zero-gradient) hydro boundaries.

Outflow is the first widening of the hot path: the paper states no hydro
boundary (periodic is the default reading), and galaxies leave a periodic box
in long collision runs.  The ghost-cell definition (two layers of edge copies of
the time-n state and potential, the step computed on the extended grid) is a
reading; these tests pin what it must do whatever its internals:
  * a uniform state, moving or not, is a fixed point;
  * cells more than 2 cells from every boundary update exactly as on a periodic
    grid (the boundary reaches no further than the stencil);
  * the canonical single-interface tubes of Table 2 on [0, 1] converge to the
    exact Riemann solutions (waves leave without a periodic image);
  * a right-moving acoustic pulse leaves the box: the state returns to the
    background (on a periodic grid it would come back);
  * mirror symmetry and axis permutation commute with the step;
  * the evaluation on windows (used by the full-size GPU tests) equals the
    whole-grid step near the boundaries.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from exact_riemann import sample
from helpers import TENSOR, permute_state, reflect_x, run_to, state_from_primitives, tube_state
from paper_1311_0861_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_uniform_moving_state_is_fixed_point():
    N = 10
    one = np.ones((N, N, N))
    P = {"xx": 0.5 * one, "yy": 0.7 * one, "zz": 0.6 * one, "xy": 0.1 * one, "xz": -0.05 * one, "yz": 0.02 * one}
    st = state_from_primitives(1.3 * one, (0.4 * one, -0.2 * one, 0.1 * one), 0.8 * one, 0.9 * one,
                               (-0.15 * one, 0.3 * one, 0.1 * one), P, 5.0 / 3.0)
    prm = O.Params(h=0.2, G=0.0, boundary="outflow")
    out, _ = O.run(st, prm, 3)
    for f in O.FIELDS:
        assert np.max(np.abs(out[f] - st[f])) <= 1e-14 * max(1.0, np.max(np.abs(st[f]))), f


def test_interior_equals_periodic():
    s = I.random_state((16, 16, 16), seed=11, rough=True)
    prm_p = O.Params(h=s.h, poisson="isolated")
    prm_o = O.Params(h=s.h, poisson="isolated", boundary="outflow")
    phi = O.solve_poisson(s.state, prm_p)
    a, _ = O.advance(s.state, phi, 2e-3, prm_p)
    b, _ = O.advance(s.state, phi, 2e-3, prm_o)
    inner = (slice(3, -3),) * 3
    edge_differs = False
    for f in O.FIELDS:
        assert np.array_equal(a[f][inner], b[f][inner]), f
        edge_differs |= not np.array_equal(a[f], b[f])
    assert edge_differs


@pytest.mark.parametrize("tid", ["1", "2"])
def test_single_interface_tubes_converge(tid):
    """Table 2 tubes on [0, 1], interface at x0, outflow ends."""
    gold = json.load(open(os.path.join(GOLD, "shock_tubes.json")))
    test, g = gold["tests"][tid], gold["gamma"]
    errs = []
    for Nx in (100, 200, 400):
        h = 1.0 / Nx
        x = (np.arange(Nx) + 0.5) * h
        left = {"rho": test["rhoL"], "v": test["vL"], "p": test["pL"]}
        right = {"rho": test["rhoR"], "v": test["vR"], "p": test["pR"]}
        st = tube_state(x, left, right, x < test["x0"], g)
        st, _ = run_to(O, st, O.Params(h=h, gamma=g, G=0.0, boundary="outflow"), test["t"])
        ex_r, ex_u, ex_p = sample((x - test["x0"]) / test["t"], test["rhoL"], test["vL"], test["pL"],
                                  test["rhoR"], test["vR"], test["pR"], g)
        rho = st["rho"][0, 0]
        errs.append((np.mean(np.abs(rho - ex_r)) / np.mean(ex_r), np.mean(np.abs(st["mx"][0, 0] / rho - ex_u)),
                     np.mean(np.abs((g - 1) * st["e"][0, 0] - ex_p)) / np.mean(ex_p)))
    errs = np.array(errs)
    assert np.all(errs[1] < errs[0] * 0.85) and np.all(errs[2] < errs[1] * 0.85), errs
    assert errs[2, 0] < {"1": 0.03, "2": 0.08}[tid], errs


def test_acoustic_pulse_leaves_the_box():
    """A right-moving linear acoustic pulse (Riemann invariant J- = 0) exits through
    the outflow boundary; on the periodic grid it is still there."""
    g, rho0, p0 = 1.4, 1.0, 1.0
    c0 = math.sqrt(g * p0 / rho0)
    Nx = 200
    h = 1.0 / Nx
    x = (np.arange(Nx) + 0.5) * h
    eps = 1e-3
    w = eps * np.exp(-((x - 0.5) / 0.05) ** 2)
    rho = (rho0 * (1 + w)).reshape(1, 1, Nx)
    v = (c0 * w).reshape(1, 1, Nx)
    p = (p0 * (1 + g * w)).reshape(1, 1, Nx)
    z = np.zeros_like(rho)
    one = np.ones_like(rho)
    P = {k: (one if k[0] == k[1] else 0 * one) for k in TENSOR}
    st = state_from_primitives(rho, (v, z, z), p, one, (z, z, z), P, g)
    t_end = 0.8 / c0   # the pulse centre travels 0.8: from 0.5 to 1.3
    res = {}
    for bc in ("outflow", "periodic"):
        out, _ = run_to(O, st, O.Params(h=h, gamma=g, G=0.0, boundary=bc), t_end)
        res[bc] = np.max(np.abs(out["rho"][0, 0] - rho0)) / (rho0 * eps)
    assert res["periodic"] > 0.3, res
    assert res["outflow"] < 0.03, res


def test_mirror_and_permutation_commute():
    s = I.random_state((12, 12, 12), seed=12, rough=True)
    prm = O.Params(h=s.h, poisson="isolated", boundary="outflow")
    a, _ = O.run(s.state, prm, 2)
    b, _ = O.run(reflect_x(s.state), prm, 2)
    c, _ = O.run(permute_state(s.state), prm, 2)
    for f in O.FIELDS:
        scale = max(1e-300, np.max(np.abs(a[f])))
        assert np.max(np.abs(reflect_x(a)[f] - b[f])) <= 1e-13 * scale, f
        assert np.max(np.abs(permute_state(a)[f] - c[f])) <= 1e-13 * scale, f


def test_windows_at_the_boundary():
    s = I.random_state((12, 12, 12), seed=13)
    prm = O.Params(h=s.h, poisson="isolated", boundary="outflow")
    phi = O.solve_poisson(s.state, prm)
    new, _ = O.advance(s.state, phi, 1e-3, prm)
    for k0, k1 in ((0, 3), (5, 7), (9, 12)):
        w, _ = O.advance_window(s.state, phi, 1e-3, prm, zslab=(k0, k1))
        for f in O.FIELDS:
            assert np.array_equal(w[f], new[f][k0:k1]), f
    cells = np.array([[0, 0, 0], [11, 5, 11], [3, 4, 5], [11, 11, 0], [1, 10, 1]])
    c, _ = O.advance_window(s.state, phi, 1e-3, prm, cells=cells)
    for f in O.FIELDS:
        assert np.array_equal(c[f], new[f][cells[:, 0], cells[:, 1], cells[:, 2]]), f
