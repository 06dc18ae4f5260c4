"""Pins of the oracle's reading B of the Lagrangian flux (Sec. 2.1, printed as a
4-term sum over the transverse diagonal neighbours of the face).

Reading B replaces the face velocity W_{i+1/2,k,l} of reading A by the mean of
W_{i+1/2,k+-1,l+-1} and upwinds by its sign.  What pins it:
  * a uniform state (moving or not) is a fixed point;
  * on a one-dimensional profile the transverse mean is the face velocity itself,
    so reading B reproduces reading A;
  * mass and total momentum are conserved exactly (flux form, periodic grid);
  * axis permutation and mirror reflection commute with the step;
  * a Sod tube at 45 degrees in the x-y plane, the one experiment that separates
    the readings: reading A converges to the exact solution along the normal,
    reading B collapses the density along the front within 30 CFL steps;
  * windowed evaluation (used by the full-size GPU tests) equals the whole grid.
"""
import json
import math
import os

import numpy as np

import oracle as O
from exact_riemann import sample
from helpers import TENSOR, permute_state, reflect_x, run_to, state_from_primitives, tube_state
from paper_1311_0861_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_diagonal_mean_by_loops():
    """The reading-B velocity of every face, summed by explicit loops."""
    rng = np.random.default_rng(5)
    nz, ny, nx = 5, 6, 7
    W = {d: rng.standard_normal((nz, ny, nx)) for d in "xyz"}
    got = O.flic_oracle._diagonal_mean(W)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                ex = {"x": 0.0, "y": 0.0, "z": 0.0}
                for a in (-1, 1):
                    for b in (-1, 1):
                        ex["x"] += W["x"][(k + b) % nz, (j + a) % ny, i]    # tangents y, z
                        ex["y"] += W["y"][(k + b) % nz, j, (i + a) % nx]    # tangents x, z
                        ex["z"] += W["z"][k, (j + b) % ny, (i + a) % nx]    # tangents x, y
                for d in "xyz":
                    assert abs(got[d][k, j, i] - 0.25 * ex[d]) <= 1e-14, (d, k, j, i)


def test_uniform_state_is_fixed_point():
    N = 8
    one = np.ones((N, N, N))
    P = {"xx": 0.5 * one, "yy": 0.7 * one, "zz": 0.6 * one, "xy": 0.1 * one, "xz": -0.05 * one, "yz": 0.02 * one}
    st = state_from_primitives(1.3 * one, (0.4 * one, -0.2 * one, 0.1 * one), 0.8 * one, 0.9 * one,
                               (-0.15 * one, 0.3 * one, 0.1 * one), P, 5.0 / 3.0)
    out, _ = O.run(st, O.Params(h=0.25, G=0.0, flux="B"), 3)
    for f in O.FIELDS:
        assert np.max(np.abs(out[f] - st[f])) <= 1e-14 * max(1.0, np.max(np.abs(st[f]))), f


def test_one_dimensional_profile_equals_reading_a():
    gold = json.load(open(os.path.join(GOLD, "shock_tubes.json")))
    test, g = gold["tests"]["1"], gold["gamma"]
    Nx = 64
    h = 4.0 / Nx
    x = (np.arange(Nx) + 0.5) * h
    in_left = (x < test["x0"]) | (x >= test["x0"] + 2.0)
    st1 = tube_state(x, {"rho": test["rhoL"], "v": test["vL"], "p": test["pL"]},
                     {"rho": test["rhoR"], "v": test["vR"], "p": test["pR"]}, in_left, g)
    st = {f: np.ascontiguousarray(np.broadcast_to(st1[f], (4, 4, Nx))) for f in O.FIELDS}
    a, _ = O.run(st, O.Params(h=h, gamma=g, G=0.0, flux="A"), 20)
    b, _ = O.run(st, O.Params(h=h, gamma=g, G=0.0, flux="B"), 20)
    for f in O.FIELDS:
        assert np.max(np.abs(a[f] - b[f])) <= 1e-13 * max(1.0, np.max(np.abs(a[f]))), f


def test_conservation_and_symmetry():
    s = I.random_state((12, 12, 12), seed=21, rough=True)
    prm = O.Params(h=s.h, flux="B")
    a, recs = O.run(s.state, prm, 2)
    vol = s.h ** 3
    for fld in ("rho", "n"):
        assert abs(np.sum(a[fld]) - np.sum(s.state[fld])) <= 1e-13 * np.sum(s.state[fld]), fld
    for ax in "xyz":
        m0 = np.sum(s.state["m" + ax] + s.state["q" + ax])
        m1 = np.sum(a["m" + ax] + a["q" + ax])
        assert abs(m1 - m0) <= 1e-12 * np.sum(s.state["rho"] + s.state["n"]), ax
    b, _ = O.run(reflect_x(s.state), prm, 2)
    c, _ = O.run(permute_state(s.state), prm, 2)
    for f in O.FIELDS:
        scale = max(1e-300, np.max(np.abs(a[f])))
        assert np.max(np.abs(reflect_x(a)[f] - b[f])) <= 1e-13 * scale, f
        assert np.max(np.abs(permute_state(a)[f] - c[f])) <= 1e-13 * scale, f
    assert vol > 0


def _oblique_sod_state(N):
    """Sod tube with its interface along x + y = L/2 on the periodic square of side
    L = 2 sqrt 2 (normal coordinate xi = (x + y)/sqrt 2, interfaces at xi = 1 and 2 = 0)."""
    gold = json.load(open(os.path.join(GOLD, "shock_tubes.json")))
    test, g = gold["tests"]["1"], gold["gamma"]
    L = 2.0 * math.sqrt(2.0)
    h = L / N
    c = (np.arange(N) + 0.5) * h
    yy, xx = np.meshgrid(c, c, indexing="ij")
    xi = ((xx + yy) % L) / math.sqrt(2.0)
    left = (xi < 1.0).reshape(1, N, N)
    z = np.zeros((1, N, N))
    one = np.ones((1, N, N))
    rho = np.where(left, test["rhoL"], test["rhoR"])
    p = np.where(left, test["pL"], test["pR"])
    P = {k: (one if k[0] == k[1] else z) for k in TENSOR}
    return state_from_primitives(rho, (z, z, z), p, one, (z, z, z), P, g), xi, h, test, g


def test_oblique_sod_reading_a_converges():
    errs = []
    for N in (48, 96):
        st, xi, h, test, g = _oblique_sod_state(N)
        st, _ = run_to(O, st, O.Params(h=h, gamma=g, G=0.0, flux="A"), test["t"])
        win = (xi > 0.55) & (xi < 1.45)
        ex_r, _, _ = sample((xi[win] - 1.0) / test["t"], test["rhoL"], test["vL"], test["pL"],
                            test["rhoR"], test["vR"], test["pR"], g)
        errs.append(np.mean(np.abs(st["rho"][0][win] - ex_r)) / np.mean(ex_r))
    assert errs[1] < 0.85 * errs[0] and errs[1] < 0.05, errs


def test_oblique_sod_reading_b_collapses():
    """The experiment that separates the readings: off the grid axes the transverse
    diagonal mean moves mass with velocities of the cells across the front, and
    the density along the front collapses within 30 CFL steps (reading A keeps it
    near the exact plateau values; both are identical on one-dimensional profiles)."""
    st0, xi, h, test, g = _oblique_sod_state(48)
    rmin = {}
    for flux in ("A", "B"):
        st, _ = O.run(st0, O.Params(h=h, gamma=g, G=0.0, flux=flux), 30)
        rmin[flux] = float(np.min(st["rho"]))
    assert rmin["A"] > 0.1, rmin              # the exact solution stays above 0.125
    assert rmin["B"] < 0.01, rmin


def test_windows():
    s = I.random_state((12, 12, 12), seed=22, rough=True)
    prm = O.Params(h=s.h, flux="B")
    phi = O.solve_poisson(s.state, prm)
    new, _ = O.advance(s.state, phi, 1e-3, prm)
    w, _ = O.advance_window(s.state, phi, 1e-3, prm, zslab=(3, 6))
    cells = np.array([[0, 0, 0], [11, 5, 11], [3, 4, 5]])
    c, _ = O.advance_window(s.state, phi, 1e-3, prm, cells=cells)
    for f in O.FIELDS:
        assert np.array_equal(w[f], new[f][3:6]), f
        assert np.array_equal(c[f], new[f][cells[:, 0], cells[:, 1], cells[:, 2]]), f
