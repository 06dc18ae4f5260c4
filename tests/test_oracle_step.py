"""Pins of the oracle's full step to invariants the method must satisfy.

* a uniform state in uniform motion is a fixed point (Sec. 2 equations);
* mass of both fluids is conserved to rounding (flux form, Sec. 2.1 Lagrangian stage);
* total momentum of both fluids is conserved to rounding: pressure and stress
  fluxes telescope and sum_c s (D Phi) = s^T D K s = 0 for the antisymmetric
  central difference D and the symmetric, translation-invariant Green operator K;
* the step commutes with axis permutations and mirror reflections of the grid
  (vector and tensor components transformed alike) -- this catches a swapped
  index, tangent or sign in any of the three face directions;
* the energy balance and kappa (Sec. 2.4) act exactly as the stated reading on
  hand-built states (tau = 0 isolates them);
* the CFL step and the diagnostics agree with closed forms on simple states;
* the windowed evaluation used for sampled large-grid parity equals the full step.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1311_0861_gb300 import inputs as I

from helpers import permute_state, reflect_x, state_from_primitives, TENSOR

FIELDS = O.FIELDS


def _uniform(shape, gamma=5.0 / 3.0):
    one = np.ones(shape)
    P = {"xx": 0.5 * one, "yy": 0.7 * one, "zz": 0.6 * one,
         "xy": 0.1 * one, "xz": -0.05 * one, "yz": 0.02 * one}
    return state_from_primitives(1.3 * one, (0.2 * one, -0.1 * one, 0.05 * one), 0.8 * one,
                                 0.9 * one, (-0.15 * one, 0.3 * one, 0.1 * one), P, gamma)


def test_uniform_state_is_fixed_point():
    st = _uniform((6, 6, 6))
    prm = O.Params(h=2.0 / 6)
    new, recs = O.run(st, prm, 3)
    for f in FIELDS:
        assert np.max(np.abs(new[f] - st[f])) <= 1e-14 * max(1.0, np.max(np.abs(st[f]))), f
    assert all(r["kappa_gas"] < 1e-14 and r["kappa_bme"] < 1e-14 for r in recs)


@pytest.mark.parametrize("rough", [False, True])
def test_mass_and_momentum_conserved(rough):
    s = I.random_state((8, 8, 8), seed=3, rough=rough)
    prm = O.Params(h=s.h, G=1.0)
    st = s.state
    d0 = O.diagnostics(st, O.solve_poisson(st, prm), prm)
    pscale = sum(np.sum(np.abs(st[f])) for f in ("mx", "my", "mz", "qx", "qy", "qz")) * s.h ** 3
    for _ in range(4):
        st, rec = O.step(st, prm)
    d1 = O.diagnostics(st, O.solve_poisson(st, prm), prm)
    assert abs(d1["mass_gas"] - d0["mass_gas"]) <= 1e-14 * d0["mass_gas"]
    assert abs(d1["mass_bme"] - d0["mass_bme"]) <= 1e-14 * d0["mass_bme"]
    for a in "xyz":
        assert abs(d1["mom_" + a] - d0["mom_" + a]) <= 1e-13 * pscale, a


def test_momentum_not_conserved_per_fluid_with_gravity():
    """Sanity of the previous pin: gravity does exchange momentum between the fluids."""
    s = I.random_state((8, 8, 8), seed=4)
    prm = O.Params(h=s.h, G=1.0)
    st, _ = O.step(s.state, prm)
    mg0 = np.sum(s.state["mx"])
    mg1 = np.sum(st["mx"])
    assert abs(mg1 - mg0) > 1e-8


def _close(a, b, tol=1e-13):
    for f in FIELDS:
        sc = max(1.0, np.max(np.abs(b[f])))
        assert np.max(np.abs(a[f] - b[f])) <= tol * sc, f


@pytest.mark.parametrize("rough", [False, True])
def test_step_commutes_with_axis_permutation(rough):
    s = I.random_state((6, 6, 6), seed=5, rough=rough)
    prm = O.Params(h=s.h, G=0.5)
    a, ra = O.run(s.state, prm, 2)
    b, rb = O.run(permute_state(s.state), prm, 2)
    _close(permute_state(a), b)
    assert abs(ra[-1]["dt"] - rb[-1]["dt"]) < 1e-15


@pytest.mark.parametrize("rough", [False, True])
def test_step_commutes_with_mirror(rough):
    s = I.random_state((6, 6, 6), seed=6, rough=rough)
    prm = O.Params(h=s.h, G=0.5)
    a, _ = O.run(s.state, prm, 2)
    b, _ = O.run(reflect_x(s.state), prm, 2)
    _close(reflect_x(a), b)
    # mirror along y and z through the permutation
    c, _ = O.run(permute_state(reflect_x(permute_state(permute_state(s.state)))), prm, 2)
    _close(permute_state(reflect_x(permute_state(permute_state(a)))), c)


def test_energy_balance_reading():
    """tau = 0: transport is the identity; only the balance of Sec. 2.4 acts."""
    shape = (1, 1, 4)
    st = _uniform(shape)
    prm = O.Params(h=0.5, eta=1e-3)
    K = (st["mx"] ** 2 + st["my"] ** 2 + st["mz"] ** 2) / (2 * st["rho"])
    st["E"] = st["E"].copy()
    st["E"][..., 0] += 0.01                    # eps_E = e + 0.01 >= eta E: e <- eps_E
    st["E"][..., 1] = K[..., 1] / (1.0 - 0.5e-3)   # eps_E = eta E / 2 < eta E: E <- e + K
    new, kap = O.advance(st, np.zeros(shape), 0.0, prm)
    assert abs(new["e"][0, 0, 0] - (st["E"][0, 0, 0] - K[0, 0, 0])) < 1e-15
    assert new["E"][0, 0, 0] == st["E"][0, 0, 0]
    assert abs(new["E"][0, 0, 1] - (st["e"][0, 0, 1] + K[0, 0, 1])) < 1e-15
    assert new["e"][0, 0, 1] == st["e"][0, 0, 1]
    assert abs(kap["kappa_gas"][0, 0, 0] - 0.01 * prm.h ** 3) < 1e-15
    # moment fluid: perturb nE_xy -> taken into Pi; make a diagonal entry negative -> reset nE
    st2 = _uniform(shape)
    st2["nExy"] = st2["nExy"].copy()
    st2["nExy"][..., 2] += 0.02
    st2["nEyy"] = st2["nEyy"].copy()
    qq = st2["qy"] ** 2 / st2["n"]
    st2["nEyy"][..., 3] = qq[..., 3] - 0.01
    new2, kap2 = O.advance(st2, np.zeros(shape), 0.0, prm)
    assert abs(new2["Pxy"][0, 0, 2] - (st2["Pxy"][0, 0, 2] + 0.02)) < 1e-15
    assert abs(kap2["kappa_bme"][0, 0, 2] - 0.02 * prm.h ** 3) < 1e-15
    assert new2["Pyy"][0, 0, 3] == st2["Pyy"][0, 0, 3]
    assert abs(new2["nEyy"][0, 0, 3] - (st2["Pyy"][0, 0, 3] + qq[0, 0, 3])) < 1e-15
    # after the balance, kappa of the new state vanishes
    _, kap3 = O.advance(new2, np.zeros(shape), 0.0, prm)
    assert np.max(kap3["kappa_bme"]) < 1e-15


def test_cfl_closed_form():
    st = _uniform((2, 2, 2))
    prm = O.Params(h=0.25, courant=0.2)
    g = prm.gamma
    cs = math.sqrt(g * 0.8 / 1.3)
    gas = max(abs(v) for v in (0.2, -0.1, 0.05)) + cs
    bme = max(abs(-0.15) + math.sqrt(3 * 0.5 / 0.9), abs(0.3) + math.sqrt(3 * 0.7 / 0.9),
              abs(0.1) + math.sqrt(3 * 0.6 / 0.9))
    assert abs(O.max_signal_speed(st, prm) - max(gas, bme)) < 1e-14
    assert abs(O.cfl_dt(st, prm) - 0.2 * 0.25 / max(gas, bme)) < 1e-15


def test_diagnostics_closed_form():
    N = 4
    st = _uniform((N, N, N))
    prm = O.Params(h=2.0 / N)
    d = O.diagnostics(st, np.zeros((N, N, N)), prm)
    V = 8.0
    assert abs(d["mass_gas"] - 1.3 * V) < 1e-13
    assert abs(d["mass_bme"] - 0.9 * V) < 1e-13
    assert abs(d["mom_y"] - (1.3 * -0.1 + 0.9 * 0.3) * V) < 1e-13
    assert abs(d["ekin_gas"] - 0.5 * 1.3 * (0.04 + 0.01 + 0.0025) * V) < 1e-13
    assert abs(d["eint_gas"] - 0.8 / (prm.gamma - 1) * V) < 1e-13
    assert abs(d["etherm_bme"] - 0.5 * 1.8 * V) < 1e-13


def test_epot_matches_direct_pair_sum():
    """E_pot = 1/2 sum s Phi h^3 with the isolated Green's function is the pair energy."""
    N = 5
    s = I.uniform(21, N ** 3).reshape(N, N, N)
    st = {f: np.ones((N, N, N)) for f in FIELDS}
    st["rho"], st["n"] = s, np.zeros((N, N, N))
    prm = O.Params(h=0.3, poisson="isolated")
    phi = O.solve_poisson(st, prm)
    d = O.diagnostics(st, phi, prm)
    idx = np.stack(np.meshgrid(*[np.arange(N)] * 3, indexing="ij"), -1).reshape(-1, 3)
    r = np.sqrt(((idx[:, None] - idx[None]) ** 2).sum(-1)) * prm.h
    with np.errstate(divide="ignore"):
        g = np.where(r > 0, -prm.h ** 3 / r, -prm.h ** 2 * O.CUBE_SELF_POTENTIAL)
    m = s.ravel()
    assert abs(d["epot"] - 0.5 * m @ g @ m * prm.h ** 3) < 1e-12 * abs(d["epot"])


def test_window_evaluation_equals_full_step():
    s = I.random_state((8, 8, 8), seed=8, rough=True)
    prm = O.Params(h=s.h)
    phi = O.solve_poisson(s.state, prm)
    tau = O.cfl_dt(s.state, prm)
    full, kap = O.advance(s.state, phi, tau, prm)
    slab, _ = O.advance_window(s.state, phi, tau, prm, zslab=(6, 10))
    for f in FIELDS:
        ref = np.concatenate([full[f][6:8], full[f][0:2]])
        assert np.array_equal(slab[f], ref), f
    cells = np.array([[0, 0, 0], [7, 3, 5], [4, 7, 7], [2, 2, 1]])
    pts, _ = O.advance_window(s.state, phi, tau, prm, cells=cells)
    for f in FIELDS:
        assert np.array_equal(pts[f], full[f][cells[:, 0], cells[:, 1], cells[:, 2]]), f
