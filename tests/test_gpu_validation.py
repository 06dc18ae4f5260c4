"""The paper's test problems (Sec. 4) on the CUDA path, through the C ABI.

A one-dimensional problem runs on an N^3 grid with its profile copied along y and
z (gravity off, periodic), so every row of the grid evolves like the oracle's 1D
run of the same problem at the same resolution:
  * parity: each row equals the oracle's run (FP64 <= 1e-10 relative L1 per field;
    mixed <= 1e-4 in the densities), and all rows are equal;
  * validation: the L1 error against the exact solution (the same exact solutions
    that pin the oracle in test_oracle_validation.py) falls from N = 64 to N = 128.
Problems: Godunov shock tubes 1-3 (Table 2), the moment-fluid shock tube (Sec. 4.2,
its exact gamma = 3 subsystem), Aksenov's simple wave (Sec. 4.3), and the
hydrostatic cloud of Sec. 4.5 with isolated gravity (3D, parity only); with
outflow boundaries, the single-interface Sod tube on [0, 1] and an acoustic
pulse that leaves the box.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from exact_riemann import sample
from helpers import TENSOR, run_to, state_from_primitives, tube_state

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
FIELDS = O.FIELDS


@pytest.fixture(scope="module")
def flic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_0861_gb300 import flic as F
    if not os.path.exists(F.LIB_PATH):
        from paper_1311_0861_gb300 import build
        build.build()
    F.load()
    return F


def rel_l1(a, b):
    den = np.sum(np.abs(b))
    return float(np.sum(np.abs(a - b)) / den) if den > 0 else float(np.sum(np.abs(a - b)))


def gpu_run_to(F, st, N, box, gamma, t_end, precision="fp64", G=0.0, poisson="periodic", courant=0.2,
               boundary="periodic"):
    """Steps the grid to t_end with CFL steps and a final partial step, as the
    oracle's run_to does; returns the final state and the number of steps."""
    h = (box[1] - box[0]) / N
    with F.Grid(N, gamma=gamma, G=G, precision=precision, box=box, poisson=poisson, boundary=boundary) as g:
        g.set_state(st)
        vmax = g.diagnostics()["vmax"]
        t, k = 0.0, 0
        while t < t_end * (1 - 1e-14):
            dt_cfl = courant * h / vmax
            if dt_cfl >= t_end - t:
                g.step(t_end - t)
            else:
                g.step()
            d = g.step_diagnostics()
            t += d["dt"]
            vmax = d["vmax"]
            k += 1
        return g.get_state(), k


def to_cube(st1, N):
    """(1, 1, N) profile -> N^3 copies along y and z."""
    return {f: np.ascontiguousarray(np.broadcast_to(st1[f], (N, N, N))) for f in FIELDS}


def check_rows(st3, st1, tol, floor=0.0):
    """Every row of the cube equals row (0, 0); row (0, 0) equals the oracle's 1D run
    (relative L1, the denominator at least ``floor`` per cell for fields that
    end near zero)."""
    for f in FIELDS:
        a = st3[f]
        scale = max(1e-300, np.max(np.abs(a)))
        assert np.max(np.abs(a - a[0:1, 0:1, :])) <= 1e-13 * scale, f
    errs = {f: float(np.sum(np.abs(st3[f][0, 0] - st1[f][0, 0])) /
                     max(np.sum(np.abs(st1[f][0, 0])), floor * st1[f][0, 0].size, 1e-300)) for f in FIELDS}
    bad = {f: e for f, e in errs.items() if e > tol and np.max(np.abs(st1[f])) > 1e-12}
    assert not bad, bad


def tube1d(test, N, g):
    """Table 2 tube on the periodic [0, 4): left state on [0, x0) and [x0 + 2, 4)."""
    h = 4.0 / N
    x = (np.arange(N) + 0.5) * h
    in_left = (x < test["x0"]) | (x >= test["x0"] + 2.0)
    left = {"rho": test["rhoL"], "v": test["vL"], "p": test["pL"]}
    right = {"rho": test["rhoR"], "v": test["vR"], "p": test["pR"]}
    return x, h, tube_state(x, left, right, in_left, g)


@pytest.mark.parametrize("tid", ["1", "2", "3"])
def test_godunov_tubes(flic, tid):
    gold = json.load(open(os.path.join(GOLD, "shock_tubes.json")))
    test, g = gold["tests"][tid], gold["gamma"]
    errs = []
    for N in (64, 128):
        x, h, st1 = tube1d(test, N, g)
        ref, k1 = run_to(O, st1, O.Params(h=h, gamma=g, G=0.0, courant=0.2), test["t"])
        out, k3 = gpu_run_to(flic, to_cube(st1, N), N, (0.0, 4.0), g, test["t"])
        assert k1 == k3
        check_rows(out, ref, 1e-10)
        win = (x > 0.05) & (x < 0.95)
        ex_r, ex_u, ex_p = sample((x[win] - test["x0"]) / test["t"], test["rhoL"], test["vL"], test["pL"],
                                  test["rhoR"], test["vR"], test["pR"], g)
        rho = out["rho"][0, 0, win]
        errs.append((np.mean(np.abs(rho - ex_r)) / np.mean(ex_r),
                     np.mean(np.abs(out["mx"][0, 0, win] / rho - ex_u)),
                     np.mean(np.abs((g - 1) * out["e"][0, 0, win] - ex_p)) / np.mean(ex_p)))
    errs = np.array(errs)
    assert np.all(errs[1] < errs[0]), errs


def test_godunov_tube1_mixed(flic):
    gold = json.load(open(os.path.join(GOLD, "shock_tubes.json")))
    test, g = gold["tests"]["1"], gold["gamma"]
    N = 128
    x, h, st1 = tube1d(test, N, g)
    ref, _ = run_to(O, st1, O.Params(h=h, gamma=g, G=0.0, courant=0.2), test["t"])
    out, _ = gpu_run_to(flic, to_cube(st1, N), N, (0.0, 4.0), g, test["t"], precision="mixed")
    for f in ("rho", "E", "e"):
        assert rel_l1(out[f][0, 0], ref[f][0, 0]) <= 1e-4, f


def test_moment_shock_tube(flic):
    gb = json.load(open(os.path.join(GOLD, "bme_shock_tube.json")))
    L, R = gb["left"], gb["right"]
    errs = []
    for N in (64, 128):
        h = 4.0 / N
        x = (np.arange(N) + 0.5) * h
        in_left = (x < gb["x0"]) | (x >= gb["x0"] + 2.0)
        gas = {"rho": 1.0, "v": 0.0, "p": 1.0}
        bl, br = dict(L), dict(R)
        for b in (bl, br):
            for k in TENSOR:
                b.setdefault("P" + k, b.get("P" + k))
        st1 = tube_state(x, gas, gas, in_left, 5.0 / 3.0, bme=(bl, br))
        ref, _ = run_to(O, st1, O.Params(h=h, G=0.0, courant=0.2), gb["t"])
        out, _ = gpu_run_to(flic, to_cube(st1, N), N, (0.0, 4.0), 5.0 / 3.0, gb["t"])
        check_rows(out, ref, 1e-10)
        win = (x > 0.05) & (x < 0.95)
        ex_n, ex_u, ex_P = sample((x[win] - gb["x0"]) / gb["t"], L["rho"], L["ux"], L["Pxx"], R["rho"], R["ux"],
                                  R["Pxx"], 3.0)
        n = out["n"][0, 0, win]
        errs.append((np.mean(np.abs(n - ex_n)) / np.mean(ex_n), np.mean(np.abs(out["qx"][0, 0, win] / n - ex_u)),
                     np.mean(np.abs(out["Pxx"][0, 0, win] - ex_P)) / np.mean(ex_P)))
    errs = np.array(errs)
    assert np.all(errs[1] < errs[0]), errs


def aksenov_exact(x, tt):
    """Riemann invariants u~ +- rho constant along dx/dtt = u~ +- rho (velocity unit
    sqrt(3), time unit 1/sqrt(3)), solved by fixed-point iteration."""
    Rp = 1.5 * np.ones_like(x)
    Rm = -1.5 * np.ones_like(x)
    for _ in range(500):
        Rp = 1.0 + 0.5 * np.cos(x - Rp * tt)
        Rm = -1.0 - 0.5 * np.cos(x - Rm * tt)
    return 0.5 * (Rp - Rm), 0.5 * (Rp + Rm) * math.sqrt(3.0)


def test_aksenov_simple_wave(flic):
    g, tt = 3.0, 1.0
    t_end = tt / math.sqrt(3.0)
    errs = []
    for N in (64, 128):
        h = 2 * np.pi / N
        x = (np.arange(N) + 0.5) * h
        rho = (1.0 + 0.5 * np.cos(x)).reshape(1, 1, N)
        z = np.zeros_like(rho)
        one = np.ones_like(rho)
        P = {k: (one if k[0] == k[1] else 0 * one) for k in TENSOR}
        st1 = state_from_primitives(rho, (z, z, z), rho ** 3, one, (z, z, z), P, g)
        ref, _ = run_to(O, st1, O.Params(h=h, gamma=g, G=0.0, courant=0.2), t_end)
        out, _ = gpu_run_to(flic, to_cube(st1, N), N, (0.0, 2 * np.pi), g, t_end)
        check_rows(out, ref, 1e-10)
        ex_r, ex_u = aksenov_exact(x, tt)
        r = out["rho"][0, 0]
        errs.append((np.mean(np.abs(r - ex_r)), np.mean(np.abs(out["mx"][0, 0] / r - ex_u))))
    errs = np.array(errs)
    assert np.all(errs[0] / errs[1] > 1.6), errs


def test_hydrostatic_cloud_isolated(flic):
    """rho0 = 1 - r and the printed p0 of Sec. 4.5, isolated gravity, 32^3: the GPU
    run equals the oracle's (both keep the cloud near rest)."""
    gold = json.load(open(os.path.join(GOLD, "cloud_test.json")))
    cp = gold["p0_poly_in_units_of_pi"]["c"]
    N, L = 32, 1.25
    h = 2 * L / N
    c = -L + (np.arange(N) + 0.5) * h
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(xx ** 2 + yy ** 2 + zz ** 2)
    rho = np.maximum(1.0 - r, 1e-3)
    p0 = sum(float(v) * r ** int(k) for k, v in cp.items()) * math.pi
    p = np.maximum(np.where(r <= 1.0, p0, 0.0), 1e-5)
    z = np.zeros_like(rho)
    one = np.ones_like(rho)
    P = {k: (1e-6 * one if k[0] == k[1] else z) for k in TENSOR}
    st = state_from_primitives(rho, (z, z, z), p, 1e-6 * one, (z, z, z), P, 5.0 / 3.0)
    ref, k1 = run_to(O, st, O.Params(h=h, G=1.0, poisson="isolated"), 0.05)
    out, k3 = gpu_run_to(flic, st, N, (-L, L), 5.0 / 3.0, 0.05, G=1.0, poisson="isolated")
    assert k1 == k3
    for f in FIELDS:
        if np.max(np.abs(ref[f])) > 1e-12:
            assert rel_l1(out[f], ref[f]) <= 1e-10, f
    inner = r < 0.7
    assert np.max(np.abs(out["mx"][inner] / out["rho"][inner])) < 0.05


def test_sod_single_interface_outflow(flic):
    gold = json.load(open(os.path.join(GOLD, "shock_tubes.json")))
    test, g = gold["tests"]["1"], gold["gamma"]
    errs = []
    for N in (64, 128):
        h = 1.0 / N
        x = (np.arange(N) + 0.5) * h
        left = {"rho": test["rhoL"], "v": test["vL"], "p": test["pL"]}
        right = {"rho": test["rhoR"], "v": test["vR"], "p": test["pR"]}
        st1 = tube_state(x, left, right, x < test["x0"], g)
        ref, k1 = run_to(O, st1, O.Params(h=h, gamma=g, G=0.0, courant=0.2, boundary="outflow"), test["t"])
        out, k3 = gpu_run_to(flic, to_cube(st1, N), N, (0.0, 1.0), g, test["t"], boundary="outflow")
        assert k1 == k3
        check_rows(out, ref, 1e-10)
        ex_r, _, _ = sample((x - test["x0"]) / test["t"], test["rhoL"], test["vL"], test["pL"],
                            test["rhoR"], test["vR"], test["pR"], g)
        errs.append(np.mean(np.abs(out["rho"][0, 0] - ex_r)) / np.mean(ex_r))
    assert errs[1] < errs[0] and errs[1] < 0.05, errs


def test_acoustic_pulse_leaves_outflow_box(flic):
    g, rho0, p0 = 1.4, 1.0, 1.0
    c0 = math.sqrt(g * p0 / rho0)
    N = 128
    h = 1.0 / N
    x = (np.arange(N) + 0.5) * h
    eps = 1e-3
    w = eps * np.exp(-((x - 0.5) / 0.05) ** 2)
    rho = (rho0 * (1 + w)).reshape(1, 1, N)
    z = np.zeros_like(rho)
    one = np.ones_like(rho)
    P = {k: (one if k[0] == k[1] else 0 * one) for k in TENSOR}
    st1 = state_from_primitives(rho, ((c0 * w).reshape(1, 1, N), z, z), (p0 * (1 + g * w)).reshape(1, 1, N), one,
                                (z, z, z), P, g)
    t_end = 0.8 / c0
    ref, _ = run_to(O, st1, O.Params(h=h, gamma=g, G=0.0, courant=0.2, boundary="outflow"), t_end)
    out, _ = gpu_run_to(flic, to_cube(st1, N), N, (0.0, 1.0), g, t_end, boundary="outflow")
    check_rows(out, ref, 1e-10, floor=rho0 * c0 * eps)   # the momentum has left with the pulse
    assert np.max(np.abs(out["rho"] - rho0)) < 0.03 * rho0 * eps


def test_cloud_collision_isolated_outflow(flic):
    """The cloud collision of Sec. 4.5 (two rho = 1 - r clouds, L0 = 2.4, v = 1) with
    isolated gravity and outflow boundaries: the GPU run equals the oracle's
    (FP64 1e-10, float32 1e-4 in the densities), and each step's mass change equals
    the closed-form flux through the boundary (test_oracle_cloud_collision.py)."""
    from paper_1311_0861_gb300 import inputs as I
    for N in (32, 48):
        s = I.cloud_collision(N)
        L = 0.5 * N * s.h
        prm = O.Params(h=s.h, gamma=s.gamma, poisson="isolated", boundary="outflow")
        ref, rrec = O.run(s.state, prm, 5)
        for precision in ("fp64", "mixed"):
            with flic.Grid(N, precision=precision, gamma=s.gamma, poisson="isolated", boundary="outflow",
                           box=(-L, L)) as g:
                g.set_state(s.state)
                m0 = g.diagnostics()["mass_gas"]
                dt0 = g.step()
                m1 = g.diagnostics()["mass_gas"]
                for _ in range(4):
                    g.step()
                out = g.get_state()
            if precision == "fp64":
                st = s.state
                flux = (np.sum(st["mx"][:, :, -1]) - np.sum(st["mx"][:, :, 0]) + np.sum(st["my"][:, -1, :])
                        - np.sum(st["my"][:, 0, :]) + np.sum(st["mz"][-1, :, :]) - np.sum(st["mz"][0, :, :]))
                assert abs((m1 - m0) + dt0 * s.h ** 2 * flux) <= 1e-12 * m0
                for f in FIELDS:
                    if np.max(np.abs(ref[f])) > 1e-9:
                        assert rel_l1(out[f], ref[f]) <= 1e-10, (N, f)
            else:
                assert rel_l1(out["rho"], ref["rho"]) <= 1e-4 and rel_l1(out["n"], ref["n"]) <= 1e-4


def rotate_axes(st, k):
    """The state with the grid and every vector/tensor component rotated k times
    by x -> y -> z -> x (a profile along x then lies along y for k = 1, z for k = 2)."""
    from helpers import permute_state
    for _ in range(k % 3):
        st = permute_state(st)
    return st


@pytest.mark.parametrize("axis", [1, 2])
def test_tubes_along_y_and_z(flic, axis):
    """Godunov tube 1 (Table 2) and the moment-fluid tube (Sec. 4.2) with their
    profiles along y or z: the z direction is the one the fused kernel marches
    (its faces live in registers and the plane ring), y the second tile axis.
    Rotated back, every row equals the oracle's 1D run (FP64 1e-10)."""
    gold = json.load(open(os.path.join(GOLD, "shock_tubes.json")))
    test, g = gold["tests"]["1"], gold["gamma"]
    N = 64
    x, h, st1 = tube1d(test, N, g)
    ref, k1 = run_to(O, st1, O.Params(h=h, gamma=g, G=0.0, courant=0.2), test["t"])
    cube = rotate_axes(to_cube(st1, N), axis)
    out, k3 = gpu_run_to(flic, cube, N, (0.0, 4.0), g, test["t"])
    assert k1 == k3
    check_rows(rotate_axes(out, 3 - axis), ref, 1e-10)

    gb = json.load(open(os.path.join(GOLD, "bme_shock_tube.json")))
    L, R = gb["left"], gb["right"]
    in_left = (x < gb["x0"]) | (x >= gb["x0"] + 2.0)
    gas = {"rho": 1.0, "v": 0.0, "p": 1.0}
    st1 = tube_state(x, gas, gas, in_left, 5.0 / 3.0, bme=(dict(L), dict(R)))
    ref, _ = run_to(O, st1, O.Params(h=h, G=0.0, courant=0.2), gb["t"])
    out, _ = gpu_run_to(flic, rotate_axes(to_cube(st1, N), axis), N, (0.0, 4.0), 5.0 / 3.0, gb["t"])
    check_rows(rotate_axes(out, 3 - axis), ref, 1e-10)
