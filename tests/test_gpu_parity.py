"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 path: every field of one step within 1e-11 of the oracle (max abs error over
the field's max abs), ten steps within 1e-10 relative L1 (sum |a-b| / sum |b|).
Mixed path (float32 bulk): ten steps within 1e-4 relative L1 in density and
1e-6 relative mass drift.  Sizes cover partial tiles (N not a multiple of the
32 x 8 tile), several tiles with ragged z chunks, radix-3 FFT lengths, and the
degenerate cases (uniform state, gravity off, fixed dt).
"""
import numpy as np
import pytest

import oracle as O
from paper_1311_0861_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FIELDS = O.FIELDS


@pytest.fixture(scope="module")
def flic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_0861_gb300 import flic as F
    import os
    if not os.path.exists(F.LIB_PATH):
        from paper_1311_0861_gb300 import build
        build.build()
    F.load()
    return F


def max_rel(a, b):
    return {f: float(np.max(np.abs(a[f] - b[f])) / max(1e-300, np.max(np.abs(b[f])))) for f in FIELDS}


def rel_l1(a, b):
    return {f: float(np.sum(np.abs(a[f] - b[f])) / max(1e-300, np.sum(np.abs(b[f])))) for f in FIELDS}


def run_gpu(F, setup, nsteps, precision="fp64", dt=0.0, G=1.0, graph=False):
    with F.Grid(setup.shape[0], gamma=setup.gamma, G=G, precision=precision,
                box=(-1.0, -1.0 + setup.h * setup.shape[0])) as g:
        g.set_state(setup.state)
        recs = []
        if graph:
            g.run(nsteps, dt)
            recs.append(g.step_diagnostics())
        else:
            for _ in range(nsteps):
                g.step(dt)
                recs.append(g.step_diagnostics())
        return g.get_state(), recs


def run_oracle(setup, nsteps, dt=None, G=1.0):
    prm = O.Params(h=setup.h, gamma=setup.gamma, G=G)
    return O.run(setup.state, prm, nsteps, dt)


@pytest.mark.parametrize("N", [8, 12, 24, 32, 48, 64])
def test_poisson_fp64(flic, N):
    s = I.random_state((N, N, N), seed=30 + N)
    prm = O.Params(h=s.h)
    ref = O.solve_poisson(s.state, prm)
    with flic.Grid(N, precision="fp64", box=(-1.0, -1.0 + s.h * N)) as g:
        g.set_state(s.state)
        phi = g.solve_poisson()
    assert np.max(np.abs(phi - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("N", [16, 48, 96])
def test_poisson_mixed(flic, N):
    s = I.random_state((N, N, N), seed=40 + N)
    prm = O.Params(h=s.h)
    ref = O.solve_poisson(s.state, prm)
    with flic.Grid(N, precision="mixed", box=(-1.0, -1.0 + s.h * N)) as g:
        g.set_state(s.state)
        phi = g.solve_poisson()
    assert np.max(np.abs(phi - ref)) <= 2e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("N,rough", [(8, True), (12, False), (24, True), (32, False), (48, True), (64, False)])
def test_one_step_fp64(flic, N, rough):
    s = I.random_state((N, N, N), seed=N, rough=rough)
    ref, rrec = run_oracle(s, 1)
    out, grec = run_gpu(flic, s, 1)
    err = max_rel(out, ref)
    assert max(err.values()) <= 1e-11, err
    g, r = grec[-1], rrec[-1]
    assert abs(g["dt"] - r["dt"]) <= 1e-14 * r["dt"]
    for k in ("mass_gas", "mass_bme", "ekin_gas", "eint_gas", "ekin_bme", "etherm_bme", "epot",
              "kappa_gas", "kappa_bme", "vmax"):
        assert abs(g[k] - r[k]) <= 1e-11 * max(abs(r[k]), 1e-300), (k, g[k], r[k])
    for a in "xyz":
        scale = r["ekin_gas"] ** 0.5 + r["mass_gas"]
        assert abs(g["mom_" + a] - r["mom_" + a]) <= 1e-12 * scale


def test_sphere_ten_steps_fp64(flic):
    """32^3 self-gravitating sphere, 10 CFL steps: relative L1 <= 1e-10 per field."""
    s = I.sphere(32)
    ref, rrec = run_oracle(s, 10)
    out, grec = run_gpu(flic, s, 10)
    err = rel_l1(out, ref)
    assert max(err.values()) <= 1e-10, err
    assert abs(grec[-1]["dt"] - rrec[-1]["dt"]) <= 1e-12 * rrec[-1]["dt"]


def test_collision_ten_steps_fp64_graph(flic):
    """32^3 two-galaxy collision through CUDA-graph replay."""
    s = I.head_on(32)
    ref, rrec = run_oracle(s, 10)
    out, grec = run_gpu(flic, s, 10, graph=True)
    err = rel_l1(out, ref)
    assert max(err.values()) <= 1e-10, err
    assert grec[-1]["step"] == 10


def test_graph_replay_equals_single_steps(flic):
    s = I.random_state((24, 24, 24), seed=5)
    a, _ = run_gpu(flic, s, 4)
    b, _ = run_gpu(flic, s, 4, graph=True)
    for f in FIELDS:
        assert np.array_equal(a[f], b[f]), f


def test_mixed_ten_steps(flic):
    """float32 bulk: 1e-4 relative L1 in density, 1e-6 relative mass drift."""
    s = I.head_on(32)
    ref, rrec = run_oracle(s, 10)
    out, grec = run_gpu(flic, s, 10, precision="mixed")
    err = rel_l1(out, ref)
    assert err["rho"] <= 1e-4 and err["n"] <= 1e-4, err
    with flic.Grid(32, precision="mixed") as g:
        g.set_state(s.state)
        m0 = g.diagnostics()
        g.run(10)
        m1 = g.diagnostics()
    assert abs(m1["mass_gas"] - m0["mass_gas"]) <= 1e-6 * m0["mass_gas"]
    assert abs(m1["mass_bme"] - m0["mass_bme"]) <= 1e-6 * m0["mass_bme"]


def test_gravity_off_and_fixed_dt(flic):
    s = I.random_state((16, 16, 16), seed=9, rough=True)
    ref, _ = run_oracle(s, 2, dt=1e-3, G=0.0)
    out, grec = run_gpu(flic, s, 2, dt=1e-3, G=0.0)
    assert grec[-1]["dt"] == 1e-3
    assert max(max_rel(out, ref).values()) <= 1e-11


def test_uniform_state_fixed_point(flic):
    N = 16
    one = np.ones((N, N, N))
    from helpers import state_from_primitives
    P = {"xx": 0.5 * one, "yy": 0.7 * one, "zz": 0.6 * one, "xy": 0.1 * one, "xz": -0.05 * one, "yz": 0.02 * one}
    st = state_from_primitives(1.3 * one, (0.2 * one, -0.1 * one, 0.05 * one), 0.8 * one, 0.9 * one,
                               (-0.15 * one, 0.3 * one, 0.1 * one), P, 5.0 / 3.0)
    s = I.Setup(st, 2.0 / N)
    out, _ = run_gpu(flic, s, 3)
    for f in FIELDS:
        assert np.max(np.abs(out[f] - st[f])) <= 1e-14 * max(1.0, np.max(np.abs(st[f]))), f


def test_state_round_trip_fp64(flic):
    s = I.random_state((12, 12, 12), seed=2, rough=True)
    with flic.Grid(12, precision="fp64") as g:
        g.set_state(s.state)
        out = g.get_state()
    for f in FIELDS:
        assert np.array_equal(out[f], s.state[f]), f


def test_diagnostics_of_current_state(flic):
    s = I.random_state((24, 24, 24), seed=3)
    prm = O.Params(h=s.h)
    phi = O.solve_poisson(s.state, prm)
    ref = O.diagnostics(s.state, phi, prm)
    with flic.Grid(24, precision="fp64", box=(-1.0, -1.0 + 24 * s.h)) as g:
        g.set_state(s.state)
        d = g.diagnostics()
    for k, v in ref.items():
        assert abs(d[k] - v) <= 1e-12 * max(1.0, abs(v)), (k, d[k], v)
    assert abs(d["vmax"] - O.max_signal_speed(s.state, prm)) <= 1e-14


def test_nonphysical_state_is_reported(flic):
    s = I.random_state((8, 8, 8), seed=4)
    st = dict(s.state)
    st["rho"] = st["rho"].copy()
    st["rho"][1, 2, 3] = -1.0
    with flic.Grid(8) as g:
        with pytest.raises(flic.FlicError) as ei:
            g.set_state(st)
        assert ei.value.code == flic.ERR_NONPHYSICAL


@pytest.mark.parametrize("field", ["mx", "qy"])
def test_step_with_overflow_is_reported(flic, field):
    # float32 storage: a momentum of 1e30 in one cell squares past the float32
    # range in the kinetic part of the energy balance (Sec. 2.4: K = |m|^2 / 2 rho,
    # q q^T / n), so the step's output there is not finite and must be flagged;
    # the float64 path steps the same state without overflow
    s = I.random_state((16, 16, 16), seed=9)
    st = {k: v.copy() for k, v in s.state.items()}
    st[field][3, 4, 5] = 1e30
    with flic.Grid(16, precision="mixed", gamma=s.gamma) as g:
        g.set_state(st)
        with pytest.raises(flic.FlicError) as ei:
            g.step()
        assert ei.value.code == flic.ERR_NONPHYSICAL
        assert g.step_diagnostics()["nonphysical"]
    with flic.Grid(16, precision="fp64", gamma=s.gamma) as g:
        g.set_state(st)
        g.step()
        assert not g.step_diagnostics()["nonphysical"]


def test_invalid_arguments(flic):
    with pytest.raises(flic.FlicError) as ei:
        flic.Grid(10)
    assert ei.value.code == flic.ERR_INVALID_ARG
    with pytest.raises(flic.FlicError):
        flic.Grid(16, gamma=1.0)


@pytest.mark.parametrize("N,precision,tol", [(8, "fp64", 1e-12), (12, "fp64", 1e-12), (24, "fp64", 1e-12),
                                             (32, "fp64", 1e-12), (48, "mixed", 2e-5), (64, "mixed", 2e-5)])
def test_poisson_isolated(flic, N, precision, tol):
    """Zero-padded solve vs the oracle's (pinned to a direct O(N^6) sum)."""
    s = I.random_state((N, N, N), seed=60 + N)
    prm = O.Params(h=s.h, poisson="isolated")
    ref = O.solve_poisson(s.state, prm)
    with flic.Grid(N, precision=precision, poisson="isolated", box=(-1.0, -1.0 + s.h * N)) as g:
        g.set_state(s.state)
        phi = g.solve_poisson()
    assert np.max(np.abs(phi - ref)) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("N", [16, 24])
def test_steps_isolated_fp64(flic, N):
    s = I.random_state((N, N, N), seed=70 + N)
    prm = O.Params(h=s.h, gamma=s.gamma, poisson="isolated")
    ref, rrec = O.run(s.state, prm, 3)
    with flic.Grid(N, precision="fp64", poisson="isolated", box=(-1.0, -1.0 + s.h * N)) as g:
        g.set_state(s.state)
        for _ in range(3):
            g.step()
        out = g.get_state()
        d = g.step_diagnostics()
    err = rel_l1(out, ref)
    assert max(err.values()) <= 1e-10, err
    assert abs(d["epot"] - rrec[-1]["epot"]) <= 1e-11 * abs(rrec[-1]["epot"])


@pytest.mark.parametrize("N,poisson,rough", [(8, "isolated", True), (12, "periodic", False), (24, "isolated", True),
                                             (48, "isolated", False), (64, "periodic", True)])
def test_one_step_outflow_fp64(flic, N, poisson, rough):
    """Outflow (zero-gradient) hydro boundaries: ghost copies of the edge cells,
    partial tiles and ragged z chunks at every face of the box."""
    s = I.random_state((N, N, N), seed=80 + N, rough=rough)
    prm = O.Params(h=s.h, gamma=s.gamma, poisson=poisson, boundary="outflow")
    ref, rrec = O.run(s.state, prm, 1)
    with flic.Grid(N, precision="fp64", gamma=s.gamma, poisson=poisson, boundary="outflow",
                   box=(-1.0, -1.0 + s.h * N)) as g:
        g.set_state(s.state)
        g.step()
        out = g.get_state()
        d = g.step_diagnostics()
    err = max_rel(out, ref)
    assert max(err.values()) <= 1e-11, err
    r = rrec[-1]
    assert abs(d["dt"] - r["dt"]) <= 1e-14 * r["dt"]
    for k in ("mass_gas", "mass_bme", "kappa_gas", "kappa_bme", "vmax", "epot"):
        assert abs(d[k] - r[k]) <= 1e-11 * max(abs(r[k]), 1e-300), (k, d[k], r[k])


def test_outflow_mixed_ten_steps(flic):
    s = I.head_on(32)
    prm = O.Params(h=s.h, gamma=s.gamma, poisson="isolated", boundary="outflow")
    ref, _ = O.run(s.state, prm, 10)
    with flic.Grid(32, precision="mixed", gamma=s.gamma, poisson="isolated", boundary="outflow") as g:
        g.set_state(s.state)
        g.run(10)
        out = g.get_state()
    err = rel_l1(out, ref)
    assert err["rho"] <= 1e-4 and err["n"] <= 1e-4, err


def test_outflow_ten_steps_fp64_graph(flic):
    s = I.random_state((24, 24, 24), seed=91)
    prm = O.Params(h=s.h, gamma=s.gamma, poisson="isolated", boundary="outflow")
    ref, _ = O.run(s.state, prm, 10)
    with flic.Grid(24, precision="fp64", gamma=s.gamma, poisson="isolated", boundary="outflow",
                   box=(-1.0, -1.0 + s.h * 24)) as g:
        g.set_state(s.state)
        g.run(10)
        out = g.get_state()
    err = rel_l1(out, ref)
    assert max(err.values()) <= 1e-10, err


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pinned_host_state_round_trip(flic, precision):
    """Page-locked host arrays (read and written in place by the conversion
    kernels) give the same state as pageable ones."""
    torch = pytest.importorskip("torch")
    s = I.random_state((24, 24, 24), seed=6, rough=True)
    pinned_in = torch.empty((22, 24, 24, 24), dtype=torch.float64, pin_memory=True)
    pinned_out = torch.empty((22, 24, 24, 24), dtype=torch.float64, pin_memory=True)
    pinned_in.numpy()[...] = I.stack(s.state)
    with flic.Grid(24, precision=precision, box=(-1.0, -1.0 + 24 * s.h)) as g:
        g.set_state([pinned_in[i] for i in range(22)])
        ref = g.get_state()
        g.get_state([pinned_out[i] for i in range(22)])
        g.step()
        a = g.get_state()
        g.set_state(s.state)
        g.step()
        b = g.get_state()
    got = I.unstack(pinned_out.numpy())
    for f in FIELDS:
        assert np.array_equal(got[f], ref[f]), f
        assert np.array_equal(a[f], b[f]), f
    if precision == "fp64":
        for f in FIELDS:
            assert np.array_equal(ref[f], s.state[f]), f


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 2e-5)])
def test_cooling_placeholder(flic, precision, tol):
    """The gas cooling placeholder q = Lambda rho^2 sqrt(eps) (reading s13): two
    steps of a rough state equal the oracle's; a uniform gas at rest decays like
    the oracle's (pinned there to the exact solution of its ODE)."""
    N = 24
    s = I.random_state((N, N, N), seed=77, rough=True)
    prm = O.Params(h=s.h, gamma=s.gamma, cooling=0.8)
    ref, _ = O.run(s.state, prm, 2)
    with flic.Grid(N, precision=precision, gamma=s.gamma, cooling=0.8, box=(-1.0, -1.0 + N * s.h)) as g:
        g.set_state(s.state)
        g.step()
        g.step()
        out = g.get_state()
    err = max_rel(out, ref)
    assert max(err.values()) <= tol, err
    from helpers import state_from_primitives
    one = np.ones((16, 16, 16))
    P = {"xx": 0.3 * one, "yy": 0.3 * one, "zz": 0.3 * one, "xy": 0 * one, "xz": 0 * one, "yz": 0 * one}
    st = state_from_primitives(1.3 * one, (0 * one, 0 * one, 0 * one), 0.8 * one, 0.5 * one,
                               (0 * one, 0 * one, 0 * one), P, 5.0 / 3.0)
    ref, _ = O.run(st, O.Params(h=2.0 / 16, G=0.0, cooling=0.7), 40, dt=0.01)
    with flic.Grid(16, precision=precision, G=0.0, cooling=0.7) as g:
        g.set_state(st)
        g.run(40, 0.01)
        out = g.get_state()
    assert np.max(np.abs(out["e"] - ref["e"])) <= 10 * tol * np.max(ref["e"])
    assert np.max(ref["e"]) < 0.85 * 1.2   # the gas cooled


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 2e-5)])
@pytest.mark.parametrize("N", [12, 24])
def test_flux_reading_b(flic, precision, tol, N):
    """Reading B of the Lagrangian transport velocity (the printed 4-term
    transverse mean, oracle Params.flux = "B") on the CUDA path: one step of a
    rough state equals the oracle's; it differs from reading A."""
    s = I.random_state((N, N, N), seed=900 + N, rough=True)
    prm = O.Params(h=s.h, gamma=s.gamma, flux="B")
    ref, rrec = O.run(s.state, prm, 1)
    refA, _ = O.run(s.state, O.Params(h=s.h, gamma=s.gamma), 1)
    with flic.Grid(N, precision=precision, gamma=s.gamma, flux="B", box=(-1.0, -1.0 + N * s.h)) as g:
        g.set_state(s.state)
        g.step()
        out = g.get_state()
        d = g.step_diagnostics()
        # setup, 5 FFT passes, 2 x 2 reading-B kernels, the reduction (1 launch over float32
        # pairs, 2 levels in float64)
        assert g.launches_per_step() == 1 + 5 + 4 + (2 if precision == "fp64" else 1)
    err = max_rel(out, ref)
    assert max(err.values()) <= tol, err
    assert max(max_rel(refA, ref).values()) > 1e-4
    r = rrec[-1]
    for k in ("mass_gas", "mass_bme", "kappa_gas", "kappa_bme", "vmax"):
        assert abs(d[k] - r[k]) <= (1e-11 if precision == "fp64" else 1e-5) * abs(r[k]), (k, d[k], r[k])


def test_flux_reading_b_ten_steps_and_limits(flic):
    s = I.head_on(32)
    prm = O.Params(h=s.h, gamma=s.gamma, flux="B")
    ref, _ = O.run(s.state, prm, 10)
    with flic.Grid(32, precision="fp64", gamma=s.gamma, flux="B") as g:
        g.set_state(s.state)
        g.run(10)
        out = g.get_state()
    err = rel_l1(out, ref)
    assert max(err.values()) <= 1e-10, err
    with pytest.raises(flic.FlicError) as ei:
        flic.Grid(16, flux="B", boundary="outflow")
    assert ei.value.code == flic.ERR_INVALID_ARG
