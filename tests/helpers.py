"""Shared test helpers: 1D states embedded in the 3D layout, error norms, transforms."""
from __future__ import annotations

import numpy as np

from paper_1311_0861_gb300.inputs import FIELDS

TENSOR = ("xx", "yy", "zz", "xy", "xz", "yz")


def state_from_primitives(rho, v, p, n, u, P, gamma):
    """22-field conserved state from primitive arrays (v, u: 3-tuples; P: dict of 6)."""
    e = p / (gamma - 1.0)
    m = [rho * vd for vd in v]
    q = [n * ud for ud in u]
    st = {"rho": rho, "mx": m[0], "my": m[1], "mz": m[2], "e": e,
          "E": e + (m[0] ** 2 + m[1] ** 2 + m[2] ** 2) / (2.0 * rho),
          "n": n, "qx": q[0], "qy": q[1], "qz": q[2]}
    qd = {"x": q[0], "y": q[1], "z": q[2]}
    for k in TENSOR:
        st["P" + k] = P[k] + 0.0 * rho
        st["nE" + k] = P[k] + qd[k[0]] * qd[k[1]] / n
    return {f: np.ascontiguousarray(np.broadcast_to(st[f], rho.shape), dtype=np.float64) for f in FIELDS}


def tube_state(x, left, right, in_left, gamma, bme=None):
    """1D gas tube along x (shape (1, 1, Nx)); ``in_left`` masks the left state.

    The moment fluid is a passive uniform state unless ``bme`` = (left, right)
    dicts of n, u_x, u_y, u_z and the 6 stress components are given."""
    sh = (1, 1, x.size)
    m = in_left.reshape(sh)

    def pick(a, b):
        return np.where(m, a, b).astype(np.float64)

    rho = pick(left["rho"], right["rho"])
    v = (pick(left["v"], right["v"]), np.zeros(sh), np.zeros(sh))
    p = pick(left["p"], right["p"])
    if bme is None:
        n = np.ones(sh)
        u = (np.zeros(sh), np.zeros(sh), np.zeros(sh))
        P = {k: (np.ones(sh) if k[0] == k[1] else np.zeros(sh)) for k in TENSOR}
    else:
        bl, br = bme
        n = pick(bl["rho"], br["rho"])
        u = (pick(bl["ux"], br["ux"]), pick(bl["uy"], br["uy"]), pick(bl["uz"], br["uz"]))
        P = {k: pick(bl["P" + k], br["P" + k]) for k in TENSOR}
    return state_from_primitives(rho, v, p, n, u, P, gamma)


def run_to(oracle, st, prm, t_end, max_steps=100000):
    t = 0.0
    k = 0
    while t < t_end * (1 - 1e-14) and k < max_steps:
        dt = min(oracle.cfl_dt(st, prm), t_end - t)
        st, _ = oracle.step(st, prm, dt)
        t += dt
        k += 1
    return st, k


def rel_l1(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.sum(np.abs(b))
    return float(np.sum(np.abs(a - b)) / den) if den > 0 else float(np.sum(np.abs(a - b)))


# -- axis permutation and reflection of a state (for equivariance pins) ------
_CYC = {"x": "y", "y": "z", "z": "x"}      # axis x -> y, y -> z, z -> x
_INV = {v: k for k, v in _CYC.items()}


def _name(prefix, comp):
    return prefix + comp


def permute_state(st):
    """Rotate the grid and every vector/tensor component by x->y->z->x."""
    out = {}
    tr = lambda a: np.ascontiguousarray(np.transpose(a, (1, 2, 0)))
    for f in ("rho", "E", "e", "n"):
        out[f] = tr(st[f])
    for pre in ("m", "q"):
        for a in "xyz":
            out[pre + a] = tr(st[pre + _INV[a]])
    for pre in ("nE", "P"):
        for k in TENSOR:
            i, j = _INV[k[0]], _INV[k[1]]
            src = pre + (i + j if (i + j) in TENSOR else j + i)
            out[pre + k] = tr(st[src])
    return out


def reflect_x(st):
    """Mirror the grid in x (i -> N-1-i) with x-odd components negated."""
    out = {}
    for f in FIELDS:
        a = st[f][..., ::-1]
        odd = f in ("mx", "qx") or f in ("nExy", "nExz", "Pxy", "Pxz")
        out[f] = np.ascontiguousarray(-a if odd else a)
    return out


def balance_branch_state(N, seed, gamma=5.0 / 3.0):
    """A rough random N^3 state whose cells, after one step, fall clearly on
    either side of the energy balance's switches (reading s11), in a pattern that
    makes neighbouring cells take different branches.

    Gas: consistent cells (E = e + K, so E - K = e >> eta E: e is taken from E)
    next to cells with E = K - e/2 (E - K < 0: E is reset from e).  Moments,
    cycling over four cell classes: consistent (nE = Pi + q q^T/n), a negative
    diagonal of Pi^E = nE - q q^T/n along x (Pi^E_xx = -Pi_xx, with the other
    two diagonal entries raised to 3 Pi_dd so the trace stays positive), the same
    along z, and a negative trace of Pi^E; all but the first are reset.
    """
    from paper_1311_0861_gb300.inputs import random_state

    s = random_state((N, N, N), seed=seed, rough=True)
    st = {f: v.copy() for f, v in s.state.items()}
    k, j, i = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    K = (st["mx"] ** 2 + st["my"] ** 2 + st["mz"] ** 2) / (2.0 * st["rho"])
    odd = (i + j + k) % 2 == 1
    st["E"] = np.where(odd, K - 0.5 * st["e"], st["e"] + K)
    cls = (i + 2 * j + 3 * k) % 4
    q = {"x": st["qx"], "y": st["qy"], "z": st["qz"]}
    for c in TENSOR:
        qq = q[c[0]] * q[c[1]] / st["n"]
        P = st["P" + c]
        dev = np.zeros_like(P)
        if c[0] == c[1]:
            dev = np.where(cls == 1, (-2.0 if c == "xx" else 2.0) * P, dev)
            dev = np.where(cls == 2, (-2.0 if c == "zz" else 2.0) * P, dev)
            dev = np.where(cls == 3, -2.0 * P, dev)
        st["nE" + c] = qq + P + dev
    return s.__class__(st, s.h, gamma)


def cold_flow_state(N, mach, gamma=5.0 / 3.0):
    """A cold, fast N^3 flow on [-1, 1]^3: both fluids stream along x at 0.5
    (the moments at 0.4 along x and 0.1 along y) with a weak shear and a 10 %
    density ripple; the gas sound speed and the moments' dispersion speed
    sqrt(3 Pi_dd / n) are 0.5 / mach, so the kinetic energy exceeds the thermal
    one by about mach^2 and E - |m|^2/(2 rho) is a small difference of large
    numbers."""
    h = 2.0 / N
    c = -1.0 + (np.arange(N) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    rho = 1.0 + 0.1 * np.sin(np.pi * x) * np.cos(np.pi * y)
    cs = 0.5 / mach
    p = rho * cs * cs / gamma
    v = (0.5 + 0.02 * np.sin(np.pi * y), 0.02 * np.cos(np.pi * z), 0.0 * rho)
    n = 0.5 * (1.0 + 0.1 * np.cos(np.pi * (x + z)))
    u = (0.4 + 0.02 * np.sin(np.pi * z), 0.1 + 0.0 * n, 0.02 * np.sin(np.pi * x))
    s2 = cs * cs / 3.0
    P = {k: (n * s2 if k[0] == k[1] else 0.0 * n) for k in TENSOR}
    return state_from_primitives(rho, v, p, n, u, P, gamma), h
