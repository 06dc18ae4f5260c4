"""Plain FP64 oracle of one FlIC/Godunov step for gas + Boltzmann-moment fluid.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Arrays are numpy float64
with shape ``(..., Nz, Ny, Nx)``: x is the fastest axis, matching the
structure-of-arrays layout ``idx = i + Nx*(j + Ny*k)``.  Optional leading axes are
batch axes, which lets the same code evaluate small periodic windows cut out of a
large grid (``advance_window``).

Readings of passages that are silent, ambiguous or garbled in the paper are
collected in ``READINGS`` and cited where they are used.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np

__all__ = [
    "FIELDS", "GAS_FIELDS", "BME_FIELDS", "READINGS", "CUBE_SELF_POTENTIAL",
    "Params", "gas_face", "bme_face", "poisson_periodic", "poisson_isolated",
    "green_isolated", "solve_poisson", "max_signal_speed", "cfl_dt", "advance",
    "advance_window", "diagnostics", "step", "run", "nonphysical",
]

# Field order of the 22-field state (also the order of the C-ABI field arrays).
GAS_FIELDS = ("rho", "mx", "my", "mz", "E", "e")
BME_FIELDS = ("n", "qx", "qy", "qz",
              "nExx", "nEyy", "nEzz", "nExy", "nExz", "nEyz",
              "Pxx", "Pyy", "Pzz", "Pxy", "Pxz", "Pyz")
FIELDS = GAS_FIELDS + BME_FIELDS

DIRS = ("x", "y", "z")
_AXIS = {"x": -1, "y": -2, "z": -3}
# Tangent directions paired with each face normal (Sec. 2.2 writes the x-face
# system with tangents y, z; the closed form is symmetric in the two tangents).
_TANGENTS = {"x": ("y", "z"), "y": ("x", "z"), "z": ("x", "y")}

# Potential at the centre of a uniform cube of unit side and unit density
# (G = 1): integral of 1/|r| over [-1/2, 1/2]^3 = 3 ln(2 + sqrt 3) - pi/2.
CUBE_SELF_POTENTIAL = 3.0 * math.log(2.0 + math.sqrt(3.0)) - 0.5 * math.pi

READINGS = {
    "s1": "Lagrangian flux (Sec. 2.1): F_{i+1/2} = W_{i+1/2} * f_upwind with W the "
          "face velocity of the same face (reading A of the garbled 4-term average); "
          "reading B (flux='B') takes the printed 4-term form literally: W is the mean "
          "of the face velocities of the same face orientation at the four transverse "
          "diagonal neighbours (k+-1, l+-1), and the upwind side follows its sign.",
    "s2": "Upwind tie W == 0 gives F = 0 either way.",
    "s3": "The transport velocity is the Eulerian-stage face solution at time n.",
    "s4": "Bracketed BME coefficients (Sec. 2.2) are arithmetic L/R means of n, "
          "Pi_nn, Pi_nt; the gas formula is used exactly as printed.",
    "s5": "Poisson symbol (Sec. 2.3) carries a minus sign: Phi_hat = -4 pi G h^2 "
          "s_hat / (6 (1 - prod_d (1 - 2/3 sin^2(pi k_d / N_d)))); the printed "
          "positive sign contradicts Laplace(Phi) = 4 pi rho (Sec. 2).",
    "s6": "Poisson zero mode Phi_hat_0 = 0 (mean-free potential).",
    "s7": "Poisson boundary periodic; 'isolated' mode is the zero-padded (2N)^3 "
          "convolution with g(r) = -G h^3/|r|, g(0) = -G h^2 * 2.3800774.",
    "s8": "Hydro boundaries periodic; 'outflow' mode (zero gradient): two layers of "
          "ghost cells along each axis copy the nearest edge cell of the time-n state "
          "and potential; the step is computed on the extended grid and cropped, so "
          "ghost cells take the Eulerian stage from their own (ghost) neighbours.",
    "s9": "Gravity: central difference of Phi^n with rho^n, m^n, n^n, q^n.",
    "s10": "CFL: tau = C h / max over cells and axes of (|v_d| + sqrt(gamma p/rho)) "
           "and (|u_d| + sqrt(3 Pi_dd / n)).",
    "s11": "Energy balance (Sec. 2.4): after measuring kappa, gas takes "
           "eps = E - |m|^2/(2 rho) when eps >= eta E, else resets E = e + |m|^2/(2 rho); "
           "BME takes Pi = nE - q q^T/n when tr >= eta tr(nE) and every diagonal "
           "entry is positive, else resets nE = Pi + q q^T/n; eta = 1e-3.",
    "s12": "Cell centres at box_min + (i + 1/2) h.",
    "s13": "No cooling by default (q = 0).  Params.cooling = Lambda > 0 switches on an "
           "analytic placeholder for the cooling function of the gas energy equations "
           "(Sec. 2; the paper's tabulated Sutherland-Dopita function is not available): "
           "q = Lambda rho^2 sqrt(eps) = Lambda rho sqrt(rho e), evaluated on the time-n "
           "state and subtracted (times tau) from both E and e in the Eulerian stage.",
    "s14": "No floors; non-positive rho, n, e, Pi_dd or a non-finite value flags "
           "the state non-physical.",
    "s15": "kappa_bme sums the 6 independent components of the symmetric tensor.",
}


@dataclass(frozen=True)
class Params:
    """Physical and numerical constants of a run (code units)."""

    h: float                   # cell width (cubic cells, Sec. 2 grid)
    gamma: float = 5.0 / 3.0   # adiabatic index of the gas
    G: float = 1.0             # gravitational constant; 0 switches gravity off
    courant: float = 0.2       # Courant number of the CFL step (reading s10)
    eta: float = 1e-3          # energy-balance switch (reading s11)
    poisson: str = "periodic"  # "periodic" (s5/s6) or "isolated" (s7)
    boundary: str = "periodic" # hydro boundaries: "periodic" or "outflow" (s8)
    flux: str = "A"            # Lagrangian transport velocity: reading "A" or "B" of s1
    cooling: float = 0.0       # Lambda of the cooling placeholder q = Lambda rho^2 sqrt(eps) (s13)


# --------------------------------------------------------------------------
# periodic shifts and face differences
# --------------------------------------------------------------------------
def _up(a, d):
    """Value at c + e_d (periodic)."""
    return np.roll(a, -1, axis=_AXIS[d])


def _dn(a, d):
    """Value at c - e_d (periodic)."""
    return np.roll(a, 1, axis=_AXIS[d])


def _delta(face, d):
    """X(c + e_d/2) - X(c - e_d/2) for a face array stored at index c = face c+1/2."""
    return face - _dn(face, d)


def _T(t, i, j):
    """Component (i, j) of a symmetric tensor stored by its 6 independent entries."""
    return t[i + j] if (i + j) in t else t[j + i]


# --------------------------------------------------------------------------
# Sec. 2.1: gas Eulerian face solution (linearised Riemann problem)
# --------------------------------------------------------------------------
def gas_face(rL, vL, pL, rR, vR, pR, gamma):
    """Face velocity V and pressure P, Sec. 2.1 closed form (both printed formulas)."""
    V = 0.5 * (vL + vR) + 0.5 * (pL - pR) * np.sqrt((rL + rR) / (rL * rR * gamma * (pL + pR)))
    P = 0.5 * (pL + pR) + 0.5 * (vL - vR) * np.sqrt(rL * rR * gamma * (pL + pR) / (rL + rR))
    return V, P


# --------------------------------------------------------------------------
# Sec. 2.2: Boltzmann-moment Eulerian face solution (6x6 linear system)
# --------------------------------------------------------------------------
def bme_face(nL, unL, ut1L, ut2L, PnnL, Pnt1L, Pnt2L,
             nR, unR, ut1R, ut2R, PnnR, Pnt1R, Pnt2R):
    """Face (u_n, u_t1, u_t2, Pi_nn, Pi_nt1, Pi_nt2), Sec. 2.2 closed form.

    The bracketed coefficients are evaluated at the arithmetic means of n, Pi_nn
    and Pi_nt (reading s4).
    """
    rho = 0.5 * (nL + nR)
    a = 0.5 * (PnnL + PnnR)
    b1 = 0.5 * (Pnt1L + Pnt1R)
    b2 = 0.5 * (Pnt2L + Pnt2R)
    s3 = math.sqrt(3.0)
    Z1 = np.sqrt(3.0 * rho * a)      # sqrt(3 rho Pi_nn): fast (longitudinal) impedance
    Z2 = np.sqrt(rho * a)            # sqrt(rho Pi_nn): slow (shear) impedance
    dPnn = 0.5 * (PnnL - PnnR)
    dun = 0.5 * (unL - unR)
    un = 0.5 * (unL + unR) + dPnn / Z1
    ut1 = 0.5 * (ut1L + ut1R) + 0.5 * (Pnt1L - Pnt1R) / Z2 + dPnn * b1 * (1.0 - s3) / (a * Z1)
    ut2 = 0.5 * (ut2L + ut2R) + 0.5 * (Pnt2L - Pnt2R) / Z2 + dPnn * b2 * (1.0 - s3) / (a * Z1)
    Pnn = 0.5 * (PnnL + PnnR) + dun * Z1
    Pnt1 = 0.5 * (Pnt1L + Pnt1R) + 0.5 * (ut1L - ut1R) * Z2 + dun * b1 * rho * (s3 - 1.0) / Z2
    Pnt2 = 0.5 * (Pnt2L + Pnt2R) + 0.5 * (ut2L - ut2R) * Z2 + dun * b2 * rho * (s3 - 1.0) / Z2
    return un, ut1, ut2, Pnn, Pnt1, Pnt2


# --------------------------------------------------------------------------
# Sec. 2.3: Poisson equation for the total potential, Laplace(Phi) = 4 pi G (rho + n)
# --------------------------------------------------------------------------
def poisson_periodic(s, h, G):
    """Periodic solve with the 27-point stencil symbol of Sec. 2.3 (readings s5, s6)."""
    nz, ny, nx = s.shape
    sh = np.fft.rfftn(s)
    kz = np.arange(nz)[:, None, None]
    ky = np.arange(ny)[None, :, None]
    kx = np.arange(nx // 2 + 1)[None, None, :]

    def f(k, n):
        return 1.0 - (2.0 / 3.0) * np.sin(np.pi * k / n) ** 2

    D = 6.0 * (1.0 - f(kz, nz) * f(ky, ny) * f(kx, nx))
    D[0, 0, 0] = 1.0
    ph = -4.0 * np.pi * G * h * h * sh / D
    ph[0, 0, 0] = 0.0
    return np.fft.irfftn(ph, s=s.shape, axes=(-3, -2, -1))


def green_isolated(shape, h, G):
    """Green's function on the (2N)^3 padded grid with wrapped distances (reading s7)."""
    axes = []
    for n in shape:
        i = np.arange(2 * n)
        axes.append(np.minimum(i, 2 * n - i).astype(np.float64))
    dz, dy, dx = np.meshgrid(*axes, indexing="ij")
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    r[0, 0, 0] = 1.0
    g = -G * h ** 3 / (h * r)
    g[0, 0, 0] = -G * h * h * CUBE_SELF_POTENTIAL
    return g


def poisson_isolated(s, h, G):
    """Zero-padded (Hockney-Eastwood) solve: linear convolution of s with g (reading s7)."""
    nz, ny, nx = s.shape
    pad = np.zeros((2 * nz, 2 * ny, 2 * nx))
    pad[:nz, :ny, :nx] = s
    g = green_isolated(s.shape, h, G)
    phi = np.fft.irfftn(np.fft.rfftn(pad) * np.fft.rfftn(g), s=pad.shape, axes=(-3, -2, -1))
    return phi[:nz, :ny, :nx].copy()


def solve_poisson(st, prm: Params):
    """Potential of the total density s = rho + n (Sec. 2.3); zero when G == 0."""
    s = st["rho"] + st["n"]
    if prm.G == 0.0:
        return np.zeros_like(s)
    if prm.poisson == "periodic":
        return poisson_periodic(s, prm.h, prm.G)
    if prm.poisson == "isolated":
        return poisson_isolated(s, prm.h, prm.G)
    raise ValueError(prm.poisson)


# --------------------------------------------------------------------------
# time step size (reading s10)
# --------------------------------------------------------------------------
def max_signal_speed(st, prm: Params):
    """max over cells and axes of |v_d| + c_gas and |u_d| + sqrt(3 Pi_dd / n)."""
    rho, n = st["rho"], st["n"]
    cs = np.sqrt(prm.gamma * (prm.gamma - 1.0) * st["e"] / rho)
    vmax = 0.0
    for d in DIRS:
        vmax = max(vmax, float(np.max(np.abs(st["m" + d] / rho) + cs)))
        vmax = max(vmax, float(np.max(np.abs(st["q" + d] / n) + np.sqrt(3.0 * st["P" + d + d] / n))))
    return vmax


def cfl_dt(st, prm: Params):
    return prm.courant * prm.h / max_signal_speed(st, prm)


# --------------------------------------------------------------------------
# one step of both fluids given Phi^n and tau
# --------------------------------------------------------------------------
def _extend(a, m):
    """Zero-gradient extension by m cells on each side of the three grid axes (s8)."""
    pad = [(0, 0)] * (a.ndim - 3) + [(m, m)] * 3
    return np.pad(a, pad, mode="edge")


def _crop(a, m):
    return a[..., m:-m, m:-m, m:-m]


def advance(st, phi, tau, prm: Params, record=None):
    """Eulerian stage, Lagrangian stage and energy balance of both fluids.

    Returns ``(new_state, kappa)`` where ``kappa`` holds the per-cell integrands of
    kappa_gas and kappa_bme (Sec. 2.4, times h^3) measured on the post-Lagrangian
    state before the balance.

    ``record``: an optional dict that receives, per cell, which branch of the
    energy balance (reading s11) was taken and how far from its switch the cell
    was (instrumentation for tests; the arithmetic is unchanged):
    ``gas_take`` (e = E - K taken), ``gas_margin`` ((E - K - eta E) / |E|),
    ``bme_take`` (Pi = nE - q q^T/n taken), ``bme_trace_margin``
    ((tr Pi^E - eta tr nE) / |tr nE|), ``bme_diag_min`` (min_d Pi^E_dd / |tr nE|).
    """
    if prm.boundary == "outflow":
        # reading s8: the update of a cell reaches 2 cells, so 2 ghost layers
        # make the periodic shifts below act as the zero-gradient boundary
        ext = {f: _extend(st[f], 2) for f in FIELDS}
        rec = {} if record is not None else None
        new, kap = advance(ext, _extend(phi, 2), tau, replace(prm, boundary="periodic"), rec)
        if record is not None:
            record.update({k: _crop(v, 2) for k, v in rec.items()})
        return {f: _crop(new[f], 2) for f in FIELDS}, {k: _crop(v, 2) for k, v in kap.items()}
    if prm.boundary != "periodic":
        raise ValueError(prm.boundary)
    h, g, eta = prm.h, prm.gamma, prm.eta
    r = tau / h
    gphi = {d: (_up(phi, d) - _dn(phi, d)) / (2.0 * h) for d in DIRS}   # reading s9

    # ---------------- gas, Sec. 2.1 ----------------
    rho = st["rho"]
    m = {d: st["m" + d] for d in DIRS}
    E, e = st["E"], st["e"]
    v = {d: m[d] / rho for d in DIRS}
    p = (g - 1.0) * e
    V, P = {}, {}
    for d in DIRS:
        V[d], P[d] = gas_face(rho, v[d], p, _up(rho, d), _up(v[d], d), _up(p, d), g)
    # Eulerian stage: pressure and gravity (Sec. 2 gas equations minus div(f v))
    m1 = {d: m[d] - r * _delta(P[d], d) - tau * rho * gphi[d] for d in DIRS}
    E1 = (E - r * sum(_delta(P[d] * V[d], d) for d in DIRS)
          - tau * sum(m[d] * gphi[d] for d in DIRS))
    e1 = e - tau * (g - 1.0) * e * sum(_delta(V[d], d) for d in DIRS) / h
    if prm.cooling != 0.0:
        # the cooling function -q of both energy equations (Sec. 2), reading s13
        q = prm.cooling * rho * np.sqrt(rho * e)
        E1 = E1 - tau * q
        e1 = e1 - tau * q
    gas1 = {"rho": rho, "mx": m1["x"], "my": m1["y"], "mz": m1["z"], "E": E1, "e": e1}

    # ---------------- Boltzmann moments, Sec. 2.2 ----------------
    n = st["n"]
    q = {i: st["q" + i] for i in DIRS}
    nE = {k: st["nE" + k] for k in ("xx", "yy", "zz", "xy", "xz", "yz")}
    Pi = {k: st["P" + k] for k in ("xx", "yy", "zz", "xy", "xz", "yz")}
    u = {i: q[i] / n for i in DIRS}
    ustar, Pstar = {}, {}      # ustar[d][i] = u_i*, Pstar[d][i] = Pi*_{i d} on axis-d faces
    for d in DIRS:
        t1, t2 = _TANGENTS[d]
        left = (n, u[d], u[t1], u[t2], _T(Pi, d, d), _T(Pi, d, t1), _T(Pi, d, t2))
        right = tuple(_up(a, d) for a in left)
        un, ut1, ut2, Pnn, Pnt1, Pnt2 = bme_face(*left, *right)
        ustar[d] = {d: un, t1: ut1, t2: ut2}
        Pstar[d] = {d: Pnn, t1: Pnt1, t2: Pnt2}
    q1 = {i: q[i] - r * sum(_delta(Pstar[d][i], d) for d in DIRS) - tau * n * gphi[i]
          for i in DIRS}
    nE1, Pi1 = {}, {}
    for k in nE:
        i, j = k[0], k[1]
        nE1[k] = (nE[k]
                  - r * sum(_delta(Pstar[d][j] * ustar[d][i] + Pstar[d][i] * ustar[d][j], d)
                            for d in DIRS)
                  - tau * (q[i] * gphi[j] + q[j] * gphi[i]))
        Pi1[k] = Pi[k] - r * sum(_T(Pi, j, d) * _delta(ustar[d][i], d)
                                 + _T(Pi, i, d) * _delta(ustar[d][j], d) for d in DIRS)
    bme1 = {"n": n, "qx": q1["x"], "qy": q1["y"], "qz": q1["z"]}
    bme1.update({"nE" + k: nE1[k] for k in nE1})
    bme1.update({"P" + k: Pi1[k] for k in Pi1})

    # ---------------- Lagrangian stage, Sec. 2.1 (reading s1) ----------------
    def transport(f1, W):
        out = f1
        for d in DIRS:
            F = W[d] * np.where(W[d] > 0.0, f1, _up(f1, d))
            out = out - r * _delta(F, d)
        return out

    Wgas = V
    Wbme = {d: ustar[d][d] for d in DIRS}
    if prm.flux == "B":
        Wgas, Wbme = _diagonal_mean(Wgas), _diagonal_mean(Wbme)
    elif prm.flux != "A":
        raise ValueError(prm.flux)
    new = {k: transport(gas1[k], Wgas) for k in GAS_FIELDS}
    new.update({k: transport(bme1[k], Wbme) for k in BME_FIELDS})

    # ---------------- Sec. 2.4: kappa, then energy balance (reading s11) --------
    vol = h ** 3
    K = (new["mx"] ** 2 + new["my"] ** 2 + new["mz"] ** 2) / (2.0 * new["rho"])
    kap_gas = np.abs(new["E"] - new["e"] - K) * vol
    epsE = new["E"] - K
    take = epsE >= eta * new["E"]
    if record is not None:
        record["gas_take"] = take
        record["gas_margin"] = (epsE - eta * new["E"]) / np.abs(new["E"])
    e2 = np.where(take, epsE, new["e"])
    E2 = np.where(take, new["E"], new["e"] + K)
    new["e"], new["E"] = e2, E2

    nq = {i: new["q" + i] for i in DIRS}
    qq = {k: nq[k[0]] * nq[k[1]] / new["n"] for k in nE}
    PiE = {k: new["nE" + k] - qq[k] for k in nE}
    kap_bme = sum(np.abs(PiE[k] - new["P" + k]) for k in nE) * vol
    tr_PiE = PiE["xx"] + PiE["yy"] + PiE["zz"]
    tr_nE = new["nExx"] + new["nEyy"] + new["nEzz"]
    take = (tr_PiE >= eta * tr_nE) & (PiE["xx"] > 0.0) & (PiE["yy"] > 0.0) & (PiE["zz"] > 0.0)
    if record is not None:
        record["bme_take"] = take
        record["bme_trace_margin"] = (tr_PiE - eta * tr_nE) / np.abs(tr_nE)
        record["bme_diag_min"] = np.minimum(np.minimum(PiE["xx"], PiE["yy"]), PiE["zz"]) / np.abs(tr_nE)
    for k in nE:
        Pk = np.where(take, PiE[k], new["P" + k])
        nEk = np.where(take, new["nE" + k], new["P" + k] + qq[k])
        new["P" + k], new["nE" + k] = Pk, nEk
    return new, {"kappa_gas": kap_gas, "kappa_bme": kap_bme}


def _diagonal_mean(W):
    """Reading B of s1: the axis-d face velocity averaged over the four transverse
    diagonal neighbours of the face, (k +- 1, l +- 1) in the two tangent directions."""
    out = {}
    for d in DIRS:
        t1, t2 = _TANGENTS[d]
        acc = 0.0
        for a in (-1, 1):
            for b in (-1, 1):
                acc = acc + np.roll(np.roll(W[d], a, axis=_AXIS[t1]), b, axis=_AXIS[t2])
        out[d] = 0.25 * acc
    return out


def _wrap_take(a, idx, axis):
    return np.take(a, idx % a.shape[axis], axis=axis)


def _clamp_take(a, idx, axis):
    return np.take(a, np.clip(idx, 0, a.shape[axis] - 1), axis=axis)


def advance_window(st, phi, tau, prm: Params, *, zslab=None, cells=None):
    """``advance`` evaluated on part of a grid.

    The update of a cell depends only on cells within L1 distance 2 (faces of its
    neighbours), so a window with a margin of 2 reproduces it exactly: indices
    wrap on a periodic grid and clamp to the edge (ghost copies, s8) on an
    outflow grid.

    zslab=(k0, k1): returns the new state on planes k0..k1-1 (full x, y extent).
    cells=(S, 3) int array of (k, j, i): returns the new state at those cells, shape (S,).
    """
    outflow = prm.boundary == "outflow"
    take = _clamp_take if outflow else _wrap_take
    if zslab is not None:
        k0, k1 = zslab
        kk = np.arange(k0 - 2, k1 + 2)
        win = {f: take(st[f], kk, 0) for f in FIELDS}
        pw = take(phi, kk, 0)
        if outflow:
            # z already holds its ghost planes; x and y get theirs here
            pad = ((0, 0), (2, 2), (2, 2))
            win = {f: np.pad(a, pad, mode="edge") for f, a in win.items()}
            pw = np.pad(pw, pad, mode="edge")
            new, kap = advance(win, pw, tau, replace(prm, boundary="periodic"))
            return ({f: new[f][2:-2, 2:-2, 2:-2] for f in FIELDS},
                    {k: v[2:-2, 2:-2, 2:-2] for k, v in kap.items()})
        new, kap = advance(win, pw, tau, prm)
        return {f: new[f][2:-2] for f in FIELDS}, {k: v[2:-2] for k, v in kap.items()}
    cells = np.asarray(cells)
    off = np.arange(-2, 3)
    K = (cells[:, 0, None] + off)[:, :, None, None]
    J = (cells[:, 1, None] + off)[:, None, :, None]
    I = (cells[:, 2, None] + off)[:, None, None, :]

    def cut(a):
        nz, ny, nx = a.shape
        if outflow:
            return a[np.clip(K, 0, nz - 1), np.clip(J, 0, ny - 1), np.clip(I, 0, nx - 1)]
        return a[K % nz, J % ny, I % nx]

    win = {f: cut(st[f]) for f in FIELDS}
    new, kap = advance(win, cut(phi), tau, replace(prm, boundary="periodic"))
    return {f: new[f][:, 2, 2, 2] for f in FIELDS}, {k: v[:, 2, 2, 2] for k, v in kap.items()}


# --------------------------------------------------------------------------
# diagnostics (Sec. 2.4 and the conserved quantities of the cloud test)
# --------------------------------------------------------------------------
def _fsum(a):
    return math.fsum(np.asarray(a, dtype=np.float64).ravel().tolist())


def diagnostics(st, phi, prm: Params):
    """Exactly rounded sums over the grid of a state and its potential."""
    vol = prm.h ** 3
    rho, n = st["rho"], st["n"]
    out = {
        "mass_gas": _fsum(rho) * vol,
        "mass_bme": _fsum(n) * vol,
        "mom_x": _fsum(st["mx"] + st["qx"]) * vol,
        "mom_y": _fsum(st["my"] + st["qy"]) * vol,
        "mom_z": _fsum(st["mz"] + st["qz"]) * vol,
        "ekin_gas": _fsum((st["mx"] ** 2 + st["my"] ** 2 + st["mz"] ** 2) / (2.0 * rho)) * vol,
        "eint_gas": _fsum(st["e"]) * vol,
        "ekin_bme": _fsum((st["qx"] ** 2 + st["qy"] ** 2 + st["qz"] ** 2) / (2.0 * n)) * vol,
        "etherm_bme": _fsum(0.5 * (st["Pxx"] + st["Pyy"] + st["Pzz"])) * vol,
        "epot": 0.5 * _fsum((rho + n) * phi) * vol,
    }
    return out


def nonphysical(st):
    """True when a density, internal energy or diagonal stress is not positive or not finite."""
    bad = False
    for f in FIELDS:
        bad |= not np.all(np.isfinite(st[f]))
    for f in ("rho", "n", "e", "Pxx", "Pyy", "Pzz"):
        bad |= bool(np.any(st[f] <= 0.0))
    return bad


def step(st, prm: Params, dt=None):
    """One full step: Poisson (Sec. 2.3), tau, both fluids (Sec. 2.1-2.2), Sec. 2.4.

    Returns ``(new_state, record)``.  The record holds the diagnostics of the state
    at the start of the step (with its potential), kappa of the post-Lagrangian
    state, the step size used and the signal speed of the new state.
    """
    phi = solve_poisson(st, prm)
    tau = dt if (dt is not None and dt > 0.0) else cfl_dt(st, prm)
    rec = diagnostics(st, phi, prm)
    new, kap = advance(st, phi, tau, prm)
    rec["kappa_gas"] = _fsum(kap["kappa_gas"])
    rec["kappa_bme"] = _fsum(kap["kappa_bme"])
    rec["dt"] = tau
    rec["vmax"] = max_signal_speed(new, prm)
    rec["nonphysical"] = nonphysical(new)
    return new, rec


def run(st, prm: Params, nsteps, dt=None):
    """``nsteps`` consecutive steps; returns the final state and the list of records."""
    recs = []
    for _ in range(nsteps):
        st, rec = step(st, prm, dt)
        recs.append(rec)
    return st, recs
