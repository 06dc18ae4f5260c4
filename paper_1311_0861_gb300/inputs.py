"""Seeded synthetic initial states (host side, numpy float64).

This module holds no arithmetic of the numerical method: it only builds initial
states (densities, velocities, pressures, dispersion tensors) from closed-form
profiles and a counter-based random generator.  Both the CUDA path's tests and the
oracle's tests draw their inputs from here.

Random numbers come from splitmix64 used as a counter-based generator: draw k of
stream ``seed`` is ``mix(seed + (k + 1) * 0x9E3779B97F4A7C15)`` with Steele, Lea
and Flood's 64-bit finaliser; a uniform variate is its top 53 bits / 2**53 and a
normal variate uses the Box-Muller transform.

States are dicts of 22 float64 arrays of shape (N, N, N) indexed [k, j, i] (x
fastest), in the field order ``FIELDS``.  The box is [-1, 1]^3 with cell centres at
-1 + (i + 1/2) h, h = 2/N.  The galaxy recipes are the synthetic stand-ins for the
paper's collision runs (Sec. 5): a gas disc with circular rotation from the
enclosed mass plus a collisionless component with a velocity-dispersion tensor.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FIELDS = ("rho", "mx", "my", "mz", "E", "e",
          "n", "qx", "qy", "qz",
          "nExx", "nEyy", "nEzz", "nExy", "nExz", "nEyz",
          "Pxx", "Pyy", "Pzz", "Pxy", "Pxz", "Pyz")
NFIELDS = len(FIELDS)

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+count-1 of the splitmix64 stream ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """U[0, 1) variates from the top 53 bits."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def normal(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """N(0, 1) variates by Box-Muller from draw pairs (2k, 2k+1)."""
    u = uniform(seed, 2 * count, 2 * offset)
    u1 = 1.0 - u[0::2]          # in (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


@dataclass
class Setup:
    """An initial state plus the constants it was built for."""

    state: dict
    h: float
    gamma: float = 5.0 / 3.0
    G: float = 1.0
    courant: float = 0.2
    poisson: str = "periodic"
    name: str = ""
    info: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.state["rho"].shape


def grid(N: int):
    """Cell-centre coordinates (z, y, x) of the N^3 grid on [-1, 1]^3 and h."""
    h = 2.0 / N
    c = -1.0 + (np.arange(N) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return z, y, x, h


def _finish(rho, mx, my, mz, p, n, qx, qy, qz, P, gamma):
    """Builds the conserved 22-field state from primitive gas and moment fields.

    P is a dict of the 6 dispersion-tensor components (Pi_ij).
    """
    e = p / (gamma - 1.0)
    E = e + (mx * mx + my * my + mz * mz) / (2.0 * rho)
    st = {"rho": rho, "mx": mx, "my": my, "mz": mz, "E": E, "e": e,
          "n": n, "qx": qx, "qy": qy, "qz": qz}
    q = {"x": qx, "y": qy, "z": qz}
    for k in ("xx", "yy", "zz", "xy", "xz", "yz"):
        st["nE" + k] = P[k] + q[k[0]] * q[k[1]] / n
        st["P" + k] = P[k]
    return {f: np.ascontiguousarray(st[f], dtype=np.float64) for f in FIELDS}


# ---------------------------------------------------------------------------
# configuration 1: isolated self-gravitating sphere (32^3)
# ---------------------------------------------------------------------------
def sphere(N: int = 32, seed: int = 1, gamma: float = 5.0 / 3.0) -> Setup:
    """Gas sphere rho = 1/(1+(r/0.2)^2) cut at r = 0.8 (background 1e-3) with 1e-3
    uniform noise, p = 0.1 rho^gamma, at rest; collisionless component 0.5 x the
    unperturbed profile with isotropic dispersion 0.05."""
    z, y, x, h = grid(N)
    r = np.sqrt(x * x + y * y + z * z)
    prof = np.where(r <= 0.8, 1.0 / (1.0 + (r / 0.2) ** 2), 1e-3)
    U = uniform(seed, N ** 3).reshape(N, N, N)
    rho = prof * (1.0 + 1e-3 * (2.0 * U - 1.0))
    p = 0.1 * rho ** gamma
    zero = np.zeros_like(rho)
    n = 0.5 * prof
    P = {"xx": 0.05 * n, "yy": 0.05 * n, "zz": 0.05 * n, "xy": zero, "xz": zero, "yz": zero}
    st = _finish(rho, zero, zero, zero, p, n, zero, zero, zero, P, gamma)
    return Setup(st, h, gamma, name=f"sphere-{N}^3")


# ---------------------------------------------------------------------------
# the paper's cloud collision test (Sec. 4.5)
# ---------------------------------------------------------------------------
def cloud_collision(N: int = 32, half_width: float = 2.5, separation: float = 2.4, v_collide: float = 1.0,
                    gamma: float = 5.0 / 3.0) -> Setup:
    """Two copies of the hydrostatic gas sphere of Sec. 4.5 (rho = 1 - r inside
    r = 1 with the printed pressure p0(r) = -pi r^2 (9 r^2 - 28 r + 24)/36 + 5 pi/36,
    G = 1) centred at x = -+separation/2, approaching along x at relative speed
    v_collide (each at +-v_collide/2); background rho = 1e-3, p = 1e-5, moving
    with the nearer cloud.  The collisionless component is a cold passive tracer
    (n = 1e-6, Pi = 1e-12 I) with the gas velocity.  The box is
    [-half_width, half_width]^3 (isolated gravity and outflow boundaries are the
    intended settings)."""
    h = 2.0 * half_width / N
    c = -half_width + (np.arange(N) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    rho = np.full(x.shape, 1e-3)
    p = np.full(x.shape, 1e-5)
    for cx in (-0.5 * separation, 0.5 * separation):
        r = np.sqrt((x - cx) ** 2 + y * y + z * z)
        inside = r <= 1.0
        p0 = -np.pi * r * r * (9.0 * r * r - 28.0 * r + 24.0) / 36.0 + 5.0 * np.pi / 36.0
        rho = np.where(inside, np.maximum(1.0 - r, 1e-3), rho)
        p = np.where(inside, np.maximum(p0, 1e-5), p)
    vx = np.where(x < 0.0, 0.5 * v_collide, -0.5 * v_collide)
    zero = np.zeros_like(rho)
    n = np.full(x.shape, 1e-6)
    P = {"xx": 1e-12 + zero, "yy": 1e-12 + zero, "zz": 1e-12 + zero, "xy": zero, "xz": zero, "yz": zero}
    st = _finish(rho, rho * vx, zero, zero, p, n, n * vx, zero, zero, P, gamma)
    return Setup(st, h, gamma, poisson="isolated", name=f"cloud-collision-{N}^3")


# ---------------------------------------------------------------------------
# galaxy pieces
# ---------------------------------------------------------------------------
def _rot_y(theta):
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def _enclosed_mass(r, dens, h, rq):
    """M(<rq): mass of ``dens`` in cells whose centre lies within radius rq."""
    order = np.argsort(r, axis=None)
    rs = r.ravel()[order]
    cm = np.cumsum(dens.ravel()[order]) * h ** 3
    idx = np.searchsorted(rs, rq, side="left")
    return np.where(idx > 0, cm[np.maximum(idx - 1, 0)], 0.0)


def _galaxy(N, centre, mass, vel, incl_deg, rcut=0.35, sigma2=0.05):
    """One galaxy: exponential gas disc (scales 0.15, 0.02) rotating at the circular
    speed of its enclosed mass, plus a collisionless core 0.5/(1+(r/0.2)^2) with
    isotropic dispersion sigma2, both truncated at rcut and moving with ``vel``."""
    z, y, x, h = grid(N)
    rvec = np.stack([x - centre[0], y - centre[1], z - centre[2]])
    r = np.sqrt((rvec ** 2).sum(0))
    Rm = _rot_y(math.radians(incl_deg))          # disc frame -> box frame
    loc = np.tensordot(Rm.T, rvec, axes=1)        # box -> disc frame
    R = np.sqrt(loc[0] ** 2 + loc[1] ** 2)
    inside = r <= rcut
    rho_d = np.where(inside, mass * np.exp(-R / 0.15) * np.exp(-np.abs(loc[2]) / 0.02), 0.0)
    n_g = np.where(inside, mass * 0.5 / (1.0 + (r / 0.2) ** 2), 0.0)
    Menc = _enclosed_mass(r, rho_d + n_g, h, R)
    vc = np.sqrt(np.where(R > 0, Menc / np.maximum(R, 1e-300), 0.0))
    with np.errstate(invalid="ignore", divide="ignore"):
        phx = np.where(R > 0, -loc[1] / R, 0.0)
        phy = np.where(R > 0, loc[0] / R, 0.0)
    vloc = np.stack([vc * phx, vc * phy, np.zeros_like(vc)])
    vrot = np.tensordot(Rm, vloc, axes=1)
    vgas = vrot + np.asarray(vel)[:, None, None, None]
    return rho_d, vgas, n_g, sigma2


def collision(N: int = 256, seed: int = 3, *, centres=((-0.4, 0.0, 0.0), (0.4, 0.0, 0.0)),
              masses=(1.0, 0.7), speed=0.5, incl=(30.0, 30.0), sigma2=0.05,
              gamma=5.0 / 3.0, poisson="periodic", name=None) -> Setup:
    """Two galaxies approaching along x at relative speed ``speed`` in their
    centre-of-mass frame (total momentum zero), discs inclined about y."""
    z, y, x, h = grid(N)
    mA, mB = masses
    vA = np.array([speed * mB / (mA + mB), 0.0, 0.0])
    vB = np.array([-speed * mA / (mA + mB), 0.0, 0.0])
    rho = np.full((N, N, N), 1e-3)
    m = np.zeros((3, N, N, N))
    n = np.full((N, N, N), 5e-4)
    q = np.zeros((3, N, N, N))
    for c, mass, v, inc in ((centres[0], mA, vA, incl[0]), (centres[1], mB, vB, incl[1])):
        rho_d, vgas, n_g, s2 = _galaxy(N, c, mass, v, inc, sigma2=sigma2)
        rho += rho_d
        m += rho_d * vgas
        n += n_g
        q += n_g * v[:, None, None, None]
    pert = np.exp(1e-3 * normal(seed, N ** 3).reshape(N, N, N))
    rho_p = rho * pert
    m *= pert
    p = 1e-2 * rho_p ** gamma
    zero = np.zeros_like(rho)
    P = {"xx": sigma2 * n, "yy": sigma2 * n, "zz": sigma2 * n, "xy": zero, "xz": zero, "yz": zero}
    st = _finish(rho_p, m[0], m[1], m[2], p, n, q[0], q[1], q[2], P, gamma)
    return Setup(st, h, gamma, poisson=poisson, name=name or f"collision-{N}^3")


def head_on(N: int = 256, seed: int = 3) -> Setup:
    """Two-galaxy head-on collision: mass ratio 1:0.7, centres +-0.4 on x,
    approach speed 0.5, discs inclined 30 degrees."""
    return collision(N, seed, name=f"head-on collision {N}^3")


def off_axis(N: int = 512, seed: int = 5) -> Setup:
    """Off-axis collision: impact parameter 0.2, ratio 1:1, inclinations +45/-20
    degrees, isotropic dispersion 0.05, isolated gravity."""
    return collision(N, seed, centres=((-0.4, -0.1, 0.0), (0.4, 0.1, 0.0)), masses=(1.0, 1.0),
                     incl=(45.0, -20.0), poisson="isolated", name=f"off-axis collision {N}^3")


def disc(N: int = 128, seed: int = 2, gamma=5.0 / 3.0) -> Setup:
    """Single rotating disc galaxy: exponential gas disc (floor 1e-3, 1e-3
    lognormal noise) in circular rotation, p = 1e-2 rho^gamma, inside a capped
    NFW-like collisionless halo with dispersions (R, phi, z) = (0.03, 0.02, 0.03)."""
    z, y, x, h = grid(N)
    r = np.sqrt(x * x + y * y + z * z)
    R = np.sqrt(x * x + y * y)
    rho_d = np.maximum(np.exp(-R / 0.15) * np.exp(-np.abs(z) / 0.02), 1e-3)
    rho = rho_d * np.exp(1e-3 * normal(seed, N ** 3).reshape(N, N, N))
    rs = np.maximum(r / 0.1, 1e-300)
    n = np.minimum(1e3, 1.0 / (rs * (1.0 + rs) ** 2))
    Menc = _enclosed_mass(r, rho + n, h, R)
    vc = np.sqrt(np.where(R > 0, Menc / np.maximum(R, 1e-300), 0.0))
    with np.errstate(invalid="ignore", divide="ignore"):
        cph = np.where(R > 0, x / R, 1.0)
        sph = np.where(R > 0, y / R, 0.0)
    mx, my, mz = -rho * vc * sph, rho * vc * cph, np.zeros_like(rho)
    p = 1e-2 * rho ** gamma
    sR, sP, sZ = 0.03, 0.02, 0.03
    P = {"xx": n * (sR * cph ** 2 + sP * sph ** 2),
         "yy": n * (sR * sph ** 2 + sP * cph ** 2),
         "zz": n * sZ * np.ones_like(n),
         "xy": n * (sR - sP) * cph * sph,
         "xz": np.zeros_like(n), "yz": np.zeros_like(n)}
    zero = np.zeros_like(rho)
    st = _finish(rho, mx, my, mz, p, n, zero, zero, zero, P, gamma)
    return Setup(st, h, gamma, name=f"disc galaxy {N}^3")


def ensemble_member(r: int) -> Setup:
    """Run r of the 64-run ensemble: N drawn from {32, 48, 64, 96}; impact
    parameter U[0, 0.3] in y, mass ratio U[0.3, 1], inclination U[0, 90] degrees,
    approach speed U[0.3, 0.8]."""
    seed = 4000 + r
    u = uniform(seed, 6, offset=0)
    N = (32, 48, 64, 96)[min(int(u[0] * 4), 3)]
    b = 0.3 * u[1]
    ratio = 0.3 + 0.7 * u[2]
    inc = 90.0 * u[3]
    spd = 0.3 + 0.5 * u[4]
    return collision(N, seed + 100000, centres=((-0.4, -0.5 * b, 0.0), (0.4, 0.5 * b, 0.0)),
                     masses=(1.0, ratio), speed=spd, incl=(inc, -inc),
                     name=f"ensemble run {r} ({N}^3)")


# ---------------------------------------------------------------------------
# generic smooth / rough random states for parity and symmetry tests
# ---------------------------------------------------------------------------
def _smooth_field(shape, seed, nmodes=6, kmax=3):
    """Sum of a few random low-wavenumber periodic cosines, scaled to [-1, 1]."""
    nz, ny, nx = shape
    u = uniform(seed, nmodes * 5)
    k = np.arange(nz)[:, None, None] / nz, np.arange(ny)[None, :, None] / ny, np.arange(nx)[None, None, :] / nx
    f = np.zeros(shape)
    for m in range(nmodes):
        kz, ky, kx = (np.floor(u[5 * m + i] * (2 * kmax + 1)) - kmax for i in range(3))
        ph = 2.0 * np.pi * u[5 * m + 3]
        amp = 0.5 + 0.5 * u[5 * m + 4]
        f = f + amp * np.cos(2.0 * np.pi * (kz * k[0] + ky * k[1] + kx * k[2]) + ph)
    mx = np.max(np.abs(f))
    return f / mx if mx > 0 else f


def random_state(shape, seed: int = 7, rough: bool = False, gamma=5.0 / 3.0, box=2.0) -> Setup:
    """A valid random state: rho, p, n in [0.5, 1.5], velocities in [-0.3, 0.3],
    diagonally dominant dispersion tensors.  ``rough`` uses independent per-cell
    values (every face is a jump); otherwise smooth periodic modes."""
    shape = tuple(shape)
    cnt = int(np.prod(shape))

    def fld(i):
        if rough:
            return 2.0 * uniform(seed * 1000 + i, cnt).reshape(shape) - 1.0
        return _smooth_field(shape, seed * 1000 + i)

    rho = 1.0 + 0.5 * fld(0)
    v = [0.3 * fld(1 + d) for d in range(3)]
    p = 1.0 + 0.5 * fld(4)
    n = 1.0 + 0.5 * fld(5)
    u = [0.3 * fld(6 + d) for d in range(3)]
    P = {"xx": n * (0.6 + 0.2 * fld(9)), "yy": n * (0.6 + 0.2 * fld(10)),
         "zz": n * (0.6 + 0.2 * fld(11)), "xy": n * 0.1 * fld(12),
         "xz": n * 0.1 * fld(13), "yz": n * 0.1 * fld(14)}
    st = _finish(rho, rho * v[0], rho * v[1], rho * v[2], p, n, n * u[0], n * u[1], n * u[2], P, gamma)
    h = box / shape[-1]
    return Setup(st, h, gamma, name=f"random{'-rough' if rough else ''} {shape}")


def stack(state, dtype=np.float64) -> np.ndarray:
    """(22, Nz, Ny, Nx) contiguous array in field order."""
    return np.ascontiguousarray(np.stack([state[f] for f in FIELDS]).astype(dtype, copy=False))


def unstack(arr) -> dict:
    return {f: np.asarray(arr[i], dtype=np.float64) for i, f in enumerate(FIELDS)}
