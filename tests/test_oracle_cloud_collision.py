"""The paper's cloud collision test (Sec. 4.5) on the oracle, with isolated
gravity and outflow boundaries: pins that do not come from the oracle itself.

* Mass through the boundary: an outflow ghost cell copies the edge cell, so the
  face between them separates two equal states; the gas face solution of Sec.
  2.1 then gives the edge cell's velocity, the moment face solution of Sec. 2.2
  its u_n, and the Lagrangian flux of density through that face is the edge
  cell's momentum m_n (q_n) whichever side is upwind.  One step therefore
  changes the total mass by exactly -tau h^2 times the sum of the edge cells'
  outward m_n, a closed form that does not involve the scheme's interior (the
  background flows in through the x faces here, so it is not zero).
* Mirror symmetry: the collision is symmetric under x -> -x with x-odd
  components negated, so the state stays symmetric and the total x momentum
  stays zero to rounding.
"""
import numpy as np
import pytest

import oracle as O
from helpers import reflect_x
from paper_1311_0861_gb300 import inputs as I


def boundary_outflow(ax, ay, az):
    """Sum over the six faces of the box of the outward normal component (ax, ay,
    az along x, y, z) at the edge cells."""
    return (np.sum(ax[:, :, -1]) - np.sum(ax[:, :, 0]) + np.sum(ay[:, -1, :]) - np.sum(ay[:, 0, :])
            + np.sum(az[-1, :, :]) - np.sum(az[0, :, :]))


@pytest.mark.parametrize("N", [16, 24])
def test_mass_change_equals_boundary_flux(N):
    s = I.cloud_collision(N)
    prm = O.Params(h=s.h, gamma=s.gamma, poisson="isolated", boundary="outflow")
    st = s.state
    for _ in range(3):
        tau = O.cfl_dt(st, prm)
        new, _ = O.step(st, prm, dt=tau)
        h2 = s.h ** 2
        for dens, mom in (("rho", "m"), ("n", "q")):
            out = boundary_outflow(st[mom + "x"], st[mom + "y"], st[mom + "z"])
            m0 = np.sum(st[dens]) * s.h ** 3
            m1 = np.sum(new[dens]) * s.h ** 3
            want = -tau * h2 * out
            assert abs((m1 - m0) - want) <= 1e-12 * m0 + 1e-12 * abs(want), (dens, m1 - m0, want)
        st = new


def test_inflow_makes_the_mass_pin_nontrivial():
    s = I.cloud_collision(16)
    for mom in ("m", "q"):
        out = boundary_outflow(s.state[mom + "x"], s.state[mom + "y"], s.state[mom + "z"])
        assert out < -1e-3 * np.sum(np.abs(s.state[mom + "x"][:, :, 0]))   # inflow through both x faces


def test_collision_stays_mirror_symmetric():
    s = I.cloud_collision(24)
    prm = O.Params(h=s.h, gamma=s.gamma, poisson="isolated", boundary="outflow")
    a, _ = O.run(s.state, prm, 3)
    b = reflect_x(a)
    for f in O.FIELDS:
        scale = max(1e-300, np.max(np.abs(a[f])))
        assert np.max(np.abs(a[f] - b[f])) <= 1e-12 * scale, f
    assert abs(np.sum(a["mx"])) <= 1e-12 * np.sum(np.abs(a["mx"]))
