"""The cooling placeholder of the gas energy equations (Sec. 2, reading s13):
q = Lambda rho^2 sqrt(eps), subtracted from E and e in the Eulerian stage.

Pins that do not come from the oracle:
* a uniform gas at rest has no fluxes, so e obeys de/dt = -Lambda rho^(3/2) e^(1/2),
  whose exact solution is sqrt(e(t)) = sqrt(e0) - Lambda rho^(3/2) t / 2; the
  explicit step converges to it at first order in the step size;
* a uniform moving gas loses the same energy from E and e, so E - e (the
  kinetic energy) is unchanged and the state stays uniform;
* Lambda = 0 is the adiabatic step exactly.
"""
import math

import numpy as np

import oracle as O
from helpers import state_from_primitives, TENSOR
from paper_1311_0861_gb300 import inputs as I


def uniform(N, rho, v, p, gamma=5.0 / 3.0):
    one = np.ones((N, N, N))
    P = {k: (0.3 * one if k[0] == k[1] else 0.0 * one) for k in TENSOR}
    return state_from_primitives(rho * one, tuple(vd * one for vd in v), p * one, 0.5 * one,
                                 (0 * one, 0 * one, 0 * one), P, gamma)


def test_uniform_decay_converges_to_exact_solution():
    N, rho, p, lam, T = 4, 1.3, 0.8, 0.7, 0.4
    gamma = 5.0 / 3.0
    e0 = p / (gamma - 1.0)
    exact = (math.sqrt(e0) - lam * rho ** 1.5 * T / 2.0) ** 2
    errs = []
    for nsteps in (20, 40, 80):
        st = uniform(N, rho, (0.0, 0.0, 0.0), p)
        prm = O.Params(h=2.0 / N, G=0.0, cooling=lam)
        st, _ = O.run(st, prm, nsteps, dt=T / nsteps)
        assert np.ptp(st["e"]) == 0.0 and np.ptp(st["rho"]) == 0.0
        errs.append(abs(st["e"][0, 0, 0] - exact))
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2, errs
    assert errs[2] < 2e-3 * exact


def test_moving_gas_keeps_its_kinetic_energy():
    N = 4
    st = uniform(N, 0.9, (0.3, -0.2, 0.1), 0.6)
    prm = O.Params(h=2.0 / N, G=0.0, cooling=0.5)
    new, _ = O.step(st, prm, dt=0.01)
    K = 0.5 * 0.9 * (0.3 ** 2 + 0.2 ** 2 + 0.1 ** 2)
    assert np.allclose(new["E"] - new["e"], K, rtol=1e-13, atol=0)
    assert np.all(new["e"] < st["e"])
    for f in ("rho", "mx", "my", "mz"):
        assert np.allclose(new[f], st[f], rtol=1e-15, atol=1e-16)


def test_zero_lambda_is_the_adiabatic_step():
    s = I.random_state((8, 8, 8), seed=3, rough=True)
    a, _ = O.step(s.state, O.Params(h=s.h))
    b, _ = O.step(s.state, O.Params(h=s.h, cooling=0.0))
    for f in O.FIELDS:
        assert np.array_equal(a[f], b[f])
