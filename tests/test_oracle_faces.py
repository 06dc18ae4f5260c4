"""Pins of the oracle's Eulerian face solutions (Sec. 2.1, Sec. 2.2).

Each closed form is compared with the Godunov state of the same linear system
built independently: the face state sum over waves of r_k (l_k . q_L) for
lambda_k > 0 and r_k (l_k . q_R) for lambda_k < 0 equals
(q_L + q_R)/2 + sign(A) (q_L - q_R)/2, with the matrix sign function
sign(A) = A |A|^-1 and |A| the principal square root of A^2 (scipy's sqrtm;
A^2 has positive eigenvalues, so this stays robust for the repeated shear
eigenvalues of the moment system).  For the gas, the small-jump limit is also
compared with the exact nonlinear Riemann solution.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1311_0861_gb300 import inputs as I

from exact_riemann import star_state


def godunov_linear(A, qL, qR):
    from scipy.linalg import sqrtm
    S = A @ np.linalg.inv(np.real(sqrtm(A @ A)))
    assert np.max(np.abs(S @ S - np.eye(len(qL)))) < 1e-10
    return 0.5 * (qL + qR) + 0.5 * S @ (qL - qR)


def _rand(seed, k):
    return I.uniform(seed, k)


def test_gas_face_is_linear_godunov_state():
    """(v, p) system of Sec. 2.1 frozen at harmonic-mean rho and arithmetic-mean p."""
    g = 1.4
    for t in range(200):
        u = _rand(100 + t, 6)
        rL, rR = 0.2 + 2 * u[0], 0.2 + 2 * u[1]
        vL, vR = u[2] - 0.5, u[3] - 0.5
        pL, pR = 0.1 + 3 * u[4], 0.1 + 3 * u[5]
        rho_star = 2 * rL * rR / (rL + rR)
        p_star = 0.5 * (pL + pR)
        A = np.array([[0.0, 1.0 / rho_star], [g * p_star, 0.0]])
        ref = godunov_linear(A, np.array([vL, pL]), np.array([vR, pR]))
        V, P = O.gas_face(rL, vL, pL, rR, vR, pR, g)
        assert abs(V - ref[0]) < 1e-13 and abs(P - ref[1]) < 1e-13 * max(1.0, abs(ref[1]))


def test_gas_face_matches_exact_riemann_for_small_jumps():
    """Error against the exact star state falls as the square of the jump."""
    g = 1.4
    errs = []
    for eps in (1e-2, 5e-3, 2.5e-3):
        rL, vL, pL = 1.0 + eps, 0.1 + 0.5 * eps, 1.0 + 2 * eps
        rR, vR, pR = 1.0, 0.1, 1.0
        ps, us = star_state(rL, vL, pL, rR, vR, pR, g)
        V, P = O.gas_face(rL, vL, pL, rR, vR, pR, g)
        errs.append(max(abs(V - us), abs(P - ps)))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


def bme_matrix(rho, a, b1, b2):
    """Sec. 2.2 matrix for (u_n, u_t1, u_t2, Pi_nn, Pi_nt1, Pi_nt2)."""
    A = np.zeros((6, 6))
    A[0, 3] = A[1, 4] = A[2, 5] = 1.0 / rho
    A[3, 0] = 3.0 * a
    A[4, 0], A[4, 1] = 2.0 * b1, a
    A[5, 0], A[5, 2] = 2.0 * b2, a
    return A


def test_bme_face_is_linear_godunov_state():
    for t in range(300):
        u = _rand(500 + t, 14)
        nL, nR = 0.2 + 2 * u[0], 0.2 + 2 * u[1]
        unL, unR = u[2] - 0.5, u[3] - 0.5
        t1L, t1R = u[4] - 0.5, u[5] - 0.5
        t2L, t2R = u[6] - 0.5, u[7] - 0.5
        PnnL, PnnR = 0.1 + 2 * u[8], 0.1 + 2 * u[9]
        P1L, P1R = 0.3 * (u[10] - 0.5), 0.3 * (u[11] - 0.5)
        P2L, P2R = 0.3 * (u[12] - 0.5), 0.3 * (u[13] - 0.5)
        A = bme_matrix(0.5 * (nL + nR), 0.5 * (PnnL + PnnR), 0.5 * (P1L + P1R), 0.5 * (P2L + P2R))
        qL = np.array([unL, t1L, t2L, PnnL, P1L, P2L])
        qR = np.array([unR, t1R, t2R, PnnR, P1R, P2R])
        ref = godunov_linear(A, qL, qR)
        got = np.array(O.bme_face(nL, unL, t1L, t2L, PnnL, P1L, P2L,
                                  nR, unR, t1R, t2R, PnnR, P1R, P2R))
        assert np.max(np.abs(got - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref))), (t, got, ref)


def test_bme_matrix_eigenvalues_are_printed_ones():
    """Sec. 2.2: eigenvalues +-sqrt(3 Pi_nn/rho) and +-sqrt(Pi_nn/rho) (twice)."""
    rho, a = 1.3, 0.7
    lam = np.sort(np.linalg.eigvals(bme_matrix(rho, a, 0.2, -0.1)).real)
    f, s = math.sqrt(3 * a / rho), math.sqrt(a / rho)
    assert np.allclose(lam, np.sort([f, -f, s, s, -s, -s]), atol=1e-12)


def test_bme_fast_block_is_gamma3_acoustics():
    """With equal L/R density the (u_n, Pi_nn) face values are the gas face values
    for gamma = 3 and p = Pi_nn (the fast subsystem is gamma = 3 gas dynamics)."""
    for t in range(50):
        u = _rand(900 + t, 5)
        n = 0.5 + u[0]
        unL, unR = u[1] - 0.5, u[2] - 0.5
        PL, PR = 0.2 + u[3], 0.2 + u[4]
        un, _, _, Pnn, _, _ = O.bme_face(n, unL, 0, 0, PL, 0, 0, n, unR, 0, 0, PR, 0, 0)
        V, P = O.gas_face(n, unL, PL, n, unR, PR, 3.0)
        assert abs(un - V) < 1e-14 and abs(Pnn - P) < 1e-14


def test_bme_face_tangent_symmetry():
    """Swapping the two tangents swaps the tangential outputs (normal ones unchanged)."""
    args = (1.1, 0.1, 0.2, -0.3, 0.9, 0.05, -0.07, 0.8, -0.2, 0.1, 0.4, 1.2, -0.02, 0.03)
    a = O.bme_face(*args)
    sw = list(args)
    for base in (0, 7):
        sw[base + 2], sw[base + 3] = sw[base + 3], sw[base + 2]
        sw[base + 5], sw[base + 6] = sw[base + 6], sw[base + 5]
    b = O.bme_face(*sw)
    assert np.allclose([a[0], a[1], a[2], a[3], a[4], a[5]], [b[0], b[2], b[1], b[3], b[5], b[4]],
                       rtol=0, atol=1e-15)
