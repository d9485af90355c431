"""Pins of the oracle's implicit pseudo-time step (Sect. 2.1: backward Euler
with local time steps, linearised once) and of its local time step."""
import math

import numpy as np
import pytest

import coronal_inputs as ci
import oracle
from _util import oracle_grid, problem


def fast_speed(rho, p, B, n, gamma):
    """Textbook fast magnetosonic speed along the unit normal n."""
    a2 = gamma * p / rho
    b2 = np.dot(B, B) / rho
    bn2 = np.dot(B, n) ** 2 / rho
    return math.sqrt(0.5 * (a2 + b2 + math.sqrt((a2 + b2) ** 2 - 4 * a2 * bn2)))


def test_local_dt_uniform_box():
    """Uniform state in a periodic box: dt = V / sum_f (|u.n| + c_f) |S_f| with
    two faces per axis of area h_j h_k (c_h small enough not to matter)."""
    L = (1.0, 2.0, 0.5)
    g = oracle.box(3, 4, 5, lengths=L, c_h=0.01)
    rho, V, B, p = 1.3, np.array([0.4, -0.7, 0.2]), np.array([0.5, 0.3, -0.9]), 0.8
    W = np.zeros((9,) + g.shape)
    W[0], W[7] = rho, p
    W[1:4] = V[:, None, None, None]
    W[4:7] = B[:, None, None, None]
    U = ci.prim_to_cons(W, g.gamma)
    h = [L[a] / g.shape[a] for a in range(3)]
    vol = h[0] * h[1] * h[2]
    s = 0.0
    for a in range(3):
        n = np.eye(3)[a]
        area = vol / h[a]
        s += 2 * (abs(V[a]) + fast_speed(rho, p, B, n, g.gamma)) * area
    np.testing.assert_allclose(oracle.local_dt(g, U), vol / s, rtol=1e-14)


def test_local_dt_static_unmagnetised_shell():
    """V = 0, B = 0 on the shell: every face has lambda = max(a, c_h), so dt_c =
    V_c / (lambda sum_f |S_f|), the face areas from the oracle's geometry."""
    shape = (5, 6, 8)
    g = oracle_grid(shape, c_h=0.3)
    W = np.zeros((9,) + shape)
    W[0] = 1.0 + np.linspace(0, 1, shape[0])[:, None, None]
    W[7] = 0.2
    U = ci.prim_to_cons(W, g.gamma)
    vol, S0, S1, S2 = oracle.geometry(g)
    a = lambda v: np.linalg.norm(v, axis=-1)
    area = a(S0[:-1]) + a(S0[1:]) + a(S1[:, :-1]) + a(S1[:, 1:]) + a(S2[:, :, :-1]) + a(S2[:, :, 1:])
    lam = np.maximum(np.sqrt(g.gamma * W[7] / W[0]), 0.3)
    np.testing.assert_allclose(oracle.local_dt(g, U), vol / (lam * area), rtol=1e-13)


def test_backward_euler_small_cfl_expansion():
    """(D/c - J) dU = R with D = diag(1/dt) gives dU = c dt R + c dt J (c dt R)
    + O(c^3): the first-order error falls 4x and the second-order error 8x per
    halving of c (pins the sign of J and the per-cell scaling of the shift)."""
    shape = (4, 4, 8)
    U, Br = problem(shape, perturb=3)
    g = oracle_grid(shape)
    J = oracle.jacobian(g, U, Br)
    dt = np.broadcast_to(oracle.local_dt(g, U), U.shape)
    R = oracle.residual(g, U, Br)["R"]
    e1, e2 = [], []
    for c in (1e-3, 5e-4, 2.5e-4):
        dU, R2 = oracle.backward_euler_step(g, U, Br, c, J=J)
        assert np.array_equal(R2, R)
        first = c * dt * R
        second = first + c * dt * oracle.residual_jvp(g, U, Br, first, np.zeros_like(Br))[1]
        e1.append(np.linalg.norm(dU - first))
        e2.append(np.linalg.norm(dU - second))
    assert 3.7 < e1[0] / e1[1] < 4.3 and 3.7 < e1[1] / e1[2] < 4.3
    assert 7.0 < e2[0] / e2[1] < 9.0 and 7.0 < e2[1] / e2[2] < 9.0


def test_backward_euler_dense_and_gmres_agree():
    shape = (4, 4, 8)
    for bc in ({}, dict(inner_bc="low_e_wp", vr_star=1935.07 / ci.V_REF)):
        U, Br = problem(shape, perturb=5)
        g = oracle_grid(shape, **bc)
        a, _ = oracle.backward_euler_step(g, U, Br, 20.0, solver="dense")
        b, _ = oracle.backward_euler_step(g, U, Br, 20.0, solver="gmres", rtol=1e-13)
        assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(a)


def test_backward_euler_keeps_a_free_stream():
    """A uniform field-aligned flow in a periodic box has R = 0, so dU = 0."""
    g = oracle.box(4, 4, 4)
    W = np.zeros((9,) + g.shape)
    W[0], W[7] = 1.0, 0.6
    W[1:4] = np.array([0.3, 0.2, -0.1])[:, None, None, None]
    W[4:7] = 2.0 * W[1:4]
    U = ci.prim_to_cons(W, g.gamma)
    dU, R = oracle.backward_euler_step(g, U, None, 50.0)
    assert np.abs(R).max() < 1e-14
    assert np.abs(dU).max() < 1e-12


def test_backward_euler_large_cfl_is_newton():
    """As the CFL grows the step tends to the Newton step -J^-1 R."""
    shape = (4, 4, 8)
    U, Br = problem(shape, perturb=3)
    g = oracle_grid(shape, inner_bc="low_e_wp", vr_star=1935.07 / ci.V_REF)
    J = oracle.jacobian(g, U, Br)
    R = oracle.residual(g, U, Br)["R"]
    newton = np.linalg.solve(-J, R.ravel()).reshape(U.shape)
    d1, _ = oracle.backward_euler_step(g, U, Br, 1e6, J=J)
    d2, _ = oracle.backward_euler_step(g, U, Br, 2e6, J=J)
    e1, e2 = np.linalg.norm(d1 - newton), np.linalg.norm(d2 - newton)
    assert e1 < 1e-3 * np.linalg.norm(newton)
    assert 1.8 < e1 / e2 < 2.2      # first order in 1/CFL


def test_steady_sensitivity_matches_finite_differences_of_steady_states():
    """dg = -gbar . J^-1 (dR/dB dB) at a steady state R(U*, B) = 0 against
    (g(U*(B + e dB)) - g(U*(B - e dB))) / 2e, the steady states found by
    pseudo-transient continuation (backward-Euler steps, Sect. 2.1) and
    polished by Newton with the dense Jacobian (6 x 6 x 12 shell, low-E with
    the V_r* magnitude, dipole; g = mean outer-layer density)."""
    shape = (6, 6, 12)
    g = oracle_grid(shape, inner_bc="low_e_wp", vr_star=1935.07 / ci.V_REF)
    U, info = ci.background(*shape)
    Br = ci.magnetogram(6, 12, dipole_only=True)
    gm1 = g.gamma - 1.0

    def newton(U, Br, steps):
        for _ in range(steps):
            R = oracle.residual(g, U, Br)["R"]
            U = U + np.linalg.solve(oracle.jacobian(g, U, Br), -R.ravel()).reshape(U.shape)
        return U

    cfl, r0 = 2.0, None
    for it in range(150):
        if it and it % 10 == 0:
            cfl = min(2 * cfl, 128.0)
        dU, R = oracle.backward_euler_step(g, U, Br, cfl, solver="gmres", rtol=1e-4)
        r0 = r0 or np.linalg.norm(R)
        if np.linalg.norm(R) < 1e-6 * r0:
            break
        W = oracle.cons_to_prim(g, U)
        rho, V, B, p = W[0], W[1:4], W[4:7], W[7]
        dp = gm1 * (dU[7] - np.sum(V * dU[1:4], 0) + 0.5 * np.sum(V * V, 0) * dU[0] - np.sum(B * dU[4:7], 0))
        U = U + min(1.0, 0.3 / max(np.max(np.abs(dU[0]) / rho), np.max(np.abs(dp) / p))) * dU
    U = newton(U, Br, 4)
    assert np.linalg.norm(oracle.residual(g, U, Br)["R"]) < 1e-12
    gbar = np.zeros_like(U)
    gbar[0, -1] = 1.0 / (6 * 12)
    dB = np.random.default_rng(1).standard_normal(Br.shape)
    s = oracle.steady_sensitivity(g, U, Br, gbar, dB, rtol=1e-11)
    e = 1e-5
    fd = (np.sum(gbar * newton(U, Br + e * dB, 2)) - np.sum(gbar * newton(U, Br - e * dB, 2))) / (2 * e)
    assert abs(fd - s) <= 1e-5 * abs(s)
