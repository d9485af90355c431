"""Pins of the oracle's boundary variants against the paper's statements:
every outer law of Table 2 (Sect. 4.1) and the rho ~ r^-2.5 law (Sect. 4.2),
the large-E (Wind-Predict) inner formulation of Sect. 3.2, and the contrast
of the boundary electric field between the two inner formulations."""
import json
import math
import os

import numpy as np
import pytest

import coronal_inputs as ci
import oracle
from _util import oracle_grid, problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def table2():
    with open(os.path.join(GOLDEN, "table2_outer_bc.json")) as f:
        return json.load(f)["cases"]


def laws_to_params(case):
    """Table 2 row -> oracle outer-law parameters."""
    rho = float(case["rho"])
    # p follows rho in every row; "B=I" (case 1) is the zero-gradient law, i.e. exponent 0 like rho there
    assert case["p"] == rho or (case["p"] == "B=I" and rho == 0)
    return dict(outer_rho_exp=rho, outer_br_exp=float(case["Br"]), outer_bphi_exp=float(case["Bphi"]),
                outer_vr_mass=case["Vr"] == "mass", outer_vphi_exp=float(case["Vphi"]),
                outer_psi_extrap=case["psi"] == "G=I")


def spherical(W, g):
    _, tc, pc = ci.cell_centres(*g.shape)
    T, P = np.meshgrid(tc, pc, indexing="ij")
    er = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)])
    et = np.stack([np.cos(T) * np.cos(P), np.cos(T) * np.sin(P), -np.sin(T)])
    ep = np.stack([-np.sin(P), np.cos(P), np.zeros_like(P)])
    V, B = W[1:4], W[4:7]
    dot = lambda a, e: np.einsum("cji,cji->ji", a, e)
    return ({"r": dot(V, er), "t": dot(V, et), "p": dot(V, ep)},
            {"r": dot(B, er), "t": dot(B, et), "p": dot(B, ep)}, (er, et, ep))


@pytest.mark.parametrize("case", [str(c) for c in range(1, 10)])
def test_outer_ghost_follows_table2(case):
    """Each Table 2 row, law by law, with G the ghost and I the last interior
    cell at radii r_G = 2 r_out - r_I and r_I."""
    law = table2()[case]
    g = oracle_grid((6, 6, 8), **laws_to_params(law))
    U, info = ci.background(*g.shape)
    U = ci.perturb(info["W"], seed=int(case), amp=0.2)
    Br = ci.magnetogram(g.n_theta, g.n_phi, dipole_only=True)
    _, Wout = oracle.ghosts(g, U, Br)
    WI = oracle.cons_to_prim(g, U)[:, -1]
    rf = ci.radial_faces(g.n_r)
    rI = 0.5 * (rf[-2] + rf[-1])
    rG = 2 * g.r_out - rI
    VI, BI, _ = spherical(WI, g)
    VG, BG, _ = spherical(Wout, g)
    tol = dict(rtol=1e-12, atol=1e-15)
    if law["rho"] == 0:
        np.testing.assert_allclose(Wout[0], WI[0], **tol)
    else:
        np.testing.assert_allclose(Wout[0] * rG ** law["rho"], WI[0] * rI ** law["rho"], **tol)
    if law["p"] == "B=I":    # boundary value = interior value: mirrored ghost = I
        np.testing.assert_allclose(Wout[7], WI[7], **tol)
    else:
        np.testing.assert_allclose(Wout[7] * rG ** law["p"], WI[7] * rI ** law["p"], **tol)
    np.testing.assert_allclose(BG["r"] * rG ** law["Br"], BI["r"] * rI ** law["Br"], **tol)
    np.testing.assert_allclose(BG["t"], BI["t"], **tol)
    np.testing.assert_allclose(BG["p"] * rG ** law["Bphi"], BI["p"] * rI ** law["Bphi"], **tol)
    if law["Vr"] == "mass":  # V_r r^2 rho = const
        np.testing.assert_allclose(VG["r"] * rG ** 2 * Wout[0], VI["r"] * rI ** 2 * WI[0], **tol)
    else:
        np.testing.assert_allclose(VG["r"], VI["r"], **tol)
    np.testing.assert_allclose(VG["t"], VI["t"], **tol)
    np.testing.assert_allclose(VG["p"] * rG ** law["Vphi"], VI["p"] * rI ** law["Vphi"], **tol)
    if law["psi"] == "B=0":
        np.testing.assert_allclose(Wout[8] + WI[8], 0.0, atol=1e-17)
    else:
        np.testing.assert_allclose(Wout[8], WI[8], **tol)


def test_outer_density_law_r_minus_2_5():
    """Sect. 4.2: rho (and p) extended as r^-2.5."""
    g = oracle_grid((6, 6, 8), outer_rho_exp=2.5)
    U, info = ci.background(*g.shape)
    _, Wout = oracle.ghosts(g, U, ci.magnetogram(6, 8, dipole_only=True))
    WI = oracle.cons_to_prim(g, U)[:, -1]
    rf = ci.radial_faces(g.n_r)
    rI = 0.5 * (rf[-2] + rf[-1])
    rG = 2 * g.r_out - rI
    np.testing.assert_allclose(Wout[0] * rG ** 2.5, WI[0] * rI ** 2.5, rtol=1e-12)


def test_large_e_inner_boundary_equations():
    """The Wind-Predict form of Sect. 3.2 at the face: B_r, B_theta prescribed,
    V_par = V_r* B_r / B_pol^2, V_r = V_par B_r, V_theta = V_par B_theta,
    V_phi = 0; B_phi Neumann; psi_b = 0."""
    vr_star = 1935.07 / ci.V_REF
    g = oracle_grid((4, 12, 16), inner_bc="large_e", vr_star=vr_star, rho_b=1.0, p_b=0.2)
    U, info = ci.background(*g.shape)
    U = ci.perturb(info["W"], seed=2, amp=0.2)
    Bb = ci.potential_field(g.n_theta, g.n_phi, lmax=6, seed=17)
    Win, _ = oracle.ghosts(g, U, Bb)
    WI = oracle.cons_to_prim(g, U)[:, 0]
    V, B, _ = spherical(0.5 * (Win + WI), g)
    _, BI, _ = spherical(WI, g)
    br, bt = Bb
    vpar = vr_star * br / (br ** 2 + bt ** 2)
    np.testing.assert_allclose(B["r"], br, atol=1e-14)
    np.testing.assert_allclose(B["t"], bt, atol=1e-14)
    np.testing.assert_allclose(B["p"], BI["p"], atol=1e-14)
    np.testing.assert_allclose(V["r"], vpar * br, rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(V["t"], vpar * bt, rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(V["p"], 0.0, atol=1e-18)
    np.testing.assert_allclose(0.5 * (Win[8] + WI[8]), 0.0, atol=1e-17)
    assert np.all(Win[0] == 1.0) and np.all(Win[7] == 0.2)


def test_boundary_electric_field_low_vs_large_e():
    """E = -V_b x B_b at the inner faces: zero (to round-off) for the low-E
    formulation, and non-zero wherever B_phi differs from zero for the large-E
    one (V_b is poloidal there, B_b keeps the interior B_phi)."""
    shape = (4, 12, 16)
    U, info = ci.background(*shape)
    U = ci.perturb(info["W"], seed=4, amp=0.2)
    Bb = ci.potential_field(shape[1], shape[2], lmax=6, seed=17)
    low = oracle_grid(shape)
    large = oracle_grid(shape, inner_bc="large_e", vr_star=1935.07 / ci.V_REF)
    E_low = oracle.boundary_efield(low, U, Bb[0])
    E_large = oracle.boundary_efield(large, U, Bb)
    Win, _ = oracle.ghosts(low, U, Bb[0])
    WI = oracle.cons_to_prim(low, U)[:, 0]
    Wb = 0.5 * (Win + WI)
    scale = np.linalg.norm(Wb[1:4], axis=0) * np.linalg.norm(Wb[4:7], axis=0)
    assert np.max(np.linalg.norm(E_low, axis=0) / scale) < 1e-14
    assert np.median(np.linalg.norm(E_large, axis=0)) > 1e3 * np.max(np.linalg.norm(E_low, axis=0))


def test_potential_field_generator():
    """B_theta of the potential field: sin(theta)/2 for the dipole; for one
    quadrupole harmonic the closed form of -dY_20/dtheta / 3."""
    _, tc, pc = ci.cell_centres(2, 8, 16)
    d = ci.potential_field(8, 16, dipole_only=True)
    np.testing.assert_allclose(d[1], 0.5 * np.sin(tc)[:, None] * np.ones((1, 16)), atol=1e-15)
    T, P = np.meshgrid(tc, pc, indexing="ij")
    ys = dict(((l, m), Y) for l, m, Y in ci.real_sh(2, T, P))
    c20 = math.sqrt(5 / (16 * math.pi))
    np.testing.assert_allclose(ys[(2, 0)], c20 * (3 * np.cos(T) ** 2 - 1), atol=1e-14)
    hi = dict(((l, m), Y) for l, m, Y in ci.real_sh(2, T + 1e-6, P))
    lo = dict(((l, m), Y) for l, m, Y in ci.real_sh(2, T - 1e-6, P))
    num = (hi[(2, 0)] - lo[(2, 0)]) / 2e-6
    np.testing.assert_allclose(num, -6 * c20 * np.cos(T) * np.sin(T), atol=1e-8)


@pytest.mark.parametrize("variant", ["large_e", "case9", "low_e_wp"])
def test_jvp_of_boundary_variants(variant):
    """The dual-number JVP through the new ghost maps against central
    differences (unlimited reconstruction, h = 1e-8; B_r and B_theta perturbed)."""
    kw = dict(limiter="none", r_out=3.0)
    if variant in ("large_e", "low_e_wp"):
        kw.update(inner_bc=variant, vr_star=1935.07 / ci.V_REF)
    else:
        kw.update(laws_to_params(table2()["9"]))
    g = oracle_grid((6, 6, 8), **kw)
    U, info = ci.background(*g.shape, r_out=3.0)
    U = ci.perturb(info["W"], seed=6, amp=0.02)
    Bb = ci.potential_field(6, 8, lmax=3, seed=2)
    if variant != "large_e":
        Bb = Bb[0]
    rng = np.random.default_rng(7)
    dU = rng.standard_normal(U.shape) * (np.abs(U) + 1e-3)
    dB = rng.standard_normal(Bb.shape)
    _, Jv = oracle.residual_jvp(g, U, Bb, dU, dB)
    h = 1e-8
    fd = (oracle.residual(g, U + h * dU, Bb + h * dB)["R"] - oracle.residual(g, U - h * dU, Bb - h * dB)["R"]) / (2 * h)
    for v in range(9):
        assert np.linalg.norm(fd[v] - Jv[v]) <= 1e-5 * np.linalg.norm(Jv[v]) + 1e-12, v


def test_thin_last_cell_mesh():
    """The Sect. 4.3 mesh (r_out = 25, last cell [r_last, r_out]): the cell
    volumes still add up to the shell's (4 pi / 3)(r_out^3 - r_in^3), the last
    cell has the prescribed thickness, the faces below r_last are geometric,
    and the outer ghost obeys its law at the mirrored radius 2 r_out - r_I."""
    r_last, r_out = 24.95, 25.0
    g = oracle_grid((12, 6, 8), r_out=r_out, r_last=r_last)
    vol, S0, _, _ = oracle.geometry(g)
    assert vol.sum() == pytest.approx(4 * math.pi / 3 * (r_out ** 3 - 1.0), rel=1e-13)
    shell_r = np.sqrt(np.abs(S0).sum(axis=(1, 2, 3)) / np.abs(S0).sum(axis=(1, 2, 3))[0])
    # |S| of a full radial face layer grows as r^2 (sum of |S_x|+|S_y|+|S_z| scales alike)
    np.testing.assert_allclose(shell_r[-1], r_out, rtol=1e-12)
    np.testing.assert_allclose(shell_r[-2], r_last, rtol=1e-12)
    ratio = shell_r[1:-1] / shell_r[:-2]
    np.testing.assert_allclose(ratio, (r_last / 1.0) ** (1.0 / 11), rtol=1e-12)
    np.testing.assert_allclose(np.sum(vol, axis=(1, 2))[-1],
                               4 * math.pi / 3 * (r_out ** 3 - r_last ** 3), rtol=1e-12)
    U, info = ci.background(*g.shape, r_out=r_out, r_last=r_last)
    _, Wout = oracle.ghosts(g, U, ci.magnetogram(6, 8, dipole_only=True))
    WI = oracle.cons_to_prim(g, U)[:, -1]
    rI = 0.5 * (r_last + r_out)
    rG = 2 * r_out - rI
    np.testing.assert_allclose(Wout[0] * rG ** 2, WI[0] * rI ** 2, rtol=1e-12)
    np.testing.assert_allclose(ci.radial_faces(12, 1.0, r_out, r_last)[-2:], [r_last, r_out])


def test_volume_efield_closed_form():
    """E = -V x B per cell.  Radial Parker wind V = v r_hat through the dipole
    (B_r = cos t / r^3, B_theta = sin t / (2 r^3)) gives E = -v B_theta phi_hat
    exactly; the field-aligned start of Sect. 3.1 gives E = 0 to round-off."""
    shape = (5, 8, 16)
    g = oracle_grid(shape)
    U, info = ci.background(*shape)
    E = oracle.efield(g, U)
    rc, tc, pc = ci.cell_centres(*shape)
    R, T, P = np.meshgrid(rc, tc, pc, indexing="ij")
    W = info["W"]
    v = np.sqrt(W[1] ** 2 + W[2] ** 2 + W[3] ** 2)
    ephi = -v * np.sin(T) / (2 * R ** 3)
    want = np.stack([-np.sin(P) * ephi, np.cos(P) * ephi, np.zeros_like(ephi)])
    np.testing.assert_allclose(E, want, rtol=1e-12, atol=1e-14 * np.abs(ephi).max())
    U0, info0 = ci.background(*shape, efree=True)
    E0 = oracle.efield(g, U0)
    W0 = info0["W"]
    scale = np.linalg.norm(W0[1:4], axis=0) * np.linalg.norm(W0[4:7], axis=0)
    assert np.max(np.linalg.norm(E0, axis=0) / scale) < 1e-14
    # same speed, same density: only the direction of V changed
    np.testing.assert_allclose(np.linalg.norm(W0[1:4], axis=0), v, rtol=1e-14)


def test_low_e_wind_predict_magnitude_equations():
    """Low-E with the Wind-Predict outflow magnitude: face-mean V_b = V_r* B_r
    B_b / |B_b|^2 with B_b = B_r rhat + tangential interior B, so V_b x B_b = 0,
    V_b . rhat = V_r* B_r^2 / |B_b|^2, and V_b does not move with V_I."""
    vr_star = 1935.07 / ci.V_REF
    shape = (4, 12, 16)
    g = oracle_grid(shape, inner_bc="low_e_wp", vr_star=vr_star)
    U, info = ci.background(*shape)
    U = ci.perturb(info["W"], seed=8, amp=0.2)
    Br = ci.magnetogram(12, 16, lmax=6, seed=5)
    Win, _ = oracle.ghosts(g, U, Br)
    WI = oracle.cons_to_prim(g, U)[:, 0]
    V, B, _ = spherical(0.5 * (Win + WI), g)
    _, BI, _ = spherical(WI, g)
    np.testing.assert_allclose(B["r"], Br, atol=1e-14)
    np.testing.assert_allclose(B["t"], BI["t"], atol=1e-14)
    np.testing.assert_allclose(B["p"], BI["p"], atol=1e-14)
    b2 = B["r"] ** 2 + B["t"] ** 2 + B["p"] ** 2
    q = vr_star * Br / b2
    for c in "rtp":
        np.testing.assert_allclose(V[c], q * B[c], rtol=1e-12, atol=1e-18)
    def face_v(W):
        Ux = ci.prim_to_cons(W)
        return 0.5 * (oracle.ghosts(g, Ux, Br)[0][1:4] + oracle.cons_to_prim(g, Ux)[1:4, 0])
    W2 = info["W"].copy()
    W2[1:4] *= 1.7
    np.testing.assert_allclose(face_v(W2), face_v(info["W"]), rtol=1e-12, atol=1e-18)


def test_inner_boundary_growing_mode():
    """On the Parker + dipole state the low-E ghost with the interior-projected
    |V_b| gives the semi-discrete operator a growing mode at the inner layer
    (an eigenvalue of diag(dt_c) dR/dU with real part near +1, i.e. growth on
    the local time-step scale, mostly in the energy); the large-E ghost and
    the low-E ghost with the prescribed V_r* magnitude have none.  This is why
    the backward-Euler iteration of Sect. 2.1 diverges with the former."""
    shape = (4, 4, 8)
    U, Br = problem(shape)
    top = {}
    for bc in ("low_e", "large_e", "low_e_wp"):
        kw = {} if bc == "low_e" else dict(inner_bc=bc, vr_star=1935.07 / ci.V_REF)
        g = oracle_grid(shape, **kw)
        B = ci.potential_field(4, 8, dipole_only=True) if bc == "large_e" else Br
        J = oracle.jacobian(g, U, B)
        dt = np.broadcast_to(oracle.local_dt(g, U), U.shape).ravel()
        top[bc] = np.linalg.eigvals(J * dt[:, None]).real.max()
    assert top["low_e"] > 0.5
    assert top["large_e"] < 0.0 and top["low_e_wp"] < 0.0
