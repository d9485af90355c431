"""GPU parity of the boundary variants: the nine outer laws of Table 2
(Sect. 4.1), the rho ~ r^-2.5 law (Sect. 4.2), the large-E inner form
(Sect. 3.2), the boundary E-field diagnostic, and the VJP through them.
Error metric and bars as in the main parity tests."""
import json
import os

import numpy as np
import pytest

import coronal_inputs as ci
import oracle
from _util import check_fp32, oracle_grid, problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_BOUND = 1e-12
FP32_BOUND = 2e-5
VR_STAR = 1935.07 / ci.V_REF


def table2_params(case):
    with open(os.path.join(os.path.dirname(__file__), "golden", "table2_outer_bc.json")) as f:
        law = json.load(f)["cases"][case]
    return dict(outer_rho_exp=float(law["rho"]), outer_br_exp=float(law["Br"]),
                outer_bphi_exp=float(law["Bphi"]), outer_vr_mass=law["Vr"] == "mass",
                outer_vphi_exp=float(law["Vphi"]), outer_psi_extrap=law["psi"] == "G=I")


VARIANTS = {f"case{c}": table2_params(str(c)) for c in range(1, 10)}
VARIANTS["r-2.5"] = dict(outer_rho_exp=2.5)
VARIANTS["large_e"] = dict(inner_bc="large_e", vr_star=VR_STAR)
VARIANTS["large_e+case9"] = dict(inner_bc="large_e", vr_star=VR_STAR, **table2_params("9"))
VARIANTS["low_e_wp"] = dict(inner_bc="low_e_wp", vr_star=VR_STAR)
VARIANTS["low_e_wp+case9"] = dict(inner_bc="low_e_wp", vr_star=VR_STAR, **table2_params("9"))
# GLM damping of the cleaning scalar (source -alpha psi)
VARIANTS["psi_damp"] = dict(psi_damp=0.5)
# the Sect. 4.3 mesh: domain to 25 R_sun with a thin outermost cell
VARIANTS["thin_last+case1"] = dict(r_out=25.0, r_last=24.95, **table2_params("1"))
VARIANTS["thin_last+case9"] = dict(r_out=25.0, r_last=24.95, **table2_params("9"))


def inputs(shape, variant, seed=7):
    U, Br = problem(shape, perturb=seed)
    if VARIANTS[variant].get("inner_bc") == "large_e":
        Br = ci.potential_field(shape[1], shape[2], lmax=6, seed=11)
    return U, Br


def gpu(shape, precision, kw, limiter="vanalbada", kernel="tiled"):
    import paper_2209_04481_gb300 as pg
    return pg.Grid(*shape, precision=precision, limiter=limiter, kernel=kernel,
                   p_b=ci.parker_sound_speed2(), **kw)


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("precision,kernel,bound", [("fp64", "tiled", FP64_BOUND),
                                                    ("fp64", "cellwise", FP64_BOUND),
                                                    ("fp32", "tiled", FP32_BOUND)])
def test_residual_parity(variant, precision, kernel, bound):
    shape = (10, 12, 24)
    kw = VARIANTS[variant]
    U, Br = inputs(shape, variant)
    ref = oracle.residual(oracle_grid(shape, **kw), U, Br, want_scale=True)
    g = gpu(shape, precision, kw, kernel=kernel)
    g.set_inner_boundary(dev(Br))
    norms = torch.zeros(9, dtype=torch.float64, device="cuda")
    dtmin = torch.zeros(1, dtype=torch.float64, device="cuda")
    R = g.residual(dev(U, g.dtype), norms=norms, dtmin=dtmin)
    g.sync_status()
    if precision == "fp32":
        check_fp32(R.double().cpu().numpy(), ref, oracle_grid(shape, **kw), U, norms.cpu().numpy(),
                   float(dtmin.cpu()[0]))
        return
    err = rel_err(R.double().cpu().numpy(), ref["R"], ref["scale"])
    assert np.all(err <= bound), err
    np.testing.assert_allclose(norms.cpu().numpy(), ref["norms"], rtol=1e-11)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_large_e_full_size(precision):
    """Large-E inner form on the 128 x 64 x 128 workload (every cell)."""
    shape = (128, 64, 128)
    kw = VARIANTS["large_e"]
    U, _ = problem("shell128")
    Br = ci.potential_field(64, 128, lmax=15, seed=1, target_max=5.0)
    ref = oracle.residual(oracle_grid(shape, **kw), U, Br, want_scale=True)
    g = gpu(shape, precision, kw)
    g.set_inner_boundary(dev(Br))
    R = g.residual(dev(U, g.dtype))
    g.sync_status()
    err = rel_err(R.double().cpu().numpy(), ref["R"], ref["scale"])
    assert np.all(err <= (FP64_BOUND if precision == "fp64" else FP32_BOUND)), err


@pytest.mark.parametrize("variant", ["case3", "large_e"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_boundary_efield(variant, precision):
    """crn_boundary_efield against the oracle's E = -V_b x B_b; bound relative
    to |V_b||B_b| (FP32 storage of U rounds V and B to 2^-24)."""
    shape = (6, 16, 32)
    kw = VARIANTS[variant]
    U, Br = inputs(shape, variant)
    og = oracle_grid(shape, **kw)
    E_ref = oracle.boundary_efield(og, U, Br)
    Win, _ = oracle.ghosts(og, U, Br)
    Wb = 0.5 * (Win + oracle.cons_to_prim(og, U)[:, 0])
    scale = np.max(np.linalg.norm(Wb[1:4], axis=0) * np.linalg.norm(Wb[4:7], axis=0))
    g = gpu(shape, precision, kw)
    g.set_inner_boundary(dev(Br))
    E = g.boundary_efield(dev(U, g.dtype)).cpu().numpy()
    g.sync_status()
    tol = 1e-13 if precision == "fp64" else 1e-5
    assert np.max(np.abs(E - E_ref)) <= tol * scale
    if variant == "case3":   # low-E: the face field vanishes
        assert np.max(np.abs(E)) <= tol * scale


@pytest.mark.parametrize("variant", ["large_e", "case9", "case5", "large_e+case9", "low_e_wp", "low_e_wp+case9", "psi_damp"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_vjp_dot_product(variant, precision, tol):
    """<Rbar, J v> (oracle dual numbers) = <J^T Rbar, v> (GPU VJP), including
    the cotangent of the prescribed (B_r, B_theta)."""
    shape = (10, 12, 24)
    kw = VARIANTS[variant]
    U, Br = inputs(shape, variant, seed=3)
    og = oracle_grid(shape, **kw)
    Rbar = np.random.default_rng(4).standard_normal(U.shape)
    g = gpu(shape, precision, kw)
    g.set_inner_boundary(dev(Br))
    Ub, Brb = g.residual_vjp(dev(U, g.dtype), dev(Rbar, g.dtype))
    g.sync_status()
    Ub, Brb = Ub.double().cpu().numpy(), Brb.cpu().numpy()
    assert Brb.shape == Br.shape
    for seed in (100, 101):
        r = np.random.default_rng(seed)
        dU = r.standard_normal(U.shape) * (np.abs(U) + 1e-3)
        dBr = r.standard_normal(Br.shape)
        _, Jv = oracle.residual_jvp(og, U, Br, dU, dBr)
        lhs = np.sum(Rbar * Jv)
        rhs = np.sum(Ub * dU) + np.sum(Brb * dBr)
        assert abs(lhs - rhs) <= tol * np.sum(np.abs(Rbar * Jv)), (lhs, rhs)


def test_large_e_boundary_cotangent_per_entry():
    """Each entry of (dR/d(B_r, B_theta))^T Rbar on a 4 x 4 x 8 shell against
    the oracle's JVP columns, one unit direction per boundary value."""
    shape = (4, 4, 8)
    kw = dict(VARIANTS["large_e"], r_out=3.0)
    U, info = ci.background(*shape, r_out=3.0)
    U = ci.perturb(info["W"], seed=5, amp=0.05)
    Br = ci.potential_field(4, 8, lmax=3, seed=2)
    og = oracle_grid(shape, **kw)
    Rbar = np.random.default_rng(9).standard_normal(U.shape)
    g = gpu(shape, "fp64", kw)
    g.set_inner_boundary(dev(Br))
    _, Brb = g.residual_vjp(dev(U), dev(Rbar))
    g.sync_status()
    Brb = Brb.cpu().numpy()
    for idx in np.ndindex(Br.shape):
        e = np.zeros_like(Br)
        e[idx] = 1.0
        _, Jv = oracle.residual_jvp(og, U, Br, np.zeros_like(U), e)
        want = np.sum(Rbar * Jv)
        assert abs(Brb[idx] - want) <= 1e-12 * (np.sum(np.abs(Rbar * Jv)) + 1e-300), idx


@pytest.mark.parametrize("efree", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_volume_efield(precision, efree):
    """crn_efield against the oracle's cell-wise E = -V x B, relative to
    max |V||B|; the field-aligned start gives E = 0 to the storage precision."""
    shape = (10, 12, 24)
    U, info = ci.background(*shape, efree=efree)
    og = oracle_grid(shape)
    E_ref = oracle.efield(og, U)
    W = info["W"]
    scale = np.max(np.linalg.norm(W[1:4], axis=0) * np.linalg.norm(W[4:7], axis=0))
    g = gpu(shape, precision, {})
    Ud = dev(U, g.dtype)
    E = g.efield(Ud).cpu().numpy()
    assert g.last_launch_count == 1
    # FP64: the same operations as the oracle; FP32: U rounded to 2^-24
    tol = 1e-15 if precision == "fp64" else 1e-6
    assert np.max(np.abs(E - E_ref)) <= tol * scale
    if efree:
        assert np.max(np.abs(E)) <= tol * scale

