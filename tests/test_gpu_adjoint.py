"""Magnetogram sensitivity of a steady state (crn_adjoint_solve): the GPU's
adjoint sensitivity dg/dB_b = -(dR/dB_b)^T J^-T dg/dU against the oracle's
tangent definition -dg/dU . J^-1 (dR/dB_b dB) in random directions dB, at
the steady state the GPU's Newton-Krylov solve reaches."""
import numpy as np
import pytest

import coronal_inputs as ci
import oracle
from _util import oracle_grid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VR = 1935.07 / ci.V_REF


def steady(shape, bc, precision):
    import paper_2209_04481_gb300 as pg
    U, info = ci.background(*shape)
    kw = dict(inner_bc=bc, vr_star=VR)
    if bc == "large_e":
        Br = ci.potential_field(shape[1], shape[2], dipole_only=True)
    else:
        Br = ci.magnetogram(shape[1], shape[2], dipole_only=True)
    g = pg.Grid(*shape, precision=precision, p_b=info["p_b"], **kw)
    g.set_inner_boundary(torch.from_numpy(Br).cuda())
    U64 = torch.from_numpy(U).cuda()
    g.steady_solve(U64, max_steps=200, tol_drop=1e-8 if precision == "fp64" else 1e-4)
    return g, U64, Br, oracle_grid(shape, **kw)


def objectives(shape, U):
    """Mean outer-layer density and mean outer-layer radial field."""
    nt, np_ = shape[1], shape[2]  # U is not needed: the functionals are linear
    g_rho = np.zeros((9,) + shape)
    g_rho[0, -1] = 1.0 / (nt * np_)
    _, tc, pc = ci.cell_centres(*shape)
    T, P = np.meshgrid(tc, pc, indexing="ij")
    g_br = np.zeros((9,) + shape)
    g_br[4, -1] = np.sin(T) * np.cos(P) / (nt * np_)
    g_br[5, -1] = np.sin(T) * np.sin(P) / (nt * np_)
    g_br[6, -1] = np.cos(T) / (nt * np_)
    return {"rho": g_rho, "B_r": g_br}


@pytest.mark.parametrize("bc", ["low_e_wp", "large_e"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-6), ("fp32", 2e-2)])
@pytest.mark.parametrize("precond", [0, 1])
def test_adjoint_sensitivity_matches_oracle_tangent(bc, precision, tol, precond):
    shape = (6, 6, 16)
    g, U64, Br, og = steady(shape, bc, precision)
    U = U64.cpu().numpy()
    rng = np.random.default_rng(7)
    for name, gbar in objectives(shape, U).items():
        sens, _, st = g.adjoint_solve(U64, torch.from_numpy(gbar).cuda(), krylov_dim=300, max_restarts=5,
                                      lin_rtol=1e-11 if precision == "fp64" else 1e-6, precond=precond)
        g.sync_status()
        assert sens.shape == Br.shape
        s = sens.cpu().numpy()
        for _ in range(2):
            dB = rng.standard_normal(Br.shape)
            ref = oracle.steady_sensitivity(og, U, Br, gbar, dB, rtol=1e-11)
            got = float(np.sum(s * dB))
            assert abs(got - ref) <= tol * np.sum(np.abs(s * dB)), (name, got, ref, st)


@pytest.mark.parametrize("precond", [0, 1])
def test_adjoint_lambda_solves_the_transposed_system(precond):
    """J^T lambda = gbar, checked with the GPU VJP itself: (dR/dU)^T lambda."""
    shape = (8, 8, 16)
    g, U64, Br, og = steady(shape, "low_e_wp", "fp64")
    gbar = torch.from_numpy(objectives(shape, None)["rho"]).cuda()
    lam = torch.empty_like(U64)
    g.adjoint_solve(U64, gbar, lam=lam, krylov_dim=300, max_restarts=5, lin_rtol=1e-11, precond=precond)
    Ub, _ = g.residual_vjp(U64, lam)
    g.sync_status()
    assert torch.linalg.vector_norm(Ub - gbar) <= 1e-8 * torch.linalg.vector_norm(gbar)


@pytest.mark.parametrize("fgmres", [30, 0])
@pytest.mark.parametrize("precond", [0, 1])
@pytest.mark.parametrize("bc", ["low_e_wp", "large_e"])
def test_pseudo_time_adjoint_matches_oracle_tangent(bc, precond, fgmres):
    """The pseudo-time adjoint iteration (adjoint_cfl > 0), accelerated by
    flexible GMRES (adjoint_fgmres = 30, the default) and plain: the same
    sensitivity as the oracle's tangent definition, J^T lambda = gbar checked
    with the GPU VJP, and the iteration's own residual below lin_rtol."""
    shape = (6, 6, 16)
    g, U64, Br, og = steady(shape, bc, "fp64")
    U = U64.cpu().numpy()
    rng = np.random.default_rng(11)
    for name, gbar in objectives(shape, U).items():
        gb = torch.from_numpy(gbar).cuda()
        lam = torch.empty_like(U64)
        sens, _, st = g.adjoint_solve(U64, gb, lam=lam, krylov_dim=30, lin_rtol=1e-10, precond=precond,
                                      adjoint_cfl=100.0, adjoint_outer=400, adjoint_fgmres=fgmres)
        g.sync_status()
        assert st["lin_rel"] <= 1e-10, st
        Ub, _ = g.residual_vjp(U64, lam)
        assert torch.linalg.vector_norm(Ub - gb) <= 1e-9 * torch.linalg.vector_norm(gb)
        s = sens.cpu().numpy()
        for _ in range(2):
            dB = rng.standard_normal(Br.shape)
            ref = oracle.steady_sensitivity(og, U, Br, gbar, dB, rtol=1e-11)
            got = float(np.sum(s * dB))
            assert abs(got - ref) <= 1e-6 * np.sum(np.abs(s * dB)), (name, got, ref, st)


@pytest.mark.parametrize("bc", ["low_e_wp", "large_e"])
def test_pseudo_time_adjoint_on_fp32_bulk_grid_mixed_precision(bc):
    """FP32-bulk grid, accelerated pseudo-time adjoint with outer_fp64 = 1
    (the default): the passes use the FP32 VJP, the outer products, the true
    residual and the sensitivity the FP64 VJP of the FP64 state, so the solve
    reaches lin_rtol 1e-10 (far below the FP32 VJP's rounding) and the
    sensitivity matches the oracle's tangent definition at 1e-6.  lambda is
    checked with the VJP of an FP64 grid of the same shell."""
    import paper_2209_04481_gb300 as pg
    shape = (6, 6, 16)
    g, U64, Br, og = steady(shape, bc, "fp32")
    U = U64.cpu().numpy()
    g64 = pg.Grid(*shape, precision="fp64", p_b=ci.background(*shape)[1]["p_b"], inner_bc=bc, vr_star=VR)
    g64.set_inner_boundary(torch.from_numpy(Br).cuda())
    rng = np.random.default_rng(13)
    for name, gbar in objectives(shape, U).items():
        gb = torch.from_numpy(gbar).cuda()
        lam = torch.empty_like(U64)
        sens, _, st = g.adjoint_solve(U64, gb, lam=lam, krylov_dim=30, lin_rtol=1e-10, precond=1,
                                      adjoint_cfl=100.0, adjoint_outer=400)
        g.sync_status()
        assert st["lin_rel"] <= 1e-10, st
        Ub, _ = g64.residual_vjp(U64, lam)
        g64.sync_status()
        assert torch.linalg.vector_norm(Ub - gb) <= 1e-9 * torch.linalg.vector_norm(gb)
        s = sens.cpu().numpy()
        for _ in range(2):
            dB = rng.standard_normal(Br.shape)
            ref = oracle.steady_sensitivity(og, U, Br, gbar, dB, rtol=1e-11)
            got = float(np.sum(s * dB))
            assert abs(got - ref) <= 1e-6 * np.sum(np.abs(s * dB)), (name, got, ref, st)
    g64.close()
