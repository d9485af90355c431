"""The hand-written residual VJP (crn_residual_vjp) against the oracle's
forward-mode JVP (dot-product identity and, on a tiny grid, the full
Jacobian), against central finite differences of the GPU residual, and
through torch.autograd.gradcheck."""
import numpy as np
import pytest

import coronal_inputs as ci
import oracle
from _util import oracle_grid, problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def gpu_grid(shape, precision, limiter="vanalbada"):
    import paper_2209_04481_gb300 as pg
    return pg.Grid(*shape, precision=precision, limiter=limiter, p_b=ci.parker_sound_speed2())


def gpu_vjp(shape, U, Br, Rbar, precision, limiter="vanalbada"):
    g = gpu_grid(shape, precision, limiter)
    dt = torch.float64 if precision == "fp64" else torch.float32
    g.set_inner_boundary(torch.from_numpy(Br).cuda())
    Ub, Brb = g.residual_vjp(torch.from_numpy(U).to("cuda", dt),
                             torch.from_numpy(Rbar).to("cuda", dt))
    g.sync_status()
    return Ub.double().cpu().numpy(), Brb.cpu().numpy()


@pytest.mark.parametrize("shape", [(8, 8, 16), (10, 12, 24), (64, 32, 64)])
@pytest.mark.parametrize("limiter", ["vanalbada", "minmod", "none"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_dot_product_identity(shape, limiter, precision, tol):
    """<Rbar, J v>_oracle (dual numbers) = <J^T Rbar, v>_GPU for random Rbar, v."""
    if shape == (64, 32, 64):
        U, Br = problem("shell64")
    else:
        U, Br = problem(shape, perturb=3)
    og = oracle_grid(shape, limiter=limiter)
    rng = np.random.default_rng(4)
    Rbar = rng.standard_normal(U.shape)
    Ub, Brb = gpu_vjp(shape, U, Br, Rbar, precision, limiter)
    for seed in (100, 101):
        r = np.random.default_rng(seed)
        dU = r.standard_normal(U.shape) * (np.abs(U) + 1e-3)
        dBr = r.standard_normal(Br.shape)
        _, Jv = oracle.residual_jvp(og, U, Br, dU, dBr)
        lhs = np.sum(Rbar * Jv)
        rhs = np.sum(Ub * dU) + np.sum(Brb * dBr)
        scale = np.sum(np.abs(Rbar * Jv))
        assert abs(lhs - rhs) <= tol * scale, (lhs, rhs, scale)


def test_full_jacobian_tiny_grid():
    """Every entry of J^T Rbar on a 4 x 4 x 8 shell against the oracle's
    Jacobian assembled column by column from dual-number JVPs."""
    import paper_2209_04481_gb300 as pg
    shape = (4, 4, 8)
    og = oracle_grid(shape, r_out=3.0)
    U, info = ci.background(*shape, r_out=3.0)
    U = ci.perturb(info["W"], seed=5, amp=0.02)
    Br = ci.magnetogram(shape[1], shape[2], lmax=2, seed=6)
    g = pg.Grid(*shape, precision="fp64", r_out=3.0, p_b=ci.parker_sound_speed2())
    Rbar = np.random.default_rng(9).standard_normal(U.shape)
    g.set_inner_boundary(torch.from_numpy(Br).cuda())
    Ub, Brb = g.residual_vjp(torch.from_numpy(U).cuda(), torch.from_numpy(Rbar).cuda())
    Ub, Brb = Ub.cpu().numpy(), Brb.cpu().numpy()
    n = U.size
    ref = np.zeros(n)
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        _, col = oracle.residual_jvp(og, U, Br, e.reshape(U.shape), np.zeros_like(Br))
        ref[q] = np.sum(Rbar * col)
    refb = np.zeros(Br.size)
    for q in range(Br.size):
        e = np.zeros(Br.size)
        e[q] = 1.0
        _, col = oracle.residual_jvp(og, U, Br, np.zeros_like(U), e.reshape(Br.shape))
        refb[q] = np.sum(Rbar * col)
    ref = ref.reshape(U.shape)
    for v in range(9):
        sc = np.abs(ref[v]).max() + 1e-300
        assert np.abs(Ub[v] - ref[v]).max() <= 1e-11 * sc, v
    assert np.abs(Brb.ravel() - refb).max() <= 1e-11 * (np.abs(refb).max() + 1e-300)


@pytest.mark.parametrize("limiter,h,bound", [("none", 1e-8, 1e-5), ("vanalbada", 1e-8, 1e-4)])
def test_finite_differences_50_directions(limiter, h, bound):
    """<Rbar, (R(U + h v) - R(U - h v)) / 2h> of the GPU FP64 residual against
    <VJP(Rbar), v> on 50 random directions (seeds 100..149), 64 x 32 x 64
    perturbed shell, N(0, 1) cotangent (seed 4).  Step 1e-8: the kinks of
    |u_n| and of the max in lambda lie within 1e-7..1e-6 of these states in
    some directions (a 1e-6 step straddles them), and the smooth van Albada
    form varies on the scale sqrt(eps) = 1e-6 of its slope arguments; the
    exact derivatives are pinned elementwise against the oracle's dual
    numbers above.  At this step FP64 rounding of the residual differences
    (1.2 M terms) limits the agreement to ~1e-6 relative."""
    shape = (64, 32, 64)
    U, Br = problem("shell64")
    Rbar = ci.cotangent(U.shape, seed=4)
    g = gpu_grid(shape, "fp64", limiter)
    Br_d = torch.from_numpy(Br).cuda()
    g.set_inner_boundary(Br_d)
    Ud = torch.from_numpy(U).cuda()
    Rb = torch.from_numpy(Rbar).cuda()
    Ub, Brb = g.residual_vjp(Ud, Rb)
    errs = []
    for seed in range(100, 150):
        r = np.random.default_rng(seed)
        v = torch.from_numpy(r.standard_normal(U.shape) * (np.abs(U) + 1e-3)).cuda()
        dBr = torch.from_numpy(r.standard_normal(Br.shape)).cuda()
        g.set_inner_boundary(Br_d + h * dBr)
        Rp = g.residual(Ud + h * v)
        g.set_inner_boundary(Br_d - h * dBr)
        Rm = g.residual(Ud - h * v)
        fd = torch.sum(Rb * (Rp - Rm)).item() / (2 * h)
        ad = torch.sum(Ub * v).item() + torch.sum(Brb * dBr).item()
        errs.append(abs(fd - ad) / (abs(ad) + 1e-300))
    assert np.median(errs) < bound and max(errs) < 100 * bound, (np.median(errs), max(errs))


def test_autograd_gradcheck():
    import paper_2209_04481_gb300 as pg
    shape = (4, 4, 8)
    U, info = ci.background(*shape, r_out=3.0)
    U = ci.perturb(info["W"], seed=8, amp=0.02)
    Br = ci.magnetogram(shape[1], shape[2], lmax=2, seed=3)
    # unlimited reconstruction: smooth at the scale of the numerical Jacobian's step
    g = pg.Grid(*shape, precision="fp64", limiter="none", r_out=3.0, p_b=ci.parker_sound_speed2())
    Ut = torch.from_numpy(U).cuda().requires_grad_(True)
    Bt = torch.from_numpy(Br).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda u, b: pg.residual(u, b, g), (Ut, Bt), eps=1e-8,
                                    atol=1e-5, rtol=1e-4, nondet_tol=0.0)
