"""The tiled VJP (vjp_radial + vjp_lateral in vjp_tiled.cuh) on the shapes
where its tiling has edges: n_theta of 2 and 3 (a tile's 3-cell halo crosses
a pole twice), n_phi below the tile width, ragged tiles and column groups,
radial blocks that end at the inner boundary, in the interior and next to the
outer boundary, every limiter and the boundary variants of Sect. 3.2 /
Table 2; in FP32 (its default) and FP64 (on request: FP64 grids default to
the face/cell VJP).

Checked against the oracle's dual-number JVP through the dot-product
identity <Rbar, J v> = <J^T Rbar, v> (exact up to rounding), and element by
element against the face/cell VJP of the reference kernels (vjp.cuh), which
shares only the per-face adjoint arithmetic with it and none of its
stencil, halo, pole or chunk handling.
"""
import numpy as np
import pytest

import coronal_inputs as ci
import oracle
from _util import oracle_grid, problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}
# tiled against reference: the same derivatives summed in another order
ELEM = {"fp64": 1e-11, "fp32": 2e-4}


def run(shape, U, Br, Rbar, precision, monkeypatch, limiter="vanalbada", vjp="tiled", **kw):
    """The VJP through crn_residual_vjp; vjp = "tiled" (vjp_tiled.cuh) or
    "faces" (the face/cell pair of vjp.cuh), chosen with CRN_VJP_KERNEL."""
    import paper_2209_04481_gb300 as pg
    monkeypatch.setenv("CRN_VJP_KERNEL", vjp)
    g = pg.Grid(*shape, precision=precision, limiter=limiter, p_b=ci.parker_sound_speed2(), **kw)
    dt = torch.float64 if precision == "fp64" else torch.float32
    g.set_inner_boundary(torch.from_numpy(np.ascontiguousarray(Br)).cuda())
    Ub, Brb = g.residual_vjp(torch.from_numpy(U).to("cuda", dt), torch.from_numpy(Rbar).to("cuda", dt))
    g.sync_status()
    nl = g.last_launch_count
    out = Ub.double().cpu().numpy(), Brb.cpu().numpy(), nl
    g.close()
    monkeypatch.delenv("CRN_VJP_KERNEL", raising=False)
    return out


def dot_identity(og, U, Br, Rbar, Ub, Brb, tol):
    for seed in (100, 101):
        r = np.random.default_rng(seed)
        dU = r.standard_normal(U.shape) * (np.abs(U) + 1e-3)
        dBr = r.standard_normal(Br.shape)
        _, Jv = oracle.residual_jvp(og, U, Br, dU, dBr)
        assert np.all(np.isfinite(Jv))
        lhs = np.sum(Rbar * Jv)
        rhs = np.sum(Ub * dU) + np.sum(Brb * dBr)
        scale = np.sum(np.abs(Rbar * Jv))
        assert abs(lhs - rhs) <= tol * scale, (seed, lhs, rhs, scale)


def elementwise(A, B, tol):
    A = A.reshape(A.shape[0], -1) if A.ndim > 1 else A[None]
    B = B.reshape(A.shape)
    for v in range(A.shape[0]):
        sc = np.abs(B[v]).max() + 1e-300
        err = np.abs(A[v] - B[v]).max() / sc
        assert err <= tol, (v, err)


SHAPES = [(2, 2, 8), (3, 3, 8), (5, 4, 16), (7, 10, 40), (12, 17, 48), (16, 8, 64)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("limiter", ["vanalbada", "minmod", "none"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tiled_vjp_dot_product_identity(shape, limiter, precision, monkeypatch):
    if limiter == "none" and precision == "fp32":
        # unlimited radial reconstruction on fewer than ~20 planes over
        # 1..21.5 R_sun extrapolates to negative face densities and
        # pressures; the derivative is still defined (and checked in FP64),
        # but FP32 rounding then decides the sign of the fast-speed
        # discriminant.  32 planes keep every face state physical.
        shape = (32,) + tuple(shape[1:])
    U, Br = problem(shape, perturb=3)
    Rbar = np.random.default_rng(4).standard_normal(U.shape)
    Ub, Brb, nl = run(shape, U, Br, Rbar, precision, monkeypatch, limiter)
    assert nl == 2
    dot_identity(oracle_grid(shape, limiter=limiter), U, Br, Rbar, Ub, Brb, TOL[precision])


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tiled_vjp_matches_reference_vjp(shape, precision, monkeypatch):
    U, Br = problem(shape, perturb=8)
    Rbar = np.random.default_rng(12).standard_normal(U.shape)
    Ut, Bt, _ = run(shape, U, Br, Rbar, precision, monkeypatch)
    Ur, Brr, nl = run(shape, U, Br, Rbar, precision, monkeypatch, vjp="faces")
    assert nl == (3 if precision == "fp64" else 2)
    elementwise(Ut, Ur, ELEM[precision])
    elementwise(Bt, Brr, ELEM[precision])


@pytest.mark.parametrize("nr", [12, 13, 14, 15, 26, 27, 40])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tiled_vjp_radial_blocks(nr, precision, monkeypatch):
    """The radial pass works on blocks of 13 planes: a block with one plane
    missing, a whole block, a last block of 1 or 2 planes, of 13 + 13, 13 + 1
    and 13 + 1 planes (block ends at both boundaries and in the interior);
    8 x 32 = 256 columns, so that the 16-column groups are whole."""
    shape = (nr, 8, 32)
    U, Br = problem(shape, perturb=9)
    Rbar = np.random.default_rng(5).standard_normal(U.shape)
    Ut, Bt, _ = run(shape, U, Br, Rbar, precision, monkeypatch)
    Uf, Bf, _ = run(shape, U, Br, Rbar, precision, monkeypatch, vjp="faces")
    elementwise(Ut, Uf, ELEM[precision])
    elementwise(Bt, Bf, ELEM[precision])
    if nr in (14, 27):
        dot_identity(oracle_grid(shape), U, Br, Rbar, Ut, Bt, TOL[precision])


@pytest.mark.parametrize("variant", ["large_e", "low_e_wp", "case9", "r-2.5", "psi_damp",
                                     "thin_last+case1", "large_e+case9"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tiled_vjp_boundary_variants(variant, precision, monkeypatch):
    from test_gpu_bc_variants import VARIANTS, inputs
    shape = (10, 12, 24)
    kw = VARIANTS[variant]
    U, Br = inputs(shape, variant)
    Rbar = np.random.default_rng(6).standard_normal(U.shape)
    Ub, Brb, _ = run(shape, U, Br, Rbar, precision, monkeypatch, **kw)
    dot_identity(oracle_grid(shape, **kw), U, Br, Rbar, Ub, Brb, TOL[precision])
    Ur, Brr, _ = run(shape, U, Br, Rbar, precision, monkeypatch, vjp="faces", **kw)
    elementwise(Ub, Ur, ELEM[precision])
    elementwise(Brb, Brr, ELEM[precision])


def test_tiled_vjp_is_deterministic(monkeypatch):
    """Fixed-order gathers, no atomics: two calls agree bit for bit."""
    import paper_2209_04481_gb300 as pg
    shape = (16, 24, 96)
    U, Br = problem(shape, perturb=2)
    Rbar = np.random.default_rng(1).standard_normal(U.shape).astype(np.float32)
    monkeypatch.delenv("CRN_VJP_KERNEL", raising=False)
    g = pg.Grid(*shape, precision="fp32", p_b=ci.parker_sound_speed2())
    g.set_inner_boundary(torch.from_numpy(Br).cuda())
    Ud = torch.from_numpy(U).to("cuda", torch.float32)
    Rd = torch.from_numpy(Rbar).cuda()
    a = [t.cpu().numpy() for t in g.residual_vjp(Ud, Rd)]
    b = [t.cpu().numpy() for t in g.residual_vjp(Ud, Rd)]
    g.sync_status()
    assert g.last_launch_count == 2   # FP32 grids default to the tiled VJP
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    g.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_vjp_full_size_128x64x128(precision, monkeypatch):
    """The benchmark's workload and launch configuration (128 x 64 x 128,
    Parker wind + dipole + l <= 15 field, N(0, 1) cotangent seed 4; the
    grid's default VJP: tiled in FP32, face/cell in FP64).

    Dot-product identity against the oracle's JVP.  At this size and field
    strength the identity is ill-conditioned in FP64: the sum of 9.4 M terms
    cancels to 1 part in 1300 of its absolute sum, and the fast speed's max
    and |u_n| sit near their kinks at some faces, so a 1-ulp change of the
    inputs moves the oracle's own value by ~1e-9 of the absolute sum (more
    than 1e-12).  The FP64 bar is therefore measured in the test: four times
    the spread of the oracle's value under two random 1-ulp perturbations of
    U.  FP32: the 2e-5 bar of the other tests.

    Then the tiled and the face/cell VJP element by element, on the same
    field with the 1 % perturbation of the adjoint workload (seed 3): the
    unperturbed Parker wind is exactly radial, so V.n of every phi face is
    zero up to rounding, and where the fast speed sets lambda the sign of
    that rounding (which differs with the FMA contraction of each kernel)
    picks the one-sided derivative of |u_n| at about 80 cells."""
    w = ci.workload("shell128")
    U, Br = w["U"], w["Br"]
    shape = U.shape[1:]
    Rbar = ci.cotangent(U.shape, seed=4)
    monkeypatch.delenv("CRN_VJP_KERNEL", raising=False)
    import paper_2209_04481_gb300 as pg
    g = pg.Grid(*shape, precision=precision, p_b=w["p_b"])
    dt = torch.float64 if precision == "fp64" else torch.float32
    g.set_inner_boundary(torch.from_numpy(Br).cuda())
    Ub, Brb = g.residual_vjp(torch.from_numpy(U).to("cuda", dt), torch.from_numpy(Rbar).to("cuda", dt))
    g.sync_status()
    assert g.last_launch_count == (3 if precision == "fp64" else 2)
    Ub, Brb = Ub.double().cpu().numpy(), Brb.cpu().numpy()
    g.close()
    og = oracle_grid(shape, p_b=w["p_b"])
    if precision == "fp32":
        dot_identity(og, U, Br, Rbar, Ub, Brb, TOL[precision])
    else:
        r = np.random.default_rng(100)
        dU = r.standard_normal(U.shape) * (np.abs(U) + 1e-3)
        dBr = r.standard_normal(Br.shape)
        vals = []
        for s in (0, 1, 2):
            Up = U if s == 0 else U * (1 + np.random.default_rng(s).choice([-1.0, 1.0], U.shape) * 2.0 ** -52)
            _, Jv = oracle.residual_jvp(og, Up, Br, dU, dBr)
            assert np.all(np.isfinite(Jv))
            vals.append(np.sum(Rbar * Jv))
        spread = max(abs(vals[1] - vals[0]), abs(vals[2] - vals[0]))
        rhs = np.sum(Ub * dU) + np.sum(Brb * dBr)
        assert abs(vals[0] - rhs) <= 4 * spread, (vals, rhs)
    _, info = ci.background(*shape)
    Up = ci.perturb(info["W"], seed=3)
    Ut, Bt, _ = run(shape, Up, Br, Rbar, precision, monkeypatch, vjp="tiled")
    Uf, Bf, _ = run(shape, Up, Br, Rbar, precision, monkeypatch, vjp="faces")
    elementwise(Ut, Uf, ELEM[precision])
    elementwise(Bt, Bf, ELEM[precision])
