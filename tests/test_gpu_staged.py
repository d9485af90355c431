"""GPU parity of the TMA-staged FP32 residual kernel (residual_staged.cuh).

The staged kernel runs on request (kernel "staged") for FP32-bulk grids that
tile into whole 8 x 32 (theta, phi) blocks.  It is checked element by element
against the FP64 oracle on shapes that reach the poles and the periodic seam
from every block, with radial chunks of 1, 2, 3, 5 planes and the default
(chunk starts at the inner boundary, in the interior and one or two planes
before the outer boundary), the three limiters and the boundary variants of
Sect. 3.2 and Table 2; and against the register-staged tiled kernel, which
shares no staging code with it.
"""
import numpy as np
import pytest

import coronal_inputs as ci
import oracle
from _util import check_fp32, oracle_grid, problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VR_STAR = 1935.07 / ci.V_REF


def run(shape, U, Br, monkeypatch, limiter="vanalbada", kchunk=None, kernel="staged", **kw):
    import paper_2209_04481_gb300 as pg
    if kchunk is not None:
        monkeypatch.setenv("CRN_KCHUNK", str(kchunk))
    g = pg.Grid(*shape, precision="fp32", limiter=limiter, kernel=kernel, p_b=ci.parker_sound_speed2(), **kw)
    monkeypatch.delenv("CRN_KCHUNK", raising=False)
    g.set_inner_boundary(torch.from_numpy(np.ascontiguousarray(Br)).cuda())
    norms = torch.zeros(9, dtype=torch.float64, device="cuda")
    dtmin = torch.zeros(1, dtype=torch.float64, device="cuda")
    R = g.residual(torch.from_numpy(U).to("cuda", torch.float32), norms=norms, dtmin=dtmin)
    g.sync_status()
    kern = g.last_kernel
    out = R.double().cpu().numpy(), norms.cpu().numpy(), float(dtmin.cpu()[0]), kern
    g.close()
    return out


SHAPES = [(2, 8, 32), (5, 16, 64), (13, 24, 32), (20, 8, 96)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("limiter", ["vanalbada", "minmod", "none"])
def test_staged_parity(shape, limiter, monkeypatch):
    U, Br = problem(shape, perturb=5)
    ref = oracle.residual(oracle_grid(shape, limiter=limiter), U, Br, want_scale=True)
    R, norms, dtmin, kern = run(shape, U, Br, monkeypatch, limiter)
    assert kern == "staged"
    check_fp32(R, ref, oracle_grid(shape, limiter=limiter), U, norms, dtmin)


@pytest.mark.parametrize("kchunk", [1, 2, 3, 5])
def test_staged_radial_chunks(kchunk, monkeypatch):
    """Chunk boundaries everywhere: R does not depend on where a CTA starts."""
    shape = (13, 16, 32)
    U, Br = problem(shape, perturb=9)
    ref = oracle.residual(oracle_grid(shape), U, Br, want_scale=True)
    R, norms, dtmin, kern = run(shape, U, Br, monkeypatch, kchunk=kchunk)
    assert kern == "staged"
    check_fp32(R, ref, oracle_grid(shape), U, norms, dtmin)


@pytest.mark.parametrize("variant", ["large_e", "low_e_wp", "case9", "r-2.5"])
def test_staged_boundary_variants(variant, monkeypatch):
    from test_gpu_bc_variants import VARIANTS, inputs
    shape = (10, 16, 32)
    kw = VARIANTS[variant]
    U, Br = inputs(shape, variant)
    ref = oracle.residual(oracle_grid(shape, **kw), U, Br, want_scale=True)
    R, norms, dtmin, kern = run(shape, U, Br, monkeypatch, **kw)
    assert kern == "staged"
    check_fp32(R, ref, oracle_grid(shape, **kw), U, norms, dtmin)


def test_staged_matches_register_tiled(monkeypatch):
    """The two FP32 tiled kernels agree to FP32 rounding of the flux arithmetic;
    the default kernel is the register-staged one."""
    shape = (24, 32, 64)
    U, Br = problem(shape, perturb=4)
    ref = oracle.residual(oracle_grid(shape), U, Br, want_scale=True)
    Rs, ns, ds, ks = run(shape, U, Br, monkeypatch)
    Rt, nt_, dt_, kt = run(shape, U, Br, monkeypatch, kernel="tiled")
    assert ks == "staged" and kt == "tiled_regs"
    assert np.all(rel_err(Rs, Rt, ref["scale"]) <= 2e-6)
    np.testing.assert_allclose(ns, nt_, rtol=1e-4)
    assert ds == pytest.approx(dt_, rel=1e-5)


def test_staged_is_deterministic_and_unaligned_state_falls_back(monkeypatch):
    """Two calls give bitwise equal R, norms and dtmin; a state that is not
    16-byte aligned cannot feed the tensor map and takes the register-staged
    kernel, with the same result to rounding."""
    import paper_2209_04481_gb300 as pg
    shape = (9, 16, 32)
    U, Br = problem(shape, perturb=2)
    g = pg.Grid(*shape, precision="fp32", kernel="staged", p_b=ci.parker_sound_speed2())
    g.set_inner_boundary(torch.from_numpy(Br).cuda())
    Ud = torch.from_numpy(U).to("cuda", torch.float32)
    outs = []
    for _ in range(2):
        norms = torch.zeros(9, dtype=torch.float64, device="cuda")
        R = g.residual(Ud, norms=norms)
        g.sync_status()
        assert g.last_kernel == "staged"
        outs.append((R.cpu().numpy(), norms.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    buf = torch.empty(Ud.numel() + 1, dtype=torch.float32, device="cuda")
    Uoff = buf[1:].view(Ud.shape)
    Uoff.copy_(Ud)
    R2 = g.residual(Uoff)
    g.sync_status()
    assert g.last_kernel == "tiled_regs"
    ref = oracle.residual(oracle_grid(shape), U, Br, want_scale=True)
    assert np.all(rel_err(R2.double().cpu().numpy(), outs[0][0], ref["scale"]) <= 2e-6)
    g.close()
