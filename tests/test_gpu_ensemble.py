"""The ensemble (crn_ensemble_*): uneven grids in one persistent launch give
every member exactly its own crn_residual / crn_pseudo_time_step result,
agree with the oracle, and keep R under the tile autotuner."""
import numpy as np
import pytest

import coronal_inputs as ci
import oracle
from _util import oracle_grid, problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(12, 8, 32), (20, 16, 48), (9, 24, 64), (33, 12, 40), (7, 6, 8)]


VR_STAR = 1935.07 / ci.V_REF


def members(precision, limiter="vanalbada", shapes=SHAPES, perturb=3, **kw):
    import paper_2209_04481_gb300 as pg
    gs, Us, Brs = [], [], []
    for m, shape in enumerate(shapes):
        U, Br = problem(shape, seed=100 + m, perturb=None if perturb is None else perturb + m)
        g = pg.Grid(*shape, precision=precision, limiter=limiter, p_b=ci.parker_sound_speed2(), **kw)
        g.set_inner_boundary(torch.from_numpy(Br).cuda())
        gs.append(g)
        Us.append(U)
        Brs.append(Br)
    return gs, Us, Brs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("limiter", ["vanalbada", "minmod"])
def test_ensemble_equals_member_launches(precision, limiter):
    import paper_2209_04481_gb300 as pg
    gs, Us, Brs = members(precision, limiter)
    dt = gs[0].dtype
    Ud = [torch.from_numpy(U).to("cuda", dt) for U in Us]
    n = len(gs)
    norms = torch.zeros((n, 9), dtype=torch.float64, device="cuda")
    dtmin = torch.zeros(n, dtype=torch.float64, device="cuda")
    ens = pg.Ensemble(gs)
    Rs = ens.residual(Ud, norms=norms, dtmin=dtmin)
    assert ens.last_launch_count == 1
    torch.cuda.synchronize()
    for m, g in enumerate(gs):
        nm = torch.zeros(9, dtype=torch.float64, device="cuda")
        dm = torch.zeros(1, dtype=torch.float64, device="cuda")
        R = g.residual(Ud[m], norms=nm, dtmin=dm)
        g.sync_status()
        assert torch.equal(R, Rs[m]), m
        assert torch.equal(nm, norms[m]) and torch.equal(dm[0], dtmin[m]), m
    ens.close()


def test_ensemble_members_match_oracle():
    import paper_2209_04481_gb300 as pg
    for precision, bound in (("fp64", 1e-12), ("fp32", 2e-5)):
        gs, Us, Brs = members(precision)
        ens = pg.Ensemble(gs)
        Rs = ens.residual([torch.from_numpy(U).to("cuda", gs[0].dtype) for U in Us])
        for m, shape in enumerate(SHAPES):
            ref = oracle.residual(oracle_grid(shape), Us[m], Brs[m], want_scale=True)
            err = rel_err(Rs[m].double().cpu().numpy(), ref["R"], ref["scale"])
            assert np.all(err <= bound), (m, err)
        gs[0].sync_status()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_autotune_keeps_the_residual(precision):
    """The radial chunk only moves where a CTA starts marching (the first r
    face of a chunk is evaluated on the preamble path), so R agrees to
    rounding and the norms differ only in summation order."""
    import paper_2209_04481_gb300 as pg
    gs, Us, Brs = members(precision)
    Ud = [torch.from_numpy(U).to("cuda", gs[0].dtype) for U in Us]
    ens = pg.Ensemble(gs)
    base = [R.clone() for R in ens.residual(Ud)]
    k = ens.autotune(Ud, [torch.empty_like(U) for U in Ud])
    assert k in (0, 4, 6, 8, 12, 16, 24, 32, 48) and ens.kchunk == k
    # every member runs the (tile, chunk) its size class was given
    for m in range(len(gs)):
        tile, kc = ens.member_config(m)
        assert tile in ((8, 32), (16, 16)) and 1 <= kc
    tuned = ens.residual(Ud)
    tol = 1e-13 if precision == "fp64" else 1e-6
    for m in range(len(gs)):
        scale = base[m].abs().amax(dim=(1, 2, 3), keepdim=True)
        assert torch.all((tuned[m] - base[m]).abs() <= tol * scale), m
    for kc in (4, 7, 0):
        ens.kchunk = kc
        norms = torch.zeros((len(gs), 9), dtype=torch.float64, device="cuda")
        Rs = ens.residual(Ud, norms=norms)
        tol = 1e-13 if precision == "fp64" else 1e-6
        for m in range(len(gs)):
            scale = base[m].abs().amax(dim=(1, 2, 3), keepdim=True)
            assert torch.all((Rs[m] - base[m]).abs() <= tol * scale), (kc, m)
        ref = torch.stack([torch.linalg.vector_norm(R.double().reshape(9, -1), dim=1) for R in Rs])
        torch.testing.assert_close(norms, ref, rtol=1e-6 if precision == "fp32" else 1e-12, atol=0)
    gs[0].sync_status()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ensemble_pseudo_time_steps_equal_member_steps(precision):
    import paper_2209_04481_gb300 as pg
    gs, Us, Brs = members(precision, shapes=SHAPES[:3], perturb=None)
    U_ens = [torch.from_numpy(U).cuda() for U in Us]
    U_one = [U.clone() for U in U_ens]
    logs = torch.zeros((len(gs), 9), dtype=torch.float64, device="cuda")
    ens = pg.Ensemble(gs)
    ens.pseudo_time_step(U_ens, 5, 0.4, res_log10=logs)
    assert ens.last_launch_count == 10 + (len(gs) if precision == "fp32" else 0)
    for m, g in enumerate(gs):
        log1 = torch.zeros(5 * 9, dtype=torch.float64, device="cuda")
        g.pseudo_time_step(U_one[m], 5, 0.4, res_log10=log1)
        g.sync_status()
        assert torch.equal(U_ens[m], U_one[m]), m
        assert torch.equal(logs[m], log1[36:45]), m


def test_ensemble_rejects_mixed_members():
    import paper_2209_04481_gb300 as pg
    a = pg.Grid(8, 8, 16, precision="fp32")
    b = pg.Grid(8, 8, 16, precision="fp64")
    with pytest.raises(pg.CoronaError, match="precision"):
        pg.Ensemble([a, b])
    c = pg.Grid(8, 8, 16, precision="fp32", limiter="minmod")
    with pytest.raises(pg.CoronaError, match="limiter"):
        pg.Ensemble([a, c])
    e = pg.Ensemble([a])
    with pytest.raises(pg.CoronaError, match="set_inner_boundary"):
        e.residual([torch.zeros((9, 8, 8, 16), device="cuda")])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_ensemble_launches_replay_from_a_cuda_graph(precision):
    """After one call has uploaded the member records, ensemble residual calls
    (a counter memset and the persistent kernel) capture into a CUDA graph whose
    replay gives exactly the direct call's R and norms."""
    import paper_2209_04481_gb300 as pg
    gs, Us, Brs = members(precision)
    Ud = [torch.from_numpy(U).to("cuda", gs[0].dtype) for U in Us]
    n = len(gs)
    ens = pg.Ensemble(gs)
    norms = torch.zeros((n, 9), dtype=torch.float64, device="cuda")
    ref = [R.clone() for R in ens.residual(Ud, norms=norms)]
    ref_norms = norms.clone()
    torch.cuda.synchronize()   # calls on other streams must not overlap this one
    Rs = [torch.zeros_like(u) for u in Ud]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ens.residual(Ud, Rs, norms=norms, stream=s)   # uploads the records for these buffers
    s.synchronize()
    for R in Rs:
        R.zero_()
    norms.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        for _ in range(3):
            ens.residual(Ud, Rs, norms=norms, stream=s)
    graph.replay()
    torch.cuda.synchronize()
    for m in range(n):
        assert torch.equal(Rs[m], ref[m]), m
    assert torch.equal(norms, ref_norms)
    gs[0].sync_status()


# 30 consecutive steps: the master state against the oracle's, relative to how
# far the state moved (FP64: round-off of the steps; FP32 bulk: the residual's
# FP32 error accumulated over the steps, measured below 1e-4)
MARCH_BOUND = {"fp64": 1e-10, "fp32": 5e-4}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ensemble_time_marching_matches_oracle(precision):
    """Time marching with the low-E ghost that keeps the prescribed outflow
    magnitude (Sect. 3.2: the low-E run used the large-E setup apart from
    V_b x B_b = 0): 30 consecutive explicit steps at CFL 0.4 of every member in
    one ensemble call against the oracle's own 30 steps, and the res(a)
    monitor of the last step."""
    import paper_2209_04481_gb300 as pg
    shapes = SHAPES[:3]
    kw = dict(inner_bc="low_e_wp", vr_star=VR_STAR)
    gs, Us, Brs = members(precision, shapes=shapes, perturb=None, **kw)
    U64 = [torch.from_numpy(U.copy()).cuda() for U in Us]
    logs = torch.zeros((len(gs), 9), dtype=torch.float64, device="cuda")
    ens = pg.Ensemble(gs)
    ens.pseudo_time_step(U64, 30, 0.4, res_log10=logs)
    for g in gs:
        g.sync_status()
    for m, shape in enumerate(shapes):
        U_ref, res_ref, _ = oracle.pseudo_time_step(oracle_grid(shape, **kw), Us[m], Brs[m], 30, 0.4)
        change = np.abs(U_ref - Us[m]).reshape(9, -1).max(axis=1)
        err = np.abs(U64[m].cpu().numpy() - U_ref).reshape(9, -1).max(axis=1) / change
        assert np.all(err < MARCH_BOUND[precision]), (m, err)
        np.testing.assert_allclose(logs[m].cpu().numpy(), res_ref[-1],
                                   atol=1e-8 if precision == "fp64" else 1e-3)
    ens.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tile_shapes_keep_the_residual(precision):
    """Every member evaluated with the 16 x 16 tile, and members split between
    the two tile shapes (one persistent launch per shape), give R equal to the
    members' own 8 x 32 launches to rounding and within the oracle bounds."""
    import paper_2209_04481_gb300 as pg
    gs, Us, Brs = members(precision)
    Ud = [torch.from_numpy(U).to("cuda", gs[0].dtype) for U in Us]
    own = []
    for m, g in enumerate(gs):
        own.append(g.residual(Ud[m]).clone())
        g.sync_status()
    ens = pg.Ensemble(gs)
    tol = 1e-13 if precision == "fp64" else 1e-6
    for layout in ("all16", "mixed"):
        for m in range(len(gs)):
            tile = (16, 16) if layout == "all16" or m % 2 else (8, 32)
            ens.set_member_config(m, tile=tile, kchunk=0)
        norms = torch.zeros((len(gs), 9), dtype=torch.float64, device="cuda")
        Rs = ens.residual(Ud, norms=norms)
        assert ens.last_launch_count == (1 if layout == "all16" else 2)
        torch.cuda.synchronize()
        for m, shape in enumerate(SHAPES):
            assert ens.member_config(m)[0] == ((16, 16) if layout == "all16" or m % 2 else (8, 32))
            scale = own[m].abs().amax(dim=(1, 2, 3), keepdim=True)
            assert torch.all((Rs[m] - own[m]).abs() <= tol * scale), (layout, m)
            ref = oracle.residual(oracle_grid(shape), Us[m], Brs[m], want_scale=True)
            err = rel_err(Rs[m].double().cpu().numpy(), ref["R"], ref["scale"])
            assert np.all(err <= (1e-12 if precision == "fp64" else 2e-6)), (layout, m, err)
        ref_n = torch.stack([torch.linalg.vector_norm(R.double().reshape(9, -1), dim=1) for R in Rs])
        torch.testing.assert_close(norms, ref_n, rtol=1e-6 if precision == "fp32" else 1e-12, atol=0)
    gs[0].sync_status()
    ens.close()
