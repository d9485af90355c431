"""crn_residual_static: the residual entry point that allocates nothing.

It serves callers that cannot call cudaMalloc (a fixed device-memory budget
owned by a host framework, a plugin that may not allocate during a solve).
Checked through the C ABI against the FP64 oracle element by element (its
geometry is built on the device, independently of crn_grid_create's host
geometry) and against crn_residual on the same inputs, on two calls in a row,
for every limiter and inner boundary and a ragged shape; then across geometry
changes at the same sizes, and with a call recorded in a CUDA graph that is
replayed after a call with another geometry.  This file is collected last so
that a failure here comes after every other test.
"""
import ctypes

import numpy as np
import pytest

import coronal_inputs as ci
import oracle
from _util import check_fp32, oracle_grid, problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOUNDS = {"fp64": 1e-12, "fp32": 2e-5}
VR_STAR = 1935.07 / ci.V_REF
INNER = {"low_e": {}, "large_e": dict(inner_bc="large_e", vr_star=VR_STAR),
         "low_e_wp": dict(inner_bc="low_e_wp", vr_star=VR_STAR)}


def _lib():
    import paper_2209_04481_gb300 as pg
    lib = pg.load_library()
    f = lib.crn_residual_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(pg.GridDesc)] + [ctypes.c_void_p] * 6
    return pg, lib


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _inputs(shape, inner, seed=11):
    U, Br = problem(shape, perturb=seed)
    if inner == "large_e":
        Br = ci.potential_field(shape[1], shape[2], lmax=6, seed=11)
    return U, Br


def _static(lib, desc, Brd, Ud, stream=None):
    R = torch.full_like(Ud, float("nan"))
    n = torch.zeros(9, dtype=torch.float64, device="cuda")
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = lib.crn_residual_static(ctypes.byref(desc), _p(Brd), _p(Ud), _p(R), _p(n), _p(d),
                                 ctypes.c_void_p(st.cuda_stream))
    assert rc == 0, lib.crn_last_error().decode()
    return R, n, d


@pytest.mark.parametrize("shape", [(32, 16, 64), (24, 12, 40)])
@pytest.mark.parametrize("inner", list(INNER))
@pytest.mark.parametrize("limiter", ["vanalbada", "minmod", "none"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_entry_point_matches_oracle_and_crn_residual(precision, limiter, inner, shape):
    pg, lib = _lib()
    kw = INNER[inner]
    U, Br = _inputs(shape, inner)
    ref = oracle.residual(oracle_grid(shape, limiter=limiter, **kw), U, Br, want_scale=True)
    assert np.all(np.isfinite(ref["R"]))  # the input keeps every reconstructed state physical
    dt = torch.float64 if precision == "fp64" else torch.float32
    Ud = torch.from_numpy(U).to("cuda", dt)
    Brd = torch.from_numpy(np.ascontiguousarray(Br)).cuda()
    g = pg.Grid(*shape, precision=precision, limiter=limiter, p_b=ci.parker_sound_speed2(), **kw)
    g.set_inner_boundary(Brd)
    n_ref = torch.zeros(9, dtype=torch.float64, device="cuda")
    d_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    R_ref = g.residual(Ud, norms=n_ref, dtmin=d_ref)
    g.sync_status()
    desc = g.desc
    for _ in range(2):  # two calls in a row share the static scratch
        R, n, d = _static(lib, desc, Brd, Ud)
        torch.cuda.synchronize()
        Rh = R.double().cpu().numpy()
        # the oracle directly: the device-built geometry is pinned on its own
        if precision == "fp32":
            check_fp32(Rh, ref, oracle_grid(shape, limiter=limiter, **kw), U, n.cpu().numpy(),
                       float(d.cpu()[0]))
        else:
            err = rel_err(Rh, ref["R"], ref["scale"])
            assert np.all(err <= BOUNDS[precision]), err
            np.testing.assert_allclose(n.cpu().numpy(), ref["norms"], rtol=1e-10)
        # crn_residual: the same kernel on the host-built geometry
        err = rel_err(Rh, R_ref.double().cpu().numpy(), ref["scale"])
        assert np.all(err <= BOUNDS[precision]), err
        rtol = 1e-10 if precision == "fp64" else 1e-5
        np.testing.assert_allclose(n.cpu().numpy(), n_ref.cpu().numpy(), rtol=rtol)
        assert float(d.cpu()[0]) == pytest.approx(float(d_ref.cpu()[0]), rel=rtol)
    g.close()


def _desc_for(pg, shape, precision, **kw):
    d = pg.GridDesc()
    pg.load_library().crn_grid_desc_default(ctypes.byref(d), *shape)
    d.precision = pg.FP64 if precision == "fp64" else pg.FP32_BULK
    d.p_b = ci.parker_sound_speed2()
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_geometry_follows_each_call(precision):
    """Same sizes, r_out changed and changed back (and g0 changed): every call
    uses its own descriptor's geometry, checked against the oracle."""
    pg, lib = _lib()
    shape = (12, 8, 32)
    U, Br = problem(shape, perturb=3)
    dt = torch.float64 if precision == "fp64" else torch.float32
    Ud = torch.from_numpy(U).to("cuda", dt)
    Brd = torch.from_numpy(Br).cuda()
    for r_out, g0 in ((21.5, ci.G0_SOLAR), (30.0, ci.G0_SOLAR), (21.5, ci.G0_SOLAR), (21.5, 0.5)):
        desc = _desc_for(pg, shape, precision, r_out=r_out, g0=g0)
        R, n, _ = _static(lib, desc, Brd, Ud)
        torch.cuda.synchronize()
        ref = oracle.residual(oracle_grid(shape, r_out=r_out, g0=g0), U, Br, want_scale=True)
        err = rel_err(R.double().cpu().numpy(), ref["R"], ref["scale"])
        assert np.all(err <= BOUNDS[precision]), (r_out, g0, err)


def test_static_call_in_a_graph_keeps_its_geometry():
    """A call captured in a CUDA graph replays with the geometry it was
    captured with, after direct calls with another geometry."""
    pg, lib = _lib()
    shape = (12, 8, 32)
    U, Br = problem(shape, perturb=6)
    Ud = torch.from_numpy(U).to("cuda", torch.float64)
    Brd = torch.from_numpy(Br).cuda()
    dA = _desc_for(pg, shape, "fp64", r_out=21.5)
    dB = _desc_for(pg, shape, "fp64", r_out=30.0)
    _static(lib, dA, Brd, Ud)             # first call on the device: set-up, outside the capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    R = torch.full_like(Ud, float("nan"))
    n = torch.zeros(9, dtype=torch.float64, device="cuda")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        rc = lib.crn_residual_static(ctypes.byref(dA), _p(Brd), _p(Ud), _p(R), _p(n), None,
                                     ctypes.c_void_p(s.cuda_stream))
    assert rc == 0, lib.crn_last_error().decode()
    _static(lib, dB, Brd, Ud)             # another geometry, built directly
    torch.cuda.synchronize()
    graph.replay()
    torch.cuda.synchronize()
    refA = oracle.residual(oracle_grid(shape, r_out=21.5), U, Br, want_scale=True)
    assert np.all(rel_err(R.cpu().numpy(), refA["R"], refA["scale"]) <= BOUNDS["fp64"])
    # and a direct call after the replay uses its own geometry again
    RB, _, _ = _static(lib, dB, Brd, Ud)
    torch.cuda.synchronize()
    refB = oracle.residual(oracle_grid(shape, r_out=30.0), U, Br, want_scale=True)
    assert np.all(rel_err(RB.cpu().numpy(), refB["R"], refB["scale"]) <= BOUNDS["fp64"])


def test_static_entry_point_rejects_oversized_grids():
    pg, lib = _lib()
    d = pg.GridDesc()
    lib.crn_grid_desc_default(ctypes.byref(d), 16, 256, 256)   # 65536 columns > 32768
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = lib.crn_residual_static(ctypes.byref(d), _p(x), _p(x), ctypes.c_void_p(x.data_ptr() + 8192),
                                 None, None, None)
    assert rc == 1
    assert "32768" in lib.crn_last_error().decode()


def test_static_entry_point_rejects_thin_last_cell():
    """The thin-outer-cell mesh (r_last != 0) is a crn_grid_create option only."""
    pg, lib = _lib()
    d = pg.GridDesc()
    lib.crn_grid_desc_default(ctypes.byref(d), 8, 8, 32)
    d.r_out, d.r_last = 25.0, 24.95
    x = torch.zeros(9 * 8 * 8 * 32, dtype=torch.float32, device="cuda")
    br = torch.zeros(8 * 32, dtype=torch.float64, device="cuda")
    rc = lib.crn_residual_static(ctypes.byref(d), _p(br), _p(x), _p(torch.empty_like(x)),
                                 None, None, None)
    assert rc == 1
    assert "r_last" in lib.crn_last_error().decode()
