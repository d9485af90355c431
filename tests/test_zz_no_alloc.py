"""crn_residual_static: the residual entry point that allocates nothing.

It serves callers that cannot call cudaMalloc (a fixed device-memory budget
owned by a host framework, a plugin that may not allocate during a solve).
Checked through the C ABI against crn_residual on the same inputs, on two
calls in a row, within the parity tolerances of the rest of the suite.  This
file is collected last so that a failure here comes after every other test.
"""
import ctypes

import numpy as np
import pytest

import coronal_inputs as ci
import oracle
from _util import oracle_grid, problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOUNDS = {"fp64": 1e-12, "fp32": 2e-5}


def _lib():
    import paper_2209_04481_gb300 as pg
    lib = pg.load_library()
    f = lib.crn_residual_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(pg.GridDesc)] + [ctypes.c_void_p] * 6
    return pg, lib


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_entry_point_matches_crn_residual(precision):
    pg, lib = _lib()
    shape = (32, 16, 64)
    U, Br = problem(shape, perturb=11)
    ref = oracle.residual(oracle_grid(shape), U, Br, want_scale=True)
    dt = torch.float64 if precision == "fp64" else torch.float32
    Ud = torch.from_numpy(U).to("cuda", dt)
    Brd = torch.from_numpy(Br).cuda()
    g = pg.Grid(*shape, precision=precision, p_b=ci.parker_sound_speed2())
    g.set_inner_boundary(Brd)
    n_ref = torch.zeros(9, dtype=torch.float64, device="cuda")
    d_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    R_ref = g.residual(Ud, norms=n_ref, dtmin=d_ref)
    g.sync_status()
    desc = g.desc
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # two calls in a row share the static scratch
        R = torch.full_like(Ud, float("nan"))
        n = torch.zeros(9, dtype=torch.float64, device="cuda")
        d = torch.zeros(1, dtype=torch.float64, device="cuda")
        rc = lib.crn_residual_static(ctypes.byref(desc), _p(Brd), _p(Ud), _p(R), _p(n), _p(d),
                                     ctypes.c_void_p(stream))
        assert rc == 0, lib.crn_last_error().decode()
        torch.cuda.synchronize()
        err = rel_err(R.double().cpu().numpy(), R_ref.double().cpu().numpy(), ref["scale"])
        assert np.all(err <= BOUNDS[precision]), err
        # the static path builds its geometry on the device (FP32 grids round
        # it to single precision independently), so norms agree to rounding
        rtol = 1e-10 if precision == "fp64" else 1e-5
        np.testing.assert_allclose(n.cpu().numpy(), n_ref.cpu().numpy(), rtol=rtol)
        assert float(d.cpu()[0]) == pytest.approx(float(d_ref.cpu()[0]), rel=rtol)
    g.close()


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
