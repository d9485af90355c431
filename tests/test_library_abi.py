"""The C-ABI library builds for sm_103a, loads, exports every declared entry
point and validates descriptors on the host (no GPU needed)."""
import ctypes

import pytest

import paper_2209_04481_gb300 as pg


@pytest.fixture(scope="module")
def lib():
    return pg.load_library()


def test_header_declares_the_boundary():
    names = pg.exported_symbols()
    for required in ("crn_grid_create", "crn_grid_destroy", "crn_set_inner_boundary",
                     "crn_residual", "crn_residual_vjp", "crn_pseudo_time_step",
                     "crn_sync_status", "crn_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in pg.exported_symbols():
        assert hasattr(lib, name), name


def test_descriptor_defaults(lib):
    d = pg.GridDesc()
    assert lib.crn_grid_desc_default(ctypes.byref(d), 128, 64, 128) == 0
    assert (d.n_r, d.n_theta, d.n_phi) == (128, 64, 128)
    assert d.r_in == 1.0 and d.r_out == 21.5 and d.gamma == 1.05 and d.c_h == 1.0
    assert abs(d.g0 - 0.82712) < 1e-4
    assert d.precision == pg.FP32_BULK and d.limiter == pg.LIMITERS["vanalbada"]
    assert d.outer_rho_exp == 2.0 and d.outer_br_exp == 2.0


@pytest.mark.parametrize("field,value,needle", [
    ("n_phi", 12, "n_phi"), ("n_r", 1, "n_r"), ("gamma", 1.0, "gamma"),
    ("r_out", 0.5, "r_in"), ("precision", 7, "precision"), ("limiter", 9, "limiter"),
    ("p_b", -1.0, "p_b"), ("c_h", -1.0, "c_h"), ("lim_eps", 0.0, "van Albada")])
def test_create_rejects_bad_descriptors_before_any_device_work(lib, field, value, needle):
    d = pg.GridDesc()
    lib.crn_grid_desc_default(ctypes.byref(d), 8, 8, 16)
    setattr(d, field, value)
    h = ctypes.c_void_p()
    assert lib.crn_grid_create(ctypes.byref(d), ctypes.byref(h)) == 1  # CRN_E_ARG
    assert h.value is None
    assert needle in lib.crn_last_error().decode()


def test_null_arguments_are_rejected(lib):
    assert lib.crn_residual(None, None, None, None, None, None) == 1
    assert lib.crn_pseudo_time_step(None, None, 1, 0.4, None, None) == 1
    assert lib.crn_grid_destroy(None) == 0


def test_newton_krylov_option_defaults(lib):
    """The NK option structs round-trip through the library (layout check) with
    the CFL law of Sect. 4.1 as default: 2, doubling, up to 128."""
    o = pg.SteadyOptions()
    assert lib.crn_steady_options_default(ctypes.byref(o)) == 0
    assert (o.cfl0, o.cfl_max, o.cfl_double_every, o.max_steps, o.tol_drop) == (2.0, 128.0, 10, 500, 1e-6)
    assert (o.nk.krylov_dim, o.nk.max_restarts, o.nk.lin_rtol, o.nk.fd_rel, o.nk.max_rel_change,
            o.nk.fd_central, o.nk.precond, o.nk.basis_fp32) == (30, 0, 1e-3, 0.0, 0.3, 1, 0, -1)
    n = pg.NkOptions()
    assert lib.crn_nk_options_default(ctypes.byref(n)) == 0
    assert n.krylov_dim == 30 and n.lin_rtol == 1e-3
    assert (n.adjoint_outer, n.adjoint_cfl, n.outer_fp64, n.adjoint_fgmres) == (200, 0.0, 1, 30)
    assert (o.nk.adjoint_outer, o.nk.adjoint_cfl, o.nk.outer_fp64, o.nk.adjoint_fgmres) == (200, 0.0, 1, 30)
    assert lib.crn_newton_krylov_step(None, None, 2.0, None, None, None, None) == 1
    assert lib.crn_steady_solve(None, None, None, None, None, 0, None) == 1


@pytest.mark.parametrize("field,value", [("inner_bc", 3), ("r_last", 0.5), ("r_last", 30.0), ("psi_damp", -1.0)])
def test_create_rejects_bad_boundary_fields(lib, field, value):
    d = pg.GridDesc()
    lib.crn_grid_desc_default(ctypes.byref(d), 8, 8, 16)
    setattr(d, field, value)
    h = ctypes.c_void_p()
    assert lib.crn_grid_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert field in lib.crn_last_error().decode()


def test_ensemble_arguments_checked_on_the_host(lib):
    h = ctypes.c_void_p()
    assert lib.crn_ensemble_create(None, 0, ctypes.byref(h)) == 1
    assert lib.crn_ensemble_residual(None, None, None, None, None, None) == 1
    assert lib.crn_ensemble_set_kchunk(None, 4) == 1
    assert lib.crn_ensemble_destroy(None) == 0


def _makespan(nr, ntiles, slots, kc, overhead):
    """List scheduling of the tiled launch, written independently of the library."""
    import heapq
    nch = -(-nr // kc)
    rem = nr - (nch - 1) * kc
    free = [0] * min(slots, nch * ntiles)
    heapq.heapify(free)
    end = 0
    for y in range(nch):
        dur = (rem if y == nch - 1 else kc) + overhead
        for _ in range(ntiles):
            t = heapq.heappop(free) + dur
            end = max(end, t)
            heapq.heappush(free, t)
    return end


@pytest.mark.parametrize("nr,ntiles,slots", [(128, 32, 304), (128, 32, 152), (96, 18, 304), (32, 2, 304),
                                             (192, 72, 304), (48, 3, 152), (3, 4, 10)])
def test_radial_chunk_minimises_the_makespan(lib, nr, ntiles, slots):
    f = lib.crn_tiled_radial_chunk
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32]
    kc = f(nr, ntiles, slots, 3)
    kmin = min(nr, 4)
    spans = {k: _makespan(nr, ntiles, slots, k, 3) for k in range(kmin, nr + 1)}
    best = min(spans.values())
    assert spans[kc] == best and kc == max(k for k, v in spans.items() if v == best)
    if (nr, ntiles, slots) == (128, 32, 304):
        assert kc == 14          # measured fastest on the 128x64x128 FP32 workload
    if (nr, ntiles, slots) == (128, 32, 152):
        assert kc == 29
    assert f(0, 1, 1, 3) == -1


def test_static_entry_point_rejects_van_albada_without_eps(lib):
    """crn_residual_static validates its descriptor on the host before any
    device work, like crn_grid_create: the smooth van Albada form is 0/0
    where both slopes vanish, so lim_eps must be > 0."""
    f = lib.crn_residual_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(pg.GridDesc)] + [ctypes.c_void_p] * 6
    d = pg.GridDesc()
    lib.crn_grid_desc_default(ctypes.byref(d), 8, 8, 32)
    d.lim_eps = 0.0
    assert f(ctypes.byref(d), None, None, None, None, None, None) == 1  # CRN_E_ARG
    assert "lim_eps" in lib.crn_last_error().decode()
    d.limiter = pg.LIMITERS["minmod"]     # other limiters ignore lim_eps
    assert f(ctypes.byref(d), None, None, None, None, None, None) == 1
    assert "NULL" in lib.crn_last_error().decode()


def test_kernel_selector_values(lib):
    """The descriptor accepts the tiled, cellwise, register-staged and
    TMA-staged kernel values and rejects others before any device work."""
    d = pg.GridDesc()
    lib.crn_grid_desc_default(ctypes.byref(d), 8, 8, 32)
    d.kernel = 7
    h = ctypes.c_void_p()
    assert lib.crn_grid_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert "kernel" in lib.crn_last_error().decode()
    assert (pg.KERNEL_TILED, pg.KERNEL_CELLWISE, pg.KERNEL_TILED_REGS, pg.KERNEL_STAGED) == (0, 1, 2, 3)
    assert lib.crn_last_kernel(None) == -1
