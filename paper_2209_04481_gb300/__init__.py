"""GB300 (sm_103a) library for the MHD + GLM residual of a global coronal model.

Thin Python binding of the C ABI in ``include/corona.h`` (argument marshalling
only: every step of the residual runs in the library's CUDA kernels).  PyTorch
provides device memory and streams.  The library is built in-tree by
``paper_2209_04481_gb300.build`` (nvcc, sm_103a); if it cannot be built or
loaded, importing the binding raises -- there is no CPU fallback.

Paper: arXiv 2209.04481 (Brchnelova et al., "To E or not to E: Numerical
Nuances of Global Coronal Models"): second-order finite volumes with
hyperbolic divergence cleaning (Sect. 2.1), ideal MHD with gravity
(Sect. 2.2), the low-E inner boundary (Sect. 3.2) and the outer extrapolation
laws (Sect. 4.1, Table 2).
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = ["Grid", "Residual", "residual", "load_library", "CoronaError", "FP64", "FP32_BULK",
           "LIMITERS", "KERNEL_TILED", "KERNEL_CELLWISE", "KERNEL_TILED_REGS", "KERNEL_STAGED",
           "exported_symbols"]

FP64, FP32_BULK = 0, 1
KERNEL_TILED, KERNEL_CELLWISE, KERNEL_TILED_REGS, KERNEL_STAGED = 0, 1, 2, 3
LIMITERS = {"none": 0, "minmod": 1, "vanalbada": 2}
_STATUS = {0: "CRN_OK", 1: "CRN_E_ARG", 2: "CRN_E_CUDA", 3: "CRN_E_NONPHYSICAL",
           4: "CRN_E_TIMEOUT", 5: "CRN_E_STATE"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None


class CoronaError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class GridDesc(ctypes.Structure):
    _fields_ = [
        ("n_r", ctypes.c_int32), ("n_theta", ctypes.c_int32), ("n_phi", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("limiter", ctypes.c_int32), ("kernel", ctypes.c_int32),
        ("r_in", ctypes.c_double), ("r_out", ctypes.c_double),
        ("gamma", ctypes.c_double), ("c_h", ctypes.c_double), ("g0", ctypes.c_double),
        ("lim_eps", ctypes.c_double),
        ("outer_rho_exp", ctypes.c_double), ("outer_br_exp", ctypes.c_double),
        ("rho_b", ctypes.c_double), ("p_b", ctypes.c_double),
        ("inner_bc", ctypes.c_int32), ("outer_vr_mass", ctypes.c_int32),
        ("outer_psi_extrap", ctypes.c_int32), ("reserved_", ctypes.c_int32),
        ("vr_star", ctypes.c_double), ("outer_bphi_exp", ctypes.c_double),
        ("outer_vphi_exp", ctypes.c_double), ("r_last", ctypes.c_double),
        ("psi_damp", ctypes.c_double),
    ]


class NkOptions(ctypes.Structure):
    _fields_ = [("krylov_dim", ctypes.c_int32), ("max_restarts", ctypes.c_int32),
                ("lin_rtol", ctypes.c_double), ("fd_rel", ctypes.c_double),
                ("max_rel_change", ctypes.c_double), ("fd_central", ctypes.c_int32),
                ("precond", ctypes.c_int32), ("basis_fp32", ctypes.c_int32),
                ("adjoint_outer", ctypes.c_int32), ("adjoint_cfl", ctypes.c_double),
                ("outer_fp64", ctypes.c_int32), ("adjoint_fgmres", ctypes.c_int32)]


class NkStats(ctypes.Structure):
    _fields_ = [("res_l2", ctypes.c_double), ("lin_rel", ctypes.c_double),
                ("alpha", ctypes.c_double), ("krylov_iters", ctypes.c_int32),
                ("residual_evals", ctypes.c_int32)]


class SteadyOptions(ctypes.Structure):
    _fields_ = [("cfl0", ctypes.c_double), ("cfl_max", ctypes.c_double),
                ("cfl_double_every", ctypes.c_int32), ("max_steps", ctypes.c_int32),
                ("tol_drop", ctypes.c_double), ("nk", NkOptions)]


class SteadyStats(ctypes.Structure):
    _fields_ = [("res0", ctypes.c_double), ("res_final", ctypes.c_double),
                ("steps", ctypes.c_int32), ("krylov_iters", ctypes.c_int32),
                ("residual_evals", ctypes.c_int32), ("converged", ctypes.c_int32)]


def _struct_dict(st):
    return {name: getattr(st, name) for name, _ in st._fields_}


def library_path() -> str:
    from . import build as _build
    return _build.LIB


def load_library(build_if_needed: bool = True):
    """Load libcorona.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build
        if build_if_needed:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libcorona.so is missing and could not be built")
        lib = ctypes.CDLL(_build.LIB)
        vp, i32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
        D = ctypes.POINTER(GridDesc)
        sigs = {
            "crn_grid_desc_default": (ctypes.c_int, [D, i32, i32, i32]),
            "crn_grid_create": (ctypes.c_int, [D, ctypes.POINTER(vp)]),
            "crn_grid_destroy": (ctypes.c_int, [vp]),
            "crn_set_inner_boundary": (ctypes.c_int, [vp, vp, vp]),
            "crn_residual": (ctypes.c_int, [vp, vp, vp, vp, vp, vp]),
            "crn_residual_vjp": (ctypes.c_int, [vp, vp, vp, vp, vp, vp]),
            "crn_pseudo_time_step": (ctypes.c_int, [vp, vp, i32, dbl, vp, vp]),
            "crn_sync_status": (ctypes.c_int, [vp, vp]),
            "crn_last_bad_cell": (ctypes.c_int64, [vp]),
            "crn_last_error": (ctypes.c_char_p, []),
            "crn_last_launch_count": (i32, [vp]),
            "crn_last_kernel": (i32, [vp]),
            "crn_boundary_efield": (ctypes.c_int, [vp, vp, vp, vp]),
            "crn_efield": (ctypes.c_int, [vp, vp, vp, vp]),
            "crn_nk_options_default": (ctypes.c_int, [ctypes.POINTER(NkOptions)]),
            "crn_steady_options_default": (ctypes.c_int, [ctypes.POINTER(SteadyOptions)]),
            "crn_local_dt": (ctypes.c_int, [vp, vp, dbl, vp, vp]),
            "crn_newton_krylov_step": (ctypes.c_int, [vp, vp, dbl, ctypes.POINTER(NkOptions), vp,
                                                      ctypes.POINTER(NkStats), vp]),
            "crn_steady_solve": (ctypes.c_int, [vp, vp, ctypes.POINTER(SteadyOptions),
                                                ctypes.POINTER(SteadyStats), vp, i32, vp]),
            "crn_residual_host_batch": (ctypes.c_int, [vp, vp, vp, vp, vp, i32, vp]),
            "crn_adjoint_solve": (ctypes.c_int, [vp, vp, vp, vp, vp, ctypes.POINTER(NkOptions),
                                                 ctypes.POINTER(NkStats), vp]),
            "crn_ensemble_create": (ctypes.c_int, [vp, i32, ctypes.POINTER(vp)]),
            "crn_ensemble_destroy": (ctypes.c_int, [vp]),
            "crn_ensemble_set_kchunk": (ctypes.c_int, [vp, i32]),
            "crn_ensemble_kchunk": (i32, [vp]),
            "crn_ensemble_set_member_config": (ctypes.c_int, [vp, i32, i32, i32]),
            "crn_ensemble_member_config": (ctypes.c_int, [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
            "crn_ensemble_launch_count": (i32, [vp]),
            "crn_ensemble_residual": (ctypes.c_int, [vp, vp, vp, vp, vp, vp]),
            "crn_ensemble_pseudo_time_step": (ctypes.c_int, [vp, vp, i32, dbl, vp, vp]),
            "crn_ensemble_autotune": (ctypes.c_int, [vp, vp, vp, vp, ctypes.POINTER(i32)]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def exported_symbols():
    """Names of the C ABI functions the header declares (parsed from include/corona.h)."""
    import re
    hdr = os.path.join(os.path.dirname(_HERE), "include", "corona.h")
    with open(hdr) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*[\w\s\*]*?\b(crn_\w+)\s*\(", text, flags=re.M)))


def _check(rc):
    if rc != 0:
        msg = _lib.crn_last_error().decode(errors="replace")
        raise CoronaError(rc, msg)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Grid:
    """A spherical-shell grid on the current CUDA device (``crn_grid``).

    Parameters mirror ``crn_grid_desc``; unspecified ones take the library
    defaults of ``crn_grid_desc_default`` (r in [1, 21.5], gamma = 1.05,
    c_h = 1, solar g0, van Albada, Table 2 case 3 outer law).
    """

    def __init__(self, n_r, n_theta, n_phi, precision="fp32", limiter="vanalbada",
                 kernel="tiled", **kw):
        lib = load_library()
        d = GridDesc()
        _check(lib.crn_grid_desc_default(ctypes.byref(d), n_r, n_theta, n_phi))
        d.precision = {"fp64": FP64, "fp32": FP32_BULK, "fp32_bulk": FP32_BULK}[precision]
        d.limiter = LIMITERS[limiter]
        d.kernel = {"tiled": KERNEL_TILED, "cellwise": KERNEL_CELLWISE, "tiled_regs": KERNEL_TILED_REGS,
                    "staged": KERNEL_STAGED}[kernel]
        if "inner_bc" in kw and isinstance(kw["inner_bc"], str):
            kw["inner_bc"] = {"low_e": 0, "large_e": 1, "low_e_wp": 2}[kw["inner_bc"]]
        for k, v in kw.items():
            if not hasattr(d, k):
                raise TypeError(f"unknown grid parameter {k}")
            setattr(d, k, v)
        self.desc = d
        h = ctypes.c_void_p()
        _check(lib.crn_grid_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.shape = (n_r, n_theta, n_phi)
        self.ncell = n_r * n_theta * n_phi
        self.precision = precision
        self._br = None

    # -- lifetime ----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.crn_grid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.desc.precision == FP64 else torch.float32

    @property
    def last_launch_count(self):
        return int(_lib.crn_last_launch_count(self._h))

    @property
    def last_kernel(self):
        """Kernel of the last residual evaluation: "cellwise", "tiled_regs" or "staged"."""
        k = int(_lib.crn_last_kernel(self._h))
        return {KERNEL_CELLWISE: "cellwise", KERNEL_TILED_REGS: "tiled_regs", KERNEL_STAGED: "staged"}.get(k)

    # -- calls ---------------------------------------------------------------
    @property
    def boundary_shape(self):
        """(n_theta, n_phi) for B_r; (2, n_theta, n_phi) for (B_r, B_theta) with large-E."""
        return (2,) + self.shape[1:] if self.desc.inner_bc == 1 else self.shape[1:]

    def set_inner_boundary(self, Br, stream=None):
        """Prescribe B_r (and B_theta for the large-E form) at the inner face centres."""
        import torch
        if Br.dtype != torch.float64 or not Br.is_cuda or not Br.is_contiguous():
            raise ValueError("Br must be a contiguous float64 CUDA tensor")
        if tuple(Br.shape) != self.boundary_shape:
            raise ValueError(f"Br must have shape {self.boundary_shape}")
        _check(_lib.crn_set_inner_boundary(self._h, _ptr(Br), _stream_handle(stream)))
        self._br = Br

    def _state_check(self, t, name, dtype=None):
        dtype = dtype or self.dtype
        if t.dtype != dtype or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {dtype} CUDA tensor")
        if t.numel() != 9 * self.ncell:
            raise ValueError(f"{name} must hold 9 x {self.shape} elements")

    def residual(self, U, R=None, norms=None, dtmin=None, stream=None):
        """R = dU/dt for U of shape (9, n_r, n_theta, n_phi) in the grid's dtype."""
        import torch
        self._state_check(U, "U")
        if R is None:
            R = torch.empty_like(U)
        self._state_check(R, "R")
        _check(_lib.crn_residual(self._h, _ptr(U), _ptr(R), _ptr(norms), _ptr(dtmin),
                                 _stream_handle(stream)))
        return R

    def residual_vjp(self, U, Rbar, Ubar=None, Brbar=None, want_br=True, stream=None):
        """(Ubar, Brbar) = ((dR/dU)^T Rbar, (dR/dB_r)^T Rbar) through crn_residual_vjp."""
        import torch
        self._state_check(U, "U")
        self._state_check(Rbar, "Rbar")
        if Ubar is None:
            Ubar = torch.empty_like(U)
        if Brbar is None and want_br:
            Brbar = torch.empty(self.boundary_shape, dtype=torch.float64, device=U.device)
        _check(_lib.crn_residual_vjp(self._h, _ptr(U), _ptr(Rbar), _ptr(Ubar), _ptr(Brbar),
                                     _stream_handle(stream)))
        return Ubar, Brbar

    def pseudo_time_step(self, U64, nsteps, cfl, res_log10=None, stream=None):
        """nsteps explicit steps on the FP64 master state U64 (in place)."""
        import torch
        self._state_check(U64, "U64", torch.float64)
        _check(_lib.crn_pseudo_time_step(self._h, _ptr(U64), int(nsteps), float(cfl),
                                         _ptr(res_log10), _stream_handle(stream)))
        return U64

    def boundary_efield(self, U, E=None, stream=None):
        """E = -V_b x B_b at the inner faces, (3, n_theta, n_phi) float64."""
        import torch
        self._state_check(U, "U")
        if E is None:
            E = torch.empty((3,) + self.shape[1:], dtype=torch.float64, device=U.device)
        _check(_lib.crn_boundary_efield(self._h, _ptr(U), _ptr(E), _stream_handle(stream)))
        return E

    def efield(self, U, E=None, stream=None):
        """E = -V x B of every cell, (3, n_r, n_theta, n_phi) float64 (crn_efield)."""
        import torch
        self._state_check(U, "U")
        if E is None:
            E = torch.empty((3,) + self.shape, dtype=torch.float64, device=U.device)
        _check(_lib.crn_efield(self._h, _ptr(U), _ptr(E), _stream_handle(stream)))
        return E

    def local_dt(self, U64, cfl=1.0, out=None, stream=None):
        """cfl x the local pseudo-time step of every cell, (n_r, n_theta, n_phi) float64."""
        import torch
        self._state_check(U64, "U64", torch.float64)
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device=U64.device)
        _check(_lib.crn_local_dt(self._h, _ptr(U64), float(cfl), _ptr(out), _stream_handle(stream)))
        return out

    @staticmethod
    def _nk_options(**kw):
        o = NkOptions()
        _check(_lib.crn_nk_options_default(ctypes.byref(o)))
        for k, v in kw.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown Newton-Krylov option {k}")
            setattr(o, k, v)
        return o

    def newton_krylov_step(self, U64, cfl, dU=None, stream=None, **options):
        """One backward-Euler pseudo-time step solved by Newton-Krylov
        (crn_newton_krylov_step); U64 is updated in place.  Returns the step's
        figures as a dict."""
        import torch
        self._state_check(U64, "U64", torch.float64)
        if dU is not None:
            self._state_check(dU, "dU", torch.float64)
        o = self._nk_options(**options)
        st = NkStats()
        _check(_lib.crn_newton_krylov_step(self._h, _ptr(U64), float(cfl), ctypes.byref(o), _ptr(dU),
                                           ctypes.byref(st), _stream_handle(stream)))
        return _struct_dict(st)

    def adjoint_solve(self, U64, gbar, lam=None, stream=None, **options):
        """dg/dB_b at the steady state U64 for dg/dU = gbar (crn_adjoint_solve):
        returns (sensitivity of the boundary shape, lambda or None, stats dict)."""
        import torch
        self._state_check(U64, "U64", torch.float64)
        self._state_check(gbar, "gbar", torch.float64)
        if lam is not None:
            self._state_check(lam, "lambda", torch.float64)
        sens = torch.empty(self.boundary_shape, dtype=torch.float64, device=U64.device)
        o = self._nk_options(**options)
        st = NkStats()
        _check(_lib.crn_adjoint_solve(self._h, _ptr(U64), _ptr(gbar), _ptr(lam), _ptr(sens), ctypes.byref(o),
                                      ctypes.byref(st), _stream_handle(stream)))
        return sens, lam, _struct_dict(st)

    def steady_solve(self, U64, history_len=None, stream=None, nk=None, **options):
        """Newton-Krylov steps under the CFL law (crn_steady_solve); U64 is
        updated in place.  Returns (stats dict, history array of rows
        (cfl, |R|_2, alpha, krylov_iters))."""
        import numpy as np
        import torch
        self._state_check(U64, "U64", torch.float64)
        o = SteadyOptions()
        _check(_lib.crn_steady_options_default(ctypes.byref(o)))
        for k, v in options.items():
            if not hasattr(o, k) or k == "nk":
                raise TypeError(f"unknown steady-solve option {k}")
            setattr(o, k, v)
        for k, v in (nk or {}).items():
            if not hasattr(o.nk, k):
                raise TypeError(f"unknown Newton-Krylov option {k}")
            setattr(o.nk, k, v)
        n = (o.max_steps + 1) if history_len is None else int(history_len)
        hist = np.zeros((n, 4))
        st = SteadyStats()
        _check(_lib.crn_steady_solve(self._h, _ptr(U64), ctypes.byref(o), ctypes.byref(st),
                                     hist.ctypes.data_as(ctypes.c_void_p), n, _stream_handle(stream)))
        stats = _struct_dict(st)
        passes = stats["steps"] + 1
        return stats, hist[:min(passes, n)]

    def sync_status(self, stream=None):
        """Synchronise and raise CoronaError if a kernel flagged a non-physical state."""
        _check(_lib.crn_sync_status(self._h, _stream_handle(stream)))

    @property
    def last_bad_cell(self):
        return int(_lib.crn_last_bad_cell(self._h))

    def residual_host_batch(self, U_hosts, R_hosts, norms=None, dtmin=None, stream=None):
        """R_hosts[i] = R(U_hosts[i]) for CPU tensors (pinned for overlap) through
        crn_residual_host_batch: copies in/out overlapped with the residuals.
        norms (count, 9) and dtmin (count,) are optional float64 CPU tensors."""
        import torch
        if len(U_hosts) != len(R_hosts):
            raise ValueError("one R buffer per state")
        for t in list(U_hosts) + list(R_hosts):
            if t.is_cuda or t.dtype != self.dtype or not t.is_contiguous() or t.numel() != 9 * self.ncell:
                raise ValueError(f"host buffers must be contiguous {self.dtype} CPU tensors of 9 x {self.shape}")
        for t in (norms, dtmin):
            if t is not None and (t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous()):
                raise ValueError("norms / dtmin must be contiguous float64 CPU tensors")
        _check(_lib.crn_residual_host_batch(self._h, _ptr_array(U_hosts), _ptr_array(R_hosts), _ptr(norms),
                                            _ptr(dtmin), len(U_hosts), _stream_handle(stream)))
        return R_hosts

    def residual_host(self, U_host, R_host, norms=None, dtmin=None, stream=None):
        """End-to-end call on host (pinned) buffers: copy U in, evaluate, copy R out.

        Uses device staging tensors allocated once per grid; the copies and the
        kernel run in order on ``stream``.
        """
        import torch
        if not hasattr(self, "_stage"):
            self._stage = (torch.empty((9,) + self.shape, dtype=self.dtype, device="cuda"),
                           torch.empty((9,) + self.shape, dtype=self.dtype, device="cuda"))
        Ud, Rd = self._stage
        s = stream or torch.cuda.current_stream()
        with torch.cuda.stream(s):
            Ud.copy_(U_host, non_blocking=True)
            self.residual(Ud, Rd, norms, dtmin, stream=s)
            R_host.copy_(Rd, non_blocking=True)
        return R_host


def _make_residual_function():
    import torch

    class Residual(torch.autograd.Function):
        """R = dU/dt as a differentiable function of (U, B_r) on a Grid.

        forward: crn_set_inner_boundary + crn_residual; backward: the
        hand-written adjoint crn_residual_vjp (gradients for U and B_r).
        """

        @staticmethod
        def forward(ctx, U, Br, grid):
            grid.set_inner_boundary(Br)
            R = grid.residual(U.contiguous())
            ctx.save_for_backward(U, Br)
            ctx.grid = grid
            return R

        @staticmethod
        def backward(ctx, Rbar):
            U, Br = ctx.saved_tensors
            grid = ctx.grid
            grid.set_inner_boundary(Br)
            Ubar, Brbar = grid.residual_vjp(U.contiguous(), Rbar.contiguous(),
                                            want_br=ctx.needs_input_grad[1])
            return Ubar, Brbar, None

    return Residual


class _Lazy:
    fn = None


def residual(U, Br, grid):
    """Differentiable residual (see Residual)."""
    if _Lazy.fn is None:
        _Lazy.fn = _make_residual_function()
    return _Lazy.fn.apply(U, Br, grid)


def __getattr__(name):
    if name == "Residual":
        if _Lazy.fn is None:
            _Lazy.fn = _make_residual_function()
        return _Lazy.fn
    raise AttributeError(name)


def _ptr_array(tensors):
    arr = (ctypes.c_void_p * len(tensors))(*[t.data_ptr() for t in tensors])
    return arr


class Ensemble:
    """Many grids (one precision and limiter, any sizes) evaluated by one
    persistent launch (``crn_ensemble_*``).  The grids must outlive the
    ensemble; per-member tensors are passed as lists in member order."""

    def __init__(self, grids):
        lib = load_library()
        self.grids = list(grids)
        hs = (ctypes.c_void_p * len(self.grids))(*[g._h.value for g in self.grids])
        h = ctypes.c_void_p()
        _check(lib.crn_ensemble_create(hs, len(self.grids), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.crn_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def kchunk(self):
        return int(_lib.crn_ensemble_kchunk(self._h))

    @kchunk.setter
    def kchunk(self, k):
        _check(_lib.crn_ensemble_set_kchunk(self._h, int(k)))

    @property
    def last_launch_count(self):
        return int(_lib.crn_ensemble_launch_count(self._h))

    TILES = {0: (8, 32), 1: (16, 16)}

    def member_config(self, m):
        """(tile shape (theta, phi), radial chunk) member m runs with."""
        t, k = ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.crn_ensemble_member_config(self._h, int(m), ctypes.byref(t), ctypes.byref(k)))
        return self.TILES[t.value], k.value

    def set_member_config(self, m, tile=(8, 32), kchunk=0):
        """Tile shape ((8, 32) or (16, 16)) and radial chunk (0: the member's own) of member m."""
        code = {v: c for c, v in self.TILES.items()}[tuple(tile)]
        _check(_lib.crn_ensemble_set_member_config(self._h, int(m), code, int(kchunk)))

    def _check_states(self, Us, name, dtype=None):
        if len(Us) != len(self.grids):
            raise ValueError(f"{name}: one tensor per member")
        for g, U in zip(self.grids, Us):
            g._state_check(U, name, dtype)

    def residual(self, Us, Rs=None, norms=None, dtmin=None, stream=None):
        """Rs[m] = R(Us[m]) for all members in one launch; optional norms
        (n, 9) and dtmin (n,) float64 device tensors."""
        import torch
        self._check_states(Us, "U")
        if Rs is None:
            Rs = [torch.empty_like(U) for U in Us]
        self._check_states(Rs, "R")
        _check(_lib.crn_ensemble_residual(self._h, _ptr_array(Us), _ptr_array(Rs), _ptr(norms), _ptr(dtmin),
                                          _stream_handle(stream)))
        return Rs

    def pseudo_time_step(self, U64s, nsteps, cfl, res_log10=None, stream=None):
        """nsteps explicit steps of every member's FP64 master state (in place)."""
        import torch
        self._check_states(U64s, "U64", torch.float64)
        _check(_lib.crn_ensemble_pseudo_time_step(self._h, _ptr_array(U64s), int(nsteps), float(cfl),
                                                  _ptr(res_log10), _stream_handle(stream)))
        return U64s

    def autotune(self, Us, Rs, stream=None):
        """Time the candidate radial chunks and keep the fastest; returns it."""
        self._check_states(Us, "U")
        self._check_states(Rs, "R")
        k = ctypes.c_int32()
        _check(_lib.crn_ensemble_autotune(self._h, _ptr_array(Us), _ptr_array(Rs), _stream_handle(stream),
                                          ctypes.byref(k)))
        return int(k.value)
