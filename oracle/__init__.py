"""Plain FP64 CPU oracle of the MHD + GLM residual (arXiv 2209.04481).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference arm may import this package.  It shares
no code with ``paper_2209_04481_gb300`` (the CUDA library) and imports nothing
from it; both follow the same definitions, written out independently.

The arithmetic lives in ``corona_oracle.cpp`` (plain scalar C++ loops, face by
face, compiled with ``-ffp-contract=off``); this module compiles it with g++
on first use and marshals numpy arrays through ctypes.

Beyond the residual and its JVP, ``backward_euler_step`` solves the implicit
pseudo-time step of Sect. 2.1 exactly (dense Jacobian from dual-number JVPs,
or scipy's GMRES on them), the definition the GPU Newton-Krylov step is
checked against.

Array layout: conservative state ``U`` of shape ``(9, n0, n1, n2)`` float64,
variables (rho, rho Vx, rho Vy, rho Vz, Bx, By, Bz, E, psi); for the spherical
shell the axes are (r, theta, phi), phi fastest.  ``Br`` has shape
``(n_theta, n_phi)``: the prescribed radial field at the inner face centres.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "corona_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

GEOM_SPHERE, GEOM_BOX = 0, 1
BC_PERIODIC, BC_COPY = 0, 1
LIMITERS = {"none": 0, "minmod": 1, "vanalbada": 2}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (g++, -O2, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Desc(ctypes.Structure):
    _fields_ = [
        ("geom", ctypes.c_int32),
        ("n0", ctypes.c_int32), ("n1", ctypes.c_int32), ("n2", ctypes.c_int32),
        ("r_in", ctypes.c_double), ("r_out", ctypes.c_double),
        ("len0", ctypes.c_double), ("len1", ctypes.c_double), ("len2", ctypes.c_double),
        ("bc0", ctypes.c_int32), ("bc1", ctypes.c_int32), ("bc2", ctypes.c_int32),
        ("limiter", ctypes.c_int32),
        ("lim_eps", ctypes.c_double),
        ("gamma", ctypes.c_double), ("c_h", ctypes.c_double), ("g0", ctypes.c_double),
        ("outer_rho_exp", ctypes.c_double), ("outer_br_exp", ctypes.c_double),
        ("rho_b", ctypes.c_double), ("p_b", ctypes.c_double),
        ("inner_bc", ctypes.c_int32), ("outer_vr_mass", ctypes.c_int32),
        ("outer_psi_extrap", ctypes.c_int32), ("pad_", ctypes.c_int32),
        ("vr_star", ctypes.c_double), ("outer_bphi_exp", ctypes.c_double),
        ("outer_vphi_exp", ctypes.c_double), ("r_last", ctypes.c_double),
        ("psi_damp", ctypes.c_double),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(ctypes.c_double)
            D = ctypes.POINTER(_Desc)
            lib.orc_residual.argtypes = [D, P, P, P, P, P, P, P]
            lib.orc_residual_jvp.argtypes = [D, P, P, P, P, P, P]
            lib.orc_flux.argtypes = [P, P, P, ctypes.c_double, ctypes.c_double, P, P]
            lib.orc_cons_to_prim.argtypes = [D, P, P]
            lib.orc_geometry.argtypes = [D, P, P, P, P]
            lib.orc_ghosts.argtypes = [D, P, P, P, P]
            lib.orc_boundary_efield.argtypes = [D, P, P, P]
            lib.orc_boundary_efield.restype = ctypes.c_int
            lib.orc_efield.argtypes = [D, P, P]
            lib.orc_efield.restype = ctypes.c_int
            lib.orc_local_dt.argtypes = [D, P, P]
            lib.orc_local_dt.restype = ctypes.c_int
            lib.orc_pseudo_time_step.argtypes = [D, P, P, ctypes.c_int, ctypes.c_double, P, P]
            for f in (lib.orc_residual, lib.orc_residual_jvp, lib.orc_flux, lib.orc_cons_to_prim,
                      lib.orc_geometry, lib.orc_ghosts, lib.orc_pseudo_time_step):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclass
class Grid:
    """Problem description: the spherical shell (default) or a Cartesian box.

    Defaults are the solar-wind configuration: r in [1, 21.5] R_sun, gamma = 1.05,
    c_h = 1 (Sect. 3.3), g0 = G M_sun / (R_sun V_ref^2) with V_ref the Alfven speed
    of the Sect. 2.1 reference values, outer law of Table 2 case 3.
    """
    n_r: int = 32
    n_theta: int = 16
    n_phi: int = 32
    r_in: float = 1.0
    r_out: float = 21.5
    gamma: float = 1.05
    c_h: float = 1.0
    g0: float = 0.0
    limiter: str = "vanalbada"
    lim_eps: float = 1e-12
    outer_rho_exp: float = 2.0
    outer_br_exp: float = 2.0
    rho_b: float = 1.0
    p_b: float = 0.0
    inner_bc: str = "low_e"          # "low_e" | "large_e" | "low_e_wp"
    vr_star: float = 0.0
    outer_bphi_exp: float = 0.0
    outer_vphi_exp: float = 0.0
    outer_vr_mass: bool = False
    outer_psi_extrap: bool = False
    r_last: float = 0.0              # > 0: thin last cell [r_last, r_out] (Sect. 4.3)
    psi_damp: float = 0.0            # GLM damping rate alpha (source -alpha psi)
    geom: int = GEOM_SPHERE
    lengths: tuple = (1.0, 1.0, 1.0)
    bcs: tuple = (BC_PERIODIC, BC_PERIODIC, BC_PERIODIC)
    _desc: _Desc = field(default=None, init=False, repr=False)

    @property
    def shape(self):
        return (self.n_r, self.n_theta, self.n_phi)

    @property
    def ncell(self):
        return self.n_r * self.n_theta * self.n_phi

    def desc(self) -> _Desc:
        d = _Desc()
        d.geom = self.geom
        d.n0, d.n1, d.n2 = self.n_r, self.n_theta, self.n_phi
        d.r_in, d.r_out = self.r_in, self.r_out
        d.len0, d.len1, d.len2 = self.lengths
        d.bc0, d.bc1, d.bc2 = self.bcs
        d.limiter = LIMITERS[self.limiter]
        d.lim_eps = self.lim_eps
        d.gamma, d.c_h, d.g0 = self.gamma, self.c_h, self.g0
        d.outer_rho_exp, d.outer_br_exp = self.outer_rho_exp, self.outer_br_exp
        d.rho_b, d.p_b = self.rho_b, self.p_b
        d.inner_bc = {"low_e": 0, "large_e": 1, "low_e_wp": 2}[self.inner_bc]
        d.outer_vr_mass = int(bool(self.outer_vr_mass))
        d.outer_psi_extrap = int(bool(self.outer_psi_extrap))
        d.vr_star = self.vr_star
        d.outer_bphi_exp, d.outer_vphi_exp = self.outer_bphi_exp, self.outer_vphi_exp
        d.r_last = self.r_last
        d.psi_damp = self.psi_damp
        return d

    @property
    def boundary_shape(self):
        """Shape of the inner-boundary input: B_r, or (B_r, B_theta) for large-E."""
        nb = 2 if self.inner_bc == "large_e" else 1
        return (self.n_theta, self.n_phi) if nb == 1 else (2, self.n_theta, self.n_phi)


def box(nx, ny, nz, lengths=(1.0, 1.0, 1.0), bcs=(BC_PERIODIC,) * 3, **kw) -> Grid:
    """Cartesian box grid (axis 0 = x slowest, axis 2 = z fastest); no gravity."""
    return Grid(n_r=nx, n_theta=ny, n_phi=nz, geom=GEOM_BOX, lengths=tuple(lengths),
                bcs=tuple(bcs), g0=0.0, **kw)


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != tuple(shape):
        a = a.reshape(shape)
    return a


def residual(grid: Grid, U, Br=None, want_scale=False, want_bflux=False):
    """Residual R = dU/dt of shape (9, n0, n1, n2), per-variable L2 norms and dtmin.

    Returns a dict with keys ``R``, ``norms`` (9,), ``dtmin`` and optionally
    ``scale`` (flux-magnitude scale, same shape as R) and ``bflux`` ((2, 9): the
    sum of F*|S| over the inner and the outer boundary faces).
    """
    lib = _load()
    U = _f64(U, (9,) + grid.shape)
    if grid.geom == GEOM_SPHERE:
        Br = _f64(Br, grid.boundary_shape)
    R = np.empty_like(U)
    norms = np.empty(9)
    dtmin = np.empty(1)
    scale = np.empty_like(U) if want_scale else None
    bflux = np.empty(18) if want_bflux else None
    d = grid.desc()
    rc = lib.orc_residual(ctypes.byref(d), _ptr(U), _ptr(Br), _ptr(R), _ptr(norms),
                          _ptr(dtmin), _ptr(scale), _ptr(bflux))
    if rc:
        raise ValueError("oracle rejected the problem description")
    out = {"R": R, "norms": norms, "dtmin": float(dtmin[0])}
    if want_scale:
        out["scale"] = scale
    if want_bflux:
        out["bflux"] = bflux.reshape(2, 9)
    return out


def residual_jvp(grid: Grid, U, Br, dU, dBr):
    """(R, dR) with dR = dR/dU . dU + dR/dBr . dBr (forward-mode dual numbers)."""
    lib = _load()
    U = _f64(U, (9,) + grid.shape)
    dU = _f64(dU, (9,) + grid.shape)
    if grid.geom == GEOM_SPHERE:
        Br = _f64(Br, grid.boundary_shape)
        dBr = _f64(dBr, grid.boundary_shape)
    R = np.empty_like(U)
    dR = np.empty_like(U)
    d = grid.desc()
    rc = lib.orc_residual_jvp(ctypes.byref(d), _ptr(U), _ptr(Br), _ptr(dU), _ptr(dBr),
                              _ptr(R), _ptr(dR))
    if rc:
        raise ValueError("oracle rejected the problem description")
    return R, dR


def flux(wl, wr, n, gamma=1.05, c_h=1.0):
    """Rusanov + GLM flux through unit normal n for primitive states; returns (F, lambda)."""
    lib = _load()
    wl, wr, n = _f64(wl), _f64(wr), _f64(n)
    F = np.empty(9)
    lam = np.empty(1)
    lib.orc_flux(_ptr(wl), _ptr(wr), _ptr(n), gamma, c_h, _ptr(F), _ptr(lam))
    return F, float(lam[0])


def cons_to_prim(grid: Grid, U):
    lib = _load()
    U = _f64(U, (9,) + grid.shape)
    W = np.empty_like(U)
    d = grid.desc()
    if lib.orc_cons_to_prim(ctypes.byref(d), _ptr(U), _ptr(W)):
        raise ValueError("bad description")
    return W


def geometry(grid: Grid):
    """Cell volumes and face-area vectors of the three face families."""
    lib = _load()
    n0, n1, n2 = grid.shape
    vol = np.empty((n0, n1, n2))
    S0 = np.empty((n0 + 1, n1, n2, 3))
    S1 = np.empty((n0, n1 + 1, n2, 3))
    S2 = np.empty((n0, n1, n2 + 1, 3))
    d = grid.desc()
    if lib.orc_geometry(ctypes.byref(d), _ptr(vol), _ptr(S0), _ptr(S1), _ptr(S2)):
        raise ValueError("bad description")
    return vol, S0, S1, S2


def ghosts(grid: Grid, U, Br):
    """Primitive ghost planes (inner, outer), each of shape (9, n_theta, n_phi)."""
    lib = _load()
    U = _f64(U, (9,) + grid.shape)
    Br = _f64(Br, grid.boundary_shape)
    Win = np.empty((9, grid.n_theta, grid.n_phi))
    Wout = np.empty_like(Win)
    d = grid.desc()
    if lib.orc_ghosts(ctypes.byref(d), _ptr(U), _ptr(Br), _ptr(Win), _ptr(Wout)):
        raise ValueError("bad description")
    return Win, Wout


def pseudo_time_step(grid: Grid, U, Br, nsteps: int, cfl: float):
    """Explicit pseudo-time steps; returns (U_new, res_log10 (nsteps, 9), dt (nsteps,))."""
    lib = _load()
    U = _f64(U, (9,) + grid.shape).copy()
    if grid.geom == GEOM_SPHERE:
        Br = _f64(Br, grid.boundary_shape)
    res = np.empty((max(nsteps, 1), 9))
    dts = np.empty(max(nsteps, 1))
    d = grid.desc()
    if lib.orc_pseudo_time_step(ctypes.byref(d), _ptr(U), _ptr(Br), int(nsteps), float(cfl),
                                _ptr(res), _ptr(dts)):
        raise ValueError("bad description")
    return U, res[:nsteps], dts[:nsteps]


def local_dt(grid: Grid, U):
    """Local pseudo-time step dt_c = V_c / sum_f max(|V.n_f| + c_f, c_h)|S_f| of
    every cell from its own state, shape (n0, n1, n2)."""
    lib = _load()
    U = _f64(U, (9,) + grid.shape)
    dt = np.empty(grid.shape)
    if lib.orc_local_dt(ctypes.byref(grid.desc()), _ptr(U), _ptr(dt)):
        raise ValueError("bad description")
    return dt


def jacobian(grid: Grid, U, Br=None):
    """Dense dR/dU (9N x 9N, state flattened in SoA order), column by column
    from the dual-number JVP; for grids of a few hundred cells."""
    n = 9 * grid.ncell
    J = np.empty((n, n))
    e = np.zeros(n)
    dB = None if Br is None else np.zeros(np.shape(Br))
    for c in range(n):
        e[c] = 1.0
        J[:, c] = residual_jvp(grid, U, Br, e.reshape((9,) + grid.shape), dB)[1].ravel()
        e[c] = 0.0
    return J


def backward_euler_step(grid: Grid, U, Br, cfl, solver="dense", rtol=1e-12, J=None):
    """One step of the implicit pseudo-time iteration of Sect. 2.1 (backward
    Euler, linearised once, local time steps): the solution dU of

        (diag(1 / (cfl dt_c)) - dR/dU) dU = R(U),

    dt_c from ``local_dt`` (shared by the nine variables of a cell), J = dR/dU
    exact (dual numbers).  cfl = inf gives the Newton step.  solver "dense"
    assembles J and solves directly; "gmres" runs scipy's GMRES on the
    dual-number JVP to ``rtol``.  Returns (dU, R)."""
    U = _f64(U, (9,) + grid.shape)
    R = residual(grid, U, Br)["R"]
    dtau = cfl * local_dt(grid, U)
    diag = np.broadcast_to(1.0 / dtau, U.shape).ravel()
    if solver == "dense":
        if J is None:
            J = jacobian(grid, U, Br)
        dU = np.linalg.solve(np.diag(diag) - J, R.ravel())
    else:
        from scipy.sparse.linalg import LinearOperator, gmres
        dB = None if Br is None else np.zeros(np.shape(Br))

        def apply(x):
            jv = residual_jvp(grid, U, Br, x.reshape(U.shape), dB)[1].ravel()
            return diag * x - jv

        n = U.size
        A = LinearOperator((n, n), matvec=apply, dtype=np.float64)
        dU, info = gmres(A, R.ravel(), rtol=rtol, atol=0.0, restart=200, maxiter=50)
        if info != 0:
            raise RuntimeError(f"GMRES did not reach rtol {rtol} (info {info})")
    return dU.reshape(U.shape), R


def steady_sensitivity(grid: Grid, U, Br, gbar, dBr, rtol=1e-12):
    """Directional sensitivity of g at a steady state R(U*, B) = 0 by the
    implicit function theorem: dg = -gbar . J^-1 (dR/dB . dBr), J = dR/dU at
    U (dual-number JVPs; scipy GMRES on J to rtol)."""
    from scipy.sparse.linalg import LinearOperator, gmres
    U = _f64(U, (9,) + grid.shape)
    zero_b = np.zeros(np.shape(Br))
    v = residual_jvp(grid, U, Br, np.zeros_like(U), dBr)[1].ravel()
    n = U.size
    A = LinearOperator((n, n), matvec=lambda x: residual_jvp(grid, U, Br, x.reshape(U.shape), zero_b)[1].ravel(),
                       dtype=np.float64)
    w, info = gmres(A, v, rtol=rtol, atol=0.0, restart=300, maxiter=100)
    if info != 0:
        raise RuntimeError(f"GMRES did not reach rtol {rtol} (info {info})")
    return -float(np.dot(np.ravel(gbar), w))


def efield(grid: Grid, U):
    """Cell-centred E = -V x B of every cell, shape (3, n_r, n_theta, n_phi)."""
    lib = _load()
    U = _f64(U, (9,) + grid.shape)
    E = np.empty((3,) + grid.shape)
    if lib.orc_efield(ctypes.byref(grid.desc()), _ptr(U), _ptr(E)):
        raise ValueError("bad description")
    return E


def boundary_efield(grid: Grid, U, Br):
    """E = -V_b x B_b of the face-mean state at the inner faces, shape (3, n_theta, n_phi)."""
    lib = _load()
    U = _f64(U, (9,) + grid.shape)
    Br = _f64(Br, grid.boundary_shape)
    E = np.empty((3, grid.n_theta, grid.n_phi))
    d = grid.desc()
    if lib.orc_boundary_efield(ctypes.byref(d), _ptr(U), _ptr(Br), _ptr(E)):
        raise ValueError("bad description")
    return E
