"""Seeded synthetic inputs for the coronal MHD residual (arXiv 2209.04481).

This module holds no arithmetic of the method itself (no fluxes, ghosts,
reconstruction or geometry of the finite-volume operator).  It only builds the
INPUTS that both the CUDA library and the CPU oracle consume, in place of the
paper's MDI magnetogram and converged states, which are not available:

* ``parker_mach``      isothermal Parker wind Mach number, transonic branch
                       (the paper's initial velocity is a fit of it, Sect. 3.1);
* ``background``       Parker wind + aligned dipole state (Sect. 3.2's steady
                       dipole set-up), conservative SoA float64;
* ``magnetogram``      dipole + seeded real spherical-harmonic field l <= lmax,
                       coefficient variance ~ l^-2, scaled to a given max |B_r|;
* ``perturb``          1 % seeded Gaussian perturbation of a state;
* ``cotangent``        seeded N(0, 1) residual cotangent.

Units: lengths in R_sun, speeds in units of the Alfven speed of the Sect. 2.1
reference values (rho_ref = 1.67e-13 kg/m^3, B_ref = 2.2e-4 T).
"""
from __future__ import annotations

import math

import numpy as np

# Sect. 2.1 reference values and the derived dimensionless gravity constant.
RHO_REF = 1.67e-13            # kg m^-3
B_REF = 2.2e-4                # T
MU0 = 4e-7 * math.pi
V_REF = B_REF / math.sqrt(MU0 * RHO_REF)   # Alfven speed, 4.80e5 m/s
GM_SUN = 1.3271244e20         # m^3 s^-2
R_SUN = 6.957e8               # m
G0_SOLAR = GM_SUN / (R_SUN * V_REF ** 2)   # 0.827

GAMMA = 1.05
R_IN, R_OUT = 1.0, 21.5
PARKER_RC = 5.0               # sonic-point radius of the background wind


def radial_faces(n_r, r_in=R_IN, r_out=R_OUT, r_last=None):
    """Geometric radial stretch r_k = r_in (r_top/r_in)^(k/M), k = 0..M.

    Without ``r_last``: M = N_r, r_top = r_out.  With it (the mesh of Sect. 4.3
    with a thin outermost cell): M = N_r - 1 cells up to r_top = r_last, then
    one cell [r_last, r_out].
    """
    M = n_r - 1 if r_last else n_r
    r_top = r_last if r_last else r_out
    k = np.arange(M + 1, dtype=np.float64)
    rf = r_in * (r_top / r_in) ** (k / M)
    rf[0], rf[-1] = r_in, r_top
    if r_last:
        rf = np.append(rf, r_out)
    return rf


def cell_centres(n_r, n_theta, n_phi, r_in=R_IN, r_out=R_OUT, r_last=None):
    """Coordinate midpoints (r_c, theta_c, phi_c) as 1D arrays."""
    rf = radial_faces(n_r, r_in, r_out, r_last)
    rc = 0.5 * (rf[:-1] + rf[1:])
    tf = math.pi * np.arange(n_theta + 1) / n_theta
    pf = 2.0 * math.pi * np.arange(n_phi + 1) / n_phi
    return rc, 0.5 * (tf[:-1] + tf[1:]), 0.5 * (pf[:-1] + pf[1:])


def parker_mach(r, r_c=PARKER_RC):
    """Mach number M = v/c_s of the transonic isothermal Parker wind.

    Solves M^2 - ln M^2 = 4 ln(r/r_c) + 4 r_c/r - 3 with M < 1 inside r_c and
    M > 1 outside, by bisection in ln M to full double precision.
    """
    r = np.asarray(r, dtype=np.float64)
    rhs = 4.0 * np.log(r / r_c) + 4.0 * r_c / r - 3.0
    sup = r > r_c
    lo = np.where(sup, 0.0, -60.0)
    hi = np.where(sup, 10.0, 0.0)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        f = np.exp(2.0 * mid) - 2.0 * mid - rhs
        # f is decreasing in ln M on the subsonic branch, increasing on the supersonic
        go_up = np.where(sup, f < 0.0, f > 0.0)
        lo = np.where(go_up, mid, lo)
        hi = np.where(go_up, hi, mid)
    return np.exp(0.5 * (lo + hi))


def parker_sound_speed2(g0=G0_SOLAR, r_c=PARKER_RC):
    """c_s^2 = g0 / (2 r_c): the sonic point of an isothermal wind."""
    return g0 / (2.0 * r_c)


def dipole_field(r, theta, phi):
    """Aligned dipole with |B| = 1 at the pole of r = 1: B_r = cos t / r^3, B_t = sin t / (2 r^3)."""
    br = np.cos(theta) / r ** 3
    bt = 0.5 * np.sin(theta) / r ** 3
    st, ct, sp, cp = np.sin(theta), np.cos(theta), np.sin(phi), np.cos(phi)
    bx = br * st * cp + bt * ct * cp
    by = br * st * sp + bt * ct * sp
    bz = br * ct - bt * st
    return bx, by, bz


def background(n_r, n_theta, n_phi, gamma=GAMMA, g0=G0_SOLAR, r_c=PARKER_RC,
               r_in=R_IN, r_out=R_OUT, r_last=None, efree=False):
    """Parker wind + aligned dipole on cell centres.

    Returns (U, info): U is the conservative SoA state of shape
    (9, n_r, n_theta, n_phi) float64; info holds rho_b, p_b (the inner boundary
    density and pressure: the wind at r = r_in), c_s^2 and the primitives.

    ``efree``: the electric-field-free start of Sect. 3.1 -- the Parker speed is
    kept but the velocity is turned along the field, V = v sgn(B_r) B/|B|
    (sgn 0 = +1), so that V x B = 0 in every cell.  Otherwise V is radial.
    """
    rc, tc, pc = cell_centres(n_r, n_theta, n_phi, r_in, r_out, r_last)
    R, T, P = np.meshgrid(rc, tc, pc, indexing="ij")
    cs2 = parker_sound_speed2(g0, r_c)
    cs = math.sqrt(cs2)
    m_in = float(parker_mach(np.array([r_in]), r_c)[0])
    mach = np.broadcast_to(parker_mach(rc, r_c)[:, None, None], R.shape)
    v = mach * cs
    rho = (m_in / mach) * (r_in / R) ** 2        # rho v r^2 = const, rho(r_in) = 1
    p = rho * cs2
    st, ct, sp, cp = np.sin(T), np.cos(T), np.sin(P), np.cos(P)
    bx, by, bz = dipole_field(R, T, P)
    if efree:
        bmag = np.sqrt(bx * bx + by * by + bz * bz)
        br = bx * st * cp + by * st * sp + bz * ct
        f = v * np.where(br < 0.0, -1.0, 1.0) / bmag
        vx, vy, vz = f * bx, f * by, f * bz
    else:
        vx, vy, vz = v * st * cp, v * st * sp, v * ct
    W = np.stack([rho, vx, vy, vz, bx, by, bz, p, np.zeros_like(rho)])
    U = prim_to_cons(W, gamma)
    info = {"rho_b": 1.0, "p_b": cs2, "cs2": cs2, "W": W}
    return U, info


def prim_to_cons(W, gamma=GAMMA):
    """Conservative variables of a primitive SoA array (input construction only)."""
    rho, vx, vy, vz, bx, by, bz, p, psi = W
    E = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) \
        + 0.5 * (bx * bx + by * by + bz * bz)
    return np.stack([rho, rho * vx, rho * vy, rho * vz, bx, by, bz, E, psi])


def _normalised_legendre(lmax, x):
    """Fully normalised associated Legendre functions Pbar[l][m](x), m >= 0.

    Normalised so that Pbar_lm(cos t) * {1 (m = 0) | sqrt(2) cos(m phi) |
    sqrt(2) sin(m phi)} are orthonormal on the unit sphere.
    """
    x = np.asarray(x, dtype=np.float64)
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    P = [[None] * (lmax + 1) for _ in range(lmax + 1)]
    P[0][0] = np.full_like(x, 1.0 / math.sqrt(4.0 * math.pi))
    for m in range(1, lmax + 1):
        P[m][m] = math.sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * P[m - 1][m - 1]
    for m in range(0, lmax):
        P[m + 1][m] = math.sqrt(2.0 * m + 3.0) * x * P[m][m]
    for m in range(0, lmax + 1):
        for l in range(m + 2, lmax + 1):
            a = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
            b = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
            P[l][m] = a * (x * P[l - 1][m] - b * P[l - 2][m])
    return P


def real_sh(lmax, theta, phi):
    """Orthonormal real spherical harmonics, list of (l, m, Y) in (l asc, m = -l..l) order."""
    P = _normalised_legendre(lmax, np.cos(theta))
    out = []
    for l in range(0, lmax + 1):
        for m in range(-l, l + 1):
            if m == 0:
                Y = P[l][0]
            elif m > 0:
                Y = math.sqrt(2.0) * P[l][m] * np.cos(m * phi)
            else:
                Y = math.sqrt(2.0) * P[l][-m] * np.sin(-m * phi)
            out.append((l, m, Y))
    return out


def potential_field(n_theta, n_phi, lmax=15, seed=2209, target_max=5.0, dipole_only=False,
                    dtheta=1e-6):
    """(B_r, B_theta) at r = 1 of the source-free exterior potential field whose
    radial component is ``magnetogram(...)``: B = -grad Phi with
    Phi = sum_lm a_lm r^-(l+1) Y_lm / (l + 1), so B_theta(r=1) =
    -sum_lm a_lm / (l + 1) dY_lm/dtheta (the dipole part cos(theta) gives
    sin(theta)/2).  It stands in for the PFSS B_theta that the paper's large-E
    boundary prescribes (Sect. 3.2).  Returns shape (2, n_theta, n_phi)."""
    br = magnetogram(n_theta, n_phi, lmax=lmax, seed=seed, target_max=target_max,
                     dipole_only=dipole_only)
    _, tc, pc = cell_centres(2, n_theta, n_phi)
    T, P = np.meshgrid(tc, pc, indexing="ij")
    bt = 0.5 * np.sin(T)
    if not dipole_only:
        scale = _magnetogram_scale(n_theta, n_phi, lmax, seed, target_max)
        rng = np.random.default_rng(seed)
        hi = real_sh(lmax, T + dtheta, P)
        lo = real_sh(lmax, T - dtheta, P)
        for (l, m, Yp), (_, _, Ym) in zip(hi, lo):
            if l == 0:
                continue
            a = rng.standard_normal() / l
            bt -= scale * a / (l + 1) * (Yp - Ym) / (2.0 * dtheta)
    return np.stack([br, bt])


def potential_background(n_r, n_theta, n_phi, lmax=15, seed=2209, target_max=5.0, dipole_only=False,
                         efree=False, gamma=GAMMA, g0=G0_SOLAR, r_c=PARKER_RC, r_in=R_IN, r_out=R_OUT,
                         dtheta=1e-6):
    """Parker wind with the source-free potential field of the magnetogram.

    The field is B = -grad Phi, Phi = cos(theta) / (2 r^2) + s sum_lm a_lm
    r^-(l+1) Y_lm / (l + 1) with the coefficients and scale of
    ``magnetogram(...)``, so that B_r at r = r_in = 1 is that magnetogram: the
    dipole part is the aligned dipole of ``background`` and each further
    multipole falls as r^-(l+2).  It stands in for the PFSS initial field the
    paper starts from (Sect. 3.1): the initial state then agrees with the
    prescribed inner B_r instead of jumping from it to the dipole.
    ``efree`` turns the wind velocity along B as in ``background``.
    Returns (U, info) like ``background``."""
    U, info = background(n_r, n_theta, n_phi, gamma=gamma, g0=g0, r_c=r_c, r_in=r_in, r_out=r_out)
    W = info["W"].copy()
    if not dipole_only:
        rc, tc, pc = cell_centres(n_r, n_theta, n_phi, r_in, r_out)
        T, P = np.meshgrid(tc, pc, indexing="ij")
        scale = _magnetogram_scale(n_theta, n_phi, lmax, seed, target_max)
        rng = np.random.default_rng(seed)
        ys = real_sh(lmax, T, P)
        hi = real_sh(lmax, T + dtheta, P)
        lo = real_sh(lmax, T - dtheta, P)
        by_l = {}
        for (l, m, Y), (_, _, Yp), (_, _, Ym) in zip(ys, hi, lo):
            if l == 0:
                continue
            a = scale * rng.standard_normal() / l
            gr, gt, gp = by_l.setdefault(l, [np.zeros_like(T), np.zeros_like(T), np.zeros_like(T)])
            gr += a * Y
            gt += -a / (l + 1) * (Yp - Ym) / (2.0 * dtheta)
            gp += -a / (l + 1) * _dphi_real_sh(l, m, T, P) / np.sin(T)
        R = rc[:, None, None]
        br = np.zeros((n_r, n_theta, n_phi))
        bt = np.zeros_like(br)
        bp = np.zeros_like(br)
        for l, (gr, gt, gp) in by_l.items():
            f = R ** (-(l + 2))
            br += f * gr[None]
            bt += f * gt[None]
            bp += f * gp[None]
        st, ct, sp, cp = np.sin(T), np.cos(T), np.sin(P), np.cos(P)
        W[4] += br * (st * cp)[None] + bt * (ct * cp)[None] - bp * sp[None]
        W[5] += br * (st * sp)[None] + bt * (ct * sp)[None] + bp * cp[None]
        W[6] += br * ct[None] - bt * st[None]
    if efree:
        rc, tc, pc = cell_centres(n_r, n_theta, n_phi, r_in, r_out)
        R3, T3, P3 = np.meshgrid(rc, tc, pc, indexing="ij")
        v = np.sqrt(W[1] ** 2 + W[2] ** 2 + W[3] ** 2)
        bmag = np.sqrt(W[4] ** 2 + W[5] ** 2 + W[6] ** 2)
        brad = W[4] * np.sin(T3) * np.cos(P3) + W[5] * np.sin(T3) * np.sin(P3) + W[6] * np.cos(T3)
        f = v * np.where(brad < 0.0, -1.0, 1.0) / bmag
        W[1], W[2], W[3] = f * W[4], f * W[5], f * W[6]
    info = dict(info, W=W)
    return prim_to_cons(W, gamma), info


def _dphi_real_sh(l, m, theta, phi):
    """d/dphi of the orthonormal real harmonic Y_lm of ``real_sh``."""
    if m == 0:
        return np.zeros_like(theta)
    P = _normalised_legendre(l, np.cos(theta))[l][abs(m)]
    if m > 0:
        return -m * math.sqrt(2.0) * P * np.sin(m * phi)
    return -m * math.sqrt(2.0) * P * np.cos(-m * phi)


def _magnetogram_scale(n_theta, n_phi, lmax, seed, target_max):
    """The factor s of magnetogram(): max |cos(theta) + s f| = target_max."""
    _, tc, pc = cell_centres(2, n_theta, n_phi)
    T, P = np.meshgrid(tc, pc, indexing="ij")
    dip = np.cos(T)
    rng = np.random.default_rng(seed)
    f = np.zeros_like(T)
    for (l, m, Y) in real_sh(lmax, T, P):
        if l == 0:
            continue
        f += (rng.standard_normal() / l) * Y

    def peak(s):
        return float(np.max(np.abs(dip + s * f)))
    hi = 1.0
    while peak(hi) < target_max:
        hi *= 2.0
    lo = 0.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if peak(mid) < target_max:
            lo = mid
        else:
            hi = mid
    return hi


def magnetogram(n_theta, n_phi, lmax=15, seed=2209, target_max=5.0, dipole_only=False):
    """Prescribed inner-boundary B_r at the inner face centres, shape (n_theta, n_phi).

    B_r = cos(theta) + s f(theta, phi), f = sum_{l=1..lmax} sum_m a_lm Y_lm with
    a_lm = N(0, 1)/l drawn in (l ascending, m = -l..l) order from
    numpy.random.default_rng(seed); s > 0 is the unique root of max |B_r| = target_max.
    ``dipole_only`` returns cos(theta).
    """
    _, tc, pc = cell_centres(2, n_theta, n_phi)
    T, P = np.meshgrid(tc, pc, indexing="ij")
    dip = np.cos(T)
    if dipole_only:
        return dip
    rng = np.random.default_rng(seed)
    f = np.zeros_like(T)
    for (l, m, Y) in real_sh(lmax, T, P):
        if l == 0:
            continue
        f += (rng.standard_normal() / l) * Y
    def peak(s):
        return float(np.max(np.abs(dip + s * f)))
    hi = 1.0
    while peak(hi) < target_max:
        hi *= 2.0
    lo = 0.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if peak(mid) < target_max:
            lo = mid
        else:
            hi = mid
    return dip + hi * f


def perturb(W, seed=3, amp=0.01, gamma=GAMMA):
    """Perturbed conservative state from a primitive state W (9, ...).

    rho, V, B and p are multiplied component-wise by (1 + amp xi), xi ~ N(0, 1)
    from numpy.random.default_rng(seed); psi = amp xi |B|.
    """
    W = np.asarray(W, dtype=np.float64)
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal(W.shape)
    Wp = W * (1.0 + amp * xi)
    bmag = np.sqrt(W[4] ** 2 + W[5] ** 2 + W[6] ** 2)
    Wp[8] = amp * xi[8] * bmag
    return prim_to_cons(Wp, gamma)


def cotangent(shape, seed=4):
    """N(0, 1) cotangent of the residual, one value per cell and variable."""
    return np.random.default_rng(seed).standard_normal(shape)


def workload(name):
    """Named synthetic workloads (sizes and inputs of the measured configurations).

    'shell32'  : 32 x 16 x 32, inner B_r = dipole (pseudo-time stepping case);
    'shell128' : 128 x 64 x 128, inner B_r = dipole + l <= 15 field, seed 2209;
    'shell64'  : 64 x 32 x 64, shell32-type background + 1 % perturbation (seed 3);
    'shell96'  : 96 x 48 x 96, magnetogram as shell128.
    Returns dict(shape, U, Br, rho_b, p_b).
    """
    shapes = {"shell32": (32, 16, 32), "shell128": (128, 64, 128),
              "shell64": (64, 32, 64), "shell96": (96, 48, 96)}
    shape = shapes[name]
    U, info = background(*shape)
    if name == "shell32":
        Br = magnetogram(shape[1], shape[2], dipole_only=True)
    elif name == "shell64":
        Br = magnetogram(shape[1], shape[2], dipole_only=True)
        U = perturb(info["W"], seed=3)
    else:
        Br = magnetogram(shape[1], shape[2], seed=2209)
    return {"shape": shape, "U": U, "Br": Br, "rho_b": info["rho_b"], "p_b": info["p_b"]}


def ensemble_members(n=32, seed=5):
    """Shapes and magnetogram seeds of the ensemble workload: n shells with
    N_r ~ U{48..192} and (N_theta, N_phi) drawn uniformly from {24 x 48,
    48 x 96, 96 x 192} (numpy default_rng(seed), N_r first, then the angular
    choice); member m takes magnetogram seed m (l <= min(15, N_theta / 2),
    max |B_r| = 5).  Returns a list of (shape, magnetogram seed)."""
    rng = np.random.default_rng(seed)
    nr = rng.integers(48, 193, size=n)
    ang = rng.integers(0, 3, size=n)
    choices = [(24, 48), (48, 96), (96, 192)]
    return [((int(nr[m]),) + choices[int(ang[m])], m) for m in range(n)]


def ensemble_member(shape, mseed, start="potential"):
    """The member's initial state and magnetogram (l <= min(15, N_theta / 2),
    max |B_r| = 5): Parker wind with the potential field of that magnetogram
    (``start="potential"``, the time-marching start) or with the dipole alone
    (``start="dipole"``)."""
    lmax = min(15, shape[1] // 2)
    Br = magnetogram(shape[1], shape[2], seed=mseed, lmax=lmax)
    if start == "potential":
        U, info = potential_background(*shape, lmax=lmax, seed=mseed)
    else:
        U, info = background(*shape)
    return U, Br, info["p_b"]
