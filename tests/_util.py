"""Shared helpers of the test-suite: oracle/GPU problem set-up and the error metric."""
import numpy as np

import coronal_inputs as ci
import oracle


def oracle_grid(shape, limiter="vanalbada", g0=ci.G0_SOLAR, rho_b=1.0, p_b=None, **kw):
    p_b = ci.parker_sound_speed2() if p_b is None else p_b
    return oracle.Grid(*shape, limiter=limiter, g0=g0, rho_b=rho_b, p_b=p_b, **kw)


def problem(name_or_shape, seed=2209, perturb=None, dipole_only=None):
    """Seeded synthetic inputs: a named workload or the background on any shape."""
    if isinstance(name_or_shape, str):
        w = ci.workload(name_or_shape)
        return w["U"], w["Br"]
    shape = tuple(name_or_shape)
    U, info = ci.background(*shape)
    if perturb is not None:
        U = ci.perturb(info["W"], seed=perturb, amp=0.01)
    if dipole_only is None:
        dipole_only = shape[1] < 8
    Br = ci.magnetogram(shape[1], shape[2], seed=seed, dipole_only=dipole_only,
                        lmax=min(15, shape[1] // 2))
    return U, Br


def rel_err(R, R_ref, scale):
    """Per-variable max |R - R_ref| / max |M|, M the oracle's flux-magnitude scale."""
    R = np.asarray(R, dtype=np.float64).reshape(9, -1)
    R_ref = np.asarray(R_ref).reshape(9, -1)
    scale = np.asarray(scale).reshape(9, -1)
    return np.abs(R - R_ref).max(axis=1) / scale.max(axis=1)
