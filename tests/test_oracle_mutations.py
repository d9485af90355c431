"""Planted mistakes in the CPU oracle must fail its pins.

Each case copies the oracle's source, changes one term the way a plausible
slip would (a flipped sign, a dropped term, a wrong factor), compiles the copy
into a temporary library, points the ``oracle`` package at it for the duration
of the case, and checks that the pins named for that term fail.  The oracle
itself is not modified; the mutated copies live in a temporary directory.

These are pins of the pins: they show that the energy flux's magnetic work
term -B_n (V.B), the gravity work rho g.V and the other terms below (paper
Sect. 2.2 fluxes and sources, the Rusanov dissipation) each have a test that
depends on them.
"""
import ctypes
import os
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "corona_oracle.cpp")

# (name, original text, mutated text, pins that must fail)
MUTATIONS = [
    ("energy flux magnetic work sign",
     "f[U_E] = (en + pt) * un - bn * vb;", "f[U_E] = (en + pt) * un + bn * vb;",
     [pins.test_flux_energy_is_enthalpy_plus_poynting, pins.test_boosted_alfven_wave_energy_converges]),
    ("energy flux magnetic work dropped",
     "f[U_E] = (en + pt) * un - bn * vb;", "f[U_E] = (en + pt) * un;",
     [pins.test_flux_energy_is_enthalpy_plus_poynting, pins.test_boosted_alfven_wave_energy_converges]),
    ("gravity work sign",
     "res.R[U_E * N + id] += mg;", "res.R[U_E * N + id] -= mg;",
     [pins.test_free_stream_gravity_source]),
    ("gravity momentum sign",
     "res.R[U_MX * N + id] += rho * g[0];", "res.R[U_MX * N + id] -= rho * g[0];",
     [pins.test_free_stream_gravity_source]),
    ("magnetic tension sign",
     "f[U_MX] = rho * vx * un + pt * n[0] - bx * bn;", "f[U_MX] = rho * vx * un + pt * n[0] + bx * bn;",
     [pins.test_flux_magnetostatic_limit]),
    ("GLM gradient term dropped",
     "f[U_BX] = un * bx - bn * vx + psi * n[0];", "f[U_BX] = un * bx - bn * vx;",
     [pins.test_flux_magnetostatic_limit]),
    ("Rusanov dissipation sign",
     "- 0.5 * lam * (ur[v] - ul[v]);", "+ 0.5 * lam * (ur[v] - ul[v]);",
     [pins.test_flux_rotation_invariance_and_dissipation]),
]


def _build_mutant(tmp_path, original, mutated):
    src = open(SRC).read()
    assert src.count(original) == 1, original
    path = tmp_path / "mutant.cpp"
    path.write_text(src.replace(original, mutated))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                    "-shared", "-o", str(lib), str(path)], check=True)
    return str(lib)


@pytest.mark.parametrize("name,original,mutated,must_fail", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_its_pins(tmp_path, monkeypatch, name, original, mutated, must_fail):
    good = oracle._load()
    lib = ctypes.CDLL(_build_mutant(tmp_path, original, mutated))
    # same signatures as the real library
    for fname in ("orc_residual", "orc_residual_jvp", "orc_flux", "orc_cons_to_prim", "orc_geometry",
                  "orc_ghosts", "orc_pseudo_time_step"):
        f, g = getattr(lib, fname), getattr(good, fname)
        f.argtypes, f.restype = g.argtypes, g.restype
    monkeypatch.setattr(oracle, "_lib", lib)
    for pin in must_fail:
        with pytest.raises(AssertionError):
            pin()
