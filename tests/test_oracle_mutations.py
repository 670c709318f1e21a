"""The oracle's pins catch plausible mistakes.

Each case plants one mistake (dropped term, wrong sign, wrong neighbour index,
swapped operand, wrong constant) into a copy of gs_oracle.c, compiles it on
the CPU, points the oracle module at the mutant and checks that at least one
pin from test_oracle_pins.py fails.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "gs_oracle.c")

MUTANTS = {
    "drop_zp_term": ("su = su + u[czp];", "su = su;"),
    "feed_sign": ("du = du + F * (1.0 - uc);", "du = du - F * (1.0 - uc);"),
    "xp_index": ("int xm = (x + L - 1) % L, xp = (x + 1) % L;",
                 "int xm = (x + L - 1) % L, xp = (x + 2) % L;"),
    "zm_uses_y": ("int64_t czm = x  + (int64_t)L * y  + LL * zm;",
                  "int64_t czm = x  + (int64_t)L * ym + LL * z;"),
    "uvv_swapped": ("double uvv = uc * (vc * vc);", "double uvv = vc * (uc * uc);"),
    "lap_wrong_centre": ("double lapv = (sv - 6.0 * vc) / 6.0;",
                         "double lapv = (sv - 6.0 * uc) / 6.0;"),
    "kill_sign": ("dv = dv - (F + k) * vc;", "dv = dv - (F - k) * vc;"),
    "dt_dropped": ("un[c] = uc + du * dt;", "un[c] = uc + du;"),
    "noise_in_v": ("dv = Dv * lapv + uvv;", "dv = Dv * lapv + uvv + noise * r;"),
    "hash_shift": ("h ^= h >> 13;", "h ^= h >> 12;"),
    "hash_key_order": ("return code_to_r(oracle_fmix32(oracle_fmix32(c ^ k1) ^ k2));",
                       "return code_to_r(oracle_fmix32(oracle_fmix32(c ^ k2) ^ k1));"),
    "field_key_order": ("r[c] = code_to_r(oracle_fmix32(oracle_fmix32((uint32_t)c ^ k1) ^ k2));",
                        "r[c] = code_to_r(oracle_fmix32(oracle_fmix32((uint32_t)c ^ k2) ^ k1));"),
    "step_key_order": (
        "double r = code_to_r(oracle_fmix32(oracle_fmix32((uint32_t)c ^ k1) ^ k2));",
        "double r = code_to_r(oracle_fmix32(oracle_fmix32((uint32_t)c ^ k2) ^ k1));"),
    "conv_tap_flip": ("int64_t q = cell_at(L, z + dz, yy + dy, xx + dx);",
                      "int64_t q = cell_at(L, z - dz, yy + dy, xx + dx);"),
    "bwd_data_tap": ("int64_t q = cell_at(L, z - dz, yy - dyo, xx - dxo);",
                     "int64_t q = cell_at(L, z - dz, yy - dyo, xx + dxo);"),
    "bwd_weight_tap": ("int64_t q = cell_at(L, z + dz, yy + dyo, xx + dxo);",
                       "int64_t q = cell_at(L, z + dz, yy - dyo, xx + dxo);"),
    "bf16_no_tie_even": ("bits += 0x7fffu + lsb;", "bits += 0x8000u;"),
    "held_face_off_by_one": ("x == L - 1 || y == L - 1 || z == L - 1;", "x == L - 2 || y == L - 1 || z == L - 1;"),
    "held_neighbour": ("su = su + u[c + L];", "su = su + u[c - L];"),
    "held_copies_u_into_v": ("vn[c] = v[c];", "vn[c] = u[c];"),
    "diffuse_D_dropped": ("b[c] = a[c] + dt * (D * lap);", "b[c] = a[c] + dt * lap;"),
    "diffuse_zp": ("sum = sum + a[x + (int64_t)L * y + LL * zp];", "sum = sum + a[x + (int64_t)L * y + LL * zm];"),
}

# pins exercised against every mutant (cheap ones)
PINS = [
    lambda o: pins.test_fmix32_published_vectors(o),
    lambda o: pins.test_noise_field_matches_numpy_restatement(o, 42, 1),
    lambda o: pins.test_fixed_point_is_exact(o, 3),
    lambda o: pins.test_octahedral_symmetry(o),
    lambda o: pins.test_sine_mode_diffusion_closed_form(o, 16, (1, 2, 3)),
    lambda o: pins.test_sine_mode_with_feed(o),
    lambda o: pins.test_v_mode_with_kill(o),
    lambda o: pins.test_brute_force_tiny_grids(o, 4, 0.1),
    lambda o: pins.test_brute_force_tiny_grids(o, 3, 0.0),
    lambda o: pins.test_light_cone(o),
    lambda o: pins.test_conv_fwd_matches_fft(o, 4),
    lambda o: pins.test_conv_adjoints(o),
    lambda o: pins.test_bf16_round_matches_torch(o),
    lambda o: pins.test_held_faces_unchanged_and_interior_as_periodic(o),
    lambda o: pins.test_held_dirichlet_mode_closed_form(o, 9, (3, 1, 2)),
    lambda o: pins.test_held_brute_force_tiny_grids(o, 5),
    lambda o: pins.test_diffuse_periodic_mode_closed_form(o, 9, (4, 0, 2)),
    lambda o: pins.test_diffuse_held_dirichlet_closed_form(o, 9, (2, 3, 1)),
    lambda o: pins.test_diffuse_brute_force_tiny_grids(o, 3, True),
]


@pytest.fixture(scope="module")
def src():
    return open(SRC).read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(src, name, monkeypatch, orc):
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    with tempfile.TemporaryDirectory() as d:
        csrc = os.path.join(d, "mut.c")
        so = os.path.join(d, "libmut.so")
        open(csrc, "w").write(src.replace(old, new))
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-shared",
                        "-fPIC", "-o", so, csrc], check=True)
        monkeypatch.setattr(oracle, "_lib", None)
        monkeypatch.setattr(oracle, "_LIB", so)
        monkeypatch.setattr(oracle, "build_oracle", lambda force=False: so)
        caught = []
        for i, pin in enumerate(PINS):
            try:
                with np.errstate(all="ignore"):
                    pin(oracle)
            except (AssertionError, RuntimeError):
                caught.append(i)
        monkeypatch.setattr(oracle, "_lib", None)
    assert caught, f"no pin caught mutant {name}"
