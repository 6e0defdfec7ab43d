"""Planted mistakes (CPU): each is written into a private copy of the
oracle's source, compiled, and must fail a pin that the unmodified copy
passes: the brute-force pin of the right-hand side (quadrature of the
pointwise weak form of Eq. 8 with the Lax-Friedrichs flux and lambda of
Eq. 10, and the truncated auxiliary system of Sect. 3), the closed-form
integral of the mass diagnostic, or the temporal order of the SSP-RK schemes
under a time-dependent open-sea boundary (which sees the stage times).  The
oracle itself is never modified: the copies live in pytest's temporary
directory."""
import importlib.util
import os
import shutil

import numpy as np
import pytest

import dgref
import oracle as O_REAL
from test_oracle_scheme import (MASS_TOL, mass_errors, random_state, scale_state_means, tide_order_rate,
                                tiny_meshes)

SRC_DIR = os.path.dirname(os.path.abspath(O_REAL.__file__))

MUTANTS = {
    # the neighbour's pressure trace on an edge with the bathymetry term's sign flipped
    "neighbour_pressure_sign": ("double pres = g * (0.5 * xo[i] * xo[j] + xo[i] * ho[j]);",
                                "double pres = g * (0.5 * xo[i] * xo[j] - xo[i] * ho[j]);"),
    # lambda of Eq. (10) from the own side only
    "lambda_own_side_only": ("double lam = fmax(fabs(un_a), fabs(un_b)) + fmax(sqrt(g * Ha), sqrt(g * Hb));",
                             "double lam = fabs(un_a) + sqrt(g * Ha);"),
    # the auxiliary system without the truncation of Sect. 3
    "no_truncation": ("static int Ktr(int i, int j) { int d = g_deg[i] > g_deg[j] ? g_deg[i] : g_deg[j]; return KP[d]; }",
                      "static int Ktr(int i, int j) { (void)i; (void)j; return KMAX; }"),
    # the bathymetry source's x and y components swapped
    "source_components_swapped": ("r[1][q] += g * m->dhb[2 * e] * xi[q]", "r[1][q] += g * m->dhb[2 * e + 1] * xi[q]"),
    # xi^2 / 2 of the volume pressure with a wrong factor
    "volume_pressure_factor": ("double pres = g * (0.5 * xi[i] * xi[j] + xi[i] * hb[j]);",
                               "double pres = g * (0.45 * xi[i] * xi[j] + xi[i] * hb[j]);"),
}

# mistakes that the right-hand side cannot see, each with the pin that must catch it
OTHER_MUTANTS = {
    # mass summed with the element area instead of sqrt|Omega_e| (the integral of phi_{e,1})
    "mass_area_scale": (("s += sqrt(m->area[e]) * c[e];", "s += m->area[e] * c[e];"), "mass"),
    # the third stage of SSP-RK3 evaluated at t + dt instead of t + dt/2
    "rk3_third_stage_time": (("tau3[3] = {0.0, 1.0, 0.5}", "tau3[3] = {0.0, 1.0, 1.0}"), "rk3"),
    # the second stage of SSP-RK2 evaluated at t instead of t + dt
    "rk2_second_stage_time": (("tau2[2] = {0.0, 1.0}", "tau2[2] = {0.0, 0.0}"), "rk2"),
}


def other_pin_passes(O, pin):
    if pin == "mass":
        return all(max(mass_errors(O, f)) <= MASS_TOL[f] for f in ("poly", "sine"))
    rk = 3 if pin == "rk3" else 2
    return abs(tide_order_rate(O, rk) - rk) < 0.3


def load_copy(tmp_path, name, mutation):
    d = tmp_path / name
    d.mkdir()
    shutil.copy(os.path.join(SRC_DIR, "oracle.py"), d / "oracle.py")
    src = open(os.path.join(SRC_DIR, "swe_oracle.c")).read()
    if mutation is not None:
        old, new = mutation
        assert src.count(old) >= 1, name
        src = src.replace(old, new)
    (d / "swe_oracle.c").write_text(src)
    spec = importlib.util.spec_from_file_location(f"oracle_copy_{name}", d / "oracle.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    return mod


def brute_force_pin_passes(O):
    """the checks of test_rhs_equals_brute_force_weak_form with the given oracle copy"""
    for case in range(3):
        for seed in (0, 1):
            xy, tri = tiny_meshes()[case]
            rng = np.random.default_rng(100 * case + seed)
            ne = len(tri)
            orders = rng.integers(0, 5, size=ne).astype(np.int8)
            hv = 1.0 + 0.3 * rng.uniform(size=len(xy))
            g = 9.81
            m = O.Mesh(xy, tri, hv, orders)
            c = scale_state_means(random_state(ne, orders, rng), m.geometry()["area"])
            r, u = m.rhs(O.Params(g=g), c, t=0.0, with_u=True)
            msh = dgref.Tri(xy, tri)
            u_ref = dgref.solve_u(msh, hv, orders, c)
            if np.abs(u - u_ref).max() > 1e-13 * max(1.0, np.abs(u_ref).max()):
                return False
            rb = dgref.brute_force_rhs(msh, hv, orders, c, u, g)
            if np.abs(r - rb).max() > 1e-12 * max(1.0, np.abs(rb).max()):
                return False
    return True


def test_unmodified_copy_passes(tmp_path):
    assert brute_force_pin_passes(load_copy(tmp_path, "unmodified", None))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_the_pin(tmp_path, name):
    assert not brute_force_pin_passes(load_copy(tmp_path, name, MUTANTS[name]))


def test_unmodified_copy_passes_the_other_pins(tmp_path):
    O = load_copy(tmp_path, "unmodified_other", None)
    assert all(other_pin_passes(O, pin) for pin in ("mass", "rk2", "rk3"))


@pytest.mark.parametrize("name", sorted(OTHER_MUTANTS))
def test_planted_mistake_fails_its_pin(tmp_path, name):
    mutation, pin = OTHER_MUTANTS[name]
    O = load_copy(tmp_path, name, mutation)
    assert brute_force_pin_passes(O)  # invisible to the right-hand side ...
    assert not other_pin_passes(O, pin)  # ... but not to its own pin
