"""Planted mistakes (CPU): each is written into a private copy of the
oracle's source, compiled, and must fail a pin that the unmodified copy
passes: the brute-force pin of the right-hand side (quadrature of the
pointwise weak form of Eq. 8 with the Lax-Friedrichs flux and lambda of
Eq. 10, land and open-sea edges, and the truncated auxiliary system of
Sect. 3), the same pin with bottom friction and Coriolis (Eq. 5), the
closed-form integral of the mass diagnostic, the temporal order of the SSP-RK
schemes under a time-dependent open-sea boundary (which sees the stage
times), the closed-form CFL step, the hand-computed decisions of the
adaptivity indicator, the open-sea elevation against the tide formula, or the
base part of the separated form against the
brute-force weak form of the degree-1 truncation.  The oracle itself is never modified: the copies live
in pytest's temporary directory."""
import importlib.util
import os
import shutil

import pytest

import oracle as O_REAL
from test_oracle_scheme import (MASS_TOL, base_part_pin_error, cfl_pin_error, indicator_pin_failures, mass_errors, rhs_pin_errors, tide_pin_error,
                                source_pin_errors, tide_order_rate)

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
    # the land boundary's ghost state without the mirrored normal momentum
    "wall_not_mirrored": ("Uo[i] = U[i] - 2.0 * nx * qn; Vo[i] = V[i] - 2.0 * ny * qn;",
                          "Uo[i] = U[i]; Vo[i] = V[i];"),
    # the open-sea ghost state with zero momentum instead of q+ = q
    "open_sea_momentum_zero": ("xo[i] = 0.0; Uo[i] = U[i]; Vo[i] = V[i];", "xo[i] = 0.0; Uo[i] = 0.0; Vo[i] = 0.0;"),
}

# mistakes that the right-hand side cannot see, each with the pin that must catch it
OTHER_MUTANTS = {
    # mass summed with the element area instead of sqrt|Omega_e| (the integral of phi_{e,1})
    "mass_area_scale": (("s += sqrt(m->area[e]) * c[e];", "s += m->area[e] * c[e];"), "mass"),
    # the third stage of SSP-RK3 evaluated at t + dt instead of t + dt/2
    "rk3_third_stage_time": (("tau3[3] = {0.0, 1.0, 0.5}", "tau3[3] = {0.0, 1.0, 1.0}"), "rk3"),
    # the second stage of SSP-RK2 evaluated at t instead of t + dt
    "rk2_second_stage_time": (("tau2[2] = {0.0, 1.0}", "tau2[2] = {0.0, 0.0}"), "rk2"),
    # the second stage of SSP-RK3 combined half and half (still consistent)
    "rk3_second_stage_weights": (("a3[3] = {0.0, 0.75, 1.0 / 3.0}, b3[3] = {1.0, 0.25, 2.0 / 3.0}",
                                  "a3[3] = {0.0, 0.5, 1.0 / 3.0}, b3[3] = {1.0, 0.5, 2.0 / 3.0}"), "rk3"),
    # Coriolis with the wrong sense of rotation
    "coriolis_sign": (("- tau * uu[q] + P->f_c * V[q];", "- tau * uu[q] - P->f_c * V[q];"), "source"),
    # the quadratic friction law with |u|^2 instead of |u|
    "friction_quadratic_law": (("P->fric_quad * sqrt(um * um + vm * vm);", "P->fric_quad * (um * um + vm * vm);"),
                               "source"),
    # the CFL step without the order factor 1 / (2p + 1)
    "cfl_without_order_factor": (("(sp * (2.0 * m->p[e] + 1.0))", "(sp * (m->p[e] + 1.0))"), "cfl"),
    # the base part with the own side's edge products whose second coefficient
    # index is of degree >= 2 (the sum of the two parts, and so the whole rhs,
    # unchanged; in the volume terms the same products vanish by orthogonality)
    "base_part_with_higher_products": (("if (i < Kx && j < Kx && use_term(part, q < 3 && i < 3 && j < 3)) {",
                                        "if (i < Kx && j < Kx && use_term(part, q < 3 && i < 3)) {"), "base"),
    # the tide's phase with the wrong sign
    "tide_phase_sign": (("sin(2.0 * M_PI * t / P->tide_period + P->tide_phase)",
                         "sin(2.0 * M_PI * t / P->tide_period - P->tide_phase)"), "tide"),
    # the indicator's energy fraction with the mean mode in the denominator
    "indicator_counts_the_mean": (("for (int i = 1; i < K; ++i) {\n      double x = C_(c, 0, i, e, ne);",
                                   "for (int i = 0; i < K; ++i) {\n      double x = C_(c, 0, i, e, ne);"),
                                  "indicator"),
}


def other_pin_passes(O, pin):
    if pin == "mass":
        return all(max(mass_errors(O, f)) <= MASS_TOL[f] for f in ("poly", "sine"))
    if pin == "source":
        return all(source_pin_errors(O, case)[0] <= 1e-12 for case in range(3))
    if pin == "tide":
        return tide_pin_error(O) <= 1e-13
    if pin == "base":
        return base_part_pin_error(O) <= 1e-12
    if pin == "cfl":
        return cfl_pin_error(O) <= 1e-15
    if pin == "indicator":
        return indicator_pin_failures(O) == []
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
            eu, er = rhs_pin_errors(O, case, seed)
            if eu > 1e-13 or er > 1e-12:
                return False
    return True


def test_unmodified_copy_passes(tmp_path):
    assert brute_force_pin_passes(load_copy(tmp_path, "unmodified", None))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_the_pin(tmp_path, name):
    assert not brute_force_pin_passes(load_copy(tmp_path, name, MUTANTS[name]))


def test_unmodified_copy_passes_the_other_pins(tmp_path):
    O = load_copy(tmp_path, "unmodified_other", None)
    assert all(other_pin_passes(O, pin) for pin in ("mass", "rk2", "rk3", "source", "cfl", "indicator", "base", "tide"))


@pytest.mark.parametrize("name", sorted(OTHER_MUTANTS))
def test_planted_mistake_fails_its_pin(tmp_path, name):
    mutation, pin = OTHER_MUTANTS[name]
    O = load_copy(tmp_path, name, mutation)
    assert brute_force_pin_passes(O)  # invisible to the right-hand side ...
    assert not other_pin_passes(O, pin)  # ... but not to its own pin
