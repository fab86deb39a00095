"""The pins catch plausible slips: each mutant below plants one mistake in a copy of the
oracle source, on the CPU, and at least one pin of test_oracle_pins must fail on it."""
import ctypes
import os
import subprocess
import tempfile

import pytest

import test_oracle_pins as PINS
from oracle import oracle as O

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "wp_oracle.c")

MUTANTS = {
    "kinetic_sign": ("double th = -p->hbar * k2 * tau / (2.0 * p->mass);",
                     "double th = p->hbar * k2 * tau / (2.0 * p->mass);"),
    "no_negative_wavenumbers": ("int64_t js = (j < n / 2) ? j : j - n;", "int64_t js = j;"),
    "vkv_second_half_at_t_n": ("apply_potential_phase(p, nterms, terms, psi, time_of(p, s + 1), 0.5 * dt);",
                               "apply_potential_phase(p, nterms, terms, psi, time_of(p, s), 0.5 * dt);"),
    "kvk_potential_at_t_n": ("apply_potential_phase(p, nterms, terms, psi, time_of(p, s) + 0.5 * dt, dt);",
                             "apply_potential_phase(p, nterms, terms, psi, time_of(p, s), dt);"),
    "missing_1_over_N": ("psih[idx] = psih[idx] * CMPLX(cos(th), sin(th)) * inv_n;",
                         "psih[idx] = psih[idx] * CMPLX(cos(th), sin(th));"),
    "mass_dropped": ("double th = -p->hbar * k2 * tau / (2.0 * p->mass);",
                     "double th = -p->hbar * k2 * tau / (2.0);"),
    "twiddle_sign": ("double wr = cos(ang), wi = sign * sin(ang);", "double wr = cos(ang), wi = -sign * sin(ang);"),
    "grid_offset": ("return p->xmin[d] + (double)i * (p->L[d] / (double)p->n[d]);",
                    "return p->xmin[d] + (double)(i + 1) * (p->L[d] / (double)p->n[d]);"),
    "gaussian_width": ("v *= CMPLX(cos(ph), sin(ph)) * exp(-u * u / (sigma[d] * sigma[d]));",
                       "v *= CMPLX(cos(ph), sin(ph)) * exp(-u * u / (2.0 * sigma[d] * sigma[d]));"),
    "momentum_without_hbar": ("rec[5 + d] = p->hbar * sp[d] * dvk;", "rec[5 + d] = sp[d] * dvk;"),
    "energy_without_potential": ("rec[11] = rec[12] + rec[13];", "rec[11] = rec[12];"),
    "half_step_not_halved": ("apply_potential_phase(p, nterms, terms, psi, time_of(p, s), 0.5 * dt);",
                             "apply_potential_phase(p, nterms, terms, psi, time_of(p, s), dt);"),
    "quad_without_half": ("r += 0.5 * tm->a[d] * u * u;", "r += tm->a[d] * u * u;"),
    "centre_velocity_sign": ("double u = x[d] - (tm->c0[d] + tm->v[d] * t);\n        r += 0.5",
                             "double u = x[d] - (tm->c0[d] - tm->v[d] * t);\n        r += 0.5"),
    "y_axis_takes_x_index": ("double x[3] = {coord(p, 0, i), p->ndim > 1 ? coord(p, 1, j) : 0.0,\n"
                             "                       p->ndim > 2 ? coord(p, 2, k) : 0.0};\n"
                             "        int64_t idx = (i * n1 + j) * n2 + k;\n        double v",
                             "double x[3] = {coord(p, 0, i), p->ndim > 1 ? coord(p, 1, i) : 0.0,\n"
                             "                       p->ndim > 2 ? coord(p, 2, k) : 0.0};\n"
                             "        int64_t idx = (i * n1 + j) * n2 + k;\n        double v"),
    "morse_sign": ("double e = 1.0 - exp(-tm->a[1] * u);", "double e = 1.0 - exp(tm->a[1] * u);"),
    "grid_dropped_in_phase": ("double v = orc_potential_at(p, nterms, terms, x, t) + (p->vgrid ? p->vgrid[idx] : 0.0);",
                              "double v = orc_potential_at(p, nterms, terms, x, t);"),
    "grid_dropped_in_energy": ("sv += (orc_potential_at(p, nterms, terms, x, t) + (p->vgrid ? p->vgrid[idx] : 0.0)) * rho;",
                               "sv += orc_potential_at(p, nterms, terms, x, t) * rho;"),
    "autocorr_overlap_with_current_state": ("cplx c = conj(psi0[idx]) * psi[idx];",
                                            "cplx c = conj(psi[idx]) * psi[idx];"),
}

PIN_TESTS = [
    lambda: PINS.test_fft_matches_bruteforce_dft(16, -1),
    lambda: PINS.test_fft_3d_matches_bruteforce_per_axis(),
    lambda: PINS.test_free_gaussian_closed_form_1d("vkv"),
    lambda: PINS.test_plane_wave_kinetic_phase_and_momentum(64 - 5),
    lambda: PINS.test_harmonic_ground_state_energy_and_width(),
    lambda: PINS.test_driven_trap_1d_follows_verlet_map("vkv"),
    lambda: PINS.test_driven_trap_1d_follows_verlet_map("kvk"),
    lambda: PINS.test_laser_trap_2d_follows_verlet_map_per_axis(),
    lambda: PINS.test_potential_terms_pointwise(),
    lambda: PINS.test_constant_grid_potential_is_a_global_phase("vkv"),
    lambda: PINS.test_harmonic_grid_potential_ground_state_3d(),
    lambda: PINS.test_morse_eigenstates_energy_and_stationarity(),
    lambda: PINS.test_free_gaussian_autocorrelation_closed_form_1d("vkv"),
]


def _build_mutant(old, new, tmpdir):
    src = open(SRC).read()
    assert src.count(old) >= 1, old
    path = os.path.join(tmpdir, "mutant.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new, 1))
    so = os.path.join(tmpdir, "libmutant.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", path, "-o", so, "-lm"], check=True)
    return so


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, monkeypatch):
    old, new = MUTANTS[name]
    with tempfile.TemporaryDirectory() as tmp:
        so = _build_mutant(old, new, tmp)
        saved = O._lib
        O._lib = None
        monkeypatch.setattr(O._build, "build", lambda force=False: so)
        caught = []
        try:
            for pin in PIN_TESTS:
                try:
                    pin()
                except (AssertionError, FloatingPointError, ValueError):
                    caught.append(pin)
                    break
        finally:
            O._lib = saved
        assert caught, f"no pin fails on mutant {name}"
