"""Planted mistakes in the oracle, on the CPU: a copy of oracle/goc_oracle.c
with one plausible mistake is compiled into a temporary library and run
against the pin meant to catch it; the pin must fail.  This checks that the
pins in test_oracle_pins.py are sharp enough, not the oracle itself."""
import os
import subprocess

import pytest

import oracle
import oracle.oracle as oracle_mod
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle_mod.__file__), "goc_oracle.c")

# (name, text in the oracle, planted replacement, pin that must fail)
MUTATIONS = [
    ("mie_source_sign", "    Y[1] = H * ((U[0] * B[1] - B[0] * U[1]) * t21);",
     "    Y[1] = -H * ((U[0] * B[1] - B[0] * U[1]) * t21);",
     pins.test_curvilinear_mie_reaches_the_steady_solution_of_its_equation),
    ("mie_gradient_theta21_dropped", "dB1[c] = -(L1 + 0.5 * csm2 * h1 * h1 * h2 * (t11 + t21) * B[c])",
     "dB1[c] = -(L1 + 0.5 * csm2 * h1 * h1 * h2 * (t11) * B[c])",
     pins.test_curvilinear_mie_reaches_the_steady_solution_of_its_equation),
    ("rest_force_theta12_dropped", "double Ft2 = h1 * (fx2 + (t12 - t22) * P",
     "double Ft2 = h1 * (fx2 + (-t22) * P",
     pins.test_rest_is_exact_and_mass_conserved_on_a_general_orthogonal_grid),
    ("tau_c_coefficients_swapped",
     "    *tc11 = rho * (ze + nu) * U2 * t12 + rho * (ze - nu) * U1 * t21;",
     "    *tc11 = rho * (ze - nu) * U2 * t12 + rho * (ze + nu) * U1 * t21;",
     pins.test_correction_coefficients_match_the_E3_E4_form),
    ("tau_c_index_transposed",
     "    *tc22 = rho * (ze + nu) * U1 * t21 + rho * (ze - nu) * U2 * t12;",
     "    *tc22 = rho * (ze + nu) * U1 * t12 + rho * (ze - nu) * U2 * t21;",
     pins.test_correction_coefficients_match_the_E3_E4_form),
    ("C3_theta21_bracket_swapped", "+ U1 * ((3 + a1) * h2 / h1 + 2 * h1 / h2 - h1 * h2 / cs2) * t21",
     "+ U1 * ((3 + a1) * h1 / h2 + 2 * h2 / h1 - h1 * h2 / cs2) * t21",
     pins.test_correction_coefficients_match_the_E3_E4_form),
    ("q21_printed_sign", "    double q21 = (1 - h2) * (h1 - 1) * (h1 - 1) / h1;",
     "    double q21 = -(1 - h2) * (h1 - 1) * (h1 - 1) / h1;",
     pins.test_central_equilibria_are_the_binomial_transform_of_the_raw_ones),
    ("centrifugal_sign", "- 2 * t12 * rho * U1 * U2 - t21 * (tau22 - rho * U2 * U2));",
     "- 2 * t12 * rho * U1 * U2 + t21 * (tau22 - rho * U2 * U2));",
     pins.test_taylor_couette_on_the_annulus_converges_at_second_order),
]


@pytest.mark.parametrize("name,old,new,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_each_pin_catches_its_planted_mistake(tmp_path, monkeypatch, name, old, new, pin):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    mutated = tmp_path / "goc_oracle_mutated.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libgoc_oracle_mutated.so"
    subprocess.run(["gcc", "-O3", "-march=native", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", str(lib),
                    str(mutated), "-lm"], check=True)
    monkeypatch.setattr(oracle_mod, "build", lambda force=False: str(lib))
    monkeypatch.setattr(oracle_mod, "_lib", None)   # the next Oracle loads the mutated library
    with pytest.raises(AssertionError):
        pin()
