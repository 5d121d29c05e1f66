"""Plant plausible mistakes in the oracle (on the CPU) and check a pin fails.

Each case patches one oracle function with a typical slip -- a wrong
coefficient, a flipped sign, a dropped factor, a transposed operand, an
off-by-one index -- and runs an existing pin, which must now fail.
"""

import numpy as np
import pytest

import synth
import test_oracle_adapt as ta
import test_oracle_evolve as te
import test_oracle_hamiltonian as th
import test_oracle_mapping as tm
import test_oracle_pool as tp
from oracle import adapt, evolve, fermion, mapping


def test_wrong_taylor_coefficient_is_caught(monkeypatch):
    good = evolve.taylor_coefficients

    def bad(theta):
        c = good(theta)
        c[5] = theta ** 5 / 100.0
        return c

    monkeypatch.setattr(evolve, "taylor_coefficients", bad)
    with pytest.raises(AssertionError):
        te.test_nilpotent_block_is_exact()


def test_dropped_taylor_term_is_caught(monkeypatch):
    good = evolve.taylor_coefficients
    monkeypatch.setattr(evolve, "taylor_coefficients", lambda t: good(t)[:5] + [0.0])
    with pytest.raises(AssertionError):
        te.test_scalar_case_is_truncated_series()


def test_flipped_y_sign_is_caught(monkeypatch):
    good = mapping.ladder_strings

    def bad(j, n, mp, create):
        (c1, s1), (c2, s2) = good(j, n, mp, create)
        return [(c1, s1), (-c2, s2)]

    monkeypatch.setattr(mapping, "ladder_strings", bad)
    with pytest.raises(AssertionError):
        th.test_route_b_equals_route_a(mapping.BK, 2, 5)


def test_parity_set_off_by_one_is_caught(monkeypatch):
    good = mapping.parity_set
    monkeypatch.setattr(mapping, "parity_set", lambda j, mp: good(j + 1, mp) if j + 1 < 6 else good(j, mp))
    with pytest.raises(AssertionError):
        tm.test_bk_sets_brute_force(6)


def test_missing_half_in_two_body_is_caught(monkeypatch):
    good = fermion.spin_orbital_integrals

    def bad(h, g):
        H1, G = good(h, g)
        return H1, 2.0 * G

    monkeypatch.setattr(fermion, "spin_orbital_integrals", bad)
    with pytest.raises(AssertionError):
        th.test_hf_energy_closed_form(mapping.JW, "c0")


def test_transposed_generator_in_gradient_is_caught(monkeypatch):
    def bad(H, pool, psi):
        w = H @ psi
        n = float(np.vdot(psi, psi).real)
        return np.array([2.0 * np.vdot(w, A.T @ psi).real / n for A in pool])

    monkeypatch.setattr(adapt, "gradients", bad)
    with pytest.raises(AssertionError):
        tp.test_gradient_equals_commutator_and_finite_difference()


def test_transposed_generator_in_chain_is_caught(monkeypatch):
    good = evolve.taylor5
    monkeypatch.setattr(evolve, "taylor5", lambda A, psi, theta: good(A.T, psi, theta))
    ints, ne = synth.config0()
    sysm = adapt.build_system(ints, ne, mapping.JW)
    with pytest.raises(AssertionError):
        te.test_chain_equals_closed_form(sysm, 0.05)


def test_wrong_line_search_term_is_caught(monkeypatch):
    good = adapt.line_energy

    def bad(coef, theta):
        H00, H01, H02, H11, H12, H22 = coef
        return good((H00, H01, H02, H11, -H12, H22), theta)

    monkeypatch.setattr(adapt, "line_energy", bad)
    ints, ne = synth.config0()
    sysm = adapt.build_system(ints, ne, mapping.JW)
    with pytest.raises(AssertionError):
        ta.test_line_search_energy_curve((ints, ne, sysm))
