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
import test_oracle_families as tfam
import test_oracle_fcidump as tf
import test_oracle_hamiltonian as th
import test_oracle_mapping as tm
import test_oracle_pool as tp
import test_oracle_sector as ts
import test_oracle_vqe as tv
from oracle import adapt, evolve, families, fcidump, fermion, mapping, sector, vqe


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


# ---------------------------------------------------------------- more slips


def test_ladder_parity_mask_off_by_one_is_caught(monkeypatch):
    # route A's parity counted over the modes at or below j instead of below
    # j: every annihilator picks up an extra sign.  (The string on the modes
    # above j instead, Eq. (4) as printed, is no slip: for the
    # number-conserving strings of H and the pool it gives the same matrix.)
    def bad(states, amps, j, create):
        occ = (states >> j) & 1
        valid = (occ == 0) if create else (occ == 1)
        upto = states & ((1 << (j + 1)) - 1)
        sign = np.where(np.bitwise_count(upto) & 1, -1.0, 1.0)
        return states ^ (1 << j), amps * sign * valid

    monkeypatch.setattr(fermion, "apply_ladder", bad)
    with pytest.raises(AssertionError):
        th.test_route_b_equals_route_a(mapping.JW, 2, 5)


def test_pool_without_mixed_spin_doubles_is_caught(monkeypatch):
    good = fermion.excitations

    def bad(n_spatial, n_electrons):
        return [e for e in good(n_spatial, n_electrons) if not (len(e) == 4 and e[0] % 2 != e[1] % 2)]

    monkeypatch.setattr(fermion, "excitations", bad)
    with pytest.raises(AssertionError):
        tp.test_pool_sizes_of_workloads()


def test_fenwick_range_off_by_one_is_caught(monkeypatch):
    def bad(k):
        return range(k + 1 - mapping.lowbit(k), k + 1)      # lowbit(k) for lowbit(k + 1)

    monkeypatch.setattr(mapping, "fenwick_range", bad)
    with pytest.raises(AssertionError):
        tm.test_bk_matrix_power_of_two_blocks()


def test_hf_state_not_encoded_is_caught(monkeypatch):
    good = adapt.hf_state
    monkeypatch.setattr(adapt, "hf_state", lambda nq, ne, mp: good(nq, ne, mapping.JW))
    with pytest.raises(AssertionError):
        th.test_hf_energy_closed_form(mapping.BK, "c0")


def test_energy_without_normalisation_is_caught(monkeypatch):
    def bad(H, psi):
        w = H @ psi
        return float(np.vdot(psi, w).real), w

    ints, ne = synth.config0()
    c0 = (ints, ne, adapt.build_system(ints, ne, mapping.JW))
    monkeypatch.setattr(adapt, "energy", bad)
    with pytest.raises(AssertionError):
        ta.test_rayleigh_quotient_scale_invariant(c0)


def test_tie_to_the_highest_index_is_caught(monkeypatch):
    def bad(g, precision=adapt.FP64):
        ag = np.abs(np.asarray(g))
        gmax = float(ag.max())
        tau = adapt.TIE_REL_FP64 * max(1.0, gmax) if precision == adapt.FP64 else adapt.TIE_ABS_C64
        return int(np.nonzero(ag >= gmax - tau)[0][-1]), gmax

    monkeypatch.setattr(adapt, "select", bad)
    with pytest.raises(AssertionError):
        ta.test_tie_rule()


def test_adjoint_derivative_missing_a_term_is_caught(monkeypatch):
    def bad(A, phi, theta):
        v, acc, coef = phi, np.zeros_like(phi), 1.0
        for m in range(4):                                 # stops one term short
            acc = acc + coef * v
            v = A @ v
            coef = coef * theta / (m + 1)
        return A @ acc

    monkeypatch.setattr(vqe, "taylor4_derivative", bad)
    with pytest.raises(AssertionError):
        tv.test_taylor4_derivative_is_the_series_derivative()


def test_colex_rank_off_by_one_is_caught(monkeypatch):
    from math import comb
    monkeypatch.setattr(sector, "subset_rank", lambda cs: sum(comb(c, j) for j, c in enumerate(sorted(cs))))
    with pytest.raises(AssertionError):
        ts.test_colex_rank_textbook()


def test_fcidump_read_in_physicist_order_is_caught(monkeypatch):
    good = fcidump.read

    def bad(path):
        h, g, e, n, ne, ms2 = good(path)
        return h, g.transpose(0, 2, 1, 3).copy(), e, n, ne, ms2   # (ij|kl) taken as <ij|kl>

    monkeypatch.setattr(fcidump, "read", bad)
    with pytest.raises(AssertionError):
        tf.test_hand_written_file()


def test_smallest_first_colouring_is_caught(monkeypatch):
    def bad(n, edges):
        nbr = [set() for _ in range(n)]
        for i, j in edges:
            nbr[i].add(j)
            nbr[j].add(i)
        family, members = [-1] * n, []
        for v in sorted(range(n), key=lambda v: len(nbr[v])):   # Algorithm 1 takes the largest first
            for f, mem in enumerate(members):
                if not (nbr[v] & mem):
                    family[v] = f
                    mem.add(v)
                    break
            else:
                family[v] = len(members)
                members.append({v})
        return family

    monkeypatch.setattr(families, "greedy_families", bad)
    with pytest.raises(AssertionError):
        tfam.test_hand_traced_example()


def test_conjugated_y_phase_in_csr_is_caught(monkeypatch):
    # the element formula with i^(-ny) for i^(ny): the same as scaling each
    # coefficient by (-1)^ny before the correct formula.  H is real
    # symmetric, so its strings all have an even number of Y and it cannot
    # show this slip; the real antisymmetric generators (odd ny) do.
    from oracle import pauli
    good = pauli.pauli_to_csr

    def bad(ps, drop_rel=1e-12):
        ny = np.bitwise_count(ps.x & ps.z).astype(np.int64)
        flipped = pauli.PauliSum(ps.n_qubits, ps.x, ps.z, ps.c * (1 - 2 * (ny & 1)))
        return good(flipped, drop_rel)

    monkeypatch.setattr(pauli, "pauli_to_csr", bad)
    with pytest.raises(AssertionError):
        tp.test_generators_route_a_equals_route_b(mapping.BK)


def test_sector_basis_not_encoded_is_caught(monkeypatch):
    # the sector's qubit indices taken as occupation indices under BK too
    good = sector.qubit_basis
    monkeypatch.setattr(sector, "qubit_basis", lambda n, na, nb, mp: good(n, na, nb, mapping.JW))
    with pytest.raises(AssertionError):
        ts.test_jw_and_bk_restrictions_are_the_same_matrix("c0")


def test_adjoint_sweep_with_the_forward_angle_is_caught(monkeypatch):
    # the adjoint state carried back through a factor with +theta instead of
    # its inverse (-theta)
    def bad(system, ops, thetas, psi0):
        phis = [psi0]
        for k, th in zip(ops, thetas):
            phis.append(evolve.taylor5(system.pool[k], phis[-1], th))
        psi = phis[-1]
        nrm = float(np.vdot(psi, psi).real)
        E, w = adapt.energy(system.H, psi)
        chi = w - E * psi
        grad = np.zeros(len(ops))
        for j in range(len(ops) - 1, -1, -1):
            A = system.pool[ops[j]]
            grad[j] = 2.0 * np.vdot(chi, vqe.taylor4_derivative(A, phis[j], thetas[j])).real / nrm
            chi = evolve.taylor5(A, chi, thetas[j])
        return E, grad

    monkeypatch.setattr(vqe, "energy_and_gradient", bad)
    with pytest.raises(AssertionError):
        tv.test_adjoint_gradient_matches_finite_differences(0)


def test_commuting_pairs_taken_as_edges_is_caught(monkeypatch):
    # the commutation test on the anticommutator AB + BA instead of AB - BA
    def bad(pool_matrices):
        mats = [A.toarray() if hasattr(A, "toarray") else np.asarray(A) for A in pool_matrices]
        return {(i, j) for i in range(len(mats)) for j in range(i + 1, len(mats))
                if np.abs(mats[i] @ mats[j] + mats[j] @ mats[i]).max() > 1e-12}

    monkeypatch.setattr(families, "full_edges", bad)
    with pytest.raises(AssertionError):
        tfam.test_full_edges_match_the_commutator_definition_on_a_tiny_pool()


def test_first_tied_sample_is_caught(monkeypatch):
    """The line search's tie reading: "first sample within tolerance" in
    place of "smallest |theta|" picks the far minimum, about pi away."""

    def bad(e, samples):
        emin = min(e)
        tol = adapt.LINE_SEARCH_TIE * max(1.0, abs(emin))
        return next(m for m in range(samples) if e[m] <= emin + tol)

    monkeypatch.setattr(adapt, "_pick_sample", bad)
    with pytest.raises(AssertionError):
        ta.test_line_search_tie_takes_the_near_minimum(mapping.BK)
    with pytest.raises(AssertionError):
        ta.test_line_search_tie_takes_the_near_minimum(mapping.JW)
