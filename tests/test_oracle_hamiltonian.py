"""Pins of the oracle's qubit Hamiltonian (no GPU).

Route B (Pauli algebra, Eq. (3)) is checked against route A (Eq. (2) applied
on occupation states), against dense Kronecker products, against the
Slater-Condon closed form of the Hartree-Fock energy, and against the
symmetries the molecular Hamiltonian has.
"""

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import adapt, fermion, mapping, pauli


def _pi(N, mp):
    d = 1 << N
    perm = mapping.permutation(N, mp)
    return sp.csr_matrix((np.ones(d), (perm, np.arange(d))), shape=(d, d))


@pytest.mark.parametrize("mp", [mapping.JW, mapping.BK])
@pytest.mark.parametrize("n,seed", [(1, 3), (2, 5), (3, 7), (4, 0), (5, 11)])
def test_route_b_equals_route_a(mp, n, seed):
    ints = synth.integrals(n, seed)
    HA = fermion.hamiltonian_matrix(ints.h, ints.g, 0.25)
    Pi = _pi(2 * n, mp)
    ref = Pi @ HA @ Pi.T
    ps = pauli.qubit_hamiltonian(ints.h, ints.g, 0.25, mp)
    HB = pauli.pauli_to_csr(ps)
    scale = abs(ref).max()
    assert abs(HB - ref).max() <= 1e-14 * max(1.0, scale) * 8
    # identical sparsity pattern (no spurious or missing entries)
    assert HB.nnz == ref.count_nonzero()


def test_route_b_equals_route_a_strong_variant():
    ints = synth.integrals(4, 9, strong=True, n_electrons=4)
    HA = fermion.hamiltonian_matrix(ints.h, ints.g)
    for mp in (mapping.JW, mapping.BK):
        Pi = _pi(8, mp)
        HB = pauli.pauli_to_csr(pauli.qubit_hamiltonian(ints.h, ints.g, 0.0, mp))
        assert abs(HB - Pi @ HA @ Pi.T).max() <= 1e-13


@pytest.mark.parametrize("mp", [mapping.JW, mapping.BK])
@pytest.mark.parametrize("n", [2, 3, 4])
def test_csr_equals_dense_kron(mp, n):
    ints = synth.integrals(n, 100 + n)
    ps = pauli.qubit_hamiltonian(ints.h, ints.g, 0.0, mp)
    dense = pauli.pauli_to_dense(ps)
    csr = pauli.pauli_to_csr(ps).toarray()
    kept = csr != 0
    # kept entries: the two sides sum the same terms in different orders
    assert np.abs(csr - dense)[kept].max() <= 8e-16 * np.abs(ps.c).sum()
    # dropped entries: exact zeros up to rounding, below the drop threshold
    assert np.abs(dense[~kept]).max() <= 1e-12 * np.abs(ps.c).max()


@pytest.mark.parametrize("mp", [mapping.JW, mapping.BK])
def test_hamiltonian_real_symmetric(mp):
    ints = synth.integrals(4, 0)
    H = pauli.pauli_to_csr(pauli.qubit_hamiltonian(ints.h, ints.g, 0.0, mp))
    assert abs(H.imag).max() == 0.0
    assert abs(H - H.T).max() <= 1e-15


def test_jw_bk_isospectral():
    # The paper reports mapping-independent energies (Table III, Sec. IV-B).
    ints, _ = synth.config0()
    ev = []
    for mp in (mapping.JW, mapping.BK):
        H = pauli.pauli_to_csr(pauli.qubit_hamiltonian(ints.h, ints.g, 0.0, mp))
        ev.append(np.linalg.eigvalsh(H.toarray()))
    assert np.abs(ev[0] - ev[1]).max() <= 1e-12


def test_jw_bk_same_structure():
    ints = synth.integrals(5, 21)
    a = pauli.qubit_hamiltonian(ints.h, ints.g, 0.0, mapping.JW)
    b = pauli.qubit_hamiltonian(ints.h, ints.g, 0.0, mapping.BK)
    Ha, Hb = pauli.pauli_to_csr(a), pauli.pauli_to_csr(b)
    assert Ha.nnz == Hb.nnz
    assert a.xgroups().size == b.xgroups().size
    assert sorted(np.diff(Ha.indptr)) == sorted(np.diff(Hb.indptr))


@pytest.mark.parametrize("mp", [mapping.JW, mapping.BK])
def test_number_and_sz_conserved(mp):
    ints = synth.integrals(3, 4)
    N = 6
    H = pauli.pauli_to_csr(pauli.qubit_hamiltonian(ints.h, ints.g, 0.0, mp))
    Pi = _pi(N, mp)
    Hocc = (Pi.T @ H @ Pi).tocoo()
    n = np.arange(1 << N)
    num = np.bitwise_count(n)
    sz = np.bitwise_count(n & 0x15) - np.bitwise_count(n & 0x2A)
    assert np.all(num[Hocc.row] == num[Hocc.col])
    assert np.all(sz[Hocc.row] == sz[Hocc.col])


def hf_energy_closed_form(h, g, n_electrons):
    """Slater-Condon: sum_I h_II + 1/2 sum_IJ [(II|JJ) - delta_s (IJ|JI)]."""
    occ = range(n_electrons)
    e = sum(h[I // 2, I // 2] for I in occ)
    for I in occ:
        for J in occ:
            i, j = I // 2, J // 2
            e += 0.5 * g[i, i, j, j]
            if I % 2 == J % 2:
                e -= 0.5 * g[i, j, j, i]
    return e


@pytest.mark.parametrize("mp", [mapping.JW, mapping.BK])
@pytest.mark.parametrize("cfg", ["c0", "c1", "c2"])
def test_hf_energy_closed_form(mp, cfg):
    ints, ne = {"c0": synth.config0, "c1": synth.config1, "c2": synth.config2}[cfg]()
    ps = pauli.qubit_hamiltonian(ints.h, ints.g, ints.e_const, mp)
    H = pauli.pauli_to_csr(ps)
    psi = adapt.hf_state(2 * ints.n_spatial, ne, mp)
    E, _ = adapt.energy(H, psi)
    assert abs(E - hf_energy_closed_form(ints.h, ints.g, ne)) <= 1e-12


def test_constant_shift():
    # Table III: absolute energy = active-space energy + shifts; a constant
    # e_const moves every eigenvalue by exactly that amount.
    ints, ne = synth.config0()
    H0 = pauli.pauli_to_csr(pauli.qubit_hamiltonian(ints.h, ints.g, 0.0, mapping.JW))
    H1 = pauli.pauli_to_csr(pauli.qubit_hamiltonian(ints.h, ints.g, -25.295232 + 3.577234, mapping.JW))
    psi = synth.random_state(8, 1)
    assert abs(adapt.energy(H1, psi)[0] - adapt.energy(H0, psi)[0] - (-25.295232 + 3.577234)) <= 1e-12


def test_table3_arithmetic():
    rows = [l.split() for l in open(__file__.rsplit("/", 1)[0] + "/golden/table3_energies.txt")
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        parts = [float(v) for v in r[1:4]]
        assert abs(sum(parts) - float(r[4])) <= 1.5e-6
