"""Pins of the oracle's excitation pool and gradients (no GPU)."""

import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import adapt, evolve, fermion, mapping, pauli

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def pool_size_formula(n, ne):
    o = ne // 2
    v = n - o
    return 2 * o * v + 2 * math.comb(o, 2) * math.comb(v, 2) + (o * v) ** 2


def _table2():
    rows = []
    for line in open(os.path.join(GOLDEN, "table2_complexity.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append(line.split())
    return rows


def test_table2_dimensions_and_pool_sizes():
    rows = _table2()
    assert len(rows) == 3
    for label, nq, dim, elems, m, n, ne in rows:
        nq, dim, elems, m, n, ne = map(int, (nq, dim, elems, m, n, ne))
        assert dim == 2 ** nq and elems == 4 ** nq and n == nq // 2
        if ne < 0:
            continue   # 4-qubit entry: active electrons not determinable (unpinned)
        assert len(fermion.excitations(n, ne)) == m
        assert pool_size_formula(n, ne) == m


def test_pool_sizes_of_workloads():
    assert len(fermion.excitations(4, 4)) == 26
    assert len(fermion.excitations(6, 4)) == 92
    assert len(fermion.excitations(6, 8)) == 92
    assert len(fermion.excitations(7, 6)) == 204
    for n in range(1, 10):
        for ne in range(0, 2 * n + 1, 2):
            assert len(fermion.excitations(n, ne)) == pool_size_formula(n, ne)


def test_pool_order_and_spin():
    exc = fermion.excitations(4, 4)
    singles = [e for e in exc if len(e) == 2]
    doubles = [e for e in exc if len(e) == 4]
    assert exc == singles + doubles
    assert singles == sorted(singles) and doubles == sorted(doubles)
    for e in exc:
        occ, vir = e[: len(e) // 2], e[len(e) // 2:]
        assert all(p < 4 for p in occ) and all(p >= 4 for p in vir)
        assert sum(p % 2 for p in occ) == sum(p % 2 for p in vir)


@pytest.mark.parametrize("mp", [mapping.JW, mapping.BK])
def test_generators_route_a_equals_route_b(mp):
    n, ne = 4, 4
    N, d = 8, 256
    perm = mapping.permutation(N, mp)
    Pi = sp.csr_matrix((np.ones(d), (perm, np.arange(d))), shape=(d, d))
    exc, pps = pauli.pool_pauli(n, ne, mp)
    for e, p in zip(exc, pps):
        ref = Pi @ fermion.generator_matrix(N, e) @ Pi.T
        A = pauli.pauli_to_csr(p)
        assert abs(A - ref).max() == 0.0
        assert A.nnz == ref.count_nonzero()
        assert np.abs(pauli.pauli_to_dense(p) - ref.toarray()).max() == 0.0


@pytest.mark.parametrize("mp", [mapping.JW, mapping.BK])
def test_generator_structure(mp):
    n, ne = 5, 4
    N, d = 10, 1024
    exc, pps = pauli.pool_pauli(n, ne, mp)
    for e, p in zip(exc, pps):
        A = pauli.pauli_to_csr(p)
        assert abs(A.imag).max() == 0.0
        assert abs(A + A.T).max() == 0.0                      # real antisymmetric
        assert set(np.unique(A.data.real)) <= {-1.0, 1.0}      # entries +-1
        assert np.diff(A.indptr).max() <= 1                    # <= 1 nnz per row
        assert np.bincount(A.indices, minlength=d).max() <= 1  # and per column
        assert A.nnz == (d // 2 if len(e) == 2 else d // 8)
        assert np.unique(p.x).size == 1                        # one X-mask
        assert p.n_terms == (2 if len(e) == 2 else 8)
        A3 = A @ A @ A
        assert abs(A3 + A).max() == 0.0                        # A^3 = -A


def slater_condon_gradient_magnitude(h, g, n_electrons, exc):
    occ = range(n_electrons)
    if len(exc) == 2:
        I, A = exc
        i, a = I // 2, A // 2
        f = h[i, a]
        for J in occ:
            j = J // 2
            f += g[i, a, j, j]
            if J % 2 == I % 2:
                f -= g[i, j, j, a]
        return 2 * abs(f)
    I, J, A, B = exc
    i, j, a, b = I // 2, J // 2, A // 2, B // 2
    v = 0.0
    if I % 2 == A % 2 and J % 2 == B % 2:
        v += g[i, a, j, b]
    if I % 2 == B % 2 and J % 2 == A % 2:
        v -= g[i, b, j, a]
    return 2 * abs(v)


@pytest.mark.parametrize("mp", [mapping.JW, mapping.BK])
def test_hf_gradients_slater_condon(mp):
    ints, ne = synth.config0()
    sysm = adapt.build_system(ints, ne, mp)
    psi = adapt.hf_state(8, ne, mp)
    g = adapt.gradients(sysm.H, sysm.pool, psi)
    ref = np.array([slater_condon_gradient_magnitude(ints.h, ints.g, ne, e) for e in sysm.excitations])
    assert np.abs(np.abs(g) - ref).max() <= 1e-13
    assert np.abs(ref).min() > 0   # non-trivial: no gradient is identically zero


def test_gradient_equals_commutator_and_finite_difference():
    ints, ne = synth.config0()
    sysm = adapt.build_system(ints, ne, mapping.BK)
    psi = synth.random_state(8, 5) * 1.7   # unnormalised on purpose
    g = adapt.gradients(sysm.H, sysm.pool, psi)
    h = 1e-4
    for k in (0, 3, 11, 25):
        A = sysm.pool[k]
        assert abs(g[k] - adapt.gradient_commutator(sysm.H, A, psi)) <= 1e-13
        ep = adapt.energy(sysm.H, evolve.expm_dense(A, h) @ psi)[0]
        em = adapt.energy(sysm.H, evolve.expm_dense(A, -h) @ psi)[0]
        assert abs(g[k] - (ep - em) / (2 * h)) <= 1e-7
