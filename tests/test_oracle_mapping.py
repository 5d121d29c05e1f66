"""Pins of the oracle's fermion-to-qubit mappings (no GPU).

Each check compares the oracle against something other than itself: the
occupation-number definition of the ladder operators, the canonical
anticommutation relations, and the binary-tree structure of the encoding.
"""

import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fermion, mapping, pauli


def _gf2_rank(M):
    M = M.copy() % 2
    r = 0
    rows, cols = M.shape
    for c in range(cols):
        piv = None
        for i in range(r, rows):
            if M[i, c]:
                piv = i
                break
        if piv is None:
            continue
        M[[r, piv]] = M[[piv, r]]
        for i in range(rows):
            if i != r and M[i, c]:
                M[i] ^= M[r]
        r += 1
    return r


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 7, 8, 12, 14, 16, 18, 30])
def test_bk_encoding_invertible(N):
    B = mapping.encoding_matrix(N, mapping.BK)
    assert _gf2_rank(B) == N
    assert np.all(np.diag(B) == 1)
    assert np.all(np.triu(B, 1) == 0)


def test_bk_matrix_power_of_two_blocks():
    # The Fenwick encoding for N = 4 is the textbook 4 x 4 BK matrix, and for
    # N = 2^k the top-left blocks are the smaller BK matrices.
    B4 = mapping.encoding_matrix(4, mapping.BK)
    ref = np.array([[1, 0, 0, 0], [1, 1, 0, 0], [0, 0, 1, 0], [1, 1, 1, 1]])
    assert np.array_equal(B4, ref)
    B8 = mapping.encoding_matrix(8, mapping.BK)
    assert np.array_equal(B8[:4, :4], B4)
    assert np.array_equal(B8[4:, 4:], B4)
    assert np.all(B8[7, :] == 1)


@pytest.mark.parametrize("N", [3, 5, 6, 8])
def test_bk_sets_brute_force(N):
    # Update, parity and flip sets against b = B n for every occupation n.
    B = mapping.encoding_matrix(N, mapping.BK)
    for j in range(N):
        U = mapping.update_set(j, N, mapping.BK)
        col = {k for k in range(N) if B[k, j]} - {j}
        assert set(U) == col
    for n in range(1 << N):
        bits = np.array([(n >> i) & 1 for i in range(N)])
        b = (B @ bits) % 2
        for j in range(N):
            P = mapping.parity_set(j, mapping.BK)
            F = mapping.flip_set(j, mapping.BK)
            assert sum(b[k] for k in P) % 2 == bits[:j].sum() % 2
            assert (b[j] + sum(b[k] for k in F)) % 2 == bits[j]


@pytest.mark.parametrize("N", [4, 8, 14, 16, 18, 30])
def test_bk_weight_logarithmic(N):
    # Sec. II-A-2: BK strings have O(log N) weight; JW strings have O(N).
    bound = 2 * math.ceil(math.log2(N)) + 1
    for j in range(N):
        for cre in (True, False):
            for _, lab in mapping.ladder_strings(j, N, mapping.BK, cre):
                assert np.count_nonzero(lab) <= bound
            jw = mapping.ladder_strings(j, N, mapping.JW, cre)
            assert max(np.count_nonzero(l) for _, l in jw) == j + 1


def _ladder_dense(j, N, mp, create):
    terms = mapping.ladder_strings(j, N, mp, create)
    x, z = pauli.label_masks(np.stack([t[1] for t in terms]))
    ps = pauli.PauliSum(N, x, z, np.array([t[0] for t in terms]))
    return pauli.pauli_to_dense(ps)


@pytest.mark.parametrize("mp", [mapping.JW, mapping.BK])
@pytest.mark.parametrize("N", [3, 4, 5])
def test_ladder_strings_match_occupation_definition(mp, N):
    # a_j^+ as Pauli strings equals Pi a_j^+ Pi^T with a_j^+ defined on
    # occupation states (route A) and Pi the basis map |n> -> |B n>.
    d = 1 << N
    perm = mapping.permutation(N, mp)
    Pi = sp.csr_matrix((np.ones(d), (perm, np.arange(d))), shape=(d, d))
    for j in range(N):
        for cre in (True, False):
            ref = (Pi @ fermion.operator_matrix(N, [(1.0, [(j, cre)])]) @ Pi.T).toarray()
            assert np.abs(_ladder_dense(j, N, mp, cre) - ref).max() == 0.0


@pytest.mark.parametrize("mp", [mapping.JW, mapping.BK])
def test_canonical_anticommutation(mp):
    N = 4
    a = [_ladder_dense(j, N, mp, False) for j in range(N)]
    ad = [_ladder_dense(j, N, mp, True) for j in range(N)]
    eye = np.eye(1 << N)
    for i in range(N):
        for j in range(N):
            assert np.allclose(a[i] @ ad[j] + ad[j] @ a[i], eye * (i == j), atol=0)
            assert np.allclose(a[i] @ a[j] + a[j] @ a[i], 0, atol=0)


def test_jw_matches_eq4_form():
    # Eq. (4) with the parity string on the lower qubits: Z..Z (X - iY)/2.
    N = 6
    for j in range(N):
        (c1, s1), (c2, s2) = mapping.ladder_strings(j, N, mapping.JW, True)
        assert c1 == 0.5 and c2 == -0.5j
        assert list(s1[:j]) == [mapping.Z_] * j and s1[j] == mapping.X_
        assert list(s2[:j]) == [mapping.Z_] * j and s2[j] == mapping.Y_
        assert not s1[j + 1:].any() and not s2[j + 1:].any()
