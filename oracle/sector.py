"""Sector-restricted basis: fixed numbers of alpha and beta electrons.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's method works in the full 2^N space (Sec. II-A, Table II).  This
module is the restriction P_S M P_S of the same operators to the subspace S
of occupation-number states with n_alpha electrons in the even spin
orbitals (alpha, P = 2p) and n_beta in the odd ones (beta, P = 2p + 1).
H of Eq. (2) conserves both counts (its integrals couple equal spins
only), and so does every spin-conserving pool generator, so the
restriction changes no energy, gradient or Taylor-5 result for a state
that lives in S.

Basis order: rank(occ) = rank_a * C(n, n_beta) + rank_b, where rank_a
(rank_b) is the colexicographic rank of the occupied alpha (beta) spatial
orbitals {c_1 < ... < c_k}: sum_j C(c_j, j) (j from 1).  The qubit-space
index of basis state i is the mapping's encoding of its occupation index
(identity for JW, B n for BK).
"""

from itertools import combinations
from math import comb

import numpy as np

from . import mapping


def subset_rank(cs):
    """Colexicographic rank of a set of non-negative integers."""
    return sum(comb(c, j + 1) for j, c in enumerate(sorted(cs)))


def dimension(n_spatial, n_alpha, n_beta):
    return comb(n_spatial, n_alpha) * comb(n_spatial, n_beta)


def spins(occ, n_spatial):
    """(alpha orbitals, beta orbitals) occupied in occupation index ``occ``."""
    a = [p for p in range(n_spatial) if (occ >> (2 * p)) & 1]
    b = [p for p in range(n_spatial) if (occ >> (2 * p + 1)) & 1]
    return a, b


def rank(occ, n_spatial, n_alpha, n_beta):
    """Rank of occupation index ``occ`` in S, or -1 if it is not in S."""
    a, b = spins(occ, n_spatial)
    if len(a) != n_alpha or len(b) != n_beta or occ >> (2 * n_spatial):
        return -1
    return subset_rank(a) * comb(n_spatial, n_beta) + subset_rank(b)


def basis(n_spatial, n_alpha, n_beta):
    """Occupation indices of S, in rank order."""
    out = np.zeros(dimension(n_spatial, n_alpha, n_beta), dtype=np.int64)
    for a in combinations(range(n_spatial), n_alpha):
        for b in combinations(range(n_spatial), n_beta):
            occ = sum(1 << (2 * p) for p in a) + sum(1 << (2 * p + 1) for p in b)
            out[rank(occ, n_spatial, n_alpha, n_beta)] = occ
    return out


def qubit_basis(n_spatial, n_alpha, n_beta, mp):
    """Qubit-space indices of S in rank order under mapping ``mp``."""
    B = mapping.encoding_matrix(2 * n_spatial, mp)
    return np.array([mapping.encode_index(int(o), B) for o in basis(n_spatial, n_alpha, n_beta)],
                    dtype=np.int64)


def restrict(M, qidx):
    """P_S M P_S as a dim(S) x dim(S) matrix (rows and columns in rank order)."""
    return M[qidx][:, qidx]


def embed(psi_s, qidx, n_qubits):
    """Full-space vector equal to ``psi_s`` on S and zero elsewhere."""
    psi = np.zeros(1 << n_qubits, dtype=np.complex128)
    psi[qidx] = psi_s
    return psi


def hf_state(n_spatial, n_electrons, n_alpha, n_beta):
    """The lowest determinant (spin orbitals P < n_electrons) as a vector of S."""
    occ = (1 << n_electrons) - 1
    r = rank(occ, n_spatial, n_alpha, n_beta)
    if r < 0:
        raise ValueError("the lowest determinant is not in this sector")
    psi = np.zeros(dimension(n_spatial, n_alpha, n_beta), dtype=np.complex128)
    psi[r] = 1.0
    return psi


class SectorSystem:
    """A full-space oracle system (``adapt.System``) restricted to S."""

    def __init__(self, system, n_alpha, n_beta):
        self.full = system
        self.n_spatial = system.n_spatial
        self.n_electrons = system.n_electrons
        self.mapping = system.mapping
        self.n_alpha, self.n_beta = n_alpha, n_beta
        self.qidx = qubit_basis(system.n_spatial, n_alpha, n_beta, system.mapping)
        self.H = restrict(system.H, self.qidx)
        self.pool = [restrict(A, self.qidx) for A in system.pool]
        self.excitations = system.excitations

    @property
    def dim(self):
        return len(self.qidx)
