"""Route A: fermionic operators on occupation-number basis states.

Oracle (test infrastructure).  Basis state ``|n>`` is the integer whose bit
``P`` is the occupation of spin orbital ``P``; spin orbitals are interleaved,
``P = 2 p + sigma`` (sigma 0 = alpha, 1 = beta).  A ladder operator on mode
``j`` carries the sign ``(-1)^(number of occupied modes below j)``, which is
the Jordan-Wigner convention with the parity string on the lower qubits (the
reading of Eq. (4) used throughout; the paper's printed form puts the string
on the upper qubits, which differs only by a diagonal +-1 similarity).

Nothing here uses Pauli algebra: these matrices are the independent
definition that the Pauli route in ``oracle.pauli`` is checked against.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _popcount(a):
    return np.bitwise_count(np.asarray(a, dtype=np.int64)).astype(np.int64)


def apply_ladder(states, amps, j, create):
    """Apply ``a_j^dagger`` (create) or ``a_j`` to basis states, vectorised.

    ``states`` are int64 basis indices, ``amps`` their amplitudes.  Returns
    the new states and amplitudes; amplitudes are 0 where the operator
    annihilates the state.
    """
    occ = (states >> j) & 1
    valid = (occ == 0) if create else (occ == 1)
    below = states & ((1 << j) - 1)
    sign = np.where(_popcount(below) & 1, -1.0, 1.0)
    return states ^ (1 << j), amps * sign * valid


def operator_matrix(n_modes, terms):
    """Sparse D x D matrix of ``sum_t coef_t * op_string_t``.

    ``terms`` is a list of ``(coef, ops)`` with ``ops`` a list of
    ``(mode, create)`` written left to right as in the operator product; the
    rightmost acts first.
    """
    d = 1 << n_modes
    cols = np.arange(d, dtype=np.int64)
    rows_all, cols_all, vals_all = [], [], []
    for coef, ops in terms:
        if coef == 0:
            continue
        st = cols.copy()
        amp = np.ones(d)
        for mode, create in reversed(ops):
            st, amp = apply_ladder(st, amp, mode, create)
        nz = amp != 0
        rows_all.append(st[nz])
        cols_all.append(cols[nz])
        vals_all.append(coef * amp[nz])
    if not rows_all:
        return sp.csr_matrix((d, d), dtype=np.complex128)
    r = np.concatenate(rows_all)
    c = np.concatenate(cols_all)
    v = np.concatenate(vals_all).astype(np.complex128)
    return sp.coo_matrix((v, (r, c)), shape=(d, d)).tocsr()


def spin_orbital_integrals(h, g):
    """Spin-orbital integrals from spatial ones (interleaved ordering).

    ``h_PQ = h_pq delta(s_P, s_Q)`` and
    ``(PQ|RS) = (pq|rs) delta(s_P, s_Q) delta(s_R, s_S)``.
    """
    n = h.shape[0]
    N = 2 * n
    sp_of = np.arange(N) // 2
    sg = np.arange(N) % 2
    H1 = h[np.ix_(sp_of, sp_of)] * (sg[:, None] == sg[None, :])
    G = g[np.ix_(sp_of, sp_of, sp_of, sp_of)]
    G = G * (sg[:, None, None, None] == sg[None, :, None, None])
    G = G * (sg[None, None, :, None] == sg[None, None, None, :])
    return H1, G


def hamiltonian_terms(h, g):
    """Fermionic terms of Eq. (2) in chemist notation.

    The paper writes ``1/2 sum h_ijkl a_i^+ a_j^+ a_l a_k`` with physicist
    integrals; with ``<ij|kl> = (ik|jl)`` this is
    ``1/2 sum_{PQRS} (PQ|RS) a_P^+ a_R^+ a_S a_Q``.
    """
    H1, G = spin_orbital_integrals(h, g)
    N = H1.shape[0]
    terms = []
    for P in range(N):
        for Q in range(N):
            if H1[P, Q] != 0.0:
                terms.append((H1[P, Q], [(P, True), (Q, False)]))
    for P in range(N):
        for Q in range(N):
            for R in range(N):
                for S in range(N):
                    v = G[P, Q, R, S]
                    if v != 0.0 and P != R and Q != S:
                        terms.append((0.5 * v, [(P, True), (R, True), (S, False), (Q, False)]))
    return terms


def hamiltonian_matrix(h, g, e_const=0.0):
    """Route A Hamiltonian of Eq. (2) on the 2^N occupation basis."""
    N = 2 * h.shape[0]
    H = operator_matrix(N, hamiltonian_terms(h, g))
    if e_const:
        H = H + e_const * sp.identity(1 << N, dtype=np.complex128, format="csr")
    return H.tocsr()


# --------------------------------------------------------------------------
# Excitation pool (Sec. III-E; sizes in Table II)
# --------------------------------------------------------------------------

def excitations(n_spatial, n_electrons):
    """Spin-conserving occupied -> virtual singles then doubles.

    Occupied spin orbitals are ``P < n_electrons`` (interleaved ordering).
    Singles ``(i, a)`` with equal spin; doubles ``(i, j, a, b)`` with
    ``i < j``, ``a < b`` and conserved S_z.  Each list is in lexicographic
    order; singles come first.  This reading reproduces the pool sizes 92
    (12 qubits) and 204 (14 qubits) of Table II.
    """
    N = 2 * n_spatial
    occ = list(range(n_electrons))
    vir = list(range(n_electrons, N))
    singles = [(i, a) for i in occ for a in vir if i % 2 == a % 2]
    doubles = []
    for ii, i in enumerate(occ):
        for j in occ[ii + 1:]:
            for aa, a in enumerate(vir):
                for b in vir[aa + 1:]:
                    if (i % 2) + (j % 2) == (a % 2) + (b % 2):
                        doubles.append((i, j, a, b))
    return singles + doubles


def excitation_ops(exc):
    """``(tau, tau^dagger)`` as operator strings (left to right)."""
    if len(exc) == 2:
        i, a = exc
        tau = [(a, True), (i, False)]
        tau_d = [(i, True), (a, False)]
    else:
        i, j, a, b = exc
        tau = [(a, True), (b, True), (j, False), (i, False)]
        tau_d = [(i, True), (j, True), (b, False), (a, False)]
    return tau, tau_d


def generator_matrix(n_modes, exc):
    """Anti-Hermitian pool generator ``A = tau - tau^dagger`` (route A)."""
    tau, tau_d = excitation_ops(exc)
    return operator_matrix(n_modes, [(1.0, tau), (-1.0, tau_d)])


def hf_occupation_index(n_electrons):
    """Occupation-basis index of the lowest-index determinant."""
    return (1 << n_electrons) - 1
