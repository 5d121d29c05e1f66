"""Fermion-to-qubit mappings as Pauli strings (oracle, test infrastructure).

Jordan-Wigner follows Eq. (4) with the parity string on the qubits below
``j`` (reading; see ``oracle.fermion``).  The paper describes Bravyi-Kitaev
only as a binary-tree encoding with O(log N) weight (Sec. II-A-2) and gives
no formula; the reading used here is the Fenwick-tree encoding: qubit ``k``
stores the parity of the modes ``k + 1 - lowbit(k + 1) .. k``.  For this
encoding the creation operator is

    a_j^+ = 1/2 X_U(j) ( X_j Z_P(j) - i Y_j Z_R(j) )

with U the update set (qubits above ``j`` whose stored parity includes mode
``j``), P the parity set (qubits whose stored parities add up to the parity
of modes below ``j``), F the flip set (members of P inside ``j``'s own
range) and R = P minus F.  Jordan-Wigner is the special case U = F = {},
P = R = {0..j-1}.
"""

from __future__ import annotations

import numpy as np

JW = 0
BK = 1

# Pauli letter codes used by the label arrays.
I_, X_, Y_, Z_ = 0, 1, 2, 3


def lowbit(i):
    return i & (-i)


def fenwick_range(k):
    """Modes whose parity qubit ``k`` stores (0-indexed, inclusive range)."""
    lo = k + 1 - lowbit(k + 1)
    return range(lo, k + 1)


def encoding_matrix(n_modes, mapping):
    """Binary matrix ``B`` with qubit bits ``b = B n (mod 2)``."""
    B = np.zeros((n_modes, n_modes), dtype=np.int64)
    for k in range(n_modes):
        if mapping == JW:
            B[k, k] = 1
        else:
            for i in fenwick_range(k):
                B[k, i] = 1
    return B


def update_set(j, n_modes, mapping):
    if mapping == JW:
        return []
    return [k for k in range(j + 1, n_modes) if j in fenwick_range(k)]


def parity_set(j, mapping):
    if mapping == JW:
        return list(range(j))
    out = []
    i = j                      # prefix of length j, 1-indexed Fenwick walk
    while i > 0:
        out.append(i - 1)
        i -= lowbit(i)
    return sorted(out)


def flip_set(j, mapping):
    if mapping == JW:
        return []
    own = set(fenwick_range(j))
    return [k for k in parity_set(j, mapping) if set(fenwick_range(k)) <= own]


def remainder_set(j, mapping):
    f = set(flip_set(j, mapping))
    return [k for k in parity_set(j, mapping) if k not in f]


def ladder_strings(j, n_modes, mapping, create):
    """``a_j^+`` (create) or ``a_j`` as ``[(coef, label), (coef, label)]``.

    A label is a uint8 array of length ``n_modes``; entry ``q`` is the Pauli
    letter on qubit ``q`` (codes I=0, X=1, Y=2, Z=3).
    """
    U = update_set(j, n_modes, mapping)
    P = parity_set(j, mapping)
    R = remainder_set(j, mapping)
    s1 = np.zeros(n_modes, dtype=np.uint8)
    s2 = np.zeros(n_modes, dtype=np.uint8)
    for q in U:
        s1[q] = X_
        s2[q] = X_
    s1[j] = X_
    s2[j] = Y_
    for q in P:
        s1[q] = Z_
    for q in R:
        s2[q] = Z_
    c2 = -0.5j if create else 0.5j
    return [(0.5 + 0j, s1), (c2, s2)]


def encode_index(n_index, B):
    """Qubit-basis index of occupation index ``n`` under encoding ``B``."""
    N = B.shape[0]
    bits = np.array([(n_index >> i) & 1 for i in range(N)], dtype=np.int64)
    b = (B @ bits) & 1
    return int(sum(int(b[k]) << k for k in range(N)))


def permutation(n_modes, mapping):
    """``perm[n] = index of |B n>``, the basis map from occupation to qubits."""
    B = encoding_matrix(n_modes, mapping)
    d = 1 << n_modes
    n = np.arange(d, dtype=np.int64)
    out = np.zeros(d, dtype=np.int64)
    for k in range(n_modes):
        bit = np.zeros(d, dtype=np.int64)
        for i in range(n_modes):
            if B[k, i]:
                bit ^= (n >> i) & 1
        out |= bit << k
    return out
