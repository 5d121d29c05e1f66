"""Route B: Pauli-string algebra and Pauli sum -> CSR (oracle, test infrastructure).

A Pauli sum is held as label arrays (one letter per qubit, little-endian:
position q acts on qubit q, so the dense matrix is kron(P_{N-1}, ..., P_0)).
It is exported in the packed form ``(x, z, c)``: bit q of ``x`` is set for X
or Y on qubit q, bit q of ``z`` for Z or Y, and ``c`` is the coefficient of
the Hermitian label.  On a basis state,

    P |b> = i^{popcount(x & z)} (-1)^{popcount(b & z)} |b xor x>,

so ``H[r, c] = sum_{p : x_p = r xor c} c_p i^{ny_p} (-1)^{popcount(c & z_p)}``
(Eq. (3) written out element by element).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import fermion, mapping

I_, X_, Y_, Z_ = mapping.I_, mapping.X_, mapping.Y_, mapping.Z_

# Single-qubit products: letter a times letter b = phase * letter.
_MUL = np.zeros((4, 4), dtype=np.uint8)
_PH = np.ones((4, 4), dtype=np.complex128)
for _a in range(4):
    _MUL[0, _a] = _a
    _MUL[_a, 0] = _a
    _MUL[_a, _a] = 0
_MUL[X_, Y_], _PH[X_, Y_] = Z_, 1j
_MUL[Y_, X_], _PH[Y_, X_] = Z_, -1j
_MUL[Y_, Z_], _PH[Y_, Z_] = X_, 1j
_MUL[Z_, Y_], _PH[Z_, Y_] = X_, -1j
_MUL[Z_, X_], _PH[Z_, X_] = Y_, 1j
_MUL[X_, Z_], _PH[X_, Z_] = Y_, -1j

_PAULI_2x2 = [
    np.eye(2, dtype=np.complex128),
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
]


def mul_labels(la, lb):
    """Row-wise product of label arrays ``[T, N]``: returns (labels, phases)."""
    out = _MUL[la, lb]
    ph = np.prod(_PH[la, lb], axis=1)
    return out, ph


def label_masks(labels):
    """Packed ``(x, z)`` int64 masks of label arrays ``[T, N]``."""
    N = labels.shape[1]
    w = (np.int64(1) << np.arange(N, dtype=np.int64))
    xb = (labels == X_) | (labels == Y_)
    zb = (labels == Z_) | (labels == Y_)
    return (xb.astype(np.int64) * w).sum(axis=1), (zb.astype(np.int64) * w).sum(axis=1)


@dataclass
class PauliSum:
    """Canonical Pauli sum: terms sorted by (x, z), like terms combined."""

    n_qubits: int
    x: np.ndarray      # int64 [K]
    z: np.ndarray      # int64 [K]
    c: np.ndarray      # complex128 [K], coefficient of the Hermitian label

    @property
    def n_terms(self):
        return self.x.size

    def xgroups(self):
        """Distinct X-masks in ascending order."""
        return np.unique(self.x)


def combine(x, z, c, n_qubits, drop_rel=1e-12):
    """Merge like terms, drop ``|c| <= drop_rel * max|c|``, sort by (x, z)."""
    key = (x.astype(np.int64) << 32) | z.astype(np.int64)
    uk, inv = np.unique(key, return_inverse=True)
    cr = np.bincount(inv, weights=c.real, minlength=uk.size)
    ci = np.bincount(inv, weights=c.imag, minlength=uk.size)
    cc = cr + 1j * ci
    mx = np.abs(cc).max() if cc.size else 0.0
    keep = np.abs(cc) > drop_rel * mx
    uk, cc = uk[keep], cc[keep]
    return PauliSum(n_qubits, uk >> 32, uk & ((1 << 32) - 1), cc)


def _ladder_tables(n_modes, mp):
    """Per mode: coefficient [2] and label [2, N] of a^+ and of a."""
    cre_c = np.zeros((n_modes, 2), dtype=np.complex128)
    ann_c = np.zeros((n_modes, 2), dtype=np.complex128)
    cre_l = np.zeros((n_modes, 2, n_modes), dtype=np.uint8)
    ann_l = np.zeros((n_modes, 2, n_modes), dtype=np.uint8)
    for j in range(n_modes):
        for t, (c, lab) in enumerate(mapping.ladder_strings(j, n_modes, mp, True)):
            cre_c[j, t], cre_l[j, t] = c, lab
        for t, (c, lab) in enumerate(mapping.ladder_strings(j, n_modes, mp, False)):
            ann_c[j, t], ann_l[j, t] = c, lab
    return cre_c, cre_l, ann_c, ann_l


def _product_terms(coef, ops_idx, ops_create, tables):
    """Expand products of ladder operators into Pauli terms, vectorised.

    ``ops_idx[T, m]`` are mode indices, ``ops_create[m]`` flags (same for all
    T rows), ``coef[T]`` the fermionic coefficients.  Returns label arrays,
    and complex coefficients for all 2^m string choices.
    """
    cre_c, cre_l, ann_c, ann_l = tables
    T, m = ops_idx.shape
    labs_out, coef_out = [], []
    for choice in range(1 << m):
        lab = None
        cc = coef.astype(np.complex128).copy()
        for o in range(m):
            t = (choice >> o) & 1
            if ops_create[o]:
                lo, co = cre_l[ops_idx[:, o], t], cre_c[ops_idx[:, o], t]
            else:
                lo, co = ann_l[ops_idx[:, o], t], ann_c[ops_idx[:, o], t]
            cc = cc * co
            if lab is None:
                lab = lo
            else:
                lab, ph = mul_labels(lab, lo)
                cc = cc * ph
        labs_out.append(lab)
        coef_out.append(cc)
    return np.concatenate(labs_out), np.concatenate(coef_out)


def qubit_hamiltonian(h, g, e_const, mp, drop_rel=1e-12):
    """Qubit Hamiltonian of Eq. (3) from the fermionic one of Eq. (2).

    One-body ``h_PQ a_P^+ a_Q`` and two-body ``1/2 (PQ|RS) a_P^+ a_R^+ a_S a_Q``
    terms are expanded with the ladder strings of the chosen mapping,
    multiplied letter by letter, and like terms are merged.  The constant
    ``e_const`` is added to the identity.
    """
    H1, G = fermion.spin_orbital_integrals(h, g)
    N = H1.shape[0]
    tables = _ladder_tables(N, mp)
    labs, coefs = [], []
    P, Q = np.nonzero(H1)
    if P.size:
        lb, cf = _product_terms(H1[P, Q], np.stack([P, Q], 1), [True, False], tables)
        labs.append(lb)
        coefs.append(cf)
    P, Q, R, S = np.nonzero(G)
    keep = (P != R) & (Q != S)
    P, Q, R, S = P[keep], Q[keep], R[keep], S[keep]
    if P.size:
        lb, cf = _product_terms(0.5 * G[P, Q, R, S], np.stack([P, R, S, Q], 1),
                                [True, True, False, False], tables)
        labs.append(lb)
        coefs.append(cf)
    lab = np.concatenate(labs)
    coef = np.concatenate(coefs)
    x, z = label_masks(lab)
    x = np.concatenate([x, [0]])
    z = np.concatenate([z, [0]])
    coef = np.concatenate([coef, [complex(e_const)]])
    ps = combine(x, z, coef, N, drop_rel)
    # Hermitian: label coefficients are real.
    assert np.all(np.abs(ps.c.imag) <= 1e-12 * max(1.0, np.abs(ps.c).max()))
    ps.c = ps.c.real.astype(np.complex128)
    return ps


def generator_pauli(exc, n_modes, mp):
    """Pool generator ``A = tau - tau^+`` as a Pauli sum (Sec. III-E step 1)."""
    tables = _ladder_tables(n_modes, mp)
    tau, tau_d = fermion.excitation_ops(exc)
    labs, coefs = [], []
    for sgn, ops in ((1.0, tau), (-1.0, tau_d)):
        idx = np.array([[m for m, _ in ops]], dtype=np.int64)
        cr = [c for _, c in ops]
        lb, cf = _product_terms(np.array([sgn]), idx, cr, tables)
        labs.append(lb)
        coefs.append(cf)
    lab = np.concatenate(labs)
    x, z = label_masks(lab)
    return combine(x, z, np.concatenate(coefs), n_modes, drop_rel=1e-12)


def pool_pauli(n_spatial, n_electrons, mp):
    exc = fermion.excitations(n_spatial, n_electrons)
    return exc, [generator_pauli(e, 2 * n_spatial, mp) for e in exc]


def pauli_to_csr(ps, drop_rel=1e-12):
    """CSR of a Pauli sum by the element formula (module docstring).

    Entries of one X-mask group are summed in canonical term order; entries
    with ``|v| <= drop_rel * max|c|`` are dropped; columns are ascending.
    Returns ``scipy.sparse.csr_matrix`` (complex128).
    """
    N = ps.n_qubits
    d = 1 << N
    rows = np.arange(d, dtype=np.int64)
    ny = np.bitwise_count(ps.x & ps.z).astype(np.int64)
    cp = ps.c * (1j ** (ny % 4))
    tol = drop_rel * (np.abs(ps.c).max() if ps.n_terms else 0.0)
    R, C, V = [], [], []
    for xg in ps.xgroups():
        sel = np.nonzero(ps.x == xg)[0]
        col = rows ^ xg
        val = np.zeros(d, dtype=np.complex128)
        for p in sel:
            sgn = 1 - 2 * (np.bitwise_count(col & ps.z[p]).astype(np.int64) & 1)
            val = val + cp[p] * sgn
        keep = np.abs(val) > tol
        R.append(rows[keep])
        C.append(col[keep])
        V.append(val[keep])
    r = np.concatenate(R)
    c = np.concatenate(C)
    v = np.concatenate(V)
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rowptr = np.zeros(d + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return sp.csr_matrix((v, c, rowptr), shape=(d, d))


def pauli_to_dense(ps):
    """Dense matrix ``sum c_p kron(P_{N-1}, ..., P_0)`` (small N only)."""
    N = ps.n_qubits
    d = 1 << N
    out = np.zeros((d, d), dtype=np.complex128)
    for x, z, c in zip(ps.x, ps.z, ps.c):
        m = np.ones((1, 1), dtype=np.complex128)
        for q in range(N - 1, -1, -1):
            xb = (int(x) >> q) & 1
            zb = (int(z) >> q) & 1
            letter = {(0, 0): I_, (1, 0): X_, (1, 1): Y_, (0, 1): Z_}[(xb, zb)]
            m = np.kron(m, _PAULI_2x2[letter])
        out += c * m
    return out
