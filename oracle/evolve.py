"""Fifth-order Taylor state update and exact exponentials (oracle, test infrastructure)."""

from __future__ import annotations

import math

import numpy as np
import scipy.sparse.linalg as spla

TAYLOR_ORDER = 5


def taylor_coefficients(theta):
    """``theta^k / k!`` for k = 0..5 (the scalars of Eq. (8))."""
    return [theta ** k / math.factorial(k) for k in range(TAYLOR_ORDER + 1)]


def taylor5(A, psi, theta):
    """Sec. III-C: ``psi' = sum_{k=0..5} (theta A)^k psi / k!``.

    Computed as the paper does: the chain ``v_k = A v_{k-1}`` of Eq. (7)
    (five sparse matrix-vector products), then the accumulation of Eq. (8)
    in the order ``psi + theta v1 + theta^2/2 v2 + ... + theta^5/120 v5``.
    No renormalisation (the paper has none).
    """
    v = [np.asarray(psi, dtype=np.complex128)]
    for _ in range(TAYLOR_ORDER):
        v.append(A @ v[-1])
    coef = taylor_coefficients(theta)
    out = v[0].copy()
    for k in range(1, TAYLOR_ORDER + 1):
        out = out + coef[k] * v[k]
    return out


def normalise(psi):
    return psi / math.sqrt(float(np.vdot(psi, psi).real))


def expm_dense(A, theta):
    """``exp(theta A)`` for anti-Hermitian A via ``eigh`` of the Hermitian ``iA``."""
    Ad = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    lam, V = np.linalg.eigh(1j * Ad)
    return (V * np.exp(-1j * theta * lam)) @ V.conj().T


def expm_apply(A, psi, theta):
    """``exp(theta A) psi`` by SciPy's Krylov/Taylor ``expm_multiply`` (larger N)."""
    return spla.expm_multiply(theta * A.tocsc(), np.asarray(psi, dtype=np.complex128))
