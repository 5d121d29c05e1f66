"""Energy, pool gradients and the ADAPT iteration (oracle, test infrastructure).

States may be unnormalised; every scalar is the Rayleigh quotient form of
Eq. (1), i.e. divided by <psi|psi>.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import evolve, fermion, mapping, pauli

FP64 = "fp64"
C64 = "c64"

# Tie rule for the operator choice (the paper is silent; alpha/beta partners
# tie exactly): the lowest index whose |g| is within tau of the maximum.
TIE_REL_FP64 = 1e-9
TIE_ABS_C64 = 1e-5

LINE_SEARCH_SAMPLES = 4096


@dataclass
class System:
    """Hamiltonian and pool of one synthetic molecule under one mapping."""

    n_spatial: int
    n_electrons: int
    mapping: int
    H: object                 # scipy CSR, complex128
    ham_pauli: pauli.PauliSum
    excitations: list
    pool: list                # scipy CSR per generator
    pool_pauli: list = field(default_factory=list)

    @property
    def n_qubits(self):
        return 2 * self.n_spatial

    @property
    def dim(self):
        return 1 << self.n_qubits


def build_system(ints, n_electrons, mp):
    """Sec. III-D steps 1-2: map the Hamiltonian, generate the pool, compile CSR."""
    ps = pauli.qubit_hamiltonian(ints.h, ints.g, ints.e_const, mp)
    H = pauli.pauli_to_csr(ps)
    exc, pool_ps = pauli.pool_pauli(ints.n_spatial, n_electrons, mp)
    pool = [pauli.pauli_to_csr(p) for p in pool_ps]
    return System(ints.n_spatial, n_electrons, mp, H, ps, exc, pool, pool_ps)


def hf_state(n_qubits, n_electrons, mp):
    """Hartree-Fock basis state: lowest determinant, encoded by the mapping."""
    B = mapping.encoding_matrix(n_qubits, mp)
    idx = mapping.encode_index(fermion.hf_occupation_index(n_electrons), B)
    psi = np.zeros(1 << n_qubits, dtype=np.complex128)
    psi[idx] = 1.0
    return psi


def energy(H, psi):
    """Eq. (1): ``E = Re<psi|H|psi> / <psi|psi>``; also returns ``w = H psi``."""
    w = H @ psi
    return float(np.vdot(psi, w).real / np.vdot(psi, psi).real), w


def gradients(H, pool, psi):
    """Eq. (5): ``g_j = <psi|[H, A_j]|psi> = 2 Re<H psi|A_j psi>`` (H = H^+, A = -A^+)."""
    w = H @ psi
    nrm = float(np.vdot(psi, psi).real)
    return np.array([2.0 * np.vdot(w, A @ psi).real / nrm for A in pool])


def gradient_commutator(H, A, psi):
    """Eq. (5) literally: ``<psi|(H A - A H)|psi> / <psi|psi>``."""
    v = H @ (A @ psi) - A @ (H @ psi)
    return float(np.vdot(psi, v).real / np.vdot(psi, psi).real)


def select(g, precision=FP64):
    """Sec. III-D step 3: the operator with the largest |g_j| (tie rule above)."""
    ag = np.abs(np.asarray(g))
    gmax = float(ag.max()) if ag.size else 0.0
    tau = TIE_REL_FP64 * max(1.0, gmax) if precision == FP64 else TIE_ABS_C64
    k = int(np.nonzero(ag >= gmax - tau)[0][0]) if ag.size else -1
    return k, gmax


def line_search_coefficients(H, A, psi):
    """Matrix elements of H in the span of ``psi, A psi, A^2 psi``.

    Because ``A^3 = -A`` for every pool generator, ``exp(theta A) psi =
    psi + sin(theta) A psi + (1 - cos(theta)) A^2 psi`` and the energy along
    that curve depends on six numbers.  Returns ``(H00, H01, H02, H11, H12,
    H22)``, each divided by ``<psi|psi>``.
    """
    u0 = psi
    u1 = A @ u0
    u2 = A @ u1
    w0, w1, w2 = H @ u0, H @ u1, H @ u2
    n = float(np.vdot(psi, psi).real)
    return (np.vdot(u0, w0).real / n, np.vdot(w0, u1).real / n,
            np.vdot(w0, u2).real / n, np.vdot(u1, w1).real / n,
            np.vdot(w1, u2).real / n, np.vdot(u2, w2).real / n)


def line_energy(coef, theta):
    H00, H01, H02, H11, H12, H22 = coef
    s, u = math.sin(theta), 1.0 - math.cos(theta)
    return H00 + 2 * s * H01 + 2 * u * H02 + s * s * H11 + 2 * s * u * H12 + u * u * H22


def _line_d1(coef, theta):
    _, H01, H02, H11, H12, H22 = coef
    s, c = math.sin(theta), math.cos(theta)
    u = 1.0 - c
    return 2 * c * H01 + 2 * s * H02 + 2 * s * c * H11 + 2 * (c * u + s * s) * H12 + 2 * u * s * H22


def _line_d2(coef, theta):
    _, H01, H02, H11, H12, H22 = coef
    s, c = math.sin(theta), math.cos(theta)
    u = 1.0 - c
    return (-2 * s * H01 + 2 * c * H02 + 2 * (c * c - s * s) * H11
            + 2 * (3 * s * c - s * u) * H12 + 2 * (s * s + u * c) * H22)


LINE_SEARCH_TIE = 1e-10


def _sample_theta(m, samples):
    return -math.pi + 2.0 * math.pi * (m + 1) / samples


def _pick_sample(e, samples):
    """The tie rule of the line search: among the samples within
    ``1e-10 * max(1, |E_min|)`` of the lowest energy, the one with the
    smallest |theta|, then the lowest index."""
    emin = min(e)
    tol = LINE_SEARCH_TIE * max(1.0, abs(emin))
    best_m = None
    for m in range(samples):
        if e[m] <= emin + tol:
            if best_m is None or abs(_sample_theta(m, samples)) < abs(_sample_theta(best_m, samples)):
                best_m = m
    return best_m


def line_search(coef, samples=LINE_SEARCH_SAMPLES):
    """Global minimiser of the energy along ``exp(theta A) psi`` on (-pi, pi].

    Reading (the paper does not say how the new angle is chosen): sample
    ``theta_m = -pi + 2 pi (m + 1) / samples``; among the samples whose
    energy is within ``1e-10 * max(1, |E_min|)`` of the lowest, take the one
    with the smallest |theta| (then the lowest m).  The tolerance matters:
    when psi lies inside the generator's support the curve is pi-periodic
    and its two minima tie up to rounding.  Then polish with up to eight
    Newton steps on dE/dtheta that stay within one sample spacing of the
    chosen sample and are kept only if they do not raise the energy.
    """
    e = [line_energy(coef, _sample_theta(m, samples)) for m in range(samples)]
    best_m = _pick_sample(e, samples)
    th0 = _sample_theta(best_m, samples)
    e0 = e[best_m]
    h = 2.0 * math.pi / samples
    th = th0
    for _ in range(8):
        d2 = _line_d2(coef, th)
        if not d2 > 0.0:
            break
        step = _line_d1(coef, th) / d2
        nt = th - step
        if abs(nt - th0) > h:
            break
        th = nt
        if abs(step) < 1e-15:
            break
    if line_energy(coef, th) > e0:
        th = th0
    return th


@dataclass
class StepResult:
    energy: float
    max_grad: float
    selected: int
    converged: bool
    theta: float
    gradients: np.ndarray


def adapt_step(system, psi, eps, theta=None, precision=FP64, renormalise=True,
               force_k=None):
    """One iteration of Sec. III-D steps 3-4.

    Energy and gradients at ``psi``; the operator with the largest |g|; stop
    if ``max|g| < eps``; otherwise Taylor-5 with the given angle, or the
    line-search angle when ``theta`` is None.  ``force_k`` overrides the
    choice (used to compare trajectories step by step).
    """
    E, _ = energy(system.H, psi)
    g = gradients(system.H, system.pool, psi)
    k, gmax = select(g, precision)
    if force_k is not None:
        k = int(force_k)
    if gmax < eps:
        return StepResult(E, gmax, k, True, 0.0, g), psi
    A = system.pool[k]
    if theta is None:
        theta = line_search(line_search_coefficients(system.H, A, psi))
    out = evolve.taylor5(A, psi, theta)
    if renormalise:
        out = evolve.normalise(out)
    return StepResult(E, gmax, k, False, float(theta), g), out


def trajectory(system, psi0, eps, thetas=None, n_iter=20, precision=FP64):
    """Repeated ``adapt_step``; ``thetas`` (if given) supplies the angles."""
    psi = psi0
    out = []
    n = len(thetas) if thetas is not None else n_iter
    for it in range(n):
        th = None if thetas is None else float(thetas[it])
        r, psi = adapt_step(system, psi, eps, th, precision)
        out.append(r)
        if r.converged:
            break
    return out, psi
