"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws random numbers and arranges them into the shapes the
method consumes (molecular integrals, rotation angles, batch and arrival
recipes).  It holds none of the method's arithmetic: no fermion-to-qubit
mapping, no operator construction, no state evolution.  Both the CPU oracle
and the CUDA library read their inputs from here, and neither imports the
other.

Integral recipe (the paper uses molecular integrals, Eq. (2), which are not
available; these shape-matched stand-ins replace them):

* ``h`` is symmetric n x n.  Its diagonal is n draws of U[-2, 1] Ha, sorted
  ascending; its upper off-diagonal, drawn row-major, is N(0, 0.05) (0.05 read
  as the standard deviation) and mirrored.
* ``g[p,q,r,s] = sum_{l<6} L_l[p,q] L_l[r,s]`` with each ``L_l`` symmetric,
  upper triangle including the diagonal drawn row-major from N(0, 0.1) and
  mirrored.  The result has the 8-fold symmetry of real chemist integrals
  ``(pq|rs)``.
* The "strongly correlated" variant doubles the off-diagonal of ``h``, scales
  every ``L_l`` by 3 (so ``g`` by 9), and makes the HOMO/LUMO pair
  near-degenerate: ``h[LUMO,LUMO] = h[HOMO,HOMO] + 1e-3`` with
  ``HOMO = n_e/2 - 1``, ``LUMO = n_e/2``.

Draw order within one generator: diagonal, off-diagonal, then the six
Cholesky-like factors, all from ``numpy.random.default_rng(seed)`` (PCG64).
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

N_FACTORS = 6

# Seeds of the workloads (one generator per seed).
SEED_CONFIG0 = 0          # 8 qubits, 4 spatial orbitals, 4 electrons
SEED_CONFIG1 = 1          # 12 qubits, 6 spatial orbitals, 8 electrons
SEED_CONFIG2 = 2          # 14 qubits, strongly correlated, 6 electrons
SEED_T5_BATCH = 3         # batched Taylor-5 headline workload
SEED_TRAJ_BASE = 1000     # batched trajectories: seed 1000 + i
SEED_CATALOGUE_BASE = 2000  # serving catalogue: seed 2000 + j
SEED_ARRIVALS = 4         # serving arrival process


@dataclass(frozen=True)
class Integrals:
    """Real chemist-notation integrals of one synthetic molecule."""

    n_spatial: int
    h: np.ndarray        # (n, n) float64, symmetric
    g: np.ndarray        # (n, n, n, n) float64, (pq|rs), 8-fold symmetric
    e_const: float       # constant energy shift (0 for every synthetic case)


def integrals(n_spatial: int, seed: int, strong: bool = False,
              n_electrons: int | None = None) -> Integrals:
    """Draw one synthetic integral set (recipe in the module docstring)."""
    n = int(n_spatial)
    if n < 1:
        raise ValueError("n_spatial must be >= 1")
    rng = np.random.default_rng(seed)
    h = np.zeros((n, n))
    h[np.arange(n), np.arange(n)] = np.sort(rng.uniform(-2.0, 1.0, n))
    for p in range(n):
        for q in range(p + 1, n):
            v = rng.normal(0.0, 0.05)
            h[p, q] = v
            h[q, p] = v
    L = np.zeros((N_FACTORS, n, n))
    for l in range(N_FACTORS):
        for p in range(n):
            for q in range(p, n):
                v = rng.normal(0.0, 0.1)
                L[l, p, q] = v
                L[l, q, p] = v
    if strong:
        off = ~np.eye(n, dtype=bool)
        h[off] *= 2.0
        L *= 3.0
        if n_electrons is None:
            raise ValueError("the strongly correlated variant needs n_electrons")
        homo = n_electrons // 2 - 1
        lumo = n_electrons // 2
        if 0 <= homo and lumo < n:
            h[lumo, lumo] = h[homo, homo] + 1e-3
    g = np.einsum("lpq,lrs->pqrs", L, L)
    return Integrals(n, h, g, 0.0)


def electrons_for(n_spatial: int) -> int:
    """Electron count used when a recipe leaves it open: 2*floor(n/2)."""
    return 2 * (n_spatial // 2)


def config0() -> tuple[Integrals, int]:
    """8 qubits: 4 spatial orbitals, 4 electrons, seed 0."""
    return integrals(4, SEED_CONFIG0), 4


def config1() -> tuple[Integrals, int]:
    """12 qubits: 6 spatial orbitals, 8 electrons, seed 0 + 1."""
    return integrals(6, SEED_CONFIG1), 8


def config2() -> tuple[Integrals, int]:
    """14 qubits, strongly correlated: 7 spatial orbitals, 6 electrons."""
    return integrals(7, SEED_CONFIG2, strong=True, n_electrons=6), 6


def t5_batch(n_states: int, pool_size: int, seed: int = SEED_T5_BATCH,
             prep_ops: int = 3):
    """Recipe of the batched Taylor-5 workload.

    Each of ``n_states`` states starts from the Hartree-Fock state and is
    prepared by ``prep_ops`` rotations (op index uniform over the pool, angle
    N(0, 0.1)); it is then assigned one more op and angle for the timed
    update.  Returns ``(prep_k[n_states, prep_ops], prep_theta[...],
    k[n_states], theta[n_states])``.
    """
    rng = np.random.default_rng(seed)
    prep_k = rng.integers(0, pool_size, size=(n_states, prep_ops), dtype=np.int64)
    prep_theta = rng.normal(0.0, 0.1, size=(n_states, prep_ops))
    k = rng.integers(0, pool_size, size=n_states, dtype=np.int64)
    theta = rng.normal(0.0, 0.1, size=n_states)
    return prep_k.astype(np.int32), prep_theta, k.astype(np.int32), theta


@dataclass(frozen=True)
class Trajectory:
    """One independent ADAPT trajectory of the batched workload."""

    index: int
    n_spatial: int
    n_electrons: int
    mapping: int          # 0 = Jordan-Wigner, 1 = Bravyi-Kitaev
    thetas: np.ndarray    # angles used at successive iterations
    seed: int


def trajectories(n_traj: int = 256, qubit_choices=(10, 12, 14, 16),
                 max_len: int = 30, seed_base: int = SEED_TRAJ_BASE):
    """Recipe of the batched-trajectory workload (one generator per trajectory).

    Qubit count uniform over ``qubit_choices``, mapping 50/50, angle vector
    length uniform over 1..``max_len`` with entries N(0, 0.1); the electron
    count is 2*floor(n/2).  Integrals come from ``integrals(n, seed)``.
    """
    out = []
    for i in range(n_traj):
        seed = seed_base + i
        rng = np.random.default_rng(seed + 10_000_000)
        nq = int(rng.choice(np.asarray(qubit_choices)))
        mapping = int(rng.integers(0, 2))
        length = int(rng.integers(1, max_len + 1))
        thetas = rng.normal(0.0, 0.1, size=length)
        n = nq // 2
        out.append(Trajectory(i, n, electrons_for(n), mapping, thetas, seed))
    return out


@dataclass(frozen=True)
class Arrival:
    t: float          # arrival time, seconds from start
    kind: int         # 0 evolve, 1 energy, 2 pool gradients
    session: int      # target resident state
    op: int           # pool op for evolve (taken modulo the pool size)
    theta: float


def arrivals(rate_hz: float, duration_s: float, n_sessions: int,
             seed: int = SEED_ARRIVALS, mix=(0.5, 0.3, 0.2)):
    """Poisson arrival stream of the serving workload."""
    rng = np.random.default_rng(seed)
    n_expected = int(rate_hz * duration_s * 1.2) + 16
    gaps = rng.exponential(1.0 / rate_hz, size=n_expected)
    times = np.cumsum(gaps)
    times = times[times < duration_s]
    n = times.size
    kinds = rng.choice(3, size=n, p=np.asarray(mix))
    sessions = rng.integers(0, n_sessions, size=n)
    ops = rng.integers(0, 1 << 30, size=n)
    thetas = rng.normal(0.0, 0.1, size=n)
    return [Arrival(float(times[i]), int(kinds[i]), int(sessions[i]),
                    int(ops[i]), float(thetas[i])) for i in range(n)]


def catalogue(qubits=(12, 14, 16, 18), per_size: int = 4,
              seed_base: int = SEED_CATALOGUE_BASE):
    """Serving catalogue: (n_spatial, n_electrons, mapping, seed) per Hamiltonian."""
    out = []
    j = 0
    for nq in qubits:
        for _ in range(per_size):
            n = nq // 2
            out.append((n, electrons_for(n), j % 2, seed_base + j))
            j += 1
    return out


def random_state(n_qubits: int, seed: int) -> np.ndarray:
    """A normalised random complex128 state (for unit tests of single steps)."""
    rng = np.random.default_rng(seed)
    d = 1 << n_qubits
    v = rng.normal(size=d) + 1j * rng.normal(size=d)
    return v / math.sqrt(float(np.vdot(v, v).real))
