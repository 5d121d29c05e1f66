"""Pins for ADAPT-VQE with re-optimised angles (oracle).

The adjoint gradient is checked against central finite differences of the
energy and against the pool gradient of Eq. (5) at theta = 0; the optimiser
against the variational bound and the stationarity of its result; the loop
against exact diagonalisation where the ansatz is complete (two electrons
in four spin orbitals) and for monotone energies.
"""

import numpy as np
import pytest

import synth
from oracle import adapt, evolve, sector, vqe


def _sys(cfg, mp):
    ints, ne = {"c0": synth.config0, "n2": lambda: (synth.integrals(2, 9), 2),
                "n3": lambda: (synth.integrals(3, 6), 2)}[cfg]()
    return adapt.build_system(ints, ne, mp), ne


@pytest.mark.parametrize("mp", [0, 1])
def test_adjoint_gradient_matches_finite_differences(mp):
    s, ne = _sys("c0", mp)
    psi0 = adapt.hf_state(8, ne, mp)
    rng = np.random.default_rng(4)
    ops = [3, 17, 0, 25, 9, 3]                  # repeats allowed
    th = rng.normal(0, 0.4, size=len(ops))
    E, g = vqe.energy_and_gradient(s, ops, th, psi0)
    assert abs(E - adapt.energy(s.H, vqe.ansatz_state(s, ops, th, psi0))[0]) <= 1e-13
    h = 1e-5
    for j in range(len(ops)):
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        fd = (vqe.energy_and_gradient(s, ops, tp, psi0)[0] - vqe.energy_and_gradient(s, ops, tm, psi0)[0]) / (2 * h)
        assert abs(g[j] - fd) <= 1e-8, j


def test_taylor4_derivative_is_the_series_derivative():
    s, ne = _sys("c0", 0)
    phi = synth.random_state(8, 2)
    A = s.pool[5]
    for th in (0.0, 0.3, -1.2):
        h = 1e-6
        fd = (evolve.taylor5(A, phi, th + h) - evolve.taylor5(A, phi, th - h)) / (2 * h)
        assert np.allclose(vqe.taylor4_derivative(A, phi, th), fd, atol=1e-8)


@pytest.mark.parametrize("mp", [0, 1])
def test_single_operator_at_zero_is_the_pool_gradient(mp):
    s, ne = _sys("c0", mp)
    psi0 = adapt.hf_state(8, ne, mp)
    g_pool = adapt.gradients(s.H, s.pool, psi0)
    for k in (0, 4, len(s.pool) - 1):
        _, g = vqe.energy_and_gradient(s, [k], [0.0], psi0)
        assert abs(g[0] - g_pool[k]) <= 1e-13


def test_reoptimize_is_stationary_and_variational():
    s, ne = _sys("c0", 1)
    psi0 = adapt.hf_state(8, ne, 1)
    ops = [int(k) for k in np.argsort(-np.abs(adapt.gradients(s.H, s.pool, psi0)))[:4]]
    th, E = vqe.reoptimize(s, ops, np.zeros(4), psi0, gtol=1e-10)
    _, g = vqe.energy_and_gradient(s, ops, th, psi0)
    assert np.abs(g).max() <= 1e-8
    assert E <= adapt.energy(s.H, psi0)[0]
    ground = np.linalg.eigvalsh(sector.restrict(s.H, sector.qubit_basis(4, 2, 2, 1)).toarray())[0]
    assert E >= ground - 1e-12


@pytest.mark.parametrize("mp", [0, 1])
def test_two_electrons_reach_the_exact_ground_state(mp):
    """2 electrons in 2 spatial orbitals: the (1, 1) sector has dimension 4 and
    the pool (2 singles, 1 double) is complete; ADAPT-VQE reaches FCI."""
    s, ne = _sys("n2", mp)
    ops, th, energies = vqe.adapt_vqe(s, adapt.hf_state(4, ne, mp), 1e-8, max_ops=6, gtol=1e-12)
    fci = np.linalg.eigvalsh(sector.restrict(s.H, sector.qubit_basis(2, 1, 1, mp)).toarray())[0]
    assert abs(energies[-1] - fci) <= 1e-9
    assert all(b <= a + 1e-12 for a, b in zip(energies, energies[1:]))


def test_adapt_vqe_beats_greedy_steps_and_is_monotone():
    s, ne = _sys("n3", 0)
    psi0 = adapt.hf_state(6, ne, 0)
    ops, th, energies = vqe.adapt_vqe(s, psi0, 1e-6, max_ops=5)
    assert all(b <= a + 1e-12 for a, b in zip(energies, energies[1:]))
    res, _ = adapt.trajectory(s, psi0, 1e-6, n_iter=len(ops))
    # re-optimising every angle can only lower the energy of the same number of steps
    assert energies[-1] <= min(r.energy for r in res) + 1e-9
