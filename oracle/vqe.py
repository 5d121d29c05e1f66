"""ADAPT-VQE with every angle re-optimised after each selection.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's loop (Sec. III-D) updates the state with the new operator only;
it does not describe re-optimising earlier angles.  This module is the
standard ADAPT-VQE form of that loop, built on the same Taylor-5 factor
U_j(theta) = sum_{m<=5} (theta A_j)^m / m! of Eqs. (6)-(8):

    psi(theta) = U_n(theta_n) ... U_1(theta_1) psi_0,
    E(theta)   = Re<psi|H|psi> / <psi|psi>            (Eq. (1); U is not unitary)

and its exact gradient by reverse accumulation:

    dE/dtheta_j = 2 Re<chi_j | U_j'(theta_j) phi_{j-1}> / <psi|psi>,
    phi_j = U_j phi_{j-1},  chi_n = (H - E) psi,  chi_{j-1} = U_j^T chi_j,

with U_j' = A_j sum_{m<=4} (theta A_j)^m / m! (the series differentiated
term by term) and U_j^T = U_j(-theta) because A_j is real antisymmetric.
"""

import numpy as np
from scipy.optimize import minimize

from . import adapt, evolve


def taylor4_derivative(A, phi, theta):
    """U'(theta) phi = A sum_{m<=4} (theta A)^m phi / m!."""
    v = phi
    acc = np.zeros_like(phi)
    coef = 1.0
    for m in range(5):
        acc = acc + coef * v
        v = A @ v
        coef = coef * theta / (m + 1)
    return A @ acc


def ansatz_state(system, ops, thetas, psi0):
    """psi(theta): the Taylor-5 factors applied in order, no renormalisation."""
    psi = psi0
    for k, th in zip(ops, thetas):
        psi = evolve.taylor5(system.pool[k], psi, th)
    return psi


def energy_and_gradient(system, ops, thetas, psi0):
    """E(theta) and dE/dtheta by one forward and one adjoint sweep."""
    phis = [psi0]
    for k, th in zip(ops, thetas):
        phis.append(evolve.taylor5(system.pool[k], phis[-1], th))
    psi = phis[-1]
    nrm = float(np.vdot(psi, psi).real)
    E, w = adapt.energy(system.H, psi)
    chi = w - E * psi
    grad = np.zeros(len(ops))
    for j in range(len(ops) - 1, -1, -1):
        A = system.pool[ops[j]]
        grad[j] = 2.0 * np.vdot(chi, taylor4_derivative(A, phis[j], thetas[j])).real / nrm
        chi = evolve.taylor5(A, chi, -thetas[j])
    return E, grad


def reoptimize(system, ops, thetas0, psi0, gtol=1e-8, max_iter=200):
    """All angles by BFGS on E(theta) with the adjoint gradient."""
    if len(ops) == 0:
        return np.zeros(0), adapt.energy(system.H, psi0)[0]
    res = minimize(lambda t: energy_and_gradient(system, ops, t, psi0)[0], np.asarray(thetas0, dtype=float),
                   jac=lambda t: energy_and_gradient(system, ops, t, psi0)[1], method="BFGS",
                   options={"gtol": gtol, "maxiter": max_iter})
    return res.x, float(res.fun)


def adapt_vqe(system, psi0, eps, max_ops=20, precision=adapt.FP64, gtol=1e-8):
    """ADAPT-VQE: pool gradients at psi(theta), select (tie rule of
    ``adapt.select``), stop if max|g| < eps, else append the operator with
    angle 0 and re-optimise every angle.  Returns (ops, thetas, energies)
    with energies[i] the optimised energy after i + 1 operators."""
    ops, thetas, energies = [], np.zeros(0), []
    for _ in range(max_ops):
        psi = ansatz_state(system, ops, thetas, psi0)
        g = adapt.gradients(system.H, system.pool, psi)
        k, gmax = adapt.select(g, precision)
        if gmax < eps:
            break
        ops.append(k)
        thetas, E = reoptimize(system, ops, np.append(thetas, 0.0), psi0, gtol=gtol)
        energies.append(E)
    return ops, thetas, energies
