"""Pins of the oracle's Taylor-5 update (Eqs. (6)-(8)) and exponentials (no GPU)."""

import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import synth
from oracle import adapt, evolve, mapping, pauli

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _const(name):
    for line in open(os.path.join(GOLDEN, "paper_constants.txt")):
        if line.startswith(name + " "):
            return [float(v) for v in line.split()[1:]]
    raise KeyError(name)


def test_coefficients_are_the_printed_scalars():
    # Eq. (8) and Sec. III-D step 4: 1, theta, 1/2, 1/6, 1/24, 1/120.
    ref = _const("taylor_scalars")
    assert evolve.taylor_coefficients(1.0) == ref


def test_nilpotent_block_is_exact():
    # For a 6 x 6 shift matrix J (J^6 = 0) the truncated series IS the
    # exponential, so the chain must reproduce scipy's expm exactly.
    J = np.diag(np.ones(5), -1)
    for theta in (0.3, -1.7, 2.5):
        psi = np.arange(1, 7) + 0.5j
        out = evolve.taylor5(sp.csr_matrix(J), psi, theta)
        assert np.abs(out - sla.expm(theta * J) @ psi).max() <= 1e-13


def test_scalar_case_is_truncated_series():
    a = np.array([0.3, -1.1, 2.0])
    theta = 0.7
    out = evolve.taylor5(sp.diags(a), np.ones(3), theta)
    ref = sum((theta * a) ** k / math.factorial(k) for k in range(6))
    assert np.abs(out - ref).max() <= 1e-15


@pytest.fixture(scope="module")
def sys8():
    ints, ne = synth.config0()
    return adapt.build_system(ints, ne, mapping.JW)


def _closed_form_t5(A, psi, theta):
    return (psi + (theta - theta ** 3 / 6 + theta ** 5 / 120) * (A @ psi)
            + (theta ** 2 / 2 - theta ** 4 / 24) * (A @ (A @ psi)))


def _closed_form_exp(A, psi, theta):
    return psi + math.sin(theta) * (A @ psi) + (1 - math.cos(theta)) * (A @ (A @ psi))


@pytest.mark.parametrize("theta", [0.05, -0.2, 0.4, 1.0])
def test_chain_equals_closed_form(sys8, theta):
    psi = synth.random_state(8, 3)
    for A in sys8.pool[::5]:
        assert np.abs(evolve.taylor5(A, psi, theta) - _closed_form_t5(A, psi, theta)).max() <= 1e-15


@pytest.mark.parametrize("theta", [0.05, 0.4, -0.9])
def test_expm_routines_equal_closed_form(sys8, theta):
    psi = synth.random_state(8, 4)
    for A in sys8.pool[::7]:
        ref = _closed_form_exp(A, psi, theta)
        assert np.abs(evolve.expm_dense(A, theta) @ psi - ref).max() <= 1e-13
        assert np.abs(evolve.expm_apply(A, psi, theta) - ref).max() <= 1e-12


@pytest.mark.parametrize("theta", [0.05, 0.1, 0.4, -0.3])
def test_truncation_bound_and_fidelity(sys8, theta):
    psi = synth.random_state(8, 6)
    floor = _const("fidelity_floor")[0]
    for A in sys8.pool:
        t5 = evolve.taylor5(A, psi, theta)
        ex = evolve.expm_dense(A, theta) @ psi
        err = np.linalg.norm(ex - t5)
        assert err <= abs(theta) ** 6 / 720 * np.linalg.norm(psi) * (1 + 1e-9) + 1e-15
        fid = abs(np.vdot(ex, t5)) ** 2 / (np.vdot(t5, t5).real * np.vdot(ex, ex).real)
        assert fid > floor


@pytest.mark.parametrize("theta", [0.05, 0.4, 1.3])
def test_norm_growth_formula(sys8, theta):
    psi = synth.random_state(8, 7)
    for A in sys8.pool[::3]:
        t5 = evolve.taylor5(A, psi, theta)
        Apsi = A @ psi
        ref = (np.vdot(psi, psi).real + (theta ** 6 / 360 - theta ** 8 / 960 + theta ** 10 / 14400)
               * np.vdot(Apsi, Apsi).real)
        assert abs(np.vdot(t5, t5).real - ref) <= 1e-14
        ex = evolve.expm_dense(A, theta) @ psi
        assert abs(np.vdot(ex, ex).real - np.vdot(psi, psi).real) <= 1e-13


def test_dense_operator_estimate():
    # Sec. IV-C: 2^28 complex128 elements is about 4.3 GB.
    gb = _const("dense_operator_gb")[0]
    assert abs(2 ** 28 * 16 / 1e9 - gb) < 0.05
    assert _const("table1_dimension")[0] == 2 ** 14
    assert _const("table1_elements")[0] == 2 ** 28
