"""Pins of the oracle's energy, selection, line search and ADAPT loop (no GPU)."""

import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import adapt, evolve, fermion, mapping, pauli
from test_oracle_hamiltonian import hf_energy_closed_form
from test_oracle_pool import slater_condon_gradient_magnitude


def det_energy(h, g, occ):
    e = sum(h[I // 2, I // 2] for I in occ)
    for I in occ:
        for J in occ:
            i, j = I // 2, J // 2
            e += 0.5 * g[i, i, j, j]
            if I % 2 == J % 2:
                e -= 0.5 * g[i, j, j, i]
    return e


@pytest.fixture(scope="module", params=[mapping.JW, mapping.BK])
def c0(request):
    ints, ne = synth.config0()
    return ints, ne, adapt.build_system(ints, ne, request.param)


def test_config0_one_step_closed_form(c0):
    """Config 0: one ADAPT step from HF, theta = 0.05, in closed form.

    From |HF>, A|HF> = +-|Phi_k> and A^2|HF> = -|HF>, so
    T5|HF> = c5|HF> + s5 A|HF> and the energy follows from Slater-Condon
    matrix elements.
    """
    ints, ne, sysm = c0
    psi = adapt.hf_state(8, ne, sysm.mapping)
    res, out = adapt.adapt_step(sysm, psi, eps=1e-3, theta=0.05, renormalise=False)
    e_hf = hf_energy_closed_form(ints.h, ints.g, ne)
    assert abs(res.energy - e_hf) <= 1e-12
    mags = np.array([slater_condon_gradient_magnitude(ints.h, ints.g, ne, e) for e in sysm.excitations])
    k_ref = int(np.nonzero(mags >= mags.max() - 1e-9 * max(1, mags.max()))[0][0])
    assert res.selected == k_ref
    assert abs(res.max_grad - mags.max()) <= 1e-13
    th = 0.05
    c5 = 1 - th ** 2 / 2 + th ** 4 / 24
    s5 = th - th ** 3 / 6 + th ** 5 / 120
    exc = sysm.excitations[k_ref]
    half = len(exc) // 2
    occ = (set(range(ne)) - set(exc[:half])) | set(exc[half:])
    e_k = det_energy(ints.h, ints.g, sorted(occ))
    h0k = res.gradients[k_ref] / 2.0      # <HF|H A|HF> = g/2 (signed)
    e_ref = (c5 ** 2 * e_hf + s5 ** 2 * e_k + 2 * c5 * s5 * h0k) / (c5 ** 2 + s5 ** 2)
    assert abs(adapt.energy(sysm.H, out)[0] - e_ref) <= 1e-12
    ex = evolve.expm_dense(sysm.pool[k_ref], th) @ psi
    fid = abs(np.vdot(ex, out)) ** 2 / np.vdot(out, out).real
    assert fid > 0.999999 and np.linalg.norm(ex - out) <= th ** 6 / 720 + 1e-15


def test_rayleigh_quotient_scale_invariant(c0):
    _, _, sysm = c0
    psi = synth.random_state(8, 9)
    e1 = adapt.energy(sysm.H, psi)[0]
    e2 = adapt.energy(sysm.H, 3.5j * psi)[0]
    assert abs(e1 - e2) <= 1e-13
    dense = sysm.H.toarray()
    assert abs(e1 - (psi.conj() @ dense @ psi).real) <= 1e-12


def test_tie_rule():
    g = np.array([0.1, -0.3, 0.3, 0.3 - 5e-10, 0.29])
    assert adapt.select(g, adapt.FP64) == (1, 0.3)
    g = np.array([0.1, 0.3 - 2e-9, -0.3])
    assert adapt.select(g, adapt.FP64)[0] == 2
    g = np.array([0.1, 0.3 - 5e-6, -0.3])
    assert adapt.select(g, adapt.C64)[0] == 1


def test_line_search_energy_curve(c0):
    _, _, sysm = c0
    psi = evolve.normalise(synth.random_state(8, 12))
    for k in (0, 7, 20):
        A = sysm.pool[k]
        coef = adapt.line_search_coefficients(sysm.H, A, psi)
        for th in (-2.0, -0.3, 0.0, 0.11, 1.4, math.pi):
            ref = adapt.energy(sysm.H, evolve.expm_dense(A, th) @ psi)[0]
            assert abs(adapt.line_energy(coef, th) - ref) <= 1e-12
        ths = adapt.line_search(coef)
        grid = np.linspace(-math.pi, math.pi, 20001)
        emin = min(adapt.line_energy(coef, t) for t in grid)
        assert adapt.line_energy(coef, ths) <= emin + 1e-12
        assert abs(adapt._line_d1(coef, ths)) <= 1e-9


def test_line_search_derivatives():
    rng = np.random.default_rng(0)
    coef = tuple(rng.normal(size=6))
    h = 1e-6
    for th in (-1.0, 0.2, 2.9):
        d1 = (adapt.line_energy(coef, th + h) - adapt.line_energy(coef, th - h)) / (2 * h)
        d2 = (adapt._line_d1(coef, th + h) - adapt._line_d1(coef, th - h)) / (2 * h)
        assert abs(d1 - adapt._line_d1(coef, th)) <= 1e-8
        assert abs(d2 - adapt._line_d2(coef, th)) <= 1e-7


@pytest.mark.slow
def test_adapt_trajectory_invariants():
    """Config-1 shape, shortened: monotone energy, variational bound, JW == BK."""
    ints, ne = synth.config1()
    energies = {}
    for mp in (mapping.JW, mapping.BK):
        sysm = adapt.build_system(ints, ne, mp)
        psi = adapt.hf_state(12, ne, mp)
        res, _ = adapt.trajectory(sysm, psi, eps=1e-3, n_iter=5)
        e = [r.energy for r in res]
        assert all(b <= a + 1e-9 for a, b in zip(e, e[1:]))
        energies[mp] = (e, [r.selected for r in res])
        if mp == mapping.JW:
            # lowest eigenvalue in the n_e = 8 sector (occupation basis = JW)
            n = np.arange(1 << 12)
            sector = np.nonzero(np.bitwise_count(n) == ne)[0]
            Hs = sysm.H[sector][:, sector]
            lam = spla.eigsh(Hs.real, k=1, which="SA")[0][0]
            assert min(e) >= lam - 1e-10
    assert energies[mapping.JW][1] == energies[mapping.BK][1]
    assert np.abs(np.array(energies[mapping.JW][0]) - np.array(energies[mapping.BK][0])).max() <= 1e-10


@pytest.mark.parametrize("mp", [mapping.JW, mapping.BK])
def test_line_search_tie_takes_the_near_minimum(mp):
    """The line search's tie reading, pinned by a closed form.

    From psi = |HF>, every pool generator gives A|HF> = +-|Phi_k> and
    A^2|HF> = -|HF>, so exp(theta A)|HF> = cos(theta)|HF> + sin(theta)A|HF>
    and the energy along the curve is

        E(theta) = a + b cos(2 theta) + c sin(2 theta),
        a = (E_HF + E_k)/2,  b = (E_HF - E_k)/2,  c = <HF|H A|HF>,

    with E_HF and E_k the Slater-Condon determinant energies and |c| half
    the Slater-Condon gradient magnitude.  The curve is pi-periodic: its two
    minima, theta_1 = atan2(-c, -b)/2 in (-pi/2, pi/2] and theta_1 -+ pi,
    tie exactly.  The reading (smallest |theta| among tied samples) must
    return theta_1.  The sign of c is read off the dense exponential's
    energy at theta = pi/4 (E = a + c there), not off the oracle's
    line-search coefficients.
    """
    ints, ne = synth.config0()
    sysm = adapt.build_system(ints, ne, mp)
    psi = adapt.hf_state(8, ne, mp)
    e_hf = hf_energy_closed_form(ints.h, ints.g, ne)
    partner_below = 0
    checked = 0
    for k, exc in enumerate(sysm.excitations):
        half = len(exc) // 2
        occ = (set(range(ne)) - set(exc[:half])) | set(exc[half:])
        e_k = det_energy(ints.h, ints.g, sorted(occ))
        a, b = 0.5 * (e_hf + e_k), 0.5 * (e_hf - e_k)
        cmag = 0.5 * slater_condon_gradient_magnitude(ints.h, ints.g, ne, exc)
        if cmag < 1e-6:
            continue                    # no unique pair of minima to tell apart
        e_quarter = adapt.energy(sysm.H, evolve.expm_dense(sysm.pool[k], math.pi / 4) @ psi)[0]
        c = math.copysign(cmag, e_quarter - a)
        assert abs(abs(e_quarter - a) - cmag) <= 1e-10
        th_ref = 0.5 * math.atan2(-c, -b)
        partner = th_ref - math.pi if th_ref > 0 else th_ref + math.pi
        coef = adapt.line_search_coefficients(sysm.H, sysm.pool[k], psi)
        assert abs(adapt.line_energy(coef, partner) - adapt.line_energy(coef, th_ref)) <= 1e-12
        th = adapt.line_search(coef)
        assert abs(th - th_ref) <= 1e-9, (k, th, th_ref)
        checked += 1
        partner_below += partner < -math.pi / 2
    assert checked >= 20
    assert partner_below >= 1          # a case where the far minimum comes first in sample order
