"""Oracle pins for the sector-restricted basis (fixed alpha and beta counts).

The restriction is checked against the full-space oracle, which is pinned
on its own: H and every pool generator are block-diagonal over sectors, the
sector spectra together are the full spectrum, JW and BK restrictions are
the same matrix, and energies, gradients and Taylor-5 updates of a state in
a sector equal the full-space ones.
"""

from itertools import product
from math import comb

import numpy as np
import pytest

import synth
from oracle import adapt, evolve, fermion, mapping, sector


def test_colex_rank_textbook():
    # 2-subsets of {0,1,2,3} in colexicographic order
    order = [(0, 1), (0, 2), (1, 2), (0, 3), (1, 3), (2, 3)]
    assert [sector.subset_rank(s) for s in order] == list(range(6))
    assert sector.subset_rank([]) == 0
    assert sector.subset_rank([4]) == 4


@pytest.mark.parametrize("n,na,nb", [(1, 0, 1), (3, 1, 2), (4, 2, 2), (5, 3, 2), (6, 4, 4)])
def test_basis_is_the_filtered_occupation_space(n, na, nb):
    b = sector.basis(n, na, nb)
    assert len(b) == comb(n, na) * comb(n, nb) == sector.dimension(n, na, nb)
    # brute force: every occupation index with the right counts, exactly once
    brute = [o for o in range(1 << (2 * n))
             if bin(o & int("01" * n, 2)).count("1") == na and bin(o & int("10" * n, 2)).count("1") == nb]
    assert sorted(b.tolist()) == brute
    assert [sector.rank(int(o), n, na, nb) for o in b] == list(range(len(b)))
    assert sector.rank(1 << (2 * n), n, na, nb) == -1


def _system(cfg, mp):
    ints, ne = {"c0": synth.config0, "n3": lambda: (synth.integrals(3, 6), 2)}[cfg]()
    return adapt.build_system(ints, ne, mp)


@pytest.mark.parametrize("cfg,mp", [("n3", 0), ("n3", 1), ("c0", 0), ("c0", 1)])
def test_operators_block_diagonal_and_spectrum_partitions(cfg, mp):
    sysm = _system(cfg, mp)
    n, N = sysm.n_spatial, 2 * sysm.n_spatial
    H = sysm.H.toarray()
    eig_sectors = []
    covered = np.zeros(1 << N, dtype=bool)
    for na, nb in product(range(n + 1), repeat=2):
        q = sector.qubit_basis(n, na, nb, mp)
        covered[q] = True
        out = np.ones(1 << N, dtype=bool)
        out[q] = False
        assert np.all(H[np.ix_(q, np.nonzero(out)[0])] == 0)       # no coupling out of S
        for A in sysm.pool:
            Ad = A.toarray()
            assert np.all(Ad[np.ix_(np.nonzero(out)[0], q)] == 0)  # A maps S into S
        eig_sectors.extend(np.linalg.eigvalsh(sector.restrict(sysm.H, q).toarray()))
    assert covered.all()
    full = np.linalg.eigvalsh(H)
    assert np.allclose(np.sort(eig_sectors), full, atol=1e-10)


@pytest.mark.parametrize("cfg", ["n3", "c0"])
def test_jw_and_bk_restrictions_are_the_same_matrix(cfg):
    jw, bk = _system(cfg, 0), _system(cfg, 1)
    n = jw.n_spatial
    for na, nb in [(1, 1), (2, 1), (2, 2)]:
        if na > n or nb > n:
            continue
        a = sector.SectorSystem(jw, na, nb)
        b = sector.SectorSystem(bk, na, nb)
        scale = np.abs(jw.H.data).max()
        assert np.abs((a.H - b.H).toarray()).max() <= 1e-13 * scale
        for A, B in zip(a.pool, b.pool):
            assert np.abs((A - B).toarray()).max() <= 1e-14


@pytest.mark.parametrize("mp", [0, 1])
def test_restricted_generators_are_signed_involution_pairs(mp):
    s = sector.SectorSystem(_system("c0", mp), 2, 2)
    for A in s.pool:
        Ad = A.toarray()
        assert np.allclose(Ad, -Ad.conj().T)
        assert set(np.unique(Ad.real)) <= {-1.0, 0.0, 1.0} and np.all(Ad.imag == 0)
        assert np.all((Ad != 0).sum(axis=1) <= 1)


@pytest.mark.parametrize("mp", [0, 1])
def test_energy_gradients_update_equal_full_space(mp):
    full = _system("c0", mp)
    s = sector.SectorSystem(full, 2, 2)
    rng = np.random.default_rng(11)
    psi_s = rng.normal(size=s.dim) + 1j * rng.normal(size=s.dim)
    psi = sector.embed(psi_s, s.qidx, 8)
    E_s, w_s = adapt.energy(s.H, psi_s)
    E, w = adapt.energy(full.H, psi)
    assert abs(E_s - E) <= 1e-12 * max(1.0, abs(E))
    assert np.allclose(sector.embed(w_s, s.qidx, 8), w, atol=1e-12)
    assert np.allclose(adapt.gradients(s.H, s.pool, psi_s), adapt.gradients(full.H, full.pool, psi), atol=1e-12)
    for k in (0, 5, len(s.pool) - 1):
        out_s = evolve.taylor5(s.pool[k], psi_s, 0.3)
        out = evolve.taylor5(full.pool[k], psi, 0.3)
        assert np.allclose(sector.embed(out_s, s.qidx, 8), out, atol=1e-12)


@pytest.mark.parametrize("mp", [0, 1])
def test_hf_state_embeds_to_the_full_space_hf(mp):
    s = sector.SectorSystem(_system("c0", mp), 2, 2)
    hf = sector.hf_state(4, 4, 2, 2)
    assert hf[0] == 1.0                      # the lowest determinant has rank 0
    assert np.array_equal(sector.embed(hf, s.qidx, 8), adapt.hf_state(8, 4, mp))
    with pytest.raises(ValueError):
        sector.hf_state(4, 4, 3, 1)


def test_adapt_step_in_the_sector_matches_full_space():
    full = _system("c0", 1)
    s = sector.SectorSystem(full, 2, 2)
    r_s, psi_s = adapt.adapt_step(s, sector.hf_state(4, 4, 2, 2), 1e-3)
    r, psi = adapt.adapt_step(full, adapt.hf_state(8, 4, 1), 1e-3)
    assert r_s.selected == r.selected and abs(r_s.theta - r.theta) <= 1e-10
    assert abs(r_s.energy - r.energy) <= 1e-12
    assert np.allclose(sector.embed(psi_s, s.qidx, 8), psi, atol=1e-12)
