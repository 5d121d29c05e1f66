"""GPU parity for ADAPT-VQE with re-optimised angles.

The device energy and adjoint gradient of the Taylor-5 product ansatz, and
the device BFGS loop, against the oracle (``oracle.vqe``) on the same
inputs; in the full space and in a sector.
"""

import numpy as np
import pytest

import paper_2606_29692_gb300 as tq
import synth
from gpu_util import rel_l2, to_state
from oracle import adapt, sector, vqe

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return tq.Context(0)


CFG = {"c0": synth.config0, "c1": synth.config1, "n2": lambda: (synth.integrals(2, 9), 2)}
_SYS = {}


def osys(cfg, mp):
    if (cfg, mp) not in _SYS:
        ints, ne = CFG[cfg]()
        _SYS[(cfg, mp)] = (ints, ne, adapt.build_system(ints, ne, mp))
    return _SYS[(cfg, mp)]


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
@pytest.mark.parametrize("cfg,mp", [("c0", 0), ("c0", 1), ("c1", 1)])
def test_ansatz_energy_and_gradient_match_oracle(ctx, cfg, mp, prec):
    ints, ne, s = osys(cfg, mp)
    nq = 2 * ints.n_spatial
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, mp, prec)
    pool = tq.build_pool(ctx, ints.n_spatial, ne, mp)
    rng = np.random.default_rng(7)
    ops = rng.integers(0, len(s.pool), size=7)
    th = rng.normal(0, 0.3, size=7)
    psi0 = adapt.hf_state(nq, ne, mp)
    st0 = to_state(ctx, psi0, nq, prec)
    out = tq.State(ctx, nq, prec)
    E, g = tq.ansatz_energy_grad(ctx, ham, pool, st0, ops, th, psi_out=out)
    E_ref, g_ref = vqe.energy_and_gradient(s, list(ops), th, psi0)
    if prec == tq.TQ_C128:
        assert abs(E - E_ref) <= 1e-10
        assert np.abs(g - g_ref).max() <= 1e-9
        assert rel_l2(out.numpy(), vqe.ansatz_state(s, list(ops), th, psi0)) <= 1e-12
    else:
        assert abs(E - E_ref) <= 1e-6
        assert np.abs(g - g_ref).max() <= 2e-5
    assert np.array_equal(st0.numpy(), psi0.astype(st0.numpy().dtype))       # psi0 untouched
    E0, g0 = tq.ansatz_energy_grad(ctx, ham, pool, st0, [], [])
    assert abs(E0 - adapt.energy(s.H, psi0)[0]) <= (1e-10 if prec == tq.TQ_C128 else 1e-6) and g0.size == 0


@pytest.mark.parametrize("mp", [0, 1])
def test_adapt_vqe_matches_oracle(ctx, mp):
    ints, ne, s = osys("c0", mp)
    psi0 = adapt.hf_state(8, ne, mp)
    ops_ref, th_ref, en_ref = vqe.adapt_vqe(s, psi0, 1e-3, max_ops=6, gtol=1e-9)
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, mp, tq.TQ_C128)
    pool = tq.build_pool(ctx, 4, ne, mp)
    st0 = to_state(ctx, psi0, 8, tq.TQ_C128)
    out = tq.State(ctx, 8, tq.TQ_C128)
    ops, th, en = tq.adapt_vqe(ctx, ham, pool, st0, 1e-3, max_ops=6, gtol=1e-9, psi_out=out)
    assert ops.tolist() == ops_ref
    assert np.abs(en - np.array(en_ref)).max() <= 1e-9
    assert np.abs(th - th_ref).max() <= 1e-4
    E_out = adapt.energy(s.H, out.numpy())[0]
    assert abs(E_out - en[-1]) <= 1e-10


def test_adapt_vqe_two_electrons_reaches_fci_in_a_sector(ctx):
    ints, ne, s = osys("n2", 1)
    ham = tq.build_hamiltonian_sector(ctx, ints.h, ints.g, ints.e_const, 1, tq.TQ_C128, 1, 1)
    pool = tq.build_pool_sector(ctx, 2, ne, 1, 1, 1)
    st0 = tq.State(ctx, 4, tq.TQ_C128, sector=(1, 1))
    tq.state_set_hf(st0, ne, 1)
    ops, th, en = tq.adapt_vqe(ctx, ham, pool, st0, 1e-8, max_ops=6, gtol=1e-12)
    fci = np.linalg.eigvalsh(sector.restrict(s.H, sector.qubit_basis(2, 1, 1, 1)).toarray())[0]
    assert abs(en[-1] - fci) <= 1e-9
    assert np.all(np.diff(en) <= 1e-12)


def test_sector_and_full_space_adapt_vqe_agree(ctx):
    ints, ne = synth.config1()
    mp = 1
    na, nb = (ne + 1) // 2, ne // 2
    hs = tq.build_hamiltonian_sector(ctx, ints.h, ints.g, 0.0, mp, tq.TQ_C128, na, nb)
    ps = tq.build_pool_sector(ctx, 6, ne, mp, na, nb)
    ss = tq.State(ctx, 12, tq.TQ_C128, sector=(na, nb))
    tq.state_set_hf(ss, ne, mp)
    hf = tq.build_hamiltonian(ctx, ints.h, ints.g, 0.0, mp, tq.TQ_C128)
    pf = tq.build_pool(ctx, 6, ne, mp)
    sf = tq.State(ctx, 12, tq.TQ_C128)
    tq.state_set_hf(sf, ne, mp)
    a = tq.adapt_vqe(ctx, hs, ps, ss, 1e-3, max_ops=4, gtol=1e-9)
    b = tq.adapt_vqe(ctx, hf, pf, sf, 1e-3, max_ops=4, gtol=1e-9)
    assert a[0].tolist() == b[0].tolist()
    assert np.abs(a[2] - b[2]).max() <= 1e-9


def test_ansatz_rejects_bad_input(ctx):
    ints, ne, s = osys("c0", 0)
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, 0.0, 0, tq.TQ_C128)
    pool = tq.build_pool(ctx, 4, ne, 0)
    st0 = to_state(ctx, adapt.hf_state(8, ne, 0), 8, tq.TQ_C128)
    with pytest.raises(tq.TQError):
        tq.ansatz_energy_grad(ctx, ham, pool, st0, [999], [0.1])
    with pytest.raises(tq.TQError):
        tq.ansatz_energy_grad(ctx, ham, pool, st0, [1], [float("nan")])
    with pytest.raises(tq.TQError):
        tq.adapt_vqe(ctx, ham, pool, st0, -1.0)
