"""GPU parity: energy (CSR and matrix-free) and pool gradients."""

import numpy as np
import pytest

import paper_2606_29692_gb300 as tq
import synth
from gpu_util import to_state
from oracle import adapt as oadapt
from oracle import evolve

pytestmark = pytest.mark.gpu

CFG = {"c0": synth.config0, "c1": synth.config1, "c2": synth.config2}


@pytest.fixture(scope="module")
def ctx():
    return tq.Context(0)


_SYS = {}


def osys(cfg, mp):
    if (cfg, mp) not in _SYS:
        ints, ne = CFG[cfg]()
        _SYS[(cfg, mp)] = (ints, ne, oadapt.build_system(ints, ne, mp))
    return _SYS[(cfg, mp)]


def _states(sysm, nq, ne, mp):
    hf = oadapt.hf_state(nq, ne, mp)
    # a correlated state: HF rotated by a few generators
    psi = hf
    for k, th in ((0, 0.1), (len(sysm.pool) - 1, -0.2), (len(sysm.pool) // 2, 0.15)):
        psi = evolve.taylor5(sysm.pool[k], psi, th)
    return {"hf": hf, "corr": psi, "rand": synth.random_state(nq, 4) * 0.7}


@pytest.mark.parametrize("sched", [32, tq.TQ_SPMV_XELL])
@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
@pytest.mark.parametrize("cfg,mp", [("c0", 0), ("c0", 1), ("c1", 0), ("c1", 1), ("c2", 1)])
def test_energy_and_gradients_match_oracle(ctx, cfg, mp, prec, sched):
    ctx.set_spmv_schedule(sched)
    try:
        _energy_and_gradients(ctx, cfg, mp, prec)
    finally:
        ctx.set_spmv_schedule(tq.TQ_SPMV_XELL)


def _energy_and_gradients(ctx, cfg, mp, prec):
    ints, ne, sysm = osys(cfg, mp)
    nq = 2 * ints.n_spatial
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, mp, prec)
    pool = tq.build_pool(ctx, ints.n_spatial, ne, mp)
    for name, psi in _states(sysm, nq, ne, mp).items():
        st = to_state(ctx, psi, nq, prec)
        if prec == tq.TQ_C64:
            psi = st.numpy()          # compare on the state the GPU actually holds
        E_ref, _ = oadapt.energy(sysm.H, psi)
        g_ref = oadapt.gradients(sysm.H, sysm.pool, psi)
        E = tq.energy(ctx, ham, st)
        E_mf = tq.energy_matrix_free(ctx, ham, st)
        g = tq.pool_gradients(ctx, ham, pool, st)
        if prec == tq.TQ_C128:
            assert abs(E - E_ref) <= 1e-10, name
            assert abs(E_mf - E_ref) <= 1e-10, name
            assert np.abs(g - g_ref).max() <= 1e-10, name
        else:
            assert abs(E - E_ref) <= 1e-6, name
            assert abs(E_mf - E_ref) <= 1e-10, name   # matrix-free sums in float64
            assert np.abs(g - g_ref).max() <= 1e-6, name


def test_gradients_device_output(ctx):
    import torch
    ints, ne, sysm = osys("c1", 1)
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, 0.0, 1, tq.TQ_C128)
    pool = tq.build_pool(ctx, 6, ne, 1)
    psi = _states(sysm, 12, ne, 1)["corr"]
    st = to_state(ctx, psi, 12, tq.TQ_C128)
    out = torch.zeros(pool.M, dtype=torch.float64, device="cuda")
    tq.pool_gradients(ctx, ham, pool, st, out=out)
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - oadapt.gradients(sysm.H, sysm.pool, psi)).max() <= 1e-10


def test_energy_rejects_mismatch(ctx):
    ints, ne, _ = osys("c0", 0)
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, 0.0, 0, tq.TQ_C128)
    st64 = to_state(ctx, synth.random_state(8, 1), 8, tq.TQ_C64)
    with pytest.raises(tq.TQError):
        tq.energy(ctx, ham, st64)
    st10 = to_state(ctx, synth.random_state(10, 1), 10, tq.TQ_C128)
    with pytest.raises(tq.TQError):
        tq.energy(ctx, ham, st10)


def test_every_spmv_schedule_agrees(ctx):
    ints, ne, sysm = osys("c2", 1)
    for prec in (tq.TQ_C128, tq.TQ_C64):
        ham = tq.build_hamiltonian(ctx, ints.h, ints.g, 0.0, 1, prec)
        psi = _states(sysm, 14, ne, 1)["corr"]
        st = to_state(ctx, psi, 14, prec)
        ref = oadapt.energy(sysm.H, st.numpy())[0]
        for lanes in (4, 8, 16, 32, tq.TQ_SPMV_XELL):
            ctx.set_spmv_schedule(lanes)
            assert abs(tq.energy(ctx, ham, st) - ref) <= (1e-10 if prec == tq.TQ_C128 else 1e-6)
        best, ms = tq.autotune_spmv(ctx, ham, st)
        assert best in (4, 8, 16, 32, tq.TQ_SPMV_XELL) and ms > 0
    ctx.set_spmv_schedule(tq.TQ_SPMV_XELL)
