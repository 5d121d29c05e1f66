"""GPU checkpoints, replay and the FCIDUMP loader end to end.

State checkpoints round-trip bit for bit and refuse a mismatched target; an
ADAPT trajectory replayed from its recorded operators and angles
reproduces the state bit for bit (the kernels are deterministic); a
Hamiltonian built from FCIDUMP integrals has the original's energies.
"""

import numpy as np
import pytest

import paper_2606_29692_gb300 as tq
import synth
from gpu_util import to_state
from oracle import adapt
from test_oracle_hamiltonian import hf_energy_closed_form

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return tq.Context(0)


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
def test_state_checkpoint_round_trip(ctx, prec, tmp_path):
    psi = synth.random_state(10, 3)
    a = to_state(ctx, psi, 10, prec)
    path = str(tmp_path / "s.bin")
    tq.state_save(a, path)
    b = tq.State(ctx, 10, prec)
    tq.state_load(b, path)
    assert np.array_equal(a.numpy(), b.numpy())
    other = tq.State(ctx, 10, tq.TQ_C64 if prec == tq.TQ_C128 else tq.TQ_C128)
    with pytest.raises(tq.TQError):
        tq.state_load(other, path)
    with pytest.raises(tq.TQError):
        tq.state_load(tq.State(ctx, 12, prec), path)
    with pytest.raises(tq.TQError):
        tq.state_load(tq.State(ctx, 10, prec, sector=(2, 3)), path)


def test_sector_state_checkpoint(ctx, tmp_path):
    a = to_state(ctx, np.arange(tq.sector_dim(5, 2, 3)) * (1 + 0.5j), 10, tq.TQ_C64, sector=(2, 3))
    path = str(tmp_path / "s.bin")
    tq.state_save(a, path)
    b = tq.State(ctx, 10, tq.TQ_C64, sector=(2, 3))
    tq.state_load(b, path)
    assert np.array_equal(a.numpy(), b.numpy())
    with pytest.raises(tq.TQError):
        tq.state_load(tq.State(ctx, 10, tq.TQ_C64, sector=(3, 2)), path)


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
def test_trajectory_replay_is_bit_exact(ctx, prec, tmp_path):
    ints, ne = synth.config1()
    mp = 1
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, 0.0, mp, prec)
    pool = tq.build_pool(ctx, 6, ne, mp)
    st = tq.State(ctx, 12, prec)
    tq.state_set_hf(st, ne, mp)
    ops, ths, energies = [], [], []
    for _ in range(8):
        r = tq.adapt_step(ctx, ham, pool, st, 1e-3)
        if r["converged"]:
            break
        ops.append(r["selected"])
        ths.append(r["theta"])
        energies.append(r["energy"])
    path = str(tmp_path / "traj.bin")
    tq.state_save(st, path)
    # replay from HF in a fresh state
    re = tq.State(ctx, 12, prec)
    tq.state_set_hf(re, ne, mp)
    tq.replay(ctx, pool, re, ops, ths)
    assert np.array_equal(re.numpy(), st.numpy())
    # and the checkpoint restores it
    back = tq.State(ctx, 12, prec)
    tq.state_load(back, path)
    assert np.array_equal(back.numpy(), st.numpy())
    assert tq.energy(ctx, ham, back) == tq.energy(ctx, ham, st)


@pytest.mark.parametrize("mp", [0, 1])
def test_fcidump_loader_end_to_end(ctx, mp, tmp_path):
    ints = synth.integrals(7, 44)
    path = str(tmp_path / "FCIDUMP")
    tq.write_fcidump(path, ints.h, ints.g, 0.5, 6)
    r = tq.read_fcidump(path)
    ham = tq.build_hamiltonian(ctx, r.h, r.g, r.e_const, mp, tq.TQ_C128)
    st = tq.State(ctx, 14, tq.TQ_C128)
    tq.state_set_hf(st, r.n_electrons, mp)
    assert abs(tq.energy(ctx, ham, st) - (hf_energy_closed_form(ints.h, ints.g, 6) + 0.5)) <= 1e-10
    ref = tq.build_hamiltonian(ctx, ints.h, ints.g, 0.5, mp, tq.TQ_C128)
    psi = to_state(ctx, synth.random_state(14, 5), 14, tq.TQ_C128)
    assert tq.energy(ctx, ham, psi) == tq.energy(ctx, ref, psi)
