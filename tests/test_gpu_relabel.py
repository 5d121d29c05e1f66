"""GPU parity: relabelled encodings (JW/BK with the qubits moved to other
index bits, or the basis index carried by an invertible GF(2) map: a
memory layout only).

A relabelled state holds the base mapping's amplitude b at index
relabel[b].  Energies, gradients and ADAPT steps must equal the oracle's
base-mapping values; the support-only and full-state updates must give the
natural layout's amplitudes, moved by the relabelling, bit for bit (the
same products on the same pairs)."""

import numpy as np
import pytest

import paper_2606_29692_gb300 as tq
import synth
from gpu_util import fidelity, rel_l2, to_state
from oracle import adapt as oadapt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return tq.Context(0)


def _random_invertible(N, rng):
    while True:
        rows = rng.integers(0, 1 << N, size=N, dtype=np.int64).astype(np.uint64)
        if np.linalg.matrix_rank(((rows[:, None] >> np.arange(N, dtype=np.uint64)) & 1).astype(np.float64)) < N:
            continue                       # real rank below N: singular over GF(2) as well
        try:
            tq.mapping_linear(0, rows)     # the library's GF(2) check decides
            return rows
        except tq.TQError:
            continue


def _layout(n, ne, mp, which):
    """(mapping id, index map) of a relabelled layout of the base mapping."""
    N = 2 * n
    if which in ("sector", "random"):
        order = (tq.pool_sector_order(n, ne, mp, 4) if which == "sector"
                 else np.random.default_rng(5 + mp).permutation(N).astype(np.int32))
        return tq.mapping_relabelled(mp, order), tq.relabel_index(order)
    rows = (tq.pool_sector_basis(n, ne, mp) if which == "linear"
            else _random_invertible(N, np.random.default_rng(9 + mp)))
    return tq.mapping_linear(mp, rows), tq.linear_index(rows)


@pytest.mark.parametrize("which", ["sector", "random", "linear", "random_linear"])
@pytest.mark.parametrize("mp", [0, 1])
@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
def test_relabelled_energy_gradients_step_match_oracle(ctx, mp, prec, which):
    ints, ne = synth.config1()
    n, N = ints.n_spatial, 12
    rl, ix = _layout(n, ne, mp, which)
    sysm = oadapt.build_system(ints, ne, mp)
    psi = synth.random_state(N, 31 + mp)
    e_ref, _ = oadapt.energy(sysm.H, psi)
    g_ref = oadapt.gradients(sysm.H, sysm.pool, psi)
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, rl, prec)
    pool = tq.build_pool(ctx, n, ne, rl)
    moved = np.zeros_like(psi)
    moved[ix] = psi
    st = to_state(ctx, moved, N, prec)
    tol = 1e-10 if prec == tq.TQ_C128 else 1e-6
    assert abs(tq.energy(ctx, ham, st) - e_ref) <= tol
    assert np.abs(tq.pool_gradients(ctx, ham, pool, st) - g_ref).max() <= tol
    # one ADAPT step with the line search from HF
    tq.state_set_hf(st, ne, rl)
    r = tq.adapt_step(ctx, ham, pool, st, 1e-3)
    ref, nxt = oadapt.adapt_step(sysm, oadapt.hf_state(N, ne, mp), 1e-3, None,
                                 oadapt.FP64 if prec == tq.TQ_C128 else oadapt.C64)
    assert r["selected"] == ref.selected and abs(r["energy"] - ref.energy) <= tol
    got = st.numpy()[ix]
    if prec == tq.TQ_C128:
        assert rel_l2(got, nxt) <= 1e-12
    else:
        assert fidelity(got, nxt) > 0.999999


@pytest.mark.parametrize("which", ["sector", "linear"])
@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
def test_relabelled_support_update_is_the_natural_one_moved(ctx, prec, which):
    """The headline shape (14 qubits, BK, pool of 204) on 512 states: the
    support-only update in a sector-packed layout (qubit order or GF(2)
    map) equals the natural layout's result moved by the index map, bit for
    bit, for every schedule; so does the full-state update."""
    import torch
    n, ne, mp = 7, 6, 1
    N = 14
    rl, ixn = _layout(n, ne, mp, which)
    ix = torch.as_tensor(ixn).cuda()
    pool_n = tq.build_pool(ctx, n, ne, mp)
    pool_r = tq.build_pool(ctx, n, ne, rl)
    S = 512
    rng = np.random.default_rng(17)
    dt = torch.complex128 if prec == tq.TQ_C128 else torch.complex64
    psi = torch.as_tensor(np.stack([synth.random_state(N, 7000 + b) for b in range(S)])).to(dt).cuda()
    k = torch.as_tensor(rng.integers(0, pool_n.M, size=S).astype(np.int32)).cuda()
    th = torch.as_tensor(rng.normal(0.0, 0.2, size=S)).cuda()
    for ppt in (1, -1, 4):
        ctx.set_support_schedule(prec, ppt)
        a = psi.clone()
        b = torch.zeros_like(psi)
        b[:, ix] = psi
        na = torch.ones(S, dtype=torch.float64, device="cuda")
        nb = na.clone()
        tq.evolve_taylor5_batch_support(ctx, pool_n, a, k, th, na, prec=prec)
        tq.evolve_taylor5_batch_support(ctx, pool_r, b, k, th, nb, prec=prec)
        assert torch.equal(b[:, ix], a), ppt
        assert torch.allclose(na, nb, rtol=1e-12 if prec == tq.TQ_C128 else 1e-6, atol=0), ppt
    ctx.set_support_schedule(prec, -1 if prec == tq.TQ_C64 else 4)
    a = psi.clone()
    b = torch.zeros_like(psi)
    b[:, ix] = psi
    tq.evolve_taylor5_batch(ctx, pool_n, a, k, th, prec=prec)
    tq.evolve_taylor5_batch(ctx, pool_r, b, k, th, prec=prec)
    assert torch.equal(b[:, ix], a)


def test_relabelled_sector_basis_is_the_natural_one_moved(ctx):
    """Sector-restricted objects take relabelled mappings too: the basis is
    the natural basis moved by the relabelling, and the sector energy is the
    full-space one."""
    import torch
    ints, ne = synth.config1()
    n = ints.n_spatial
    order = tq.pool_sector_order(n, ne, 1, 3)
    rl = tq.mapping_relabelled(1, order)
    ix = tq.relabel_index(order)
    nat = tq.sector_basis(n, 4, 4, 1).astype(np.int64)
    got = tq.sector_basis(n, 4, 4, rl).astype(np.int64)
    assert np.array_equal(got, ix[nat])
    ham_s = tq.build_hamiltonian_sector(ctx, ints.h, ints.g, ints.e_const, rl, tq.TQ_C128, 4, 4)
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, rl, tq.TQ_C128)
    v = synth.random_state(12, 99)[: nat.size]
    full = np.zeros(1 << 12, dtype=np.complex128)
    full[got] = v
    st_s = tq.State(ctx, 12, tq.TQ_C128, tensor=torch.as_tensor(v).cuda(), sector=(4, 4))
    st = to_state(ctx, full, 12, tq.TQ_C128)
    assert abs(tq.energy(ctx, ham_s, st_s) - tq.energy(ctx, ham, st)) <= 1e-10
