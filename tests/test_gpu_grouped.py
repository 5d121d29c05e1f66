"""GPU parity: the support-only update for groups of states that share a
generator, interleaved amplitude-major within each group (TQ_GROUP_C64 = 4
complex64 or TQ_GROUP_C128 = 2 complex128 states per 32-byte sector).

Each state's amplitudes must be those the per-state support update gives
it, bit for bit (the same products on the same pairs), for every schedule;
its carried norm agrees to rounding; a few states are checked against the
oracle's chain of Eqs. (7)-(8)."""

import numpy as np
import pytest

import paper_2606_29692_gb300 as tq
import synth
from gpu_util import fidelity, rel_l2
from oracle import evolve, pauli

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return tq.Context(0)


def _setup(n, ne, mp, n_groups, prec, seed):
    G = tq.TQ_GROUP_C128 if prec == tq.TQ_C128 else tq.TQ_GROUP_C64
    N = 2 * n
    D = 1 << N
    rng = np.random.default_rng(seed)
    psi = np.stack([synth.random_state(N, seed * 1000 + b) for b in range(n_groups * G)])
    return G, D, rng, psi


def _interleave(t, n_groups, G, D):
    return t.reshape(n_groups, G, D).permute(0, 2, 1).contiguous()


def _deinterleave(t, n_groups, G, D):
    return t.reshape(n_groups, D, G).permute(0, 2, 1).reshape(n_groups * G, D)


@pytest.mark.parametrize("prec", [tq.TQ_C64, tq.TQ_C128])
@pytest.mark.parametrize("n,ne,mp", [(4, 4, 0), (6, 8, 1), (7, 6, 1)])
def test_grouped_equals_per_state_update(ctx, n, ne, mp, prec):
    import torch
    pool = tq.build_pool(ctx, n, ne, mp)
    n_groups = 48
    G, D, rng, psi = _setup(n, ne, mp, n_groups, prec, 11 + n + mp)
    dt = torch.complex128 if prec == tq.TQ_C128 else torch.complex64
    kg = rng.integers(0, pool.M, size=n_groups).astype(np.int32)
    kg[:3] = [0, pool.M - 1, pool.M // 2]
    th = rng.normal(0.0, 0.3, size=n_groups * G)
    th[0] = 0.0
    ks = np.repeat(kg, G).astype(np.int32)
    ref = torch.as_tensor(psi).to(dt).cuda()
    n0 = (ref.abs().double() ** 2).sum(dim=1)
    nref = n0.clone()
    tq.evolve_taylor5_batch_support(ctx, pool, ref, torch.as_tensor(ks).cuda(), torch.as_tensor(th).cuda(), nref,
                                    prec=prec)
    scheds = [(lanes, ppt) for lanes in ((1, 2) if prec == tq.TQ_C128 else (1, 2, 4)) for ppt in (1, 2, 4)]
    for sched in scheds:
        ctx.set_grouped_schedule(prec, *sched)
        gpsi = _interleave(torch.as_tensor(psi).to(dt).cuda(), n_groups, G, D)
        ng = n0.clone()
        tq.evolve_taylor5_batch_grouped(ctx, pool, gpsi, torch.as_tensor(kg).cuda(), torch.as_tensor(th).cuda(), ng,
                                        prec=prec)
        got = _deinterleave(gpsi, n_groups, G, D)
        assert torch.equal(torch.view_as_real(got), torch.view_as_real(ref)), sched
        tol = 1e-12 if prec == tq.TQ_C128 else 1e-6
        assert (ng - nref).abs().max().item() <= tol * nref.max().item(), sched
    ctx.set_grouped_schedule(prec, 1, 1)
    # a few states against the oracle
    pps = pauli.pool_pauli(n, ne, mp)[1]
    out = got.cpu().numpy()
    for b in (0, 5, G * n_groups - 1):
        o = evolve.taylor5(pauli.pauli_to_csr(pps[int(ks[b])]), psi[b], th[b])
        if prec == tq.TQ_C128:
            assert rel_l2(out[b], o) <= 1e-12
        else:
            assert fidelity(out[b], o) > 0.999999


def test_grouped_bad_op_and_alignment(ctx):
    import torch
    n, ne, mp = 4, 4, 1
    pool = tq.build_pool(ctx, n, ne, mp)
    G, D, rng, psi = _setup(n, ne, mp, 3, tq.TQ_C64, 5)
    gpsi = _interleave(torch.as_tensor(psi).to(torch.complex64).cuda(), 3, G, D)
    before = gpsi.clone()
    kg = torch.as_tensor(np.array([1, pool.M, 2], dtype=np.int32)).cuda()
    th = torch.full((3 * G,), 0.2, dtype=torch.float64, device="cuda")
    n2 = torch.ones(3 * G, dtype=torch.float64, device="cuda")
    tq.evolve_taylor5_batch_grouped(ctx, pool, gpsi, kg, th, n2)
    assert torch.equal(torch.view_as_real(gpsi[1]), torch.view_as_real(before[1]))   # untouched group
    assert torch.isnan(n2[G:2 * G]).all() and torch.isfinite(n2[:G]).all()
    # a state buffer off the 32-byte boundary is refused before any launch
    from paper_2606_29692_gb300._native import call
    flat = torch.zeros(3 * G * D + 4, dtype=torch.complex64, device="cuda")
    with pytest.raises(tq.TQError):
        call("tq_evolve_taylor5_batch_grouped", ctx.handle, pool.handle, 3, tq.TQ_C64,
             flat[1:].data_ptr(), kg.data_ptr(), th.data_ptr(), None, None)
    for bad in ((1, 0), (1, 3), (1, 8), (3, 1), (0, 2), (8, 1)):
        with pytest.raises(tq.TQError):
            ctx.set_grouped_schedule(tq.TQ_C64, *bad)
    with pytest.raises(tq.TQError):
        ctx.set_grouped_schedule(tq.TQ_C128, 4, 1)   # two complex128 states per row
