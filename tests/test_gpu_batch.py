"""GPU parity: independent ADAPT trajectories advanced together (graph-replayed)."""

import numpy as np
import pytest

import paper_2606_29692_gb300 as tq
import synth
from gpu_util import fidelity, rel_l2
from oracle import adapt as oadapt

pytestmark = pytest.mark.gpu

# (n_spatial, n_electrons, mapping, seed, length)
SMALL = [(4, 4, 0, 11, 3), (5, 4, 1, 12, 5), (6, 8, 0, 13, 2), (4, 2, 1, 14, 1),
         (3, 2, 0, 15, 4), (6, 6, 1, 16, 6), (2, 2, 1, 17, 3)]


@pytest.fixture(scope="module")
def ctx():
    return tq.Context(0)


def _thetas(seed, length):
    return np.random.default_rng(seed + 7).normal(0.0, 0.1, size=length)


def _build(ctx, spec, prec, eps=1e-3):
    hams, pools, ne, mp, th = [], [], [], [], []
    for n, e, m, seed, L in spec:
        ints = synth.integrals(n, seed)
        hams.append(tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, m, prec))
        pools.append(tq.build_pool(ctx, n, e, m))
        ne.append(e)
        mp.append(m)
        th.append(_thetas(seed, L))
    return tq.Batch(ctx, hams, pools, ne, mp, th, eps), th


def _oracle(spec, th, eps=1e-3, precision=oadapt.FP64):
    out = []
    for (n, e, m, seed, L), t in zip(spec, th):
        sysm = oadapt.build_system(synth.integrals(n, seed), e, m)
        res, psi = oadapt.trajectory(sysm, oadapt.hf_state(2 * n, e, m), eps, thetas=t,
                                     precision=precision)
        out.append((res, psi))
    return out


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
def test_small_batch_matches_oracle(ctx, prec):
    b, th = _build(ctx, SMALL, prec)
    b.run(use_graph=True)
    got = b.results()
    ref = _oracle(SMALL, th, precision=oadapt.FP64 if prec == tq.TQ_C128 else oadapt.C64)
    tolE = 1e-10 if prec == tq.TQ_C128 else 1e-6
    for t, ((res, psi), g) in enumerate(zip(ref, got)):
        assert g["n_iter"] == len(res), t
        assert g["converged"] == res[-1].converged, t
        for i, r in enumerate(res):
            assert g["selected"][i] == r.selected, (t, i)
            assert abs(g["energy"][i] - r.energy) <= tolE, (t, i)
            assert abs(g["max_grad"][i] - r.max_grad) <= tolE, (t, i)
            assert g["theta"][i] == (0.0 if r.converged else r.theta), (t, i)
        out = b.state(t)
        if prec == tq.TQ_C128:
            assert rel_l2(out, psi) <= 1e-12, t
        else:
            assert fidelity(out, psi) > 0.999999, t


def test_graph_direct_and_schedules_agree(ctx):
    b, th = _build(ctx, SMALL, tq.TQ_C128)
    b.run(use_graph=False)
    base = b.results()
    states = [b.state(t) for t in range(len(SMALL))]
    for lpr in (tq.TQ_SPMV_XELL, 4, 8, 16, 32):
        b.set_schedule(lpr)
        b.run(use_graph=True)
        r = b.results()
        for t in range(len(SMALL)):
            assert np.array_equal(r[t]["selected"], base[t]["selected"])
            assert np.abs(r[t]["energy"] - base[t]["energy"]).max(initial=0) <= 1e-12
            assert rel_l2(b.state(t), states[t]) <= 1e-13
    best, ms = b.autotune()
    assert best in (tq.TQ_SPMV_XELL, 4, 8, 16, 32) and ms > 0
    b.run()
    assert [x["n_iter"] for x in b.results()] == [x["n_iter"] for x in base]


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
def test_repeated_runs_are_bit_identical(ctx, prec):
    """Every sum of the batch is taken in a fixed order (energy items, the
    gradient chunks of each op, the final norm), and the device-side item
    numbering and tickets start afresh each run: graph replays and a direct
    run give the same bits."""
    b, _ = _build(ctx, SMALL, prec)
    runs = []
    for use_graph in (True, True, False):
        b.run(use_graph=use_graph)
        runs.append((b.results(), [b.state(t) for t in range(len(SMALL))]))
    (r0, s0) = runs[0]
    for r, st in runs[1:]:
        for t in range(len(SMALL)):
            assert r[t]["n_iter"] == r0[t]["n_iter"]
            for key in ("energy", "max_grad", "selected", "theta"):
                assert np.array_equal(r[t][key], r0[t][key]), (t, key)
            assert np.array_equal(st[t], s0[t]), t


def test_immediate_convergence_keeps_hf(ctx):
    spec = [(4, 4, 0, 11, 3), (3, 2, 1, 15, 2)]
    b, th = _build(ctx, spec, tq.TQ_C128, eps=1e3)
    b.run()
    for t, r in enumerate(b.results()):
        assert r["n_iter"] == 1 and r["converged"] and r["theta"][0] == 0.0
        n, e, m = spec[t][:3]
        assert np.array_equal(b.state(t), oadapt.hf_state(2 * n, e, m))


def test_full_size_batch_sampled(ctx):
    """256 trajectories of 10-16 qubits (the batched workload), sampled."""
    import torch
    trajs = synth.trajectories()
    hams, pools = [], []
    for tr in trajs:
        ints = synth.integrals(tr.n_spatial, tr.seed)
        hams.append(tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, tr.mapping, tq.TQ_C64))
        pools.append(tq.build_pool(ctx, tr.n_spatial, tr.n_electrons, tr.mapping))
    b = tq.Batch(ctx, hams, pools, [t.n_electrons for t in trajs], [t.mapping for t in trajs],
                 [t.thetas for t in trajs], 1e-3)
    b.autotune()
    b.run(use_graph=True)
    got = b.results()
    torch.cuda.synchronize()
    picks = {}
    for tr in trajs:                       # one short trajectory per size up to 14 qubits
        q = 2 * tr.n_spatial
        if q <= 14 and len(tr.thetas) <= 6 and q not in picks:
            picks[q] = tr
    assert len(picks) == 3
    for q, tr in picks.items():
        sysm = oadapt.build_system(synth.integrals(tr.n_spatial, tr.seed), tr.n_electrons, tr.mapping)
        res, psi = oadapt.trajectory(sysm, oadapt.hf_state(q, tr.n_electrons, tr.mapping), 1e-3,
                                     thetas=tr.thetas, precision=oadapt.C64)
        g = got[tr.index]
        assert g["n_iter"] == len(res)
        for i, r in enumerate(res):
            assert g["selected"][i] == r.selected
            assert abs(g["energy"][i] - r.energy) <= 1e-6
        assert fidelity(b.state(tr.index), psi) > 0.999999
    assert all(np.isfinite(x["energy"]).all() for x in got)


def test_zero_length_and_single_trajectory(ctx):
    spec = [(3, 2, 0, 15, 0), (2, 2, 1, 17, 1)]
    b, th = _build(ctx, spec, tq.TQ_C128)
    b.run()
    r = b.results()
    assert r[0]["n_iter"] == 0 and r[0]["energy"].size == 0
    assert np.array_equal(b.state(0), oadapt.hf_state(6, 2, 0))
    ref = _oracle(spec[1:], th[1:])[0]
    assert r[1]["n_iter"] == len(ref[0]) == 1
    assert abs(r[1]["energy"][0] - ref[0][0].energy) <= 1e-10
    assert rel_l2(b.state(1), ref[1]) <= 1e-12
