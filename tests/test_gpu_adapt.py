"""GPU parity: the ADAPT iteration (selection, line search, update)."""

import numpy as np
import pytest

import paper_2606_29692_gb300 as tq
import synth
from gpu_util import fidelity, rel_l2, to_state
from oracle import adapt as oadapt
from oracle import evolve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return tq.Context(0)


@pytest.mark.parametrize("mp", [0, 1])
def test_config0_one_step(ctx, mp):
    """8 qubits, JW/BK, complex128: one step from HF at theta = 0.05."""
    ints, ne = synth.config0()
    sysm = oadapt.build_system(ints, ne, mp)
    psi0 = oadapt.hf_state(8, ne, mp)
    ref, psi_ref = oadapt.adapt_step(sysm, psi0, 1e-3, theta=0.05)
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, 0.0, mp, tq.TQ_C128)
    pool = tq.build_pool(ctx, 4, ne, mp)
    st = tq.State(ctx, 8, tq.TQ_C128)
    tq.state_set_hf(st, ne, mp)
    r = tq.adapt_step(ctx, ham, pool, st, 1e-3, 0.05)
    assert abs(r["energy"] - ref.energy) <= 1e-10
    assert abs(r["max_grad"] - ref.max_grad) <= 1e-10
    assert r["selected"] == ref.selected and not r["converged"]
    assert r["theta"] == 0.05
    out = st.numpy()
    assert rel_l2(out, psi_ref) <= 1e-12
    ex = evolve.expm_dense(sysm.pool[ref.selected], 0.05) @ psi0
    assert fidelity(out, ex) > 0.999999


def _teacher_forced(ctx, mp, prec, n_iter):
    ints, ne = synth.config1()
    sysm = oadapt.build_system(ints, ne, mp)
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, 0.0, mp, prec)
    pool = tq.build_pool(ctx, 6, ne, mp)
    psi = oadapt.hf_state(12, ne, mp)
    precision = oadapt.FP64 if prec == tq.TQ_C128 else oadapt.C64
    tau = 1e-9 if prec == tq.TQ_C128 else 1e-5
    for it in range(n_iter):
        ref, nxt = oadapt.adapt_step(sysm, psi, 1e-3, None, precision)
        st = to_state(ctx, psi, 12, prec)
        held = st.numpy()
        r = tq.adapt_step(ctx, ham, pool, st, 1e-3)
        tolE = 1e-10 if prec == tq.TQ_C128 else 1e-6
        assert abs(r["energy"] - ref.energy) <= tolE, it
        assert abs(r["max_grad"] - ref.max_grad) <= tolE, it
        # selection: identical, or a tie within tau of the maximum
        assert abs(abs(ref.gradients[r["selected"]]) - ref.max_grad) <= tau + tolE, it
        if r["selected"] == ref.selected:
            assert abs(r["theta"] - ref.theta) <= 1e-9 * max(1, abs(ref.theta)) + (1e-5 if prec else 0), it
            if prec == tq.TQ_C128:
                assert rel_l2(st.numpy(), nxt) <= 1e-12, it
            else:
                _, nxt_held = oadapt.adapt_step(sysm, held, 1e-3, r["theta"], precision,
                                                force_k=r["selected"])
                assert fidelity(st.numpy(), nxt_held) > 0.999999, it
        psi = nxt
        if ref.converged:
            break


@pytest.mark.parametrize("mp", [0, 1])
def test_config1_teacher_forced_fp64(ctx, mp):
    _teacher_forced(ctx, mp, tq.TQ_C128, 20)


@pytest.mark.parametrize("mp", [0, 1])
def test_config1_teacher_forced_c64(ctx, mp):
    _teacher_forced(ctx, mp, tq.TQ_C64, 8)


@pytest.mark.parametrize("sched", [32, tq.TQ_SPMV_XELL])
@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
def test_config1_free_running(ctx, prec, sched):
    """20 iterations on the GPU alone vs the oracle's own trajectory, with
    the H pass on the CSR and on the XOR-ELL layout."""
    ctx.set_spmv_schedule(sched)
    try:
        _free_running(ctx, prec)
    finally:
        ctx.set_spmv_schedule(tq.TQ_SPMV_XELL)


def _free_running(ctx, prec):
    ints, ne = synth.config1()
    mp = 1
    sysm = oadapt.build_system(ints, ne, mp)
    res, psi_ref = oadapt.trajectory(sysm, oadapt.hf_state(12, ne, mp), 1e-3, n_iter=20)
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, 0.0, mp, prec)
    pool = tq.build_pool(ctx, 6, ne, mp)
    st = tq.State(ctx, 12, prec)
    tq.state_set_hf(st, ne, mp)
    for it, ref in enumerate(res):
        r = tq.adapt_step(ctx, ham, pool, st, 1e-3)
        tolE = 1e-10 if prec == tq.TQ_C128 else 1e-6
        assert r["selected"] == ref.selected, it
        assert abs(r["energy"] - ref.energy) <= tolE, it
    assert fidelity(st.numpy(), psi_ref) > 0.999999


def test_config2_c64_vs_fp64(ctx):
    """14 qubits, BK, strongly correlated: full-pool screen, complex64 vs float64."""
    ints, ne = synth.config2()
    mp = 1
    out = {}
    for prec in (tq.TQ_C128, tq.TQ_C64):
        ham = tq.build_hamiltonian(ctx, ints.h, ints.g, 0.0, mp, prec)
        pool = tq.build_pool(ctx, 7, ne, mp)
        st = tq.State(ctx, 14, prec)
        tq.state_set_hf(st, ne, mp)
        es = []
        for _ in range(4):
            es.append(tq.adapt_step(ctx, ham, pool, st, 1e-3, 0.1))
        out[prec] = (es, st.numpy())
    for a, b in zip(out[tq.TQ_C128][0], out[tq.TQ_C64][0]):
        assert a["selected"] == b["selected"]
        assert abs(a["energy"] - b["energy"]) <= 1e-6
    assert fidelity(out[tq.TQ_C128][1], out[tq.TQ_C64][1]) > 0.999999
    # and the float64 path against the oracle
    sysm = oadapt.build_system(ints, ne, mp)
    res, psi = oadapt.trajectory(sysm, oadapt.hf_state(14, ne, mp), 1e-3, thetas=[0.1] * 4)
    for a, ref in zip(out[tq.TQ_C128][0], res):
        assert a["selected"] == ref.selected and abs(a["energy"] - ref.energy) <= 1e-10
    assert rel_l2(out[tq.TQ_C128][1], psi) <= 1e-12


def test_converged_step_leaves_state(ctx):
    ints, ne = synth.config0()
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, 0.0, 0, tq.TQ_C128)
    pool = tq.build_pool(ctx, 4, ne, 0)
    st = tq.State(ctx, 8, tq.TQ_C128)
    tq.state_set_hf(st, ne, 0)
    before = st.numpy()
    r = tq.adapt_step(ctx, ham, pool, st, 1e3)     # eps above every gradient
    assert r["converged"]
    assert np.array_equal(st.numpy(), before)


@pytest.mark.parametrize("mp", [0, 1])
def test_line_search_16q_c64_follows_c128(ctx, mp):
    """Ten line-search steps at 16 qubits (rows of up to ~280 non-zeros):
    complex64 takes the same operators and the same angles as complex128.
    When psi lies in a generator's support the energy curve has two tied
    minima half a period apart; the line-search products must resolve that
    tie (to 1e-10) in complex64 too, else the update takes the far minimum,
    where Taylor-5 is no longer accurate, and the energy rises."""
    n = 8
    ne = synth.electrons_for(n)
    ints = synth.integrals(n, 4242)
    runs = {}
    for prec in (tq.TQ_C128, tq.TQ_C64):
        ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, mp, prec)
        pool = tq.build_pool(ctx, n, ne, mp)
        st = tq.State(ctx, 2 * n, prec)
        tq.state_set_hf(st, ne, mp)
        runs[prec] = [tq.adapt_step(ctx, ham, pool, st, 0.0, float("nan")) for _ in range(10)]
    a, b = runs[tq.TQ_C128], runs[tq.TQ_C64]
    for i, (ra, rb) in enumerate(zip(a, b)):
        assert ra["selected"] == rb["selected"], i
        assert abs(ra["theta"] - rb["theta"]) <= 1e-4, (i, ra["theta"], rb["theta"])
        assert abs(ra["energy"] - rb["energy"]) <= 1e-5, i
        assert abs(rb["theta"]) <= np.pi / 2 + 1e-9, i
    e = [r["energy"] for r in b]
    assert all(e[i + 1] <= e[i] + 1e-6 for i in range(len(e) - 1)), e


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
@pytest.mark.parametrize("given", [False, True])
def test_adapt_run_equals_repeated_steps(ctx, prec, given):
    """The graph-replayed run gives, bit for bit, what n_iter calls of
    tq_adapt_step give (results and final state), with the line search or
    with given angles; the oracle's trajectory checks the first steps."""
    ints, ne = synth.config1()
    mp = 1
    n = 12
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, mp, prec)
    pool = tq.build_pool(ctx, ints.n_spatial, ne, mp)
    thetas = np.random.default_rng(5).normal(0.0, 0.1, size=n) if given else None
    a = tq.State(ctx, 12, prec)
    tq.state_set_hf(a, ne, mp)
    ref = [tq.adapt_step(ctx, ham, pool, a, 1e-3, float(thetas[i]) if given else float("nan")) for i in range(n)]
    b = tq.State(ctx, 12, prec)
    tq.state_set_hf(b, ne, mp)
    got, done = tq.adapt_run(ctx, ham, pool, b, 1e-3, n, thetas)
    assert done == n
    for r, g in zip(ref, got):
        assert r == g
    assert np.array_equal(a.numpy(), b.numpy())
    # a converged run stops changing the state and reports where it stopped
    c_ = tq.State(ctx, 12, prec)
    tq.state_set_hf(c_, ne, mp)
    got2, done2 = tq.adapt_run(ctx, ham, pool, c_, 10.0, 3, None)
    assert done2 == 1 and got2[0]["converged"] and got2[2]["converged"]
    assert abs(c_.numpy()[tq.hf_index(12, ne, mp)]) == 1.0
