"""GPU: the continuous-batching request loop.

Every request must give the same result alone (its own tick) and in a mix
(batched with others), and both must match the oracle replaying the same
request script session by session.
"""

import time

import numpy as np
import pytest

import paper_2606_29692_gb300 as tq
import synth
from oracle import adapt as oadapt
from oracle import evolve

pytestmark = pytest.mark.gpu

HAMS = [(4, 4, 0, 31), (5, 4, 1, 32)]            # (n_spatial, n_electrons, mapping, seed)
SESSIONS = [0, 1, 0, 1, 1, 0]                     # Hamiltonian of each session


def _script(n=48, seed=9):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        kind = int(rng.choice(3, p=[0.5, 0.3, 0.2]))
        sess = int(rng.integers(0, len(SESSIONS)))
        out.append((kind, sess, int(rng.integers(0, 1 << 20)), float(rng.normal(0, 0.1)), i))
    return out


def _server(prec):
    ctx = tq.Context(0)
    srv = tq.Server(ctx, prec, hbm_budget=256 << 20, max_batch=64)
    pools = []
    for n, ne, mp, seed in HAMS:
        ints = synth.integrals(n, seed)
        ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, mp, prec)
        pool = tq.build_pool(ctx, n, ne, mp)
        srv.add_hamiltonian(ham, pool)
        pools.append(pool.M)
    for h in SESSIONS:
        n, ne, mp, _ = HAMS[h]
        srv.add_session(h, ne, mp)
    srv.start()
    return ctx, srv, pools


def _submit(srv, pools, req):
    kind, sess, op, th, tag = req
    srv.submit(kind, sess, op % pools[SESSIONS[sess]], th, tag)


def _collect(srv, n, timeout_s=30.0):
    got = {}
    t0 = time.time()
    while len(got) < n and time.time() - t0 < timeout_s:
        for c in srv.poll(2000):
            got[c["tag"]] = c
    assert len(got) == n, f"only {len(got)} of {n} completions"
    return got


def _run(prec, alone):
    ctx, srv, pools = _server(prec)
    script = _script()
    got = {}
    if alone:
        for req in script:
            _submit(srv, pools, req)
            got.update(_collect(srv, 1))
    else:
        for req in script:
            _submit(srv, pools, req)
        got = _collect(srv, len(script))
    srv.stop()
    states = [srv.state(s) for s in range(len(SESSIONS))]
    stats = srv.stats()
    return script, got, states, stats, pools


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
def test_alone_and_mixed_identical(prec):
    script, a, sa, st_a, _ = _run(prec, alone=True)
    _, b, sb, st_b, _ = _run(prec, alone=False)
    assert st_a["ticks"] == len(script)             # one request per tick
    assert st_b["ticks"] < len(script)               # the mix really batched
    for kind, sess, op, th, tag in script:
        x, y = a[tag], b[tag]
        assert x["status"] == 0 and y["status"] == 0
        for f in ("energy", "max_grad", "norm2", "argmax"):
            assert x[f] == y[f], (tag, f, x[f], y[f])
    for u, v in zip(sa, sb):
        assert np.array_equal(u, v)


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
def test_mixed_run_matches_oracle(prec):
    script, got, states, _, pools = _run(prec, alone=False)
    systems = []
    for n, ne, mp, seed in HAMS:
        systems.append(oadapt.build_system(synth.integrals(n, seed), ne, mp))
    psi = []
    for h in SESSIONS:
        n, ne, mp, _ = HAMS[h]
        psi.append(oadapt.hf_state(2 * n, ne, mp))
    tol = 1e-10 if prec == tq.TQ_C128 else 1e-6
    precision = oadapt.FP64 if prec == tq.TQ_C128 else oadapt.C64
    for kind, sess, op, th, tag in script:
        sysm = systems[SESSIONS[sess]]
        c = got[tag]
        if kind == tq.TQ_REQ_EVOLVE:
            k = op % len(sysm.pool)
            out = evolve.taylor5(sysm.pool[k], psi[sess], th)
            assert abs(c["norm2"] - np.vdot(out, out).real) <= (1e-12 if prec == tq.TQ_C128 else 1e-6)
            psi[sess] = evolve.normalise(out)
        else:
            assert abs(c["energy"] - oadapt.energy(sysm.H, psi[sess])[0]) <= tol
            if kind == tq.TQ_REQ_GRADIENTS:
                g = oadapt.gradients(sysm.H, sysm.pool, psi[sess])
                k, gmax = oadapt.select(g, precision)
                assert abs(c["max_grad"] - gmax) <= tol
                assert abs(abs(g[c["argmax"]]) - gmax) <= (1e-9 if prec == tq.TQ_C128 else 1e-5) + tol
    for s, u in enumerate(states):
        ref = psi[s]
        err = np.linalg.norm(u - ref) / np.linalg.norm(ref)
        assert err <= (1e-12 if prec == tq.TQ_C128 else 2e-6)


def test_admission_and_errors():
    ctx = tq.Context(0)
    srv = tq.Server(ctx, tq.TQ_C64, hbm_budget=64 << 20, max_batch=8)
    ints = synth.integrals(4, 1)
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, 0.0, 0, tq.TQ_C64)
    pool = tq.build_pool(ctx, 4, 4, 0)
    h = srv.add_hamiltonian(ham, pool)
    s0 = srv.add_session(h, 4, 0)
    # a Hamiltonian of another precision is refused
    ham128 = tq.build_hamiltonian(ctx, ints.h, ints.g, 0.0, 0, tq.TQ_C128)
    with pytest.raises(tq.TQError):
        srv.add_hamiltonian(ham128, pool)
    srv.start()
    assert srv.poll(1000) == []                          # nothing pending: timeout
    with pytest.raises(tq.TQError):
        srv.submit(tq.TQ_REQ_EVOLVE, s0, pool.M, 0.1)     # op out of range
    with pytest.raises(tq.TQError):
        srv.submit(tq.TQ_REQ_ENERGY, 99)                  # unknown session
    srv.submit(tq.TQ_REQ_ENERGY, s0, tag=5)
    c = _collect(srv, 1)
    assert c[5]["status"] == 0 and np.isfinite(c[5]["energy"])
    srv.stop()


def test_session_budget_is_enforced():
    ctx = tq.Context(0)
    srv = tq.Server(ctx, tq.TQ_C64, hbm_budget=64 << 20, max_batch=8)
    ints = synth.integrals(8, 2)
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, 0.0, 1, tq.TQ_C64)
    pool = tq.build_pool(ctx, 8, 8, 1)
    h = srv.add_hamiltonian(ham, pool)
    n = 0
    with pytest.raises(tq.TQError) as e:
        for _ in range(100):                              # 512 KiB each, 32 MiB cap
            srv.add_session(h, 8, 1)
            n += 1
    assert e.value.code == -5 and n == 64
