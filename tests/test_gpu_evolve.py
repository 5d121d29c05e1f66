"""GPU parity: the Taylor-5 update (pair path, CSR cluster path, batched)."""

import numpy as np
import pytest
import scipy.sparse as sp

import paper_2606_29692_gb300 as tq
import synth
from gpu_util import fidelity, rel_l2, to_state
from oracle import adapt as oadapt
from oracle import evolve, pauli

pytestmark = pytest.mark.gpu

THETAS = (0.05, -0.4, 1.1, 0.0)


@pytest.fixture(scope="module")
def ctx():
    return tq.Context(0)


_POOLS = {}


def oracle_pool(n, ne, mp):
    key = (n, ne, mp)
    if key not in _POOLS:
        exc, pps = pauli.pool_pauli(n, ne, mp)
        _POOLS[key] = (exc, pps, {})
    return _POOLS[key]


def oracle_A(n, ne, mp, k):
    exc, pps, cache = oracle_pool(n, ne, mp)
    if k not in cache:
        cache[k] = pauli.pauli_to_csr(pps[k])
    return cache[k]


def _ks(M):
    return sorted(set([0, 1, M // 2, M - 1] + list(range(0, M, max(1, M // 6)))))


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
@pytest.mark.parametrize("n,ne,mp", [(2, 2, 0), (2, 2, 1), (4, 4, 0), (4, 4, 1), (6, 8, 0), (7, 6, 1)])
def test_pair_path_matches_oracle(ctx, n, ne, mp, prec):
    N = 2 * n
    pool = tq.build_pool(ctx, n, ne, mp)
    psi0 = synth.random_state(N, 11 + n)
    for k in _ks(pool.M):
        A = oracle_A(n, ne, mp, k)
        for th in THETAS:
            st = to_state(ctx, psi0, N, prec)
            tq.evolve_taylor5(ctx, pool, k, th, st)
            out = st.numpy()
            ref = evolve.taylor5(A, psi0, th)
            if prec == tq.TQ_C128:
                assert rel_l2(out, ref) <= 1e-12, (k, th)
            else:
                assert rel_l2(out, ref) <= 2e-6, (k, th)
                assert fidelity(out, ref) > 0.999999


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
def test_pair_path_renormalises(ctx, prec):
    n, ne, mp = 6, 8, 1
    pool = tq.build_pool(ctx, n, ne, mp)
    psi0 = synth.random_state(12, 3) * 2.5
    for k, th in [(5, 0.3), (60, -1.2)]:
        st = to_state(ctx, psi0, 12, prec)
        tq.evolve_taylor5(ctx, pool, k, th, st, renormalize=True)
        ref = evolve.normalise(evolve.taylor5(oracle_A(n, ne, mp, k), psi0, th))
        tol = 1e-12 if prec == tq.TQ_C128 else 2e-6
        assert rel_l2(st.numpy(), ref) <= tol


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
@pytest.mark.parametrize("n,ne,mp", [(4, 4, 0), (6, 8, 1), (7, 6, 1), (8, 8, 0), (9, 8, 1)])
def test_csr_cluster_path_matches_oracle(ctx, n, ne, mp, prec):
    """Generator CSR compiled on the GPU, then the shared-memory-staged update.

    14 qubits runs on a cluster of 2 (complex64) or 4 (complex128) CTAs, 16
    qubits on 8 or 16, 18 qubits on the unfused fallback.
    """
    import torch
    N = 2 * n
    pool = tq.build_pool(ctx, n, ne, mp)
    psi0 = synth.random_state(N, 5 + n)
    for k in (0, pool.M // 3, pool.M - 1):
        rp, cl, vl, nnz = tq.pool_csr(ctx, pool, k, prec)
        A = oracle_A(n, ne, mp, k)
        for th, ren in ((0.07, False), (-0.6, True)):
            st = to_state(ctx, psi0, N, prec)
            tq.evolve_taylor5_csr(ctx, N, rp, cl, vl, th, st, renormalize=ren)
            ref = evolve.taylor5(A, psi0, th)
            if ren:
                ref = evolve.normalise(ref)
            tol = 1e-12 if prec == tq.TQ_C128 else 2e-6
            assert rel_l2(st.numpy(), ref) <= tol, (k, th, ren)
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
@pytest.mark.parametrize("nq", [6, 10, 14])
def test_csr_path_general_operator(ctx, nq, prec):
    """A non-pool operator: random real antisymmetric, several non-zeros per row."""
    import torch
    D = 1 << nq
    rng = np.random.default_rng(nq)
    nnz_row = 5
    rows = np.repeat(np.arange(D), nnz_row)
    cols = rng.integers(0, D, size=D * nnz_row)
    vals = rng.normal(0, 0.3, size=D * nnz_row)
    M = sp.coo_matrix((vals, (rows, cols)), shape=(D, D)).tocsr()
    A = (M - M.T).tocsr()
    A.sort_indices()
    A.eliminate_zeros()
    vt = torch.float64 if prec == tq.TQ_C128 else torch.float32
    rp = torch.as_tensor(A.indptr.astype(np.int32)).cuda()
    cl = torch.as_tensor(A.indices.astype(np.int32)).cuda()
    vl = torch.as_tensor(A.data.real).to(vt).cuda()
    Aref = sp.csr_matrix((vl.cpu().double().numpy(), A.indices, A.indptr), shape=(D, D))
    psi0 = synth.random_state(nq, 99)
    for th in (0.1, -0.35):
        st = to_state(ctx, psi0, nq, prec)
        tq.evolve_taylor5_csr(ctx, nq, rp.data_ptr(), cl.data_ptr(), vl.data_ptr(), th, st)
        ref = evolve.taylor5(Aref, psi0, th)
        tol = 1e-12 if prec == tq.TQ_C128 else 5e-6
        assert rel_l2(st.numpy(), ref) <= tol


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
def test_batched_matches_oracle(ctx, prec):
    import torch
    n, ne, mp = 7, 6, 1
    N = 14
    pool = tq.build_pool(ctx, n, ne, mp)
    S = 48
    rng = np.random.default_rng(21)
    psi = np.stack([synth.random_state(N, 1000 + b) for b in range(S)])
    k = rng.integers(0, pool.M, size=S).astype(np.int32)
    th = rng.normal(0, 0.3, size=S)
    dt = torch.complex128 if prec == tq.TQ_C128 else torch.complex64
    dpsi = torch.as_tensor(psi).to(dt).cuda()
    dk = torch.as_tensor(k).cuda()
    dth = torch.as_tensor(th).cuda()
    dn = torch.zeros(S, dtype=torch.float64, device="cuda")
    tq.evolve_taylor5_batch(ctx, pool, dpsi, dk, dth, dn, prec=prec)
    torch.cuda.synchronize()
    out = dpsi.cpu().numpy().astype(np.complex128)
    nrm = dn.cpu().numpy()
    for b in range(S):
        ref = evolve.taylor5(oracle_A(n, ne, mp, int(k[b])), psi[b], th[b])
        tol = 1e-12 if prec == tq.TQ_C128 else 2e-6
        assert rel_l2(out[b], ref) <= tol, b
        assert abs(nrm[b] - np.vdot(out[b], out[b]).real) <= 1e-12 * nrm[b] + (1e-6 if prec else 0)
        if prec == tq.TQ_C128:
            assert abs(nrm[b] - np.vdot(ref, ref).real) <= 1e-12


def test_batched_host_buffers_equal_device_path(ctx):
    import torch
    n, ne, mp = 6, 8, 0
    pool = tq.build_pool(ctx, n, ne, mp)
    S = 300
    rng = np.random.default_rng(5)
    psi = (rng.normal(size=(S, 4096)) + 1j * rng.normal(size=(S, 4096))).astype(np.complex64)
    k = rng.integers(0, pool.M, size=S).astype(np.int32)
    th = rng.normal(0, 0.1, size=S)
    dpsi = torch.as_tensor(psi.copy()).cuda()
    dn = torch.zeros(S, dtype=torch.float64, device="cuda")
    tq.evolve_taylor5_batch(ctx, pool, dpsi, torch.as_tensor(k).cuda(), torch.as_tensor(th).cuda(), dn)
    hpsi = torch.as_tensor(psi.copy()).pin_memory()
    hn = torch.zeros(S, dtype=torch.float64).pin_memory()
    tq.evolve_taylor5_batch_host(ctx, pool, hpsi, torch.as_tensor(k), torch.as_tensor(th), hn)
    torch.cuda.synchronize()
    assert np.array_equal(hpsi.numpy(), dpsi.cpu().numpy())
    assert np.array_equal(hn.numpy(), dn.cpu().numpy())


def test_full_size_batch_sampled(ctx):
    """The benchmark's launch: 8192 complex64 states of 14 qubits, sampled."""
    import torch
    n, ne, mp = 7, 6, 1
    N, S = 14, 8192
    pool = tq.build_pool(ctx, n, ne, mp)
    tq.autotune_pair(ctx, pool, tq.TQ_C64, n_states=2048)     # as the benchmark does
    prep_k, prep_th, k, th = synth.t5_batch(S, pool.M)
    hf = tq.hf_index(N, ne, mp)
    psi = torch.zeros((S, 1 << N), dtype=torch.complex64, device="cuda")
    psi[:, hf] = 1.0
    for j in range(prep_k.shape[1]):
        tq.evolve_taylor5_batch(ctx, pool, psi, torch.as_tensor(prep_k[:, j].copy()).cuda(),
                                torch.as_tensor(prep_th[:, j].copy()).cuda())
    dn = torch.zeros(S, dtype=torch.float64, device="cuda")
    tq.evolve_taylor5_batch(ctx, pool, psi, torch.as_tensor(k).cuda(), torch.as_tensor(th).cuda(), dn)
    torch.cuda.synchronize()
    sample = [0, 1, 777, 4095, 4096, 8190, 8191] + list(np.random.default_rng(0).integers(0, S, 9))
    for b in sample:
        ref = oadapt.hf_state(N, ne, mp)
        for j in range(prep_k.shape[1]):
            ref = evolve.taylor5(oracle_A(n, ne, mp, int(prep_k[b, j])), ref, prep_th[b, j])
        ref = evolve.taylor5(oracle_A(n, ne, mp, int(k[b])), ref, th[b])
        out = psi[b].cpu().numpy().astype(np.complex128)
        assert rel_l2(out, ref) <= 2e-6
        assert fidelity(out, ref) > 0.999999
        assert abs(dn[b].item() - np.vdot(ref, ref).real) <= 1e-6


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
def test_every_schedule_gives_identical_results(ctx, prec):
    import torch
    pool = tq.build_pool(ctx, 6, 8, 1)
    S = 40
    rng = np.random.default_rng(8)
    psi = np.stack([synth.random_state(12, 50 + b) for b in range(S)])
    k = torch.as_tensor(rng.integers(0, pool.M, size=S).astype(np.int32)).cuda()
    th = torch.as_tensor(rng.normal(0, 0.2, size=S)).cuda()
    dt = torch.complex128 if prec == tq.TQ_C128 else torch.complex64
    outs = []
    for upt in (1, 2, 4, 8):
        ctx.set_pair_schedule(prec, upt)
        d = torch.as_tensor(psi).to(dt).cuda()
        n = torch.zeros(S, dtype=torch.float64, device="cuda")
        tq.evolve_taylor5_batch(ctx, pool, d, k, th, n, prec=prec)
        torch.cuda.synchronize()
        outs.append((d.cpu().numpy(), n.cpu().numpy()))
    # complex64 norms: per-thread float32 partials of <= 32 squares, grouped
    # by the schedule, so schedules agree to float32 rounding of those
    # partials; the cross-thread sums are compensated and widened to float64
    tol = 1e-12 if prec == tq.TQ_C128 else 2e-6
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0])
        assert np.abs(o[1] - outs[0][1]).max() <= tol * outs[0][1].max()
    best, ms = tq.autotune_pair(ctx, pool, prec, n_states=64)
    assert best in (1, 2, 4, 8) and ms > 0 and ctx.pair_schedule(prec) == best
    with pytest.raises(tq.TQError):
        ctx.set_pair_schedule(prec, 3)


def test_invalid_op_index_poisons_norm(ctx):
    import torch
    pool = tq.build_pool(ctx, 4, 4, 0)
    psi = torch.zeros((3, 256), dtype=torch.complex64, device="cuda")
    psi[:, 5] = 1.0
    before = psi.clone()
    k = torch.as_tensor(np.array([0, pool.M, -1], dtype=np.int32)).cuda()
    th = torch.as_tensor(np.array([0.1, 0.1, 0.1])).cuda()
    n = torch.zeros(3, dtype=torch.float64, device="cuda")
    tq.evolve_taylor5_batch(ctx, pool, psi, k, th, n)
    torch.cuda.synchronize()
    assert np.isfinite(n[0].item()) and np.isnan(n[1].item()) and np.isnan(n[2].item())
    assert torch.equal(psi[1:], before[1:])


def test_empty_batch_is_a_noop(ctx):
    import torch
    pool = tq.build_pool(ctx, 4, 4, 0)
    for prec, dt in ((tq.TQ_C64, torch.complex64), (tq.TQ_C128, torch.complex128)):
        psi = torch.zeros((0, 256), dtype=dt, device="cuda")
        k = torch.zeros(0, dtype=torch.int32, device="cuda")
        th = torch.zeros(0, dtype=torch.float64, device="cuda")
        tq.evolve_taylor5_batch(ctx, pool, psi, k, th, None, prec=prec)
        tq.evolve_taylor5_batch_host(ctx, pool, psi.cpu(), k.cpu(), th.cpu(), None, prec=prec)


def test_evolve_rejects_bad_arguments(ctx):
    pool = tq.build_pool(ctx, 4, 4, 0)
    st = to_state(ctx, synth.random_state(8, 1), 8, tq.TQ_C128)
    with pytest.raises(tq.TQError):
        tq.evolve_taylor5(ctx, pool, pool.M, 0.1, st)
    with pytest.raises(tq.TQError):
        tq.evolve_taylor5(ctx, pool, -1, 0.1, st)
    with pytest.raises(tq.TQError):
        tq.evolve_taylor5(ctx, pool, 0, float("nan"), st)
    st10 = to_state(ctx, synth.random_state(10, 1), 10, tq.TQ_C128)
    with pytest.raises(tq.TQError):
        tq.evolve_taylor5(ctx, pool, 0, 0.1, st10)
