"""GPU parity: the support-only batched Taylor-5 update (Sec. III-C).

Only the rows on each generator's support are read and written; the tests
check the amplitudes against the oracle's five-product chain, the equality
with the full-state kernel, that rows off the support keep their bits, and
the carried squared norm."""

import numpy as np
import pytest

import paper_2606_29692_gb300 as tq
import synth
from gpu_util import fidelity, rel_l2
from oracle import adapt as oadapt
from oracle import evolve, pauli

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return tq.Context(0)


_A = {}


def oracle_A(n, ne, mp, k):
    key = (n, ne, mp)
    if key not in _A:
        _A[key] = (pauli.pool_pauli(n, ne, mp)[1], {})
    pps, cache = _A[key]
    if k not in cache:
        cache[k] = pauli.pauli_to_csr(pps[k])
    return cache[k]


def _inputs(n_q, S, M, seed, prec):
    import torch
    rng = np.random.default_rng(seed)
    psi = np.stack([synth.random_state(n_q, seed * 1000 + b) for b in range(S)])
    k = (np.arange(S) % M).astype(np.int32)          # every generator at least once when S >= M
    rng.shuffle(k)
    th = rng.normal(0, 0.3, size=S)
    th[0] = 0.0
    dt = torch.complex128 if prec == tq.TQ_C128 else torch.complex64
    return psi, k, th, dt


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
@pytest.mark.parametrize("n,ne,mp", [(2, 2, 0), (2, 2, 1), (4, 4, 0), (4, 4, 1), (6, 8, 0), (7, 6, 1)])
def test_support_update_matches_oracle(ctx, n, ne, mp, prec):
    import torch
    N = 2 * n
    pool = tq.build_pool(ctx, n, ne, mp)
    S = max(pool.M, 24) if N <= 12 else 64
    psi, k, th, dt = _inputs(N, S, pool.M, 3 + n + mp, prec)
    dpsi = torch.as_tensor(psi).to(dt).cuda()
    n_in = (dpsi.abs().double() ** 2).sum(dim=1)
    dn = n_in.clone()
    tq.evolve_taylor5_batch_support(ctx, pool, dpsi, torch.as_tensor(k).cuda(), torch.as_tensor(th).cuda(), dn,
                                    prec=prec)
    torch.cuda.synchronize()
    out = dpsi.cpu().numpy().astype(np.complex128)
    nrm = dn.cpu().numpy()
    for b in range(S):
        ref = evolve.taylor5(oracle_A(n, ne, mp, int(k[b])), psi[b], th[b])
        tol = 1e-12 if prec == tq.TQ_C128 else 2e-6
        assert rel_l2(out[b], ref) <= tol, b
        if prec == tq.TQ_C128:
            assert abs(nrm[b] - np.vdot(ref, ref).real) <= 1e-12, b
        else:
            assert abs(nrm[b] - np.vdot(out[b], out[b]).real) <= 1e-6, b


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
@pytest.mark.parametrize("n,ne,mp", [(6, 8, 0), (6, 8, 1), (7, 6, 1)])
def test_support_update_equals_full_state_kernel(ctx, n, ne, mp, prec):
    """Same amplitudes as the full-state pair kernel, rows off the support
    bit-for-bit untouched, every schedule identical."""
    import torch
    N = 2 * n
    pool = tq.build_pool(ctx, n, ne, mp)
    S = 96
    psi, k, th, dt = _inputs(N, S, pool.M, 40 + n + mp, prec)
    dk = torch.as_tensor(k).cuda()
    dth = torch.as_tensor(th).cuda()
    full = torch.as_tensor(psi).to(dt).cuda()
    n_full = torch.zeros(S, dtype=torch.float64, device="cuda")
    tq.evolve_taylor5_batch(ctx, pool, full, dk, dth, n_full, prec=prec)
    before = torch.as_tensor(psi).to(dt).cuda()
    n_in = (before.abs().double() ** 2).sum(dim=1)
    outs = []
    for ppt in (1, 2, 4, 8, -1, -2, -4, -8):
        ctx.set_support_schedule(prec, ppt)
        d = before.clone()
        dn = n_in.clone()
        tq.evolve_taylor5_batch_support(ctx, pool, d, dk, dth, dn, prec=prec)
        torch.cuda.synchronize()
        outs.append((d, dn))
    ctx.set_support_schedule(prec, 4 if prec == tq.TQ_C128 else -1)
    fv = torch.view_as_real(full)
    bv = torch.view_as_real(before)
    for d, dn in outs:
        assert torch.equal(torch.view_as_real(d), fv)       # values (a -0.0 equals +0.0)
        assert torch.equal(torch.view_as_real(d), torch.view_as_real(outs[0][0]))
        tol = 1e-12 if prec == tq.TQ_C128 else 2e-6
        assert (dn - n_full).abs().max().item() <= tol * n_full.max().item()
    # rows off the support: identical bits
    d = outs[-1][0]
    ib = bv.view(torch.int64) if prec == tq.TQ_C128 else bv.view(torch.int32)
    io = torch.view_as_real(d).view(torch.int64) if prec == tq.TQ_C128 else torch.view_as_real(d).view(torch.int32)
    for b in range(0, S, 7):
        A = oracle_A(n, ne, mp, int(k[b]))
        on = np.zeros(1 << N, dtype=bool)
        on[np.unique(A.tocoo().row)] = True
        off = torch.as_tensor(~on).cuda()
        assert torch.equal(io[b][off], ib[b][off])


def test_full_size_batch_sampled(ctx):
    """8192 complex64 states of 14 qubits (the batched benchmark's launch),
    norms carried over two updates, sampled against the oracle."""
    import torch
    n, ne, mp = 7, 6, 1
    N, S = 14, 8192
    pool = tq.build_pool(ctx, n, ne, mp)
    prep_k, prep_th, k, th = synth.t5_batch(S, pool.M)
    hf = tq.hf_index(N, ne, mp)
    psi = torch.zeros((S, 1 << N), dtype=torch.complex64, device="cuda")
    psi[:, hf] = 1.0
    dn = torch.ones(S, dtype=torch.float64, device="cuda")
    for j in range(prep_k.shape[1]):
        tq.evolve_taylor5_batch_support(ctx, pool, psi, torch.as_tensor(prep_k[:, j].copy()).cuda(),
                                        torch.as_tensor(prep_th[:, j].copy()).cuda(), dn)
    tq.evolve_taylor5_batch_support(ctx, pool, psi, torch.as_tensor(k).cuda(), torch.as_tensor(th).cuda(), dn)
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
def test_single_large_state_splits_tiles(ctx, prec):
    """One 18-qubit state: the state is split over many tiles."""
    import torch
    n, ne, mp = 9, 8, 1
    N = 18
    pool = tq.build_pool(ctx, n, ne, mp)
    for kk in (0, pool.M // 3, pool.M - 1):
        psi = synth.random_state(N, 77 + kk)
        dt = torch.complex128 if prec == tq.TQ_C128 else torch.complex64
        d = torch.as_tensor(psi[None, :]).to(dt).cuda()
        dn = torch.ones(1, dtype=torch.float64, device="cuda")
        tq.evolve_taylor5_batch_support(ctx, pool, d, torch.as_tensor(np.array([kk], np.int32)).cuda(),
                                        torch.as_tensor(np.array([0.37])).cuda(), dn, prec=prec)
        torch.cuda.synchronize()
        ref = evolve.taylor5(oracle_A(n, ne, mp, kk), psi, 0.37)
        out = d[0].cpu().numpy().astype(np.complex128)
        assert rel_l2(out, ref) <= (1e-12 if prec == tq.TQ_C128 else 2e-6)
        assert abs(dn[0].item() - np.vdot(ref, ref).real) <= (1e-12 if prec == tq.TQ_C128 else 1e-6)


def test_invalid_index_empty_batch_and_sector_pool(ctx):
    import torch
    pool = tq.build_pool(ctx, 4, 4, 0)
    psi = torch.zeros((3, 256), dtype=torch.complex64, device="cuda")
    psi[:, 5] = 1.0
    before = psi.clone()
    k = torch.as_tensor(np.array([0, pool.M, -1], dtype=np.int32)).cuda()
    th = torch.as_tensor(np.array([0.1, 0.1, 0.1])).cuda()
    n = torch.ones(3, dtype=torch.float64, device="cuda")
    tq.evolve_taylor5_batch_support(ctx, pool, psi, k, th, n)
    torch.cuda.synchronize()
    assert np.isfinite(n[0].item()) and np.isnan(n[1].item()) and np.isnan(n[2].item())
    assert torch.equal(psi[1:], before[1:])
    empty = torch.zeros((0, 256), dtype=torch.complex64, device="cuda")
    tq.evolve_taylor5_batch_support(ctx, pool, empty, k[:0], th[:0], None)
    spool = tq.build_pool_sector(ctx, 4, 4, 0, 2, 2)
    with pytest.raises(tq.TQError):
        tq.evolve_taylor5_batch_support(ctx, spool, psi, k, th, n)
    with pytest.raises(tq.TQError):
        ctx.set_support_schedule(tq.TQ_C64, 3)


def test_autotuner_picks_a_valid_schedule(ctx):
    pool = tq.build_pool(ctx, 6, 8, 1)
    for prec in (tq.TQ_C64, tq.TQ_C128):
        best, ms = tq.autotune_support(ctx, pool, prec, n_states=64)
        assert best in (1, 2, 4, 8, -1, -2, -4, -8) and ms > 0
    ctx.set_support_schedule(tq.TQ_C128, 4)
    ctx.set_support_schedule(tq.TQ_C64, -1)


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
def test_states_in_host_memory(ctx, prec):
    """The same update on page-locked host states, read and written in
    place by the kernel: bit-identical to the device-memory path."""
    import torch
    n, ne, mp = 7, 6, 1
    pool = tq.build_pool(ctx, n, ne, mp)
    S = 40
    psi, k, th, dt = _inputs(14, S, pool.M, 91, prec)
    dev = torch.as_tensor(psi).to(dt).cuda()
    n_in = (dev.abs().double() ** 2).sum(dim=1)
    dn = n_in.clone()
    tq.evolve_taylor5_batch_support(ctx, pool, dev, torch.as_tensor(k).cuda(), torch.as_tensor(th).cuda(), dn,
                                    prec=prec)
    host = torch.as_tensor(psi).to(dt).pin_memory()
    hn = n_in.cpu().clone()
    tq.evolve_taylor5_batch_support_host(ctx, pool, host, k, th, hn.numpy(), prec=prec)
    torch.cuda.synchronize()
    assert torch.equal(torch.view_as_real(host), torch.view_as_real(dev.cpu()))
    assert torch.equal(hn, dn.cpu())
    # memory the device cannot reach is refused before any launch
    with pytest.raises(tq.TQError):
        tq.evolve_taylor5_batch_support_host(ctx, pool, torch.as_tensor(psi).to(dt).numpy(), k, th, None,
                                             prec=prec)


def test_l2_fetch_granularity_round_trip(ctx):
    default = ctx.l2_fetch()
    assert default in (32, 64, 128)
    for b in (32, 64, 128):
        ctx.set_l2_fetch(b)
        assert ctx.l2_fetch() == b
    ctx.set_l2_fetch(0)
    assert ctx.l2_fetch() == default
    with pytest.raises(tq.TQError):
        ctx.set_l2_fetch(48)


def test_fp64_fma_rate(ctx):
    """The float64 roofline of the complex128 updates: a positive, finite
    rate within the range any float64 pipe of one GPU can have (10^9 to
    10^14 FMA lane operations per second), repeatable within a factor of 2,
    and arguments out of range rejected."""
    r1 = tq.fp64_fma_rate(ctx, 1024)
    r2 = tq.fp64_fma_rate(ctx, 4096)
    for r in (r1, r2):
        assert np.isfinite(r) and 1e9 < r < 1e14
    assert 0.5 < r1 / r2 < 2.0
    for bad in (0, -1, (1 << 20) + 1):
        with pytest.raises(tq.TQError):
            tq.fp64_fma_rate(ctx, bad)


@pytest.mark.parametrize("prec", [tq.TQ_C64, tq.TQ_C128])
def test_occupancy_knob_keeps_every_bit(ctx, prec):
    """Resident CTAs per SM (tq_ctx_set_support_occupancy) change only the
    persistent grid: amplitudes and carried norms are bit-identical for every
    setting, and bad settings are refused."""
    import torch
    n, ne, mp = 7, 6, 1
    pool = tq.build_pool(ctx, n, ne, mp)
    S = 600                                      # more states than one wave of CTAs at 2 per SM
    psi, k, th, dt = _inputs(14, S, pool.M, 71, prec)
    outs = []
    for occ in (0, 1, 2, 3):
        ctx.set_support_occupancy(prec, occ)
        d = torch.as_tensor(psi).to(dt).cuda()
        dn = torch.ones(S, dtype=torch.float64, device="cuda")
        tq.evolve_taylor5_batch_support(ctx, pool, d, torch.as_tensor(k).cuda(), torch.as_tensor(th).cuda(), dn,
                                        prec=prec)
        outs.append((d.cpu(), dn.cpu()))
    ctx.set_support_occupancy(prec, 0)
    for d, dn in outs[1:]:
        assert torch.equal(torch.view_as_real(d), torch.view_as_real(outs[0][0]))
        assert torch.equal(dn, outs[0][1])
    for bad in (-1, 33):
        with pytest.raises(tq.TQError):
            ctx.set_support_occupancy(prec, bad)


def test_l2_read_rate(ctx):
    """The L2 read-rate probe returns a rate between the HBM copy rate's
    order and a bound no GB300 L2 reaches, and refuses bad sizes."""
    r = tq.l2_read_rate(ctx, 16 << 20, 16)
    assert 1e12 < r < 1e14
    for nbytes, reps in ((1 << 19, 4), ((256 << 20) + 16, 4), ((1 << 20) + 8, 4), (1 << 20, 0)):
        with pytest.raises(tq.TQError):
            tq.l2_read_rate(ctx, nbytes, reps)


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
def test_support_touch_keeps_every_bit(ctx, prec):
    """The memory-only form of the update (the bench's floor for the access
    pattern) writes every support row back as it read it: the states and
    the carried norms keep their bits under either schedule."""
    import torch
    n, ne, mp = 7, 6, 1
    pool = tq.build_pool(ctx, n, ne, mp)
    S = 256
    psi, k, th, dt = _inputs(14, S, pool.M, 77, prec)
    ref = torch.as_tensor(psi).to(dt).cuda()
    n_in = (ref.abs().double() ** 2).sum(dim=1)
    for ppt in (-2, 4):
        ctx.set_support_schedule(prec, ppt)
        a = ref.clone()
        n2 = n_in.clone()
        tq.evolve_taylor5_batch_support_touch(ctx, pool, a, torch.as_tensor(k).cuda(), n2, prec=prec)
        torch.cuda.synchronize()
        assert torch.equal(torch.view_as_real(a), torch.view_as_real(ref)), ppt
        assert torch.equal(n2, n_in), ppt
    ctx.set_support_schedule(prec, 4 if prec == tq.TQ_C128 else -1)
