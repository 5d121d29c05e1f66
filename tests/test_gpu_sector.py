"""GPU parity in the sector-restricted basis (fixed alpha/beta counts).

The CUDA sector path against the oracle's restriction of the full-space
operators: CSR (indices bit-exact), generator tables (exact), energies,
gradients, Taylor-5 (single, batched, host buffers) and free-running ADAPT.
At 18 qubits, where the oracle cannot build the full space, the sector
energy of a state equals the full-space GPU energy of the same state
embedded, and sampled CSR rows match the element formula.
"""

import numpy as np
import pytest

import paper_2606_29692_gb300 as tq
import synth
from gpu_util import dev_to_numpy, fidelity, ham_csr_numpy, oracle_split, rel_l2, to_state
from oracle import adapt, evolve, pauli, sector

pytestmark = pytest.mark.gpu

CFG = {"c0": synth.config0, "c1": synth.config1, "c2": synth.config2,
       "n3": lambda: (synth.integrals(3, 6), 2)}


@pytest.fixture(scope="module")
def ctx():
    return tq.Context(0)


_SYS = {}


def osec(cfg, mp, na, nb):
    key = (cfg, mp, na, nb)
    if key not in _SYS:
        if (cfg, mp) not in _SYS:
            ints, ne = CFG[cfg]()
            _SYS[(cfg, mp)] = (ints, ne, adapt.build_system(ints, ne, mp))
        ints, ne, full = _SYS[(cfg, mp)]
        _SYS[key] = (ints, ne, sector.SectorSystem(full, na, nb))
    return _SYS[key]


def hf_sector(ne):
    return (ne + 1) // 2, ne // 2


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
@pytest.mark.parametrize("cfg,mp,shift", [("n3", 0, 0), ("n3", 1, 1), ("c0", 0, 0), ("c0", 1, 0), ("c1", 1, 0),
                                          ("c1", 0, 1), ("c2", 1, 0)])
def test_sector_hamiltonian_csr_matches_oracle(ctx, cfg, mp, shift, prec):
    ints, ne = CFG[cfg]()
    na, nb = hf_sector(ne)
    na, nb = na - shift, nb + shift
    _, _, s = osec(cfg, mp, na, nb)
    ham = tq.build_hamiltonian_sector(ctx, ints.h, ints.g, ints.e_const, mp, prec, na, nb)
    assert ham.dim == s.dim and ham.n_ambiguous == 0
    rowptr, col, val, diag = ham_csr_numpy(ham)
    orp, ocol, oval, odiag = oracle_split(s.H)
    assert np.array_equal(rowptr, orp) and np.array_equal(col, ocol)
    maxc = np.abs(s.full.ham_pauli.c).max()
    if prec == tq.TQ_C128:
        assert val.size == 0 or np.abs(val - oval).max() <= 1e-14 * maxc
    else:
        ref32 = oval.astype(np.float32)
        assert np.all(np.abs(val.astype(np.float64) - ref32.astype(np.float64)) <= np.spacing(np.abs(ref32)))
    assert np.abs(diag - odiag).max() <= 1e-14 * np.abs(s.full.ham_pauli.c).sum()


@pytest.mark.parametrize("cfg,mp", [("c0", 0), ("c0", 1), ("c1", 1), ("c2", 1)])
def test_sector_pool_tables_match_oracle(ctx, cfg, mp):
    ints, ne = CFG[cfg]()
    na, nb = hf_sector(ne)
    _, _, s = osec(cfg, mp, na, nb)
    pool = tq.build_pool_sector(ctx, ints.n_spatial, ne, mp, na, nb)
    dim, cp, sp = tq.pool_sector_table(pool)
    assert dim == s.dim and pool.M == len(s.pool)
    col = dev_to_numpy(cp, pool.M * dim, "<i4").reshape(pool.M, dim)
    sgn = dev_to_numpy(sp, pool.M * dim, "|i1").reshape(pool.M, dim)
    rows = np.arange(dim)
    for k, A in enumerate(s.pool):
        Ad = A.toarray().real
        nz = Ad.any(axis=1)
        assert np.array_equal(sgn[k] != 0, nz)
        assert np.array_equal(col[k][~nz], rows[~nz])
        assert np.array_equal(Ad[rows[nz], col[k][nz]], sgn[k][nz].astype(float))


def _states(s, ne, seed=5):
    rng = np.random.default_rng(seed)
    hf = sector.hf_state(s.n_spatial, ne, s.n_alpha, s.n_beta)
    corr = hf.copy()
    for k, th in [(0, 0.2), (len(s.pool) // 2, -0.3), (len(s.pool) - 1, 0.15)]:
        corr = evolve.taylor5(s.pool[k], corr, th)
    rand = rng.normal(size=s.dim) + 1j * rng.normal(size=s.dim)
    return {"hf": hf, "corr": corr, "rand": rand * 0.3}


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
@pytest.mark.parametrize("cfg,mp", [("c0", 0), ("c1", 1), ("c2", 1)])
def test_sector_energy_and_gradients(ctx, cfg, mp, prec):
    ints, ne = CFG[cfg]()
    na, nb = hf_sector(ne)
    _, _, s = osec(cfg, mp, na, nb)
    nq = 2 * ints.n_spatial
    ham = tq.build_hamiltonian_sector(ctx, ints.h, ints.g, ints.e_const, mp, prec, na, nb)
    pool = tq.build_pool_sector(ctx, ints.n_spatial, ne, mp, na, nb)
    for name, psi in _states(s, ne).items():
        st = to_state(ctx, psi, nq, prec, sector=(na, nb))
        if prec == tq.TQ_C64:
            psi = st.numpy()
        E_ref, _ = adapt.energy(s.H, psi)
        g_ref = adapt.gradients(s.H, s.pool, psi)
        tol = 1e-10 if prec == tq.TQ_C128 else 1e-6
        assert abs(tq.energy(ctx, ham, st) - E_ref) <= tol, name
        assert np.abs(tq.pool_gradients(ctx, ham, pool, st) - g_ref).max() <= tol, name


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
@pytest.mark.parametrize("mp", [0, 1])
def test_sector_taylor5_single_and_batched(ctx, mp, prec):
    import torch
    ints, ne = CFG["c2"]()
    na, nb = hf_sector(ne)
    _, _, s = osec("c2", mp, na, nb)
    pool = tq.build_pool_sector(ctx, ints.n_spatial, ne, mp, na, nb)
    psi0 = _states(s, ne)["corr"]
    for k, th in [(3, 0.37), (len(s.pool) - 2, -1.1)]:
        st = to_state(ctx, psi0, 14, prec, sector=(na, nb))
        start = st.numpy() if prec == tq.TQ_C64 else psi0
        tq.evolve_taylor5(ctx, pool, k, th, st, renormalize=False)
        ref = evolve.taylor5(s.pool[k], start, th)
        if prec == tq.TQ_C128:
            assert rel_l2(st.numpy(), ref) <= 1e-12
        else:
            assert rel_l2(st.numpy(), ref) <= 2e-6
    # batched: each state its own op and angle, norms returned
    rng = np.random.default_rng(9)
    B = 37
    ks = rng.integers(0, len(s.pool), size=B).astype(np.int32)
    ths = rng.normal(0, 0.4, size=B)
    dt = torch.complex128 if prec == tq.TQ_C128 else torch.complex64
    batch = np.stack([_states(s, ne, seed=b)["rand"] for b in range(B)])
    dev = torch.as_tensor(batch, dtype=dt).cuda().contiguous()
    start = dev.cpu().numpy().astype(np.complex128)
    n2 = torch.zeros(B, dtype=torch.float64, device="cuda")
    tq.evolve_taylor5_batch(ctx, pool, dev, torch.as_tensor(ks).cuda(), torch.as_tensor(ths).cuda(), n2, prec=prec)
    out = dev.cpu().numpy()
    host = torch.as_tensor(batch, dtype=dt).contiguous()
    hn2 = torch.zeros(B, dtype=torch.float64)
    tq.evolve_taylor5_batch_host(ctx, pool, host, torch.as_tensor(ks), torch.as_tensor(ths), hn2, prec=prec)
    for b in range(B):
        ref = evolve.taylor5(s.pool[ks[b]], start[b], ths[b])
        tol = 1e-12 if prec == tq.TQ_C128 else 2e-6
        assert rel_l2(out[b], ref) <= tol
        assert np.array_equal(out[b], host.numpy()[b])
        assert abs(n2[b].item() - np.vdot(ref, ref).real) <= tol * 4 * np.vdot(ref, ref).real
        assert n2[b].item() == hn2[b].item()


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
def test_sector_free_running_adapt_matches_oracle_and_full_space(ctx, prec):
    ints, ne = synth.config1()
    mp = 1
    na, nb = hf_sector(ne)
    _, _, s = osec("c1", mp, na, nb)
    res, psi_ref = adapt.trajectory(s, sector.hf_state(6, ne, na, nb), 1e-3, n_iter=20)
    ham = tq.build_hamiltonian_sector(ctx, ints.h, ints.g, 0.0, mp, prec, na, nb)
    pool = tq.build_pool_sector(ctx, 6, ne, mp, na, nb)
    st = tq.State(ctx, 12, prec, sector=(na, nb))
    tq.state_set_hf(st, ne, mp)
    full_h = tq.build_hamiltonian(ctx, ints.h, ints.g, 0.0, mp, prec)
    full_p = tq.build_pool(ctx, 6, ne, mp)
    fst = tq.State(ctx, 12, prec)
    tq.state_set_hf(fst, ne, mp)
    tolE = 1e-10 if prec == tq.TQ_C128 else 1e-6
    for it, ref in enumerate(res):
        r = tq.adapt_step(ctx, ham, pool, st, 1e-3)
        rf = tq.adapt_step(ctx, full_h, full_p, fst, 1e-3)
        assert r["selected"] == ref.selected == rf["selected"], it
        assert abs(r["energy"] - ref.energy) <= tolE, it
        assert abs(r["energy"] - rf["energy"]) <= tolE, it
    assert fidelity(st.numpy(), psi_ref) > 0.999999
    # the sector state is the full-space state's restriction
    assert fidelity(st.numpy(), fst.numpy()[s.qidx]) > 0.999999


def test_jw_and_bk_sector_matrices_are_identical_on_gpu(ctx):
    ints, ne = synth.config2()
    na, nb = hf_sector(ne)
    a = ham_csr_numpy(tq.build_hamiltonian_sector(ctx, ints.h, ints.g, 0.0, 0, tq.TQ_C128, na, nb))
    b = ham_csr_numpy(tq.build_hamiltonian_sector(ctx, ints.h, ints.g, 0.0, 1, tq.TQ_C128, na, nb))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    scale = np.abs(a[2]).max()
    assert np.abs(a[2] - b[2]).max() <= 1e-13 * scale and np.abs(a[3] - b[3]).max() <= 1e-13 * scale


def test_sector_mismatches_are_rejected(ctx):
    ints, ne = synth.config0()
    ham = tq.build_hamiltonian_sector(ctx, ints.h, ints.g, 0.0, 0, tq.TQ_C128, 2, 2)
    pool = tq.build_pool_sector(ctx, 4, ne, 0, 2, 2)
    full = tq.State(ctx, 8, tq.TQ_C128)
    other = tq.State(ctx, 8, tq.TQ_C128, sector=(1, 3))
    for st in (full, other):
        with pytest.raises(tq.TQError):
            tq.energy(ctx, ham, st)
        with pytest.raises(tq.TQError):
            tq.evolve_taylor5(ctx, pool, 0, 0.1, st)
    with pytest.raises(tq.TQError):
        tq.state_set_hf(other, ne, 0)                       # HF is in (2, 2)
    st = tq.State(ctx, 8, tq.TQ_C128, sector=(2, 2))
    with pytest.raises(tq.TQError):
        tq.energy_matrix_free(ctx, ham, st)
    with pytest.raises(tq.TQError):
        tq.autotune_pair(ctx, pool, tq.TQ_C64, 8)
    with pytest.raises(tq.TQError):
        tq.Batch(ctx, [ham], [pool], [ne], [0], [[0.1]])
    with pytest.raises(tq.TQError):
        tq.build_hamiltonian_sector(ctx, ints.h, ints.g, 0.0, 0, tq.TQ_C128, 5, 0)


@pytest.mark.parametrize("mp", [0, 1])
def test_18_qubit_sector_energy_equals_full_space(ctx, mp):
    """n = 9, 4 + 4 electrons: 15876 amplitudes instead of 262144."""
    import torch
    n, ne = 9, 8
    ints = synth.integrals(n, 2012)
    na, nb = hf_sector(ne)
    hs = tq.build_hamiltonian_sector(ctx, ints.h, ints.g, ints.e_const, mp, tq.TQ_C128, na, nb)
    hf = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, mp, tq.TQ_C128)
    qidx = torch.as_tensor(tq.sector_basis(n, na, nb, mp).astype(np.int64)).cuda()
    g = torch.Generator("cuda").manual_seed(3)
    psi_s = torch.randn(hs.dim, dtype=torch.complex128, device="cuda", generator=g)
    full = torch.zeros(1 << 18, dtype=torch.complex128, device="cuda")
    full[qidx] = psi_s
    e_s = tq.energy(ctx, hs, tq.State(ctx, 18, tq.TQ_C128, tensor=psi_s, sector=(na, nb)))
    e_f = tq.energy(ctx, hf, tq.State(ctx, 18, tq.TQ_C128, tensor=full))
    assert abs(e_s - e_f) <= 1e-10 * max(1.0, abs(e_f))
    # sampled sector rows against the element formula of the oracle's Pauli sum
    ps = pauli.qubit_hamiltonian(ints.h, ints.g, ints.e_const, mp)
    rp, cp, vp, dp = tq.ham_csr(hs)
    rowptr = dev_to_numpy(rp, hs.dim + 1, "<i4")
    q = qidx.cpu().numpy()
    pos = {int(v): i for i, v in enumerate(q)}
    maxc = np.abs(ps.c).max()
    groups = np.unique(ps.x[ps.x != 0])
    for r in np.random.default_rng(mp).integers(0, hs.dim, size=4):
        a, b = int(rowptr[r]), int(rowptr[r + 1])
        cols = dev_to_numpy(cp + 4 * a, b - a, "<i4")
        vals = dev_to_numpy(vp + 8 * a, b - a, "<f8")
        e = int(q[r])
        expect = {}
        for gx in groups:
            c = e ^ int(gx)
            if c in pos:
                sel = np.nonzero(ps.x == gx)[0]
                v = 0.0
                for p_ in sel:
                    ny = bin(int(ps.x[p_]) & int(ps.z[p_])).count("1")
                    sgn = -1.0 if bin(c & int(ps.z[p_])).count("1") & 1 else 1.0
                    v += (ps.c[p_] * (1j ** (ny % 4))).real * sgn
                if abs(v) > 1e-12 * maxc:
                    expect[pos[c]] = v
        assert sorted(expect) == list(cols)
        for c, v in zip(cols, vals):
            assert abs(v - expect[int(c)]) <= 1e-14 * maxc
