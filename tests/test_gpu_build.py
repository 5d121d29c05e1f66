"""GPU parity: Pauli -> CSR compilation and the pool layout (CUDA vs oracle)."""

import numpy as np
import pytest

import paper_2606_29692_gb300 as tq
import synth
from gpu_util import dev_to_numpy, ham_csr_numpy, oracle_split
from oracle import pauli

pytestmark = pytest.mark.gpu

CFG = {"c0": synth.config0, "c1": synth.config1, "c2": synth.config2,
       "n1": lambda: (synth.integrals(1, 5), 2), "n3": lambda: (synth.integrals(3, 6), 2)}


@pytest.fixture(scope="module")
def ctx():
    return tq.Context(0)


_ORACLE = {}


def oracle_h(cfg, mp):
    key = (cfg, mp)
    if key not in _ORACLE:
        ints, ne = CFG[cfg]()
        ps = pauli.qubit_hamiltonian(ints.h, ints.g, ints.e_const, mp)
        _ORACLE[key] = (ints, ne, ps, pauli.pauli_to_csr(ps))
    return _ORACLE[key]


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
@pytest.mark.parametrize("cfg,mp", [("n1", 0), ("n3", 1), ("c0", 0), ("c0", 1), ("c1", 0), ("c1", 1),
                                    ("c2", 1), ("c2", 0)])
def test_hamiltonian_csr_matches_oracle(ctx, cfg, mp, prec):
    ints, ne, ps, H = oracle_h(cfg, mp)
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, mp, prec)
    rowptr, col, val, diag = ham_csr_numpy(ham)
    orp, ocol, oval, odiag = oracle_split(H)
    assert ham.n_pauli == ps.n_terms
    assert ham.n_ambiguous == 0
    assert np.array_equal(rowptr, orp), "rowptr differs"
    assert np.array_equal(col, ocol), "column indices differ"
    # The library's Pauli coefficients come from its own (symplectic) route,
    # which merges like terms in a different order than the oracle: entries
    # agree to rounding, 1e-14 relative to the largest coefficient.
    maxc = np.abs(ps.c).max()
    if val.size == 0:
        assert oval.size == 0
    elif prec == tq.TQ_C128:
        assert np.abs(val - oval).max() <= 1e-14 * maxc
    else:
        ref32 = oval.astype(np.float32)
        ulp = np.spacing(np.abs(ref32)).astype(np.float64)
        assert np.all(np.abs(val.astype(np.float64) - ref32.astype(np.float64)) <= ulp)
    # the diagonal is kept dense (no zero-drop): entries that vanish exactly
    # (e.g. the vacuum row) carry a rounding residue on either side
    assert np.abs(diag - odiag).max() <= 1e-14 * np.abs(ps.c).sum()


def xell_numpy(ham, prec):
    nb, npairs, xp, xm, xv = tq.ham_xell(ham)
    xptr = dev_to_numpy(xp, nb + 1, "<i4")
    xmask = dev_to_numpy(xm, npairs, "<u4") if npairs else np.zeros(0, np.uint32)
    vt = "<f8" if prec == tq.TQ_C128 else "<f4"
    xval = dev_to_numpy(xv, 8 * npairs, vt).reshape(npairs, 8) if npairs else np.zeros((0, 8))
    return nb, xptr, xmask, xval


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
@pytest.mark.parametrize("cfg,mp", [("n1", 0), ("n3", 1), ("c0", 0), ("c1", 0), ("c1", 1), ("c2", 1)])
def test_hamiltonian_xell_matches_oracle(ctx, cfg, mp, prec):
    """The XOR-ELL layout holds exactly the CSR's entries: per block of 8
    rows, the X-masks r ^ c of the oracle's off-diagonal entries (ascending,
    bit-exact), the oracle's value where the entry exists and exact zero
    where it does not; values equal the library's own CSR bit for bit."""
    ints, ne, ps, H = oracle_h(cfg, mp)
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, mp, prec)
    nb, xptr, xmask, xval = xell_numpy(ham, prec)
    rowptr, col, val, _ = ham_csr_numpy(ham)
    orp, ocol, oval, _ = oracle_split(H)
    D = len(orp) - 1
    assert nb == (D + 7) // 8 and xptr[0] == 0
    maxc = np.abs(ps.c).max()
    for R in range(nb):
        rows = range(8 * R, min(8 * R + 8, D))
        expect = sorted({r ^ int(c) for r in rows for c in ocol[orp[r]:orp[r + 1]]})
        got = xmask[xptr[R]:xptr[R + 1]]
        assert got.tolist() == expect, f"block {R}: X-masks differ"
        blk = xval[xptr[R]:xptr[R + 1]]
        for i, r in enumerate(rows):
            oc = {int(c): v for c, v in zip(ocol[orp[r]:orp[r + 1]], oval[orp[r]:orp[r + 1]])}
            mine = {int(c): v for c, v in zip(col[rowptr[r]:rowptr[r + 1]], val[rowptr[r]:rowptr[r + 1]])}
            for j, x in enumerate(expect):
                c = r ^ x
                if c in oc:
                    assert blk[j, i] == mine[c]
                    assert abs(float(blk[j, i]) - oc[c]) <= (1e-14 * maxc if prec == tq.TQ_C128
                                                            else float(np.spacing(np.float32(abs(oc[c])))))
                else:
                    assert blk[j, i] == 0.0
        for i in range(len(rows), 8):
            assert np.all(blk[:, i] == 0.0)


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
@pytest.mark.parametrize("n,ne,mp", [(2, 2, 0), (4, 4, 0), (4, 4, 1), (6, 8, 1), (7, 6, 1)])
def test_pool_csr_matches_oracle(ctx, n, ne, mp, prec):
    exc, pps = pauli.pool_pauli(n, ne, mp)
    pool = tq.build_pool(ctx, n, ne, mp)
    assert pool.M == len(exc)
    assert [tuple(int(v) for v in row[: len(e)]) for row, e in zip(pool.idx4, exc)] == exc
    ks = range(pool.M) if pool.M <= 92 else list(range(0, pool.M, 17)) + [pool.M - 1]
    D = 1 << (2 * n)
    for k in ks:
        rp, cl, vl, nnz = tq.pool_csr(ctx, pool, k, prec)
        A = pauli.pauli_to_csr(pps[k])
        assert nnz == A.nnz
        assert np.array_equal(dev_to_numpy(rp, D + 1, "<i4"), A.indptr)
        assert np.array_equal(dev_to_numpy(cl, nnz, "<i4"), A.indices)
        v = dev_to_numpy(vl, nnz, "<f8" if prec == tq.TQ_C128 else "<f4")
        assert np.array_equal(v.astype(np.float64), A.data.real)


def test_build_rejects_bad_arguments(ctx):
    ints, _ = synth.config0()
    with pytest.raises(tq.TQError):
        tq.build_hamiltonian(ctx, ints.h, ints.g, 0.0, 3, tq.TQ_C128)
    with pytest.raises(tq.TQError):
        tq.build_hamiltonian(ctx, ints.h, ints.g, 0.0, 0, 7)
    with pytest.raises(tq.TQError):
        tq.build_pool(ctx, 1, 1, 0)        # empty pool
    with pytest.raises(tq.TQError):
        tq.build_hamiltonian(ctx, ints.h, ints.g, float("inf"), 0, tq.TQ_C128)


@pytest.mark.parametrize("mode", [tq.TQ_COMMUTE_FULL, tq.TQ_COMMUTE_QWC])
def test_pool_families_of_a_device_pool_equal_the_host_ones(ctx, mode):
    for n, ne, mp in [(4, 4, 0), (7, 6, 1)]:
        pool = tq.build_pool(ctx, n, ne, mp)
        fam, order, k = tq.pool_families(pool, mode)
        hfam, horder, hk = tq.pool_families_host(n, ne, mp, mode)
        assert np.array_equal(fam, hfam) and np.array_equal(order, horder) and k == hk
