"""C ABI checks that need no GPU.

The library must load without a device, export every entry point declared
in include/tq.h, and its host-side algebra (Pauli sums, pool, Hartree-Fock
index) must match the oracle: masks bit-exact, coefficients to rounding.
"""

import os
import re
import subprocess

import numpy as np
import pytest

import synth
from oracle import adapt as oadapt
from oracle import fermion, mapping, pauli

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:const\s+char\s*\*|int|void)\s+(tq_\w+)\s*\(", txt, re.M))
    return names


@pytest.fixture(scope="module")
def tq():
    from paper_2606_29692_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    import paper_2606_29692_gb300 as m
    m.lib()
    return m


def test_every_declared_symbol_is_exported(tq):
    from paper_2606_29692_gb300 import _native
    declared = _declared_symbols()
    assert len(declared) >= 25
    out = subprocess.run(["nm", "-D", "--defined-only", _native.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (tq_\w+)", out))
    assert declared <= exported, declared - exported
    # the Python binding declares every one of them too
    assert declared <= set(_native.SIGNATURES)


def test_no_gpu_needed_to_load(tq):
    assert tq.lib().tq_version() == 100


def _oracle_matrix_coefs(ps):
    ny = np.bitwise_count(ps.x & ps.z).astype(np.int64)
    return (ps.c * (1j ** (ny % 4)))


@pytest.mark.parametrize("mp", [mapping.JW, mapping.BK])
@pytest.mark.parametrize("cfg", ["c0", "c1", "c2", "n5"])
def test_pauli_hamiltonian_matches_oracle(tq, mp, cfg):
    if cfg == "n5":
        ints, ne = synth.integrals(5, 77), 4
    else:
        ints, ne = {"c0": synth.config0, "c1": synth.config1, "c2": synth.config2}[cfg]()
    x, z, c = tq.pauli_hamiltonian(ints.h, ints.g, 0.5, mp)
    ps = pauli.qubit_hamiltonian(ints.h, ints.g, 0.5, mp)
    assert np.array_equal(x.astype(np.int64), ps.x)
    assert np.array_equal(z.astype(np.int64), ps.z)
    cm = _oracle_matrix_coefs(ps)
    assert np.abs(cm.imag).max() == 0.0
    assert np.abs(c - cm.real).max() <= 1e-14 * np.abs(c).max()


def test_pool_excitations_match_oracle(tq):
    for n, ne in [(4, 4), (6, 8), (7, 6), (5, 2), (8, 8)]:
        idx = tq.pool_excitations(n, ne)
        ref = fermion.excitations(n, ne)
        assert idx.shape[0] == len(ref)
        for row, e in zip(idx, ref):
            assert tuple(int(v) for v in row[: len(e)]) == e
            assert all(v == -1 for v in row[len(e):])


@pytest.mark.parametrize("mp", [mapping.JW, mapping.BK])
def test_pauli_pool_matches_oracle(tq, mp):
    n, ne = 7, 6
    x, nt, z, c = tq.pauli_pool(n, ne, mp)
    _, ref = pauli.pool_pauli(n, ne, mp)
    assert len(ref) == x.size == 204
    for k, ps in enumerate(ref):
        assert nt[k] == ps.n_terms
        assert np.all(ps.x == int(x[k]))
        assert np.array_equal(z[k, : nt[k]].astype(np.int64), ps.z)
        cm = _oracle_matrix_coefs(ps)
        assert np.array_equal(c[k, : nt[k]], cm.real)    # dyadic: exact
        assert np.abs(cm.imag).max() == 0.0


@pytest.mark.parametrize("mp", [mapping.JW, mapping.BK])
def test_hf_index_matches_oracle(tq, mp):
    for nq, ne in [(8, 4), (12, 8), (14, 6), (16, 8), (18, 8), (30, 10)]:
        B = mapping.encoding_matrix(nq, mp)
        assert tq.hf_index(nq, ne, mp) == mapping.encode_index(fermion.hf_occupation_index(ne), B)


def test_invalid_arguments_are_rejected(tq):
    with pytest.raises(tq.TQError) as e:
        tq.pool_excitations(0, 0)
    assert e.value.code == -1
    with pytest.raises(tq.TQError):
        tq.pool_excitations(4, 9)
    with pytest.raises(tq.TQError):
        tq.hf_index(8, 4, 7)
    ints, _ = synth.config0()
    with pytest.raises(tq.TQError):
        tq.pauli_hamiltonian(ints.h, ints.g, 0.0, 5)


@pytest.mark.parametrize("mp", [mapping.JW, mapping.BK])
def test_sector_basis_matches_oracle(tq, mp):
    from oracle import sector
    for n, na, nb in [(1, 1, 0), (3, 1, 2), (4, 2, 2), (6, 4, 4), (7, 3, 3), (7, 2, 4)]:
        assert tq.sector_dim(n, na, nb) == sector.dimension(n, na, nb)
        got = tq.sector_basis(n, na, nb, mp).astype(np.int64)
        assert np.array_equal(got, sector.qubit_basis(n, na, nb, mp))
    # the largest sector a device state can hold (26 qubits): dimension only
    assert tq.sector_dim(13, 6, 7) == sector.dimension(13, 6, 7)


def test_sector_arguments_are_rejected(tq):
    for args in [(0, 0, 0), (14, 7, 7), (4, 5, 0), (4, 0, -1)]:
        with pytest.raises(tq.TQError):
            tq.sector_dim(*args)
    with pytest.raises(tq.TQError):
        tq.sector_basis(4, 2, 2, 7)


@pytest.mark.parametrize("mp", [mapping.JW, mapping.BK])
def test_pool_families_match_oracle(tq, mp):
    """Algorithm 1 in the library (Pauli-algebra commutators) against the
    oracle (dense commutators; qubit-wise from Pauli labels): identical
    families, family-major order, and count."""
    from oracle import families, pauli
    cases = [(4, 4, tq.TQ_COMMUTE_FULL), (4, 4, tq.TQ_COMMUTE_QWC), (3, 2, tq.TQ_COMMUTE_FULL),
             (6, 8, tq.TQ_COMMUTE_QWC), (7, 6, tq.TQ_COMMUTE_QWC)]
    for n, ne, mode in cases:
        exc, pool_ps = pauli.pool_pauli(n, ne, mp)
        if mode == tq.TQ_COMMUTE_FULL:
            edges = families.full_edges([pauli.pauli_to_csr(p) for p in pool_ps])
        else:
            edges = families.qwc_edges([families.labels(p) for p in pool_ps])
        ref = families.greedy_families(len(exc), edges)
        fam, order, k = tq.pool_families_host(n, ne, mp, mode)
        assert fam.tolist() == ref, (n, ne, mode)
        assert order.tolist() == families.family_order(ref)
        assert k == max(ref) + 1


def test_pool_families_rejects_bad_mode(tq):
    with pytest.raises(tq.TQError):
        tq.pool_families_host(4, 4, 0, 5)


def test_fcidump_reader_matches_the_golden_expansion(tq):
    from test_oracle_fcidump import GOLD, expected_2orb
    h, g, meta = expected_2orb()
    ints = tq.read_fcidump(os.path.join(GOLD, "fcidump_2orb.txt"))
    assert np.array_equal(ints.h, h) and np.array_equal(ints.g, g)
    assert ints.e_const == meta["e"] and ints.n_electrons == meta["nelec"] and ints.ms2 == meta["ms2"]


def test_fcidump_round_trips_with_the_oracle(tq, tmp_path):
    from oracle import fcidump
    for n, seed in [(3, 6), (6, 1), (9, 2012)]:
        ints = synth.integrals(n, seed)
        a = str(tmp_path / "oracle.txt")
        fcidump.write(a, ints.h, ints.g, 0.375, 2 * (n // 2), ms2=0)
        r = tq.read_fcidump(a)                                   # library reads the oracle's file
        assert np.array_equal(r.h, ints.h) and np.array_equal(r.g, ints.g) and r.e_const == 0.375
        b = str(tmp_path / "lib.txt")
        tq.write_fcidump(b, ints.h, ints.g, -1.5, 2 * (n // 2))
        h, g, e, nn, ne, ms2 = fcidump.read(b)                   # oracle reads the library's file
        assert np.array_equal(h, ints.h) and np.array_equal(g, ints.g) and e == -1.5 and nn == n


def test_fcidump_errors(tq, tmp_path):
    bad = tmp_path / "bad.txt"
    for text in ["no header at all\n", " &FCI NELEC=2, &END\n 1.0 1 1 1 1\n",
                 " &FCI NORB=2,NELEC=2 &END\n 1.0 3 1 1 1\n", " &FCI NORB=2,NELEC=2 &END\n 1.0 1 x 1 1\n"]:
        bad.write_text(text)
        with pytest.raises(tq.TQError):
            tq.read_fcidump(str(bad))
    with pytest.raises(tq.TQError):
        tq.read_fcidump(str(tmp_path / "missing.txt"))


def _insert_zero(v, b):
    return ((v >> b) << (b + 1)) | (v & ((1 << b) - 1))


@pytest.mark.parametrize("n,ne,mp", [(2, 2, mapping.JW), (2, 2, mapping.BK), (4, 4, mapping.JW),
                                     (4, 4, mapping.BK), (6, 8, mapping.BK), (7, 6, mapping.JW),
                                     (7, 6, mapping.BK)])
def test_support_pair_enumeration_covers_the_oracle_support(tq, n, ne, mp):
    """Pairs enumerated from the exported support form (the formula the
    support-only update and the gradients run) are exactly the oracle
    generator's non-zero rows, each pair once, every row in range."""
    N = 2 * n
    f = tq.pool_support_forms(n, ne, mp)
    x, _, _, _ = tq.pauli_pool(n, ne, mp)
    _, pps = pauli.pool_pauli(n, ne, mp)
    for k, ps in enumerate(pps):
        m = int(f["m"][k])
        piv = [int(p) for p in f["pivots"][k, :m]]
        assert piv == sorted(piv) and all(0 <= p < N for p in piv)
        u = np.arange(1 << (N - m - 1), dtype=np.int64)
        r = _insert_zero(u, int(f["rep_pos"][k]))
        for p in piv:
            r = _insert_zero(r, p)
        for i, p in enumerate(piv):
            par = np.array([bin(int(v) & int(f["masks"][k, i])).count("1") & 1 for v in r], dtype=np.int64)
            r = r | (((int(f["target"][k]) >> i) & 1) ^ par) << p
        q = r ^ int(x[k])
        assert r.max() < (1 << N) and np.all((r >> int(f["rep_bit"][k])) & 1 == 0)
        rows = np.concatenate([r, q])
        assert np.unique(rows).size == rows.size                     # each pair once
        A = pauli.pauli_to_csr(ps).tocoo()
        assert np.array_equal(np.sort(rows), np.unique(A.row))


def _permute_bits(v, order):
    v = np.asarray(v, dtype=np.int64)
    out = np.zeros_like(v)
    for k, o in enumerate(order):
        out |= ((v >> k) & 1) << int(o)
    return out


def _relabel_sum(x, z, c, order):
    """A Pauli sum with its qubits relabelled, in the canonical (x, z) order."""
    xp, zp = _permute_bits(x, order), _permute_bits(z, order)
    i = np.lexsort((zp, xp))
    return xp[i], zp[i], np.asarray(c)[i]


@pytest.mark.parametrize("mp", [mapping.JW, mapping.BK])
def test_relabelled_mapping_is_the_oracle_mapping_with_permuted_qubits(tq, mp):
    """A relabelled encoding (qubit k stored at bit order[k]) gives the
    oracle's JW/BK Pauli strings with every mask's bits moved by the order:
    same coefficients, same pool, Hartree-Fock index moved the same way."""
    ints, ne = synth.config1()
    n, N = ints.n_spatial, 2 * ints.n_spatial
    order = np.random.default_rng(11 + mp).permutation(N)
    rl = tq.mapping_relabelled(mp, order)
    assert rl >= 16 and tq.mapping_relabelled(mp, order) == rl        # registered once
    x, z, c = tq.pauli_hamiltonian(ints.h, ints.g, 0.25, rl)
    ps = pauli.qubit_hamiltonian(ints.h, ints.g, 0.25, mp)
    rx, rz, rc = _relabel_sum(ps.x, ps.z, _oracle_matrix_coefs(ps).real, order)
    assert np.array_equal(x.astype(np.int64), rx) and np.array_equal(z.astype(np.int64), rz)
    assert np.abs(c - rc).max() <= 1e-14 * np.abs(c).max()
    px, nt, pz, pc = tq.pauli_pool(n, ne, rl)
    _, pref = pauli.pool_pauli(n, ne, mp)
    for k, p in enumerate(pref):
        assert int(px[k]) == int(_permute_bits(p.x[:1], order)[0])
        rx, rz, rc = _relabel_sum(p.x, p.z, _oracle_matrix_coefs(p).real, order)
        assert np.array_equal(pz[k, : nt[k]].astype(np.int64), rz)
        assert np.array_equal(pc[k, : nt[k]], rc)                     # dyadic: exact
    B = mapping.encoding_matrix(N, mp)
    hf = mapping.encode_index(fermion.hf_occupation_index(ne), B)
    assert tq.hf_index(N, ne, rl) == int(_permute_bits([hf], order)[0])
    ix = tq.relabel_index(order)
    assert np.array_equal(np.sort(ix), np.arange(1 << N))
    # a mapping registered for 12 qubits is refused at another size
    with pytest.raises(tq.TQError):
        tq.hf_index(14, 6, rl)


def test_relabelled_mapping_rejects_bad_orders(tq):
    for base, order in [(2, list(range(8))), (0, [0, 1, 2, 2]), (1, [0, 1, 4, 2]), (0, [])]:
        with pytest.raises(tq.TQError) as e:
            tq.mapping_relabelled(base, order)
        assert e.value.code == -1


def _support_masks(f, k):
    return [int(f["masks"][k, i]) for i in range(int(f["m"][k]))]


def test_sector_order_first_pair_is_the_brute_force_best(tq):
    """The greedy qubit order's two lowest bits are the pair that minimises
    the touched 32-byte sectors of the pool's supports, counted row by row
    from the exported support form (brute force over all pairs)."""
    import itertools
    n, ne, mp = 7, 6, mapping.BK
    N = 2 * n
    f = tq.pool_support_forms(n, ne, mp)
    x, _, _, _ = tq.pauli_pool(n, ne, mp)
    rows = []
    for k in range(x.size):
        m = int(f["m"][k])
        r = np.arange(1 << N, dtype=np.int64)
        keep = np.ones(r.size, dtype=bool)
        for i, e in enumerate(_support_masks(f, k)):
            keep &= (np.bitwise_count(r & e) & 1) == ((int(f["target"][k]) >> i) & 1)
        rows.append(r[keep])
        assert rows[-1].size == 1 << (N - m)

    def touched(pair):
        msk = (1 << pair[0]) | (1 << pair[1])
        return sum(np.unique(r & ~msk).size for r in rows)

    cost = {p: touched(p) for p in itertools.combinations(range(N), 2)}
    best = min(cost.values())
    order = tq.pool_sector_order(n, ne, mp, 2)
    low = tuple(sorted(int(np.nonzero(order == b)[0][0]) for b in (0, 1)))
    assert cost[low] == best
    assert cost[low] < cost[(0, 1)]                      # better than the natural order
    assert np.array_equal(np.sort(order), np.arange(N))
    # the rest keep their base order
    rest = [q for q in range(N) if q not in low]
    assert [int(order[q]) for q in rest] == list(range(2, N))


def _dense_from_terms(x, z, c, N):
    """Dense matrix of sum_t c_t X^{x_t} Z^{z_t} (the library's real form:
    <s ^ x| X^x Z^z |s> = (-1)^{popcount(s & z)})."""
    s = np.arange(1 << N, dtype=np.int64)
    H = np.zeros((1 << N, 1 << N))
    for xt, zt, ct in zip(np.asarray(x, dtype=np.int64), np.asarray(z, dtype=np.int64), c):
        sign = 1.0 - 2.0 * (np.bitwise_count(s & zt) & 1)
        np.add.at(H, (s ^ xt, s), ct * sign)
    return H


def _random_invertible(N, rng):
    while True:
        rows = rng.integers(0, 1 << N, size=N, dtype=np.int64)
        a = [int(r) for r in rows]
        rank = 0
        for bit in range(N):
            piv = next((i for i in range(rank, N) if (a[i] >> bit) & 1), None)
            if piv is None:
                continue
            a[rank], a[piv] = a[piv], a[rank]
            for i in range(N):
                if i != rank and (a[i] >> bit) & 1:
                    a[i] ^= a[rank]
            rank += 1
        if rank == N:
            return rows.astype(np.uint64)


@pytest.mark.parametrize("mp", [mapping.JW, mapping.BK])
def test_linear_mapping_is_the_base_mapping_under_its_index_map(tq, mp):
    """Under an invertible GF(2) index map r' = M r the Hamiltonian, every
    pool generator and the Hartree-Fock state are the base mapping's with
    rows and columns moved by the map: H'[M r, M s] = H[r, s] (8 qubits,
    dense, from the library's own Pauli terms; the base terms are pinned
    to the oracle by the test above)."""
    ints, ne = synth.config0()
    n, N = ints.n_spatial, 2 * ints.n_spatial
    rows = _random_invertible(N, np.random.default_rng(5 + mp))
    ml = tq.mapping_linear(mp, rows)
    assert ml >= 16 and tq.mapping_linear(mp, rows) == ml
    ix = tq.linear_index(rows)
    assert np.array_equal(np.sort(ix), np.arange(1 << N))
    Hb = _dense_from_terms(*tq.pauli_hamiltonian(ints.h, ints.g, 0.25, mp), N)
    Hl = _dense_from_terms(*tq.pauli_hamiltonian(ints.h, ints.g, 0.25, ml), N)
    assert np.abs(Hl[np.ix_(ix, ix)] - Hb).max() <= 1e-13 * np.abs(Hb).max()
    bx, bnt, bz, bc = tq.pauli_pool(n, ne, mp)
    lx, lnt, lz, lc = tq.pauli_pool(n, ne, ml)
    for k in range(bx.size):
        Ab = _dense_from_terms([bx[k]] * bnt[k], bz[k, : bnt[k]], bc[k, : bnt[k]], N)
        Al = _dense_from_terms([lx[k]] * lnt[k], lz[k, : lnt[k]], lc[k, : lnt[k]], N)
        assert np.array_equal(Al[np.ix_(ix, ix)], Ab), k          # dyadic coefficients: exact
    assert tq.hf_index(N, ne, ml) == int(ix[tq.hf_index(N, ne, mp)])


def test_linear_mapping_of_a_permutation_is_the_relabelled_mapping(tq):
    order = np.random.default_rng(3).permutation(12)
    rows = np.zeros(12, dtype=np.uint64)
    for k, o in enumerate(order):
        rows[o] = 1 << k
    assert tq.mapping_linear(mapping.BK, rows) == tq.mapping_relabelled(mapping.BK, order)
    assert np.array_equal(tq.linear_index(rows), tq.relabel_index(order))


def test_linear_mapping_rejects_bad_maps(tq):
    singular = np.array([1, 2, 3, 8], dtype=np.uint64)                  # row 2 = row 0 ^ row 1
    wide = np.array([1, 2, 4, 16], dtype=np.uint64)                     # bit 4 of a 4-qubit index
    for base, rows in [(mapping.BK, singular), (mapping.JW, wide), (2, np.array([1, 2], dtype=np.uint64))]:
        with pytest.raises(tq.TQError) as e:
            tq.mapping_linear(base, rows)
        assert e.value.code == -1


def _touched_sectors(tq, n, ne, mp):
    """Support rows of every pool generator (numpy, from the exported support
    form) and the 32-byte sectors (4 complex64 amplitudes) they touch."""
    N = 2 * n
    f = tq.pool_support_forms(n, ne, mp)
    r = np.arange(1 << N, dtype=np.int64)
    n_rows = n_sect = 0
    for k in range(f["m"].size):
        keep = np.ones(r.size, dtype=bool)
        for i, e in enumerate(_support_masks(f, k)):
            keep &= (np.bitwise_count(r & e) & 1) == ((int(f["target"][k]) >> i) & 1)
        n_rows += int(keep.sum())
        n_sect += np.unique(r[keep] >> 2).size
    return n_rows, n_sect


def test_sector_basis_packs_supports_tighter_than_any_qubit_order(tq):
    """The greedy GF(2) basis for the 14-qubit BK pool: an invertible map,
    and its supports touch fewer 32-byte sectors (counted row by row) than
    the best qubit order's: 170496 against 201216 for 565248 rows (fill
    0.83 against 0.70)."""
    n, ne, mp = 7, 6, mapping.BK
    rows = tq.pool_sector_basis(n, ne, mp)
    ml = tq.mapping_linear(mp, rows)                                    # raises if singular
    order = tq.pool_sector_order(n, ne, mp, 14)
    nr_l, ns_l = _touched_sectors(tq, n, ne, ml)
    nr_o, ns_o = _touched_sectors(tq, n, ne, tq.mapping_relabelled(mp, order))
    assert nr_l == nr_o == 565248
    assert (ns_l, ns_o) == (170496, 201216)
