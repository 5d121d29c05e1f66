"""Pins for the commuting-family partition (Sec. III-F, Algorithm 1)."""

import os

import numpy as np
import pytest

import synth
from oracle import adapt, families, fermion

GOLD = os.path.join(os.path.dirname(__file__), "golden", "algorithm1_trace.txt")


def _read_trace():
    d = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        key, *rest = line.split()
        d[key] = rest
    n = int(d["n"][0])
    edges = {tuple(sorted(map(int, e.split("-")))) for e in d["edges"]}
    return n, edges, [int(v) for v in d["family"]]


def test_hand_traced_example():
    n, edges, fam = _read_trace()
    assert families.greedy_families(n, edges) == fam


def test_textbook_graphs():
    k4 = {(i, j) for i in range(4) for j in range(i + 1, 4)}
    assert sorted(set(families.greedy_families(4, k4))) == [0, 1, 2, 3]
    c5 = {(i, (i + 1) % 5) if i < (i + 1) % 5 else ((i + 1) % 5, i) for i in range(5)}
    assert len(set(families.greedy_families(5, c5))) == 3
    c6 = {tuple(sorted((i, (i + 1) % 6))) for i in range(6)}
    assert families.greedy_families(6, c6) == [0, 1, 0, 1, 0, 1]
    star = {(0, j) for j in range(1, 5)}
    assert families.greedy_families(5, star) == [0, 1, 1, 1, 1]
    assert families.greedy_families(3, set()) == [0, 0, 0]


def _pool(cfg, mp):
    ints, ne = {"c0": synth.config0, "n3": lambda: (synth.integrals(3, 6), 2)}[cfg]()
    return adapt.build_system(ints, ne, mp)


def _valid(fam, edges):
    return all(fam[i] != fam[j] for i, j in edges)


@pytest.mark.parametrize("cfg", ["n3", "c0"])
def test_pool_partitions_are_valid_and_bounded(cfg):
    jw, bk = _pool(cfg, 0), _pool(cfg, 1)
    full_jw = families.full_edges(jw.pool)
    full_bk = families.full_edges(bk.pool)
    assert full_jw == full_bk                                # commutation does not depend on the basis
    for s in (jw, bk):
        qwc = families.qwc_edges([families.labels(p) for p in s.pool_pauli])
        assert full_jw <= qwc                                # qubit-wise commuting implies commuting
        for edges in (full_jw, qwc):
            fam = families.greedy_families(len(s.pool), edges)
            assert _valid(fam, edges)
            deg = np.bincount(np.array(sorted(edges)).ravel(), minlength=len(s.pool)) if edges else [0]
            assert max(fam) + 1 <= max(deg) + 1              # greedy bound
            order = families.family_order(fam)
            assert sorted(order) == list(range(len(s.pool)))
            assert [fam[v] for v in order] == sorted(fam)


@pytest.mark.parametrize("mp", [0, 1])
def test_generators_on_disjoint_modes_commute(mp):
    s = _pool("c0", mp)
    full = families.full_edges(s.pool)
    for i, a in enumerate(s.excitations):
        for j, b in enumerate(s.excitations):
            if i < j and not set(a) & set(b):
                assert (i, j) not in full
    # and the pool does have non-commuting pairs
    assert full


def test_full_edges_match_the_commutator_definition_on_a_tiny_pool():
    # 2 spatial orbitals, 2 electrons: singles 0->2, 1->3 and the double 01->23
    exc = fermion.excitations(2, 2)
    mats = [fermion.generator_matrix(4, e) for e in exc]
    edges = families.full_edges(mats)
    # the two singles act on disjoint modes; each single fails to commute with the double
    assert exc == [(0, 2), (1, 3), (0, 1, 2, 3)]
    assert edges == {(0, 2), (1, 2)}
