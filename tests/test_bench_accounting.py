"""The benchmark's algorithmic byte count, checked on the CPU.

The roofline of the support-only update counts, per state, the rows of its
generator's support (read and written once each).  The benchmark rebuilds
those rows from the library's exported support forms; here they must be
exactly the rows where the oracle's generator matrix (Sec. III-C: A_k from
its Pauli strings) has an entry: every support row once, no other row.
"""

import numpy as np
import pytest

import bench
import paper_2606_29692_gb300 as tq
from oracle import pauli


@pytest.mark.parametrize("n,ne,mp", [(4, 4, 0), (4, 4, 1), (6, 8, 1), (7, 6, 1)])
def test_support_rows_are_the_oracle_support(n, ne, mp):
    rows = bench.support_rows(tq, n, ne, mp)
    _, pps = pauli.pool_pauli(n, ne, mp)
    assert len(rows) == len(pps)
    for k, (r, p) in enumerate(zip(rows, pps)):
        ref = np.unique(pauli.pauli_to_csr(p).nonzero()[0])
        got = np.sort(np.asarray(r, dtype=np.int64))
        assert np.array_equal(got, ref), k


def test_headline_byte_model():
    """The 14-qubit BK pool: singles touch D/2 rows and doubles D/8, so the
    mean over the pool is (24 D/2 + 180 D/8) / 204 rows per update."""
    D = 1 << 14
    rows = bench.support_rows(tq, 7, 6, 1)
    sizes = np.array([r.size for r in rows])
    assert sizes.size == 204
    assert sorted(set(sizes.tolist())) == [D // 8, D // 2]
    assert (sizes == D // 2).sum() == 24
    assert abs(sizes.mean() - (24 * D / 2 + 180 * D / 8) / 204) < 1e-9
