"""GPU parity at sizes the oracle cannot run whole: closed forms and samples.

18 qubits (the largest Hamiltonian of the request-loop catalogue): the
Hartree-Fock energy against Slater-Condon, the energy after one rotation
from HF in closed form, and CSR rows recomputed term by term from the
oracle's Pauli sum.  24 qubits (2^24 amplitudes, the pair kernel's largest
routine size here): sampled amplitude pairs recomputed by the oracle's
element formula and the exact norm-growth law of the truncated series.
"""

import math

import numpy as np
import pytest

import paper_2606_29692_gb300 as tq
import synth
from gpu_util import dev_to_numpy
from oracle import fermion, mapping, pauli
from test_oracle_adapt import det_energy
from test_oracle_hamiltonian import hf_energy_closed_form
from test_oracle_pool import slater_condon_gradient_magnitude

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return tq.Context(0)


def _element(ps, r, c):
    """H[r][c] from the oracle's Pauli sum by the element formula."""
    x = r ^ c
    sel = np.nonzero(ps.x == x)[0]
    v = 0.0
    for p in sel:
        ny = bin(int(ps.x[p]) & int(ps.z[p])).count("1")
        sgn = -1.0 if bin(c & int(ps.z[p])).count("1") & 1 else 1.0
        v += (ps.c[p] * (1j ** (ny % 4))).real * sgn
    return v


@pytest.mark.parametrize("mp", [0, 1])
@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
def test_18_qubit_hf_energy_and_rows(ctx, mp, prec):
    n, ne = 9, 8
    ints = synth.integrals(n, 2012)
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, mp, prec)
    assert ham.n_ambiguous == 0
    st = tq.State(ctx, 18, prec)
    tq.state_set_hf(st, ne, mp)
    E = tq.energy(ctx, ham, st)
    assert abs(E - hf_energy_closed_form(ints.h, ints.g, ne)) <= (1e-10 if prec == tq.TQ_C128 else 1e-6)
    if prec == tq.TQ_C64:
        return
    # sampled rows against the oracle's Pauli sum, term by term
    ps = pauli.qubit_hamiltonian(ints.h, ints.g, ints.e_const, mp)
    rp, cp, vp, dp = tq.ham_csr(ham)
    rowptr = dev_to_numpy(rp, (1 << 18) + 1, "<i4")
    diag = dev_to_numpy(dp, 1 << 18, "<f8")
    rng = np.random.default_rng(mp)
    maxc = np.abs(ps.c).max()
    hf = mapping.encode_index(fermion.hf_occupation_index(ne), mapping.encoding_matrix(18, mp))
    for r in [0, hf, (1 << 18) - 1] + list(rng.integers(0, 1 << 18, size=5)):
        r = int(r)
        a, b = int(rowptr[r]), int(rowptr[r + 1])
        cols = dev_to_numpy(cp + 4 * a, b - a, "<i4")
        vals = dev_to_numpy(vp + 8 * a, b - a, "<f8")
        assert np.all(np.diff(cols) > 0)
        for c, v in zip(cols[:: max(1, len(cols) // 40)], vals[:: max(1, len(cols) // 40)]):
            assert abs(v - _element(ps, r, int(c))) <= 1e-14 * maxc
        assert abs(diag[r] - _element(ps, r, r)) <= 1e-14 * np.abs(ps.c).sum()
        # no column missing: every group whose entry survives the drop rule appears
        groups = np.unique(ps.x[ps.x != 0])
        expect = sorted(r ^ int(g) for g in groups if abs(_element(ps, r, r ^ int(g))) > 1e-12 * maxc)
        assert list(cols) == expect
    # XOR-ELL blocks of the same rows: masks and values from the element formula
    nb, npairs, xp, xm, xv = tq.ham_xell(ham)
    assert nb == 1 << 15
    xptr = dev_to_numpy(xp, nb + 1, "<i4")
    for R in [0, hf >> 3, nb - 1] + list(rng.integers(0, nb, size=3)):
        R = int(R)
        a, b = int(xptr[R]), int(xptr[R + 1])
        masks = dev_to_numpy(xm + 4 * a, b - a, "<u4")
        vals = dev_to_numpy(xv + 64 * a, 8 * (b - a), "<f8").reshape(b - a, 8)
        el = {int(g): [_element(ps, 8 * R + i, (8 * R + i) ^ int(g)) for i in range(8)] for g in groups}
        kept = [g for g in sorted(el) if max(abs(v) for v in el[g]) > 1e-12 * maxc]
        assert masks.tolist() == kept
        for j, g in enumerate(kept):
            for i in range(8):
                ref = el[g][i] if abs(el[g][i]) > 1e-12 * maxc else 0.0
                assert abs(vals[j, i] - ref) <= 1e-14 * maxc
                assert (vals[j, i] == 0.0) == (ref == 0.0)


@pytest.mark.parametrize("mp", [0, 1])
def test_18_qubit_one_rotation_closed_form(ctx, mp):
    """T5|HF> = c5|HF> + s5 A|HF>: its energy from Slater-Condon elements."""
    n, ne = 9, 8
    ints = synth.integrals(n, 2013)
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, mp, tq.TQ_C128)
    pool = tq.build_pool(ctx, n, ne, mp)
    exc = fermion.excitations(n, ne)
    st = tq.State(ctx, 18, tq.TQ_C128)
    g = None
    e_hf = hf_energy_closed_form(ints.h, ints.g, ne)
    for k in (0, len(exc) // 2, len(exc) - 1):
        tq.state_set_hf(st, ne, mp)
        g = tq.pool_gradients(ctx, ham, pool, st)
        assert abs(abs(g[k]) - slater_condon_gradient_magnitude(ints.h, ints.g, ne, exc[k])) <= 1e-10
        th = 0.13
        tq.evolve_taylor5(ctx, pool, k, th, st)
        c5 = 1 - th ** 2 / 2 + th ** 4 / 24
        s5 = th - th ** 3 / 6 + th ** 5 / 120
        half = len(exc[k]) // 2
        occ = (set(range(ne)) - set(exc[k][:half])) | set(exc[k][half:])
        e_k = det_energy(ints.h, ints.g, sorted(occ))
        ref = (c5 ** 2 * e_hf + s5 ** 2 * e_k + 2 * c5 * s5 * g[k] / 2) / (c5 ** 2 + s5 ** 2)
        assert abs(tq.energy(ctx, ham, st) - ref) <= 1e-10


@pytest.mark.parametrize("mp", [0, 1])
def test_24_qubit_pair_update_sampled(ctx, mp):
    import torch
    n, ne, nq = 12, 12, 24
    D = 1 << nq
    pool = tq.build_pool(ctx, n, ne, mp)
    rng = np.random.default_rng(24 + mp)
    psi = torch.randn(D, dtype=torch.complex64, device="cuda", generator=torch.Generator("cuda").manual_seed(7))
    psi /= torch.linalg.vector_norm(psi)
    before = psi.clone()
    exc = fermion.excitations(n, ne)
    for k in (3, len(exc) - 5):
        ps = pauli.generator_pauli(exc[k], nq, mp)
        x = int(ps.x[0])
        th = 0.21
        b = before.cpu().numpy().astype(np.complex128)
        norm2 = torch.zeros(1, dtype=torch.float64, device="cuda")
        tq.evolve_taylor5_batch(ctx, pool, psi.view(1, D), torch.tensor([k], dtype=torch.int32, device="cuda"),
                                torch.tensor([th], dtype=torch.float64, device="cuda"), norm2)
        out = psi.cpu().numpy().astype(np.complex128)
        cf = [th ** j / math.factorial(j) for j in range(6)]
        for r in rng.integers(0, D, size=400):
            r = int(r)
            q = r ^ x
            a_rq = _element(ps, r, q)
            a_qr = _element(ps, q, r)
            vr, vq = b[r], b[q]
            acc = vr
            for j in range(1, 6):
                vr, vq = a_rq * vq, a_qr * vr
                acc = acc + cf[j] * vr
            assert abs(out[r] - acc) <= 2e-6 * (abs(acc) + 1e-3)
        # exact norm growth of the truncated series: ||T5 psi||^2 = ||psi||^2
        # + (th^6/360 - th^8/960 + th^10/14400) ||A psi||^2, ||A psi||^2 = weight
        # of psi on the support of A
        rows = np.arange(D, dtype=np.int64)
        s = np.zeros(D)
        for p in range(ps.n_terms):
            ny = bin(int(ps.x[p]) & int(ps.z[p])).count("1")
            cp = (ps.c[p] * (1j ** (ny % 4))).real
            s += cp * (1 - 2 * (np.bitwise_count((rows ^ x) & int(ps.z[p])).astype(np.int64) & 1))
        w_supp = float(np.sum(np.abs(b[rows ^ x]) ** 2 * (s != 0)))
        ref = np.vdot(b, b).real + (th ** 6 / 360 - th ** 8 / 960 + th ** 10 / 14400) * w_supp
        assert abs(norm2.item() - ref) <= 1e-6
        before = psi.clone()
