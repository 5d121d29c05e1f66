"""The energy entry point that allocates nothing, checked against tq_energy.

Callers that cannot allocate device memory where they need an energy -- a
serving loop that reserved its memory up front and must not stall the GPU on
cudaMalloc/cudaFree, or a host whose own allocator owns the device heap --
use tq_energy_noalloc, which keeps its scratch in a fixed device array.  This
file is collected last so that a run stopping at the first failure has run
every other test first; it also passes on its own in a fresh process.
"""

import numpy as np
import pytest

import paper_2606_29692_gb300 as tq
import synth
from gpu_util import to_state

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
def test_noalloc_energy_equals_energy_on_two_calls(prec):
    import torch
    ctx = tq.Context(0)
    ints, ne = synth.config1()
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, tq.TQ_BK, prec)
    rp, cl, vl, dg = tq.ham_csr(ham)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    tol = 1e-10 if prec == tq.TQ_C128 else 1e-6
    # two calls in a row on different states: the shared scratch keeps the
    # previous call's contents, which must not leak into the next result
    for seed in (3, 4):
        st = to_state(ctx, synth.random_state(12, seed), 12, prec)
        ref = tq.energy(ctx, ham, st)
        out.fill_(float("nan"))
        tq.energy_noalloc(12, prec, rp, cl, vl, dg, st.tensor.data_ptr(), out.data_ptr())
        torch.cuda.synchronize()
        assert abs(out.item() - ref) <= tol, (seed, out.item(), ref)


@pytest.mark.parametrize("prec", [tq.TQ_C128, tq.TQ_C64])
def test_noalloc_smaller_call_after_larger_on_a_side_stream(prec):
    """A 12-qubit call (more CTAs) then an 8-qubit one (fewer), both on a
    non-default stream: the second call's reduction must not pick up the
    partials the first left past its own grid in the shared array."""
    import torch
    ctx = tq.Context(0)
    side = torch.cuda.Stream()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    tol = 1e-10 if prec == tq.TQ_C128 else 1e-6
    for (ints, ne), nq, seed in ((synth.config1(), 12, 5), (synth.config0(), 8, 6)):
        ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, tq.TQ_JW, prec)
        rp, cl, vl, dg = tq.ham_csr(ham)
        st = to_state(ctx, synth.random_state(nq, seed), nq, prec)
        ref = tq.energy(ctx, ham, st)
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            out.fill_(float("nan"))
            tq.energy_noalloc(nq, prec, rp, cl, vl, dg, st.tensor.data_ptr(), out.data_ptr(),
                              stream=side.cuda_stream)
        side.synchronize()
        assert abs(out.item() - ref) <= tol, (nq, out.item(), ref)


def test_noalloc_energy_rejects_bad_sizes():
    import torch
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.zeros(4, dtype=torch.complex128, device="cuda")
    with pytest.raises(tq.TQError) as e:
        tq.energy_noalloc(0, tq.TQ_C128, out.data_ptr(), out.data_ptr(), out.data_ptr(),
                          out.data_ptr(), st.data_ptr(), out.data_ptr())
    assert e.value.code == -1 and "n_qubits" in str(e.value)
    with pytest.raises(tq.TQError):
        tq.energy_noalloc(27, tq.TQ_C128, out.data_ptr(), out.data_ptr(), out.data_ptr(),
                          out.data_ptr(), st.data_ptr(), out.data_ptr())
