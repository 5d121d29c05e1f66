"""Failure detection on the GPU without a fault: a bounded wait that runs out.

The XOR-ELL energy pass waits on shared-memory copy barriers with a time
limit.  With the test flag set its producer never copies the first chunk,
so the consumers' waits run out; the call must come back with TQ_ETIMEOUT
(not hang, not fault), and the same context must then give the normal
energy again.
"""

import time

import pytest

import paper_2606_29692_gb300 as tq
import synth

pytestmark = pytest.mark.gpu


def test_withheld_chunk_times_out_and_the_context_recovers():
    ctx = tq.Context(0)
    ints, ne = synth.config1()
    for prec in (tq.TQ_C64, tq.TQ_C128):
        ham = tq.build_hamiltonian(ctx, ints.h, ints.g, 0.0, 1, prec)
        st = tq.State(ctx, 12, prec)
        tq.state_set_hf(st, ne, 1)
        ctx.set_spmv_schedule(tq.TQ_SPMV_XELL)
        E0 = tq.energy(ctx, ham, st)
        ctx.set_test_flags(tq.TQ_TEST_WITHHOLD_CHUNK)
        t0 = time.monotonic()
        with pytest.raises(tq.TQError) as err:
            tq.energy(ctx, ham, st)
        dt = time.monotonic() - t0
        assert err.value.code == -4                       # TQ_ETIMEOUT
        assert 1.0 < dt < 30.0                            # the bound, not a hang
        ctx.set_test_flags(0)
        assert tq.energy(ctx, ham, st) == E0              # the context is still usable
        ctx.set_spmv_schedule(tq.TQ_SPMV_XELL)
    with pytest.raises(tq.TQError):
        ctx.set_test_flags(8)
