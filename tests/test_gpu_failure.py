"""Failure detection on the GPU without a GPU fault: the staged streaming
kernel's waits for its state copies are bounded (about 0.25 s of wall-clock
time each). The C-ABI test hook makes one launch withhold the copies of a
tile per block, so nothing ever completes those waits; the kernel must end
by itself, report the waits that gave up (mucite_tally returns
MUCITE_E_TIMEOUT), and leave the context usable once the instance is
resumed."""
import time

import pytest

from paper_2609_31258_b300 import workloads as W

pytestmark = pytest.mark.gpu


def test_withheld_staged_copy_times_out_and_context_recovers():
    import torch
    from paper_2609_31258_b300 import build, mucite
    build.build()
    n = 5000
    w = W.ring_stack(n_packs=n, n_steps=0, seed=3, precision=0, nr=129, nz=513)
    w.fields.gas_p[:] = 0.0  # collision-free: single steps take the staged streaming kernel
    ctx = mucite.Context(0)
    ctx.set_tuning(1, 256)
    mucite.load_workload(ctx, w, 0)
    ctx.step(0, 3)
    T0 = ctx.tally(0)
    assert T0["pack_steps"] == 3 * n
    ctx.test_hook(mucite.HOOK_HOLD_STAGED_COPY, 0)
    t0 = time.perf_counter()
    ctx.step(0, 1)
    with pytest.raises(mucite.MuciteError) as e:
        ctx.tally(0)
    assert e.value.status == mucite.E_TIMEOUT
    assert time.perf_counter() - t0 < 30.0  # the waits are bounded
    # the hook acts on one launch; after a resume (counters reset) the
    # context steps and tallies again
    ctx.resume(0, n, T0["step"] + 1)
    ctx.step(0, 4)
    T = ctx.tally(0)
    assert T["pack_steps"] > 0 and T["step"] == T0["step"] + 5
    with pytest.raises(mucite.MuciteError) as e:
        ctx.test_hook(99, 0)
    assert e.value.status == mucite.E_ARG
    torch.cuda.synchronize()
    ctx.close()
