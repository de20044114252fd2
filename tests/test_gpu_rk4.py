"""RK4 pusher, dt segments and Eq. 1 limits on the GPU against the oracle."""
import math

import numpy as np
import pytest

from paper_2609_31258_b300 import workloads as W
from helpers import download, fp32_state_from_oracle, fp64_state_from_oracle, rel_pos_error, upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    from paper_2609_31258_b300 import build, mucite
    build.build()
    return mucite


def _ring_vacuum(precision, n=1500):
    w = W.ring_stack(n_packs=n, n_steps=0, precision=precision, nr=129, nz=513, seed=41)
    w.fields.gas_p[:] = 0.0
    w.source.T_vel = 3000.0
    w.run.integrator = 1
    return w


def test_rk4_collision_free_fp32(mc, orc):
    w = _ring_vacuum(0)
    s = orc.Sim(w)
    s.inject()
    ctx = mc.Context(0)
    ctx.set_tuning(1000, 128)
    mc.load_workload(ctx, w, 0)
    upload(ctx, 0, fp32_state_from_oracle(s))
    ctx.step(0, 8000)
    got = download(ctx, 0, 1500)
    s.steps(8000)
    act = (got["status"] == 0) & (s.status[:1500] == 0)
    assert act.mean() > 0.5
    err = rel_pos_error(w.fields.grid, {k: got[k][act] for k in ("x", "y", "z")}, s.x[:1500][act],
                        s.y[:1500][act], s.z[:1500][act])
    assert err.max() < 1e-5, err.max()


def test_rk4_fp64_and_dt_segments(mc, orc):
    w = _ring_vacuum(1, n=500)
    s = orc.Sim(w)
    s.inject()
    ctx = mc.Context(0)
    mc.load_workload(ctx, w, 0)
    upload(ctx, 0, fp64_state_from_oracle(s))
    ctx.step(0, 700)
    s.steps(700)
    ctx.set_dt(0, 0.35e-9)
    s.set_dt(0.35e-9)
    ctx.step(0, 600)
    s.steps(600)
    got = download(ctx, 0, 500)
    err = rel_pos_error(w.fields.grid, got, s.x[:500], s.y[:500], s.z[:500], lattice=False)
    assert np.median(err) < 1e-12 and err.max() < 1e-9


def test_eq1_limits_match_oracle(mc, orc):
    for precision in (0, 1):
        w = W.ring_stack(n_packs=3000, n_steps=0, precision=precision, nr=129, nz=513, seed=43)
        w.run.langevin = 1
        s = orc.Sim(w)
        s.inject()
        s.steps(200)
        ctx = mc.Context(0)
        mc.load_workload(ctx, w, 0)
        st = fp32_state_from_oracle(s) if precision == 0 else fp64_state_from_oracle(s)
        upload(ctx, 0, st, step=200)
        got = ctx.dt_limits(0)
        ref = s.dt_limits()
        for k in range(6):
            if math.isinf(ref[k]):
                assert math.isinf(got[k])
            else:
                assert abs(got[k] / ref[k] - 1) < 1e-4, (k, got[k], ref[k])
        assert got[4] == 2e-9 and got[0] == pytest.approx(0.05e-6)
