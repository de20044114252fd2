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


def test_rk4_is_the_integrator_applied(mc, orc):
    """The FP32 path with RK4 selected (and neither Eq. 7 nor the Langevin
    branch) follows the oracle's RK4 and not its leapfrog: at dt = 5 ns (200
    steps per RF period) the two integrators separate well beyond the FP32
    tolerance."""
    import dataclasses
    w = _ring_vacuum(0, n=1000)
    w.run.dt = 5e-9
    s = orc.Sim(w)
    s.inject()
    st = fp32_state_from_oracle(s)
    lf = orc.Sim(dataclasses.replace(w, run=dataclasses.replace(w.run, integrator=0)))
    lf.inject()
    fp32_state_from_oracle(lf)
    ctx = mc.Context(0)
    ctx.set_tuning(500, 128)
    mc.load_workload(ctx, w, 0)
    upload(ctx, 0, st)
    ctx.step(0, 2000)
    got = download(ctx, 0, 1000)
    s.steps(2000)
    lf.steps(2000)
    act = (got["status"] == 0) & (s.status[:1000] == 0) & (lf.status[:1000] == 0)
    assert act.mean() > 0.5
    pos = {k: got[k][act] for k in ("x", "y", "z")}
    e_rk4 = rel_pos_error(w.fields.grid, pos, s.x[:1000][act], s.y[:1000][act], s.z[:1000][act])
    e_lf = rel_pos_error(w.fields.grid, pos, lf.x[:1000][act], lf.y[:1000][act], lf.z[:1000][act])
    assert np.median(e_rk4) < 1e-5, np.median(e_rk4)
    assert np.median(e_lf) > 10 * np.median(e_rk4), (np.median(e_lf), np.median(e_rk4))
