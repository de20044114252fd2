"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (2000 fused micro steps per launch, 256 threads per block).

- ring stack 512 x 2048, 100,000 packs of 15 kDa/+8: the oracle injects and
  advances every pack (packs are independent without space charge); the GPU
  path starts from the same state; compared pack by pack (status agreement,
  close trajectories for the packs whose random decisions agree) and as
  ensembles (KS on KE and T_eff, mean T_eff within 0.5 %);
- cylinder with space charge, 1,000,000 packs prefilled: the int64 deposit on
  the 256 x 1024 PIC grid is bit-exact and the solve meets the 1e-6 residual
  on the oracle's operator.
"""
import numpy as np
import pytest
from scipy import stats

from paper_2609_31258_b300 import workloads as W
from helpers import download, fp32_state_from_oracle, rel_pos_error, upload

pytestmark = pytest.mark.gpu


def test_ring_stack_full_size(orc):
    from paper_2609_31258_b300 import build, mucite
    build.build()
    n = 100_000
    w = W.ring_stack(n_packs=n, n_steps=0, seed=1, precision=0)
    s = orc.Sim(w)
    s.inject()
    st = fp32_state_from_oracle(s)
    ctx = mucite.Context(0)
    ctx.set_tuning(2000, 256)
    mucite.load_workload(ctx, w, 0)
    upload(ctx, 0, st)
    ctx.step(0, 2000)
    got = download(ctx, 0, n)
    s.steps(2000)
    T = ctx.tally(0)
    assert T["candidate_overflow"] == 0
    assert abs(T["pack_steps"] / int(s.nsteps[:n].sum()) - 1) < 1e-3
    same_status = got["status"] == s.status[:n]
    assert same_status.mean() > 0.999
    err = rel_pos_error(w.fields.grid, {k: got[k] for k in ("x", "y", "z")}, s.x[:n], s.y[:n], s.z[:n])
    assert np.median(err) < 1e-5
    m = w.ion.mass_da * W.DALTON
    a = (got["status"] == 0) & (s.status[:n] == 0)
    ke_g = 0.5 * m * (got["vx"][a].astype(np.float64) ** 2 + got["vy"][a] ** 2 + got["vz"][a] ** 2)
    ke_o = 0.5 * m * (s.vx[:n][a] ** 2 + s.vy[:n][a] ** 2 + s.vz[:n][a] ** 2)
    assert stats.ks_2samp(ke_g, ke_o).pvalue > 0.01
    Tg = np.array([orc.T_of_eint(w.ion, e) for e in got["eint"][a][::10].astype(np.float64)])
    To = np.array([orc.T_of_eint(w.ion, e) for e in s.eint[:n][a][::10]])
    assert stats.ks_2samp(Tg, To).pvalue > 0.01
    assert abs(Tg.mean() / To.mean() - 1) < 0.005
    ctx.close()


def test_space_charge_full_size_deposit_and_solve(orc):
    from oracle import poisson
    from paper_2609_31258_b300 import build, mucite
    build.build()
    n = 1_000_000
    w = W.cylinder_space_charge(n_packs=n, n_steps=0, precision=0)
    s = orc.Sim(w)
    s.inject()
    ctx = mucite.Context(0)
    mucite.load_workload(ctx, w, 0)
    upload(ctx, 0, fp32_state_from_oracle(s))
    ctx.pic_update(0)
    got = ctx.pic_read(0)
    Q = s.deposit()
    assert (got["Q"] == Q).all()
    assert Q.sum() == n * w.source.weight * 2 ** 30
    # the paper's Poisson tolerance (Table S2: rtol 1e-6), on the residual the
    # library reports and on the oracle's own recomputation of it from the
    # returned potential; the two are the same quantity in FP64
    res = poisson.residual(w.fields.pic, Q, got["phi"])
    assert got["rel_residual"] <= 1e-6 and res <= 1e-6, (got["rel_residual"], res)
    assert abs(res - got["rel_residual"]) <= 1e-3 * res + 1e-12, (got["rel_residual"], res)
    ctx.close()


@pytest.mark.parametrize("graphs", [False, True])
def test_space_charge_every_update_meets_tolerance(orc, graphs):
    """Cylinder with space charge at the benchmark's size (1e6 packs, 256 x
    1024 PIC grid every 10 micro steps), 300 micro steps: every warm-started
    solve that can be read back -- each update when issued directly, the
    second of every two when two macro steps are replayed as graphs -- meets
    the paper's 1e-6 tolerance, on the residual the library reports and on the
    oracle's FP64 recomputation from the returned potential and charge. The
    solves start from the last two solutions extrapolated in time and take one
    correction pass once that start exists (at most two at any update)."""
    import torch
    from oracle import poisson
    from paper_2609_31258_b300 import build, mucite
    build.build()
    w = W.cylinder_space_charge(n_packs=1_000_000, n_steps=0, precision=0)
    ctx = mucite.Context(0, torch.cuda.Stream())
    ctx.set_launch_mode(0, graphs)
    mucite.load_workload(ctx, w, 0)
    per_call = 20 if graphs else 10
    passes = []
    for call in range(300 // per_call):
        ctx.step(0, per_call)
        got = ctx.pic_read(0)
        res = poisson.residual(w.fields.pic, got["Q"], got["phi"])
        assert got["rel_residual"] <= 1e-6 and res <= 1e-6, (call, got["rel_residual"], res)
        assert abs(res - got["rel_residual"]) <= 1e-3 * res + 1e-12, (call, got["rel_residual"], res)
        passes.append(got["iterations"])
    ctx.close()
    assert max(passes[2:]) <= 2, passes
    assert sum(p == 1 for p in passes[2:]) >= 0.8 * len(passes[2:]), passes
