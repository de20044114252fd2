"""Hybrid Langevin branch on the GPU against the oracle (FP32 fused path:
ensemble statistics; plain FP64 path: pack-for-pack tracking)."""
import numpy as np
import pytest
from scipy import stats

from paper_2609_31258_b300 import workloads as W
from helpers import binomial_band, download, fp32_state_from_oracle, fp64_state_from_oracle, upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    from paper_2609_31258_b300 import build, mucite
    build.build()
    return mucite


def _lv_workload(precision, n=3000, seed=31):
    w = W.tiny_cylinder(n_packs=n, n_steps=0, precision=precision, seed=seed)
    w.source.z_plane = 10e-3
    w.source.half_space = 0
    w.run.z_exit = 10.6e-3
    w.run.langevin, w.run.lv_z0, w.run.lv_z1, w.run.lv_switch = 1, 9.0e-3, 10.4e-3, 0.05
    w.ion = W.IonTemplate(mass_da=1000.0, charge=1, ccs_m2=300e-20, n_atoms=100, dH_kJmol=100.0, dS_JmolK=-80.0,
                          T_init=700.0)
    return w


def test_langevin_ensemble_fp32(mc, orc):
    w = _lv_workload(0)
    s = orc.Sim(w)
    s.inject()
    ctx = mc.Context(0)
    ctx.set_tuning(500, 128)
    mc.load_workload(ctx, w, 0)
    upload(ctx, 0, fp32_state_from_oracle(s))
    ctx.step(0, 9000)
    got = download(ctx, 0, 3000)
    s.steps(9000)
    n = 3000
    for lab in (1, 4):
        assert binomial_band((got["status"] == lab).sum(), (s.status[:n] == lab).sum(), n), lab
    assert (got["status"] == 1).sum() > 300
    a_g, a_o = got["status"] == 0, s.status[:n] == 0
    m = 1000 * W.DALTON
    ke_g = 0.5 * m * (got["vx"][a_g].astype(np.float64) ** 2 + got["vy"][a_g] ** 2 + got["vz"][a_g] ** 2)
    ke_o = 0.5 * m * (s.vx[:n][a_o] ** 2 + s.vy[:n][a_o] ** 2 + s.vz[:n][a_o] ** 2)
    assert stats.ks_2samp(ke_g, ke_o).pvalue > 0.01
    # the aggregated step neither heats nor dissociates: compare mean SY too
    sy_g, sy_o = np.exp(got["lnsy"].astype(np.float64)).mean(), np.exp(s.lnsy[:n]).mean()
    assert abs(sy_g / sy_o - 1) < 0.005


def test_langevin_fp64_tracks_oracle(mc, orc):
    w = _lv_workload(1, n=1000, seed=33)
    s = orc.Sim(w)
    s.inject()
    ctx = mc.Context(0)
    mc.load_workload(ctx, w, 0)
    upload(ctx, 0, fp64_state_from_oracle(s))
    ctx.step(0, 300)
    got = download(ctx, 0, 1000)
    s.steps(300)
    same = np.abs(got["vz"] - s.vz[:1000]) <= 1e-9 * (np.abs(s.vz[:1000]) + 1.0)
    assert same.mean() > 0.99
