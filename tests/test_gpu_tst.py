"""Eq. 7 on the GPU against the oracle: transition-state dissociation with
the survival yield accumulated per pack."""
import math

import numpy as np
import pytest

from paper_2609_31258_b300 import workloads as W
from helpers import download, fp32_state_from_oracle, fp64_state_from_oracle, upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    from paper_2609_31258_b300 import build, mucite
    build.build()
    return mucite


@pytest.mark.parametrize("precision", [0, 1])
def test_survival_constant_teff(mc, orc, precision):
    w = W.tiny_cylinder(n_packs=2000, n_steps=0, precision=precision)
    w.fields.gas_p[:] = 0.0
    w.fields.phi_dc[:] = 0.0
    w.ion = W.IonTemplate(mass_da=1000.0, charge=1, ccs_m2=300e-20, n_atoms=100, T_init=900.0,
                          dH_kJmol=100.0, dS_JmolK=-80.0)
    w.source.z_plane = 10e-3
    ctx = mc.Context(0)
    ctx.set_tuning(1000, 128)
    mc.load_workload(ctx, w, 0)
    n = 6000
    ctx.step(0, n)
    got = download(ctx, 0, 2000)
    expect = -orc.eyring_rate(w.ion, 900.0) * n * w.run.dt
    tol = 1e-12 if precision == 1 else 2e-5
    assert np.abs(got["lnsy"] / expect - 1).max() < tol
    T = ctx.tally(0)
    assert abs(T["sum_w_sy"][0] / 2000 / math.exp(expect) - 1) < tol


def test_survival_ensemble_hot_collisions(mc, orc):
    """Ions injected hot cool in the gas while dissociating; the FP32 fused
    path follows the oracle's mean survival yield."""
    w = W.tiny_cylinder(n_packs=3000, n_steps=0, precision=0, seed=17)
    w.fields.phi_dc[:] = 0.0
    w.source.z_plane = 10e-3
    w.ion = W.IonTemplate(mass_da=556.27, charge=1, ccs_m2=1.62e-18, n_atoms=77, T_init=1100.0,
                          dH_kJmol=111.7, dS_JmolK=-38.1)
    s = orc.Sim(w)
    s.inject()
    ctx = mc.Context(0)
    ctx.set_tuning(500, 128)
    mc.load_workload(ctx, w, 0)
    upload(ctx, 0, fp32_state_from_oracle(s))
    ctx.step(0, 4000)
    got = download(ctx, 0, 3000)
    s.steps(4000)
    sy_g, sy_o = np.exp(got["lnsy"].astype(np.float64)), np.exp(s.lnsy[:3000])
    assert 0.05 < sy_o.mean() < 0.95  # the yield is exercised
    assert abs(sy_g.mean() / sy_o.mean() - 1) < 0.005
    # packs follow the oracle pack for pack until a borderline decision differs
    close = np.abs(sy_g - sy_o) < 1e-3
    assert close.mean() > 0.9


def test_fp64_survival_tracks_oracle(mc, orc):
    w = W.tiny_cylinder(n_packs=1000, n_steps=0, precision=1, seed=19)
    w.fields.phi_dc[:] = 0.0
    w.source.z_plane = 10e-3
    w.ion = W.IonTemplate(mass_da=556.27, charge=1, ccs_m2=1.62e-18, n_atoms=77, T_init=1100.0,
                          dH_kJmol=111.7, dS_JmolK=-38.1)
    s = orc.Sim(w)
    s.inject()
    ctx = mc.Context(0)
    mc.load_workload(ctx, w, 0)
    upload(ctx, 0, fp64_state_from_oracle(s))
    ctx.step(0, 300)
    got = download(ctx, 0, 1000)
    s.steps(300)
    same = np.abs(got["lnsy"] - s.lnsy[:1000]) <= 1e-9 * np.abs(s.lnsy[:1000]) + 1e-15
    assert same.mean() > 0.99
