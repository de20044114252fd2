"""Pins of the oracle's hybrid Langevin branch (Methods: "optional hybrid
Langevin branch"; Table S2: switch at lambda dt >= 0.05).

- stationary state: ion velocities Maxwellian at the gas temperature;
- drift: mean axial velocity K E with the Mason-Schamp low-field mobility;
- explicit vs hybrid: the same transmission within binomial noise (the
  paper's explicit-vs-hybrid cross-check of Table 1, on synthetic fields);
- T_eff is not updated inside the window; outside it collisions stay explicit.
"""
import math

import numpy as np
from scipy import stats

from paper_2609_31258_b300 import workloads as W

KB, E, DA = W.K_B, W.E_CHARGE, W.DALTON


def _box(Ez=0.0, langevin=1, n_packs=2000, seed=3, T_init=300.0, window=(0.0, 20e-3)):
    w = W.tiny_cylinder(n_packs=n_packs, n_steps=0, seed=seed)
    w.fields = W.uniform_axial_fields(w.fields.grid, Ez=Ez, p=200.0)
    w.source.z_plane = 10e-3
    w.source.half_space = 0
    w.ion = W.IonTemplate(mass_da=1000.0, charge=1, ccs_m2=300e-20, n_atoms=100, T_init=T_init)
    w.run.langevin, w.run.lv_z0, w.run.lv_z1, w.run.lv_switch = langevin, window[0], window[1], 0.05
    return w


def _K():
    N = 200.0 / (KB * 300.0)
    mu = 1000 * 28 / 1028 * DA
    return 3 * E / (16 * N) * math.sqrt(2 * math.pi / (mu * KB * 300.0)) / 300e-20


def test_langevin_stationary_maxwellian_and_frozen_teff(orc):
    w = _box(T_init=500.0)
    s = orc.Sim(w)
    s.inject()
    e0 = s.eint[: s.n].copy()
    s.steps(6000)
    sd = math.sqrt(KB * 300.0 / (1000 * DA))
    assert stats.kstest(s.vx[: s.n] / sd, "norm").pvalue > 0.01
    assert stats.kstest(s.vz[: s.n] / sd, "norm").pvalue > 0.01
    assert (s.eint[: s.n] == e0).all()          # T_eff not updated by the aggregated step
    assert s.ncoll[: s.n].sum() == 0


def test_langevin_drift_is_mobility_times_field(orc):
    w = _box(Ez=2000.0)
    s = orc.Sim(w)
    s.inject()
    s.steps(3000)
    za = s.z[: s.n].copy()
    s.steps(12000)
    act = s.status[: s.n] == 0
    vd = (s.z[: s.n][act] - za[act]).mean() / (12000 * w.run.dt)
    assert abs(vd / (_K() * 2000.0) - 1) < 0.01, vd


def test_explicit_vs_hybrid_transmission(orc):
    res = []
    for lv in (0, 1):
        w = _box(Ez=2000.0, langevin=lv, n_packs=3000, seed=23)
        w.run.z_exit = 10.6e-3
        s = orc.Sim(w)
        s.inject()
        s.steps(9000)
        res.append((s.status[: s.n] == W.ST_TRANSMITTED).sum())
    n = 3000
    p = 0.5 * (res[0] + res[1]) / n
    assert 0.2 < p < 0.8
    assert abs(res[0] - res[1]) / n < 3 * math.sqrt(2 * p * (1 - p) / n), res


def test_window_and_switch(orc):
    # window away from the packs: collisions stay explicit
    w = _box(window=(15e-3, 20e-3))
    s = orc.Sim(w)
    s.inject()
    s.steps(500)
    assert s.ncoll[: s.n].sum() > 0
    # switch threshold above the local lambda dt (~0.07): explicit as well
    w = _box()
    w.run.lv_switch = 0.5
    s = orc.Sim(w)
    s.inject()
    s.steps(500)
    assert s.ncoll[: s.n].sum() > 0
