"""Pins of the oracle's transition-state dissociation (Eq. 7).

- Eyring rate: k(T) = (k_B T / h) exp(dS/R) exp(-dH/(R T)); its Arrhenius
  form gives d ln(k/T) / d(1/T) = -dH/R exactly and k/T at 1/T -> 0 equal to
  (k_B/h) exp(dS/R);
- with collisions off and a fixed E_int, T_eff is constant and the survival
  yield is exactly exp(-k t) after t = n dt;
- with the paper's Table S3 templates at 300 K the yield stays ~1 (the
  activation barrier is far above k_B T).
"""
import json
import math
import os

import numpy as np

from paper_2609_31258_b300 import workloads as W

H = 6.62607015e-34
R = W.K_B * 6.02214076e23


def test_eyring_arrhenius_form(orc):
    ion = W.IonTemplate(mass_da=556.27, charge=1, ccs_m2=1.62e-18, n_atoms=77, dH_kJmol=111.7,
                        dS_JmolK=-38.1)
    T1, T2 = 600.0, 900.0
    k1, k2 = orc.eyring_rate(ion, T1), orc.eyring_rate(ion, T2)
    slope = (math.log(k2 / T2) - math.log(k1 / T1)) / (1 / T2 - 1 / T1)
    assert abs(slope / (-111.7e3 / R) - 1) < 1e-12
    pre = (k1 / T1) * math.exp(111.7e3 / (R * T1))
    assert abs(pre / ((W.K_B / H) * math.exp(-38.1 / R)) - 1) < 1e-12
    off = W.IonTemplate(mass_da=556.27, charge=1, ccs_m2=1.62e-18, n_atoms=77)
    assert orc.eyring_rate(off, 800.0) == 0.0


def test_survival_closed_form_constant_teff(orc):
    w = W.tiny_cylinder(n_packs=64, n_steps=0)
    w.fields.gas_p[:] = 0.0                      # no collisions: E_int and T_eff stay fixed
    w.fields.phi_dc[:] = 0.0
    w.ion = W.IonTemplate(mass_da=1000.0, charge=1, ccs_m2=300e-20, n_atoms=100, T_init=900.0,
                          dH_kJmol=100.0, dS_JmolK=-80.0)
    w.source.z_plane = 10e-3
    s = orc.Sim(w)
    s.inject()
    n = 5000
    s.steps(n)
    k = orc.eyring_rate(w.ion, 900.0)
    expect = -k * n * w.run.dt
    act = s.status[:64] == 0
    assert act.all()
    assert np.allclose(s.lnsy[:64], expect, rtol=1e-10)
    T = s.tally()
    assert abs(T["sum_w_sy"][0] / 64 - math.exp(expect)) < 1e-12


def test_table_s3_templates_stable_at_room_temperature(orc):
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table_s3_ion_templates.json")))
    for t in gold["templates"].values():
        ion = W.IonTemplate(mass_da=t["mass_da"], charge=t["charge"], ccs_m2=t["ccs_m2"], n_atoms=t["n_atoms"],
                            dH_kJmol=t["dH_kJ_per_mol"], dS_JmolK=t["dS_J_per_mol_K"])
        # over the paper's 4 ms runs at T_eff = 300 K almost nothing dissociates
        assert orc.eyring_rate(ion, 300.0) * 4e-3 < 1e-6
