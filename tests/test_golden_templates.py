"""The paper's two ion templates (Table S3) at the stage pressures of the
Experiments section: the oracle's thermalised collision rate against
n sigma sqrt(8kT/(pi mu)) and the equilibrium T_eff, with the classical heat
capacity standing in for the unpublished "drags"/"peptide" profiles."""
import json
import math
import os

import numpy as np
import pytest

from paper_2609_31258_b300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table_s3_ion_templates.json")))


@pytest.mark.parametrize("name", sorted(GOLD["templates"]))
def test_table_s3_template_thermal_rate(orc, name):
    t = GOLD["templates"][name]
    ion = W.IonTemplate(mass_da=t["mass_da"], charge=t["charge"], ccs_m2=t["ccs_m2"], n_atoms=t["n_atoms"],
                        T_init=t["T_init_K"])
    w = W.tiny_cylinder(n_packs=1500, n_steps=0, seed=21)
    w.fields = W.uniform_axial_fields(w.fields.grid, Ez=0.0, p=t["stage_pressure_Pa"])
    w.source.z_plane, w.source.half_space = 10e-3, 0
    w.ion = ion
    s = orc.Sim(w)
    s.inject()
    s.steps(3000)
    c0, n0 = s.ncoll.sum(), s.nsteps.sum()
    s.steps(6000)
    rate = (s.ncoll.sum() - c0) / (s.nsteps.sum() - n0) / w.run.dt
    mu = t["mass_da"] * 28.0 / (t["mass_da"] + 28.0) * W.DALTON
    n = t["stage_pressure_Pa"] / (W.K_B * 300.0)
    expect = n * t["ccs_m2"] * math.sqrt(8 * W.K_B * 300.0 / (math.pi * mu))
    assert abs(rate / expect - 1) < 0.02, (rate, expect)
    T = np.array([orc.T_of_eint(ion, e) for e in s.eint[: s.n]])
    assert abs(T.mean() / 300.0 - 1) < 0.01
