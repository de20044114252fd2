"""Pins of the oracle's mask-aware Poisson solve (Phi = 0 at metal nodes).

A grounded metal tube at r >= a inside the domain makes the interior problem
the one of a grounded cylinder of radius a: a uniformly charged core then has
the closed-form potential rho (b^2 - r^2)/(4 eps0) + rho b^2 ln(a/b)/(2 eps0)
(core radius b) at mid-length, with second-order convergence; metal nodes
carry exactly zero potential and the masked system's residual is at rounding.
"""
import math

import numpy as np

from paper_2609_31258_b300 import workloads as W


def _tube_case(nr):
    from oracle import poisson
    R, L = 4e-3, 40e-3
    nz = 10 * (nr - 1) + 1
    pic = W.Grid(nr, nz, R, 0.0, L)
    dr, dz = pic.dr, pic.dz
    ka = (nr - 1) // 2          # metal for r >= a = ka dr (all z)
    kb = ka // 4                # core r <= b, b = (kb + 1/2) dr
    a, b = ka * dr, (kb + 0.5) * dr
    metal = np.zeros((nz, nr), bool)
    metal[:, ka:] = True
    rho = 1e-6
    vol = np.array([math.pi * (dr / 2) ** 2 * dz] + [2 * math.pi * i * dr * dr * dz for i in range(1, nr)])
    Q = np.tile(np.where(np.arange(nr) <= kb, rho * vol, 0.0) / poisson.Q_UNIT, (nz, 1))
    phi = poisson.solve_masked(pic, Q, metal)
    r = np.arange(nr) * dr
    ins = r <= a
    exact = np.where(r <= b, rho * (b * b - r * r) / (4 * W.EPS0) + rho * b * b * math.log(a / b) / (2 * W.EPS0),
                     rho * b * b * np.log(a / np.maximum(r, 1e-30)) / (2 * W.EPS0))
    err = np.abs(phi[nz // 2][ins] - exact[ins]).max() / exact.max()
    return err, phi, metal, pic, Q


def test_grounded_tube_closed_form_and_convergence():
    from oracle import poisson
    e1, phi, metal, pic, Q = _tube_case(17)
    e2, *_ = _tube_case(33)
    assert e1 < 3e-2 and e2 < 1e-2 and e2 < e1 / 3.0, (e1, e2)
    assert (phi[metal] == 0.0).all()
    assert poisson.residual_masked(pic, Q, phi, metal) < 1e-10


def test_pic_metal_resampling_of_ring_stack():
    from oracle import poisson
    g = W.Grid(129, 513, 5e-3, 0.0, 40e-3)
    pic = W.Grid(33, 129, 5e-3, 0.0, 40e-3)
    idx = W.ring_stack_mask(g)
    metal = poisson.pic_metal_from_static(g, idx >= 0, pic)
    # the first ring (z in [5, 5.5] mm, r >= 4 mm) appears on the PIC grid
    j = int(round(5.25e-3 / pic.dz))
    assert metal[j, -1] and not metal[j, 0]
    assert not metal[int(round(2e-3 / pic.dz))].any()
