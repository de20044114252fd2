"""Pins of the oracle's space-charge cycle (CIC deposit + finite-volume
cylindrical Poisson + E differencing) against closed forms:

- uniformly charged infinite cylinder inside a grounded tube (mid-plane of a
  long domain): Phi = rho (a^2 - r^2)/(4 eps0) + rho a^2 ln(R/a)/(2 eps0)
  inside, rho a^2 ln(R/r)/(2 eps0) outside; second-order convergence;
- ring charges in a grounded cylinder with grounded end caps: the Fourier-
  Bessel Green's function summed over N <= 200 charges (brute force);
- deposit invariants: total charge, first radial/axial moments.
"""
import math

import numpy as np
import pytest
from scipy import special

from paper_2609_31258_b300 import workloads as W

EPS0 = W.EPS0


def _cyl_error(nr, a_cells=None):
    from oracle import poisson
    R, L = 2e-3, 40e-3
    nz = 8 * (nr - 1) * 5 + 1  # dz = dr, L = 20 R
    pic = W.Grid(nr, nz, R, 0.0, L)
    dr, dz = pic.dr, pic.dz
    k = (nr - 1) // 4          # a = (k + 1/2) dr: control volumes align with r = a
    a = (k + 0.5) * dr
    rho = 1e-6                 # C/m^3
    vol = np.array([math.pi * (dr / 2) ** 2 * dz] + [2 * math.pi * i * dr * dr * dz for i in range(1, nr)])
    Qrow = np.where(np.arange(nr) <= k, rho * vol, 0.0) / poisson.Q_UNIT
    Q = np.tile(Qrow, (nz, 1))
    phi = poisson.solve(pic, Q)
    r = np.arange(nr) * dr
    exact = np.where(r <= a, rho * (a * a - r * r) / (4 * EPS0) + rho * a * a * math.log(R / a) / (2 * EPS0),
                     rho * a * a * np.log(R / np.maximum(r, 1e-30)) / (2 * EPS0))
    mid = phi[nz // 2]
    return np.abs(mid - exact).max() / exact.max(), poisson.residual(pic, Q, phi)


def test_uniform_cylinder_closed_form():
    e1, res1 = _cyl_error(17)
    e2, res2 = _cyl_error(33)
    assert e1 < 1e-2 and e2 < 3e-3, (e1, e2)
    assert e2 < e1 / 3.0  # second order
    assert res1 < 1e-10 and res2 < 1e-10


def _green_ring(r, z, rp, zp, q, R, L, nterms=400):
    """Potential at (r, z) of a ring charge q at (rp, zp) in a grounded
    cylinder of radius R, 0 <= z <= L, grounded ends."""
    n = np.arange(1, nterms + 1)[:, None]
    k = n * math.pi / L
    rl, rg = np.minimum(r, rp), np.maximum(r, rp)
    t1 = special.i0e(k * rl) * special.k0e(k * rg) * np.exp(k * (rl - rg))
    t2 = special.k0e(k * R) * special.i0e(k * rg) * special.i0e(k * rl) / special.i0e(k * R) * \
        np.exp(k * (rg + rl - 2 * R))
    terms = q / (math.pi * L * EPS0) * np.sin(k * zp) * np.sin(k * z) * (t1 - t2)
    return terms.sum(0)


@pytest.mark.parametrize("npart", [1, 200])
def test_ring_green_function_vs_pic(orc, npart):
    from oracle import poisson
    R, L = 2e-3, 8e-3
    pic = W.Grid(65, 257, R, 0.0, L)
    rng = np.random.default_rng(17 + npart)
    rp = rng.uniform(0.0, 0.6e-3, npart) if npart > 1 else np.array([0.4e-3])
    th = rng.uniform(0, 2 * math.pi, npart)
    zp = rng.uniform(3.5e-3, 4.5e-3, npart) if npart > 1 else np.array([4.0e-3])
    x, y = rp * np.cos(th), rp * np.sin(th)
    xq, yq, zq = orc.quantize(R, 0.0, L, x, y, zp)
    qw = 1000
    Q = orc.deposit_fixed(pic, xq, yq, zq, np.zeros(npart, np.uint8), qw)
    phi = poisson.solve(pic, Q)
    rn, zn = W.node_coords(pic)
    # evaluation nodes at least 1.2 mm away from the charge cloud
    jj = np.nonzero((np.abs(zn - 4e-3) > 1.7e-3) & (zn > 0.5e-3) & (zn < L - 0.5e-3))[0][::8]
    ii = np.arange(0, pic.nr - 4, 6)
    rr, zz = np.meshgrid(rn[ii], zn[jj])
    ref = np.zeros(rr.size)
    for p in range(npart):
        rq = math.hypot(xq[p] * R / 2 ** 30, yq[p] * R / 2 ** 30)
        ref += _green_ring(rr.reshape(-1), zz.reshape(-1), rq, zq[p] * L / 2 ** 30, qw * W.E_CHARGE, R, L)
    got = phi[np.ix_(jj, ii)].reshape(-1)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < 0.02, err


def test_deposit_invariants(orc):
    pic = W.Grid(33, 65, 2e-3, 0.0, 8e-3)
    rng = np.random.default_rng(5)
    n = 500
    xq = rng.integers(-(2 ** 30) // 2, 2 ** 30 // 2, n).astype(np.int32)
    yq = rng.integers(-(2 ** 30) // 2, 2 ** 30 // 2, n).astype(np.int32)
    zq = rng.integers(0, 2 ** 30, n).astype(np.int32)
    st = np.zeros(n, np.uint8)
    st[::7] = 1  # terminal packs deposit nothing
    qw = 8 * 1000
    Q = orc.deposit_fixed(pic, xq, yq, zq, st, qw)
    act = st == 0
    assert Q.sum() == qw * 2 ** 30 * act.sum()
    assert (Q >= 0).all()
    # first moments: CIC reproduces r and z to the 15-bit fraction resolution
    r = np.floor(np.sqrt(xq.astype(np.float64) ** 2 + yq.astype(np.float64) ** 2))
    ri = np.arange(pic.nr)[None, :] * (2 ** 30 / (pic.nr - 1))
    zj = np.arange(pic.nz)[:, None] * (2 ** 30 / (pic.nz - 1))
    m_r = (Q * ri).sum() / (qw * 2 ** 30)
    m_z = (Q * zj).sum() / (qw * 2 ** 30)
    cell_r, cell_z = 2 ** 30 / (pic.nr - 1), 2 ** 30 / (pic.nz - 1)
    assert abs(m_r - r[act].sum()) < act.sum() * cell_r * 2 ** -14
    assert abs(m_z - zq[act].astype(np.float64).sum()) < act.sum() * cell_z * 2 ** -14
    # a pack exactly on a node deposits everything there
    Q1 = orc.deposit_fixed(pic, np.array([0], np.int32), np.array([0], np.int32),
                           np.array([(2 ** 30 // (pic.nz - 1)) * 0], np.int32), np.zeros(1, np.uint8), 3)
    assert Q1[0, 0] == 3 * 2 ** 30 and Q1.sum() == 3 * 2 ** 30
