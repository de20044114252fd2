"""Pins of the oracle's discrete decisions and bookkeeping: terminal
classification on hand-placed packs (geometry fixed by the workload, not by
the code), tie-breaks, tallies (conservation of represented weight and
recounts), the continuous-current accumulator of Eq. 5, source sampling
distributions and the E-from-potential differencing."""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2609_31258_b300 import workloads as W

S30 = 2 ** 30


def _ring_sim(orc):
    w = W.ring_stack(n_packs=16, n_steps=0, nr=65, nz=257)
    w.run.z_exit = 36e-3
    w.run.r_det = 2e-3
    return w, orc.Sim(w)


def _q(w, r, z, th=0.3):
    g = w.fields.grid
    x, y = r * math.cos(th), r * math.sin(th)
    return (int(round(x / g.R * S30)), int(round(y / g.R * S30)),
            int(round((z - g.z0) / (g.z1 - g.z0) * S30)))


def test_classification_hand_placed(orc):
    w, s = _ring_sim(orc)
    F = s.fields_struct()
    cases = [
        ((0.1e-3, 2e-3), W.ST_ACTIVE),          # gas, before the first ring
        ((4.5e-3, 5.25e-3), W.ST_ELECTRODE),    # inside ring 0 (r >= 4 mm)
        ((0.2e-3, 33.75e-3), W.ST_ACTIVE),      # on axis inside the last ring's bore (r_in = 1 mm)
        ((1.5e-3, 33.75e-3), W.ST_ELECTRODE),   # inside the last ring
        ((3.9e-3, 4.0e-3), W.ST_ACTIVE),        # gap region, far from metal
        ((5.2e-3, 2.0e-3), W.ST_RADIAL),        # beyond R, no metal at z = 2 mm
        ((1.0e-3, 36.5e-3), W.ST_TRANSMITTED),  # crossed the plane inside r_det
        ((3.0e-3, 36.5e-3), W.ST_AXIAL),        # crossed the plane outside r_det
        ((1.0e-3, -0.1e-3), W.ST_AXIAL),        # left through z < z0
    ]
    xq, yq, zq = zip(*[_q(w, r, z) for (r, z), _ in cases])
    st = orc.classify_fixed(F, w.run, np.array(xq), np.array(yq), np.array(zq))
    assert list(st) == [c for _, c in cases]


def test_classification_tie_breaks(orc):
    w, s = _ring_sim(orc)
    F = s.fields_struct()
    g = w.fields.grid
    zexit_q = math.ceil((w.run.z_exit - g.z0) / (g.z1 - g.z0) * S30)
    rdet_q = math.floor(w.run.r_det / g.R * S30)
    xq = np.array([rdet_q, rdet_q + 1, 100, 100, S30, S30 - 1], np.int32)
    zq = np.array([zexit_q, zexit_q, zexit_q, zexit_q - 1, 1000, 1000], np.int32)
    st = orc.classify_fixed(F, w.run, xq, np.zeros(6, np.int32), zq)
    # z == z_exit counts as crossed, r == r_det counts as transmitted, r == R is lost
    assert list(st) == [W.ST_TRANSMITTED, W.ST_AXIAL, W.ST_TRANSMITTED, W.ST_ACTIVE, W.ST_RADIAL,
                        W.ST_ACTIVE]


def test_electrode_hit_distance(orc):
    """A node next to metal is a hit when its stored distance is within the
    hit distance and not otherwise."""
    w, s = _ring_sim(orc)
    g = w.fields.grid
    d = s.dmask
    # gas node adjacent (radially) to ring 0's inner face
    j = int(round((5.25e-3 - g.z0) / g.dz))
    i_metal = np.nonzero(w.fields.mask[j])[0][0]
    i = i_metal - 1
    assert d[j, i] > 0 and abs(d[j, i] - g.dr) < 1e-9
    xq = np.array([int(round(i * g.dr / g.R * S30))], np.int32)
    zq = np.array([int(round(j * g.dz / (g.z1 - g.z0) * S30))], np.int32)
    for hit, expect in ((g.dr * 1.01, W.ST_ELECTRODE), (g.dr * 0.99, W.ST_ACTIVE)):
        w.run.hit_dist = hit
        st = orc.classify_fixed(s.fields_struct(), w.run, xq, np.zeros(1, np.int32), zq)
        assert st[0] == expect


def test_tally_conservation_and_recount(orc):
    w, s = _ring_sim(orc)
    rng = np.random.default_rng(2)
    n = 3000
    st = rng.choice([0, 1, 2, 3, 4, 255], n, p=[0.3, 0.3, 0.2, 0.1, 0.05, 0.05]).astype(np.uint8)
    xq = rng.integers(-S30 // 3, S30 // 3, n).astype(np.int32)
    yq = rng.integers(-S30 // 3, S30 // 3, n).astype(np.int32)
    zq = rng.integers(0, S30, n).astype(np.int32)
    v = rng.normal(0, 30, (3, n))
    e = rng.uniform(1e6, 3e6, n)
    tt = rng.integers(0, 80000, n).astype(np.int32)
    W_ = 1000
    w.source.weight = W_
    T = s.tally(xq, yq, zq, v[0], v[1], v[2], e, st, tt)
    for lab in range(5):
        assert T["count"][lab] == (st == lab).sum()
        assert T["weight"][lab] == W_ * (st == lab).sum()
    emitted = (st != 255).sum()
    assert T["count"][:5].sum() == emitted  # emitted = active + sum(terminal)
    tr = st == 1
    assert T["exit_hist"].sum() == W_ * tr.sum() == T["ke_hist"].sum() == T["teff_hist"].sum()
    assert T["loss_map"].sum() == W_ * (st == 2).sum()
    ref_exit = np.bincount(np.minimum(tt[tr] // w.run.exit_bin_steps, w.run.n_exit_bins - 1),
                           minlength=w.run.n_exit_bins) * W_
    assert (T["exit_hist"] == ref_exit).all()
    ke = 0.5 * w.ion.mass_da * W.DALTON * (v ** 2).sum(0) / W.E_CHARGE
    assert abs(T["sum_w_ke"][1] - W_ * ke[tr].sum()) < 1e-9 * W_ * ke[tr].sum()


def test_source_accumulator_eq5(orc):
    I, q, dt, Wt = 1e-9, 1, 0.5e-9, 1000
    acc = 0.0
    total = 0
    for chunk in (10, 10, 1000, 37, 200000):
        k, acc = orc.source_emit(I, q, dt, Wt, chunk, acc)
        total += k
    steps = 10 + 10 + 1000 + 37 + 200000
    real = I * steps * dt / (q * W.E_CHARGE)
    assert total == math.floor(real / Wt + 1e-9)
    assert abs(total * Wt + acc - real) < 1e-6 * real


def test_injection_distributions(orc):
    w = W.cylinder_space_charge(n_packs=20000, n_steps=0)
    s = orc.Sim(w)
    s.inject()
    r = np.hypot(s.x[: s.n], s.y[: s.n])
    sig, a = w.source.sigma, w.source.radius
    cdf = lambda x: -np.expm1(-x * x / (2 * sig * sig)) / -math.expm1(-a * a / (2 * sig * sig))
    assert r.max() < a
    assert stats.kstest(r, cdf).pvalue > 0.01
    assert stats.kstest(s.z[: s.n] / 20e-3, "uniform").pvalue > 0.01
    sd = math.sqrt(W.K_B * 300.0 / (1000 * W.DALTON))
    assert stats.kstest(s.vx[: s.n] / sd, "norm").pvalue > 0.01
    assert (s.vz[: s.n] >= 0).all()
    assert stats.kstest(s.vz[: s.n] / sd, stats.halfnorm.cdf).pvalue > 0.01
    w1 = W.tiny_cylinder(n_packs=20000, n_steps=0)
    s1 = orc.Sim(w1)
    s1.inject()
    r1 = np.hypot(s1.x[: s1.n], s1.y[: s1.n])
    assert stats.kstest((r1 / 1e-3) ** 2, "uniform").pvalue > 0.01  # uniform over the disc area
    assert (s1.z[: s1.n] == 0).all() and (s1.eint[: s1.n] == 3 * 100 * 300.0).all()


def test_efield_from_phi():
    import oracle
    g = W.Grid(33, 65, 2e-3, 0.0, 8e-3)
    r, z = W.node_coords(g)
    zz, rr = np.meshgrid(z, r, indexing="ij")
    phi = 3.0 * zz ** 2 - 1.5 * rr ** 2 + 7.0 * zz  # quadratic: central differences exact
    er, ez = oracle.efield_from_phi(phi, g.dr, g.dz)
    assert np.allclose(er[:, 1:-1], 3.0 * rr[:, 1:-1], rtol=1e-10, atol=1e-12)
    assert (er[:, 0] == 0).all()
    assert np.allclose(ez[1:-1], -(6.0 * zz[1:-1] + 7.0), rtol=1e-10)
    # one-sided at the edges
    assert np.allclose(ez[0], -(phi[1] - phi[0]) / g.dz)


def _teff_by_quadrature(ion, eint_over_kb):
    """T with E_int(T)/k_B = eint, E_int(T) = integral of Cv from 0 to T and
    Cv/k_B = 3N min(1, c0 + c1 T), inverted by root finding on the
    numerically integrated heat capacity (no closed form involved)."""
    from scipy import integrate, optimize
    n3 = 3.0 * ion.n_atoms
    knee = (1.0 - ion.cv_c0) / ion.cv_c1 if ion.cv_c1 > 0 else math.inf

    def E(T):
        pts = [knee] if 0.0 < knee < T else None
        return integrate.quad(lambda t: n3 * min(1.0, ion.cv_c0 + ion.cv_c1 * t), 0.0, T, points=pts,
                              epsabs=0.0, epsrel=1e-13, limit=200)[0]

    return np.array([optimize.brentq(lambda T: E(T) - e, 0.0, 1e5, xtol=1e-12, rtol=1e-14) for e in eint_over_kb])


def _bins_fp64(x, n):
    """floor(x * n) clamped to [0, n-1], with a flag for values within 1e-6
    (relative to one bin) of a bin edge, where the FP32/FP64 decision of the
    oracle may fall on either side."""
    y = np.asarray(x, np.float64) * n
    b = np.clip(np.floor(y), 0, n - 1).astype(np.int64)
    near = np.abs(y - np.rint(y)) < 1e-6
    return b, near


def test_tally_histogram_bins_recounted(orc):
    """Every bin of the exit-radius, KE, T_eff and loss-map histograms,
    recounted from the physical definitions in FP64: r in [0, r_det) over
    n_r bins, KE = M v^2 / 2 in [0, ke_max) eV, T_eff (the temperature whose
    integrated heat capacity is E_int) in [0, teff_max), and the loss map
    over r in [0, R) x z in [z0, z1); values beyond the range land in the last
    bin. A wrong bin scale, offset or axis swap fails here even though the
    totals are unchanged (Eq. 8 and the terminal-event observables of the
    Methods' terminal-events section)."""
    w, s = _ring_sim(orc)
    g, run, ion = w.fields.grid, w.run, w.ion
    rng = np.random.default_rng(11)
    n = 4000
    st = rng.choice([1, 2], n, p=[0.6, 0.4]).astype(np.uint8)
    # radius: transmitted packs over [0, 1.15 r_det], electrode hits over [0, R)
    r = np.where(st == 1, rng.uniform(0, 1.15 * run.r_det, n), rng.uniform(0, 0.999 * g.R, n))
    th = rng.uniform(0, 2 * math.pi, n)
    xq = np.rint(r * np.cos(th) / g.R * S30).astype(np.int32)
    yq = np.rint(r * np.sin(th) / g.R * S30).astype(np.int32)
    zq = rng.integers(0, S30, n).astype(np.int32)
    M = ion.mass_da * W.DALTON
    ke = rng.uniform(0, 1.15 * run.ke_max_ev, n)
    sp = np.sqrt(2.0 * ke * W.E_CHARGE / M)
    u = rng.normal(size=(3, n))
    u /= np.linalg.norm(u, axis=0)
    v = sp * u
    e = rng.uniform(0.0, 1.2 * 3.0 * ion.n_atoms * (run.teff_max - 350.0), n)
    tt = rng.integers(0, 80000, n).astype(np.int32)
    W_ = 7
    w.source.weight = W_
    T = s.tally(xq, yq, zq, v[0], v[1], v[2], e, st, tt)

    tr, lo = st == 1, st == 2
    r_lat = np.hypot(xq.astype(np.float64), yq.astype(np.float64)) * g.R / S30  # radius the lattice encodes
    ke_v = 0.5 * M * (v ** 2).sum(0) / W.E_CHARGE
    te = _teff_by_quadrature(ion, e[tr])
    checks = [("r_hist", r_lat[tr] / run.r_det, run.n_r_bins),
              ("ke_hist", ke_v[tr] / run.ke_max_ev, run.n_ke_bins),
              ("teff_hist", te / run.teff_max, run.n_teff_bins)]
    for name, x, nb in checks:
        b, near = _bins_fp64(x, nb)
        ref = np.bincount(b, minlength=nb) * W_
        got = T[name]
        assert got.sum() == ref.sum() == W_ * tr.sum(), name
        if not near.any():
            assert (got == ref).all(), (name, np.nonzero(got != ref)[0][:8])
        else:  # a value on an edge may fall on either side
            assert np.abs(got - ref).sum() <= 2 * W_ * near.sum(), name
        assert (np.bincount(b, minlength=nb) > 0).sum() >= nb - 1, name  # every bin exercised
    br, nr_ = _bins_fp64(r_lat[lo] / g.R, run.n_loss_r)
    zf = zq[lo].astype(np.float64) / S30  # (z - z0) / (z1 - z0) on the lattice
    bz, nz_ = _bins_fp64(zf, run.n_loss_z)
    ref = np.zeros(run.n_loss_z * run.n_loss_r, np.int64)
    np.add.at(ref, bz * run.n_loss_r + br, W_)
    near = nr_ | nz_
    got = np.asarray(T["loss_map"]).reshape(-1)  # [z bin][r bin]
    assert got.sum() == ref.sum()
    assert np.abs(got - ref).sum() <= 2 * W_ * near.sum()
    if not near.any():
        assert (got == ref).all()
