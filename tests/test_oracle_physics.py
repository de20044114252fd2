"""Pins of the oracle's push and collision physics against closed forms.

- uniform field, no gas: leapfrog positions follow the exact discrete parabola;
- static DC field, no gas: kinetic + potential energy conserved;
- RF ring guide (Dehmelt): radial secular frequency from the pseudopotential,
  axial secular frequency twice the radial one;
- collision rate at a frozen ion velocity: n sigma gbar(w), with gbar the mean
  relative speed against a Maxwellian (closed form with erf);
- optical depth carried across steps: at frozen velocities the accepted
  events of each pack over many steps are Poisson with mean
  n sigma gbar(w) N dt (mean and dispersion across packs);
- thermalised ions: collision rate n sigma sqrt(8kT/(pi mu));
- low-field drift: Mason-Schamp mobility K = (3q/16N) sqrt(2 pi/(mu k T))/sigma;
- internal temperature relaxes to the gas temperature; E_int equilibrium
  distribution Gamma(3N, k T) for the classical heat capacity.
"""
import math

import numpy as np
import pytest
from scipy import special, stats

from paper_2609_31258_b300 import workloads as W

KB, E, DA = W.K_B, W.E_CHARGE, W.DALTON


def _vacuum(w):
    f = w.fields
    f.gas_p[:] = 0.0
    return w


def test_uniform_field_parabola(orc):
    w = _vacuum(W.tiny_cylinder(n_packs=50, n_steps=0))
    s = orc.Sim(w)
    s.inject()
    x0, z0, vz0, vx0 = s.x[:50].copy(), s.z[:50].copy(), s.vz[:50].copy(), s.vx[:50].copy()
    n = 3000
    s.steps(n)
    a = E / (1000 * DA) * 2000.0
    dt = w.run.dt
    # v stored at half steps: z_n = z_0 + n dt v0 + a dt^2 n(n+1)/2
    zexp = z0 + n * dt * vz0 + a * dt * dt * n * (n + 1) / 2
    act = s.status[:50] == 0
    assert act.sum() > 40
    assert np.allclose(s.z[:50][act], zexp[act], rtol=1e-12, atol=1e-15)
    assert np.allclose(s.x[:50][act], x0[act] + n * dt * vx0[act], rtol=1e-12, atol=1e-15)


def test_energy_conservation_static_dc(orc):
    """Collision-free motion in the ring-stack DC field: kinetic + potential
    energy at integer steps (kinetic from the mean of the two half-step
    velocities) stays within a small fraction of one ring's potential step."""
    g = W.Grid(65, 257, 5e-3, 0.0, 40e-3)
    w = W.ring_stack(n_packs=64, n_steps=0, nr=65, nz=257)
    w.fields.gas_p[:] = 0.0
    w.run.v_rf = 0.0
    w.run.dt = 2e-9
    w.source.z_plane = 12e-3
    w.source.radius = 1.0e-3
    w.source.T_vel = 3000.0
    s = orc.Sim(w)
    s.inject()
    m, q = w.ion.mass_da * DA, w.ion.charge * E
    from scipy.interpolate import RegularGridInterpolator
    r_n, z_n = W.node_coords(g)
    phi = RegularGridInterpolator((z_n, r_n), w.fields.phi_dc * w.run.dc_scale, method="cubic")
    vel = lambda: np.stack([s.vx[:64], s.vy[:64], s.vz[:64]]).copy()
    energies = []
    for k in range(40):
        xk, yk, zk, v_minus = s.x[:64].copy(), s.y[:64].copy(), s.z[:64].copy(), vel()
        s.steps(1)
        v = 0.5 * (v_minus + vel())
        energies.append(0.5 * m * (v ** 2).sum(0) + q * phi(np.stack([zk, np.hypot(xk, yk)], -1)))
        s.steps(249)
    alive = s.status[:64] == 0
    e = np.array(energies)[:, alive]
    swing = q * w.run.dc_scale  # one ring's potential step
    drift = np.abs(e - e[0]).max(0)
    assert alive.sum() > 10
    assert np.median(drift) < 0.02 * swing, (np.median(drift), swing)


def _dehmelt_setup(nr=129, nz=513, Rmax=2e-3, half=4e-3, z0l=2e-3, r0=1e-3):
    g = W.Grid(nr, nz, Rmax, -half, half)
    r, z = W.node_coords(g)
    zz, rr = np.meshgrid(z, r, indexing="ij")
    phi = special.i0(rr / z0l) * np.cos(zz / z0l) / special.i0(r0 / z0l)
    zero = np.zeros_like(phi)
    f = W.Fields(g, zero.copy(), phi, zero.copy(), np.full_like(phi, 300.0), zero.copy(), zero.copy(),
                 np.zeros(phi.shape, np.uint8), np.full_like(phi, 1.0))
    return g, f


def _secular_frequency(t, x, T_rf):
    k = max(1, int(round(T_rf / (t[1] - t[0]))))
    xs = np.convolve(x, np.ones(k) / k, mode="valid")
    ts = t[: xs.size] + 0.5 * (k - 1) * (t[1] - t[0])
    sgn = np.signbit(xs)
    idx = np.nonzero(sgn[1:] != sgn[:-1])[0]
    tc = ts[idx] - xs[idx] * (ts[idx + 1] - ts[idx]) / (xs[idx + 1] - xs[idx])
    return math.pi / np.mean(np.diff(tc))


@pytest.mark.parametrize("axis", ["r", "z"])
def test_dehmelt_secular_frequency(orc, axis):
    z0l, r0 = 2e-3, 1e-3
    g, f = _dehmelt_setup(z0l=z0l, r0=r0)
    ion = W.IonTemplate(mass_da=1000.0, charge=1, ccs_m2=0.0, n_atoms=100)
    V, freq = 150.0, 1e6
    Om = 2 * math.pi * freq
    dt = 1e-8
    run = W.Run(dt=dt, v_rf=V, f_rf=freq, phi_rf=0.0, dc_scale=0.0, z_exit=half_exit(g), r_det=g.R,
                hit_dist=0.0)
    src = W.Source(n_initial=1)
    w = W.Workload("dehmelt", f, ion, src, run, 0)
    s = orc.Sim(w)
    s.inject(1)
    s.x[0], s.y[0], s.z[0] = (1e-4, 0.0, 0.0) if axis == "r" else (0.0, 0.0, 1e-4)
    s.vx[0] = s.vy[0] = s.vz[0] = 0.0
    m, q = 1000 * DA, E
    I0 = special.i0(r0 / z0l)
    w_r = q * V / (math.sqrt(8.0) * m * Om * z0l ** 2 * I0)
    w_exp = w_r if axis == "r" else 2 * w_r
    n = int(6 * 2 * math.pi / w_exp / dt)
    traj = np.empty(n)
    for k in range(n):
        s.steps(1)
        traj[k] = s.x[0] if axis == "r" else s.z[0]
    assert s.status[0] == 0
    t = dt * np.arange(1, n + 1)
    w_meas = _secular_frequency(t, traj, 1.0 / freq)
    assert abs(w_meas / w_exp - 1) < 0.04, (w_meas, w_exp)


def half_exit(g):
    return g.z1


def gbar(w, s):
    """Mean |v - c| for c Maxwellian with most-probable speed s about the flow,
    at ion-flow relative speed w."""
    if w == 0:
        return 2 * s / math.sqrt(math.pi)
    x = w / s
    return s * ((x + 1 / (2 * x)) * math.erf(x) + math.exp(-x * x) / math.sqrt(math.pi))


@pytest.mark.parametrize("wrel", [0.0, 50.0, 400.0, 2000.0])
def test_collision_rate_frozen(orc, wrel):
    ion = W.ION_1KDA
    run = W.Run(dt=1e-9, seed=5)
    n, T = 200.0 / (KB * 300.0), 300.0
    u = np.array([10.0, -20.0, 30.0])
    v = u + np.array([0.0, 0.6, 0.8]) * wrel
    trials = 400_000
    cnt = orc.count_collisions_frozen(ion, run, n, T, u, v, trials)
    s = math.sqrt(2 * KB * T / (28 * DA))
    lam_dt = n * ion.ccs_m2 * gbar(wrel, s) * run.dt
    mean = cnt / trials
    assert abs(mean - lam_dt) < 4 * math.sqrt(lam_dt / trials) + 1e-9, (mean, lam_dt)


def _thermal_box(n_packs=2000, T_init=300.0, Ez=0.0, p=200.0, seed=3):
    w = W.tiny_cylinder(n_packs=n_packs, n_steps=0, seed=seed)
    g = w.fields.grid
    f = W.uniform_axial_fields(g, Ez=Ez, p=p)
    w.fields = f
    w.source.z_plane = 10e-3
    w.source.half_space = 0
    w.ion = W.IonTemplate(mass_da=1000.0, charge=1, ccs_m2=300e-20, n_atoms=100, T_init=T_init)
    return w


def test_collision_counts_poisson_across_steps(orc):
    """Frozen velocities, uniform gas at rest, no field: each pack's
    candidates are a Poisson process of constant rate, so whatever the step
    boundaries the accepted count over N steps is Poisson(n sigma gbar(w) N dt).
    A tau that is not consumed, or consumed twice, shifts the mean; candidate
    draws shared between steps or packs raise the dispersion."""
    w = _thermal_box(n_packs=2000, seed=11)
    s = orc.Sim(w)
    s.inject()
    n_st = 3000
    v = np.sqrt(s.vx[:s.n] ** 2 + s.vy[:s.n] ** 2 + s.vz[:s.n] ** 2)
    s.steps(n_st, frozen=True)
    assert (s.status[:s.n] == 0).all()
    n = 200.0 / (KB * 300.0)
    sg = math.sqrt(2 * KB * 300.0 / (28 * DA))
    expect = np.array([n * w.ion.ccs_m2 * gbar(x, sg) * n_st * w.run.dt for x in v])
    cnt = s.ncoll[:s.n].astype(np.float64)
    assert abs(cnt.sum() / expect.sum() - 1) < 4 / math.sqrt(expect.sum()), (cnt.sum(), expect.sum())
    disp = np.mean((cnt - expect) ** 2 / expect)
    assert abs(disp - 1) < 4 * math.sqrt(2 / s.n), disp


def test_thermal_collision_rate(orc):
    w = _thermal_box()
    s = orc.Sim(w)
    s.inject()
    s.steps(4000)
    c0 = s.ncoll.sum()
    st0 = s.nsteps.sum()
    s.steps(4000)
    rate = (s.ncoll.sum() - c0) / (s.nsteps.sum() - st0) / w.run.dt
    mu = 1000 * 28 / 1028 * DA
    n = 200.0 / (KB * 300.0)
    exp = n * w.ion.ccs_m2 * math.sqrt(8 * KB * 300.0 / (math.pi * mu))
    assert abs(rate / exp - 1) < 0.01, (rate, exp)


def test_mason_schamp_mobility(orc):
    w = _thermal_box(Ez=2000.0)
    s = orc.Sim(w)
    s.inject()
    s.steps(3000)  # 3 us to reach the steady drift
    z_a = s.z[: s.n].copy()
    n_mid = 12000
    s.steps(n_mid)
    act = s.status[: s.n] == 0
    vd = (s.z[: s.n][act] - z_a[act]).mean() / (n_mid * w.run.dt)
    N = 200.0 / (KB * 300.0)
    mu = 1000 * 28 / 1028 * DA
    K = 3 * E / (16 * N) * math.sqrt(2 * math.pi / (mu * KB * 300.0)) / w.ion.ccs_m2
    assert abs(vd / (K * 2000.0) - 1) < 0.03, (vd, K * 2000.0)


def test_internal_temperature_relaxation(orc):
    w = _thermal_box(T_init=600.0, seed=9)
    s = orc.Sim(w)
    s.inject()
    s.steps(25000)
    e = s.eint[: s.n]
    T = np.array([orc.T_of_eint(w.ion, x) for x in e])
    assert abs(T.mean() / 300.0 - 1) < 0.005, T.mean()
    # equilibrium E_int ~ Gamma(3N, k T) in units of k_B
    assert stats.kstest(e, stats.gamma(300.0, scale=300.0).cdf).pvalue > 0.01
    # ion velocities Maxwellian at the gas temperature
    m = 1000 * DA
    sd = math.sqrt(KB * 300.0 / m)
    assert stats.kstest(s.vx[: s.n] / sd, "norm").pvalue > 0.01
