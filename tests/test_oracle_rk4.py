"""Pins of the oracle's RK4 pusher (Methods, "Particle transport, collisions,
and effective internal temperature"), of dt segments and of the Eq. 1
micro-step limits.

- constant force: RK4 positions and velocities are exact (cubic and higher
  terms vanish);
- harmonic field (potential quadratic in z, interpolated exactly by the grid):
  halving dt cuts the RK4 position error ~16x (fourth order) and the leapfrog
  one ~4x (second order);
- a dt change keeps the RF phase continuous: after it the scalar equals
  V cos(2 pi f t + phi) at the accumulated time t;
- Eq. 1 limits against values computed by hand for a simple state.
"""
import math

import numpy as np

from paper_2609_31258_b300 import workloads as W

E, DA, KB = W.E_CHARGE, W.DALTON, W.K_B


def _vacuum_cyl(n=20, integrator=1, Ez=2000.0):
    w = W.tiny_cylinder(n_packs=n, n_steps=0)
    w.fields = W.uniform_axial_fields(w.fields.grid, Ez=Ez, p=0.0)
    w.source.z_plane = 5e-3
    w.run.integrator = integrator
    return w


def test_rk4_exact_under_constant_force(orc):
    w = _vacuum_cyl()
    s = orc.Sim(w)
    s.inject()
    z0, vz0, x0, vx0 = s.z[:20].copy(), s.vz[:20].copy(), s.x[:20].copy(), s.vx[:20].copy()
    n = 2000
    s.steps(n)
    a = E / (1000 * DA) * 2000.0
    t = n * w.run.dt
    assert np.allclose(s.z[:20], z0 + vz0 * t + 0.5 * a * t * t, rtol=1e-12)
    assert np.allclose(s.vz[:20], vz0 + a * t, rtol=1e-12)
    assert np.allclose(s.x[:20], x0 + vx0 * t, rtol=1e-12, atol=1e-18)


def _harmonic(integrator, dt):
    g = W.Grid(33, 401, 5e-3, -10e-3, 10e-3)
    r, z = W.node_coords(g)
    zz, rr = np.meshgrid(z, r, indexing="ij")
    k = 2.0e5  # V/m^2: E_z = -2 k z exactly on the grid (quadratic potential)
    phi = k * zz ** 2
    zero = np.zeros_like(phi)
    f = W.Fields(g, phi, zero.copy(), zero.copy(), np.full_like(phi, 300.0), zero.copy(), zero.copy(),
                 np.zeros(phi.shape, np.uint8), np.full_like(phi, 1.0))
    ion = W.IonTemplate(mass_da=1000.0, charge=1, ccs_m2=0.0, n_atoms=100)
    run = W.Run(dt=dt, z_exit=g.z1, r_det=g.R, hit_dist=0.0, integrator=integrator)
    return W.Workload("harmonic", f, ion, W.Source(n_initial=1), run, 0), k


def _oscillate(orc, integrator, dt, T=20e-6):
    wl, k = _harmonic(integrator, dt)
    omega = math.sqrt(2 * k * E / (1000 * DA))
    z0 = 1e-3
    s = orc.Sim(wl)
    s.inject(1)
    s.x[0] = s.y[0] = s.vx[0] = s.vy[0] = 0.0
    s.z[0] = z0
    # RK4 holds v(t_n); the leapfrog holds v(t_n - dt/2): start each exactly
    s.vz[0] = 0.0 if integrator == 1 else z0 * omega * math.sin(omega * dt / 2)
    n = int(round(T / dt))
    s.steps(n)
    return s.z[0], z0 * math.cos(omega * n * dt)


def test_rk4_fourth_order_leapfrog_second_order(orc):
    e = {}
    for integ in (0, 1):
        errs = []
        for dt in (4e-7, 2e-7):   # omega dt = 0.078, 0.039
            zn, zex = _oscillate(orc, integ, dt)
            errs.append(abs(zn - zex))
        e[integ] = errs[0] / errs[1]
    assert 13.0 < e[1] < 19.0, e   # fourth order
    assert 3.5 < e[0] < 4.5, e     # second order


def test_dt_segment_keeps_rf_phase(orc):
    w = W.ring_stack(n_packs=4, n_steps=0, nr=65, nz=257)
    w.fields.gas_p[:] = 0.0
    s = orc.Sim(w)
    s.inject()
    s.steps(1234)
    t = 1234 * w.run.dt
    s.set_dt(0.3e-9)
    s.steps(777)
    t += 777 * 0.3e-9
    got = orc.rf_scalar(s.run, s.step)
    ref = w.run.v_rf * math.cos(2 * math.pi * w.run.f_rf * t + w.run.phi_rf)
    assert abs(got - ref) < 1e-9 * w.run.v_rf


def test_eq1_limits_by_hand(orc):
    w = _vacuum_cyl(n=3, integrator=0, Ez=2000.0)
    w.fields.gas_p[:] = 200.0
    s = orc.Sim(w)
    s.inject()
    s.vx[:3], s.vy[:3], s.vz[:3] = [0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [10.0, 400.0, -50.0]
    lim = s.dt_limits()
    g = w.fields.grid
    assert math.isinf(lim[0]) and math.isinf(lim[4])
    assert abs(lim[3] - 0.5 * min(g.dr, g.dz) / 400.0) < 1e-15
    a = E / (1000 * DA) * 2000.0
    vth = math.sqrt(KB * 300.0 / (1000 * DA))
    assert abs(lim[2] / (0.1 * max(10.0, vth) / a) - 1) < 1e-12
    # collision limit: the fastest pack (w = 400 m/s) has the largest rate
    n, s_ = 200.0 / (KB * 300.0), math.sqrt(2 * KB * 300.0 / (28 * DA))
    x = 400.0 / s_
    gbar = s_ * ((x + 0.5 / x) * math.erf(x) + math.exp(-x * x) / math.sqrt(math.pi))
    assert abs(lim[1] / (0.1 / (n * 300e-20 * gbar)) - 1) < 1e-12
    assert lim[5] == min(lim[:5])
