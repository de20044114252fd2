"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle
on identical seeded inputs.

Bars (per the method's stated tolerances):
- classification labels, CIC deposit and integer tallies: bit-exact on
  identical state;
- collision-free trajectories: position within 1e-5 relative (FP32 path);
- stochastic ensembles: transmission inside a 3-sigma binomial band, KS
  p > 0.01 on kinetic energy and T_eff, mean T_eff within 0.5 %;
- Poisson: relative residual <= 1e-6 on the oracle's own operator.
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2609_31258_b300 import workloads as W
from helpers import (binomial_band, download, fp32_state_from_oracle, fp64_state_from_oracle,
                     fp64_from_lattice, lattice_from_fp64, rel_pos_error, upload)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    import torch
    from paper_2609_31258_b300 import build, mucite
    build.build()
    assert torch.cuda.is_available()
    return mucite


def _ctx(mc, w, inst=0, capacity=None, threads=256, spl=256):
    ctx = mc.Context(0)
    ctx.set_tuning(spl, threads)
    mc.load_workload(ctx, w, inst, capacity)
    return ctx


def _ring_small(n_packs=2000, seed=11, precision=0, vacuum=False):
    w = W.ring_stack(n_packs=n_packs, n_steps=0, seed=seed, precision=precision, nr=129, nz=513)
    if vacuum:
        w.fields.gas_p[:] = 0.0
    return w


# ---------------------------------------------------------------------------
# injection
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", [0, 1])
def test_inject_matches_oracle(mc, orc, precision):
    w = W.cylinder_space_charge(n_packs=3001, n_steps=0, precision=precision, pic_nr=33, pic_nz=65)
    s = orc.Sim(w)
    s.inject()
    ctx = _ctx(mc, w)
    got = download(ctx, 0, 3001)
    g = w.fields.grid
    if precision == 1:
        # sincospi on the device vs cos(2 pi u) on the host: agreement to a few
        # ulps of the component's scale, not of a component near zero
        for k in ("x", "y", "z", "vx", "vy", "vz", "eint"):
            ref = getattr(s, k)[:3001]
            assert np.allclose(got[k], ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max()), k
    else:
        xq, yq, zq = lattice_from_fp64(g, s.x[:3001], s.y[:3001], s.z[:3001])
        for a, b in ((got["x"], xq), (got["y"], yq), (got["z"], zq)):
            assert np.abs(a.astype(np.int64) - b).max() <= 1
            assert (a == b).mean() > 0.999
        assert np.allclose(got["vx"], s.vx[:3001].astype(np.float32), rtol=1e-6)
    # Exp(1) optical depth to the first collision candidate
    tol = 1e-13 if precision == 1 else 1e-6
    assert np.allclose(got["tau"], s.tau[:3001].astype(got["tau"].dtype), rtol=tol)
    assert (got["status"] == 0).all() and (got["t_term"] == -1).all()
    ctx.close()


# ---------------------------------------------------------------------------
# collision-free trajectories
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("geometry", ["cylinder", "ring_rf"])
def test_collision_free_trajectories_fp32(mc, orc, geometry):
    if geometry == "cylinder":
        w = W.tiny_cylinder(n_packs=1500, n_steps=0, precision=0)
        w.fields.gas_p[:] = 0.0
        nsteps = 5000
    else:
        w = _ring_small(n_packs=1500, vacuum=True)
        w.source.T_vel = 3000.0
        nsteps = 12000
    s = orc.Sim(w)
    s.inject()
    st = fp32_state_from_oracle(s)
    ctx = _ctx(mc, w, spl=1000)
    upload(ctx, 0, st)
    ctx.step(0, nsteps)
    got = download(ctx, 0, 1500)
    s.steps(nsteps)
    act = (s.status[:1500] == 0) & (got["status"] == 0)
    assert act.mean() > 0.5
    err = rel_pos_error(w.fields.grid, {k: got[k][act] for k in ("x", "y", "z")}, s.x[:1500][act],
                        s.y[:1500][act], s.z[:1500][act])
    assert err.max() < 1e-5, err.max()
    assert (got["status"] == s.status[:1500]).mean() > 0.999


# ---------------------------------------------------------------------------
# plain FP64 step vs oracle, with collisions: nearly every pack identical
# ---------------------------------------------------------------------------
def test_fp64_step_tracks_oracle(mc, orc):
    w = _ring_small(n_packs=1000, precision=1)
    s = orc.Sim(w)
    s.inject()
    ctx = _ctx(mc, w)
    upload(ctx, 0, fp64_state_from_oracle(s))
    ctx.step(0, 400)
    got = download(ctx, 0, 1000)
    s.steps(400)
    same = np.abs(got["vx"] - s.vx[:1000]) <= 1e-9 * (np.abs(s.vx[:1000]) + 1.0)
    assert same.mean() > 0.99, same.mean()
    err = rel_pos_error(w.fields.grid, got, s.x[:1000], s.y[:1000], s.z[:1000], lattice=False)
    assert np.median(err) < 1e-12
    assert (got["status"] == s.status[:1000]).mean() > 0.99
    T = ctx.tally(0)
    assert T["collisions"] > 0


# ---------------------------------------------------------------------------
# stochastic ensembles (FP32 fused path vs oracle)
# ---------------------------------------------------------------------------
def _ensemble_compare(orc, w, got, s, n):
    ion = w.ion
    m = ion.mass_da * W.DALTON
    st_g, st_o = got["status"], s.status[:n]
    for lab in (1, 2, 3, 4):
        assert binomial_band((st_g == lab).sum(), (st_o == lab).sum(), n), lab
    a_g, a_o = st_g == 0, st_o == 0
    ke_g = 0.5 * m * (got["vx"][a_g].astype(np.float64) ** 2 + got["vy"][a_g] ** 2 + got["vz"][a_g] ** 2)
    ke_o = 0.5 * m * (s.vx[:n][a_o] ** 2 + s.vy[:n][a_o] ** 2 + s.vz[:n][a_o] ** 2)
    assert stats.ks_2samp(ke_g, ke_o).pvalue > 0.01
    T_g = np.array([orc.T_of_eint(ion, e) for e in got["eint"][a_g].astype(np.float64)])
    T_o = np.array([orc.T_of_eint(ion, e) for e in s.eint[:n][a_o]])
    assert stats.ks_2samp(T_g, T_o).pvalue > 0.01
    assert abs(T_g.mean() / T_o.mean() - 1) < 0.005


def test_ensemble_cylinder_with_exits(mc, orc):
    w = W.tiny_cylinder(n_packs=3000, n_steps=0, precision=0, seed=4)
    w.run.z_exit = 0.6e-3
    w.run.r_det = 0.8e-3
    s = orc.Sim(w)
    s.inject()
    st = fp32_state_from_oracle(s)
    ctx = _ctx(mc, w, spl=500)
    upload(ctx, 0, st)
    ctx.step(0, 12000)
    got = download(ctx, 0, 3000)
    s.steps(12000)
    assert (got["status"] == 1).sum() > 300  # transmission exercised
    assert (got["status"] == 4).sum() > 30
    _ensemble_compare(orc, w, got, s, 3000)
    # most packs follow the oracle pack for pack (same random streams)
    assert (got["status"] == s.status[:3000]).mean() > 0.9


def test_ensemble_ring_stack_rf_gas(mc, orc):
    w = _ring_small(n_packs=2500, seed=12)
    w.run.z_exit = 9e-3
    s = orc.Sim(w)
    s.inject()
    st = fp32_state_from_oracle(s)
    ctx = _ctx(mc, w, spl=400)
    upload(ctx, 0, st)
    ctx.step(0, 6000)
    got = download(ctx, 0, 2500)
    s.steps(6000)
    _ensemble_compare(orc, w, got, s, 2500)
    T = ctx.tally(0)
    assert T["candidate_overflow"] == 0
    coll_o = s.ncoll[:2500].sum()
    assert abs(T["collisions"] / coll_o - 1) < 0.01


# ---------------------------------------------------------------------------
# discrete decisions on identical state: bit-exact
# ---------------------------------------------------------------------------
def _random_lattice(rng, n, span_r=1.1, zlo=-0.02, zhi=1.02):
    ang = rng.uniform(0, 2 * np.pi, n)
    r = span_r * np.sqrt(rng.uniform(0, 1, n)) * 2 ** 30
    xq = np.rint(r * np.cos(ang)).astype(np.int32)
    yq = np.rint(r * np.sin(ang)).astype(np.int32)
    zq = np.rint(rng.uniform(zlo, zhi, n) * 2 ** 30).astype(np.int32)
    return xq, yq, zq


@pytest.mark.parametrize("precision", [0, 1])
def test_classification_bit_exact(mc, orc, precision):
    w = _ring_small(n_packs=5000, precision=precision)
    f = w.fields
    f.phi_dc[:] = 0.0
    f.phi_rf[:] = 0.0
    f.gas_p[:] = 0.0
    w.run.z_exit, w.run.r_det = 36e-3, 2e-3
    rng = np.random.default_rng(8)
    n = 5000
    xq, yq, zq = _random_lattice(rng, n)
    # exact boundary cases
    zexit_q = math.ceil((w.run.z_exit - f.grid.z0) / (f.grid.z1 - f.grid.z0) * 2 ** 30)
    rdet_q = math.floor(w.run.r_det / f.grid.R * 2 ** 30)
    xq[:4] = [rdet_q, rdet_q + 1, 2 ** 30, 2 ** 30 - 1]
    yq[:4] = 0
    zq[:4] = [zexit_q, zexit_q, 100, 100]
    ctx = _ctx(mc, w)
    z0 = np.zeros(n)
    if precision == 0:
        arr = dict(x=xq, y=yq, z=zq, vx=z0.astype(np.float32), vy=z0.astype(np.float32),
                   vz=z0.astype(np.float32), eint=np.full(n, 1e6, np.float32), status=np.zeros(n, np.uint8),
                   t_term=np.full(n, -1, np.int32))
    else:
        x, y, z = fp64_from_lattice(f.grid, xq, yq, zq)
        arr = dict(x=x, y=y, z=z, vx=z0, vy=z0, vz=z0, eint=np.full(n, 1e6), status=np.zeros(n, np.uint8),
                   t_term=np.full(n, -1, np.int32))
    upload(ctx, 0, arr)
    ctx.step(0, 1)
    got = download(ctx, 0, n)
    s = orc.Sim(w)
    ref = orc.classify_fixed(s.fields_struct(), w.run, xq, yq, zq)
    assert (got["status"] == ref).all()
    assert (got["t_term"][ref != 0] == 1).all()
    assert len(set(ref.tolist())) == 5  # every class exercised


def _pic_workload(n, precision=0, pnr=65, pnz=257):
    return W.cylinder_space_charge(n_packs=n, n_steps=0, precision=precision, pic_nr=pnr, pic_nz=pnz)


@pytest.mark.parametrize("precision", [0, 1])
def test_deposit_bit_exact(mc, orc, precision):
    n = 20011
    w = _pic_workload(n, precision)
    rng = np.random.default_rng(3)
    xq, yq, zq = _random_lattice(rng, n, span_r=0.8, zlo=0.0, zhi=1.0)
    status = np.where(rng.uniform(size=n) < 0.9, 0, 2).astype(np.uint8)
    ctx = _ctx(mc, w)
    z0 = np.zeros(n)
    if precision == 0:
        arr = dict(x=xq, y=yq, z=zq, status=status)
    else:
        x, y, z = fp64_from_lattice(w.fields.grid, xq, yq, zq)
        arr = dict(x=x, y=y, z=z, status=status)
    upload(ctx, 0, arr)
    ctx.pic_update(0)
    got = ctx.pic_read(0)
    ref = orc.deposit_fixed(w.fields.pic, xq, yq, zq, status, w.ion.charge * w.source.weight)
    assert (got["Q"] == ref).all()
    assert got["Q"].sum() == (status == 0).sum() * w.source.weight * 2 ** 30


def test_tally_bit_exact(mc, orc):
    n = 7777
    w = _ring_small(n_packs=n)
    w.source.weight = 1000
    w.run.z_exit, w.run.r_det = 36e-3, 2e-3
    rng = np.random.default_rng(4)
    xq, yq, zq = _random_lattice(rng, n, span_r=0.9)
    status = rng.choice([0, 1, 2, 3, 4, 255], n).astype(np.uint8)
    v = rng.normal(0, 40, (3, n)).astype(np.float32)
    e = rng.uniform(1e6, 5e6, n).astype(np.float32)
    tt = rng.integers(0, 100000, n).astype(np.int32)
    ctx = _ctx(mc, w, capacity=n)
    upload(ctx, 0, dict(x=xq, y=yq, z=zq, vx=v[0], vy=v[1], vz=v[2], eint=e, status=status, t_term=tt))
    T = ctx.tally(0)
    s = orc.Sim(w)
    R = s.tally(xq, yq, zq, v[0].astype(np.float64), v[1].astype(np.float64), v[2].astype(np.float64),
                e.astype(np.float64), status, tt)
    for k in ("count", "weight", "exit_hist", "r_hist", "ke_hist", "teff_hist", "loss_map"):
        assert (T[k] == R[k]).all(), k
    assert np.allclose(T["sum_w_ke"], R["sum_w_ke"], rtol=1e-12)
    assert np.allclose(T["sum_w_teff"], R["sum_w_teff"], rtol=1e-12)
    assert T["emitted_count"] == n == T["count"][:5].sum() + (status == 255).sum()


# ---------------------------------------------------------------------------
# Poisson solve
# ---------------------------------------------------------------------------
# Radial systems: (300, 129) has more than 256 radial unknowns (tridiagonal
# sweeps on global memory); (256, 1024) and (150, 257) have 129..256 (cyclic
# reduction, 150 not a power of two); the others up to 128 (shared-memory
# staged sweeps). (3, 5) and (7, 4): fewer unknowns than one tile or one batch
# of the sweeps' row prefetch; (33, 65): one ragged tile, k range not split;
# (300, 129): k range split over clusters of 2 CTAs, (65, 257) of 4,
# (256, 1024) of 8.
@pytest.mark.parametrize("shape", [(65, 257), (256, 1024), (300, 129), (3, 5), (7, 4), (33, 65), (150, 257)])
def test_poisson_matches_direct_solve(mc, orc, shape):
    from oracle import poisson
    pnr, pnz = shape
    n = 30000
    w = _pic_workload(n, 0, pnr, pnz)
    s = orc.Sim(w)
    s.inject()
    ctx = _ctx(mc, w)
    upload(ctx, 0, fp32_state_from_oracle(s))
    ctx.pic_update(0)
    got = ctx.pic_read(0)
    Q = s.deposit()
    assert (got["Q"] == Q).all()
    ref = poisson.solve(w.fields.pic, Q)
    assert got["rel_residual"] <= 1e-6 and 1 <= got["iterations"] <= 4
    assert poisson.residual(w.fields.pic, Q, got["phi"]) <= 1e-6
    print("phi rel err", np.abs(got["phi"] - ref).max() / np.abs(ref).max(), "res", got["rel_residual"])
    assert np.abs(got["phi"] - ref).max() <= 1e-4 * np.abs(ref).max()
    er, ez = orc.efield_from_phi(ref, w.fields.pic.dr, w.fields.pic.dz)
    scale = max(np.abs(er).max(), np.abs(ez).max())
    assert np.abs(got["er"] - er).max() <= 1e-3 * scale
    assert np.abs(got["ez"] - ez).max() <= 1e-3 * scale


def test_space_charge_ensemble(mc, orc):
    """Whole cycle with space charge every 10 steps: FP32 fused path vs oracle."""
    n = 4000
    w = _pic_workload(n, 0, 65, 257)
    w.source.weight = 20_000  # strong space charge on purpose
    w.source.current_A = 0.0
    w.run.z_exit = 8e-3
    s = orc.Sim(w)
    s.inject()
    ctx = _ctx(mc, w, spl=100)
    upload(ctx, 0, fp32_state_from_oracle(s))
    for _ in range(10):
        ctx.step(0, 300)
        s.advance(300)
    got = download(ctx, 0, n)
    _ensemble_compare(orc, w, got, s, n)
    # space charge pushes packs outwards: compare radial spread
    r_g = np.hypot(*fp64_from_lattice(w.fields.grid, got["x"], got["y"], got["z"])[:2])
    r_o = np.hypot(s.x[:n], s.y[:n])
    a = (got["status"] == 0) & (s.status[:n] == 0)
    assert abs(np.median(r_g[a]) / np.median(r_o[a]) - 1) < 0.01


# ---------------------------------------------------------------------------
# invariants of the implementation
# ---------------------------------------------------------------------------
def test_launch_shape_independence(mc, orc):
    """Per-pack arithmetic does not depend on threads per block or on how many
    steps are fused per launch: states are bit-identical."""
    w = _ring_small(n_packs=3000, seed=5)
    outs = []
    for threads, spl in ((256, 250), (128, 1), (64, 777)):
        ctx = _ctx(mc, w, threads=threads, spl=spl)
        ctx.step(0, 1000)
        outs.append(download(ctx, 0, 3000))
        ctx.close()
    for o in outs[1:]:
        for k in outs[0]:
            assert (o[k] == outs[0][k]).all(), k


def test_checkpoint_resume_bit_exact(mc, orc):
    w = _ring_small(n_packs=2000, seed=6)
    ctx = _ctx(mc, w)
    ctx.step(0, 1500)
    ref = download(ctx, 0, 2000)
    ctx2 = _ctx(mc, w)
    ctx2.step(0, 700)
    mid = download(ctx2, 0, 2000)
    ctx3 = _ctx(mc, w)
    upload(ctx3, 0, mid, step=700)
    ctx3.step(0, 800)
    fin = download(ctx3, 0, 2000)
    for k in ref:
        assert (fin[k] == ref[k]).all(), k


def test_weight_conservation_with_continuous_source(mc, orc):
    w = _pic_workload(5000, 0, 65, 257)
    w.source.current_A = 2e-7  # 0.2 uA at W = 1e3: 625 packs per 1000 steps of 0.5 ns
    ctx = _ctx(mc, w, capacity=8000)
    total_new = 0
    s = orc.Sim(w, capacity=8000)
    for _ in range(4):
        ctx.step(0, 1000)
        total_new += s.emit_continuous(1000)
    T = ctx.tally(0)
    assert T["emitted_count"] == 5000 + total_new
    assert T["emitted_weight"] == T["weight"][:5].sum()
    assert T["step"] == 4000


def test_edge_cases_and_errors(mc, orc):
    w = _ring_small(n_packs=0)
    ctx = _ctx(mc, w, capacity=1)
    ctx.step(0, 10)  # empty instance
    T = ctx.tally(0)
    assert T["count"].sum() == 0 and T["pack_steps"] == 0
    with pytest.raises(mc.MuciteError) as e:
        ctx.step(5, 1)
    assert e.value.status == mc.E_STATE
    with pytest.raises(mc.MuciteError) as e:
        ctx.step(0, -1)
    assert e.value.status == mc.E_ARG
    for spl, threads in ((100, 96), (100, 512), (7000, 128)):
        with pytest.raises(mc.MuciteError) as e:
            ctx.set_tuning(spl, threads)
        assert e.value.status == mc.E_ARG
    bad = W.ring_stack(n_packs=10, n_steps=0, nr=129, nz=513)
    bad.source.n_initial = 10
    with pytest.raises(mc.MuciteError) as e:
        ctx.inject(1, bad.ion, bad.source, bad.run, capacity=5)
    assert e.value.status == mc.E_ARG
    wp = _pic_workload(10)
    ctxp = mc.Context(0)
    ctxp.load_fields(wp.fields)
    wp.source.weight = 10 ** 6
    with pytest.raises(mc.MuciteError) as e:
        ctxp.inject(0, wp.ion, wp.source, wp.run, capacity=10 ** 4)
    assert e.value.status == mc.E_OVERFLOW
    # single pack, ragged tile
    w1 = _ring_small(n_packs=1)
    c1 = _ctx(mc, w1)
    c1.step(0, 100)
    assert c1.tally(0)["pack_steps"] == 100


@pytest.mark.parametrize("graphs", [False, True])
def test_streamed_single_steps_equal_fused_launch(mc, orc, graphs):
    """One micro step per launch (the staged streaming kernel: TMA bulk
    copies of the state several tiles ahead) gives bit for bit the state and
    tallies of the same steps in one fused launch, including a partial last
    tile and packs that terminate; directly and graph-replayed."""
    import torch
    n = 20_000 + 77
    w = W.ring_stack(n_packs=n, n_steps=0, seed=23, precision=0, nr=129, nz=513)
    w.fields.gas_p[:] = 0.0
    w.source.T_vel = 3000.0
    w.run.z_exit = 6.0e-3 + 0.4e-6  # packs start on z = 6 mm moving forward: many cross within the run
    outs = []
    for spl in (1, 60):
        stream = torch.cuda.Stream(torch.device("cuda", 0)) if graphs else None
        ctx = mc.Context(0, stream)
        ctx.set_tuning(spl, 256)
        mc.load_workload(ctx, w, 0)
        ctx.step(0, 60)
        outs.append((download(ctx, 0, n), ctx.tally(0)))
        if graphs and spl == 1:
            assert ctx.graph_stats()[0] >= 2  # replayed single-step macro steps
        ctx.close()
    (a, ta), (b, tb) = outs
    for k in a:
        assert (a[k] == b[k]).all(), k
    assert (a["status"] != 0).sum() > 100 and (a["status"] == 0).sum() > 100
    for k in ("count", "exit_hist", "r_hist"):
        assert (ta[k] == tb[k]).all(), k
    assert ta["pack_steps"] == tb["pack_steps"]


# ---------------------------------------------------------------------------
# space-charge solve with the DST-I contractions on the tensor cores
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(256, 1024), (65, 257), (150, 257)])
def test_poisson_tensor_cores_matches_direct_solve(mc, orc, shape):
    """tcgen05 contractions with TF32-pair operands: the same 1e-6 residual
    (Table S2) on the oracle's operator, the potential and field of the
    direct solve, and within a few FP32 roundings of the SIMT contractions."""
    from oracle import poisson
    pnr, pnz = shape
    n = 30000
    w = _pic_workload(n, 0, pnr, pnz)
    s = orc.Sim(w)
    s.inject()
    st = fp32_state_from_oracle(s)
    out = {}
    for solver in (mc.DST_TENSOR_CORES, mc.DST_SIMT):
        ctx = mc.Context(0)
        ctx.load_fields(w.fields)
        ctx.set_pic_solver(solver)
        ctx.inject(0, w.ion, w.source, w.run)
        upload(ctx, 0, st)
        ctx.pic_update(0)
        out[solver] = ctx.pic_read(0)
        ctx.close()
    got, simt = out[mc.DST_TENSOR_CORES], out[mc.DST_SIMT]
    Q = s.deposit()
    assert (got["Q"] == Q).all()
    ref = poisson.solve(w.fields.pic, Q)
    res = poisson.residual(w.fields.pic, Q, got["phi"])
    assert got["rel_residual"] <= 1e-6 and res <= 1e-6, (got["rel_residual"], res)
    assert got["iterations"] <= simt["iterations"] + 1
    assert np.abs(got["phi"] - ref).max() <= 1e-4 * np.abs(ref).max()
    er, ez = orc.efield_from_phi(ref, w.fields.pic.dr, w.fields.pic.dz)
    scale = max(np.abs(er).max(), np.abs(ez).max())
    assert np.abs(got["er"] - er).max() <= 1e-3 * scale
    assert np.abs(got["ez"] - ez).max() <= 1e-3 * scale


def test_batched_space_charge_tensor_cores_equals_alone(mc):
    """With the tensor-core contractions, instances solved in one batch give
    bit for bit the potentials and packs of the same instances alone."""
    import torch

    def cyl(n, seed, weight):
        w = W.cylinder_space_charge(n_packs=n, n_steps=0, seed=seed, precision=0, pic_nr=65, pic_nz=257)
        w.source.current_A = 0.0
        w.source.weight = weight
        return w
    ws = [cyl(3000, 7, 20000), cyl(1000, 8, 5000)]
    ctx = mc.Context(0, torch.cuda.Stream())
    ctx.set_tuning(64, 128)
    ctx.load_fields(ws[0].fields)
    ctx.set_pic_solver(mc.DST_TENSOR_CORES)
    for i, w in enumerate(ws):
        ctx.inject(i, w.ion, w.source, w.run)
    ctx.step(-1, 200)
    for i, w in enumerate(ws):
        got = download(ctx, i, w.source.n_initial)
        pic = ctx.pic_read(i)
        c1 = mc.Context(0)
        c1.set_tuning(64, 128)
        c1.load_fields(w.fields)
        c1.set_pic_solver(mc.DST_TENSOR_CORES)
        c1.inject(0, w.ion, w.source, w.run)
        c1.step(0, 200)
        ref = download(c1, 0, w.source.n_initial)
        pref = c1.pic_read(0)
        c1.close()
        for k in ref:
            assert (got[k] == ref[k]).all(), (i, k)
        assert (pic["phi"] == pref["phi"]).all()
    ctx.close()


def test_pic_solver_choice_errors(mc):
    w = _pic_workload(100, 0, 65, 257)
    ctx = mc.Context(0)
    with pytest.raises(mc.MuciteError) as e:
        ctx.set_pic_solver(mc.DST_TENSOR_CORES)  # no PIC grid yet
    assert e.value.status == mc.E_STATE
    ctx.load_fields(w.fields)
    with pytest.raises(mc.MuciteError) as e:
        ctx.set_pic_solver(7)
    assert e.value.status == mc.E_ARG
    ctx.inject(0, w.ion, w.source, w.run)
    with pytest.raises(mc.MuciteError) as e:
        ctx.set_pic_solver(mc.DST_SIMT)  # instances already injected
    assert e.value.status == mc.E_STATE
    ctx.close()
