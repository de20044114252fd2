"""Batched stepping: many instances (different operating points, pack
counts, seeds and clocks) advanced in one fused launch per chunk -- with the
space-charge macro step batched over instances, CUDA-graph replay of whole
macro steps and the persistent launch -- must give exactly the state each
instance reaches when stepped alone. Per-pack arithmetic does not depend on
the other packs in the launch, so the comparison is bit-exact."""
import numpy as np
import pytest

from paper_2609_31258_b300 import workloads as W
from helpers import download

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    from paper_2609_31258_b300 import build, mucite
    build.build()
    return mucite


def _ring(n, seed, v_rf, dc, p_scale):
    w = W.ring_stack(n_packs=n, n_steps=0, seed=seed, precision=0, nr=129, nz=513)
    w.run.v_rf, w.run.dc_scale, w.run.p_scale = v_rf, dc, p_scale
    return w


POINTS = [(1500, 100, 50.0, 0.5, 0.5), (3333, 101, 150.0, 4.0, 2.0), (257, 102, 100.0, 2.0, 1.0)]


def _alone(mc, w, steps, spl=64):
    ctx = mc.Context(0)
    ctx.set_tuning(spl, 128)
    ctx.set_launch_mode(0, False)
    mc.load_workload(ctx, w, 0)
    for s in steps:
        ctx.step(0, s)
    out = download(ctx, 0, w.source.n_initial)
    T = ctx.tally(0)
    ctx.close()
    return out, T


@pytest.mark.parametrize("persistent,graphs", [(0, False), (0, True), (2, True)])
def test_batched_equals_alone(mc, persistent, graphs):
    import torch
    ws = [_ring(*p) for p in POINTS]
    ctx = mc.Context(0, torch.cuda.Stream())
    ctx.set_tuning(64, 128)
    ctx.set_launch_mode(persistent, graphs)
    ctx.load_fields(ws[0].fields)
    for i, w in enumerate(ws):
        ctx.inject(i, w.ion, w.source, w.run)
    ctx.step(-1, 700)
    ctx.step(-1, 333)
    if graphs:
        assert ctx.launch_count() > 0
    for i, w in enumerate(ws):
        got = download(ctx, i, w.source.n_initial)
        ref, Tref = _alone(mc, w, [700, 333])
        for k in ref:
            assert (got[k] == ref[k]).all(), (i, k)
        T = ctx.tally(i)
        assert T["pack_steps"] == Tref["pack_steps"] and T["collisions"] == Tref["collisions"]
    ctx.close()


def test_batched_mixed_clocks(mc):
    """An instance admitted later (different clock) batched with running ones."""
    ws = [_ring(*p) for p in POINTS[:2]]
    ctx = mc.Context(0)
    ctx.set_tuning(100, 128)
    ctx.load_fields(ws[0].fields)
    ctx.inject(0, ws[0].ion, ws[0].source, ws[0].run)
    ctx.step(-1, 450)
    ctx.inject(1, ws[1].ion, ws[1].source, ws[1].run)
    ctx.step(-1, 500)
    a = download(ctx, 0, ws[0].source.n_initial)
    b = download(ctx, 1, ws[1].source.n_initial)
    ra, _ = _alone(mc, ws[0], [950])
    rb, _ = _alone(mc, ws[1], [500])
    for k in ra:
        assert (a[k] == ra[k]).all(), k
        assert (b[k] == rb[k]).all(), k


@pytest.mark.parametrize("graphs", [False, True])
def test_batched_space_charge(mc, graphs):
    def cyl(n, seed, weight):
        w = W.cylinder_space_charge(n_packs=n, n_steps=0, seed=seed, precision=0, pic_nr=65, pic_nz=257)
        w.source.current_A = 0.0
        w.source.weight = weight
        return w
    import torch
    ws = [cyl(3000, 7, 20000), cyl(1000, 8, 5000), cyl(4500, 9, 1000)]
    ctx = mc.Context(0, torch.cuda.Stream())
    ctx.set_tuning(64, 128)
    ctx.set_launch_mode(0, graphs)
    ctx.load_fields(ws[0].fields)
    for i, w in enumerate(ws):
        ctx.inject(i, w.ion, w.source, w.run)
    ctx.step(-1, 300)
    for i, w in enumerate(ws):
        got = download(ctx, i, w.source.n_initial)
        pic = ctx.pic_read(i)
        c1 = mc.Context(0)
        c1.set_launch_mode(0, False)
        c1.set_tuning(64, 128)
        mc.load_workload(c1, w, 0)
        c1.step(0, 300)
        ref = download(c1, 0, w.source.n_initial)
        pref = c1.pic_read(0)
        c1.close()
        for k in ref:
            assert (got[k] == ref[k]).all(), (i, k)
        assert (pic["Q"] == pref["Q"]).all()
        assert np.abs(pic["phi"] - pref["phi"]).max() <= 1e-12 * max(np.abs(pref["phi"]).max(), 1e-30)
    ctx.close()


def test_autotune_restores_state_and_picks_a_shape(mc):
    """The tuner times shapes on the live instances and restores them: the
    run afterwards is bit-exact with an untuned run of the same instances."""
    import torch
    ws = [_ring(*p) for p in POINTS]
    outs = []
    for tune in (False, True):
        ctx = mc.Context(0, torch.cuda.Stream())
        ctx.set_tuning(64, 128)
        ctx.load_fields(ws[0].fields)
        for i, w in enumerate(ws):
            ctx.inject(i, w.ion, w.source, w.run)
        ctx.step(-1, 300)
        if tune:
            t = ctx.autotune([0, 1, 2], 600)
            assert t["n_tried"] == 12 * 1 and t["best_ms_per_step"] > 0
            assert t["threads_per_block"] in (64, 128, 256) and t["steps_per_launch"] == 250
            with pytest.raises(mc.MuciteError):
                ctx.autotune([0, 0], 10)
        ctx.step(-1, 700)
        outs.append(([download(ctx, i, w.source.n_initial) for i, w in enumerate(ws)],
                     [ctx.tally(i) for i in range(3)]))
        ctx.close()
    (sa, ta), (sb, tb) = outs
    for a, b in zip(sa, sb):
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    for a, b in zip(ta, tb):
        assert (a["count"] == b["count"]).all()
        assert a["pack_steps"] == b["pack_steps"] and a["collisions"] == b["collisions"] and a["step"] == b["step"]


@pytest.mark.parametrize("masked", [0, 1])
def test_captured_solve_loops_match_direct(mc, masked):
    """Under graph capture the correction passes (maskless solve) and the PCG
    iterations (mask-aware solve) run as device-controlled while loops that
    stop at convergence; the direct path issues the fixed pass count, whose
    passes after convergence return at once. Both must reach the same
    charge, potential, residual and iteration count. The PCG scalars come
    from order-independent grid sums, so the mask-aware solve is
    reproducible bit for bit."""
    import torch

    def ring(n, seed):
        w = W.ring_stack(n_packs=n, n_steps=0, seed=seed, precision=0, nr=129, nz=513)
        w.fields.pic = W.Grid(65, 257, w.fields.grid.R, w.fields.grid.z0, w.fields.grid.z1)
        w.run.pic_interval, w.run.pic_masked = 10, masked
        w.source.weight = 1000
        w.source.prefill_z0, w.source.prefill_z1, w.source.radius = 3e-3, 30e-3, 3.5e-3
        return w

    ws = [ring(3000, 21), ring(1200, 22)]
    out = []
    for graphs in (True, False):
        ctx = mc.Context(0, torch.cuda.Stream())
        ctx.set_tuning(64, 128)
        ctx.set_launch_mode(0, graphs)
        ctx.load_fields(ws[0].fields)
        for i, w in enumerate(ws):
            ctx.inject(i, w.ion, w.source, w.run)
        ctx.step(-1, 200)
        out.append([(download(ctx, i, w.source.n_initial), ctx.pic_read(i)) for i, w in enumerate(ws)])
        ctx.close()
    for (sg, pg), (sd, pd) in zip(*out):
        for k in sd:
            assert (sg[k] == sd[k]).all(), k
        assert (pg["Q"] == pd["Q"]).all()
        if masked:
            assert (pg["phi"] == pd["phi"]).all()
            assert pg["iterations"] == pd["iterations"]
        else:
            assert np.abs(pg["phi"] - pd["phi"]).max() <= 1e-12 * max(np.abs(pd["phi"]).max(), 1e-30)
            assert abs(int(pg["iterations"]) - int(pd["iterations"])) <= 1
        assert pg["rel_residual"] <= 1e-6 and pd["rel_residual"] <= 1e-6
        assert np.abs(pd["phi"]).max() > 0.0


def test_autotune_restores_space_charge_state(mc):
    """With a PIC grid the tuner's trials run whole macro steps (charge,
    solve, E_SCE); the snapshot restores the pool and the space-charge state
    (charge, potential, nodal and per-cell E_SCE), so the run afterwards is
    bit-exact with an untuned run."""
    import torch

    def ring(n, seed):
        w = W.ring_stack(n_packs=n, n_steps=0, seed=seed, precision=0, nr=129, nz=513)
        w.fields.pic = W.Grid(65, 257, w.fields.grid.R, w.fields.grid.z0, w.fields.grid.z1)
        w.run.pic_interval = 10
        w.source.weight = 1000
        w.source.prefill_z0, w.source.prefill_z1, w.source.radius = 3e-3, 30e-3, 3.5e-3
        return w

    ws = [ring(2000, 31), ring(900, 32)]
    outs = []
    for tune in (False, True):
        ctx = mc.Context(0, torch.cuda.Stream())
        ctx.set_tuning(64, 128)
        ctx.load_fields(ws[0].fields)
        for i, w in enumerate(ws):
            ctx.inject(i, w.ion, w.source, w.run)
        ctx.step(-1, 105)
        if tune:
            t = ctx.autotune([0, 1], 200)
            assert t["steps_per_launch"] == 64  # the PIC interval sets the macro step
            assert t["n_tried"] == 24 and t["schedule"] in (mc.SCHEDULE_BALANCED, mc.SCHEDULE_EAGER)
        ctx.step(-1, 205)
        outs.append(([download(ctx, i, w.source.n_initial) for i, w in enumerate(ws)],
                     [ctx.pic_read(i) for i in range(2)]))
        ctx.close()
    (sa, pa), (sb, pb) = outs
    for a, b in zip(sa, sb):
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    for a, b in zip(pa, pb):
        assert (a["Q"] == b["Q"]).all()
        assert np.abs(a["phi"] - b["phi"]).max() <= 1e-12 * max(np.abs(a["phi"]).max(), 1e-30)


@pytest.mark.parametrize("space_charge", [False, True])
def test_schedule_does_not_change_results(mc, space_charge):
    """The collision loop's schedule (which lanes a warp serves in an
    iteration) reorders work between lanes only: every pack takes its own
    sequence of operations, so the balanced and the eager schedule give the
    same pools, tallies and space-charge state bit for bit -- for the ring
    stack's frequent candidates and for the cylinder's rare ones, in launches
    of 10 micro steps, batched and graph-replayed."""
    import torch
    if space_charge:
        def cyl(n, seed, weight):
            w = W.cylinder_space_charge(n_packs=n, n_steps=0, seed=seed, precision=0, pic_nr=65, pic_nz=257)
            w.source.current_A = 0.0
            w.source.weight = weight
            return w
        ws = [cyl(3000, 17, 20000), cyl(1200, 18, 5000)]
    else:
        ws = [_ring(*p) for p in POINTS]
    outs = []
    for sched in (mc.SCHEDULE_BALANCED, mc.SCHEDULE_EAGER):
        ctx = mc.Context(0, torch.cuda.Stream())
        ctx.set_tuning(10, 64)
        ctx.set_schedule(sched)
        ctx.load_fields(ws[0].fields)
        for i, w in enumerate(ws):
            ctx.inject(i, w.ion, w.source, w.run)
        ctx.step(-1, 300)
        outs.append(([download(ctx, i, w.source.n_initial) for i, w in enumerate(ws)],
                     [ctx.tally(i) for i in range(len(ws))],
                     [ctx.pic_read(i) for i in range(len(ws))] if space_charge else []))
        with pytest.raises(mc.MuciteError):
            ctx.set_schedule(3)
        ctx.close()
    (sa, ta, pa), (sb, tb, pb) = outs
    for a, b in zip(sa, sb):
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    for a, b in zip(ta, tb):
        assert (a["count"] == b["count"]).all() and a["collisions"] == b["collisions"] > 0
        assert a["pack_steps"] == b["pack_steps"]
    for a, b in zip(pa, pb):
        assert (a["Q"] == b["Q"]).all()
        assert np.array_equal(a["phi"], b["phi"])
