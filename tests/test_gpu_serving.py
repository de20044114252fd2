"""Continuous batching: requests arriving while others run are admitted into
free slots and advanced together; every request's observables are the same
as when it runs alone (integer tallies bit-exact, FP64 sums to rounding).
The mix runs on a non-default stream, so its batched macro steps are
captured as CUDA graphs and replayed; the requests run alone use direct
launches on the default stream."""
import numpy as np
import pytest

from paper_2609_31258_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("policy", ["all", "srpt"])
def test_serving_mix_equals_alone(policy):
    import torch
    from paper_2609_31258_b300 import build, mucite, serving
    build.build()
    base = W.ring_stack(n_packs=1, n_steps=0, nr=129, nz=513)
    base.run.z_exit = 7.0e-3  # short stack: some packs transmit within the run
    tmpl = W.SERVING_TEMPLATES
    spec = [(0.00, 3000, 0, 11), (0.01, 5000, 1, 12), (0.02, 700, 2, 13), (0.40, 2500, 0, 14), (0.41, 4096, 1, 15)]
    ctx = mucite.Context(0, torch.cuda.Stream(torch.device("cuda", 0)))
    ctx.set_tuning(500, 128)
    ctx.load_fields(base.fields)
    reqs = [serving.make_request(i, t, n, tmpl[k], base, n_steps=3000, seed=sd)
            for i, (t, n, k, sd) in enumerate(spec)]
    # srpt with a small fill: launches take subsets of the admitted requests;
    # chunks of two 500-step launches are replayed from a captured graph
    srv = serving.Server(ctx, max_slots=3, chunk=1000, policy=policy, min_packs=4000, max_defer=0.5)
    done, wall = srv.run(reqs)
    replays, captures = ctx.graph_stats()
    assert replays >= 2 * captures > 0
    assert len(done) == len(reqs)
    assert max(len(srv.active), 0) == 0
    lat = serving.latency_summary(done)
    assert lat["n"] == len(reqs) and lat["p99_s"] >= lat["p50_s"] > 0
    for r in done:
        c1 = mucite.Context(0)
        c1.set_tuning(777, 64)
        c1.load_fields(base.fields)
        c1.inject(0, r.ion, r.source, r.run, capacity=r.n_packs)
        c1.step(0, r.n_steps)
        T = c1.tally(0)
        c1.close()
        for k in ("count", "weight", "exit_hist", "r_hist", "ke_hist", "teff_hist", "loss_map"):
            assert (r.tally[k] == T[k]).all(), (r.rid, k)
        for k in ("pack_steps", "collisions", "emitted_count", "step"):
            assert r.tally[k] == T[k], (r.rid, k)
        assert np.allclose(r.tally["sum_w_ke"], T["sum_w_ke"], rtol=1e-12)
        assert np.allclose(r.tally["sum_w_teff"], T["sum_w_teff"], rtol=1e-12)
    ctx.close()


def test_step_set_matches_step_all_and_rejects_bad_lists():
    from paper_2609_31258_b300 import build, mucite
    build.build()
    w = W.ring_stack(n_packs=2000, n_steps=0, nr=129, nz=513)
    outs = []
    for mode in ("all", "set"):
        ctx = mucite.Context(0)
        ctx.set_tuning(300, 128)
        ctx.load_fields(w.fields)
        for i in range(3):
            ctx.inject(i, w.ion, w.source, w.run, capacity=2000)
        if mode == "all":
            ctx.step(-1, 900)
        else:
            ctx.step_set([2, 0], 900)
            ctx.step_set([1], 900)
        outs.append([ctx.tally(i) for i in range(3)])
        if mode == "set":
            for bad in ([0, 0], [5]):
                with pytest.raises(mucite.MuciteError) as e:
                    ctx.step_set(bad, 10)
                assert e.value.status in (mucite.E_ARG, mucite.E_STATE)
        ctx.close()
    for a, b in zip(*outs):
        assert (a["count"] == b["count"]).all() and a["pack_steps"] == b["pack_steps"]
        assert a["collisions"] == b["collisions"]
