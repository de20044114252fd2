"""Continuous-batching serving loop over the C ABI.

Requests are sweep points (operating point, ion template, pack count,
simulated duration). A request is admitted into a free instance slot as soon
as it has arrived and its pack pool fits in free device memory; from the next
launch on its packs are advanced together with those of every other admitted
request (one batched fused launch per chunk, mucite_step on all instances);
when its clock reaches its duration it is tallied, its slot and pool are
released, and its latency (finish - arrival) is recorded. Arrival times are
wall-clock seconds from the start of `run`.

Which admitted requests share the next launch is the batch policy: "all"
steps every admitted request each chunk (all finish together when their
durations agree); "srpt" takes the requests with the least remaining work
(packs x remaining micro steps) first, adding requests until the launch
holds at least `min_packs` packs (enough to fill the GPU), and adds any
request that has waited longer than `max_defer` seconds for a step, so
small requests finish early without starving large ones.

Every request keeps its own Philox key (its seed) and its own clock, and
per-pack arithmetic does not depend on the other packs of a launch, so a
request's result is the same alone and in any mix, under either policy.

Launches: a chunk advances the selected requests by `chunk` micro steps in
one mucite_step_set call; with the context on a non-default stream and a
chunk of at least two launches, the library captures the batched macro step
as a CUDA graph once per selection and replays it. Back-pressure: the host
enqueues at most `max_ahead` chunks ahead of the device (it waits for the
event of an older chunk before enqueuing a new one), so admission and batch
decisions are taken against the device's progress, not ahead of it.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque
from typing import List, Optional

import numpy as np

from . import mucite, workloads as W


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float
    n_packs: int
    ion: W.IonTemplate
    run: W.Run
    source: W.Source
    n_steps: int
    admitted: Optional[float] = None
    finished: Optional[float] = None
    tally: Optional[dict] = None
    slot: Optional[int] = None

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival


def make_request(rid, arrival, n_packs, template, base: W.Workload, n_steps, seed=None):
    """A sweep-point request on the base workload's geometry and gas."""
    run = dataclasses.replace(base.run, seed=rid if seed is None else seed, precision=mucite.FP32)
    src = dataclasses.replace(base.source, n_initial=int(n_packs))
    return Request(rid, float(arrival), int(n_packs), template, run, src, int(n_steps))


def srpt_batch(active, clock, min_packs, waited=None, max_defer=None):
    """Slots to step next: shortest remaining work first (packs x remaining
    micro steps; ties by slot), until the selection holds `min_packs` packs,
    plus every slot whose wait since its last step exceeds `max_defer`."""
    order = sorted(active, key=lambda s: (active[s].n_packs * (active[s].n_steps - clock[s]), s))
    sel, packs = [], 0
    for s in order:
        if packs >= min_packs:
            break
        sel.append(s)
        packs += active[s].n_packs
    if waited is not None and max_defer is not None:
        sel += [s for s in order[len(sel):] if waited[s] > max_defer]
    return sel


class Server:
    def __init__(self, ctx: mucite.Context, max_slots=32, chunk=4000, mem_reserve=2 << 30, policy="srpt",
                 min_packs=None, max_defer=5.0, max_ahead=2):
        self.ctx = ctx
        self.max_slots = min(max_slots, mucite.MAX_INSTANCES)
        self.chunk = chunk
        self.max_ahead = max(1, int(max_ahead))
        self.mem_reserve = mem_reserve
        if policy not in ("all", "srpt"):
            raise ValueError(f"unknown batch policy {policy!r}")
        self.policy = policy
        if min_packs is None:
            import torch
            # two waves of the fused collision kernel (256 threads x 3 blocks per SM)
            min_packs = 2 * 768 * torch.cuda.get_device_properties(ctx.device).multi_processor_count
        self.min_packs = int(min_packs)
        self.max_defer = max_defer
        self.active = {}
        self.clock = {}
        self.last_step = {}
        self.pack_steps = 0

    def _fits(self, req):
        import torch
        free, _ = torch.cuda.mem_get_info(self.ctx.device)
        need = mucite.state_layout(mucite.FP32, max(req.n_packs, 1)).total_bytes + 256
        return free - need > self.mem_reserve

    def _admit(self, req, now):
        slot = next(s for s in range(self.max_slots) if s not in self.active)
        self.ctx.inject(slot, req.ion, req.source, req.run, capacity=max(req.n_packs, 1))
        req.slot, req.admitted = slot, now
        self.active[slot] = req
        self.clock[slot] = 0
        self.last_step[slot] = now

    def _retire(self, slot, now):
        req = self.active.pop(slot)
        req.tally = self.ctx.tally(slot)
        self.pack_steps += req.tally["pack_steps"]
        req.finished = now
        self.ctx.release(slot)
        self.clock.pop(slot)
        self.last_step.pop(slot)
        return req

    def run(self, requests: List[Request], t_limit: Optional[float] = None):
        import torch
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        done = []
        inflight = deque()
        stream = self.ctx.stream if self.ctx.stream is not None else torch.cuda.current_stream(self.ctx.device)
        t0 = time.perf_counter()
        while pending or self.active:
            now = time.perf_counter() - t0
            if t_limit is not None and now > t_limit:
                break
            while (pending and pending[0].arrival <= now and len(self.active) < self.max_slots
                   and self._fits(pending[0])):
                self._admit(pending.popleft(), now)
            if not self.active:
                if pending:
                    time.sleep(max(0.0, min(pending[0].arrival - now, 0.05)))
                continue
            if self.policy == "srpt":
                waited = {s: now - self.last_step[s] for s in self.active}
                sel = srpt_batch(self.active, self.clock, self.min_packs, waited, self.max_defer)
            else:
                sel = sorted(self.active)
            step = min(self.chunk, min(self.active[s].n_steps - self.clock[s] for s in sel))
            # back-pressure: at most max_ahead chunks queued on the device
            while len(inflight) >= self.max_ahead:
                inflight.popleft().synchronize()
            self.ctx.step_set(sel, step)
            ev = torch.cuda.Event()
            ev.record(stream)
            inflight.append(ev)
            for s in sel:
                self.clock[s] += step
                self.last_step[s] = now
            finished = [s for s in sel if self.clock[s] >= self.active[s].n_steps]
            if finished:
                self.ctx.sync()
                now = time.perf_counter() - t0
                for s in finished:
                    done.append(self._retire(s, now))
        return done, time.perf_counter() - t0


def latency_summary(done: List[Request]):
    lat = np.array([r.latency for r in done if r.latency is not None])
    if lat.size == 0:
        return {"p50_s": None, "p99_s": None, "n": 0}
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)), "n": int(lat.size),
            "mean_s": float(lat.mean())}
