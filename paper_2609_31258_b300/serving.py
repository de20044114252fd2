"""Continuous-batching serving loop over the C ABI.

Requests are sweep points (operating point, ion template, pack count,
simulated duration). A request is admitted into a free instance slot as soon
as it has arrived and its pack pool fits in free device memory; from the next
launch on its packs are advanced together with those of every other admitted
request (one batched fused launch per chunk, mucite_step on all instances);
when its clock reaches its duration it is tallied, its slot and pool are
released, and its latency (finish - arrival) is recorded. Arrival times are
wall-clock seconds from the start of `run`.

Every request keeps its own Philox key (its seed) and its own clock, and
per-pack arithmetic does not depend on the other packs of a launch, so a
request's result is the same alone and in any mix.
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


class Server:
    def __init__(self, ctx: mucite.Context, max_slots=32, chunk=2000, mem_reserve=2 << 30):
        self.ctx = ctx
        self.max_slots = min(max_slots, mucite.MAX_INSTANCES)
        self.chunk = chunk
        self.mem_reserve = mem_reserve
        self.active = {}
        self.clock = {}
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

    def _retire(self, slot, now):
        req = self.active.pop(slot)
        req.tally = self.ctx.tally(slot)
        self.pack_steps += req.tally["pack_steps"]
        req.finished = now
        self.ctx.release(slot)
        self.clock.pop(slot)
        return req

    def run(self, requests: List[Request], t_limit: Optional[float] = None):
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        done = []
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
            step = min(self.chunk, min(r.n_steps - self.clock[s] for s, r in self.active.items()))
            self.ctx.step(-1, step)
            for s in self.active:
                self.clock[s] += step
            finished = [s for s, r in self.active.items() if self.clock[s] >= r.n_steps]
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
