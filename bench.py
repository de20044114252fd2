"""Benchmark of the MuCITE ion-pack step on B300.

Workload (one GPU): the S-lens-like ring stack -- 512 x 2048 (r, z) grid,
20 rings with RF 1 MHz / 100 V peak and DC -2 V per ring, free-jet N2
1000 -> 100 Pa, 100,000 packs of 15 kDa / +8 / 1500 A^2 / 2000 atoms,
dt = 0.5 ns. One benchmark step = `--micro` micro steps of every pack
(gather, collisions, kick, drift, classification) followed by the tally of
the observables. Metric: ion-pack steps per second (active packs advanced
one dt), FP32 fused path, with the plain FP64 GPU step timed on the same
workload beside it.

Timing: CUDA events on the library's stream around each benchmark step,
L2 flushed (256 MiB write) before every timed step, W warm-up steps first,
max over ranks. With torchrun (N > 1) every rank advances its own
independent replica (seed + rank): weak scaling, no data-path collective.

--impl reference runs the FP64 CPU oracle (the reference implementation of
the method here) on the same workload and metric, on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ion-pack steps/s (FP32 batched vs plain FP64, same GPU); p50/p99 request latency"
UNIT = "pack-steps/s"
FP64_PEAK_GFLOPS = 1250.0  # nominal dense FP64 of a B300


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """Samples of the SM clock and the clock-event (throttle) reasons during
    the timed region: NVML polled every 10 ms from a thread (read-only
    queries), else nvidia-smi polled every 20 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index, period_s=0.01):
        self.index = index
        self.period = period_s
        self.proc = None
        self.nvml = None
        self.lines = []
        self.samples = []  # (sm MHz, max sm MHz, set of reason names)
        self.stop = threading.Event()
        self.nvml_error = None

    def _handle(self, nv):
        try:
            import torch
            pr = torch.cuda.get_device_properties(self.index)
            bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
            return nv.nvmlDeviceGetHandleByPciBusId(bus)
        except Exception:
            return nv.nvmlDeviceGetHandleByIndex(self.index)

    def __enter__(self):
        try:
            import pynvml as nv
            nv.nvmlInit()
            h = self._handle(nv)
            bits = [nv.nvmlClocksEventReasonHwSlowdown, nv.nvmlClocksEventReasonHwThermalSlowdown,
                    nv.nvmlClocksEventReasonSwThermalSlowdown, nv.nvmlClocksEventReasonSwPowerCap]
            mx = nv.nvmlDeviceGetMaxClockInfo(h, nv.NVML_CLOCK_SM)

            def poll():
                while not self.stop.is_set():
                    try:
                        sm = nv.nvmlDeviceGetClockInfo(h, nv.NVML_CLOCK_SM)
                        r = nv.nvmlDeviceGetCurrentClocksEventReasons(h)
                        self.samples.append((float(sm), float(mx), {n for n, b in zip(self.NAMES, bits) if r & b}))
                    except Exception:
                        pass
                    self.stop.wait(self.period)

            self.nvml = nv
            self.t = threading.Thread(target=poll, daemon=True)
            self.t.start()
            return self
        except Exception as e:
            self.nvml = None
            self.nvml_error = f"{type(e).__name__}: {e}"
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi needs a moment to start: sample before the timed work
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 3.0:
                time.sleep(0.005)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.nvml is not None:
            self.stop.set()
            self.t.join(timeout=2)
            try:
                self.nvml.nvmlShutdown()
            except Exception:
                pass
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        for a, b, r in self.samples:
            sm.append(a)
            mx.append(b)
            reasons |= r
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(self.NAMES, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm.sort()
        out = {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
               "samples": len(sm), "source": "nvml" if self.samples else "nvidia-smi"}
        if self.nvml_error:
            out["nvml_error"] = self.nvml_error
        return out


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline_run(n_packs=100_000, min_seconds=10.0, max_micro=20000, w=None):
    """The oracle as it stands on a bounded sample of the workload: the full
    pack count, advanced in chunks of 50 micro steps until at least
    `min_seconds` of CPU work (or `max_micro` micro steps) are done."""
    import oracle
    from paper_2609_31258_b300 import workloads as W
    if w is None:
        w = W.ring_stack(n_packs=n_packs, n_steps=0, precision=1)
    s = oracle.Sim(w)
    s.inject()
    s.steps(5)
    n0 = int(s.nsteps.sum())
    t0 = time.perf_counter()
    done = 0
    while done < max_micro and time.perf_counter() - t0 < min_seconds:
        s.steps(50)
        done += 50
    dt = time.perf_counter() - t0
    ps = int(s.nsteps.sum()) - n0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": ps / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "seconds": dt,
            "sample": f"{n_packs} packs x {done} micro steps of the same 512x2048 ring-stack workload "
                      f"({ps} pack-steps in {dt:.1f} s, FP64 C oracle, OpenMP over packs)"}


def cpu_baseline_rows():
    """The oracle's pack-step rate on the three workloads of the CPU-baseline
    plan, each on every host core and on one core: the tiny cylinder whole
    (2,000 packs x 20,000 micro steps), the ring stack on a same-shape subset
    (10,000 packs x 2,000 micro steps on the full 512 x 2048 fields) and the
    space-charge cylinder on a subset (100,000 packs x 200 micro steps, PIC
    256 x 1024 every 10 steps, the direct solve's factorisation included)."""
    import oracle
    from oracle import poisson
    from paper_2609_31258_b300 import workloads as W
    all_cores = os.cpu_count() or 1
    jobs = [("tiny cylinder 64x256, whole (2000 packs x 20000 steps)",
             lambda: W.tiny_cylinder(n_packs=2000, n_steps=0, precision=1), 20000, False),
            ("ring stack 512x2048, subset (10000 packs x 2000 steps)",
             lambda: W.ring_stack(n_packs=10_000, n_steps=0, precision=1), 2000, False),
            ("cylinder + PIC 256x1024 every 10 steps, subset (100000 packs x 200 steps)",
             lambda: W.cylinder_space_charge(n_packs=100_000, n_steps=0, precision=1), 200, True)]
    rows = []
    prev = oracle.threads()
    try:
        for cores in (all_cores, 1):
            used = oracle.threads(cores)
            for name, make, nsteps, pic in jobs:
                w = make()
                s = oracle.Sim(w, capacity=w.source.n_initial + 64)
                s.inject()
                poisson._cache.clear()
                t0 = time.perf_counter()
                if pic:
                    s.advance(nsteps)
                else:
                    s.steps(nsteps)
                dt = time.perf_counter() - t0
                ps = int(s.nsteps[:s.n].sum())
                rows.append({"workload": name, "cores": used, "value": ps / dt, "unit": UNIT, "seconds": dt})
    finally:
        oracle.threads(prev)
    return rows


# --------------------------------------------------------------------------
# Error against the FP64 oracle, per output. The oracle runs of the CPU
# baseline leg serve as the reference: the FP32 fused path and the plain
# FP64 GPU path start from the oracle's state (same state, same seed) or run
# their own injection with another seed (independent samples).
# --------------------------------------------------------------------------
_LAT = 2.0 ** 30


def _to_fp32_state(sim):
    """Lattice positions and FP32 velocity / E_int of the oracle's packs; the
    oracle is reset to exactly those values so both sides start equal."""
    import numpy as np
    n, g = sim.n, sim.g
    sx, sz = _LAT / g.R, _LAT / (g.z1 - g.z0)
    xq = np.rint(sim.x[:n] * sx).astype(np.int32)
    yq = np.rint(sim.y[:n] * sx).astype(np.int32)
    zq = np.rint((sim.z[:n] - g.z0) * sz).astype(np.int32)
    st = dict(x=xq, y=yq, z=zq, status=sim.status[:n].copy(), t_term=sim.t_term[:n].copy())
    for k in ("vx", "vy", "vz", "eint", "lnsy", "tau"):
        st[k] = getattr(sim, k)[:n].astype(np.float32)
        getattr(sim, k)[:n] = st[k].astype(np.float64)
    sim.x[:n] = xq.astype(np.float64) / sx
    sim.y[:n] = yq.astype(np.float64) / sx
    sim.z[:n] = g.z0 + zq.astype(np.float64) / sz
    return st


def _to_fp64_state(sim):
    n = sim.n
    return {k: getattr(sim, k)[:n].copy() for k in ("x", "y", "z", "vx", "vy", "vz", "eint", "status", "t_term",
                                                      "lnsy", "tau")}


def _gpu_run(local, stream, w, state, nsteps, spl=2000):
    """Run a workload on the library from an uploaded state (or from its own
    injection when state is None); returns the pool as numpy and the
    context (caller closes)."""
    import numpy as np
    import torch
    from paper_2609_31258_b300 import mucite
    ctx = mucite.Context(local, stream)
    ctx.set_tuning(spl, 256)
    mucite.load_workload(ctx, w, 0)
    if state is not None:
        views = ctx.state(0)
        n = len(state["status"])
        for k, a in state.items():
            views[k][:n].copy_(torch.from_numpy(np.ascontiguousarray(a)))
        torch.cuda.synchronize()
        ctx.resume(0, n, 0)
    if nsteps:
        ctx.step(0, nsteps)
    return _download(ctx), ctx


def _download(ctx):
    import torch
    ctx.sync()
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in ctx.state(0).items()}


def _pos_err(g, got, sim, n, lattice):
    import numpy as np
    if lattice:
        gx = got["x"][:n].astype(np.float64) * g.R / _LAT
        gy = got["y"][:n].astype(np.float64) * g.R / _LAT
        gz = g.z0 + got["z"][:n].astype(np.float64) * (g.z1 - g.z0) / _LAT
    else:
        gx, gy, gz = got["x"][:n], got["y"][:n], got["z"][:n]
    act = (got["status"][:n] == 0) & (sim.status[:n] == 0)
    d = np.sqrt((gx - sim.x[:n]) ** 2 + (gy - sim.y[:n]) ** 2 + (gz - sim.z[:n]) ** 2)
    nrm = np.sqrt(sim.x[:n] ** 2 + sim.y[:n] ** 2 + (sim.z[:n] - g.z0) ** 2)
    e = (d / nrm)[act]
    return {"max": float(e.max()) if e.size else None, "median": float(np.median(e)) if e.size else None,
            "packs": int(act.sum())}


def _ensemble(oracle, ion, got, n_g, sim, n_o):
    """Per terminal label the fractions and their difference in standard
    deviations of a two-sample binomial proportion; KS on KE and T_eff of
    the active packs; mean-T_eff ratio (GPU / oracle)."""
    import numpy as np
    from scipy import stats
    m = ion.mass_da * 1.66053906660e-27
    st_g, st_o = got["status"][:n_g], sim.status[:n_o]
    lab = {}
    for k, name in ((1, "transmitted"), (2, "electrode"), (3, "radial"), (4, "axial")):
        kg, ko = int((st_g == k).sum()), int((st_o == k).sum())
        p = (kg + ko) / (n_g + n_o)
        sd = math.sqrt(max(p * (1 - p), 1.0 / (n_g + n_o)) * (1.0 / n_g + 1.0 / n_o))
        lab[name] = {"gpu": kg / n_g, "oracle": ko / n_o, "sigma": abs(kg / n_g - ko / n_o) / sd}
    a_g, a_o = st_g == 0, st_o == 0
    ke = lambda vx, vy, vz: 0.5 * m * (vx.astype(np.float64) ** 2 + vy.astype(np.float64) ** 2 +
                                       vz.astype(np.float64) ** 2) / 1.602176634e-19
    ke_g = ke(got["vx"][:n_g][a_g], got["vy"][:n_g][a_g], got["vz"][:n_g][a_g])
    ke_o = ke(sim.vx[:n_o][a_o], sim.vy[:n_o][a_o], sim.vz[:n_o][a_o])
    T_of = np.vectorize(lambda e: oracle.T_of_eint(ion, float(e)))
    T_g = T_of(got["eint"][:n_g][a_g].astype(np.float64))
    T_o = T_of(sim.eint[:n_o][a_o])
    k1, k2 = stats.ks_2samp(ke_g, ke_o), stats.ks_2samp(T_g, T_o)
    return {"labels": lab, "ke_ks": {"D": float(k1.statistic), "p": float(k1.pvalue)},
            "teff_ks": {"D": float(k2.statistic), "p": float(k2.pvalue)},
            "mean_ke_ratio": float(ke_g.mean() / ke_o.mean()), "mean_teff_ratio": float(T_g.mean() / T_o.mean())}


def _pack_diffs(oracle, ion, got, sim, n):
    """Same state, same seed: label agreement and per-pack relative
    differences of KE and T_eff over the packs active on both sides."""
    import numpy as np
    agree = float((got["status"][:n] == sim.status[:n]).mean())
    a = (got["status"][:n] == 0) & (sim.status[:n] == 0)
    v2g = sum(got[k][:n][a].astype(np.float64) ** 2 for k in ("vx", "vy", "vz"))
    v2o = sum(getattr(sim, k)[:n][a] ** 2 for k in ("vx", "vy", "vz"))
    dke = np.abs(v2g / v2o - 1.0)
    T_of = np.vectorize(lambda e: oracle.T_of_eint(ion, float(e)))
    dT = np.abs(T_of(got["eint"][:n][a].astype(np.float64)) / T_of(sim.eint[:n][a]) - 1.0)
    return {"label_agreement": agree, "ke_rel_median": float(np.median(dke)), "ke_rel_p99": float(np.quantile(dke, 0.99)),
            "teff_rel_median": float(np.median(dT)), "teff_rel_p99": float(np.quantile(dT, 0.99))}


def parity_report(local, stream):
    """Error of the FP32 fused path and of the plain FP64 GPU path against
    the FP64 oracle, per output, on bounded samples of the benchmarked
    workloads (seconds of oracle work each)."""
    import numpy as np
    import oracle
    from oracle import poisson
    from paper_2609_31258_b300 import workloads as W
    out = {}
    t_start = time.perf_counter()

    # collision-free trajectories on the full ring-stack fields: position
    n = 10_000
    w = W.ring_stack(n_packs=n, n_steps=0, seed=31, precision=0)
    w.fields.gas_p[:] = 0.0
    w.source.T_vel = 3000.0
    s = oracle.Sim(w)
    s.inject()
    st32 = _to_fp32_state(s)
    st64 = _to_fp64_state(s)
    g32, c = _gpu_run(local, stream, w, st32, 4000)
    c.close()
    w.run.precision = 1
    g64, c = _gpu_run(local, stream, w, st64, 4000)
    c.close()
    s.steps(4000)
    g = w.fields.grid
    out["position_collision_free"] = {
        "workload": "ring stack 512x2048, no gas, 10000 packs at 3000 K, 4000 micro steps, same state",
        "fp32": _pos_err(g, g32, s, n, True), "fp64_gpu": _pos_err(g, g64, s, n, False),
        "label_agreement_fp32": float((g32["status"][:n] == s.status[:n]).mean()),
        "label_agreement_fp64": float((g64["status"][:n] == s.status[:n]).mean()), "bar": "max < 1e-5"}

    # collisions on the ring stack: KE, T_eff, collision rate
    w = W.ring_stack(n_packs=n, n_steps=0, seed=1, precision=0)
    s = oracle.Sim(w)
    s.inject()
    st32 = _to_fp32_state(s)
    st64 = _to_fp64_state(s)
    g32, c = _gpu_run(local, stream, w, st32, 2000)
    T32 = c.tally(0)
    c.close()
    w.run.precision = 1
    g64, c = _gpu_run(local, stream, w, st64, 2000)
    c.close()
    s.steps(2000)
    w.run.precision = 0
    gi, c = _gpu_run(local, stream, w, None, 2000)
    c.close()
    wo = W.ring_stack(n_packs=n, n_steps=0, seed=1001, precision=1)
    so = oracle.Sim(wo)
    so.inject()
    so.steps(2000)
    out["collisions_ring_stack"] = {
        "workload": "ring stack 512x2048 with gas, 10000 packs, 2000 micro steps",
        "same_state_fp32": _pack_diffs(oracle, w.ion, g32, s, n),
        "same_state_fp64": _pack_diffs(oracle, w.ion, g64, s, n),
        "collisions_per_pack_step": {"fp32": T32["collisions"] / max(T32["pack_steps"], 1),
                                     "oracle": float(s.ncoll[:n].sum() / s.nsteps[:n].sum())},
        "independent_seeds_fp32": _ensemble(oracle, w.ion, gi, n, so, n)}

    # terminal labels and transmission on the tiny cylinder with a near exit
    n = 10_000

    def cyl(seed, prec):
        w = W.tiny_cylinder(n_packs=n, n_steps=0, precision=prec, seed=seed)
        w.run.z_exit, w.run.r_det = 0.6e-3, 0.8e-3
        return w
    w = cyl(4, 0)
    s = oracle.Sim(w)
    s.inject()
    st32 = _to_fp32_state(s)
    g32, c = _gpu_run(local, stream, w, st32, 12000)
    c.close()
    s.steps(12000)
    gi, c = _gpu_run(local, stream, cyl(5, 0), None, 12000)
    c.close()
    so = oracle.Sim(cyl(1005, 1))
    so.inject()
    so.steps(12000)
    out["labels_cylinder"] = {
        "workload": "tiny cylinder 64x256, z_exit 0.6 mm, r_det 0.8 mm, 10000 packs, 12000 micro steps",
        "same_state_fp32": _pack_diffs(oracle, w.ion, g32, s, n),
        "independent_seeds_fp32": _ensemble(oracle, w.ion, gi, n, so, n)}

    # ln SY (Eq. 7) of hot dissociating ions cooling in the gas
    n = 3000

    def tst(prec):
        w = W.tiny_cylinder(n_packs=n, n_steps=0, precision=prec, seed=17)
        w.fields.phi_dc[:] = 0.0
        w.source.z_plane = 10e-3
        w.ion = W.IonTemplate(mass_da=556.27, charge=1, ccs_m2=1.62e-18, n_atoms=77, T_init=1100.0,
                              dH_kJmol=111.7, dS_JmolK=-38.1)
        return w
    w = tst(0)
    s = oracle.Sim(w)
    s.inject()
    st32 = _to_fp32_state(s)
    st64 = _to_fp64_state(s)
    g32, c = _gpu_run(local, stream, w, st32, 4000, spl=500)
    c.close()
    g64, c = _gpu_run(local, stream, tst(1), st64, 4000, spl=500)
    c.close()
    s.steps(4000)
    sy_o = np.exp(s.lnsy[:n])

    def sy(got):
        d = np.abs(got["lnsy"][:n].astype(np.float64) - s.lnsy[:n])
        return {"mean_sy_ratio": float(np.exp(got["lnsy"][:n].astype(np.float64)).mean() / sy_o.mean()),
                "ln_sy_abs_median": float(np.median(d)), "ln_sy_abs_p99": float(np.quantile(d, 0.99))}
    out["survival_yield"] = {"workload": "tiny cylinder, 556 Da/+1 at 1100 K, dH 111.7 kJ/mol, dS -38.1 J/mol/K, "
                                         "3000 packs, 4000 micro steps, same state",
                             "mean_sy_oracle": float(sy_o.mean()), "fp32": sy(g32), "fp64_gpu": sy(g64)}

    # space charge: deposit, potential, field, residual
    n = 100_000
    w = W.cylinder_space_charge(n_packs=n, n_steps=0, precision=0)
    s = oracle.Sim(w)
    s.inject()
    st32 = _to_fp32_state(s)
    st64 = _to_fp64_state(s)
    Q, phi = s.pic_update()
    pic = w.fields.pic
    res = {}
    for prec, st in ((0, st32), (1, st64)):
        w.run.precision = prec
        _, c = _gpu_run(local, stream, w, st, 0)
        c.pic_update(0)
        pr = c.pic_read(0)
        c.close()
        er, ez = oracle.efield_from_phi(phi, pic.dr, pic.dz)
        d = {"deposit_mismatched_nodes": int((pr["Q"] != Q).sum()),
             "phi_rel_max": float(np.abs(pr["phi"] - phi).max() / np.abs(phi).max()),
             "rel_residual_reported": float(pr["rel_residual"]),
             "rel_residual_recomputed": poisson.residual(pic, Q, pr["phi"]),
             "solve_passes": int(pr["iterations"])}
        scale = max(np.abs(er).max(), np.abs(ez).max())
        d["esc_rel_max"] = float(max(np.abs(pr["er"] - er).max(), np.abs(pr["ez"] - ez).max()) / scale)
        res["fp32" if prec == 0 else "fp64_gpu"] = d
    out["space_charge"] = dict(workload="cylinder 1e5 packs prefilled, PIC 256x1024, one update, same state",
                               **res)

    # the space-charge run as an ensemble: independent seeds, replicated runs
    # (in one run every pack moves in the field of that run's own charge
    # grid, whose noise is common to its packs: with the benchmark's 1e6
    # packs even the oracle against itself fails an i.i.d. KS test), ten runs
    # of 1e4 packs per side pooled
    import numpy as np
    nr, runs = 10_000, 10
    pool_g, pool_o = [], []

    def sc(seed, prec):
        w = W.cylinder_space_charge(n_packs=nr, n_steps=0, seed=seed, precision=prec)
        w.source.current_A = 0.0
        return w
    for r in range(runs):
        w = sc(2 + r, 0)
        _, ctx = _gpu_run(local, stream, w, None, 0)
        ctx.step(0, 200)
        pool_g.append(_download(ctx))
        ctx.close()
        so = oracle.Sim(sc(1002 + r, 1))
        so.inject()
        so.advance(200)
        pool_o.append(so)

    class _Pooled:
        pass
    po = _Pooled()
    for k in ("status", "vx", "vy", "vz", "eint"):
        setattr(po, k, np.concatenate([getattr(s_, k)[:nr] for s_ in pool_o]))
    pg = {k: np.concatenate([g_[k][:nr] for g_ in pool_g]) for k in ("status", "vx", "vy", "vz", "eint")}
    out["space_charge_ensemble"] = {
        "workload": "cylinder, W = 1e3, PIC 256x1024 every 10 steps, 200 micro steps; 10 runs of 1e4 packs per side "
                    "(GPU seeds 2-11, oracle seeds 1002-1011), pooled",
        "independent_seeds_fp32": _ensemble(oracle, w.ion, pg, nr * runs, po, nr * runs)}
    out["seconds"] = time.perf_counter() - t_start
    return out


def _config(args, name, ws):
    """The workload, identical for both arms (the launch shape is reported
    separately by the CUDA arm)."""
    return {"workload": name, "grid": "512x2048", "packs_per_gpu": args.packs,
            "micro_steps_per_step": args.micro,
            "l2": "flushed before every timed step (256 MiB write)",
            "parallelism": f"replicas x{ws}"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2609_31258_b300 import workloads as W
    w = W.ring_stack(n_packs=args.packs, n_steps=0, precision=1)
    steps, secs = [], []
    cb = None
    for k in range(args.warmup + args.steps):
        # each step a bounded sample (about 8 s) of the same workload
        r = cpu_baseline_run(n_packs=args.packs, min_seconds=8.0, max_micro=args.micro, w=w)
        if k >= args.warmup:
            steps.append(r["value"])
            secs.append(r["seconds"])
            cb = r
    val = sum(steps) / len(steps)
    # wall time of one timed (sampled) step
    ms_step = 1e3 * sum(secs) / len(secs)
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": _config(args, w.name, ws),
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                            "sample": "each timed step: " + cb["sample"]},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mucite", choices=["mucite", "reference"])
    ap.add_argument("--micro", type=int, default=2000, help="micro steps per benchmark step")
    ap.add_argument("--packs", type=int, default=100_000)
    ap.add_argument("--spl", type=int, default=0, help="micro steps fused per launch (0 = tuned default)")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--no-autotune", action="store_true", help="keep 2000 steps per launch, 256-pack tiles")
    ap.add_argument("--fp64-steps", type=int, default=2, help="timed steps of the plain FP64 path")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle legs (CPU baseline, its per-workload rows and the parity report)")
    ap.add_argument("--no-parity", action="store_true", help="skip the per-output error report")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-streamed", action="store_true")
    ap.add_argument("--streamed-packs", type=int, default=8_000_000)
    ap.add_argument("--streamed-threads", type=int, default=256, help="packs per tile of the streamed launch")
    ap.add_argument("--streamed-persistent", type=int, default=0,
                    help="persistent blocks per SM of the streamed launch (0: one block per tile)")
    ap.add_argument("--serve-requests", type=int, default=200, help="first arrivals served at 20 / s")
    ap.add_argument("--serve-steps", type=int, default=100_000, help="micro steps per request (50 us)")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-pic", action="store_true")
    ap.add_argument("--no-paper-grid", action="store_true")
    ap.add_argument("--pic-packs", type=int, default=1_000_000)
    ap.add_argument("--pic-steps", type=int, default=2000)
    ap.add_argument("--pic-direct", action="store_true",
                    help="space-charge and sweep sections without graph replay: the solves run their "
                         "fixed pass sequence as separate launches (a profiler cannot see the kernels of "
                         "graphs that hold device-controlled loops)")
    ap.add_argument("--sweep-instances", type=int, default=64)
    ap.add_argument("--sweep-steps", type=int, default=2000)
    ap.add_argument("--sweep-tune-steps", type=int, default=200, help="autotuner trial length (0: no tuning)")
    ap.add_argument("--serve-search-requests", type=int, default=24,
                    help="arrivals served in each trial of the sustainable-rate search (0: no search)")
    ap.add_argument("--serve-search-trials", type=int, default=3, help="most trials of the sustainable-rate search")
    ap.add_argument("--serve-policy", default="srpt", choices=["srpt", "all"],
                    help="batch policy of the serving loop")
    ap.add_argument("--section", default="all",
                    choices=["all", "fused", "streamed", "serving", "sweep", "space_charge", "paper_grid", "fp64"],
                    help="run only one timed section (for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    from paper_2609_31258_b300 import build, mucite, workloads as W

    ws, rank, local = _dist()
    if args.section == "serving":
        torch.cuda.set_device(local)
        build.build()
        print(json.dumps(_serving(args, local)))
        return
    if args.section == "paper_grid":
        torch.cuda.set_device(local)
        build.build()
        dev = torch.device("cuda", local)
        print(json.dumps(_paper_grid(args, local, torch.cuda.Stream(dev), dev)))
        return
    if args.section == "space_charge":
        torch.cuda.set_device(local)
        build.build()
        dev = torch.device("cuda", local)
        print(json.dumps(_space_charge(args, local, torch.cuda.Stream(dev), dev)))
        return
    if args.section == "sweep":
        torch.cuda.set_device(local)
        build.build()
        dev = torch.device("cuda", local)
        print(json.dumps(_sweep(args, local, torch.cuda.Stream(dev), dev)))
        return
    if args.section == "fp64":
        torch.cuda.set_device(local)
        build.build()
        dev = torch.device("cuda", local)
        w = W.ring_stack(n_packs=args.packs, n_steps=0, seed=1 + rank, precision=0)
        print(json.dumps(_fp64(args, w, local, torch.cuda.Stream(dev), dev)))
        return
    if args.section == "streamed":
        torch.cuda.set_device(local)
        build.build()
        print(json.dumps(_streamed_push(args, local, torch.cuda.Stream(torch.device("cuda", local)),
                                        torch.device("cuda", local), _peaks()[0])))
        return
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    dev = torch.device("cuda", local)
    peaks, peak_src = _peaks()

    w = W.ring_stack(n_packs=args.packs, n_steps=0, seed=1 + rank, precision=0)
    stream = torch.cuda.Stream(dev)
    ctx = mucite.Context(local, stream)
    ctx.set_tuning(args.spl or 2000, args.threads or 256)
    mucite.load_workload(ctx, w, 0)
    tuning = None
    if not args.spl and not args.threads and not args.no_autotune:
        # the library's autotuner picks the launch shape (state restored after)
        tuning = ctx.autotune([0], 2 * args.micro)
        args.spl, args.threads = tuning["steps_per_launch"], tuning["threads_per_block"]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def bench_step():
        ctx.step(0, args.micro)

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()

    # warm-up
    for _ in range(args.warmup):
        bench_step()
        ctx.tally(0)
    barrier()
    T0 = ctx.tally(0)
    l0 = ctx.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            bench_step()
            ev[k][1].record(stream)
        barrier()
    launches_step = ctx.launch_count() - l0
    T1 = ctx.tally(0)
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    pack_steps = T1["pack_steps"] - T0["pack_steps"]
    t_ms, total_ps = aggregate(t_ms, pack_steps, dev, ws)
    value = total_ps / (t_ms * 1e-3)

    # kernel-level roofline of the fused step kernel: launches of one step
    launches_per_step = launches_step / args.steps
    # each fused launch is preceded by the RF-table pre-kernel (~20 us of the
    # ~14 ms; 0.15 % of the launch list), so the step kernel's average
    # duration is the step time over the fused launches of one step
    spl = args.spl or 2000
    step_launches = -(-args.micro // spl)
    kern_ms = t_ms / args.steps / step_launches
    prof, stale = _profile_fields()
    insts = None if stale else float(prof["inst_per_pack_step"]) if "inst_per_pack_step" in prof else None
    traffic = None if stale else float(prof["dram_bytes_per_launch"]) if "dram_bytes_per_launch" in prof else None
    sm_mhz = clk.summary().get("sm_mhz") or peaks.get("sm_max_mhz", 2032.0)
    peak_ginst = 148 * 4 * 32 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e9  # lane-instructions/s, in G
    ps_per_launch = pack_steps / (args.steps * step_launches)
    ach = insts * ps_per_launch / (kern_ms * 1e-3) / 1e9 if insts else None
    roofline = {"bound": "alu", "achieved": ach, "peak": peak_ginst, "unit": "Ginst/s (thread instructions)",
                "frac": (ach / peak_ginst) if ach else None, "traffic": traffic, "profile_stale": stale,
                "kernel": "step_f32_one_kernel", "kernel_ms_per_launch": kern_ms,
                "inst_per_pack_step": insts, "pack_steps_per_launch": ps_per_launch,
                "peak_source": "148 SMs x 4 schedulers x 32 lanes x max SM clock (issue-bound ALU peak)",
                "issue_active": None if stale else prof.get("smsp__issue_active.avg.pct_of_peak_sustained_active"),
                "note": "executed thread instructions over issue slots: fewer instructions per pack-step at the "
                        "same issue activity lower this fraction while raising the pack-step rate",
                "hbm_bytes_per_pack_step_at_launch": 65.0 / (args.spl or 2000)}

    if args.section == "fused":
        print(json.dumps({"value": value, "pack_steps_per_step": pack_steps / args.steps,
                          "launches_per_step": launches_per_step, "ms_per_step": t_ms / args.steps}))
        return
    # end to end through the C ABI with host buffers: H2D of the pack state
    # from pinned memory, the steps, D2H of the tally
    e2e = _e2e(ctx, args, stream, dev, w, tuning)

    # plain FP64 GPU step on the same workload
    fp64 = None
    if not args.no_fp64:
        fp64 = _fp64(args, w, local, stream, dev)
    # the single-GPU sections (streamed push, sweep, space charge, paper grid,
    # serving) describe one device: they run at N = 1 only, so a multi-rank
    # run times the replicated step and stays short
    one = ws == 1
    streamed = None
    if one and not args.no_streamed:
        streamed = _streamed_push(args, local, stream, dev, peaks)
    sweep = None
    if one and not args.no_sweep:
        sweep = _sweep(args, local, stream, dev)
    space_charge = None
    if one and not args.no_pic:
        space_charge = _space_charge(args, local, stream, dev)
    paper = None
    if one and not args.no_paper_grid:
        paper = _paper_grid(args, local, stream, dev)
    serve = None
    if one and not args.no_serving:
        serve = _serving(args, local)

    # CPU-baseline leg (rank 0): the oracle timed on the host cores, its rows
    # on the three planned workloads, and its runs as the reference of the
    # per-output error report
    cpu = parity = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline_run()
        if one:
            cpu["rows"] = cpu_baseline_rows()
            if not args.no_parity:
                parity = parity_report(local, stream)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": _config(args, w.name, ws),
               "launch": {"steps_per_launch": args.spl or 2000, "threads_per_block": args.threads or 256,
                          "autotuned": tuning},
               "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu, "clocks": clk.summary(),
               "gpu_launches": int(launches_step), "fp64_plain": fp64,
               "speedup_fp32_vs_fp64": (value / ws) / fp64["value"] if fp64 else None,
               "streamed_push": streamed,
               "sweep": sweep,
               "space_charge": space_charge,
               "paper_grid": paper,
               "serving": serve,
               "parity": parity,
               "peaks_source": peak_src}
        print(json.dumps(out))
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def aggregate(t_ms, pack_steps, dev, ws):
    """Whole-job figures over ranks: the slowest rank's time, the sum of the
    pack-steps every rank advanced (replicas run independently; this is the
    only collective, outside the timed region)."""
    if ws <= 1:
        return float(t_ms), float(pack_steps)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(t_ms)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([float(pack_steps)], device=dev, dtype=torch.float64)
    dist.all_reduce(p)
    return float(t.item()), float(p.item())


def source_stamp(cu_name="step_fp32.cu"):
    """SHA-256 of the code a kernel is compiled from: the CUDA source and its
    local includes (transitively), comments and blank space removed, so a
    profile summary taken on other code is recognised as stale."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_2609_31258_b300", "csrc")
    seen, order = set(), []

    def visit(path):
        path = os.path.normpath(path)
        if path in seen or not os.path.exists(path):
            return
        seen.add(path)
        src = open(path).read()
        order.append((os.path.relpath(path, ROOT), src))
        for inc in re.findall(r'#include\s+"([^"]+)"', src):
            visit(os.path.join(os.path.dirname(path), inc))

    visit(os.path.join(csrc, cu_name))
    h = hashlib.sha256()
    for rel, src in sorted(order):
        code = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        code = re.sub(r"//[^\n]*", "", code)
        code = "\n".join(ln.strip() for ln in code.splitlines() if ln.strip())
        h.update(rel.encode() + b"\0" + code.encode() + b"\0")
    return h.hexdigest()


def _profile_fields(name="step_f32_ring_stack.txt", cu_name="step_fp32.cu"):
    """Figures of a committed ncu summary, and whether it was taken on the
    code that is built now (its sources_sha256 line against source_stamp)."""
    p = os.path.join(ROOT, "profiles", name)
    out = {}
    try:
        for ln in open(p):
            if ":" in ln:
                k, v = ln.split(":", 1)
                out[k.strip()] = v.strip()
    except OSError:
        return {}, "no profile summary"
    if out.get("sources_sha256", "").split(" ")[0] != source_stamp(cu_name):
        return out, f"profiles/{name} was taken on other {cu_name} sources: re-profile"
    return out, None


def _e2e(ctx, args, stream, dev, w, tuning):
    """The headline metric through the C ABI with host buffers: every step
    uploads the pack state (the instance's whole pool, one copy) from pinned
    host memory, advances it by the step's micro steps and reads the tally
    back (the step's result), one step after the other on one context: the
    value. Also timed with two contexts on their own streams taking such
    independent steps in turn, so that one step's upload, read-back and host
    turnaround overlap the other's compute, and the two steps' launches share
    the GPU -- a serving process's throughput with two jobs in flight,
    reported beside the value, not as it."""
    import torch
    from paper_2609_31258_b300 import mucite
    n = args.packs
    assert ctx.meta[0]["capacity"] == n
    pool = ctx.pool(0)
    host = torch.empty(pool.shape, dtype=torch.uint8, pin_memory=True)
    torch.cuda.synchronize(dev)
    host.copy_(pool)
    h2d = host.numel()
    step0 = ctx.tally(0)["step"]
    K = max(2, args.steps // 2)

    def submit(c, s, dst):
        with torch.cuda.stream(s):
            dst.copy_(host, non_blocking=True)
        c.resume(0, n, step0)
        c.step(0, args.micro)

    torch.cuda.synchronize(dev)
    t_start = time.perf_counter()
    for k in range(K):
        submit(ctx, stream, pool)
        T = ctx.tally(0)  # D2H of the observables, synchronises
    t_serial = time.perf_counter() - t_start
    # resume() zeroes the device counters: count the last call's pack-steps
    per_call = T["pack_steps"]
    d2h = 8 * (16 + 16 + 6) + 8 * (T["exit_hist"].size + T["r_hist"].size + T["ke_hist"].size +
                                   T["teff_hist"].size + T["loss_map"].size)

    out = {"value": per_call * K / t_serial, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h), "steps": K,
           "note": "pinned host pool -> device (one copy), micro steps, tally -> host, every step, on one "
                   "context with nothing overlapped"}
    # two jobs in flight: a second context with the same workload and launch
    # shape (a supplementary figure: a failure here leaves the value standing)
    ctx2 = None
    try:
        s2 = torch.cuda.Stream(dev)
        ctx2 = mucite.Context(dev.index, s2)
        ctx2.set_tuning(args.spl or 2000, args.threads or 256)
        if tuning:
            ctx2.set_launch_mode(tuning["persistent_blocks_per_sm"], True)
            ctx2.set_schedule(tuning["schedule"])
        mucite.load_workload(ctx2, w, 0)
        lanes = [(ctx, stream, pool), (ctx2, s2, ctx2.pool(0))]
        submit(*lanes[1])
        ctx2.tally(0)  # warm-up of the second context
        torch.cuda.synchronize(dev)
        t_start = time.perf_counter()
        submit(*lanes[0])
        done = 0
        for k in range(K):
            if k + 1 < K:
                submit(*lanes[(k + 1) % 2])
            done += lanes[k % 2][0].tally(0)["pack_steps"]  # synchronises that context's stream only
        t_pipe = time.perf_counter() - t_start
    except (RuntimeError, mucite.MuciteError) as ex:
        out["two_jobs_in_flight"] = {"value": None, "error": str(ex)}
        return out
    finally:
        if ctx2 is not None:
            ctx2.close()
    out["two_jobs_in_flight"] = {"value": done / t_pipe, "unit": UNIT,
                                   "note": "two contexts take independent steps in turn: one step's copies and "
                                           "host turnaround overlap the other's compute, and their launches "
                                           "share the GPU (more warps per scheduler than one 100,000-pack "
                                           "launch has)"}
    return out


def _streamed_push(args, local, stream, dev, peaks):
    """HBM roofline of the streamed step: one micro step per launch on a
    collision-free ring-stack workload whose pack pool exceeds L2. The
    collision-free kernel reads status, lattice position and velocity
    (1 + 12 + 12 bytes) and writes position and velocity (24 bytes) per
    pack-step: 49 algorithmic bytes."""
    import torch
    from paper_2609_31258_b300 import mucite, workloads as W
    n = args.streamed_packs
    w = W.ring_stack(n_packs=n, n_steps=0, seed=3, precision=0)
    w.fields.gas_p[:] = 0.0
    w.source.radius = 2.0e-3
    ctx = mucite.Context(local, stream)
    ctx.set_tuning(1, args.streamed_threads)
    ctx.set_launch_mode(args.streamed_persistent, True)
    mucite.load_workload(ctx, w, 0)
    K = 50
    # warm-up with the timed call's shape: the macro-step graph is captured
    # and instantiated here, not inside the timed region
    for _ in range(2):
        ctx.step(0, K)
    torch.cuda.synchronize(dev)
    T0 = ctx.tally(0)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    ctx.step(0, K)
    b.record(stream)
    torch.cuda.synchronize(dev)
    T1 = ctx.tally(0)
    ms = a.elapsed_time(b)
    ps = T1["pack_steps"] - T0["pack_steps"]
    layout = mucite.state_layout(mucite.FP32, n)
    ctx.close()
    rate = ps / (ms * 1e-3)
    gbs = 49.0 * rate / 1e9
    return {"value": rate, "unit": UNIT, "packs": n, "launches": K, "ms": ms,
            "threads": args.streamed_threads, "persistent_blocks_per_sm": args.streamed_persistent,
            "pool_bytes": int(layout.total_bytes), "bytes_per_pack_step": 49,
            "achieved_gbs": gbs, "peak_gbs": peaks["hbm_gbs"], "frac": gbs / peaks["hbm_gbs"],
            "note": "K=1 launches (graph replays of RF table + step + clock advance), no gas (push, gather, "
                    "classify), pool larger than L2"}


def _sweep(args, local, stream, dev):
    """Batched sweep (64 operating points of the ring stack: RF amplitude x DC
    gradient x inlet pressure, pack counts log-uniform in [1e4, 5e5], seeds
    100-163), each instance with its own 128 x 512 PIC grid updated every 10
    micro steps, advanced together by graph-replayed macro steps in the
    launch shape the autotuner picks."""
    import dataclasses
    import torch
    from paper_2609_31258_b300 import mucite, workloads as W
    g = W.Grid(512, 2048, 5e-3, 0.0, 40e-3)
    pic = W.Grid(128, 512, 5e-3, 0.0, 40e-3)
    f = W.ring_stack_fields(g, p_in=1000.0, pic=pic)
    base = W.ring_stack(n_packs=1, n_steps=0)
    pts = W.sweep_points(args.sweep_instances)
    ctx = mucite.Context(local, stream)
    if args.pic_direct:
        ctx.set_launch_mode(0, False)
    ctx.load_fields(f)
    for i, pt in enumerate(pts):
        run = dataclasses.replace(base.run, v_rf=pt["v_rf"], dc_scale=pt["dc_scale"], p_scale=pt["p_scale"],
                                  seed=pt["seed"], pic_interval=10)
        ctx.inject(i, base.ion, dataclasses.replace(base.source, n_initial=pt["n_packs"]), run)
    inst = list(range(len(pts)))
    tuning = ctx.autotune(inst, args.sweep_tune_steps) if args.sweep_tune_steps > 0 else None
    ctx.step(-1, 200)
    torch.cuda.synchronize(dev)
    p0 = sum(ctx.tally(i)["pack_steps"] for i in inst)
    K = args.sweep_steps
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    ctx.step(-1, K)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b)
    ps = sum(ctx.tally(i)["pack_steps"] for i in inst) - p0
    ctx.close()
    return {"value": ps / (ms * 1e-3), "unit": UNIT, "instances": len(pts),
            "packs": int(sum(pt["n_packs"] for pt in pts)), "micro_steps": K, "ms": ms,
            "pic": "128x512 per instance, every 10 micro steps", "tuning": tuning,
            "note": "macro step = batched PIC update of all instances + one launch of 10 micro steps per instance "
                    "(side by side on the context's step streams), "
                    "graph-replayed"}


def _space_charge(args, local, stream, dev):
    """Cylinder with PIC space charge: 1e6 packs of 1 kDa/+1 (W = 1e3) in a
    uniform axial field and 200 Pa N2, 256 x 1024 PIC grid updated every 10
    micro steps (deposit, DST/tridiagonal solve with FP64 refinement to 1e-6,
    E_SCE), continuous source; macro steps graph-replayed. The PIC share is
    one minus the time of the same run without space charge over the time
    with it."""
    import dataclasses
    import torch
    from paper_2609_31258_b300 import mucite, workloads as W
    w = W.cylinder_space_charge(n_packs=args.pic_packs, n_steps=0, precision=0)
    K = args.pic_steps

    def timed(run, solver=mucite.DST_SIMT):
        ctx = mucite.Context(local, stream)
        if args.pic_direct:
            ctx.set_launch_mode(0, False)
        ctx.load_fields(w.fields)
        if run.pic_interval:
            ctx.set_pic_solver(solver)
        ctx.inject(0, w.ion, w.source, run, capacity=args.pic_packs + 100_000)
        # the library's autotuner picks the launch shape (state restored after)
        tuning = None if args.no_autotune else ctx.autotune([0], 200)
        ctx.step(0, K)  # warm-up of the timed call's shape (graph capture)
        torch.cuda.synchronize(dev)
        T0 = ctx.tally(0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.step(0, K)
        b.record(stream)
        torch.cuda.synchronize(dev)
        T1 = ctx.tally(0)
        pr = ctx.pic_read(0) if run.pic_interval else {}
        rel = (pr.get("rel_residual"), pr.get("iterations"))
        ctx.close()
        return a.elapsed_time(b), T1["pack_steps"] - T0["pack_steps"], rel, tuning

    ms, ps, rel, tuning = timed(w.run)
    ms0, _, _, _ = timed(dataclasses.replace(w.run, pic_interval=0))
    # the same run with the DST-I contractions on the tensor cores (TF32 pairs)
    ms_tc, ps_tc, rel_tc, _ = timed(w.run, mucite.DST_TENSOR_CORES)
    upd = K // w.run.pic_interval
    return {"value": ps / (ms * 1e-3), "unit": UNIT, "packs": args.pic_packs, "micro_steps": K, "ms": ms,
            "pic_updates": upd, "ms_without_space_charge": ms0,
            "ms_per_pic_update": (ms - ms0) / upd, "pic_share": 1.0 - ms0 / ms,
            "last_rel_residual": rel[0], "last_iterations": rel[1], "pic_grid": "256x1024",
            "dst_contraction": "SIMT FP32 (default)",
            "tensor_core_dst": {"value": ps_tc / (ms_tc * 1e-3), "ms": ms_tc, "ms_per_pic_update": (ms_tc - ms0) / upd,
                                "pic_share": 1.0 - ms0 / ms_tc, "last_rel_residual": rel_tc[0],
                                "last_iterations": rel_tc[1],
                                "note": "tcgen05 kind::tf32 contractions with TF32-pair operands (mucite_set_pic_solver)"},
            "launch": "direct (fixed solve passes)" if args.pic_direct else "graph-replayed macro steps",
            "tuning": tuning}


def _paper_grid(args, local, stream, dev):
    """Fused FP32 step on a static grid of the paper's S-lens size (2001 x
    6501 nodes, 468 MB of node records and mask: the gathers are served from
    HBM through L2 rather than from an L2-resident table), 100,000 packs
    filling the guide, 2000 micro steps per launch."""
    import torch
    from paper_2609_31258_b300 import mucite, workloads as W
    w = W.paper_grid(n_packs=args.packs)
    ctx = mucite.Context(local, stream)
    ctx.set_tuning(2000, 256)
    mucite.load_workload(ctx, w, 0)
    for _ in range(2):
        ctx.step(0, 2000)
    torch.cuda.synchronize(dev)
    T0 = ctx.tally(0)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        ctx.step(0, 2000)
    b.record(stream)
    torch.cuda.synchronize(dev)
    T1 = ctx.tally(0)
    ctx.close()
    ms = a.elapsed_time(b)
    ps = T1["pack_steps"] - T0["pack_steps"]
    # HBM roofline of the launch: DRAM bytes per launch from the committed
    # ncu summary of the same launch (null once the kernel's sources change)
    prof, stale = _profile_fields("step_f32_paper_grid.txt")
    peak = _peaks()[0]["hbm_gbs"]
    launch_ms = ms / args.steps
    traffic = None if stale or "dram_bytes_per_launch" not in prof else float(prof["dram_bytes_per_launch"])
    ach = traffic / (launch_ms * 1e-3) / 1e9 if traffic else None
    roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak if ach else None,
            "traffic": traffic, "kernel_ms_per_launch": launch_ms, "pack_steps_per_launch": ps / args.steps,
            "dram_bytes_per_pack_step": traffic / (ps / args.steps) if traffic else None, "profile_stale": stale,
            "note": "DRAM bytes of the node gathers and of the pack state per launch: the packs' neighbourhood of the "
                    "468 MB table stays in L2 (99 % L2 hits in the ncu summary), so the launch is issue-bound like "
                    "the ring-stack launch and this fraction is far below 1"}
    return {"value": ps / (ms * 1e-3), "unit": UNIT, "grid": "2001x6501", "packs": args.packs,
            "micro_steps": 2000 * args.steps, "ms": ms,
            "collisions_per_pack_step": (T1["collisions"] - T0["collisions"]) / max(ps, 1), "roofline": roof}


def _serving(args, local):
    """Serving loop on the ring-stack geometry: Poisson arrivals at 20 / s,
    pack counts log-uniform in [1e4, 2e6], three ion templates, 50 us
    (1e5 micro steps) per request, the first --serve-requests arrivals
    (default 200). The offered load exceeds the capacity at 20 / s, so the
    latency there is queue dominated. Then the highest sustainable arrival
    rate is searched on the first --serve-search-requests arrivals, their
    arrival times stretched: starting just below the capacity the first run
    measured, the rate is lowered until the latency stops growing with the
    run (the mean latency of the last third of the requests within 1.5 x
    that of the first third plus the requests' mean service time alone)."""
    import numpy as np
    import torch
    from paper_2609_31258_b300 import mucite, serving, workloads as W
    base = W.ring_stack(n_packs=1, n_steps=0, precision=0)
    t, n, tmpl = W.serving_arrivals(n_req=args.serve_requests, rate_hz=20.0, seed=5)
    dev = torch.device("cuda", local)

    def once(rate, count):
        arr = t * (20.0 / rate)
        reqs = [serving.make_request(i, arr[i], int(n[i]), W.SERVING_TEMPLATES[int(tmpl[i])], base,
                                     n_steps=args.serve_steps, seed=1000 + i) for i in range(count)]
        # a non-default stream: the batched macro steps are graph-captured and replayed
        ctx = mucite.Context(local, torch.cuda.Stream(dev))
        ctx.set_tuning(2000, 256)
        ctx.load_fields(base.fields)
        srv = serving.Server(ctx, max_slots=64, chunk=4000, policy=args.serve_policy)
        torch.cuda.synchronize()
        done, wall = srv.run(reqs)
        replays, captures = ctx.graph_stats()
        launches = ctx.launch_count()
        ctx.close()
        lat = serving.latency_summary(done)
        work = sum(r.tally["pack_steps"] for r in done)
        by_arrival = sorted(done, key=lambda r: r.arrival)
        third = max(1, len(by_arrival) // 3)
        first = float(np.mean([r.latency for r in by_arrival[:third]]))
        last = float(np.mean([r.latency for r in by_arrival[-third:]]))
        return {"requests": len(done), "arrival_rate_hz": rate, "policy": args.serve_policy,
                "p50_latency_s": lat["p50_s"], "p99_latency_s": lat["p99_s"], "mean_latency_s": lat.get("mean_s"),
                "mean_latency_first_third_s": first, "mean_latency_last_third_s": last,
                "wall_s": wall, "pack_steps": int(work), "throughput": work / wall, "unit": UNIT,
                "graph_replays": replays, "graph_captures": captures, "gpu_launches": launches}

    first = once(20.0, args.serve_requests)
    first.update({"micro_steps_per_request": args.serve_steps, "packs": [int(x) for x in n],
                  "templates": [int(x) for x in tmpl],
                  "note": "offered load exceeds capacity at 20 / s: latency is queue dominated"})
    if args.serve_search_requests <= 0:
        return first
    m = min(args.serve_search_requests, len(n))
    # capacity in requests / s of the first m requests at the throughput measured above
    work_m = float(np.sum(n[:m])) * args.serve_steps
    cap = first["throughput"] / (work_m / m)
    service = work_m / m / first["throughput"]  # mean service time of a request alone at full throughput
    trials = []
    frac = 0.9
    best = None
    while frac >= 0.3 and len(trials) < args.serve_search_trials:
        r = once(frac * cap, m)
        ok = r["mean_latency_last_third_s"] <= 1.5 * r["mean_latency_first_third_s"] + service
        r.update({"fraction_of_capacity": frac, "bounded": bool(ok)})
        trials.append({k: r[k] for k in ("arrival_rate_hz", "fraction_of_capacity", "bounded", "p50_latency_s",
                                         "p99_latency_s", "mean_latency_first_third_s", "mean_latency_last_third_s",
                                         "wall_s")})
        if ok:
            best = r
            break
        frac -= 0.2
    first["capacity_req_per_s"] = cap
    first["sustainable_search"] = trials
    if best is not None:
        best["note"] = (f"highest bounded rate tried: first {m} arrivals stretched to {best['arrival_rate_hz']:.3f} / s "
                        f"({best['fraction_of_capacity']:.0%} of the measured capacity)")
        first["sustainable"] = best
    return first


def _fp64(args, w32, local, stream, dev):
    import torch
    from paper_2609_31258_b300 import mucite, workloads as W
    w = W.ring_stack(n_packs=args.packs, n_steps=0, seed=w32.run.seed, precision=1)
    ctx = mucite.Context(local, stream)
    mucite.load_workload(ctx, w, 0)
    micro = max(100, args.micro // 4)
    for _ in range(2):
        ctx.step(0, micro)
    torch.cuda.synchronize(dev)
    T0 = ctx.tally(0)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.fp64_steps):
        ctx.step(0, micro)
    b.record(stream)
    torch.cuda.synchronize(dev)
    T1 = ctx.tally(0)
    ms = a.elapsed_time(b)
    ps = T1["pack_steps"] - T0["pack_steps"]
    ctx.close()
    value = ps / (ms * 1e-3)
    # FP64 rate of the plain step: FP64 flops per pack-step (DADD + DMUL +
    # 2 DFMA, counted by ncu on the same launch) times the measured rate,
    # against the part's nominal FP64 peak (null once the kernel's sources
    # change after the summary was taken)
    prof, stale = _profile_fields("step_f64_ring_stack.txt", "step_fp64.cu")
    fpp = None if stale or "fp64_flop_per_pack_step" not in prof else float(prof["fp64_flop_per_pack_step"])
    ach = fpp * value / 1e9 if fpp else None
    roof = {"bound": "fp64", "achieved": ach, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
            "frac": ach / FP64_PEAK_GFLOPS if ach else None, "peak_source": "nominal B300 FP64 (no measured figure)",
            "fp64_flop_per_pack_step": fpp,
            "fp64_pipe_active": prof.get("sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active") if not stale else None,
            "profile_stale": stale}
    return {"value": value, "unit": UNIT, "micro_steps_timed": micro * args.fp64_steps,
            "ms": ms, "note": "one launch per micro step, FP64 state and fields", "roofline": roof}


if __name__ == "__main__":
    main()
