"""Thin Python binding of the C ABI in include/mucite.h.

Argument marshalling only: every step of the method runs in the CUDA library
(libmucite.so, built in-tree for sm_103a). PyTorch supplies the device pack
pool and the stream. Importing this module does not need a GPU; creating a
Context does, and fails loudly when the library or the device is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmucite.so")

OK, E_ARG, E_OOM, E_CUDA, E_OVERFLOW, E_STATE, E_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
FP32, FP64 = 0, 1
ACTIVE, TRANSMITTED, ELECTRODE, RADIAL, AXIAL, EMPTY = 0, 1, 2, 3, 4, 255
MAX_INSTANCES = 256

EXPORTS = ["mucite_create", "mucite_destroy", "mucite_last_error", "mucite_load_fields",
           "mucite_state_layout", "mucite_inject", "mucite_release", "mucite_resume", "mucite_step",
           "mucite_step_set", "mucite_autotune",
           "mucite_pic_update", "mucite_tally", "mucite_pic_read", "mucite_set_tuning", "mucite_set_launch_mode",
           "mucite_launch_count", "mucite_sync", "mucite_poisson_solve_noalloc", "mucite_set_dt",
           "mucite_dt_limits", "mucite_graph_stats", "mucite_set_pic_solver", "mucite_set_schedule",
           "mucite_test_hook"]
HOOK_HOLD_STAGED_COPY = 1
DST_SIMT, DST_TENSOR_CORES = 0, 1
SCHEDULE_BALANCED, SCHEDULE_EAGER = 1, 6


class MuciteError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"mucite status {status}: {msg}")
        self.status = status


class Grid(C.Structure):
    _fields_ = [("nr", C.c_int32), ("nz", C.c_int32), ("R", C.c_double), ("z0", C.c_double),
                ("z1", C.c_double)]


class IonTemplate(C.Structure):
    _fields_ = [("mass_da", C.c_double), ("charge", C.c_int32), ("ccs_m2", C.c_double),
                ("n_atoms", C.c_double), ("cv_c0", C.c_double), ("cv_c1", C.c_double),
                ("T_init", C.c_double), ("dH_kJmol", C.c_double), ("dS_JmolK", C.c_double)]


class Source(C.Structure):
    _fields_ = [("profile", C.c_int32), ("z_plane", C.c_double), ("radius", C.c_double),
                ("sigma", C.c_double), ("T_vel", C.c_double), ("half_space", C.c_int32),
                ("n_initial", C.c_int64), ("prefill_z0", C.c_double), ("prefill_z1", C.c_double),
                ("current_A", C.c_double), ("weight", C.c_int64)]


class Run(C.Structure):
    _fields_ = [("dt", C.c_double), ("v_rf", C.c_double), ("f_rf", C.c_double), ("phi_rf", C.c_double),
                ("dc_scale", C.c_double), ("p_scale", C.c_double), ("hit_dist", C.c_double),
                ("z_exit", C.c_double), ("r_det", C.c_double), ("m_gas_da", C.c_double),
                ("seed", C.c_uint64), ("precision", C.c_int32), ("pic_interval", C.c_int32),
                ("exit_bin_steps", C.c_int32), ("n_exit_bins", C.c_int32), ("n_r_bins", C.c_int32),
                ("n_ke_bins", C.c_int32), ("n_teff_bins", C.c_int32), ("n_loss_r", C.c_int32),
                ("n_loss_z", C.c_int32), ("ke_max_ev", C.c_double), ("teff_max", C.c_double),
                ("langevin", C.c_int32), ("lv_z0", C.c_double), ("lv_z1", C.c_double), ("lv_switch", C.c_double),
                ("pic_masked", C.c_int32), ("integrator", C.c_int32)]


class Layout(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("off_x", "off_y", "off_z", "off_vx", "off_vy", "off_vz",
                                         "off_eint", "off_status", "off_t_term", "off_lnsy", "off_tau",
                                         "total_bytes")] + \
               [("pos_bytes", C.c_int32), ("vel_bytes", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("steps_per_launch", C.c_int32), ("threads_per_block", C.c_int32),
                ("persistent_blocks_per_sm", C.c_int32), ("schedule", C.c_int32), ("n_tried", C.c_int32),
                ("best_ms_per_step", C.c_double)]


_i64p = C.POINTER(C.c_int64)


class TallyOut(C.Structure):
    _fields_ = [("count", C.c_int64 * 8), ("weight", C.c_int64 * 8), ("sum_w_ke", C.c_double * 8),
                ("sum_w_teff", C.c_double * 8), ("sum_w_sy", C.c_double * 8), ("emitted_count", C.c_int64),
                ("emitted_weight", C.c_int64), ("pack_steps", C.c_int64), ("collisions", C.c_int64),
                ("candidate_overflow", C.c_int64), ("step", C.c_int64), ("exit_hist", _i64p),
                ("r_hist", _i64p), ("ke_hist", _i64p), ("teff_hist", _i64p), ("loss_map", _i64p)]


_lib = None


def lib():
    """The loaded CUDA library. Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2609_31258_b300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, dp = C.c_void_p, C.POINTER(C.c_double)
        L.mucite_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, vp]
        L.mucite_destroy.argtypes = [vp]
        L.mucite_destroy.restype = None
        L.mucite_last_error.argtypes = [vp]
        L.mucite_last_error.restype = C.c_char_p
        L.mucite_load_fields.argtypes = [vp, C.POINTER(Grid)] + [dp] * 6 + [C.POINTER(C.c_uint8), dp,
                                                                          C.POINTER(Grid)]
        L.mucite_state_layout.argtypes = [C.c_int, C.c_int64, C.POINTER(Layout)]
        L.mucite_inject.argtypes = [vp, C.c_int, C.POINTER(IonTemplate), C.POINTER(Source), C.POINTER(Run),
                                    vp, C.c_int64]
        L.mucite_release.argtypes = [vp, C.c_int]
        L.mucite_resume.argtypes = [vp, C.c_int, C.c_int64, C.c_int64]
        L.mucite_step.argtypes = [vp, C.c_int, C.c_int]
        L.mucite_step_set.argtypes = [vp, C.POINTER(C.c_int), C.c_int, C.c_int]
        L.mucite_autotune.argtypes = [vp, C.POINTER(C.c_int), C.c_int, C.c_int, C.POINTER(Tuning)]
        L.mucite_pic_update.argtypes = [vp, C.c_int]
        L.mucite_tally.argtypes = [vp, C.c_int, C.POINTER(TallyOut)]
        L.mucite_pic_read.argtypes = [vp, C.c_int, _i64p, dp, C.POINTER(C.c_float), C.POINTER(C.c_float), dp,
                                      C.POINTER(C.c_int32)]
        L.mucite_set_tuning.argtypes = [vp, C.c_int, C.c_int]
        L.mucite_set_launch_mode.argtypes = [vp, C.c_int, C.c_int]
        L.mucite_launch_count.argtypes = [vp]
        L.mucite_launch_count.restype = C.c_int64
        L.mucite_sync.argtypes = [vp]
        L.mucite_graph_stats.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.mucite_set_pic_solver.argtypes = [vp, C.c_int]
        L.mucite_set_schedule.argtypes = [vp, C.c_int]
        L.mucite_test_hook.argtypes = [vp, C.c_int, C.c_int]
        L.mucite_poisson_solve_noalloc.argtypes = [C.c_int, vp, C.POINTER(Grid), vp, vp, vp, vp]
        L.mucite_set_dt.argtypes = [vp, C.c_int, C.c_double]
        L.mucite_dt_limits.argtypes = [vp, C.c_int, dp]
        _lib = L
    return _lib


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def grid_struct(g):
    return Grid(g.nr, g.nz, g.R, g.z0, g.z1)


def ion_struct(ion):
    return IonTemplate(ion.mass_da, int(ion.charge), ion.ccs_m2, float(ion.n_atoms), ion.cv_c0, ion.cv_c1,
                       ion.T_init, ion.dH_kJmol, ion.dS_JmolK)


def source_struct(src):
    return Source(src.profile, src.z_plane, src.radius, src.sigma, src.T_vel, src.half_space,
                  int(src.n_initial), src.prefill_z0, src.prefill_z1, src.current_A, int(src.weight))


def run_struct(run):
    return Run(run.dt, run.v_rf, run.f_rf, run.phi_rf, run.dc_scale, run.p_scale, run.hit_dist, run.z_exit,
               run.r_det, run.m_gas_da, run.seed & 0xFFFFFFFFFFFFFFFF, run.precision, run.pic_interval,
               run.exit_bin_steps, run.n_exit_bins, run.n_r_bins, run.n_ke_bins, run.n_teff_bins,
               run.n_loss_r, run.n_loss_z, run.ke_max_ev, run.teff_max, int(run.langevin), run.lv_z0, run.lv_z1,
               run.lv_switch, int(run.pic_masked), int(run.integrator))


def state_layout(precision, capacity):
    L = Layout()
    st = lib().mucite_state_layout(precision, capacity, C.byref(L))
    if st != OK:
        raise MuciteError(st, "bad layout request")
    return L


class Context:
    """One library context bound to a CUDA device and a torch stream."""

    def __init__(self, device=0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("mucite needs a CUDA device; none is visible")
        self.torch = torch
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self._p = C.c_void_p()
        st = lib().mucite_create(C.byref(self._p), device, C.c_void_p(self.stream.cuda_stream))
        if st != OK:
            raise MuciteError(st, lib().mucite_last_error(None).decode())
        self.pools = {}
        self.meta = {}
        self.grid = None

    def _check(self, st):
        if st != OK:
            raise MuciteError(st, lib().mucite_last_error(self._p).decode())

    def close(self):
        if self._p:
            lib().mucite_destroy(self._p)
            self._p = C.c_void_p()
        self.pools.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- calls with the C names ------------------------------------------------
    def load_fields(self, fields):
        g = grid_struct(fields.grid)
        keep = [_f64(a) for a in (fields.phi_dc, fields.phi_rf, fields.gas_p, fields.gas_T, fields.gas_ur,
                                  fields.gas_uz)]
        mask = np.ascontiguousarray(fields.mask, dtype=np.uint8)
        dist = _f64(fields.dist)
        pic = C.byref(grid_struct(fields.pic)) if fields.pic is not None else None
        self._check(lib().mucite_load_fields(self._p, C.byref(g), *[k[1] for k in keep],
                                             mask.ctypes.data_as(C.POINTER(C.c_uint8)), dist[1], pic))
        self.grid = fields.grid
        self.pic_grid = fields.pic

    def inject(self, instance, ion, source, run, capacity=None):
        torch = self.torch
        cap = int(capacity if capacity is not None else max(source.n_initial, 1))
        lay = state_layout(run.precision, cap)
        buf = torch.empty(lay.total_bytes + 256, dtype=torch.uint8, device=f"cuda:{self.device}")
        off = (-buf.data_ptr()) % 256
        pool = buf[off:off + lay.total_bytes]
        self._check(lib().mucite_inject(self._p, instance, C.byref(ion_struct(ion)),
                                        C.byref(source_struct(source)), C.byref(run_struct(run)),
                                        C.c_void_p(pool.data_ptr()), cap))
        self.pools[instance] = (buf, pool, lay)
        import copy
        self.meta[instance] = dict(run=copy.copy(run), ion=ion, source=source, capacity=cap)
        return pool

    def release(self, instance):
        self._check(lib().mucite_release(self._p, instance))
        self.pools.pop(instance, None)
        self.meta.pop(instance, None)

    def resume(self, instance, n_slots, step):
        self._check(lib().mucite_resume(self._p, instance, int(n_slots), int(step)))

    def step(self, instance, n_steps):
        self._check(lib().mucite_step(self._p, instance, int(n_steps)))

    def step_set(self, instances, n_steps):
        """Advance the listed instances together (one batched launch per chunk)."""
        arr = (C.c_int * len(instances))(*[int(i) for i in instances])
        self._check(lib().mucite_step_set(self._p, arr, len(instances), int(n_steps)))

    def autotune(self, instances, trial_steps):
        """Time the candidate launch shapes on the listed instances (state
        restored afterwards) and apply the fastest; returns the choice."""
        arr = (C.c_int * len(instances))(*[int(i) for i in instances])
        t = Tuning()
        self._check(lib().mucite_autotune(self._p, arr, len(instances), int(trial_steps), C.byref(t)))
        return {k: getattr(t, k) for k, _ in Tuning._fields_}

    def pic_update(self, instance):
        self._check(lib().mucite_pic_update(self._p, instance))

    def tally(self, instance):
        run = self.meta[instance]["run"]
        out = dict(exit_hist=np.zeros(run.n_exit_bins, np.int64), r_hist=np.zeros(run.n_r_bins, np.int64),
                   ke_hist=np.zeros(run.n_ke_bins, np.int64), teff_hist=np.zeros(run.n_teff_bins, np.int64),
                   loss_map=np.zeros((run.n_loss_z, run.n_loss_r), np.int64))
        T = TallyOut()
        for k in ("exit_hist", "r_hist", "ke_hist", "teff_hist", "loss_map"):
            setattr(T, k, out[k].ctypes.data_as(_i64p))
        self._check(lib().mucite_tally(self._p, instance, C.byref(T)))
        out["count"] = np.array(T.count[:], np.int64)
        out["weight"] = np.array(T.weight[:], np.int64)
        out["sum_w_ke"] = np.array(T.sum_w_ke[:])
        out["sum_w_teff"] = np.array(T.sum_w_teff[:])
        out["sum_w_sy"] = np.array(T.sum_w_sy[:])
        for k in ("emitted_count", "emitted_weight", "pack_steps", "collisions", "candidate_overflow", "step"):
            out[k] = int(getattr(T, k))
        return out

    def pic_read(self, instance):
        pg = self.pic_grid
        shape = (pg.nz, pg.nr)
        Q = np.zeros(shape, np.int64)
        phi = np.zeros(shape)
        er = np.zeros(shape, np.float32)
        ez = np.zeros(shape, np.float32)
        rel = C.c_double()
        its = C.c_int32()
        self._check(lib().mucite_pic_read(self._p, instance, Q.ctypes.data_as(_i64p),
                                          phi.ctypes.data_as(C.POINTER(C.c_double)),
                                          er.ctypes.data_as(C.POINTER(C.c_float)),
                                          ez.ctypes.data_as(C.POINTER(C.c_float)), C.byref(rel), C.byref(its)))
        return dict(Q=Q, phi=phi, er=er, ez=ez, rel_residual=rel.value, iterations=its.value)

    def set_tuning(self, steps_per_launch=0, threads_per_block=0):
        self._check(lib().mucite_set_tuning(self._p, int(steps_per_launch), int(threads_per_block)))

    def set_dt(self, instance, dt):
        self._check(lib().mucite_set_dt(self._p, instance, float(dt)))
        self.meta[instance]["run"].dt = dt

    def dt_limits(self, instance):
        out = (C.c_double * 6)()
        self._check(lib().mucite_dt_limits(self._p, instance, out))
        return np.array(out[:])

    def set_launch_mode(self, persistent_blocks_per_sm=0, use_graphs=True):
        self._check(lib().mucite_set_launch_mode(self._p, int(persistent_blocks_per_sm), int(bool(use_graphs))))

    def launch_count(self):
        return int(lib().mucite_launch_count(self._p))

    def sync(self):
        self._check(lib().mucite_sync(self._p))

    def set_pic_solver(self, contraction):
        """DST_SIMT (default) or DST_TENSOR_CORES for the space-charge solve's
        contractions; after load_fields, before injecting instances."""
        self._check(lib().mucite_set_pic_solver(self._p, int(contraction)))

    def set_schedule(self, schedule):
        """SCHEDULE_BALANCED (default) or SCHEDULE_EAGER for the collision loop
        of the per-instance collision launches (results do not depend on it)."""
        self._check(lib().mucite_set_schedule(self._p, int(schedule)))

    def test_hook(self, hook, value):
        """Failure-path test hook (see include/mucite.h); not for production runs."""
        self._check(lib().mucite_test_hook(self._p, int(hook), int(value)))

    def graph_stats(self):
        """(macro-step graphs replayed, graphs captured) since creation."""
        r, c = C.c_int64(), C.c_int64()
        self._check(lib().mucite_graph_stats(self._p, C.byref(r), C.byref(c)))
        return int(r.value), int(c.value)

    # -- views of a pack pool -------------------------------------------------
    def pool(self, instance):
        """torch uint8 view (no copy) of the instance's whole pool: the buffer
        whose layout mucite_state_layout gives, for copies of the whole state."""
        return self.pools[instance][1]

    def state(self, instance):
        """torch views (no copy) of the instance's structure-of-arrays pool."""
        torch = self.torch
        buf, pool, L = self.pools[instance]
        cap = self.meta[instance]["capacity"]
        pt = torch.int32 if L.pos_bytes == 4 else torch.float64
        vt = torch.float32 if L.vel_bytes == 4 else torch.float64
        ps, vs = L.pos_bytes, L.vel_bytes

        def v(off, n, dt):
            return pool[off:off + n].view(dt)

        return dict(x=v(L.off_x, cap * ps, pt), y=v(L.off_y, cap * ps, pt), z=v(L.off_z, cap * ps, pt),
                    vx=v(L.off_vx, cap * vs, vt), vy=v(L.off_vy, cap * vs, vt), vz=v(L.off_vz, cap * vs, vt),
                    eint=v(L.off_eint, cap * vs, vt), status=v(L.off_status, cap, torch.uint8),
                    t_term=v(L.off_t_term, cap * 4, torch.int32), lnsy=v(L.off_lnsy, cap * vs, vt),
                    tau=v(L.off_tau, cap * vs, vt))


def poisson_solve_noalloc(device, stream, pic, Q, phi, esc, rel=None):
    """Allocation-free space-charge solve on caller-provided device tensors:
    Q int64 [nz][nr] (input), phi float64 [nz][nr] and esc float32
    [nz][nr][2] (outputs), rel float64 [1] (optional output)."""
    g = grid_struct(pic)
    ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
    st = lib().mucite_poisson_solve_noalloc(device, C.c_void_p(stream.cuda_stream), C.byref(g), ptr(Q),
                                            ptr(phi), ptr(esc), ptr(rel))
    if st != OK:
        raise MuciteError(st, "mucite_poisson_solve_noalloc failed")


def load_workload(ctx, workload, instance=0, capacity=None):
    """Load a workload's fields (if not loaded) and inject its instance."""
    if ctx.grid is None:
        ctx.load_fields(workload.fields)
    return ctx.inject(instance, workload.ion, workload.source, workload.run, capacity)
