"""FP64 CPU oracle of the MuCITE ion-pack step.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check
and by the benchmark's CPU-baseline leg, never by the product path. It shares
no code with the CUDA library; both take their inputs from the seeded
generators in `paper_2609_31258_b300.workloads`, which hold none of the
method's arithmetic.

`mucite_oracle.c` holds the per-pack arithmetic (Philox, gather, collisions,
push, classification, deposit, tallies); `poisson.py` the finite-volume
cylindrical Poisson operator and its direct solve. Each function cites the
passage of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mucite_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

ACTIVE, TRANSMITTED, ELECTRODE, RADIAL, AXIAL, EMPTY = 0, 1, 2, 3, 4, 255
E_CHARGE = 1.602176634e-19
K_B = 1.380649e-23
DALTON = 1.66053906660e-27


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no contraction into FMA, OpenMP over
    packs)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(_LIB)
        _declare(_lib)
    return _lib


# --------------------------------------------------------------------------
# ctypes mirrors of the oracle's own structs
# --------------------------------------------------------------------------
_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_u8p = C.POINTER(C.c_uint8)
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)


class OrcFields(C.Structure):
    _fields_ = [("nr", C.c_int), ("nz", C.c_int), ("R", C.c_double), ("z0", C.c_double),
                ("z1", C.c_double), ("er_dc", _dp), ("ez_dc", _dp), ("er_rf", _dp), ("ez_rf", _dp),
                ("gas_p", _dp), ("gas_T", _dp), ("gas_ur", _dp), ("gas_uz", _dp), ("dmask", _fp),
                ("pnr", C.c_int), ("pnz", C.c_int), ("er_sc", _dp), ("ez_sc", _dp)]


class OrcIon(C.Structure):
    _fields_ = [("mass_da", C.c_double), ("charge", C.c_double), ("ccs_m2", C.c_double),
                ("n_atoms", C.c_double), ("cv_c0", C.c_double), ("cv_c1", C.c_double),
                ("T_init", C.c_double), ("dH_kJmol", C.c_double), ("dS_JmolK", C.c_double)]


class OrcSource(C.Structure):
    _fields_ = [("profile", C.c_int), ("z_plane", C.c_double), ("radius", C.c_double),
                ("sigma", C.c_double), ("T_vel", C.c_double), ("half_space", C.c_int),
                ("prefill_z0", C.c_double), ("prefill_z1", C.c_double)]


class OrcRun(C.Structure):
    _fields_ = [("dt", C.c_double), ("v_rf", C.c_double), ("f_rf", C.c_double),
                ("phi_rf", C.c_double), ("dc_scale", C.c_double), ("p_scale", C.c_double),
                ("hit_dist", C.c_double), ("z_exit", C.c_double), ("r_det", C.c_double),
                ("m_gas_da", C.c_double), ("seed", C.c_uint64), ("langevin", C.c_int),
                ("lv_z0", C.c_double), ("lv_z1", C.c_double), ("lv_switch", C.c_double),
                ("integrator", C.c_int), ("rf_phase0", C.c_double), ("seg_step0", C.c_int64)]


class OrcState(C.Structure):
    _fields_ = [("x", _dp), ("y", _dp), ("z", _dp), ("vx", _dp), ("vy", _dp), ("vz", _dp),
                ("eint", _dp), ("status", _u8p), ("t_term", _i32p), ("ncoll", _i64p),
                ("nsteps", _i64p), ("noverflow", _i64p), ("lnsy", _dp), ("tau", _dp)]


class OrcTally(C.Structure):
    _fields_ = [("count", C.c_int64 * 8), ("weight", C.c_int64 * 8), ("sum_w_ke", C.c_double * 8),
                ("sum_w_teff", C.c_double * 8), ("sum_w_sy", C.c_double * 8), ("exit_hist", _i64p), ("r_hist", _i64p),
                ("ke_hist", _i64p), ("teff_hist", _i64p), ("loss_map", _i64p)]


class OrcTallySpec(C.Structure):
    _fields_ = [("exit_bin_steps", C.c_int), ("n_exit_bins", C.c_int), ("n_r_bins", C.c_int),
                ("n_ke_bins", C.c_int), ("n_teff_bins", C.c_int), ("n_loss_r", C.c_int),
                ("n_loss_z", C.c_int), ("ke_max_ev", C.c_double), ("teff_max", C.c_double)]


def _declare(L):
    P = C.POINTER
    L.orc_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
    L.orc_uniforms.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, _dp]
    L.orc_eint_of_T.argtypes = [P(OrcIon), C.c_double]
    L.orc_eint_of_T.restype = C.c_double
    L.orc_T_of_eint.argtypes = [P(OrcIon), C.c_double]
    L.orc_T_of_eint.restype = C.c_double
    L.orc_cv_of_T.argtypes = [P(OrcIon), C.c_double]
    L.orc_cv_of_T.restype = C.c_double
    L.orc_eyring_rate.argtypes = [P(OrcIon), C.c_double]
    L.orc_eyring_rate.restype = C.c_double
    L.orc_efield_from_phi.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp, _dp]
    L.orc_rf_scalar.argtypes = [P(OrcRun), C.c_int64]
    L.orc_rf_scalar.restype = C.c_double
    L.orc_dt_limits.argtypes = [P(OrcFields), P(OrcIon), P(OrcRun), P(OrcState), C.c_int64, C.c_int64, _dp]
    L.orc_quantize.argtypes = [C.c_double] * 6 + [_i32p, _i32p, _i32p]
    L.orc_classify_fixed.argtypes = [P(OrcFields), P(OrcRun), C.c_int64, _i32p, _i32p, _i32p, _u8p]
    L.orc_run_steps.argtypes = [P(OrcFields), P(OrcIon), P(OrcRun), P(OrcState), C.c_int64,
                                C.c_int64, C.c_int64, C.c_int]
    L.orc_count_collisions_frozen.argtypes = [P(OrcIon), P(OrcRun), C.c_double, C.c_double, _dp,
                                              _dp, C.c_int64]
    L.orc_count_collisions_frozen.restype = C.c_int64
    L.orc_one_minus_beta.argtypes = [C.c_double, C.c_double, C.c_double]
    L.orc_one_minus_beta.restype = C.c_double
    L.orc_inject.argtypes = [P(OrcIon), P(OrcSource), P(OrcRun), P(OrcState), C.c_int64, C.c_int64]
    L.orc_source_emit.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int64, C.c_int64, _dp]
    L.orc_source_emit.restype = C.c_int64
    L.orc_deposit_fixed.argtypes = [C.c_int, C.c_int, C.c_int64, _i32p, _i32p, _i32p, _u8p,
                                    C.c_int64, _i64p]
    L.orc_threads.argtypes = [C.c_int]
    L.orc_threads.restype = C.c_int
    L.orc_tally_state.argtypes = [P(OrcFields), P(OrcIon), P(OrcRun), P(OrcTallySpec), C.c_int64,
                                  _i32p, _i32p, _i32p, _dp, _dp, _dp, _dp, _dp, _u8p, _i32p, C.c_int64,
                                  P(OrcTally)]


def _ptr(a, t):
    return a.ctypes.data_as(t) if a is not None else C.cast(None, t)


# --------------------------------------------------------------------------
# thin helpers
# --------------------------------------------------------------------------

def threads(n=0):
    """Host threads of the oracle's loops over packs: set when n > 0; returns
    the count in use."""
    return int(lib().orc_threads(int(n)))


def philox(ctr, key):
    ctr = (C.c_uint32 * 4)(*[int(c) & 0xFFFFFFFF for c in ctr])
    key = (C.c_uint32 * 2)(*[int(k) & 0xFFFFFFFF for k in key])
    out = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(ctr, key, out)
    return list(out)


def uniforms(seed, pack, step, block, purpose):
    u = np.zeros(4)
    lib().orc_uniforms(seed, pack, step, block, purpose, _ptr(u, _dp))
    return u


def efield_from_phi(phi, dr, dz):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    nz, nr = phi.shape
    er = np.empty_like(phi)
    ez = np.empty_like(phi)
    lib().orc_efield_from_phi(nr, nz, dr, dz, _ptr(phi, _dp), _ptr(er, _dp), _ptr(ez, _dp))
    return er, ez


def ion_struct(ion):
    return OrcIon(ion.mass_da, float(ion.charge), ion.ccs_m2, float(ion.n_atoms), ion.cv_c0,
                  ion.cv_c1, ion.T_init, ion.dH_kJmol, ion.dS_JmolK)


def run_struct(run):
    return OrcRun(run.dt, run.v_rf, run.f_rf, run.phi_rf, run.dc_scale, run.p_scale, run.hit_dist,
                  run.z_exit, run.r_det, run.m_gas_da, run.seed & 0xFFFFFFFFFFFFFFFF, int(run.langevin),
                  run.lv_z0, run.lv_z1, run.lv_switch, int(run.integrator), float(getattr(run, "_rf_phase0", 0.0)),
                  int(getattr(run, "_seg_step0", 0)))


def source_struct(src):
    return OrcSource(src.profile, src.z_plane, src.radius, src.sigma, src.T_vel, src.half_space,
                     src.prefill_z0, src.prefill_z1)


def tally_spec(run):
    return OrcTallySpec(run.exit_bin_steps, run.n_exit_bins, run.n_r_bins, run.n_ke_bins,
                        run.n_teff_bins, run.n_loss_r, run.n_loss_z, run.ke_max_ev, run.teff_max)


def eint_of_T(ion, T):
    s = ion_struct(ion)
    return lib().orc_eint_of_T(C.byref(s), T)


def T_of_eint(ion, e):
    s = ion_struct(ion)
    return lib().orc_T_of_eint(C.byref(s), e)


def cv_of_T(ion, T):
    s = ion_struct(ion)
    return lib().orc_cv_of_T(C.byref(s), T)


def eyring_rate(ion, T):
    s = ion_struct(ion)
    return lib().orc_eyring_rate(C.byref(s), T)


def rf_scalar(run, n):
    s = run_struct(run)
    return lib().orc_rf_scalar(C.byref(s), n)


def one_minus_beta(a, u2, u3):
    return lib().orc_one_minus_beta(a, u2, u3)


def count_collisions_frozen(ion, run, n, T, u, v, trials):
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    return lib().orc_count_collisions_frozen(C.byref(ion_struct(ion)), C.byref(run_struct(run)), n, T,
                                             _ptr(u, _dp), _ptr(v, _dp), trials)


def source_emit(current_A, charge, dt, weight, nsteps, acc):
    a = C.c_double(acc)
    n = lib().orc_source_emit(current_A, float(charge), dt, weight, nsteps, C.byref(a))
    return n, a.value


def quantize(R, z0, z1, x, y, z):
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    z = np.ascontiguousarray(z, np.float64)
    n = x.size
    xq = np.empty(n, np.int32)
    yq = np.empty(n, np.int32)
    zq = np.empty(n, np.int32)
    xa, ya, za = C.c_int32(), C.c_int32(), C.c_int32()
    f = lib().orc_quantize
    for k in range(n):
        f(R, z0, z1, x[k], y[k], z[k], C.byref(xa), C.byref(ya), C.byref(za))
        xq[k], yq[k], zq[k] = xa.value, ya.value, za.value
    return xq, yq, zq


def dmask_of(fields):
    """-1 at metal nodes, else the surface distance, stored in FP32 (the
    precision the hit comparison is taken in)."""
    d = fields.dist.astype(np.float32).copy()
    d[fields.mask != 0] = -1.0
    return np.ascontiguousarray(d)


class Sim:
    """One simulated instance on the oracle: baked fields, FP64 pack state,
    optional PIC space-charge cycle."""

    def __init__(self, workload, capacity=None):
        self.w = workload
        f = workload.fields
        g = f.grid
        self.g = g
        self.er_dc, self.ez_dc = efield_from_phi(f.phi_dc, g.dr, g.dz)
        self.er_rf, self.ez_rf = efield_from_phi(f.phi_rf, g.dr, g.dz)
        self.gas = [np.ascontiguousarray(a, np.float64) for a in (f.gas_p, f.gas_T, f.gas_ur, f.gas_uz)]
        self.dmask = dmask_of(f)
        self.pic = f.pic
        self.er_sc = self.ez_sc = None
        if self.pic is not None:
            self.er_sc = np.zeros((self.pic.nz, self.pic.nr))
            self.ez_sc = np.zeros((self.pic.nz, self.pic.nr))
        self.ion = workload.ion
        self.run = workload.run
        cap = capacity or max(workload.source.n_initial, 1)
        self.cap = cap
        self.x, self.y, self.z = (np.zeros(cap) for _ in range(3))
        self.vx, self.vy, self.vz = (np.zeros(cap) for _ in range(3))
        self.eint = np.zeros(cap)
        self.status = np.full(cap, EMPTY, np.uint8)
        self.t_term = np.full(cap, -1, np.int32)
        self.ncoll = np.zeros(cap, np.int64)
        self.nsteps = np.zeros(cap, np.int64)
        self.noverflow = np.zeros(cap, np.int64)
        self.lnsy = np.zeros(cap)
        self.tau = np.zeros(cap)
        self.n = 0
        self.step = 0
        self.src_acc = 0.0
        self.phi_sc = None

    def fields_struct(self):
        g = self.g
        keep = [self.er_dc, self.ez_dc, self.er_rf, self.ez_rf] + self.gas + [self.dmask]
        self._keep = keep
        pnr = self.pic.nr if self.pic is not None else 0
        pnz = self.pic.nz if self.pic is not None else 0
        return OrcFields(g.nr, g.nz, g.R, g.z0, g.z1, _ptr(self.er_dc, _dp), _ptr(self.ez_dc, _dp),
                         _ptr(self.er_rf, _dp), _ptr(self.ez_rf, _dp), _ptr(self.gas[0], _dp),
                         _ptr(self.gas[1], _dp), _ptr(self.gas[2], _dp), _ptr(self.gas[3], _dp),
                         _ptr(self.dmask, _fp), pnr, pnz, _ptr(self.er_sc, _dp), _ptr(self.ez_sc, _dp))

    def state_struct(self):
        return OrcState(*(_ptr(a, _dp) for a in (self.x, self.y, self.z, self.vx, self.vy, self.vz,
                                                  self.eint)),
                        _ptr(self.status, _u8p), _ptr(self.t_term, _i32p), _ptr(self.ncoll, _i64p),
                        _ptr(self.nsteps, _i64p), _ptr(self.noverflow, _i64p), _ptr(self.lnsy, _dp),
                        _ptr(self.tau, _dp))

    def inject(self, count=None):
        count = self.w.source.n_initial if count is None else count
        assert self.n + count <= self.cap
        S = self.state_struct()
        lib().orc_inject(C.byref(ion_struct(self.ion)), C.byref(source_struct(self.w.source)),
                         C.byref(run_struct(self.run)), C.byref(S), self.n, count)
        self.n += count

    def emit_continuous(self, nsteps):
        """Packs released by the continuous source over nsteps (Eq. 5); the
        new packs start on the source plane."""
        src = self.w.source
        if src.current_A <= 0:
            return 0
        k, self.src_acc = source_emit(src.current_A, self.ion.charge, self.run.dt, src.weight, nsteps,
                                      self.src_acc)
        if k:
            saved = (src.prefill_z0, src.prefill_z1)
            src.prefill_z0 = src.prefill_z1 = 0.0
            try:
                self.inject(k)
            finally:
                src.prefill_z0, src.prefill_z1 = saved
        return k

    def steps(self, nsteps, frozen=False):
        F = self.fields_struct()
        S = self.state_struct()
        lib().orc_run_steps(C.byref(F), C.byref(ion_struct(self.ion)), C.byref(run_struct(self.run)),
                            C.byref(S), self.n, self.step, nsteps, 1 if frozen else 0)
        self.step += nsteps

    def quantized(self):
        g = self.g
        return quantize(g.R, g.z0, g.z1, self.x[:self.n], self.y[:self.n], self.z[:self.n])

    def deposit(self):
        xq, yq, zq = self.quantized()
        return deposit_fixed(self.pic, xq, yq, zq, self.status[:self.n],
                             int(self.ion.charge) * int(self.w.source.weight))

    def pic_update(self):
        """Deposit -> FV Poisson (direct) -> central-difference E_SCE
        ("Axisymmetric PIC space charge update")."""
        from . import poisson
        Q = self.deposit()
        if getattr(self.run, "pic_masked", 0):
            metal = poisson.pic_metal_from_static(self.g, self.w.fields.mask, self.pic)
            phi = poisson.solve_masked(self.pic, Q, metal) if metal.any() else poisson.solve(self.pic, Q)
        else:
            phi = poisson.solve(self.pic, Q)
        self.phi_sc = phi
        er, ez = efield_from_phi(phi, self.pic.dr, self.pic.dz)
        self.er_sc[...] = er
        self.ez_sc[...] = ez
        return Q, phi

    def set_dt(self, dt):
        """Start a new dt segment at the current step: the RF phase carries
        over (frac of the phase reached), the step clock continues."""
        run = self.run
        if run.f_rf > 0:
            x = getattr(run, "_rf_phase0", 0.0) + (self.step - getattr(run, "_seg_step0", 0)) * (run.dt * run.f_rf)
            run._rf_phase0 = x - np.floor(x)
        run._seg_step0 = self.step
        run.dt = dt

    def dt_limits(self):
        out = np.zeros(6)
        lib().orc_dt_limits(C.byref(self.fields_struct()), C.byref(ion_struct(self.ion)),
                            C.byref(run_struct(self.run)), C.byref(self.state_struct()), self.n, self.step,
                            _ptr(out, _dp))
        return out

    def advance(self, nsteps):
        """Advance nsteps with the PIC cycle every pic_interval steps and the
        continuous source emitting at the start of every call."""
        self.emit_continuous(nsteps)
        P = self.run.pic_interval
        done = 0
        while done < nsteps:
            if P and self.pic is not None and self.step % P == 0:
                self.pic_update()
            chunk = nsteps - done
            if P:
                chunk = min(chunk, P - self.step % P)
            self.steps(chunk)
            done += chunk

    def tally(self, xq=None, yq=None, zq=None, vx=None, vy=None, vz=None, eint=None, status=None,
              t_term=None, lnsy=None):
        n = self.n
        if xq is None:
            xq, yq, zq = self.quantized()
            vx, vy, vz, eint = self.vx[:n], self.vy[:n], self.vz[:n], self.eint[:n]
            status, t_term, lnsy = self.status[:n], self.t_term[:n], self.lnsy[:n]
        return tally_state(self.fields_struct(), self.ion, self.run, xq, yq, zq, vx, vy, vz, eint,
                           status, t_term, self.w.source.weight, lnsy)


def classify_fixed(fields_struct, run, xq, yq, zq):
    xq, yq, zq = (np.ascontiguousarray(a, np.int32) for a in (xq, yq, zq))
    st = np.empty(xq.size, np.uint8)
    lib().orc_classify_fixed(C.byref(fields_struct), C.byref(run_struct(run)), xq.size,
                             _ptr(xq, _i32p), _ptr(yq, _i32p), _ptr(zq, _i32p), _ptr(st, _u8p))
    return st


def deposit_fixed(pic, xq, yq, zq, status, qw):
    xq, yq, zq = (np.ascontiguousarray(a, np.int32) for a in (xq, yq, zq))
    status = np.ascontiguousarray(status, np.uint8)
    Q = np.zeros((pic.nz, pic.nr), np.int64)
    lib().orc_deposit_fixed(pic.nr, pic.nz, xq.size, _ptr(xq, _i32p), _ptr(yq, _i32p), _ptr(zq, _i32p),
                            _ptr(status, _u8p), int(qw), _ptr(Q, _i64p))
    return Q


def tally_state(fields_struct, ion, run, xq, yq, zq, vx, vy, vz, eint, status, t_term, weight, lnsy=None):
    n = len(status)
    arr = lambda a, t: np.ascontiguousarray(a, t)
    xq, yq, zq = arr(xq, np.int32), arr(yq, np.int32), arr(zq, np.int32)
    vx, vy, vz, eint = (arr(a, np.float64) for a in (vx, vy, vz, eint))
    status, t_term = arr(status, np.uint8), arr(t_term, np.int32)
    lnsy = arr(lnsy, np.float64) if lnsy is not None else None
    out = dict(exit_hist=np.zeros(run.n_exit_bins, np.int64), r_hist=np.zeros(run.n_r_bins, np.int64),
               ke_hist=np.zeros(run.n_ke_bins, np.int64), teff_hist=np.zeros(run.n_teff_bins, np.int64),
               loss_map=np.zeros((run.n_loss_z, run.n_loss_r), np.int64))
    T = OrcTally()
    T.exit_hist = _ptr(out["exit_hist"], _i64p)
    T.r_hist = _ptr(out["r_hist"], _i64p)
    T.ke_hist = _ptr(out["ke_hist"], _i64p)
    T.teff_hist = _ptr(out["teff_hist"], _i64p)
    T.loss_map = _ptr(out["loss_map"], _i64p)
    spec = tally_spec(run)
    lib().orc_tally_state(C.byref(fields_struct), C.byref(ion_struct(ion)), C.byref(run_struct(run)),
                          C.byref(spec), n, _ptr(xq, _i32p), _ptr(yq, _i32p), _ptr(zq, _i32p),
                          _ptr(vx, _dp), _ptr(vy, _dp), _ptr(vz, _dp), _ptr(eint, _dp), _ptr(lnsy, _dp),
                          _ptr(status, _u8p), _ptr(t_term, _i32p), int(weight), C.byref(T))
    out["count"] = np.array(T.count[:], np.int64)
    out["weight"] = np.array(T.weight[:], np.int64)
    out["sum_w_ke"] = np.array(T.sum_w_ke[:])
    out["sum_w_teff"] = np.array(T.sum_w_teff[:])
    out["sum_w_sy"] = np.array(T.sum_w_sy[:])
    return out
