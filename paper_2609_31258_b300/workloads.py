"""Seeded synthetic inputs for the ion-pack step: grids, baked fields, ion
templates, sources and run settings.

This module is the one place both the CUDA library and the FP64 oracle take
their inputs from. It holds none of the method's arithmetic: it builds the
static inputs the paper obtains offline (the "field bake" of the Methods
section: DC and RF-basis potentials, gas fields, electrode mask and surface
distance on a common axisymmetric (r, z) grid) and the parameter sets of the
five benchmark workloads. The potentials are the solution of Laplace's
equation on a synthetic ring-stack electrode mask, computed here by red-black
SOR in FP64 with nested grids; the paper's own come from SIMION, which is not
available.

Grid convention (paper Table S2, static grid 2001 x 6501 for 20 mm / 0.01 mm):
node counts include both ends, arrays are row-major [Nz][Nr], r_i = i*R/(Nr-1),
z_j = z0 + j*(z1-z0)/(Nz-1). Units are SI throughout.
"""
from __future__ import annotations

import dataclasses
import hashlib
import math
import os
from typing import Optional

import numpy as np

# CODATA 2018 exact / recommended values.
E_CHARGE = 1.602176634e-19
K_B = 1.380649e-23
EPS0 = 8.8541878128e-12
DALTON = 1.66053906660e-27

# Status codes written into the pack state (terminal classes of the
# "Terminal events" paragraph).
ST_ACTIVE, ST_TRANSMITTED, ST_ELECTRODE, ST_RADIAL, ST_AXIAL, ST_EMPTY = 0, 1, 2, 3, 4, 255


@dataclasses.dataclass
class Grid:
    nr: int
    nz: int
    R: float
    z0: float
    z1: float

    @property
    def dr(self) -> float:
        return self.R / (self.nr - 1)

    @property
    def dz(self) -> float:
        return (self.z1 - self.z0) / (self.nz - 1)


@dataclasses.dataclass
class Fields:
    """Host FP64 arrays [Nz][Nr] on `grid` (inputs to field loading)."""
    grid: Grid
    phi_dc: np.ndarray
    phi_rf: np.ndarray
    gas_p: np.ndarray
    gas_T: np.ndarray
    gas_ur: np.ndarray
    gas_uz: np.ndarray
    mask: np.ndarray          # uint8, 1 = metal node
    dist: np.ndarray          # distance to the nearest metal node [m]
    pic: Optional[Grid] = None


@dataclasses.dataclass
class IonTemplate:
    mass_da: float
    charge: int
    ccs_m2: float
    n_atoms: float
    # heat capacity Cv/k_B = 3N * min(1, cv_c0 + cv_c1*T)
    cv_c0: float = 1.0
    cv_c1: float = 0.0
    T_init: float = 300.0
    # transition-state parameters of Eq. 7 (dH <= 0: no dissociation)
    dH_kJmol: float = 0.0
    dS_JmolK: float = 0.0


@dataclasses.dataclass
class Source:
    profile: int = 0          # 0 = uniform over a disc, 1 = truncated Gaussian
    z_plane: float = 0.0
    radius: float = 1e-3      # disc radius, or truncation radius of the Gaussian
    sigma: float = 0.0
    T_vel: float = 300.0      # Maxwell temperature of the initial velocity
    half_space: int = 1       # v_z = |v_z|
    n_initial: int = 0
    prefill_z0: float = 0.0   # if prefill_z1 > prefill_z0: z uniform in this range
    prefill_z1: float = 0.0
    current_A: float = 0.0    # continuous current (Eq. 5); 0 = none
    weight: int = 1           # real ions per pack W


@dataclasses.dataclass
class Run:
    dt: float
    v_rf: float = 0.0         # peak volts applied to the RF basis
    f_rf: float = 0.0
    phi_rf: float = 0.0
    dc_scale: float = 1.0
    p_scale: float = 1.0
    hit_dist: float = 1e-5    # electrode-hit distance (Table S2: 0.01 mm)
    z_exit: float = 0.0
    r_det: float = 0.0
    m_gas_da: float = 28.0
    seed: int = 0
    precision: int = 0        # 0 = FP32 fused path, 1 = plain FP64 path
    pic_interval: int = 0     # steps between PIC updates, 0 = no space charge
    # hybrid Langevin branch: OU relaxation instead of explicit collisions in
    # z in [lv_z0, lv_z1] where lambda*dt >= lv_switch (Table S2: 0.05)
    langevin: int = 0
    lv_z0: float = 0.0
    lv_z1: float = 0.0
    lv_switch: float = 0.05
    pic_masked: int = 0       # impose Phi = 0 on metal nodes of the PIC grid
    integrator: int = 0       # 0 leapfrog, 1 RK4
    # tally histogram layout
    exit_bin_steps: int = 1000
    n_exit_bins: int = 64
    n_r_bins: int = 64
    n_ke_bins: int = 64
    ke_max_ev: float = 1.0
    n_teff_bins: int = 64
    teff_max: float = 1000.0
    n_loss_r: int = 16
    n_loss_z: int = 64


@dataclasses.dataclass
class Workload:
    name: str
    fields: Fields
    ion: IonTemplate
    source: Source
    run: Run
    n_steps: int


# ----------------------------------------------------------------------------
# field bake helpers
# ----------------------------------------------------------------------------

def node_coords(g: Grid):
    r = np.arange(g.nr) * g.dr
    z = g.z0 + np.arange(g.nz) * g.dz
    return r, z


def ring_stack_mask(g: Grid, n_rings=20, z_first=5e-3, thick=0.5e-3, pitch=1.5e-3,
                    r_in_first=4e-3, r_in_last=1e-3):
    """Electrode index per node (-1 = gas). Ring k occupies
    z in [z_first + k*pitch, z_first + k*pitch + thick], r >= r_in(k), with the
    inner radius tapering linearly from r_in_first to r_in_last."""
    r, z = node_coords(g)
    idx = -np.ones((g.nz, g.nr), dtype=np.int32)
    eps = 1e-12
    for k in range(n_rings):
        za = z_first + k * pitch
        zb = za + thick
        rin = r_in_first + (r_in_last - r_in_first) * k / (n_rings - 1)
        jz = (z >= za - eps) & (z <= zb + eps)
        ir = r >= rin - eps
        idx[np.ix_(jz, ir)] = k
    return idx


def _sor_level(phi, fixed, dr, dz, n_iter, omega, tol=1e-10):
    """Red-black SOR for the axisymmetric Laplacian (finite-volume form),
    Dirichlet at `fixed` nodes, symmetry at r=0 and mirror (Neumann) ghosts at
    the other domain edges. The four parity sub-lattices are updated through
    strided views of a padded array."""
    nz, nr = phi.shape
    i = np.arange(nr, dtype=np.float64)
    cp = np.ones(nr)
    cm = np.ones(nr)
    cp[1:] = 1.0 + 0.5 / i[1:]
    cm[1:] = 1.0 - 0.5 / i[1:]
    cp[0] = 4.0  # axis row: 4*(phi1 - phi0)/dr^2
    cm[0] = 0.0
    ar = 1.0 / dr ** 2
    az = 1.0 / dz ** 2
    diag = np.full(nr, 2 * ar + 2 * az)
    diag[0] = 4 * ar + 2 * az
    wE = ar * cp / diag
    wW = ar * cm / diag
    wN = np.broadcast_to(az / diag, (nz, nr))
    P = np.zeros((nz + 2, nr + 2))
    P[1:-1, 1:-1] = phi
    free = (~fixed).astype(np.float64)
    subl = {0: [(0, 0), (1, 1)], 1: [(0, 1), (1, 0)]}

    def ghosts():
        P[1:-1, 0] = P[1:-1, 2]
        P[1:-1, -1] = P[1:-1, -3]
        P[0, :] = P[2, :]
        P[-1, :] = P[-3, :]

    ghosts()
    for it in range(n_iter):
        delta = 0.0
        for c in (0, 1):
            for (pj, pi) in subl[c]:
                js = slice(1 + pj, nz + 1, 2)
                is_ = slice(1 + pi, nr + 1, 2)
                C = P[js, is_]
                E = P[js, slice(2 + pi, nr + 2, 2)]
                Wv = P[js, slice(pi, nr, 2)]
                N = P[slice(2 + pj, nz + 2, 2), is_]
                S = P[slice(pj, nz, 2), is_]
                m = min(E.shape[1], Wv.shape[1], C.shape[1])
                k = min(N.shape[0], S.shape[0], C.shape[0])
                C = C[:k, :m]
                gs = wE[pi::2][:m] * E[:k, :m] + wW[pi::2][:m] * Wv[:k, :m] \
                    + wN[pj::2, pi::2][:k, :m] * (N[:k, :m] + S[:k, :m])
                upd = omega * (gs - C) * free[pj::2, pi::2][:k, :m]
                C += upd
                if upd.size:
                    delta = max(delta, float(np.abs(upd).max()))
            ghosts()
        if delta < tol:
            break
    phi[...] = P[1:-1, 1:-1]
    return phi


def _prolong(phi, nr, nz):
    rc = np.linspace(0.0, 1.0, phi.shape[1])
    zc = np.linspace(0.0, 1.0, phi.shape[0])
    rf = np.linspace(0.0, 1.0, nr)
    zf = np.linspace(0.0, 1.0, nz)
    tmp = np.empty((phi.shape[0], nr))
    for j in range(phi.shape[0]):
        tmp[j] = np.interp(rf, rc, phi[j])
    out = np.empty((nz, nr))
    for i in range(nr):
        out[:, i] = np.interp(zf, zc, tmp[:, i])
    return out


def solve_laplace_rings(g: Grid, electrode_idx, volts, tol=1e-9, fine_sweeps=400):
    """FP64 potential with electrode k held at volts[k]; nested grids coarse to
    fine (each about half the nodes of the next), each level relaxed by
    red-black SOR and bilinearly prolonged to the next (G13 of the build
    plan)."""
    levels = [(g.nr, g.nz)]
    nr, nz = g.nr, g.nz
    while nr > 48 and nz > 96:
        nr, nz = (nr + 1) // 2, (nz + 1) // 2
        levels.append((nr, nz))
    levels = levels[::-1]
    phi = None
    volts = np.asarray(volts, dtype=np.float64)
    for li, (lr, lz) in enumerate(levels):
        gl = Grid(lr, lz, g.R, g.z0, g.z1)
        eidx = electrode_idx if (lr, lz) == (g.nr, g.nz) else ring_stack_mask(gl)
        fixed = eidx >= 0
        phi = np.zeros((lz, lr)) if phi is None else _prolong(phi, lr, lz)
        phi[fixed] = volts[eidx[fixed]]
        h = min(gl.dr, gl.dz)
        span = max(g.R, g.z1 - g.z0)
        omega = min(2.0 / (1.0 + math.sin(math.pi * h / span)), 1.97)
        n_iter = 6000 if li == 0 else (fine_sweeps if (lr, lz) == (g.nr, g.nz) else 600)
        phi = _sor_level(phi, fixed, gl.dr, gl.dz, n_iter, omega if li == 0 else 1.9, tol)
    return phi


def distance_to_metal(g: Grid, mask):
    from scipy import ndimage
    if not mask.any():
        return np.full(mask.shape, 1.0)
    return ndimage.distance_transform_edt(mask == 0, sampling=(g.dz, g.dr)).astype(np.float64)


def _cache_dir():
    d = os.environ.get("MUCITE_FIELD_CACHE",
                       os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "fieldcache"))
    os.makedirs(d, exist_ok=True)
    return d


def ring_stack_fields(g: Grid, p_in=1000.0, pic: Optional[Grid] = None, cache=True) -> Fields:
    """Ring-stack S-lens-like geometry with a free-jet gas field.

    RF basis: adjacent rings at +1 / -1 V (Methods, RF basis convention).
    DC basis: ring k at -k volts (unit gradient of -1 V per ring).
    Gas: p(z) = p_in * 0.1**((z-z0)/L), u_z = 500 m/s * ((z-z0)/L) * (1-(r/R)^2),
    u_r = 0, T = 300 K (N2)."""
    key = hashlib.sha1(repr((g.nr, g.nz, g.R, g.z0, g.z1)).encode()).hexdigest()[:16]
    path = os.path.join(_cache_dir(), f"rings_{key}.npz")
    eidx = ring_stack_mask(g)
    if cache and os.path.exists(path):
        d = np.load(path)
        phi_dc, phi_rf = d["phi_dc"], d["phi_rf"]
    else:
        nrings = 20
        phi_rf = solve_laplace_rings(g, eidx, [(1.0 if k % 2 == 0 else -1.0) for k in range(nrings)])
        phi_dc = solve_laplace_rings(g, eidx, [-float(k) for k in range(nrings)])
        if cache:
            tmp = path + f".{os.getpid()}.tmp.npz"
            np.savez(tmp, phi_dc=phi_dc, phi_rf=phi_rf)
            os.replace(tmp, path)
    mask = (eidx >= 0).astype(np.uint8)
    r, z = node_coords(g)
    L = g.z1 - g.z0
    zz, rr = np.meshgrid(z, r, indexing="ij")
    gas_p = p_in * np.power(0.1, (zz - g.z0) / L)
    gas_T = np.full_like(gas_p, 300.0)
    gas_uz = 500.0 * ((zz - g.z0) / L) * (1.0 - (rr / g.R) ** 2)
    gas_ur = np.zeros_like(gas_p)
    return Fields(g, phi_dc, phi_rf, gas_p, gas_T, gas_ur, gas_uz, mask,
                  distance_to_metal(g, mask), pic)


def uniform_axial_fields(g: Grid, Ez=2000.0, p=200.0, T=300.0, pic: Optional[Grid] = None) -> Fields:
    """Cylinder without electrodes, DC potential linear in z (uniform E_z), no
    RF, static gas."""
    r, z = node_coords(g)
    zz, rr = np.meshgrid(z, r, indexing="ij")
    phi_dc = -Ez * (zz - g.z0)
    zero = np.zeros_like(phi_dc)
    mask = np.zeros(phi_dc.shape, np.uint8)
    return Fields(g, phi_dc, zero.copy(), np.full_like(zero, p), np.full_like(zero, T),
                  zero.copy(), zero.copy(), mask, np.full_like(zero, 1.0), pic)


# ----------------------------------------------------------------------------
# ion templates and workloads (the five benchmark configurations)
# ----------------------------------------------------------------------------

ION_1KDA = IonTemplate(mass_da=1000.0, charge=1, ccs_m2=300e-20, n_atoms=100)
# Cv/k_B = 3N * (0.3 + 0.7*T/1000 K), capped at 3N
ION_15KDA = IonTemplate(mass_da=15000.0, charge=8, ccs_m2=1500e-20, n_atoms=2000, cv_c0=0.3, cv_c1=7e-4)
ION_150KDA = IonTemplate(mass_da=150000.0, charge=25, ccs_m2=7500e-20, n_atoms=20000, cv_c0=0.3, cv_c1=7e-4)
ION_1KDA_LIN = IonTemplate(mass_da=1000.0, charge=1, ccs_m2=300e-20, n_atoms=100, cv_c0=0.3, cv_c1=7e-4)


def tiny_cylinder(n_packs=2000, n_steps=20000, seed=0, precision=1) -> Workload:
    """Plain method, tiny: 64x256 grid, r<=5 mm, z in [0,20] mm, uniform
    E_z=2000 V/m, static N2 at 300 K and 200 Pa, 1 kDa/+1/300 A^2/100 atoms,
    dt = 1 ns, seed 0."""
    g = Grid(64, 256, 5e-3, 0.0, 20e-3)
    f = uniform_axial_fields(g)
    src = Source(profile=0, z_plane=0.0, radius=1e-3, T_vel=300.0, half_space=1, n_initial=n_packs, weight=1)
    run = Run(dt=1e-9, z_exit=20e-3, r_det=5e-3, seed=seed, precision=precision,
              exit_bin_steps=1000, n_exit_bins=32, ke_max_ev=0.5, teff_max=600.0)
    return Workload("cylinder-64x256-2k-packs", f, ION_1KDA, src, run, n_steps)


def ring_stack(n_packs=100_000, n_steps=80_000, seed=1, precision=0, nr=512, nz=2048) -> Workload:
    """S-lens-like ring stack, no space charge: 512x2048 grid over r<=5 mm,
    z in [0,40] mm, 20 rings 0.5 mm thick at 1.5 mm pitch with inner radius
    4 -> 1 mm, RF 1 MHz 100 V peak on alternating rings, DC -2 V per ring,
    free-jet N2 1000 -> 100 Pa, 15 kDa/+8/1500 A^2/2000 atoms, dt = 0.5 ns,
    40 us, seed 1. Packs start on the paper's source plane z = 6 mm, uniform
    over the 0.25 mm source radius."""
    g = Grid(nr, nz, 5e-3, 0.0, 40e-3)
    f = ring_stack_fields(g, p_in=1000.0)
    src = Source(profile=0, z_plane=6e-3, radius=0.25e-3, T_vel=300.0, half_space=1, n_initial=n_packs, weight=1)
    run = Run(dt=0.5e-9, v_rf=100.0, f_rf=1e6, phi_rf=-math.pi / 2, dc_scale=2.0, p_scale=1.0,
              hit_dist=1e-5, z_exit=40e-3, r_det=5e-3, seed=seed, precision=precision,
              exit_bin_steps=2000, n_exit_bins=40, ke_max_ev=2.0, teff_max=1000.0)
    return Workload(f"ring-stack-{nr}x{nz}-{n_packs}-packs", f, ION_15KDA, src, run, n_steps)


def cylinder_space_charge(n_packs=1_000_000, n_steps=200_000, seed=2, precision=0,
                          pic_nr=256, pic_nz=1024) -> Workload:
    """Tiny-cylinder geometry plus PIC space charge: 1 nA continuous current at
    W = 1e3, 1e6 packs in flight (prefilled uniformly in z over [0,20] mm),
    Gaussian radial profile sigma = 0.3 mm (truncated at 3 sigma), PIC
    256x1024 every 10 steps, dt = 0.5 ns, 100 us, seed 2."""
    g = Grid(64, 256, 5e-3, 0.0, 20e-3)
    pic = Grid(pic_nr, pic_nz, 5e-3, 0.0, 20e-3)
    f = uniform_axial_fields(g, pic=pic)
    src = Source(profile=1, z_plane=0.0, radius=0.9e-3, sigma=0.3e-3, T_vel=300.0, half_space=1,
                 n_initial=n_packs, prefill_z0=0.0, prefill_z1=20e-3, current_A=1e-9, weight=1000)
    run = Run(dt=0.5e-9, z_exit=20e-3, r_det=5e-3, seed=seed, precision=precision, pic_interval=10,
              exit_bin_steps=2000, n_exit_bins=100, ke_max_ev=1.0, teff_max=600.0)
    return Workload(f"cylinder-pic-{pic_nr}x{pic_nz}-{n_packs}-packs", f, ION_1KDA, src, run, n_steps)


def paper_grid(n_packs=100_000, seed=7, precision=0, nr=2001, nz=6501) -> Workload:
    """Static grid of the paper's S-lens size (2001 x 6501 nodes at 0.01 mm,
    r <= 20 mm, z in [0, 65] mm; 468 MB of FP32 node records and mask, not
    L2-resident) with analytic fields in place of a Laplace solve: an RF
    pattern alternating every 1.5 mm, (r / 4 mm)^2 cos(pi z / 1.5 mm), a DC
    gradient of -2 V per 1.5 mm, no electrodes, and the free-jet gas of the
    ring stack over 65 mm. Packs of 15 kDa/+8 fill the guide: prefilled
    uniformly in z over [1, 64] mm, Gaussian in r with sigma = 1.5 mm
    (truncated at 4.5 mm), Maxwellian at 300 K."""
    g = Grid(nr, nz, 20e-3, 0.0, 65e-3)
    r, z = node_coords(g)
    zz, rr = np.meshgrid(z, r, indexing="ij")
    phi_rf = (rr / 4e-3) ** 2 * np.cos(np.pi * zz / 1.5e-3)
    phi_dc = -(2.0 / 1.5e-3) * zz
    L = g.z1 - g.z0
    gas_p = 1000.0 * np.power(0.1, zz / L)
    gas_T = np.full_like(gas_p, 300.0)
    gas_uz = 500.0 * (zz / L) * (1.0 - (rr / g.R) ** 2)
    mask = np.zeros(phi_dc.shape, np.uint8)
    f = Fields(g, phi_dc, phi_rf, gas_p, gas_T, np.zeros_like(gas_p), gas_uz, mask, np.full_like(gas_p, 1.0))
    src = Source(profile=1, z_plane=0.0, radius=4.5e-3, sigma=1.5e-3, T_vel=300.0, half_space=0,
                 n_initial=n_packs, prefill_z0=1e-3, prefill_z1=64e-3, weight=1)
    run = Run(dt=0.5e-9, v_rf=100.0, f_rf=1e6, phi_rf=-math.pi / 2, dc_scale=1.0, p_scale=1.0, hit_dist=1e-5,
              z_exit=65e-3, r_det=20e-3, seed=seed, precision=precision, exit_bin_steps=2000, n_exit_bins=40,
              ke_max_ev=2.0, teff_max=1000.0)
    return Workload(f"paper-grid-{nr}x{nz}-{n_packs}-packs", f, ION_15KDA, src, run, 0)


def sweep_points(n_inst=64, seed_base=100, n_min=10_000, n_max=500_000):
    """Operating points of the batched sweep: a 4x4x4 grid of RF amplitude
    (100-300 Vpp), DC gradient (-0.5 to -4 V/ring) and inlet pressure
    (500-2000 Pa); pack counts log-uniform in [n_min, n_max] drawn with the
    instance seed."""
    pts = []
    vpp = np.linspace(100.0, 300.0, 4)
    dcg = np.linspace(-0.5, -4.0, 4)
    pin = np.linspace(500.0, 2000.0, 4)
    for i in range(n_inst):
        a, b, c = (i // 16) % 4, (i // 4) % 4, i % 4
        rng = np.random.default_rng(seed_base + i)
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        pts.append(dict(v_rf=vpp[a] / 2.0, dc_scale=-dcg[b], p_scale=pin[c] / 1000.0,
                        seed=seed_base + i, n_packs=n))
    return pts


def serving_arrivals(n_req=200, rate_hz=20.0, seed=5, n_min=10_000, n_max=2_000_000):
    """Poisson arrivals of sweep-point requests: arrival time, pack count
    (log-uniform), ion template index (uniform over three)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_req))
    n = np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=n_req)).round().astype(np.int64)
    tmpl = rng.integers(0, 3, size=n_req)
    return t, n, tmpl


SERVING_TEMPLATES = [
    IonTemplate(mass_da=1000.0, charge=1, ccs_m2=300e-20, n_atoms=100, cv_c0=0.3, cv_c1=7e-4),
    ION_15KDA,
    ION_150KDA,
]
