"""Shared test plumbing: move identical pack states between the oracle and
the CUDA library's pools, and ensemble comparisons."""
import math

import numpy as np

LAT = 2.0 ** 30


def lattice_from_fp64(g, x, y, z):
    """Round FP64 positions to the int32 lattice (rint(x 2^30 / R))."""
    sx, sz = LAT / g.R, LAT / (g.z1 - g.z0)
    return (np.rint(np.asarray(x) * sx).astype(np.int32), np.rint(np.asarray(y) * sx).astype(np.int32),
            np.rint((np.asarray(z) - g.z0) * sz).astype(np.int32))


def fp64_from_lattice(g, xq, yq, zq):
    return (xq.astype(np.float64) * g.R / LAT, yq.astype(np.float64) * g.R / LAT,
            g.z0 + zq.astype(np.float64) * (g.z1 - g.z0) / LAT)


def fp32_state_from_oracle(sim):
    """Lattice positions + FP32 velocities/E_int of the oracle's packs, and the
    oracle state reset to exactly the same values (so both start equal)."""
    n = sim.n
    g = sim.g
    xq, yq, zq = lattice_from_fp64(g, sim.x[:n], sim.y[:n], sim.z[:n])
    st = dict(x=xq, y=yq, z=zq, vx=sim.vx[:n].astype(np.float32), vy=sim.vy[:n].astype(np.float32),
              vz=sim.vz[:n].astype(np.float32), eint=sim.eint[:n].astype(np.float32),
              status=sim.status[:n].copy(), t_term=sim.t_term[:n].copy(), lnsy=sim.lnsy[:n].astype(np.float32),
              tau=sim.tau[:n].astype(np.float32))
    sim.x[:n], sim.y[:n], sim.z[:n] = fp64_from_lattice(g, xq, yq, zq)
    sim.vx[:n], sim.vy[:n], sim.vz[:n] = (st[k].astype(np.float64) for k in ("vx", "vy", "vz"))
    sim.eint[:n] = st["eint"].astype(np.float64)
    sim.lnsy[:n] = st["lnsy"].astype(np.float64)
    sim.tau[:n] = st["tau"].astype(np.float64)
    return st


def fp64_state_from_oracle(sim):
    n = sim.n
    return dict(x=sim.x[:n].copy(), y=sim.y[:n].copy(), z=sim.z[:n].copy(), vx=sim.vx[:n].copy(),
                vy=sim.vy[:n].copy(), vz=sim.vz[:n].copy(), eint=sim.eint[:n].copy(),
                status=sim.status[:n].copy(), t_term=sim.t_term[:n].copy(), lnsy=sim.lnsy[:n].copy(),
                tau=sim.tau[:n].copy())


def upload(ctx, inst, arrays, step=0):
    import torch
    views = ctx.state(inst)
    n = len(arrays["status"])
    for k, a in arrays.items():
        views[k][:n].copy_(torch.from_numpy(np.ascontiguousarray(a)))
    torch.cuda.synchronize()
    ctx.resume(inst, n, step)


def download(ctx, inst, n):
    import torch
    ctx.sync()
    torch.cuda.synchronize()
    return {k: v[:n].cpu().numpy() for k, v in ctx.state(inst).items()}


def rel_pos_error(g, got, ref_x, ref_y, ref_z, lattice=True):
    """Per-pack |x_gpu - x_ref| / |x_ref - (0,0,z0)|."""
    if lattice:
        gx, gy, gz = fp64_from_lattice(g, got["x"], got["y"], got["z"])
    else:
        gx, gy, gz = got["x"], got["y"], got["z"]
    d = np.sqrt((gx - ref_x) ** 2 + (gy - ref_y) ** 2 + (gz - ref_z) ** 2)
    norm = np.sqrt(ref_x ** 2 + ref_y ** 2 + (ref_z - g.z0) ** 2)
    return d / norm


def binomial_band(k_a, k_b, n, nsig=3.0):
    """|p_a - p_b| within nsig standard deviations of a binomial proportion."""
    p = 0.5 * (k_a + k_b) / n
    sd = math.sqrt(max(p * (1 - p), 1.0 / n) / n)
    return abs(k_a - k_b) / n <= nsig * sd


def ensemble_stats(orc, ion, got, n_g, sim, n_o, labels=(1, 2, 3, 4)):
    """The stochastic-ensemble criteria of the method's parity bar for a GPU
    population `got` (downloaded pool, n_g packs) against an oracle
    population `sim` (n_o packs): per terminal label the fractions, their
    difference in standard deviations of a two-sample binomial proportion;
    two-sample KS statistic and p-value on the kinetic energy and T_eff of
    the packs still active; mean-T_eff ratio."""
    from scipy import stats
    m = ion.mass_da * 1.66053906660e-27
    st_g, st_o = got["status"][:n_g], sim.status[:n_o]
    out = {"labels": {}}
    for lab in labels:
        kg, ko = int((st_g == lab).sum()), int((st_o == lab).sum())
        pg, po = kg / n_g, ko / n_o
        p = (kg + ko) / (n_g + n_o)
        sd = math.sqrt(max(p * (1 - p), 1.0 / (n_g + n_o)) * (1.0 / n_g + 1.0 / n_o))
        out["labels"][int(lab)] = {"gpu": pg, "oracle": po, "sigma": abs(pg - po) / sd}
    a_g, a_o = st_g == 0, st_o == 0
    ke_g = 0.5 * m * (got["vx"][:n_g][a_g].astype(np.float64) ** 2 + got["vy"][:n_g][a_g].astype(np.float64) ** 2
                      + got["vz"][:n_g][a_g].astype(np.float64) ** 2)
    ke_o = 0.5 * m * (sim.vx[:n_o][a_o] ** 2 + sim.vy[:n_o][a_o] ** 2 + sim.vz[:n_o][a_o] ** 2)
    ks = stats.ks_2samp(ke_g, ke_o)
    out["ke_ks"] = {"D": float(ks.statistic), "p": float(ks.pvalue)}
    T_of = np.vectorize(lambda e: orc.T_of_eint(ion, float(e)))
    # T_eff of at most 200,000 packs per side (evenly strided) keeps the host work short
    sg = max(1, int(a_g.sum()) // 200_000)
    so = max(1, int(a_o.sum()) // 200_000)
    T_g = T_of(got["eint"][:n_g][a_g][::sg].astype(np.float64))
    T_o = T_of(sim.eint[:n_o][a_o][::so])
    ks = stats.ks_2samp(T_g, T_o)
    out["teff_ks"] = {"D": float(ks.statistic), "p": float(ks.pvalue)}
    out["mean_teff_ratio"] = float(T_g.mean() / T_o.mean())
    out["active"] = {"gpu": int(a_g.sum()), "oracle": int(a_o.sum())}
    return out


def assert_ensemble_bar(es):
    """3-sigma binomial band per label, KS p > 0.01 on KE and T_eff, mean
    T_eff within 0.5 %."""
    for lab, v in es["labels"].items():
        assert v["sigma"] <= 3.0, (lab, v)
    assert es["ke_ks"]["p"] > 0.01, es["ke_ks"]
    assert es["teff_ks"]["p"] > 0.01, es["teff_ks"]
    assert abs(es["mean_teff_ratio"] - 1.0) < 0.005, es["mean_teff_ratio"]
