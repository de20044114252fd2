"""Oracle: cylindrical finite-volume Poisson operator and its direct solve.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows "Axisymmetric PIC space charge update": the Poisson operator is a
finite-volume balance on the ring-shaped cell that surrounds each node of
the (r, z) PIC grid; dPhi/dr = 0 at r = 0 (no flux through the axis);
Phi = 0 at both axial ends and at the outer radius. Metal-mask nodes are not
imposed (the workloads with space charge have no electrodes inside the PIC
domain). The right-hand side is the node charge Q deposited by CIC, so the
discrete equation of node (i, j) is

    sum over faces of (face area) * (Phi_neighbour - Phi_ij) / spacing = -Q_ij / eps0

with radial faces at r_{i +- 1/2} = (i +- 1/2) dr (area 2 pi r dz; none inside
r = 0) and axial faces of the annulus area pi (r_{i+1/2}^2 - r_{i-1/2}^2)
(pi (dr/2)^2 on the axis). The system is solved directly (SuperLU) in FP64.
Pinned in the tests by: the uniformly charged cylinder's closed form, the
ring-charge Green's function of a grounded cylinder (brute force over
charges), and the discrete residual.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

EPS0 = 8.8541878128e-12
E_CHARGE = 1.602176634e-19
Q_UNIT = E_CHARGE / 2.0 ** 30  # one fixed-point charge unit of the CIC deposit


def fv_matrix(pic):
    """Sparse operator A on the unknown nodes i = 0..nr-2, j = 1..nz-2, and
    the map from unknown index to (j, i)."""
    nr, nz, dr, dz = pic.nr, pic.nz, pic.dr, pic.dz
    ni, nj = nr - 1, nz - 2
    idx = lambda i, j: (j - 1) * ni + i
    rows, cols, vals = [], [], []
    for j in range(1, nz - 1):
        for i in range(0, nr - 1):
            k = idx(i, j)
            r_out = (i + 0.5) * dr
            r_in = (i - 0.5) * dr if i > 0 else 0.0
            a_out = 2.0 * math.pi * r_out * dz / dr
            a_in = 2.0 * math.pi * r_in * dz / dr
            area_z = math.pi * (r_out ** 2 - r_in ** 2)
            a_z = area_z / dz
            diag = -(a_out + a_in + 2.0 * a_z)
            rows.append(k); cols.append(k); vals.append(diag)
            if i + 1 <= nr - 2:
                rows.append(k); cols.append(idx(i + 1, j)); vals.append(a_out)
            if i > 0:
                rows.append(k); cols.append(idx(i - 1, j)); vals.append(a_in)
            if j + 1 <= nz - 2:
                rows.append(k); cols.append(idx(i, j + 1)); vals.append(a_z)
            if j - 1 >= 1:
                rows.append(k); cols.append(idx(i, j - 1)); vals.append(a_z)
    n = ni * nj
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


_cache = {}


def _factor(pic):
    key = (pic.nr, pic.nz, pic.R, pic.z0, pic.z1)
    if key not in _cache:
        A = fv_matrix(pic).tocsc()
        _cache[key] = (A, spla.splu(A))
    return _cache[key]


def rhs(pic, Q):
    """-Q/eps0 on the unknown nodes, Q in fixed-point units of e*2^-30."""
    q = np.asarray(Q, dtype=np.float64)[1:-1, :-1] * Q_UNIT
    return (-q / EPS0).reshape(-1)


def solve(pic, Q):
    """Phi on the full PIC grid [nz][nr] (zeros on the Dirichlet boundary)."""
    A, lu = _factor(pic)
    x = lu.solve(rhs(pic, Q))
    phi = np.zeros((pic.nz, pic.nr))
    phi[1:-1, :-1] = x.reshape(pic.nz - 2, pic.nr - 1)
    return phi


def residual(pic, Q, phi):
    """||b - A phi|| / ||b|| of a candidate solution on the same operator."""
    A, _ = _factor(pic)
    b = rhs(pic, Q)
    x = np.asarray(phi)[1:-1, :-1].reshape(-1)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(b - A @ x) / (nb if nb > 0 else 1.0))


def masked_matrix(pic, metal):
    """Operator with Phi = 0 imposed at metal-mask nodes (the space-charge
    potential vanishes on the electrodes, as the Methods' PIC space-charge
    section states): metal unknowns get the identity row, and their coupling
    is removed from fluid rows (Phi_metal = 0 there). `metal` is a bool array
    [nz][nr]."""
    A = fv_matrix(pic).tocsr()
    m = np.asarray(metal)[1:-1, :-1].reshape(-1).astype(bool)
    keep = sp.diags((~m).astype(np.float64))
    Am = keep @ A @ keep + sp.diags(m.astype(np.float64))
    return Am.tocsc(), m


def solve_masked(pic, Q, metal):
    """Phi [nz][nr] of the masked system, direct solve (zero on metal nodes
    and on the Dirichlet boundary)."""
    Am, m = masked_matrix(pic, metal)
    b = rhs(pic, Q)
    b[m] = 0.0
    x = spla.splu(Am).solve(b)
    phi = np.zeros((pic.nz, pic.nr))
    phi[1:-1, :-1] = x.reshape(pic.nz - 2, pic.nr - 1)
    return phi


def residual_masked(pic, Q, phi, metal):
    Am, m = masked_matrix(pic, metal)
    b = rhs(pic, Q)
    b[m] = 0.0
    x = np.asarray(phi)[1:-1, :-1].reshape(-1)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(b - Am @ x) / (nb if nb > 0 else 1.0))


def pic_metal_from_static(static_grid, static_mask, pic):
    """Metal flag of each PIC node: the static-grid mask at the nearest static
    node (both grids span the same box)."""
    r = np.arange(pic.nr) * pic.dr
    z = pic.z0 + np.arange(pic.nz) * pic.dz
    i = np.clip(np.rint(r / static_grid.dr).astype(int), 0, static_grid.nr - 1)
    j = np.clip(np.rint((z - static_grid.z0) / static_grid.dz).astype(int), 0, static_grid.nz - 1)
    return np.asarray(static_mask)[np.ix_(j, i)] != 0
