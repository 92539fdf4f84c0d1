"""Tip heat equation with Joule heating (test infrastructure only), Sec. 2.1.

eq:heat   C_v dT/dt = div(kappa grad T) + J^2/sigma,  kappa = L T sigma (Wiedemann-Franz, L = 2.0e-8)
eq:cont   div(sigma grad phi_J) = 0, sigma grad phi_J = -J_e on the emitting surface (eq:bce1),
          phi_J = 0 on the bulk bottom (eq:bce3)
eq:bct1-3 kappa grad T . n = P_cath on the surface, T = T_amb on the bulk bottom.

Finite volumes on the solid tip cells.  The paper's bulk substrate is replaced by the tip
alone: the bottom faces of the k=0 solid cells are the bulk bottom (phi_J = 0, T = T_amb,
at half a cell).  Surface heat P_cath = P_N + P_vap + P_bom enters each tip face's owner
cell; emitted current leaves through the same faces.  Implicit Euler over dt_heat with
kappa and sigma evaluated at the old temperature; both linear systems are solved directly.
Cu resistivity and heat capacity are not printed (the paper defers them to earlier work):
stand-ins rho_e = 1.72e-8 T/293 Ohm m and C_v = 3.45e6 J m^-3 K^-1.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import constants as C

CV = 3.45e6
RHO293 = 1.72e-8


def sigma_of_T(T):
    return 1.0 / (RHO293 * np.asarray(T, dtype=np.float64) / 293.0)


def kappa_of_T(T):
    return C.LORENTZ * np.asarray(T, dtype=np.float64) * sigma_of_T(T)


def voxel_graph(grid):
    """Solid cells in linear order, their internal face pairs and their base (k=0) cells."""
    cells = np.nonzero(grid.solid.ravel())[0]
    index = -np.ones(grid.ncell, dtype=np.int64)
    index[cells] = np.arange(len(cells))
    nx, ny = grid.nx, grid.ny
    ci, cj, ck = cells % nx, (cells // nx) % ny, cells // (nx * ny)
    pairs = []
    for (di, dj, dk) in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
        ni, nj, nk = ci + di, cj + dj, ck + dk
        ok = (ni < nx) & (nj < ny) & (nk < grid.nz)
        nb = np.where(ok, grid.cell_index(np.minimum(ni, nx - 1), np.minimum(nj, ny - 1),
                                          np.minimum(nk, grid.nz - 1)), 0)
        ok &= grid.solid.ravel()[nb]
        a = np.nonzero(ok)[0]
        pairs.append(np.stack([a, index[nb[a]]], 1))
    pairs = np.concatenate(pairs)
    base = ck == 0
    return cells, index, pairs, base


def _laplacian(n, pairs, cface, base_coef):
    """SPD matrix sum_f c_f (u_a - u_b)^2 form plus diagonal base coupling."""
    a, b = pairs[:, 0], pairs[:, 1]
    rows = np.concatenate([a, b, a, b, np.arange(n)])
    cols = np.concatenate([a, b, b, a, np.arange(n)])
    vals = np.concatenate([cface, cface, -cface, -cface, base_coef])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def heat_step(grid, T, face_heat_W, face_current_A, dt_heat, T_amb):
    """One implicit heat step.  T: per solid cell (linear order).  face_heat_W / face_current_A:
    per face (tip faces only are used).  Returns (T_new, joule power per cell [W])."""
    cells, index, pairs, base = voxel_graph(grid)
    n = len(cells)
    dx = grid.dx
    A = dx * dx
    sig = sigma_of_T(T)
    kap = kappa_of_T(T)
    # sources per cell from tip faces
    tip = grid.face_owner >= 0
    own = index[grid.face_owner[tip]]
    S = np.zeros(n)
    np.add.at(S, own, face_heat_W[tip])
    Iin = np.zeros(n)
    np.add.at(Iin, own, face_current_A[tip])
    # current continuity: conventional current enters at emitting faces, leaves at the base
    sf = 0.5 * (sig[pairs[:, 0]] + sig[pairs[:, 1]]) * A / dx
    sb = np.where(base, 2.0 * sig * A / dx, 0.0)
    K = _laplacian(n, pairs, sf, sb)
    phiJ = spla.spsolve(K.tocsc(), Iin) if np.any(Iin != 0) else np.zeros(n)
    joule = np.zeros(n)
    pf = sf * (phiJ[pairs[:, 0]] - phiJ[pairs[:, 1]]) ** 2
    np.add.at(joule, pairs[:, 0], 0.5 * pf)
    np.add.at(joule, pairs[:, 1], 0.5 * pf)
    joule += sb * phiJ ** 2
    # heat: (C_v V/dt) (T' - T) = -K_th T' + base kappa (T_amb - T') + S + joule
    kf = 0.5 * (kap[pairs[:, 0]] + kap[pairs[:, 1]]) * A / dx
    kb = np.where(base, 2.0 * kap * A / dx, 0.0)
    Kt = _laplacian(n, pairs, kf, kb)
    m = CV * dx ** 3 / dt_heat
    M = Kt + sp.diags(np.full(n, m))
    rhs = m * T + kb * T_amb + S + joule
    Tn = spla.spsolve(M.tocsc(), rhs)
    return Tn, joule
