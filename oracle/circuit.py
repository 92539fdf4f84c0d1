"""External RC circuit and the Shockley-Ramo gap current (test infrastructure only).

The paper couples the gap to its power source by the RC circuit of ArcPIC (the passage after
the evaporative-cooling equation, Sec. 2.3.1): with applied voltage V0, resistance R and gap
capacitance C,
    V_gap(t) = V0 + (1/C) * integral_0^t (I_tot - I_gap) dt,    I_tot = (V0 - V_gap) / R,
and the gap current is the Shockley-Ramo current of the moving charges,
    I_gap = sum over charged SPs of q v . E0(r),
with E0 the Laplace field for the anode at unit potential and no space charge.

Readings (the paper gives the equations only):
  * the integral is advanced by explicit Euler once per PIC step, from V_gap and I_gap at the
    start of the step: V_gap <- V_gap + dt/C (I_tot - I_gap);
  * I_gap is taken after the push, from the new positions and the half-step velocities of
    electrons and Cu+ (q = Z e w w_min per SP) that are still in the vacuum region (SPs the
    push removed at a boundary no longer move in the gap), with E0 gathered by the same
    cloud-in-cell weights as E;
  * E0 is the node field of the unit Laplace solution by central differences (one-sided on the
    cathode and anode planes, mirrored at the lateral walls), in float64;
  * the anode potential of the step's Poisson solve is the updated V_gap.
"""
import numpy as np

from . import constants as C
from . import field


def unit_field(grid):
    """E0 = -grad(phi_1), phi_1 the Laplace solution with the anode at 1 V (units 1/m), float64
    array (nz+1, ny+1, nx+1, 3)."""
    phi1 = field.solve_poisson(grid, 1.0)
    nx, ny, nz, dx = grid.nx, grid.ny, grid.nz, grid.dx
    ii, jj = np.arange(nx + 1), np.arange(ny + 1)
    E0 = np.zeros((nz + 1, ny + 1, nx + 1, 3))
    E0[..., 0] = (phi1[:, :, field._mirror(ii - 1, nx)] - phi1[:, :, field._mirror(ii + 1, nx)]) / (2 * dx)
    E0[..., 1] = (phi1[:, field._mirror(jj - 1, ny), :] - phi1[:, field._mirror(jj + 1, ny), :]) / (2 * dx)
    E0[1:-1, ..., 2] = (phi1[:-2] - phi1[2:]) / (2 * dx)
    E0[0, ..., 2] = (phi1[0] - phi1[1]) / dx
    E0[-1, ..., 2] = (phi1[-2] - phi1[-1]) / dx
    return E0


def gather64(E0, x, y, z):
    """Cloud-in-cell (trilinear) gather of a node field at positions in cell units, float64."""
    x, y, z = (np.asarray(a, dtype=np.float64) for a in (x, y, z))
    i, j, k = np.floor(x).astype(np.int64), np.floor(y).astype(np.int64), np.floor(z).astype(np.int64)
    fx, fy, fz = x - i, y - j, z - k
    out = np.zeros((len(x), 3))
    for dk, wz in ((0, 1 - fz), (1, fz)):
        for dj, wy in ((0, 1 - fy), (1, fy)):
            for di, wx in ((0, 1 - fx), (1, fx)):
                out += (wx * wy * wz)[:, None] * E0[k + dk, j + dj, i + di]
    return out


def gap_current(E0, species, w_min):
    """I_gap = sum_s sum_i Z_s e w_i w_min v_i . E0(x_i) [A]; species: iterable of (Z, SoA)."""
    total = 0.0
    for Z, sp_ in species:
        if Z == 0 or len(sp_["x"]) == 0:
            continue
        e0 = gather64(E0, sp_["x"], sp_["y"], sp_["z"])
        v = np.stack([np.asarray(sp_[c], dtype=np.float64) for c in ("vx", "vy", "vz")], 1)
        q = Z * C.E_CHARGE * np.asarray(sp_["w"], dtype=np.float64) * w_min
        total += float(np.sum(q * np.sum(v * e0, axis=1)))
    return total


def circuit_step(V_gap, I_gap, V0, R, Cg, dt):
    """One explicit Euler step of the RC circuit: returns (V_gap_new, I_tot)."""
    I_tot = (V0 - V_gap) / R
    return V_gap + dt / Cg * (I_tot - I_gap), I_tot
