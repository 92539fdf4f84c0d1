"""Pins of the oracle's electrostatics (eq:poi, eq:bcf1-3) against closed forms."""
import math

import numpy as np
import pytest

from oracle import constants as C
from oracle import field, particles as P
from oracle.grid import Grid


def test_parallel_plate_is_linear():
    # no tip: the discrete solution of Laplace between the plates is exactly V0 z / L
    g = Grid(8, 6, 12, 1e-9, 0.0, 0.0)
    assert g.solid.sum() == 0
    phi = field.solve_poisson(g, 7.5)
    z = np.arange(g.nz + 1)[:, None, None] / g.nz
    assert np.max(np.abs(phi - 7.5 * z)) < 1e-12 * 7.5


def test_discrete_eigenfunction_with_mirror_walls():
    # sin in z (Dirichlet planes) times cos in x, y (mirror walls) is an exact eigenvector of the
    # 7-point operator; a wrong lateral condition or stencil scale breaks it
    g = Grid(10, 8, 12, 2e-9, 0.0, 0.0)
    k, j, i = np.meshgrid(np.arange(g.nz + 1), np.arange(g.ny + 1), np.arange(g.nx + 1), indexing="ij")
    u = np.sin(math.pi * k / g.nz) * np.cos(math.pi * i / g.nx) * np.cos(2 * math.pi * j / g.ny)
    lam = (2 - 2 * math.cos(math.pi / g.nz) + 2 - 2 * math.cos(math.pi / g.nx)
           + 2 - 2 * math.cos(2 * math.pi / g.ny)) / g.dx ** 2
    phi = field.solve_poisson(g, 0.0, lam * u)
    assert np.max(np.abs(phi - u)) < 1e-10


def test_gauss_law_around_deposited_charge():
    # the flux of the discrete field out of a box equals the enclosed charge / eps0
    g = Grid(12, 12, 12, 1e-9, 0.0, 0.0)
    sp_ = P.empty()
    for f, v in (("x", 6.0), ("y", 6.0), ("z", 6.0), ("vx", 0.0), ("vy", 0.0), ("vz", 0.0)):
        sp_[f] = np.array([v], np.float32)
    sp_["w"] = np.array([3], np.int32)
    sp_["id"] = np.array([0], np.uint64)
    Q = P.deposit(g, sp_, 1)
    assert Q[6, 6, 6] == 3 << 30 and Q.sum() == 3 << 30
    f = field.rhs_from_charge(g, Q, w_min=2.0)
    phi = field.solve_poisson(g, 0.0, f)
    a, b = 4, 8                    # box of nodes [a, b]^3 around the charge
    flux = 0.0
    for ax in range(3):
        for side, (inn, out) in ((0, (a, a - 1)), (1, (b, b + 1))):
            sl_in = [slice(a, b + 1)] * 3
            sl_out = [slice(a, b + 1)] * 3
            sl_in[ax] = inn
            sl_out[ax] = out
            flux += np.sum(phi[tuple(sl_in)] - phi[tuple(sl_out)]) / g.dx * g.dx ** 2
    q = 3 * 2.0 * C.E_CHARGE
    assert flux == pytest.approx(q / C.EPS0, rel=1e-9)


@pytest.mark.slow
def test_hemisphere_boss_in_uniform_field():
    # grounded hemisphere of radius R on a grounded plane in a uniform field E0:
    # phi = E0 z (1 - R^3/r^3), r from the centre on the plane (image of a sphere in a field)
    R = 8
    g = Grid(48, 48, 48, 1.0, R, R)          # tip height = radius: a bare hemispherical cap
    E0 = 1.0
    L = g.nz
    phi = field.solve_poisson(g, E0 * L * (1 - R ** 3 / L ** 3))
    k, j, i = np.meshgrid(np.arange(g.nz + 1), np.arange(g.ny + 1), np.arange(g.nx + 1), indexing="ij")
    x, y, z = i - g.ax, j - g.ay, k.astype(float)
    r = np.sqrt(x * x + y * y + z * z)
    exact = E0 * z * (1 - R ** 3 / np.maximum(r, 1e-9) ** 3)
    # a staircase of radius 8 cells and a finite mirror box: a few % from the analytic form
    for rmin, tol in ((2, 0.06), (3, 0.03)):
        m = (r >= rmin * R) & (np.sqrt(x * x + y * y) < 16) & (z > 0) & (z < L - 8)
        err = np.abs(phi[m] - exact[m]) / (E0 * z[m])
        assert err.max() < tol
    # field enhancement on top of a boss is 3 E0; one cell above the staircase apex it is lower
    assert 1.8 < phi[R + 2, 24, 24] - phi[R + 1, 24, 24] < 3.0


def test_efield_uniform_and_mirror():
    g = Grid(6, 5, 8, 1e-9, 0.0, 0.0)
    phi = field.solve_poisson(g, 4.0)
    E = field.efield(g, phi)
    assert np.allclose(E[..., 2], np.float32(-4.0 / (g.nz * g.dx)), rtol=1e-6)
    # the mirror walls make the normal component vanish exactly on x=0, x=nx, y=0, y=ny
    assert np.all(E[:, :, 0, 0] == 0) and np.all(E[:, :, -1, 0] == 0)
    assert np.all(E[:, 0, :, 1] == 0) and np.all(E[:, -1, :, 1] == 0)
    assert np.max(np.abs(E[..., :2])) < 1e-9 * 4.0 / (g.nz * g.dx)
