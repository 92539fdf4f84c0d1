"""Pins of oracle functions against values fixed outside the oracle: the published Philox
known-answer vectors, face and voxel counts of the staircased tips (a brute-force count written
here as plain loops, and the counts of the workload geometries), and closed-form values of the
field-ionization rate (eq:dfi) and the evaporation flux (Sec. 2.3.1)."""
import os

import numpy as np
import pytest

from oracle import collide, philox, surface
from oracle.grid import Grid

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_philox_matches_published_known_answer_vectors():
    """Philox4x32-10 against the three known-answer vectors published with the generator
    (Salmon et al., SC'11), read from tests/golden/philox4x32_10_kat.txt."""
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(t, 16) for t in line.split()])
    assert len(rows) == 3
    for r in rows:
        c0, c1, c2, c3, k0, k1 = r[:6]
        out = philox.philox4x32_10(c0, c1, c2, c3, k0, k1)
        assert [int(o) for o in out] == r[6:], [hex(int(o)) for o in out]


def brute_force_counts(nx, ny, nz, dx, r, h):
    """Voxels, tip faces and cathode-plane faces of the staircased tip, counted cell by cell.

    A cell is solid when its centre lies in the cylinder of radius r below z = h - r or in the
    ball of radius r about the axis point at z = h - r (the tip height includes the cap).  A tip
    face lies between a vacuum cell and a solid neighbour; a plane face is the z = 0 face of a
    vacuum cell in the bottom layer."""
    rc, hc = r / dx, h / dx
    ax, ay, zc = nx / 2.0, ny / 2.0, hc - rc

    def solid(i, j, k):
        if not (0 <= i < nx and 0 <= j < ny and 0 <= k < nz):
            return False
        x, y, z = i + 0.5 - ax, j + 0.5 - ay, k + 0.5
        if x * x + y * y <= rc * rc and z <= zc:
            return True
        return x * x + y * y + (z - zc) ** 2 <= rc * rc

    vox = tip = plane = 0
    kmax = int(hc) + 2
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                if k > kmax:          # above the tip every cell is vacuum with vacuum neighbours
                    continue
                if solid(i, j, k):
                    vox += 1
                    continue
                for di, dj, dk in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)):
                    tip += solid(i + di, j + dj, k + dk)
    plane = sum(1 for j in range(ny) for i in range(nx) if not solid(i, j, 0))
    return vox, tip, plane


def oracle_counts(g):
    vox = int(g.solid.sum())
    tip = int(np.sum(g.face_owner >= 0))
    plane = int(np.sum(g.face_owner < 0))
    return vox, tip, plane


def test_face_counts_small_workload_against_brute_force():
    """32x32x64 cells, dx 1 nm, tip r 3 nm h 20 nm: 612 voxels, 504 tip faces, 992 plane faces
    (brute force here, and the counts of the workload geometry)."""
    bf = brute_force_counts(32, 32, 64, 1e-9, 3e-9, 20e-9)
    assert bf == (612, 504, 992)
    assert oracle_counts(Grid(32, 32, 64, 1e-9, 3e-9, 20e-9)) == bf


@pytest.mark.parametrize("args", [(12, 10, 20, 1e-9, 2.5e-9, 9e-9), (16, 16, 24, 0.5e-9, 1.7e-9, 6.1e-9),
                                  (9, 9, 9, 1e-9, 0.0, 0.0)])
def test_face_counts_odd_shapes_against_brute_force(args):
    """Off-centre axes (odd cell counts), a cap cut below a half cell, and no tip at all."""
    assert oracle_counts(Grid(*args)) == brute_force_counts(*args)


@pytest.mark.slow
def test_face_counts_production_workload():
    """256x256x512 cells, dx 0.5 nm, tip r 5 nm h 60 nm: 36 872 voxels, 9 748 tip faces and
    65 220 plane faces."""
    assert oracle_counts(Grid(256, 256, 512, 0.5e-9, 5e-9, 60e-9)) == (36872, 9748, 65220)


@pytest.mark.parametrize("E,P", [(8.0, 3.0967e-4), (10.0, 8.3752e-3), (12.0, 7.1384e-2), (15.0, 0.56868)])
def test_dfi_rate_closed_form_values(E, P):
    """eq:dfi for Cu (xi = 7.726 eV, z = 1), evaluated by hand at 8, 10, 12 and 15 GV/m [1/fs]."""
    assert float(collide.adk_rate_per_fs(E)) == pytest.approx(P, rel=1e-4)


@pytest.mark.parametrize("T,phi", [(2000.0, 2.1315e24), (3000.0, 1.3235e27), (4000.0, 3.1607e28)])
def test_evaporation_flux_closed_form_values(T, phi):
    """Clausius-Clapeyron vapour pressure over the kinetic wall flux (Sec. 2.3.1) with
    E_vap = 3.43 eV, T_b = 2835 K, p_atm = 101325 Pa, m = 63.546 u [atoms / m^2 s]."""
    assert surface.evaporation_flux(T) == pytest.approx(phi, rel=1e-4)
