"""Pins of the oracle's Coulomb collisions: conservation and the turn of the relative velocity,
the small-angle deflection rate against the Rutherford cross section integrated over impact
parameters (an independent route to the same physics), isotropy of the azimuth, the integer
weight rule and its mean momentum conservation, and the pairings."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import constants as C, coulomb as CO, particles as P, philox
from oracle.grid import Grid


def _pop(g, n_per, w, v, seed, id0, spread=0.0):
    rng = np.random.default_rng(seed)
    n = n_per * g.ncell
    cells = np.repeat(np.arange(g.ncell), n_per)
    i, j, k = cells % g.nx, (cells // g.nx) % g.ny, cells // (g.nx * g.ny)
    f = rng.random((n, 3))
    sp_ = {"x": (i + f[:, 0]).astype(np.float32), "y": (j + f[:, 1]).astype(np.float32),
           "z": (k + f[:, 2]).astype(np.float32)}
    vel = np.asarray(v, dtype=np.float64) + spread * rng.normal(size=(n, 3))
    for c, name in enumerate(("vx", "vy", "vz")):
        sp_[name] = vel[:, c].astype(np.float32)
    sp_["w"] = np.full(n, w, np.int32)
    sp_["id"] = np.arange(id0, id0 + n, dtype=np.uint64)
    return P.stable_sort(g, sp_)


@pytest.mark.parametrize("ma,mb,qa,qb", [(C.M_E, C.M_E, -1, -1), (C.M_E, C.M_CU, -1, 1), (C.M_CU, C.M_CU, 1, 1)])
def test_scatter_conserves_momentum_energy_and_relative_speed(ma, mb, qa, qb):
    rng = np.random.default_rng(1)
    e = C.E_CHARGE
    for _ in range(300):
        vA, vB = rng.normal(size=3) * 3e5, rng.normal(size=3) * 1e4
        words = rng.integers(0, 2 ** 32, 4)
        a, b = CO.scatter_pair(vA, vB, qa * e, qb * e, ma, mb, 1e26, 10.0, 1e-15, words)
        p0, p1 = ma * vA + mb * vB, ma * a + mb * b
        assert np.allclose(p1, p0, rtol=0, atol=1e-11 * (np.linalg.norm(ma * vA) + np.linalg.norm(mb * vB)))
        assert ma * a @ a + mb * b @ b == pytest.approx(ma * vA @ vA + mb * vB @ vB, rel=1e-11)
        assert np.linalg.norm(a - b) == pytest.approx(np.linalg.norm(vA - vB), rel=1e-12)
    assert CO.scatter_pair(np.ones(3), np.ones(3), e, e, ma, mb, 1e26, 10.0, 1e-15, [1, 2, 3, 4]) is None


def test_small_angle_deflection_rate_is_rutherford():
    """An electron beam through Cu+ at rest: the mean square deflection per step equals
    n u dt times the integral of theta^2 over the Rutherford cross section, 8 pi b90^2 lnL with
    b90 = e^2 / (4 pi eps0 m_ab u^2), within the sampling error."""
    g = Grid(4, 4, 4, 1e-9, 0.0, 0.0)
    v = math.sqrt(2 * 200.0 * C.E_CHARGE / C.M_E)
    Wi, Ni_cell, Ne_cell = 50, 6, 4
    prm = {"dt": 2e-17, "seed": 4, "w_min": 1e-3, "coulomb_log": 10.0}
    n = Ni_cell * Wi * prm["w_min"] / g.dx ** 3
    mab = C.M_E * C.M_CU / (C.M_E + C.M_CU)
    b90 = C.E_CHARGE ** 2 / (4 * math.pi * C.EPS0 * mab * v * v)
    expect = n * v * prm["dt"] * 8 * math.pi * b90 ** 2 * prm["coulomb_log"]
    th2 = []
    for step in range(40):
        e, eo = _pop(g, Ne_cell, 1, [0, 0, v], 10 + step, 0)
        i, io = _pop(g, Ni_cell, Wi, [0, 0, 0], 50 + step, 10_000)
        v0 = np.stack([e[c].astype(np.float64) for c in ("vx", "vy", "vz")], 1)
        assert CO.coulomb_ei(g, prm, e, eo, i, io, step) == len(e["w"])
        v1 = np.stack([e[c].astype(np.float64) for c in ("vx", "vy", "vz")], 1)
        cos = np.sum(v0 * v1, 1) / (np.linalg.norm(v0, axis=1) * np.linalg.norm(v1, axis=1))
        th2.append(np.arccos(np.clip(cos, -1, 1)) ** 2)
    th2 = np.concatenate(th2)
    assert 1e-4 < expect < 1e-2            # the small-angle regime
    assert th2.mean() == pytest.approx(expect, rel=5 * math.sqrt(2.0 / len(th2)))


def test_azimuth_is_uniform_and_scattering_symmetric():
    g = Grid(4, 4, 4, 1e-9, 0.0, 0.0)
    v = 2e6
    prm = {"dt": 2e-17, "seed": 9, "w_min": 1e-3}
    dv = []
    for step in range(20):
        e, eo = _pop(g, 4, 1, [0, 0, v], 70 + step, 0)
        i, io = _pop(g, 6, 30, [0, 0, 0], 90 + step, 10_000)
        CO.coulomb_ei(g, prm, e, eo, i, io, step)
        dv.append(np.stack([e["vx"].astype(np.float64), e["vy"].astype(np.float64)], 1))
    dv = np.concatenate(dv)
    s = np.abs(dv).mean()
    assert np.all(np.abs(dv.mean(0)) < 5 * s / math.sqrt(len(dv)))
    assert (dv[:, 0] ** 2).mean() == pytest.approx((dv[:, 1] ** 2).mean(), rel=0.1)


def test_like_pairs_conserve_cell_momentum_and_energy():
    g = Grid(3, 3, 2, 1e-9, 0.0, 0.0)
    prm = {"dt": 1e-16, "seed": 2, "w_min": 1e-3}
    for N in (2, 3, 5):
        e, eo = _pop(g, N, 4, [0, 0, 0], N, 0, spread=1e6)
        v0 = np.stack([e[c].astype(np.float64) for c in ("vx", "vy", "vz")], 1)
        assert CO.coulomb_ee(g, prm, e, eo, 3) == g.ncell * (N // 2)
        v1 = np.stack([e[c].astype(np.float64) for c in ("vx", "vy", "vz")], 1)
        moved = np.any(v1 != v0, axis=1)
        assert np.all(np.add.reduceat(moved.astype(int), eo[:-1]) == 2 * (N // 2))
        for c in range(g.ncell):
            s = slice(eo[c], eo[c + 1])
            assert np.allclose(v1[s].sum(0), v0[s].sum(0), rtol=0, atol=1e-6 * np.abs(v0[s]).sum())
            assert (v1[s] ** 2).sum() == pytest.approx((v0[s] ** 2).sum(), rel=1e-6)


def test_weight_rule_exact_and_mean_momentum():
    rng = np.random.default_rng(5)
    for _ in range(2000):
        word = int(rng.integers(0, 2 ** 32))
        ws = int(rng.integers(1, 2 ** 20))
        wl = ws + int(rng.integers(0, 2 ** 20))
        assert CO.weight_keeps(word, ws, wl) == (Fraction(2 * (word >> 8) + 1, 2 ** 25) < Fraction(ws, wl))
    # ions of weight 1 and 3 in every cell: the heavier turns with probability 1/3
    g = Grid(4, 4, 4, 1e-9, 0.0, 0.0)
    prm = {"dt": 1e-14, "seed": 21, "w_min": 1e-3}
    took, pairs = 0, 0
    dp = np.zeros(3)
    scale = 0.0
    for step in range(30):
        a, _ = _pop(g, 1, 1, [0, 0, 2e4], 300 + step, 0, spread=5e3)
        b, _ = _pop(g, 1, 3, [0, 0, 0], 400 + step, 5000, spread=5e3)
        m, mo = P.stable_sort(g, {k: np.concatenate([a[k], b[k]]) for k in P.FIELDS})
        v0 = np.stack([m[c].astype(np.float64) for c in ("vx", "vy", "vz")], 1)
        CO.coulomb_ii(g, prm, m, mo, step)
        v1 = np.stack([m[c].astype(np.float64) for c in ("vx", "vy", "vz")], 1)
        heavy = m["w"] == 3
        took += int(np.sum(np.any(v1[heavy] != v0[heavy], axis=1)))
        pairs += int(heavy.sum())
        w = m["w"].astype(np.float64)[:, None]
        dp += (w * (v1 - v0)).sum(0)
        scale += float(np.sqrt((w[:, 0] ** 2 * ((v1 - v0) ** 2).sum(1)).sum()))
    assert abs(took / pairs - 1 / 3) < 4 * math.sqrt(pairs * 2 / 9) / pairs
    assert np.all(np.abs(dp) < 4 * scale / math.sqrt(30))
    assert philox.PAIR not in (CO.PAIR_EE, CO.PAIR_EI, CO.PAIR_II)
