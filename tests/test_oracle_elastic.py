"""Pins of the oracle's elastic collisions and charge exchange: the mechanics of eq:newv with
eq:du (momentum, energy, relative speed, scattering angle), isotropy, the collision rate
n sigma v, the pairings (brute force on small cells), the integer weight rule and its mean
momentum conservation."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import constants as C, elastic as EL, particles as P, philox
from oracle.grid import Grid


@pytest.mark.parametrize("mA,mB", [(C.M_E, C.M_CU), (C.M_CU, C.M_CU), (1.0, 3.0)])
def test_newv_conserves_momentum_energy_and_turns_u_by_theta(mA, mB):
    rng = np.random.default_rng(3)
    for _ in range(200):
        vA, vB = rng.normal(size=3) * 1e5, rng.normal(size=3) * 1e4
        ct, ph = 2 * rng.random() - 1, 2 * math.pi * rng.random()
        a, b = EL.elastic_velocities(vA, vB, mA, mB, ct, ph)
        p0, p1 = mA * vA + mB * vB, mA * a + mB * b
        assert np.allclose(p1, p0, rtol=0, atol=1e-11 * np.linalg.norm(mA * vA) + 1e-11 * np.linalg.norm(mB * vB))
        K0 = mA * vA @ vA + mB * vB @ vB
        assert (mA * a @ a + mB * b @ b) == pytest.approx(K0, rel=1e-11)
        u0, u1 = vA - vB, a - b
        assert np.linalg.norm(u1) == pytest.approx(np.linalg.norm(u0), rel=1e-12)
        # the relative velocity turns by the drawn scattering angle theta'
        assert u0 @ u1 / (u0 @ u0) == pytest.approx(ct, abs=1e-9)


def test_scattered_relative_velocity_is_isotropic():
    rng = np.random.default_rng(4)
    u = np.array([2.0, -1.0, 0.5])
    out = np.array([u + EL.delta_u(u, 2 * rng.random() - 1, 2 * math.pi * rng.random()) for _ in range(20000)])
    s = np.linalg.norm(u)
    assert np.allclose(np.linalg.norm(out, axis=1), s)
    assert np.all(np.abs(out.mean(axis=0)) < s * 4 / math.sqrt(3 * 20000))
    assert np.allclose((out ** 2).mean(axis=0), s * s / 3, rtol=0.03)


def test_weight_rule_is_exact_in_integers():
    rng = np.random.default_rng(5)
    for _ in range(3000):
        word = int(rng.integers(0, 2 ** 32))
        ws = int(rng.integers(1, 2 ** 20))
        wl = ws + int(rng.integers(0, 2 ** 20))
        U = Fraction(2 * (word >> 8) + 1, 2 ** 25)
        assert EL.weight_keeps(word, ws, wl) == (U < Fraction(ws, wl))
    assert EL.weight_keeps(0xFFFFFFFF, 7, 7)      # equal weights: always


def _cells_population(g, n_per, w, v, seed, id0, spread=0.0):
    """n_per SPs in every cell, weight w, velocity v (+ Gaussian spread), cell-sorted."""
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


def test_elastic_rate_equals_n_sigma_v():
    """Mono-energetic electrons through cold neutrals: the colliding fraction of electron SPs is
    1 - exp(-v n sigma dt) per step (n the real neutral density), within 3 binomial sigma."""
    g = Grid(4, 4, 4, 1e-9, 0.0, 0.0)
    v = math.sqrt(2 * 20.0 * C.E_CHARGE / C.M_E)
    wn, we, n_per_e, n_per_n = 40, 1, 2, 5
    prm = {"dt": 1e-16, "seed": 11, "w_min": 0.02, "sigma_el_en": 2e-19}
    n_real = n_per_n * wn * prm["w_min"] / g.dx ** 3
    p = -math.expm1(-v * n_real * prm["sigma_el_en"] * prm["dt"])
    total, trials = 0, 0
    for step in range(8):
        e, eo = _cells_population(g, n_per_e, we, [0, 0, v], 100 + step, 0)
        n, no = _cells_population(g, n_per_n, wn, [0, 0, 0], 200 + step, 10_000)
        v0 = e["vz"].copy()
        ev = EL.elastic_en(g, prm, e, eo, n, no, step)
        changed = int(np.sum(e["vz"] != v0))
        assert ev == changed                          # the lighter SP (weight 1) always turns
        total += ev
        trials += len(e["id"])
    assert p * trials > 100
    assert abs(total - p * trials) < 3 * math.sqrt(trials * p * (1 - p))


def test_like_species_pairs_cover_each_cell_once():
    """With P = 1 every pair collides: floor(N/2) events per cell, every SP of an even cell
    turned once, exactly one SP of an odd cell left as it was (brute force on small cells)."""
    g = Grid(3, 2, 2, 1e-9, 0.0, 0.0)
    prm = {"dt": 1e-12, "seed": 3, "w_min": 1.0, "sigma_el_nn": 1e-12}
    for N in (2, 3, 4, 5):
        n, no = _cells_population(g, N, 2, [0, 0, 0], N, 0, spread=300.0)
        before = {c: n[c].copy() for c in ("vx", "vy", "vz")}
        ev = EL.elastic_nn(g, prm, n, no, step=7)
        assert ev == g.ncell * (N // 2)
        moved = (n["vx"] != before["vx"]) | (n["vy"] != before["vy"]) | (n["vz"] != before["vz"])
        per_cell = np.add.reduceat(moved.astype(int), no[:-1])
        assert np.all(per_cell == 2 * (N // 2))
        # momentum of each cell conserved (equal masses and weights) to float32 rounding
        for c in range(g.ncell):
            s = slice(no[c], no[c + 1])
            for name in ("vx", "vy", "vz"):
                p0 = before[name][s].astype(np.float64).sum()
                p1 = n[name][s].astype(np.float64).sum()
                assert abs(p1 - p0) <= 1e-6 * (np.abs(before[name][s]).sum() + 1.0)


def test_charge_exchange_swaps_velocities_of_equal_weights():
    g = Grid(2, 2, 2, 1e-9, 0.0, 0.0)
    prm = {"dt": 1e-12, "seed": 8, "w_min": 1.0, "sigma_cx": 1e-12}
    i, io = _cells_population(g, 2, 3, [0, 0, -2e4], 1, 0, spread=500.0)
    n, no = _cells_population(g, 3, 3, [0, 0, 0], 2, 1000, spread=500.0)
    iv = np.stack([i[c].copy() for c in ("vx", "vy", "vz")], 1)
    nv = np.stack([n[c].copy() for c in ("vx", "vy", "vz")], 1)
    w0 = (i["w"].copy(), n["w"].copy())
    ev = EL.charge_exchange(g, prm, i, io, n, no, step=2)
    assert ev == 2 * g.ncell                        # P = 1: every ion (the projectile) exchanges
    iv1 = np.stack([i[c] for c in ("vx", "vy", "vz")], 1)
    nv1 = np.stack([n[c] for c in ("vx", "vy", "vz")], 1)
    # each ion now carries a neutral's old velocity and that neutral the ion's
    for a in range(len(iv1)):
        hit = np.nonzero(np.all(nv == iv1[a], axis=1))[0]
        assert len(hit) == 1 and np.array_equal(nv1[hit[0]], iv[a])
    assert np.array_equal(i["w"], w0[0]) and np.array_equal(n["w"], w0[1])
    assert np.allclose(iv1.sum(0) + nv1.sum(0), iv.sum(0) + nv.sum(0), rtol=0, atol=1e-3)


def test_weighted_pairs_conserve_momentum_on_average():
    """One neutral SP of weight 1 and one of weight 3 in every cell (P = 1): the heavier SP takes
    its post-collision velocity with probability 1/3, so the real-particle momentum change
    averages to zero."""
    g = Grid(4, 4, 4, 1e-9, 0.0, 0.0)
    prm = {"dt": 1e-12, "seed": 21, "w_min": 1.0, "sigma_el_nn": 1e-12}
    dp, took, pairs, scale = np.zeros(3), 0, 0, 0.0
    for step in range(40):
        a, ao = _cells_population(g, 1, 1, [0, 0, 3e3], 300 + step, 0, spread=1e3)
        b, bo = _cells_population(g, 1, 3, [0, 0, 0], 400 + step, 5000, spread=1e3)
        # one like-species pass over a merged cell-sorted population: pairs (light, heavy)
        m = {k: np.concatenate([a[k], b[k]]) for k in P.FIELDS}
        m, mo = P.stable_sort(g, m)
        v0 = np.stack([m[c].astype(np.float64) for c in ("vx", "vy", "vz")], 1)
        EL.elastic_nn(g, prm, m, mo, step)
        v1 = np.stack([m[c].astype(np.float64) for c in ("vx", "vy", "vz")], 1)
        w = m["w"].astype(np.float64)[:, None]
        dp += (w * (v1 - v0)).sum(0)
        heavy = m["w"] == 3
        took += int(np.sum(np.any(v1[heavy] != v0[heavy], axis=1)))
        pairs += int(heavy.sum())
        scale += float(np.sqrt((w[:, 0] ** 2 * ((v1 - v0) ** 2).sum(1)).sum()))
    assert abs(took / pairs - 1 / 3) < 4 * math.sqrt(pairs / 3 * 2 / 3) / pairs
    assert np.all(np.abs(dp) < 4 * scale / math.sqrt(40))


def test_zero_weight_pairs_do_not_collide():
    g = Grid(1, 1, 1, 1e-9, 0.0, 0.0)
    prm = {"dt": 1e-12, "seed": 1, "w_min": 1.0, "sigma_el_en": 1e-12}
    e, eo = _cells_population(g, 1, 1, [0, 0, 1e6], 1, 0)
    n, no = _cells_population(g, 2, 0, [0, 0, 0], 2, 10)
    assert EL.elastic_en(g, prm, e, eo, n, no, 0) == 0
    assert philox.PAIR not in (EL.PAIR_EN, EL.PAIR_NN, EL.PAIR_CX)
