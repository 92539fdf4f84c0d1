"""Pins of the oracle's elastic collisions and charge exchange: the mechanics of eq:newv with
eq:du (momentum, energy, relative speed, scattering angle), isotropy, the collision rate
n sigma v per sub-particle, the pairings (brute force on small cells), and the splitting of
Sec. 2.3.2 (weights, exact momentum, ids)."""
import math

import numpy as np
import pytest

from oracle import collide, constants as C, elastic as EL, particles as P, philox
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


def _sub_collisions(sp_, before_v, new):
    """Colliding sub-particles of one species in a pass: the weights of its new SPs plus the
    weights of the SPs that turned whole."""
    turned = np.any([sp_[c] != before_v[c] for c in ("vx", "vy", "vz")], axis=0)
    return int(new["w"].astype(np.int64).sum()) + int(sp_["w"][turned].astype(np.int64).sum())


def test_elastic_rate_equals_n_sigma_v():
    """Mono-energetic electrons (weight 3) through cold neutrals: each electron sub-particle
    collides with probability 1 - exp(-v n sigma dt) per step (n the real neutral density),
    within 3 binomial sigma."""
    g = Grid(4, 4, 4, 1e-9, 0.0, 0.0)
    v = math.sqrt(2 * 20.0 * C.E_CHARGE / C.M_E)
    wn, we, n_per_e, n_per_n = 40, 3, 2, 5
    prm = {"dt": 1e-16, "seed": 11, "w_min": 0.02, "sigma_el_en": 2e-19}
    n_real = n_per_n * wn * prm["w_min"] / g.dx ** 3
    p = -math.expm1(-v * n_real * prm["sigma_el_en"] * prm["dt"])
    total, trials = 0, 0
    for step in range(8):
        e, eo = _cells_population(g, n_per_e, we, [0, 0, v], 100 + step, 0)
        n, no = _cells_population(g, n_per_n, wn, [0, 0, 0], 200 + step, 10_000)
        before = {c: e[c].copy() for c in ("vx", "vy", "vz")}
        ids = collide.Counter(50_000)
        new_e, new_n, ev = EL.elastic_en(g, prm, e, eo, n, no, step, ids)
        total += _sub_collisions(e, before, new_e)
        trials += int(e["w"].sum()) + int(new_e["w"].sum())
        # both sides of an event move the same number of sub-particles
        assert int(new_n["w"].sum()) == _sub_collisions(e, before, new_e)
        assert len(new_n["w"]) == ev and ids.next_id == 50_000 + len(new_e["w"]) + len(new_n["w"])
    assert p * trials > 300
    assert abs(total - p * trials) < 3 * math.sqrt(trials * p * (1 - p))


def test_like_species_pairs_cover_each_cell_once():
    """With P = 1 and equal weights every sub-particle collides, so whole SPs turn: floor(N/2)
    events per cell, every SP of an even cell turned once, exactly one SP of an odd cell left
    as it was (brute force on small cells)."""
    g = Grid(3, 2, 2, 1e-9, 0.0, 0.0)
    prm = {"dt": 1e-12, "seed": 3, "w_min": 1.0, "sigma_el_nn": 1e-12}
    for N in (2, 3, 4, 5):
        n, no = _cells_population(g, N, 2, [0, 0, 0], N, 0, spread=300.0)
        before = {c: n[c].copy() for c in ("vx", "vy", "vz")}
        new, ev = EL.elastic_nn(g, prm, n, no, 7, collide.Counter(0))
        assert ev == g.ncell * (N // 2) and len(new["w"]) == 0
        moved = (n["vx"] != before["vx"]) | (n["vy"] != before["vy"]) | (n["vz"] != before["vz"])
        per_cell = np.add.reduceat(moved.astype(int), no[:-1])
        assert np.all(per_cell == 2 * (N // 2))
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
    new_i, new_n, ev = EL.charge_exchange(g, prm, i, io, n, no, 2, collide.Counter(0))
    assert ev == 2 * g.ncell and len(new_i["w"]) == 0 and len(new_n["w"]) == 0   # P = 1, equal weights
    iv1 = np.stack([i[c] for c in ("vx", "vy", "vz")], 1)
    nv1 = np.stack([n[c] for c in ("vx", "vy", "vz")], 1)
    # each ion now carries a neutral's old velocity and that neutral the ion's
    for a in range(len(iv1)):
        hit = np.nonzero(np.all(nv == iv1[a], axis=1))[0]
        assert len(hit) == 1 and np.array_equal(nv1[hit[0]], iv[a])
    assert np.array_equal(i["w"], w0[0]) and np.array_equal(n["w"], w0[1])


def _momentum(sps, m):
    return sum((sp_["w"].astype(np.float64)[:, None] * m *
                np.stack([sp_[c].astype(np.float64) for c in ("vx", "vy", "vz")], 1)).sum(0) for sp_ in sps)


def test_splitting_conserves_weight_and_momentum():
    """Unequal weights (Sec. 2.3.2): the colliding sub-particles leave both SPs as new SPs of
    weight N_coll, so every species keeps its weight and the real-particle momentum is conserved
    up to the float32 storage of the velocities; ids are consecutive."""
    g = Grid(3, 3, 3, 1e-9, 0.0, 0.0)
    prm = {"dt": 1e-16, "seed": 5, "w_min": 0.02, "sigma_el_en": 3e-19, "sigma_el_nn": 3e-15, "sigma_cx": 3e-16}
    v = math.sqrt(2 * 30.0 * C.E_CHARGE / C.M_E)
    e, eo = _cells_population(g, 3, 5, [0, 0, v], 1, 0, spread=0.2 * v)
    n, no = _cells_population(g, 4, 7, [0, 0, 0], 2, 1000, spread=800.0)
    i, io = _cells_population(g, 2, 4, [0, 0, -3e4], 3, 2000, spread=2e3)
    n["w"][::3] = 2
    e0, n0, i0 = (int(x["w"].sum()) for x in (e, n, i))
    ids = collide.Counter(9000)
    p_en0 = _momentum([e], C.M_E) + _momentum([n], C.M_CU)
    ne_, nn1, ev1 = EL.elastic_en(g, prm, e, eo, n, no, 0, ids)
    p_en1 = _momentum([e, ne_], C.M_E) + _momentum([n, nn1], C.M_CU)
    assert ev1 > 5 and len(ne_["w"]) > 0
    assert np.allclose(p_en1, p_en0, rtol=0, atol=1e-6 * np.abs(_momentum([e], C.M_E)).max())
    p_nn0 = _momentum([n, nn1], C.M_CU)
    nn2, ev2 = EL.elastic_nn(g, prm, n, no, 0, ids)
    assert ev2 > 5
    assert np.allclose(_momentum([n, nn1, nn2], C.M_CU), p_nn0, rtol=0, atol=1e-6 * np.abs(p_nn0).max() + 1e-30)
    p_cx0 = _momentum([i], C.M_CU) + _momentum([n, nn1, nn2], C.M_CU)
    ni_, nn3, ev3 = EL.charge_exchange(g, prm, i, io, n, no, 0, ids)
    assert ev3 > 5
    p_cx1 = _momentum([i, ni_], C.M_CU) + _momentum([n, nn1, nn2, nn3], C.M_CU)
    assert np.allclose(p_cx1, p_cx0, rtol=0, atol=1e-6 * np.abs(_momentum([i], C.M_CU)).max())
    assert int(e["w"].sum()) + int(ne_["w"].sum()) == e0
    assert int(n["w"].sum()) + sum(int(x["w"].sum()) for x in (nn1, nn2, nn3)) == n0
    assert int(i["w"].sum()) + int(ni_["w"].sum()) == i0
    new_ids = np.concatenate([x["id"] for x in (ne_, nn1, nn2, ni_, nn3)])
    assert sorted(new_ids.tolist()) == list(range(9000, ids.next_id))


def test_zero_weight_pairs_do_not_collide():
    g = Grid(1, 1, 1, 1e-9, 0.0, 0.0)
    prm = {"dt": 1e-12, "seed": 1, "w_min": 1.0, "sigma_el_en": 1e-12}
    e, eo = _cells_population(g, 1, 1, [0, 0, 1e6], 1, 0)
    n, no = _cells_population(g, 2, 0, [0, 0, 0], 2, 10)
    assert EL.elastic_en(g, prm, e, eo, n, no, 0, collide.Counter(0))[2] == 0
    assert philox.PAIR not in (EL.PAIR_EN, EL.PAIR_NN, EL.PAIR_CX)
