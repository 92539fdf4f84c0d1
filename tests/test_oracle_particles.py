"""Pins of the oracle's particle kernels (Sec. 2.2): gather, leapfrog, boundaries, sort, deposit."""
import math

import numpy as np
import pytest

from oracle import constants as C
from oracle import field, particles as P
from oracle.grid import Grid


def _sp(pos, vel=None, w=None):
    pos = np.atleast_2d(np.asarray(pos, dtype=np.float32))
    n = len(pos)
    vel = np.zeros((n, 3), np.float32) if vel is None else np.atleast_2d(np.asarray(vel, np.float32))
    w = np.ones(n, np.int32) if w is None else np.asarray(w, np.int32)
    return {"x": pos[:, 0].copy(), "y": pos[:, 1].copy(), "z": pos[:, 2].copy(),
            "vx": vel[:, 0].copy(), "vy": vel[:, 1].copy(), "vz": vel[:, 2].copy(),
            "w": w, "id": np.arange(n, dtype=np.uint64)}


def test_gather_is_exact_on_trilinear_fields():
    rng = np.random.default_rng(3)
    nx, ny, nz = 5, 4, 6
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    E = np.zeros((nz + 1, ny + 1, nx + 1, 3), np.float32)
    E[..., 0] = 2.0 * i + 0.5                 # exactly representable linear fields
    E[..., 1] = -3.0 * j + 1.0
    E[..., 2] = 0.25 * k * i                  # bilinear
    pos = rng.random((200, 3)) * np.array([nx, ny, nz])
    q = (np.floor(pos * 1024) / 1024).astype(np.float32)     # dyadic positions: every lerp exact
    e = P.gather(E, q[:, 0], q[:, 1], q[:, 2])
    x, y, z = q[:, 0].astype(float), q[:, 1].astype(float), q[:, 2].astype(float)
    assert np.array_equal(e[:, 0], (2.0 * x + 0.5).astype(np.float32))
    assert np.array_equal(e[:, 1], (-3.0 * y + 1.0).astype(np.float32))
    assert np.allclose(e[:, 2], 0.25 * z * x, rtol=1e-6)


def test_leapfrog_reproduces_uniform_field_trajectory():
    # constant E: the leapfrog positions equal x0 + v0 t + a t^2/2 at t = n dt when the stored
    # velocity is v(-dt/2) (closed form of uniformly accelerated motion)
    g = Grid(4, 4, 400, 1e-9, 0.0, 0.0)
    Ez = -2.0e7                                # V/m
    E = np.zeros((g.nz + 1, g.ny + 1, g.nx + 1, 3), np.float32)
    E[..., 2] = Ez
    E64 = E.astype(np.float64)
    dt = 5e-17
    a = -C.E_CHARGE / C.M_E * Ez
    v0 = 1.0e5
    sp_ = _sp([[2.0, 2.0, 10.0]], [[0.0, 0.0, v0 - 0.5 * a * dt]])
    sp64 = {k: v.astype(np.float64) if v.dtype == np.float32 else v.copy() for k, v in sp_.items()}
    sp64["vz"] = np.array([v0 - 0.5 * a * dt])
    qmdt = P.kick_factor(-1, C.M_E, dt)
    x64 = None
    for n in range(1, 201):
        x, y, z, vx, vy, vz = P.push_f32(sp_, E, qmdt, np.float32(dt / g.dx))
        sp_.update(x=x, y=y, z=z, vx=vx, vy=vy, vz=vz)
        x64 = P.push_f64(sp64, E64, -C.E_CHARGE / C.M_E * dt, dt / g.dx)
        sp64 = dict(sp64)
        for c, v in zip(("x", "y", "z", "vx", "vy", "vz"), x64):
            sp64[c] = np.asarray(v, dtype=np.float64)
        t = n * dt
        exact = 10.0 + (v0 * t + 0.5 * a * t * t) / g.dx
        assert sp64["z"][0] == pytest.approx(exact, rel=1e-12, abs=1e-9)
        assert float(z[0]) == pytest.approx(exact, rel=1e-5)
    # energy gain equals e E dz (work-energy) for the f64 trajectory
    dz = (sp64["z"][0] - 10.0) * g.dx
    assert 0.5 * C.M_E * ((v0 + a * 200 * dt) ** 2 - v0 ** 2) == pytest.approx(C.E_CHARGE * -Ez * dz, rel=1e-9)


def test_lone_charge_feels_no_self_force():
    g = Grid(8, 8, 8, 1e-9, 0.0, 0.0)
    sp_ = _sp([[4.0, 4.0, 4.0]], w=[5])
    Q = P.deposit(g, sp_, 1)
    phi = field.solve_poisson(g, 0.0, field.rhs_from_charge(g, Q, 1.0))
    E = field.efield(g, phi)
    e = P.gather(E, sp_["x"], sp_["y"], sp_["z"])
    scale = np.abs(E).max()
    assert np.all(np.abs(e) <= 1e-9 * scale)


def _brute_first_event(g, p0, p1, samples=20000):
    ts = (np.arange(1, samples + 1) / samples)
    pts = p0[None, :] + ts[:, None] * (p1 - p0)[None, :]
    c = np.floor(pts).astype(int)
    prev = np.floor(p0).astype(int)
    for q in range(samples):
        cc = c[q]
        if np.array_equal(cc, prev):
            continue
        out = (cc[0] < 0 or cc[0] >= g.nx or cc[1] < 0 or cc[1] >= g.ny or cc[2] < 0 or cc[2] >= g.nz)
        if out:
            if cc[2] < 0:
                return P.EV_CATHODE, g.cell_index(*prev)
            if cc[2] >= g.nz:
                return P.EV_ANODE, g.cell_index(*prev)
            return P.EV_LATERAL, g.cell_index(*prev)
        if g.solid[cc[2], cc[1], cc[0]]:
            return P.EV_SOLID, g.cell_index(*prev)
        prev = cc
    return P.EV_NONE, -1


def test_dda_matches_brute_force_traversal():
    g = Grid(8, 8, 10, 1e-9, 2.2e-9, 6e-9)
    rng = np.random.default_rng(7)
    checked = 0
    while checked < 300:
        p0 = rng.random(3) * np.array([8, 8, 10])
        c0 = np.floor(p0).astype(int)
        if g.solid[c0[2], c0[1], c0[0]]:
            continue
        p1 = p0 + rng.normal(0, 1.5, 3)
        # skip near-degenerate segments (two crossings closer than the sampling step)
        d = p1 - p0
        ts = []
        for a in range(3):
            lo, hi = sorted((p0[a], p1[a]))
            for b in range(int(np.floor(lo)) + 1, int(np.floor(hi)) + 1):
                ts.append((b - p0[a]) / d[a])
        ts = np.sort(ts)
        if len(ts) > 1 and np.min(np.diff(ts)) < 5e-4:
            continue
        ev, vcell, _ = P.first_event(g, p0, p1)
        bev, bcell = _brute_first_event(g, p0, p1)
        assert ev == bev
        if ev != P.EV_NONE:
            assert vcell == bcell
        checked += 1


def test_ion_impact_records_face_and_energy():
    g = Grid(8, 8, 10, 1e-9, 2.2e-9, 6e-9)
    # an ion just above the apex moving straight down into the tip
    top = max(k for k in range(g.nz) if g.solid[k, 3, 3])
    sp_ = _sp([[3.5, 3.5, top + 1.2]], [[0.0, 0.0, -1.0e7]], w=[4])
    new = P.push_f32(sp_, np.zeros((g.nz + 1, g.ny + 1, g.nx + 1, 3), np.float32), 0.0,
                     np.float32(5e-17 / 1e-9))
    alive, imp = P.boundary(g, sp_, new, True, C.M_CU)
    assert not alive[0] and len(imp) == 1
    f, energy, w = imp[0]
    assert g.face_dir[f] == 4 and g.face_owner[f] == g.cell_index(3, 3, top)
    assert energy == pytest.approx(0.5 * C.M_CU * 1e14 / C.E_CHARGE, rel=1e-6) and w == 4


def test_stable_sort_against_brute_force():
    g = Grid(6, 5, 7, 1e-9, 0.0, 0.0)
    rng = np.random.default_rng(11)
    n = 500
    pos = rng.random((n, 3)) * np.array([6, 5, 7])
    pos[::7] = pos[3]                      # many equal cells
    sp_ = _sp(pos)
    alive = rng.random(n) > 0.2
    out, off = P.stable_sort(g, sp_, alive)
    keys = P.cell_keys(g, sp_)
    brute = sorted([p for p in range(n) if alive[p]], key=lambda p: (keys[p], p))
    assert np.array_equal(out["id"], np.array(brute, dtype=np.uint64))
    assert off[-1] == alive.sum()
    for c in range(g.ncell):
        assert off[c + 1] - off[c] == sum(1 for p in brute if keys[p] == c)


def test_deposit_conserves_charge_and_ignores_order():
    g = Grid(6, 5, 7, 1e-9, 0.0, 0.0)
    rng = np.random.default_rng(5)
    n = 2000
    pos = rng.random((n, 3)) * np.array([6, 5, 7])
    w = rng.integers(1, 9, n)
    sp_ = _sp(pos, w=w)
    Q = P.deposit(g, sp_, -1)
    assert Q.sum() == -(int(w.sum()) << 30)
    perm = rng.permutation(n)
    Q2 = P.deposit(g, P.take(sp_, perm), -1)
    assert np.array_equal(Q, Q2)
    # a particle on a node gives everything to that node; at a cell centre, 8 equal shares
    Qn = P.deposit(g, _sp([[2.0, 3.0, 4.0]], w=[3]), 1)
    assert Qn[4, 3, 2] == 3 << 30 and np.count_nonzero(Qn) == 1
    Qc = P.deposit(g, _sp([[2.5, 3.5, 4.5]], w=[1]), 1)
    assert np.count_nonzero(Qc) == 8 and np.all(Qc[Qc != 0] == 1 << 27)
