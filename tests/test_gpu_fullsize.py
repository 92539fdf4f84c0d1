"""Parity at the production size (256x256x512 cells, 33.9M nodes, 2e7 SPs), in the launch
configuration bench.py times.  The oracle cannot step the whole instance, so it checks sampled
outputs one by one (pushes of sampled SPs, emission of sampled faces) and whole-array definitions
that are cheap in numpy (node field, face field, the discrete Poisson residual), and the rest by
properties that hold at any size (sorted keys, weight and charge conservation, unique ids).
"""
import numpy as np
import pytest

from oracle import emission as em, field, particles as P
from oracle import constants as OC
from paper_2402_08404_gb300 import synth

from _util import SPECIES, grid_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pic():
    import os
    from paper_2402_08404_gb300 import _build
    if not os.path.exists(_build.LIB):
        _build.build()
    from paper_2402_08404_gb300 import pic as m
    return m


def _weights(sim):
    return [int(sim.get_particles(s)["w"].astype(np.int64).sum()) for s in range(3)]


def test_production_size_step_stages(pic):
    cfg = dict(synth.CONFIGS["production"])
    n = cfg["n_sp"]
    pop = synth.plasma(cfg, seed=cfg["seed"])
    cap = (int(0.4 * n * 1.25), int(0.4 * n * 1.25), int(0.2 * n * 1.5))
    flags = (pic.F_ALL & ~pic.F_SURROGATE) | pic.F_FAST_INTEGRAL
    sim = pic.Pic(cfg, capacity=cap, flags=flags, mg_tol=1e-6, mg_max_cycles=60)
    for s, (k, _, _) in enumerate(SPECIES):
        sim.load_particles(s, pop[k])
    sim.set_clock(0, n)
    sim.solve_field()
    g = grid_of(cfg)
    rng = np.random.default_rng(17)

    # node field: the oracle's definition over the whole grid, bit for bit
    phi = sim.get_potential()
    E = field.efield(g, phi)
    assert np.array_equal(sim.get_efield(), E)

    # push: sampled SPs of every species against the oracle's float32 leapfrog, bit for bit
    before = [sim.get_particles(s) for s in range(3)]
    sim.push()
    after = [sim.get_particles(s) for s in range(3)]
    dtdx = np.float32(cfg["dt"] / cfg["dx"])
    for s, (k, Z, m) in enumerate(SPECIES):
        idx = np.sort(rng.choice(len(before[s]["x"]), size=3000, replace=False))
        samp = P.take(before[s], idx)
        new = P.push_f32(samp, E, P.kick_factor(Z, m, cfg["dt"]) if Z else 0.0, dtdx)
        for c, v in zip(("x", "y", "z", "vx", "vy", "vz"), new):
            assert np.array_equal(after[s][c][idx], v.astype(np.float32)), (k, c)
        assert np.array_equal(after[s]["id"], before[s]["id"])
    n_pushed = [len(a["x"]) for a in after]
    w_before = [int(a["w"].astype(np.int64).sum()) for a in before]
    del before, after

    # sort: cell keys ascending, every SP kept or counted as removed
    sim.sort()
    d = sim.diagnostics()
    for s in range(3):
        sp_ = sim.get_particles(s)
        keys = P.cell_keys(g, sp_)
        assert np.all(np.diff(keys) >= 0)
        assert len(sp_["x"]) + d["removed"][s] == n_pushed[s]
        assert not np.any(g.solid.ravel()[keys])

    # collisions: an ionization moves k units of weight from Cu to Cu+ and adds k to e-
    w0 = _weights(sim)
    sim.collide()
    w1 = _weights(sim)
    assert w1[1] + w1[2] == w0[1] + w0[2]
    assert w1[0] - w0[0] == w1[2] - w0[2]
    ids = np.concatenate([sim.get_particles(s)["id"] for s in range(3)])
    assert len(np.unique(ids)) == len(ids)

    # deposit: the fixed-point charge sums to the SP charge exactly
    sim.deposit()
    Q = sim.get_charge()
    assert int(Q.sum()) == (w1[2] - w1[0]) << 30

    # solve: the discrete Poisson residual by the oracle's definition, and the node field again
    sim.solve_field()
    d = sim.diagnostics()
    phi = sim.get_potential()
    f = field.rhs_from_charge(g, Q, cfg["w_min"])
    rel = field.relative_residual(g, phi, f, d["V0"])
    assert d["mg_residual"] <= 1e-6 and rel <= 2e-6, (d["mg_residual"], rel)
    E = field.efield(g, phi)
    assert np.array_equal(sim.get_efield(), E)

    # emission: the face field by definition over all faces; J and P_N of sampled faces against
    # the oracle's FP64 integral within the FP32-Gamow bar (1e-4 relative where J > 1e-5 A/m^2)
    sim.emit()
    Fg, J, PN = sim.face_emission()
    Fv = field.face_field(g, phi)
    assert np.array_equal(Fg, Fv)
    hot = np.nonzero(Fv > 3e9)[0]
    pick = rng.choice(hot, size=min(40, len(hot)), replace=False)
    R = np.where(g.face_owner[pick] >= 0, cfg["tip_radius"] * 1e9, np.inf)
    Jr, Pr = em.current_density_fixed(Fv[pick] * 1e-9, np.full(len(pick), cfg["T0"]), cfg["work_function"], R)
    rel_ = Jr > 1e-5
    assert rel_.sum() >= 10
    assert np.max(np.abs(J[pick][rel_] / Jr[rel_] - 1)) <= 1e-4
    assert np.max(np.abs(PN[pick][rel_] - Pr[rel_]) / (np.abs(Pr[rel_]) + 0.05 * Jr[rel_])) <= 1e-4
    sim.close()


def test_production_size_optional_processes(pic):
    """The optional processes at the production size, by properties that hold at any size:
    merging keeps every species' weight and momentum (float32 rounding) and merges in the dense
    cells; the collide stage with elastic and Coulomb passes moves weight only from Cu to Cu+
    (and adds as much to e-), keeps ids unique, and turns pairs in every Coulomb pass."""
    cfg = dict(synth.CONFIGS["production"], merge_max=8)
    n = cfg["n_sp"]
    pop = synth.plasma(cfg, seed=cfg["seed"])
    cap = (int(0.4 * n * 1.25), int(0.4 * n * 1.25), int(0.2 * n * 1.5))
    flags = (pic.F_ALL & ~pic.F_SURROGATE) | pic.F_FAST_INTEGRAL | pic.F_ELASTIC | pic.F_COULOMB | pic.F_MERGE
    sim = pic.Pic(cfg, capacity=cap, flags=flags, mg_tol=1e-6, mg_max_cycles=60)
    for s, (k, _, _) in enumerate(SPECIES):
        sim.load_particles(s, pop[k])
    sim.set_clock(0, n)
    sim.solve_field()

    def moments(s):
        sp_ = sim.get_particles(s)
        w = sp_["w"].astype(np.int64)
        p = [float((w * sp_[c].astype(np.float64)).sum()) for c in ("vx", "vy", "vz")]
        a = [float((w * np.abs(sp_[c].astype(np.float64))).sum()) for c in ("vx", "vy", "vz")]
        return int(w.sum()), p, a

    before = [moments(s) for s in range(3)]
    sim.merge()
    d = sim.diagnostics()
    assert d["merged"] > 0
    for s in range(3):
        w1, p1, _ = moments(s)
        w0, p0, a0 = before[s]
        assert w1 == w0
        for c in range(3):
            assert abs(p1[c] - p0[c]) <= 1e-5 * a0[c] + 1e-30, (s, c)

    w0 = _weights(sim)
    sim.collide()
    d = sim.diagnostics()
    w1 = _weights(sim)
    assert w1[1] + w1[2] == w0[1] + w0[2]
    assert w1[0] - w0[0] == w1[2] - w0[2]
    ids = np.concatenate([sim.get_particles(s)["id"] for s in range(3)])
    assert len(np.unique(ids)) == len(ids)
    assert d["coulomb_ee"] > 0 and d["coulomb_ei"] > 0 and d["coulomb_ii"] > 0
    sim.close()
