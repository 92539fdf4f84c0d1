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


def test_production_size_collisions_sampled_against_the_oracle(pic):
    """Impact and field ionization at the production size, with w_min raised to 1e-3 so that both
    produce events (the bench's collision-rich form), checked cell by cell against the oracle:
    every cell whose SPs the GPU changed (at most 4000 of them) and 300 random cells holding both
    e- and Cu.  The oracle's MCC and DFI on those cells' SPs alone (pairing, draws and field
    depend on the cell, its SPs and the node field only) must give the same weights (bit for
    bit), velocities (within 1e-6 of the species' largest speed) and new SPs (positions and
    weights bit for bit; ids are numbered over the whole grid and are checked for uniqueness)."""
    from oracle import collide
    cfg = dict(synth.CONFIGS["production"], w_min=1e-3)
    n = cfg["n_sp"]
    pop = synth.plasma(cfg, seed=cfg["seed"])
    cap = (int(0.4 * n * 1.5), int(0.4 * n * 1.25), int(0.2 * n * 2.0))
    flags = (pic.F_ALL & ~pic.F_SURROGATE) | pic.F_FAST_INTEGRAL
    sim = pic.Pic(cfg, capacity=cap, flags=flags, mg_tol=1e-6, mg_max_cycles=60)
    for s, (k, _, _) in enumerate(SPECIES):
        sim.load_particles(s, pop[k])
    sim.set_clock(0, n)
    sim.solve_field()
    g = grid_of(cfg)
    E = field.efield(g, sim.get_potential())
    before = [sim.get_particles(s) for s in range(3)]
    sim.collide()
    d = sim.diagnostics()
    after = [sim.get_particles(s) for s in range(3)]
    assert d["impact_ionizations"] > 100 and d["field_ionizations"] > 1000, d
    ids = np.concatenate([a["id"] for a in after])
    assert len(np.unique(ids)) == len(ids)

    keys = [P.cell_keys(g, b) for b in before]
    ne, nn, ni = (len(b["x"]) for b in before)
    changed = set()
    for s, m in ((0, ne), (1, nn)):
        moved = (after[s]["w"][:m] != before[s]["w"]) | (after[s]["vx"][:m] != before[s]["vx"])
        changed.update(np.unique(keys[s][moved]).tolist())
    rng = np.random.default_rng(5)
    changed = sorted(changed)
    if len(changed) > 4000:
        changed = sorted(rng.choice(changed, size=4000, replace=False).tolist())
    both = np.intersect1d(np.unique(keys[0]), np.unique(keys[1]))
    cells = np.union1d(changed, rng.choice(both, size=300, replace=False))
    sel = [np.isin(keys[s], cells) for s in range(2)]
    assert sel[0].sum() > 100 and sel[1].sum() > 1000

    # the oracle on the selected cells alone (cell order is kept, so the sub-arrays are sorted)
    e_sub, e_off = P.stable_sort(g, P.take(before[0], np.nonzero(sel[0])[0]))
    n_sub, n_off = P.stable_sort(g, P.take(before[1], np.nonzero(sel[1])[0]))
    prm = dict(cfg)
    ids_o = collide.Counter(1 << 40)
    ni_o, ne_o, ev = collide.impact_ionization(g, prm, e_sub, e_off, n_sub, n_off, 0, ids_o)
    ni2_o, ne2_o, ev2 = collide.field_ionization(g, prm, n_sub, E, 0, ids_o)
    assert ev > 0 and ev2 > 0

    for s, sub in ((0, e_sub), (1, n_sub)):
        idx = np.nonzero(sel[s])[0]
        got = {f: after[s][f][idx] for f in P.FIELDS}
        assert np.array_equal(got["id"], sub["id"])
        assert np.array_equal(got["w"], sub["w"]), s
        vmax = max(float(np.abs(sub[c]).max()) for c in ("vx", "vy", "vz"))
        for c in ("vx", "vy", "vz"):
            assert np.max(np.abs(got[c].astype(np.float64) - sub[c])) <= 1e-6 * vmax, (s, c)

    def products(new, s):
        k = P.cell_keys(g, new)
        m = np.isin(k, cells)
        rows = np.stack([k[m].astype(np.float64), new["x"][m], new["y"][m], new["z"][m], new["w"][m]], 1)
        return rows[np.lexsort(rows.T[::-1])]

    new_i = {f: after[2][f][ni:] for f in P.FIELDS}
    new_e = {f: after[0][f][ne:] for f in P.FIELDS}
    want_i = P.concat(ni_o, ni2_o)
    want_e = P.concat(ne_o, ne2_o)
    assert np.array_equal(products(new_i, 2), products(want_i, 2))
    assert np.array_equal(products(new_e, 0), products(want_e, 0))
    sim.close()


def test_production_size_cu2_channels_sampled_against_the_oracle(pic):
    """The Cu2+ channels at the production size (w_min 1e-3, electrons of the seeded state):
    impact ionization with the double channel and the ionization of Cu+, cell by cell against the
    oracle as above (every cell the GPU changed, up to 3000, and 300 random cells holding
    electrons and Cu or Cu+): weights bit for bit, velocities within 1e-6 of the largest speed,
    new Cu+, Cu2+ and electrons by position and weight."""
    from oracle import collide
    cfg = dict(synth.CONFIGS["production"], w_min=1e-3)
    n = cfg["n_sp"]
    pop = synth.plasma(cfg, seed=cfg["seed"])
    cap = (int(0.4 * n * 1.5), int(0.4 * n * 1.25), int(0.2 * n * 2.0), int(0.2 * n))
    flags = pic.F_IMPACT_ION | pic.F_ION2
    sim = pic.Pic(cfg, capacity=cap, flags=flags, mg_tol=1e-6, mg_max_cycles=60)
    for s, (k, _, _) in enumerate(SPECIES):
        sim.load_particles(s, pop[k])
    sim.set_clock(0, n)
    g = grid_of(cfg)
    before = [sim.get_particles(s) for s in range(3)]
    sim.collide()
    d = sim.diagnostics()
    after = [sim.get_particles(s) for s in range(4)]
    assert d["impact_ionizations"] > 100 and d["double_ionizations"] > 0 and d["ion_ionizations"] > 0, d
    ids = np.concatenate([a["id"] for a in after])
    assert len(np.unique(ids)) == len(ids)
    keys = [P.cell_keys(g, b) for b in before]
    ne, nn, ni = (len(b["x"]) for b in before)
    changed = set()
    for s, m in ((0, ne), (1, nn), (2, ni)):
        moved = (after[s]["w"][:m] != before[s]["w"]) | (after[s]["vx"][:m] != before[s]["vx"])
        changed.update(np.unique(keys[s][moved]).tolist())
    rng = np.random.default_rng(6)
    changed = sorted(changed)
    if len(changed) > 3000:
        changed = sorted(rng.choice(changed, size=3000, replace=False).tolist())
    both = np.union1d(np.intersect1d(np.unique(keys[0]), np.unique(keys[1])),
                      np.intersect1d(np.unique(keys[0]), np.unique(keys[2])))
    cells = np.union1d(changed, rng.choice(both, size=300, replace=False))
    sel = [np.isin(keys[s], cells) for s in range(3)]
    subs = [P.stable_sort(g, P.take(before[s], np.nonzero(sel[s])[0])) for s in range(3)]
    (e_sub, e_off), (n_sub, n_off), (i_sub, i_off) = subs
    ids_o = collide.Counter(1 << 40)
    ni_o, ne_o, ev, nj_o, ne2_o, ev2 = collide.impact_ionization(g, dict(cfg), e_sub, e_off, n_sub, n_off, 0, ids_o,
                                                                   double=True)
    nj3_o, ne3_o, ev3 = collide.ion_ionization(g, dict(cfg), e_sub, e_off, i_sub, i_off, 0, ids_o)
    assert ev > 0 and ev3 > 0
    for s, sub in ((0, e_sub), (1, n_sub), (2, i_sub)):
        idx = np.nonzero(sel[s])[0]
        got = {f: after[s][f][idx] for f in P.FIELDS}
        assert np.array_equal(got["id"], sub["id"]) and np.array_equal(got["w"], sub["w"]), s
        vmax = max(float(np.abs(sub[c]).max()) for c in ("vx", "vy", "vz"))
        for c in ("vx", "vy", "vz"):
            assert np.max(np.abs(got[c].astype(np.float64) - sub[c])) <= 1e-6 * vmax, (s, c)

    def products(new):
        k = P.cell_keys(g, new)
        m = np.isin(k, cells)
        rows = np.stack([k[m].astype(np.float64), new["x"][m], new["y"][m], new["z"][m], new["w"][m]], 1)
        return rows[np.lexsort(rows.T[::-1])]

    for s, start, want in ((2, ni, ni_o), (3, 0, P.concat(nj_o, nj3_o)), (0, ne, P.concat(P.concat(ne_o, ne2_o), ne3_o))):
        new = {f: after[s][f][start:] for f in P.FIELDS}
        assert np.array_equal(products(new), products(want)), s
    sim.close()
