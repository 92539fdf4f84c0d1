"""Parity of the Coulomb collisions (PIC_F_COULOMB: e-e, e-Cu+, Cu+-Cu+) with the oracle, through
the C ABI.

Bars: the pairs and the weight-rule decisions are integer work (event counts per pass, weights,
ids, positions bit for bit).  The turn itself runs in FP32 on the GPU against the oracle's FP64:
delta carries a few FP32 roundings (1e-6 of its size at most, the Box-Muller cosine by cospif),
so the velocity change k du is off by ~1e-6 of the relative speed, below 2e-6 of the largest
speed of the pair; the test allows 4e-6 of the largest speed of the species (plus 1 m/s) per
component.  A wrong weight-rule decision moves a velocity by k du, far outside that bar.
"""
import numpy as np
import pytest

from oracle import collide, coulomb as CO, elastic as EL, field, particles as P
from paper_2402_08404_gb300 import synth

from _util import SPECIES, assert_sp_equal, colocated_population, fixed_phi, grid_of, small_cfg, sorted_pop

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pic():
    import os
    from paper_2402_08404_gb300 import _build
    if not os.path.exists(_build.LIB):
        _build.build()
    from paper_2402_08404_gb300 import pic as m
    return m


def _setup(pic, flags, seed, V0=60.0, **kw):
    cfg = small_cfg(n_sp=30000, w_min=1.0, **kw)
    g = grid_of(cfg)
    sim = pic.Pic(cfg, capacity=200_000, V0=V0, flags=flags)
    pop = colocated_population(cfg, seed)
    phi = fixed_phi(field.solve_poisson(g, V0))
    sim.set_potential(phi)
    for s, (k, _, _) in enumerate(SPECIES):
        sim.load_particles(s, pop[k])
    sim.set_clock(3, cfg["n_sp"])
    st = sorted_pop(g, pop)
    offs = {k: P.stable_sort(g, st[k])[1] for k in "eni"}
    prm = {"dt": cfg["dt"], "seed": cfg["seed"], "w_min": cfg["w_min"], **kw}
    return cfg, g, sim, st, offs, prm


def _close(got, ref, before, k):
    S = max(float(np.max(np.abs(np.stack([ref[c] for c in ("vx", "vy", "vz")])))),
            float(np.max(np.abs(np.stack([before[c] for c in ("vx", "vy", "vz")])))))
    for c in ("vx", "vy", "vz"):
        a, b = got[c].astype(np.float64), ref[c].astype(np.float64)
        bad = np.nonzero(~(np.abs(a - b) <= 4e-6 * S + 1.0))[0]
        assert len(bad) == 0, (k, c, bad[:5], a[bad[:5]], b[bad[:5]], S)


def test_coulomb_passes_match_oracle(pic):
    cfg, g, sim, st, offs, prm = _setup(pic, pic.F_COULOMB, seed=31)
    before = {k: {c: st[k][c].copy() for c in ("vx", "vy", "vz")} for k in "eni"}
    ev = (CO.coulomb_ee(g, prm, st["e"], offs["e"], 3),
          CO.coulomb_ei(g, prm, st["e"], offs["e"], st["i"], offs["i"], 3),
          CO.coulomb_ii(g, prm, st["i"], offs["i"], 3))
    assert min(ev) > 500, ev
    sim.collide()
    d = sim.diagnostics()
    assert (d["coulomb_ee"], d["coulomb_ei"], d["coulomb_ii"]) == ev
    for s, (k, _, _) in enumerate(SPECIES):
        got = sim.get_particles(s)
        assert_sp_equal(got, st[k], fields=("x", "y", "z", "w", "id"))
        _close(got, st[k], before[k], k)
    # the turn is not negligible: electrons moved by much more than the bar
    assert np.max(np.abs(st["e"]["vx"].astype(np.float64) - before["e"]["vx"])) > 1e3
    sim.close()


def test_collide_stage_with_all_processes_matches_oracle(pic):
    """Impact ionization, the elastic passes, the Coulomb passes and field ionization, in the
    oracle step's order."""
    sig = dict(sigma_el_en=2e-19, sigma_el_nn=2e-15, sigma_cx=1e-16, coulomb_log=8.0)
    flags = pic.F_IMPACT_ION | pic.F_DFI | pic.F_ELASTIC | pic.F_COULOMB
    cfg, g, sim, st, offs, prm = _setup(pic, flags, seed=32, V0=420.0, **sig)
    before = {k: {c: st[k][c].copy() for c in ("vx", "vy", "vz")} for k in "eni"}
    E = field.efield(g, fixed_phi(field.solve_poisson(g, 420.0)))
    ids = collide.Counter(cfg["n_sp"])
    ni, ne, ev = collide.impact_ionization(g, prm, st["e"], offs["e"], st["n"], offs["n"], 3, ids)
    el_e, n1, _ = EL.elastic_en(g, prm, st["e"], offs["e"], st["n"], offs["n"], 3, ids)
    n2, _ = EL.elastic_nn(g, prm, st["n"], offs["n"], 3, ids)
    el_i, n3, _ = EL.charge_exchange(g, prm, st["i"], offs["i"], st["n"], offs["n"], 3, ids)
    st["n"] = P.concat(P.concat(P.concat(st["n"], n1), n2), n3)
    co = (CO.coulomb_ee(g, prm, st["e"], offs["e"], 3), CO.coulomb_ei(g, prm, st["e"], offs["e"], st["i"], offs["i"], 3),
          CO.coulomb_ii(g, prm, st["i"], offs["i"], 3))
    ni2, ne2, ev2 = collide.field_ionization(g, prm, st["n"], E, 3, ids)
    ref = {"e": P.concat(P.concat(P.concat(st["e"], ne), el_e), ne2), "n": st["n"],
           "i": P.concat(P.concat(P.concat(st["i"], ni), el_i), ni2)}
    sim.collide()
    d = sim.diagnostics()
    assert ev > 20 and ev2 > 20 and min(co) > 500
    assert (d["impact_ionizations"], d["field_ionizations"]) == (ev, ev2)
    assert (d["coulomb_ee"], d["coulomb_ei"], d["coulomb_ii"]) == co
    assert d["next_id"] == ids.next_id
    for s, (k, _, _) in enumerate(SPECIES):
        got = sim.get_particles(s)
        assert_sp_equal(got, ref[k], fields=("x", "y", "z", "w", "id"))
        _close(got, ref[k], before[k], k)
    sim.close()


def _steps(pic, flags, calls, seed=33):
    cfg = small_cfg(n_sp=20000, n_heat=3)
    pop = synth.plasma(cfg, seed=seed)
    sim = pic.Pic(cfg, capacity=200_000, flags=flags, mg_tol=1e-10)
    for s, (k, _, _) in enumerate(SPECIES):
        sim.load_particles(s, pop[k])
    sim.set_clock(0, cfg["n_sp"])
    sim.solve_field()
    diags = []
    for n in calls:
        sim.step(n)
        diags.append(sim.diagnostics())
    out = {"sp": [sim.get_particles(s) for s in range(3)], "phi": sim.get_potential(), "diag": diags}
    sim.close()
    return out


def test_steps_with_every_collision_graph_equals_eager(pic):
    base = (pic.F_ALL & ~pic.F_SURROGATE) | pic.F_ELASTIC | pic.F_COULOMB
    calls = (1, 2, 1)
    ref = _steps(pic, base, calls)
    got = _steps(pic, base | pic.F_GRAPH, calls)
    for s in range(3):
        for f in ("x", "y", "z", "vx", "vy", "vz", "w", "id"):
            assert np.array_equal(ref["sp"][s][f], got["sp"][s][f]), (s, f)
    assert np.array_equal(ref["phi"], got["phi"])
    for a, b in zip(ref["diag"], got["diag"]):
        for k in ("coulomb_ee", "coulomb_ei", "coulomb_ii", "elastic_en", "elastic_nn", "charge_exchanges", "count",
                  "next_id"):
            assert a[k] == b[k], k
    assert ref["diag"][-1]["coulomb_ee"] > 0
