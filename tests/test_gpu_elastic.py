"""Parity of the elastic e-Cu and Cu-Cu collisions and the Cu+-Cu charge exchange
(PIC_F_ELASTIC) with the oracle, through the C ABI.

Bars: the collision decisions and the splitting are integer work (event counts, weights, new
SPs, ids and slots, bit for bit); the new velocities are FP64 rotations stored in float32,
within 1e-6 of the oracle's per component (plus 1 m/s).  The cross sections are raised far above
the stand-in defaults so that a small instance has hundreds of events in every pass.
"""
import numpy as np
import pytest

from oracle import collide, elastic as EL, field, particles as P
from oracle import constants as OC
from paper_2402_08404_gb300 import synth

from _util import SPECIES, assert_sp_equal, colocated_population, fixed_phi, grid_of, small_cfg, sorted_pop

pytestmark = pytest.mark.gpu

SIGMAS = dict(sigma_el_en=2e-19, sigma_el_nn=2e-15, sigma_cx=1e-16)


@pytest.fixture(scope="module")
def pic():
    import os
    from paper_2402_08404_gb300 import _build
    if not os.path.exists(_build.LIB):
        _build.build()
    from paper_2402_08404_gb300 import pic as m
    return m


def _setup(pic, flags, V0=60.0, seed=12):
    cfg = small_cfg(n_sp=30000, w_min=1.0, **SIGMAS)
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
    prm = {"dt": cfg["dt"], "seed": cfg["seed"], "w_min": cfg["w_min"], **SIGMAS}
    return cfg, g, sim, st, offs, prm, field.efield(g, phi)


def _velocities_close(got, ref, k):
    for c in ("vx", "vy", "vz"):
        a, b = got[c].astype(np.float64), ref[c].astype(np.float64)
        bad = np.nonzero(~(np.abs(a - b) <= 1e-6 * (np.abs(b) + 1.0)))[0]
        assert len(bad) == 0, (k, c, bad[:5], a[bad[:5]], b[bad[:5]])


def _oracle_passes(g, prm, st, offs, ids):
    """The three passes on the sorted state st (modified in place); the new SPs per species."""
    el_e, n1, ev_en = EL.elastic_en(g, prm, st["e"], offs["e"], st["n"], offs["n"], 3, ids)
    n2, ev_nn = EL.elastic_nn(g, prm, st["n"], offs["n"], 3, ids)
    el_i, n3, ev_cx = EL.charge_exchange(g, prm, st["i"], offs["i"], st["n"], offs["n"], 3, ids)
    return el_e, P.concat(P.concat(n1, n2), n3), el_i, (ev_en, ev_nn, ev_cx)


def test_elastic_passes_match_oracle(pic):
    cfg, g, sim, st, offs, prm, E = _setup(pic, pic.F_ELASTIC)
    before = {k: {c: st[k][c].copy() for c in ("vx", "vy", "vz")} for k in "eni"}
    nsort = {k: len(st[k]["x"]) for k in "eni"}
    ids = collide.Counter(cfg["n_sp"])
    el_e, el_n, el_i, evs = _oracle_passes(g, prm, st, offs, ids)
    assert min(evs) > 100, evs
    assert min(len(el_e["w"]), len(el_n["w"]), len(el_i["w"])) > 20   # the splitting is exercised
    ref = {"e": P.concat(st["e"], el_e), "n": P.concat(st["n"], el_n), "i": P.concat(st["i"], el_i)}
    sim.collide()
    d = sim.diagnostics()
    assert (d["elastic_en"], d["elastic_nn"], d["charge_exchanges"]) == evs
    assert d["impact_ionizations"] == 0 and d["field_ionizations"] == 0
    assert d["next_id"] == ids.next_id
    for s_, (k, _, _) in enumerate(SPECIES):
        got = sim.get_particles(s_)
        assert_sp_equal(got, ref[k], fields=("x", "y", "z", "w", "id"))
        _velocities_close(got, ref[k], k)
        if k in "ei":   # which sorted SPs turned whole: bit-exact decisions
            m = nsort[k]
            moved_ref = np.any([ref[k][c][:m] != before[k][c] for c in ("vx", "vy", "vz")], axis=0)
            moved_got = np.any([got[c][:m] != before[k][c] for c in ("vx", "vy", "vz")], axis=0)
            assert np.array_equal(moved_got, moved_ref), k
    sim.close()


def test_collide_stage_with_elastic_matches_oracle(pic):
    """Impact ionization, then the three passes, then field ionization: the oracle step's order
    and its order of the new SPs."""
    flags = pic.F_IMPACT_ION | pic.F_DFI | pic.F_ELASTIC
    cfg, g, sim, st, offs, prm, E = _setup(pic, flags, V0=420.0, seed=13)
    ids = collide.Counter(cfg["n_sp"])
    ni, ne, ev = collide.impact_ionization(g, prm, st["e"], offs["e"], st["n"], offs["n"], 3, ids)
    el_e, el_n, el_i, evs = _oracle_passes(g, prm, st, offs, ids)
    st["n"] = P.concat(st["n"], el_n)
    ni2, ne2, ev2 = collide.field_ionization(g, prm, st["n"], E, 3, ids)
    ref = {"e": P.concat(P.concat(P.concat(st["e"], ne), el_e), ne2), "n": st["n"],
           "i": P.concat(P.concat(P.concat(st["i"], ni), el_i), ni2)}
    sim.collide()
    d = sim.diagnostics()
    assert ev > 20 and ev2 > 20 and min(evs) > 20, (ev, ev2, evs)
    assert (d["impact_ionizations"], d["field_ionizations"]) == (ev, ev2)
    assert (d["elastic_en"], d["elastic_nn"], d["charge_exchanges"]) == evs
    assert d["next_id"] == ids.next_id
    for s_, (k, _, _) in enumerate(SPECIES):
        got = sim.get_particles(s_)
        assert_sp_equal(got, ref[k], fields=("x", "y", "z", "w", "id"))
        _velocities_close(got, ref[k], k)
    sim.close()
