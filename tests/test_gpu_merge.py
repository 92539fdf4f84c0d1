"""Parity of SP merging (PIC_F_MERGE, Sec. 2.3.2) with the oracle, through the C ABI.  Merging is
FP64 arithmetic in a fixed order rounded once to float32 on both sides, so every field is compared
bit for bit; so are the merge count and the step's graph form against its eager form."""
import numpy as np
import pytest

from oracle import merge as M, particles as P
from paper_2402_08404_gb300 import synth

from _util import SPECIES, assert_sp_equal, colocated_population, grid_of, small_cfg, sorted_pop

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pic():
    import os
    from paper_2402_08404_gb300 import _build
    if not os.path.exists(_build.LIB):
        _build.build()
    from paper_2402_08404_gb300 import pic as m
    return m


@pytest.mark.parametrize("merge_max,w_max", [(2, 1024), (3, 9)])
def test_merge_stage_matches_oracle(pic, merge_max, w_max):
    cfg = small_cfg(n_sp=40000, w_min=1.0, merge_max=merge_max, w_max_units=w_max)
    g = grid_of(cfg)
    sim = pic.Pic(cfg, capacity=200_000, V0=60.0, flags=pic.F_MERGE)
    pop = colocated_population(cfg, 41)
    for s, (k, _, _) in enumerate(SPECIES):
        sim.load_particles(s, pop[k])
    st = sorted_pop(g, pop)
    done = 0
    for k in "eni":
        _, off = P.stable_sort(g, st[k])
        done += M.merge_species(st[k], off, merge_max, w_max)
    assert done > 1000
    sim.merge()
    assert sim.diagnostics()["merged"] == done
    for s, (k, _, _) in enumerate(SPECIES):
        assert_sp_equal(sim.get_particles(s), st[k])
    sim.close()


def _steps(pic, flags, calls, seed=43):
    cfg = small_cfg(n_sp=20000, n_heat=3, merge_max=1)
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


def test_steps_with_merging_graph_equals_eager(pic):
    base = (pic.F_ALL & ~pic.F_SURROGATE) | pic.F_MERGE
    calls = (1, 2)
    ref = _steps(pic, base, calls)
    got = _steps(pic, base | pic.F_GRAPH, calls)
    for s in range(3):
        for f in ("x", "y", "z", "vx", "vy", "vz", "w", "id"):
            assert np.array_equal(ref["sp"][s][f], got["sp"][s][f]), (s, f)
    assert np.array_equal(ref["phi"], got["phi"])
    for a, b in zip(ref["diag"], got["diag"]):
        assert a["merged"] == b["merged"] and a["count"] == b["count"]
    assert ref["diag"][-1]["merged"] > 0
