"""The graph form of the step (PIC_F_GRAPH: one CUDA graph per step, the Poisson refinement loop
a device-side while node) must give the eager form's results bit for bit: the same kernels run
in the same order on the same data, and the convergence test compares the same FP64 norms.
"""
import numpy as np
import pytest

from paper_2402_08404_gb300 import synth

from _util import SPECIES, small_cfg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pic():
    import os
    from paper_2402_08404_gb300 import _build
    if not os.path.exists(_build.LIB):
        _build.build()
    from paper_2402_08404_gb300 import pic as m
    return m


def _run(pic, cfg, pop, flags, steps, calls):
    sim = pic.Pic(cfg, capacity=200_000, flags=flags, mg_tol=1e-10)
    for s, (k, _, _) in enumerate(SPECIES):
        sim.load_particles(s, pop[k])
    sim.set_clock(0, cfg["n_sp"])
    sim.solve_field()
    diags = []
    for n in calls:
        sim.step(n)
        diags.append(sim.diagnostics())
    out = {"sp": [sim.get_particles(s) for s in range(3)], "phi": sim.get_potential(),
           "E": sim.get_efield(), "Q": sim.get_charge(), "acc": sim.face_accumulators(), "diag": diags}
    sim.close()
    return out


@pytest.mark.parametrize("mixed", [True, False])
def test_graph_step_equals_eager_step(pic, mixed):
    cfg = small_cfg(n_sp=20000, n_heat=3)
    pop = synth.plasma(cfg, seed=21)
    base = pic.F_ALL & ~pic.F_SURROGATE
    if not mixed:
        base &= ~pic.F_MIXED_MG
    calls = (1, 3, 2)          # first call: one eager step records the graph; then replays
    ref = _run(pic, cfg, pop, base, 6, calls)
    got = _run(pic, cfg, pop, base | pic.F_GRAPH, 6, calls)
    for s in range(3):
        for f in ("x", "y", "z", "vx", "vy", "vz", "w", "id"):
            assert np.array_equal(ref["sp"][s][f], got["sp"][s][f]), (s, f)
    assert np.array_equal(ref["phi"], got["phi"])
    assert np.array_equal(ref["E"], got["E"])
    assert np.array_equal(ref["Q"], got["Q"])
    for k in ref["acc"]:
        assert np.array_equal(ref["acc"][k], got["acc"][k]), k
    for a, b in zip(ref["diag"], got["diag"]):
        for k in ("step", "next_id", "count", "weight", "emitted", "impact_ionizations", "field_ionizations",
                  "removed", "total_charge_fixed", "mg_cycles"):
            assert a[k] == b[k], k
        assert abs(a["mg_residual"] - b["mg_residual"]) <= 1e-6 * max(a["mg_residual"], 1e-30)
    assert got["diag"][-1]["step"] == 6


def test_graph_rebuilds_after_flag_change_and_reload(pic):
    cfg = small_cfg(n_sp=8000)
    pop = synth.plasma(cfg, seed=5)
    flags = (pic.F_ALL & ~pic.F_SURROGATE) | pic.F_GRAPH
    sim = pic.Pic(cfg, capacity=100_000, flags=flags, mg_tol=1e-10)
    for s, (k, _, _) in enumerate(SPECIES):
        sim.load_particles(s, pop[k])
    sim.set_clock(0, cfg["n_sp"])
    sim.solve_field()
    sim.step(3)
    # reloading one species changes its buffer parity alone: the recorded graphs no longer fit
    sim.load_particles(1, pop["n"])
    sim.step(2)
    sim.set_flags(flags & ~pic.F_DFI)
    sim.step(2)
    d = sim.diagnostics()
    assert d["step"] == 7 and d["field_ionizations"] == 0
    sim.close()
