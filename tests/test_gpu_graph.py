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


def _ensemble_cfgs():
    return [small_cfg(n_sp=12000, apex_field=8e9, seed=1),
            small_cfg(nx=16, ny=16, nz=32, tip_radius=2e-9, tip_height=10e-9, n_sp=4000, apex_field=6e9, seed=2),
            small_cfg(nx=24, ny=24, nz=48, tip_radius=3e-9, tip_height=14e-9, n_sp=8000, apex_field=11e9, seed=3,
                      n_heat=2)]


def _build(pic, cfgs, flags, stream=None):
    sims = []
    for cfg in cfgs:
        sim = pic.Pic(cfg, capacity=100_000, flags=flags, mg_tol=1e-10, stream=stream)
        pop = synth.plasma(cfg, seed=cfg["seed"])
        for s, (k, _, _) in enumerate(SPECIES):
            sim.load_particles(s, pop[k])
        sim.set_clock(0, cfg["n_sp"])
        sim.solve_field()
        sims.append(sim)
    return sims


def _state(sim):
    return {"sp": [sim.get_particles(s) for s in range(3)], "phi": sim.get_potential(), "Q": sim.get_charge(),
            "T": sim.get_temperature(), "d": sim.diagnostics()}


def _assert_same(a, b):
    for s in range(3):
        for f in ("x", "y", "z", "vx", "vy", "vz", "w", "id"):
            assert np.array_equal(a["sp"][s][f], b["sp"][s][f]), (s, f)
    assert np.array_equal(a["phi"], b["phi"])
    assert np.array_equal(a["Q"], b["Q"])
    assert np.array_equal(a["T"], b["T"])
    for k in ("step", "next_id", "count", "weight", "removed", "impact_ionizations", "field_ionizations", "mg_cycles"):
        assert a["d"][k] == b["d"][k], k


def test_batch_equals_instances_stepped_alone(pic):
    """Three instances of different grids, fields and heat cadences: one graph launch per step
    for all of them gives each the results of stepping it alone."""
    import torch
    flags = pic.F_ALL & ~pic.F_SURROGATE
    cfgs = _ensemble_cfgs()
    ref = _build(pic, cfgs, flags)
    for sim in ref:
        sim.step(1)
        sim.step(4)
    want = [_state(sim) for sim in ref]
    for sim in ref:
        sim.close()
    st = torch.cuda.Stream()
    sims = _build(pic, cfgs, flags, stream=st)
    batch = pic.Batch(sims)
    batch.step(1)      # eager step of every instance, then the graphs are recorded
    batch.step(4)
    assert batch.ms() > 0
    for sim, w in zip(sims, want):
        _assert_same(_state(sim), w)
    batch.close()
    for sim in sims:
        sim.close()


def test_batch_rejects_mixed_streams(pic):
    import torch
    flags = pic.F_ALL & ~pic.F_SURROGATE
    cfgs = _ensemble_cfgs()[:2]
    a = _build(pic, cfgs[:1], flags, stream=torch.cuda.Stream())[0]
    b = _build(pic, cfgs[1:], flags, stream=torch.cuda.Stream())[0]
    with pytest.raises(pic.PicError):
        pic.Batch([a, b])
    with pytest.raises(pic.PicError):
        pic.Batch([a, a])
    a.close()
    b.close()


def test_autotune_keeps_results(pic):
    flags = pic.F_ALL & ~pic.F_SURROGATE
    cfg = small_cfg(n_sp=16000)
    a, b = _build(pic, [cfg, cfg], flags)
    ch = a.autotune()
    assert ch["particle_blocks_per_sm"] in (2, 4, 8, 16, 32)
    assert ch["residual_planes_per_thread"] in (1, 2, 4)
    assert len(ch["smoother_planes_per_thread"]) >= 1
    assert all(k in (1, 2, 4, 8) for k in ch["smoother_planes_per_thread"])
    for sim in (a, b):
        sim.step(3)
    _assert_same(_state(a), _state(b))
    a.close()
    b.close()
