"""Checkpoint/resume (pic_save / pic_load) and the error paths of the step.

Resume: n steps, save, load into a freshly created handle, m steps must equal n + m
uninterrupted steps bit for bit, in the eager and the graph form, with every optional process
on (the random draws are keyed by id and step, so nothing depends on the process history).

Errors: PIC_E_NOCONV when the Poisson solve cannot reach mg_tol within mg_max_cycles (eager and
graph form), PIC_E_CAPACITY when a stage would create more SPs than a species holds (the stage
adds none, ids stay unique), PIC_E_INVALID for a state file of another geometry, and a
checkpoint taken before a refused step restores the state of that moment.
"""
import os

import numpy as np
import pytest

from paper_2402_08404_gb300 import synth

from _util import SPECIES, small_cfg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pic():
    from paper_2402_08404_gb300 import _build
    if not os.path.exists(_build.LIB):
        _build.build()
    from paper_2402_08404_gb300 import pic as m
    return m


def cfg_all():
    # every optional process: circuit, elastic, Coulomb, merging, extrapolation, heat every 2 steps
    return small_cfg(n_sp=20000, n_heat=2, circuit_R=1e3, circuit_C=1e-12, merge_max=8)


def flags_all(pic):
    return ((pic.F_ALL & ~pic.F_SURROGATE) | pic.F_CIRCUIT | pic.F_ELASTIC | pic.F_COULOMB | pic.F_MERGE |
            pic.F_EXTRAPOLATE | pic.F_FAST_INTEGRAL)


def fresh(pic, cfg, flags, cap=200_000, **kw):
    return pic.Pic(cfg, capacity=cap, flags=flags, mg_tol=1e-10, **kw)


def seeded(pic, cfg, flags, seed=13, **kw):
    sim = fresh(pic, cfg, flags, **kw)
    pop = synth.plasma(cfg, seed=seed)
    for s, (k, _, _) in enumerate(SPECIES):
        sim.load_particles(s, pop[k])
    sim.set_clock(0, cfg["n_sp"])
    sim.solve_field()
    return sim


def state(sim):
    d = sim.diagnostics()
    return {"sp": [sim.get_particles(s) for s in range(3)], "phi": sim.get_potential(), "E": sim.get_efield(),
            "Q": sim.get_charge(), "T": sim.get_temperature(), "acc": sim.face_accumulators(),
            "em": sim.face_emission(), "diag": d}


DIAG_KEYS = ("step", "next_id", "count", "weight", "emitted", "evaporated", "sputtered", "impact_ionizations",
             "field_ionizations", "removed", "ion_impacts", "total_charge_fixed", "mg_cycles", "V0", "V_gap",
             "I_gap", "I_tot", "elastic_en", "elastic_nn", "charge_exchanges", "coulomb_ee", "coulomb_ei",
             "coulomb_ii", "merged", "max_T")


def assert_same(a, b):
    for s in range(3):
        for f in ("x", "y", "z", "vx", "vy", "vz", "w", "id"):
            assert np.array_equal(a["sp"][s][f], b["sp"][s][f]), (s, f)
    for k in ("phi", "E", "Q", "T"):
        assert np.array_equal(a[k], b[k]), k
    for k in a["acc"]:
        assert np.array_equal(a["acc"][k], b["acc"][k]), k
    for x, y in zip(a["em"], b["em"]):
        assert np.array_equal(x, y)
    for k in DIAG_KEYS:
        assert a["diag"][k] == b["diag"][k], (k, a["diag"][k], b["diag"][k])


@pytest.mark.parametrize("graph", [False, True])
def test_resume_repeats_the_uninterrupted_run(pic, tmp_path, graph):
    cfg = cfg_all()
    flags = flags_all(pic) | (pic.F_GRAPH if graph else 0)
    n, m = 3, 4
    ref = seeded(pic, cfg, flags)
    ref.step(n)
    path = str(tmp_path / "state.pic")
    ref.save(path)
    ref.step(m)
    want = state(ref)
    ref.close()
    # a fresh handle (its own seeded-free creation state), loaded, stepped m
    sim = fresh(pic, cfg, flags_all(pic))
    sim.load(path)
    sim.step(m)
    got = state(sim)
    sim.close()
    assert got["diag"]["step"] == n + m
    assert_same(want, got)


def test_resume_with_a_trained_surrogate(pic, tmp_path):
    """The surrogate's weights and validity map travel with the state: the production form
    (surrogate emission) resumes bit for bit."""
    cfg = small_cfg(n_sp=10000)
    flags = pic.F_PRODUCTION
    ref = seeded(pic, cfg, flags)
    ref.surrogate_train(nsamples=65536, epochs=4, batch=4096, lr=3e-3, seed=2)
    ref.step(2)
    path = str(tmp_path / "sur.pic")
    ref.save(path)
    ref.step(3)
    want = state(ref)
    ref.close()
    sim = fresh(pic, cfg, flags)
    sim.load(path)
    sim.step(3)
    got = state(sim)
    sim.close()
    assert_same(want, got)
    assert got["diag"]["surrogate_faces"] == want["diag"]["surrogate_faces"]


def test_load_refuses_another_geometry_and_short_capacity(pic, tmp_path):
    cfg = small_cfg(n_sp=8000)
    flags = pic.F_ALL & ~pic.F_SURROGATE
    sim = seeded(pic, cfg, flags)
    sim.step(1)
    path = str(tmp_path / "a.pic")
    sim.save(path)
    counts = sim.diagnostics()["count"]
    sim.close()
    other = fresh(pic, dict(cfg, tip_radius=4e-9), flags)
    with pytest.raises(pic.PicError) as e:
        other.load(path)
    assert e.value.code == pic.PIC_E_INVALID and "geometry" in str(e.value)
    other.close()
    short = fresh(pic, cfg, flags, cap=(counts[0] - 1, 200_000, 200_000))
    with pytest.raises(pic.PicError) as e:
        short.load(path)
    assert e.value.code == pic.PIC_E_CAPACITY
    short.close()
    with open(path, "r+b") as f:
        f.write(b"NOTSTATE")
    sim = fresh(pic, cfg, flags)
    with pytest.raises(pic.PicError) as e:
        sim.load(path)
    assert e.value.code == pic.PIC_E_INVALID
    sim.close()


def test_save_refuses_pushed_unsorted_state(pic, tmp_path):
    cfg = small_cfg(n_sp=4000)
    sim = seeded(pic, cfg, pic.F_ALL & ~pic.F_SURROGATE)
    sim.push()
    with pytest.raises(pic.PicError) as e:
        sim.save(str(tmp_path / "x.pic"))
    assert e.value.code == pic.PIC_E_INVALID
    sim.sort()
    sim.save(str(tmp_path / "x.pic"))
    sim.close()


@pytest.mark.parametrize("graph", [False, True])
def test_poisson_cycle_cap_gives_noconv(pic, graph):
    """mg_tol far below the FP64 floor with a cap of 3 refinement cycles: the step ends with
    PIC_E_NOCONV (in the graph form through the device-side loop's error bit); with the
    controls restored the same handle steps on."""
    cfg = small_cfg(n_sp=4000)
    flags = (pic.F_ALL & ~pic.F_SURROGATE) | (pic.F_GRAPH if graph else 0)
    sim = seeded(pic, cfg, flags)
    sim.step(2)                    # graph form: records and replays the graphs first
    sim.set_solver(1e-30, 3)
    with pytest.raises(pic.PicError) as e:
        sim.step(2)
    assert e.value.code == pic.PIC_E_NOCONV
    assert sim.diagnostics()["mg_cycles"] <= 3
    sim.set_solver(1e-10, 60)
    sim.step(1)
    sim.close()


def test_capacity_refusal_adds_no_sp_and_checkpoint_restores(pic, tmp_path):
    """The ion capacity a handful above the loaded count: ionizations overflow it, the step
    returns PIC_E_CAPACITY, the ion products of the refused pass are not added (the count stays
    within capacity, ids stay unique) and a state saved before the step restores that moment."""
    cfg = small_cfg(n_sp=20000, w_min=1.0)       # collision-rich: thousands of ionizations per step
    pop = synth.plasma(cfg, seed=13)
    ni = len(pop["i"]["x"])
    flags = pic.F_ALL & ~pic.F_SURROGATE & ~pic.F_HEAT
    sim = fresh(pic, cfg, flags, cap=(200_000, 200_000, ni + 2))
    for s, (k, _, _) in enumerate(SPECIES):
        sim.load_particles(s, pop[k])
    sim.set_clock(0, cfg["n_sp"])
    sim.solve_field()
    path = str(tmp_path / "before.pic")
    sim.save(path)
    before = state(sim)
    code = None
    for _ in range(5):
        try:
            sim.step(1)
        except pic.PicError as e:
            code = e.code
            break
    assert code == pic.PIC_E_CAPACITY
    d = sim.diagnostics()
    assert d["count"][2] <= ni + 2
    ids = np.concatenate([sim.get_particles(s)["id"] for s in range(3)])
    assert len(np.unique(ids)) == len(ids)
    assert ids.max() < d["next_id"]
    sim.load(path)
    assert_same(before, state(sim))
    sim.close()


def test_load_all_equals_species_by_species_and_stops_at_a_bad_species(pic):
    # pic_load_all (copies of the next species beside the current one's check and sort) leaves the
    # state of the pic_load_particles sequence; a species that fails its check leaves the species
    # before it loaded and itself and the rest unchanged
    import torch
    cfg = small_cfg(n_sp=20000)
    flags = pic.F_ALL & ~pic.F_SURROGATE
    a = fresh(pic, cfg, flags)
    b = fresh(pic, cfg, flags)
    pop = synth.plasma(cfg, seed=21)
    pinned = []
    for k, _, _ in SPECIES:      # pinned host copies, as a caller streaming states in would hold them
        d = {}
        for f, v in pop[k].items():
            t = torch.empty(len(v), dtype={np.float32: torch.float32, np.int32: torch.int32,
                                           np.uint64: torch.int64}[v.dtype.type], pin_memory=True)
            arr = t.numpy().view(v.dtype)
            arr[:] = v
            d[f] = arr
        pinned.append(d)
    for s, (k, _, _) in enumerate(SPECIES):
        a.load_particles(s, pop[k])
    b.load_all(pinned)
    for s in range(3):
        ga, gb = a.get_particles(s), b.get_particles(s)
        for f in ga:
            assert np.array_equal(ga[f], gb[f]), (s, f)
    # a second state whose Cu species holds an SP outside the domain
    pop2 = synth.plasma(cfg, seed=22)
    pop2["n"]["x"][17] = np.float32(cfg["nx"] + 3)
    with pytest.raises(pic.PicError):
        b.load_all([pop2[k] for k, _, _ in SPECIES])
    e_new = b.get_particles(0)
    a.load_particles(0, pop2["e"])
    e_ref = a.get_particles(0)
    for f in e_ref:
        assert np.array_equal(e_new[f], e_ref[f]), f          # species 0 was loaded
    for s in (1, 2):
        g = b.get_particles(s)
        ref = a.get_particles(s)                                # a still holds the first state there
        for f in ref:
            assert np.array_equal(g[f], ref[f]), (s, f)         # species 1, 2 unchanged
    b.step(1)                                                   # the handle stays usable
    a.close()
    b.close()


def test_dense_cell_sorts_stably_and_the_cell_limit_gives_capacity(pic):
    # 20000 electrons in one cell (a long segment: one block's bitonic sort in shared memory) sort
    # into the oracle's stable order; 40000 in one cell exceed the sort's 32768 and give
    # PIC_E_CAPACITY (the segment is left unsorted, nothing is written out of place)
    from oracle import particles as P
    from _util import grid_of
    cfg = small_cfg(n_sp=20000)
    g = grid_of(cfg)
    flags = pic.F_ALL & ~pic.F_SURROGATE
    rng = np.random.default_rng(4)

    def electrons(n_dense, n_rest):
        x = np.concatenate([np.full(n_dense, 3.5, np.float32) + rng.random(n_dense).astype(np.float32) * np.float32(0.4),
                            (rng.random(n_rest) * 8).astype(np.float32)])
        y = np.concatenate([np.full(n_dense, 4.25, np.float32), (rng.random(n_rest) * 8).astype(np.float32)])
        z = np.concatenate([np.full(n_dense, 50.5, np.float32), (50 + rng.random(n_rest) * 10).astype(np.float32)])
        perm = rng.permutation(n_dense + n_rest)      # the dense cell's SPs interleaved with the rest
        n = n_dense + n_rest
        return {"x": x[perm], "y": y[perm], "z": z[perm], "vx": np.zeros(n, np.float32), "vy": np.zeros(n, np.float32),
                "vz": np.zeros(n, np.float32), "w": np.ones(n, np.int32), "id": np.arange(n, dtype=np.uint64)}

    sim = fresh(pic, cfg, flags, cap=100_000)
    e = electrons(20000, 5000)
    sim.load_particles(0, e)
    got = sim.get_particles(0)
    want, off = P.stable_sort(g, {f: np.asarray(v) for f, v in e.items()})
    assert int(np.diff(off).max()) >= 20000
    for f in ("x", "y", "z", "id"):
        assert np.array_equal(got[f], want[f]), f
    with pytest.raises(pic.PicError):
        sim.load_particles(0, electrons(40000, 100))
    sim.close()
