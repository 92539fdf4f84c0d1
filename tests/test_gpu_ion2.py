"""The Cu2+ channels on the GPU against the oracle (Table colls: Cu + e -> Cu2+ + 3e competing
with single ionization by the total cross section, Cu+ + e -> Cu2+ + 2e; Sec. 2.2: Coulomb
collisions between all charged species, here e-Cu2+, Cu+-Cu2+, Cu2+-Cu2+).

One full step of a collision-rich state holding all four species, with every process of the
method and the Cu2+ flag, against the oracle's step from the same bits: event counts, ids,
positions and weights of every species bit for bit, velocities within 1e-6 of the species'
largest speed (FP64 rotations and FP32 Coulomb turns), and the deposited charge, which now
carries Z = 2 for Cu2+, node for node.
"""
import numpy as np
import pytest

from oracle import field, step as OS
from oracle.grid import Grid

from _util import assert_sp_equal, colocated_population

pytestmark = pytest.mark.gpu

SPECIES4 = ("e", "n", "i", "j")
CFG = dict(nx=16, ny=16, nz=32, dx=1e-9, tip_radius=2e-9, tip_height=10e-9, apex_field=8e9, n_sp=6000, dt=5e-17,
           T0=2900.0, work_function=4.5, w_min=0.05, w_max_units=1024, n_heat=0, seed=5, merge_max=2,
           circuit_R=1e3, circuit_C=1e-12, sigma_el_en=5e-19, sigma_el_nn=5e-17, sigma_cx=5e-18, coulomb_log=10.0)


@pytest.fixture(scope="module")
def pic():
    import os
    from paper_2402_08404_gb300 import _build
    if not os.path.exists(_build.LIB):
        _build.build()
    from paper_2402_08404_gb300 import pic as m
    return m


def population(cfg, seed):
    """Colocated e-, Cu, Cu+ (electrons of 20-300 eV: above the double-ionization threshold for
    most) with the last third of the ions turned into Cu2+."""
    pop = colocated_population(cfg, seed)
    ni = len(pop["i"]["x"])
    cut = ni - ni // 3
    pop["j"] = {f: v[cut:].copy() for f, v in pop["i"].items()}
    pop["i"] = {f: v[:cut].copy() for f, v in pop["i"].items()}
    return pop


def make(pic, cfg, pop, phi, V0, extra=0):
    flags = ((pic.F_ALL & ~pic.F_SURROGATE & ~pic.F_HEAT) | pic.F_ELASTIC | pic.F_COULOMB | pic.F_MERGE |
             pic.F_CIRCUIT | pic.F_ION2 | extra)
    sim = pic.Pic(cfg, capacity=100_000, flags=flags, V0=V0, mg_tol=1e-11, mg_max_cycles=100)
    sim.set_potential(phi)
    for s, k in enumerate(SPECIES4):
        sim.load_particles(s, pop[k])
    sim.set_clock(0, cfg["n_sp"])
    return sim


def setup(cfg, seed=8):
    g = Grid(cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["tip_radius"], cfg["tip_height"])
    V0 = field.calibrate_V0(g, cfg["apex_field"])
    phi = np.round(field.solve_poisson(g, V0) * 2.0 ** 40) / 2.0 ** 40
    return g, V0, phi, population(cfg, seed)


@pytest.mark.parametrize("w_min", [2.0, 30.0])
def test_step_with_cu2_channels_matches_the_oracle(pic, w_min):
    cfg = dict(CFG, w_min=w_min)
    g, V0, phi, pop = setup(cfg)
    sim = make(pic, cfg, pop, phi, V0)
    prm = dict(cfg, V0=V0, next_id=cfg["n_sp"], elastic=True, coulomb=True, ion2=True)
    st = OS.State(g, prm, pop, phi)
    OS.step(st)
    sim.step(1)
    d = sim.diagnostics()
    keys = ("impact_ionizations", "double_ionizations", "ion_ionizations", "field_ionizations", "elastic_en",
            "elastic_nn", "charge_exchanges", "coulomb_ee", "coulomb_ei", "coulomb_ii", "coulomb_ej", "coulomb_ij",
            "coulomb_jj", "merged", "emitted", "evaporated", "ion_impacts")
    for k in keys:
        assert d[k] == st.count.get(k, 0), (k, d[k], st.count.get(k))
    assert d["double_ionizations"] > 0 and d["ion_ionizations"] > 0 and d["coulomb_jj"] > 0
    assert d["next_id"] == st.next_id
    for s, k in enumerate(SPECIES4):
        got = sim.get_particles(s)
        assert_sp_equal(got, st.sp[k], fields=("x", "y", "z", "w", "id"))
        vmax = max(np.abs(st.sp[k][c]).max() for c in ("vx", "vy", "vz")) if len(got["id"]) else 0.0
        for c in ("vx", "vy", "vz"):
            assert np.max(np.abs(got[c].astype(np.float64) - st.sp[k][c]), initial=0.0) <= 1e-6 * vmax + 1.0, (k, c)
        assert d["removed"][s] == st.count.get("removed_" + k, 0)
    assert d["count"][3] == len(st.sp["j"]["id"]) and d["weight"][3] == int(st.sp["j"]["w"].astype(np.int64).sum())
    # the charge of the step (Z = 2 for Cu2+), deposited by the push and moved by merging, equals the
    # oracle's deposit after the collisions, node by node
    assert np.array_equal(sim.get_charge().ravel(), st.Q.ravel().astype(np.int64))
    # the gap current (Z = 2 for Cu2+) within the float32 rounding of v . E0: 1e-6 of sum |q| |v| max|E0|
    e0max = float(np.abs(st.E0).max())
    scale = sum(abs(z) * float(np.sum(st.sp[k]["w"] * (np.abs(st.sp[k]["vx"]) + np.abs(st.sp[k]["vy"]) +
                                                      np.abs(st.sp[k]["vz"])).astype(np.float64)))
                for k, z in (("e", -1), ("i", 1), ("j", 2))) * cfg["w_min"] * 1.602176634e-19 * e0max
    assert abs(d["I_gap"] - st.I_gap) <= 1e-6 * scale, (d["I_gap"], st.I_gap, scale)
    sim.close()


def test_graph_form_with_cu2_equals_the_eager_form(pic):
    cfg = dict(CFG, w_min=2.0)
    g, V0, phi, pop = setup(cfg, seed=9)
    a = make(pic, cfg, pop, phi, V0)
    b = make(pic, cfg, pop, phi, V0, extra=pic.F_GRAPH)
    a.step(3)
    b.step(3)      # one eager step, then the recorded graph
    da, db = a.diagnostics(), b.diagnostics()
    for k in ("next_id", "count", "weight", "double_ionizations", "ion_ionizations", "coulomb_jj", "V_gap"):
        assert da[k] == db[k], k
    for s in range(4):
        assert_sp_equal(a.get_particles(s), b.get_particles(s))
    assert np.array_equal(a.get_charge(), b.get_charge())
    a.close()
    b.close()


def test_resume_with_cu2_repeats_the_uninterrupted_run(pic, tmp_path):
    # the checkpoint holds the fourth species: n steps, save, m steps against a fresh handle loaded
    # from the file and stepped m, bit for bit
    cfg = dict(CFG, w_min=2.0)
    g, V0, phi, pop = setup(cfg, seed=11)
    ref = make(pic, cfg, pop, phi, V0)
    ref.step(2)
    path = str(tmp_path / "ion2.pic")
    ref.save(path)
    ref.step(2)
    want = [ref.get_particles(s) for s in range(4)]
    dref = ref.diagnostics()
    qref = ref.get_charge()
    ref.close()
    sim = make(pic, cfg, population(cfg, seed=12), phi, V0)   # another state, replaced by the load
    sim.load(path)
    sim.step(2)
    d = sim.diagnostics()
    for s in range(4):
        assert_sp_equal(sim.get_particles(s), want[s])
    assert np.array_equal(sim.get_charge(), qref)
    for k in ("step", "next_id", "count", "weight", "double_ionizations", "ion_ionizations", "coulomb_ej",
              "coulomb_ij", "coulomb_jj", "V_gap"):
        assert d[k] == dref[k], k
    assert dref["count"][3] > 0
    sim.close()
