"""Long runs of the small workload on the GPU against the oracle's, over eight seeds.

tests/golden/longrun_<variant>.json holds the oracle's 100-step runs of the small workload
(32x32x64 cells, 5e4 SPs, every process of the plain method, heat every 10 steps) for seeds
1..8, written by tests/golden/make_longrun.py: variant "small" as the workload is (a cold tip
that barely emits), variant "small_dense" with a 2000 K tip, a 12 GV/m apex field and w_min
0.1 (emission, impact and field ionization and the ions' space charge all act).  The CUDA path
runs the same seeds from the same initial bits (the oracle's V0 and its Laplace potential on
the fixed-point grid) in the plain form (full FP64 emission integral, FP64 V-cycles).  Variant
"small_all" adds every optional process to the dense one: elastic collisions and charge exchange,
Coulomb collisions, the Cu2+ channels, SP merging and the RC circuit.

* While both runs hold the same state, every integer of the step (counts, weights, events,
  removals, ids) is equal.  The runs would part when the potentials differ in a bit that reaches
  an integer decision: the oracle solves Poisson by CG to 1e-13, the library by multigrid to
  mg_tol, so the node field, a float32 rounding of potential differences, could differ by one
  ulp at some node, and a later position, cell or CIC fraction of an SP near it would follow.
  The test reports, for every seed, the steps before the first parting and requires at least 50
  of them (one with every optional process, whose FP32 Coulomb turn parts the positions within a
  few steps), with the emitted current within 1e-6 and the tip temperature within 2e-9 per heat
  step done over those steps.
* Over the seeds, at each quarter of the run, the mean over the 8 seeds of each inventory (SP
  count and weight per species), of each cumulative event count (emission, injection,
  ionizations, removals, ion impacts; with every optional process also the elastic, exchange,
  Coulomb and merge counts) and of each float (emitted current, tip temperature, gap voltage)
  lies within the oracle's seed-spread band: mean +- 4 sigma / sqrt(8), sigma the oracle's spread over the seeds
  (4 rather than 3 standard errors: some 70 comparisons per variant are made, and at 3 one of
  them would fall outside by chance in one run of six); the float quantities get a floor of
  1e-6 of their value.
"""
import json
import os

import numpy as np
import pytest

from oracle import field
from oracle.grid import Grid
from paper_2402_08404_gb300 import synth

from _util import SPECIES

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
VARIANTS = ("small", "small_dense", "small_all")
# Steps each seed must stay on the oracle's integer trajectory.  With every optional process the
# Coulomb turn runs in FP32 (within 4e-6 of the species' largest speed of the oracle's FP64 turn),
# so positions, and after them cells and decisions, part within a few steps; the seed bands carry
# the comparison from there.
EQUAL_FLOOR = {"small": 50, "small_dense": 50, "small_all": 1}
DIAG_INT = ("emitted", "evaporated", "sputtered", "impact_ionizations", "field_ionizations", "ion_impacts",
            "double_ionizations", "ion_ionizations", "elastic_en", "elastic_nn", "charge_exchanges", "coulomb_ee",
            "coulomb_ei", "coulomb_ii", "coulomb_ej", "coulomb_ij", "coulomb_jj", "merged", "next_id")
DIAG_FLOAT = ("emitted_current", "max_T", "V_gap")


@pytest.fixture(scope="module", params=VARIANTS)
def gold(request):
    path = os.path.join(GOLDEN, f"longrun_{request.param}.json")
    if not os.path.exists(path):
        pytest.skip(f"{os.path.basename(path)} not written (tests/golden/make_longrun.py --variant {request.param})")
    with open(path) as f:
        g = json.load(f)
    if g["steps"] < 100 or len(g["seeds"]) < 8:
        pytest.skip(f"{os.path.basename(path)} holds fewer than 100 steps of 8 seeds")
    return g


@pytest.fixture(scope="module")
def runs(gold):
    from paper_2402_08404_gb300 import _build
    if not os.path.exists(_build.LIB):
        _build.build()
    from paper_2402_08404_gb300 import pic
    out = {}
    for seed in sorted(gold["seeds"], key=int):
        out[seed] = run_gpu(pic, int(seed), gold["seeds"][seed]["V0"], gold["steps"], gold["n_heat"],
                            gold.get("overrides", {}))
    return out


def run_gpu(pic, seed, V0, steps, n_heat, overrides):
    cfg = dict(synth.CONFIGS["small"], n_heat=n_heat, seed=seed, **overrides)
    g = Grid(cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["tip_radius"], cfg["tip_height"])
    flags = pic.F_ALL & ~pic.F_SURROGATE & ~pic.F_MIXED_MG
    for key, flag in (("elastic", pic.F_ELASTIC), ("coulomb", pic.F_COULOMB), ("ion2", pic.F_ION2),
                      ("merge_max", pic.F_MERGE), ("circuit_R", pic.F_CIRCUIT)):
        if cfg.get(key):
            flags |= flag
    sim = pic.Pic(cfg, capacity=400_000, flags=flags, V0=V0, mg_tol=1e-12, mg_max_cycles=200)
    sim.set_potential(np.round(field.solve_poisson(g, V0) * 2.0 ** 40) / 2.0 ** 40)
    pop = synth.plasma(cfg, seed=seed)
    for s, (k, _, _) in enumerate(SPECIES):
        sim.load_particles(s, pop[k])
    sim.set_clock(0, cfg["n_sp"])
    rows = {k: [] for k in DIAG_INT + DIAG_FLOAT}
    for k in "enij":
        for q in ("count_", "weight_", "removed_"):
            rows[q + k] = []
    for _ in range(steps):
        sim.step(1)
        d = sim.diagnostics()
        for s, k in enumerate("enij"):
            rows["count_" + k].append(d["count"][s])
            rows["weight_" + k].append(d["weight"][s])
            rows["removed_" + k].append(d["removed"][s])
        for k in DIAG_INT + DIAG_FLOAT:
            rows[k].append(d[k])
    sim.close()
    return rows


def first_parting(gold_seed, run, keys):
    for t in range(len(run["next_id"])):
        if any(run[k][t] != gold_seed[k][t] for k in keys):
            return t + 1
    return None


def test_integers_equal_until_the_runs_part(gold, runs):
    keys = [k for k in gold["int_keys"]]
    n_heat = gold["n_heat"]
    parting, worst = {}, {}
    for seed in sorted(gold["seeds"], key=int):
        g, r = gold["seeds"][seed], runs[seed]
        part = first_parting(g, r, keys)
        upto = gold["steps"] if part is None else part - 1
        parting[seed] = upto
        if upto < gold["steps"]:
            print(f"variant {gold.get('variant', 'small')}, seed {seed} first parts at step {upto + 1}: " +
                  ", ".join(f"{k} {r[k][upto]} vs {g[k][upto]}" for k in keys if r[k][upto] != g[k][upto]))
        # while the states agree, the floats of the step: the emitted current within 1e-6 (the
        # single-step bar) and the tip temperature within 2e-9 per heat step done (each heat step
        # agrees to 1e-9 with the oracle's; the differences carry into the next)
        dj = max((abs(r["emitted_current"][t] - g["emitted_current"][t]) / max(abs(g["emitted_current"][t]), 1e-12)
                  for t in range(upto)), default=0.0)
        dt = max((abs(r["max_T"][t] - g["max_T"][t]) / g["max_T"][t] / (2e-9 * (1 + (t + 1) // n_heat))
                  for t in range(upto)), default=0.0)
        worst[seed] = (dj, dt)
    print(f"variant {gold.get('variant', 'small')}: steps with every integer equal, by seed: {parting}; "
          f"largest relative current difference and temperature difference over its bar, by seed: {worst}")
    floor = EQUAL_FLOOR[gold.get("variant", "small")]
    for seed, upto in parting.items():
        assert upto >= floor, (seed, upto)
        assert worst[seed][0] <= 1e-6 and worst[seed][1] <= 1.0, (seed, worst[seed])


@pytest.mark.parametrize("quarter", [1, 2, 3, 4])
def test_seed_means_within_the_oracle_band(gold, runs, quarter):
    seeds = sorted(gold["seeds"], key=int)
    n = len(seeds)
    assert n >= 8
    t = gold["steps"] * quarter // 4 - 1
    # SP counts and weights are states at the checkpoint; every other integer is a per-step count,
    # summed up to it
    ints = [k for k in gold["int_keys"] if k != "next_id"]
    state = {k for k in ints if k.startswith(("count_", "weight_"))}

    def value(src, k):
        if k in ints and k not in state:
            return float(np.sum(src[k][:t + 1]))
        return float(src[k][t])

    bad = []
    for k in ints + list(gold["float_keys"]):
        o = np.array([value(gold["seeds"][s], k) for s in seeds])
        g = np.array([value(runs[s], k) for s in seeds])
        # a floor for quantities the seeds hardly move (the tip temperature): the float parity bar
        # of a single step (1e-6 relative)
        band = 4.0 * o.std(ddof=1) / np.sqrt(n) + (1e-6 * abs(o.mean()) if k in gold["float_keys"] else 0.0)
        if abs(g.mean() - o.mean()) > band:
            bad.append((k, g.mean(), o.mean(), band))
    assert not bad, bad
