"""Write tests/golden/longrun_<variant>.json: the oracle's long runs of the small workload.

The small workload (32x32x64 cells, dx = 1 nm, tip r = 3 nm h = 20 nm, 8 GV/m apex field,
5e4 seeded SPs, dt = 0.05 fs) is stepped 100 times by the oracle (oracle/step.py, every
process of the plain method, heat every 10 steps) for seeds 1..8 (the seed keys both the
seeded population and the Philox streams).  Variant "small" is that workload as it is (a cold
tip that barely emits); variant "small_dense" heats the tip to 2000 K, raises the apex field to
12 GV/m and w_min to 0.1 (ten times the real particles per SP), so that emission, impact and
field ionization and the space charge of the ions act during the run; variant "small_all" adds
every optional process (elastic collisions, Coulomb collisions, the Cu2+ channels, merging, the
RC circuit).  Per step it records the integer diagnostics and the
emitted current and tip temperature, which tests/test_gpu_longrun.py compares with the CUDA
path: bit for bit while the two runs share their state, statistically over the seeds after.

The initial potential is the Laplace solution for V0 calibrated by the oracle, rounded to the
library's fixed-point grid (steps of 2^-40 V), so that both sides start from the same bits; the
test recomputes it with the oracle.  Calls only oracle/ and the seeded input generator.

  python tests/golden/make_longrun.py [--variant small|small_dense|small_all] [--steps 100] [--seeds 1-8] [--workers 8]
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

# one thread per worker process: the seeds run in parallel, and numpy's BLAS pool in every
# worker would oversubscribe the cores
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
N_HEAT = 10
DENSE = {"T0": 2000.0, "apex_field": 12e9, "w_min": 0.1}
# "small_all": the dense variant with every optional process: elastic collisions and charge
# exchange, Coulomb collisions, the Cu2+ channels, SP merging above 16 SPs of a species per
# cell, and the RC circuit (1 kOhm, 1 pF)
ALL = dict(DENSE, elastic=True, coulomb=True, ion2=True, merge_max=16, circuit_R=1e3, circuit_C=1e-12,
           coulomb_log=10.0)
VARIANTS = {"small": {}, "small_dense": DENSE, "small_all": ALL}
INT_KEYS = ("count_e", "count_n", "count_i", "weight_e", "weight_n", "weight_i", "emitted", "evaporated",
            "sputtered", "impact_ionizations", "field_ionizations", "removed_e", "removed_n", "removed_i",
            "ion_impacts", "next_id")
FLOAT_KEYS = ("emitted_current", "max_T")
# recorded for the variant with every optional process
ALL_INT_KEYS = ("count_j", "weight_j", "removed_j", "double_ionizations", "ion_ionizations", "elastic_en",
                "elastic_nn", "charge_exchanges", "coulomb_ee", "coulomb_ei", "coulomb_ii", "coulomb_ej", "coulomb_ij",
                "coulomb_jj", "merged")
ALL_FLOAT_KEYS = ("V_gap",)


def keys_of(variant):
    """(integer keys, float keys) recorded for a variant."""
    if variant == "small_all":
        return INT_KEYS + ALL_INT_KEYS, FLOAT_KEYS + ALL_FLOAT_KEYS
    return INT_KEYS, FLOAT_KEYS


def workload(variant="small"):
    from paper_2402_08404_gb300 import synth
    return dict(synth.CONFIGS["small"], n_heat=N_HEAT, **VARIANTS[variant])


def initial_state(seed, variant="small"):
    """(grid, oracle state, V0) of the seeded small workload for one seed."""
    from oracle import field, step as S
    from oracle.grid import Grid
    from paper_2402_08404_gb300 import synth
    cfg = dict(workload(variant), seed=seed)
    g = Grid(cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["tip_radius"], cfg["tip_height"])
    V0 = field.calibrate_V0(g, cfg["apex_field"])
    phi = np.round(field.solve_poisson(g, V0) * 2.0 ** 40) / 2.0 ** 40
    prm = dict(cfg, V0=V0, next_id=cfg["n_sp"])
    st = S.State(g, prm, synth.plasma(cfg, seed=seed), phi)
    return g, st, V0


def record(st):
    r = {}
    for k in "enij":
        r["count_" + k] = int(len(st.sp[k]["x"]))
        r["weight_" + k] = int(st.sp[k]["w"].astype(np.int64).sum())
    for k in ("emitted", "evaporated", "sputtered", "impact_ionizations", "field_ionizations", "removed_e",
              "removed_n", "removed_i", "removed_j", "ion_impacts", "double_ionizations", "ion_ionizations",
              "elastic_en", "elastic_nn", "charge_exchanges", "coulomb_ee", "coulomb_ei", "coulomb_ii", "coulomb_ej",
              "coulomb_ij", "coulomb_jj", "merged"):
        r[k] = int(st.count.get(k, 0))
    r["next_id"] = int(st.next_id)
    r["emitted_current"] = float(np.sum(st.last_J) * st.grid.dx ** 2)
    r["max_T"] = float(np.max(st.T))
    r["V_gap"] = float(st.V_gap)
    return r


def run_seed(args):
    seed, steps, variant = args
    from oracle import step as S
    g, st, V0 = initial_state(seed, variant)
    rows = []
    t0 = time.time()
    for _ in range(steps):
        S.step(st)
        rows.append(record(st))
    return seed, V0, rows, time.time() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--variant", default="small", choices=sorted(VARIANTS))
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--seeds", default="1-8")
    ap.add_argument("--workers", type=int, default=8)
    a = ap.parse_args()
    lo, hi = (int(v) for v in a.seeds.split("-"))
    seeds = list(range(lo, hi + 1))
    with mp.get_context("spawn").Pool(min(a.workers, len(seeds))) as pool:
        res = pool.map(run_seed, [(s, a.steps, a.variant) for s in seeds])
    cfg = workload(a.variant)
    out = {"workload": f"{a.variant}: 32x32x64 cells, dx 1 nm, tip r 3 nm h 20 nm, T0 {cfg['T0']:g} K, "
                       f"apex {cfg['apex_field'] * 1e-9:g} GV/m, w_min {cfg['w_min']:g}, 5e4 SPs, dt 0.05 fs, "
                       f"heat every {N_HEAT} steps; every process of the plain method",
           "variant": a.variant, "overrides": VARIANTS[a.variant],
           "generator": "tests/golden/make_longrun.py (oracle/step.py only)",
           "steps": a.steps, "n_heat": N_HEAT, "int_keys": list(keys_of(a.variant)[0]),
           "float_keys": list(keys_of(a.variant)[1]),
           "seeds": {}}
    for seed, V0, rows, sec in sorted(res):
        ik, fk = keys_of(a.variant)
        out["seeds"][str(seed)] = {"V0": V0, "seconds": round(sec, 1), **{k: [r[k] for r in rows] for k in ik + fk}}
    path = os.path.join(HERE, f"longrun_{a.variant}.json")
    with open(path, "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print("wrote", path, {s: out["seeds"][s]["seconds"] for s in out["seeds"]})


if __name__ == "__main__":
    main()
