#!/usr/bin/env python
"""Benchmark of the vacuum-arc PIC-MCC step on GB300 (one JSON line on stdout, rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config production]

A step is one pass of the whole path: emission + injection, gather/push/boundary, cell sort,
impact + field ionization, deposit, multigrid Poisson solve + node field (+ heat every n_heat
steps).  The workload is the seeded production instance (256x256x512 cells, dx = 0.5 nm, tip
r = 5 nm h = 60 nm, 10 GV/m apex field, 2e7 SPs).  Multi-GPU: a single instance does not
shard, so N ranks run N independent replicas (weak scaling, no collective on the data path).

value: particle updates per second (SPs advanced through a full step), whole job, inputs
resident in HBM.  e2e: the same metric through the public API with the step's particle state
copied in from pinned host memory and the diagnostics read back, every step.
--impl reference times the FP64 CPU oracle (the only reference this paper has) on a bounded
particle sample of the same workload.
"""
import os

# the CPU baseline states the threads it uses: one per process (numpy's BLAS pool would add more)
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import math
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "PIC-MCC particle-updates/s (full step)"
UNIT = "particle-updates/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
FP64_PEAK_TFLOPS = 1.25          # nominal GB300 FP64 rate (the recipe's unit table)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return PEAKS_FALLBACK, "fallback"


def workload_name(cfg, name):
    return (f"{name}: {cfg['nx']}x{cfg['ny']}x{cfg['nz']} cells dx={cfg['dx']*1e9:g} nm, tip r={cfg['tip_radius']*1e9:g} "
            f"nm h={cfg['tip_height']*1e9:g} nm, apex {cfg['apex_field']/1e9:g} GV/m, {cfg['n_sp']:.3g} SPs "
            f"(40% e-, 40% Cu, 20% Cu+), dt={cfg['dt']*1e15:g} fs")


class ClockSampler:
    """nvidia-smi clock samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                pass
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}
        return out


# ---- algorithmic traffic per stage (bytes) -------------------------------------------------------
def stage_units(cfg, counts, mg_cycles, nface, emission_evals):
    n_sp = sum(counts)
    n_chg = counts[0] + sum(counts[2:])     # e-, Cu+ (and Cu2+)
    ncell = cfg["nx"] * cfg["ny"] * cfg["nz"]
    nnode = (cfg["nx"] + 1) * (cfg["ny"] + 1) * (cfg["nz"] + 1)
    return {
        # read pos+vel+w (28 B), write pos+vel (24 B), key (4 B) per SP
        "push": ("hbm", 56.0 * n_sp),
        # key reads (8), perm write/read/fix (12), record read+write (72) per SP; per-cell scan 12 B x 3 species
        "sort": ("hbm", 92.0 * n_sp + 36.0 * ncell),
        # pos + w per charged SP (16 B); node charge cleared and accumulated (16 B/node)
        "deposit": ("hbm", 16.0 * n_chg + 16.0 * nnode),
        # per refinement cycle ~153 B/node (fixed-point residual 21, fine-level V-cycle with 3 + 3
        # sweeps 97 and its coarser levels ~14, correction 21); per solve a last residual 21 and the
        # field 24
        "solve": ("hbm", (153.0 * max(mg_cycles, 1) + 45.0) * nnode),
        # MCC + DFI: positions/offsets/velocities of e- and Cu (40 B) + neutral pass (24 B)
        "collide": ("hbm", 40.0 * (counts[0] + counts[1]) + 24.0 * counts[1]),
        # FP64 emission integral: ~640 flops per transmission evaluation (32-node Gamow quadrature,
        # turning points, supply and Nottingham kernels), counted per evaluation by the library
        "emit": ("alu64", 640.0 * emission_evals),
    }


# Algorithmic bytes of the library's kernels.  Grid kernels: bytes per work unit the library
# reports for the launch (nodes of the level; slots of the swept colour for the smoothers, colour-0
# slots for k_residual).  Particle kernels: bytes per SP of the species the kernel covers, per step.
KERNEL_BYTES_PER_UNIT = {
    "k_smooth": 13.0,        # per slot of the colour swept: f 4 + mask 1 + u write 4, other colour's u 4
    "k_smooth_first": 9.0,   # first sweep of a cycle: the other colour is zero and not read
    "k_residual": 17.0,      # per colour-0 slot: u 4 + other colour's u 4 + f 4 + mask 1 + r write 4
    "k_restrict": 21.0,      # per coarse node: the colour-0 fine residuals it covers 16 + mask 1 + f write 4
    "k_prolong": 9.5,        # per fine node: u read + write 8 + mask 1 + coarse u 0.5
    "k_residual64": 21.0,    # per node: phi 8 + charge Q 8 + mask 1 + level right-hand side write 4
    "k_correct": 21.0,       # per node: phi read + write 16 + u 4 + mask 1
    "k_dirichlet": 1.0,      # per node: mask 1 (Dirichlet values written on the mask only)
    "k_efield": 24.0,        # per node: phi 8 + E write 16
}
# DRAM bytes (read + write) per launch from one ncu capture of the unchanged kernel on the
# production grid: (workload, kernel) -> bytes.  A kernel that has changed since its capture has
# no entry (the bench then reports null).
# k_smooth: the non-first sweeps of levels 0-2 (11 launches per level and step) move 193.17, 19.32
# and 2.48 MB per launch (read + write), captured on the production grid with a tenth of the SPs
# (the smoother's traffic depends on the grid alone), 71.65 MB per launch on average.
NCU_TRAFFIC_PER_LAUNCH = {("production", "k_smooth"): 71.65e6}
KERNEL_BYTES_PER_SP = {      # (bytes, species the launches of one step cover)
    "k_push": (56.0, "all"),         # pos+vel+w read 28, pos+vel write 24, key 4 (+ 8 B per node of charge)
    "k_gather": (76.0, "all"),       # perm 4 + 36 B record read + 36 B record write
    "k_deposit": (16.0, "charged"),  # pos + w of e- and Cu+ (+ 8 B per node of charge, below)
}


# The particle kernels of the benchmark spec's figure (push with its fused charge deposit, impact and
# field ionization), their algorithmic bytes per step:
#   push + crossers + clearing the charge: 56 B per SP (read pos+vel 24 + w 4, write pos+vel 24,
#     cell key 4) + 8 B per node (the deposited charge written once) + 12 B per node (the node
#     field read once: cell-sorted SPs share their cells' corners);
#   impact ionization (count + products): read vel + w + id (24 B) per e- and Cu SP;
#   field ionization (count + products): read pos + w (16 B) per Cu SP.
PARTICLE_KERNELS = ("k_push", "k_cross", "k_mcc_count", "k_mcc_products", "k_dfi_count", "k_dfi_products")


def particle_roofline(kt, counts, nnode, steps, hbm_peak, pk_src):
    """Roofline of the push + deposit + MCC + DFI kernels over the timed region (their summed
    event-timed durations against their summed algorithmic bytes)."""
    n_all = sum(counts)
    parts = {
        "push_deposit": (("k_push", "k_cross"), 56.0 * n_all + 20.0 * nnode),
        "impact_ionization": (("k_mcc_count", "k_mcc_products"), 24.0 * (counts[0] + counts[1])),
        "field_ionization": (("k_dfi_count", "k_dfi_products"), 16.0 * counts[1]),
    }
    out, tot_b, tot_ms = {}, 0.0, 0.0
    for name, (ks, b) in parts.items():
        ms = sum(kt[k][1] for k in ks if k in kt)
        if ms <= 0:
            continue
        ach = b * steps / (ms * 1e-3) / 1e9
        out[name] = {"ms_per_step": round(ms / steps, 4), "alg_bytes_per_step": round(b), "achieved_gbs": round(ach, 1),
                     "frac": round(ach / hbm_peak, 4)}
        tot_b += b * steps
        tot_ms += ms
    if tot_ms <= 0:
        return None
    ach = tot_b / (tot_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s", "frac": round(ach / hbm_peak, 4),
            "kernels": list(PARTICLE_KERNELS), "ms_per_step": round(tot_ms / steps, 4), "parts": out,
            "alg_bytes": "56 B per SP + 8 B per node of charge + 12 B per node of field (push, crossers, charge clear + "
                         "deposit); 24 B per e- and Cu SP (impact ionization); 16 B per Cu SP (field ionization)",
            "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if pk_src == "measured" else pk_src}


def kernel_roofline(name, timing, counts, nnode, steps, hbm_peak, pk_src):
    """Roofline of one kernel from its live event timing over the timed region."""
    launches, ms, units = timing
    if name in KERNEL_BYTES_PER_UNIT:
        alg = KERNEL_BYTES_PER_UNIT[name] * units
        per_unit = f"{KERNEL_BYTES_PER_UNIT[name]:g} B per unit x {units / launches:.4g} units per launch"
    elif name in KERNEL_BYTES_PER_SP:
        b, which = KERNEL_BYTES_PER_SP[name]
        n = sum(counts) if which == "all" else counts[0] + counts[2]
        node_b = 8.0 if name in ("k_deposit", "k_push") else 0.0
        alg = b * n * steps + node_b * nnode * steps
        per_unit = f"{b:g} B per SP x {n:.4g} SPs per step" + (" + 8 B per node" if node_b else "")
    else:
        return None
    achieved = alg / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(achieved / hbm_peak, 4), "traffic": None, "kernel": name,
            "launches": int(launches), "avg_launch_us": round(1e3 * ms / launches, 2),
            "alg_bytes_per_launch": round(alg / launches), "alg_bytes": per_unit,
            "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if pk_src == "measured" else pk_src}


def timed_steps(sim, stream, steps, clk=None):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d0 = sim.diagnostics()
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    d1 = sim.diagnostics()
    return e0.elapsed_time(e1), d0, d1


def reduce_over_ranks(dist, elapsed_ms, updates, e2e_rate, device):
    """Whole-job numbers of N replicas: the slowest rank's time and the work summed over ranks
    (updates in the timed region, end-to-end update rates).  dist None: one process."""
    if dist is None:
        return elapsed_ms, updates, e2e_rate
    import torch
    t = torch.tensor([elapsed_ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([updates, e2e_rate], device=device, dtype=torch.float64)
    dist.all_reduce(u)
    return t.item(), u[0].item(), u[1].item()


def run_ours(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2402_08404_gb300 import pic, synth
    cfg = dict(synth.CONFIGS[args.config])
    cfg["seed"] = cfg["seed"] + rank
    n_sp = cfg["n_sp"]
    nnode_ = (cfg["nx"] + 1) * (cfg["ny"] + 1) * (cfg["nz"] + 1)
    pop = synth.plasma(cfg, seed=cfg["seed"])
    cap = (int(0.4 * n_sp * 1.25), int(0.4 * n_sp * 1.25), int(0.2 * n_sp * 1.5))
    prod_flags = pic.F_PRODUCTION if args.form == "production" else (pic.F_ALL & ~pic.F_SURROGATE & ~pic.F_MIXED_MG)
    if args.circuit:   # the paper's external circuit: 1 kOhm, 1 pF, Shockley-Ramo gap current
        cfg["circuit_R"], cfg["circuit_C"] = 1e3, 1e-12
        prod_flags |= pic.F_CIRCUIT
    if args.elastic:   # elastic e-Cu, Cu-Cu and Cu+-Cu charge exchange with the stand-in cross sections
        prod_flags |= pic.F_ELASTIC
    if args.extrapolate:   # each step's solve starts from 2 phi^n - phi^(n-1)
        prod_flags |= pic.F_EXTRAPOLATE
    if args.coulomb:   # e-e, e-Cu+, Cu+-Cu+ Coulomb collisions (lnL = 10)
        prod_flags |= pic.F_COULOMB
    if args.merge > 0:   # SP merging in cells above this many SPs of a species
        cfg["merge_max"] = args.merge
        prod_flags |= pic.F_MERGE
    if args.ion2:   # Cu2+: double ionization, ionization of Cu+, Coulomb pairs with Cu2+ (with --coulomb)
        prod_flags |= pic.F_ION2
        cap = cap + (int(0.2 * n_sp * 0.5),)
    plain_flags = pic.F_ALL & ~pic.F_SURROGATE & ~pic.F_MIXED_MG
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = pic.Pic(cfg, capacity=cap, flags=prod_flags, mg_tol=args.mg_tol, mg_max_cycles=60, stream=stream,
                      mg_sweeps=args.mg_sweeps)
        for s, k in enumerate("eni"):
            sim.load_particles(s, pop[k])
        sim.set_clock(0, n_sp)
        sim.solve_field()
        # launch shapes picked by the library's autotuner on this state (untimed set-up)
        tune = sim.autotune() if args.autotune else None
        sur = None
        if prod_flags & pic.F_SURROGATE:
            # the learned emission model: trained here on the library's own FP64 integral (untimed)
            sur = sim.surrogate_train(nsamples=args.sur_samples, epochs=args.sur_epochs, batch=8192, lr=3e-3,
                                      seed=cfg["seed"])
        sim.step(args.warmup)
        # find the kernel with the largest summed device time over two untimed steps; only its
        # launches are bracketed by events in the timed region
        sim.set_kernel_timing(sim.kernel_names())
        sim.step(2)
        kt_all = sim.kernel_timing()
        dom_kernel = max(kt_all, key=lambda k: kt_all[k][1])
        timed = sorted({dom_kernel, *[k for k in PARTICLE_KERNELS if k in kt_all]})
        sim.set_kernel_timing(timed)
        if dist:
            dist.barrier()
        with ClockSampler(local) as clk:
            # the timed region is the profiler range (ncu --profile-from-start off captures only it)
            torch.cuda.profiler.start()
            elapsed_ms, d0, d1 = timed_steps(sim, stream, args.steps)
            torch.cuda.profiler.stop()
        kt_live = sim.kernel_timing()
        kt_dom = kt_live.get(dom_kernel)
        sim.set_kernel_timing([])
        if dist:
            dist.barrier()
        launches = d1["kernel_launches"] - d0["kernel_launches"]
        updates = args.steps * 0.5 * (sum(d0["count"]) + sum(d1["count"]))
        sur_faces = d1["surrogate_faces"]
        # the same form replayed as one CUDA graph per step (Poisson loop as a device-side while node)
        graph = None
        if args.graph_steps > 0:
            sim.set_flags(prod_flags | pic.F_GRAPH)
            sim.step(2)     # one eager step records the graphs, one replay warms them
            gm, g0, g1 = timed_steps(sim, stream, args.graph_steps)
            graph = {"ms_per_step": gm / args.graph_steps, "steps": args.graph_steps,
                     "particle_updates_per_s": args.graph_steps * 0.5 * (sum(g0["count"]) + sum(g1["count"])) / (gm * 1e-3),
                     "mg_cycles": g1["mg_cycles"]}
            sim.set_flags(prod_flags)
        # the plain GPU form on the same state: full FP64 emission integral, FP64 V-cycles
        plain = None
        if args.plain_steps > 0 and prod_flags != plain_flags:
            sim.set_flags(plain_flags)
            sim.step(1)
            pm, p0, p1 = timed_steps(sim, stream, args.plain_steps)
            plain = {"ms_per_step": pm / args.plain_steps,
                     "stage_ms": {k: round(p1["ms"][i] / args.plain_steps, 4) for i, k in
                                  enumerate(["emit", "push", "sort", "collide", "deposit", "solve", "heat"])},
                     "mg_cycles": p1["mg_cycles"]}
            sim.set_flags(prod_flags)
        # end to end through the public API: pinned host state in, diagnostics out, every step
        pinned = {}
        for k in "eni":
            pinned[k] = {}
            for f, v in pop[k].items():
                t = torch.empty(len(v), dtype={np.float32: torch.float32, np.int32: torch.int32,
                                               np.uint64: torch.int64}[v.dtype.type], pin_memory=True)
                a = t.numpy().view(v.dtype)
                a[:] = v
                pinned[k][f] = a
        h2d = sum(a.nbytes for k in pinned for a in pinned[k].values())

        e2e_phase = {"load_ms": 0.0, "step_ms": 0.0, "diagnostics_ms": 0.0}

        def e2e_step():
            # host clock per phase (each phase ends in a stream synchronisation of the library)
            t = time.perf_counter()
            sim.load_all([pinned[k] for k in "eni"])
            t1 = time.perf_counter()
            sim.step(1)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            n = sum(sim.diagnostics()["count"])
            t3 = time.perf_counter()
            for k, v in zip(e2e_phase, (t1 - t, t2 - t1, t3 - t2)):
                e2e_phase[k] += v * 1e3
            return n

        if args.e2e_steps > 0:
            e2e_step()   # one untimed warm-up step, as for the device-timed region
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_updates = 0
        for _ in range(args.e2e_steps):
            e2e_updates += e2e_step()
        torch.cuda.synchronize()
        e2e_s = max(time.perf_counter() - t0, 1e-9)
        # the same workload at a larger w_min: more real particles per SP, so the collision
        # processes produce events every step and the solve sees the space charge of the seeded
        # plasma (untimed for the headline; its own event-timed numbers)
        rich = None
        if args.rich_steps > 0:
            sim_r = None
            try:
                cfg_r = dict(cfg, w_min=args.rich_wmin)
                sim_r = pic.Pic(cfg_r, capacity=tuple(2 * c for c in cap), flags=prod_flags, mg_tol=args.mg_tol,
                                mg_max_cycles=60, stream=stream, mg_sweeps=args.mg_sweeps)
                for s_, k in enumerate("eni"):
                    sim_r.load_particles(s_, pop[k])
                sim_r.set_clock(0, n_sp)
                sim_r.solve_field()
                if sur is not None:
                    sim_r.surrogate_copy_from(sim)
                sim_r.step(2)
                sim_r.set_kernel_timing([k for k in PARTICLE_KERNELS] + ["k_smooth", "k_residual64"])
                rm, r0, r1 = timed_steps(sim_r, stream, args.rich_steps)
                kt_r = sim_r.kernel_timing()
                mc_r = [0.5 * (a + b) for a, b in zip(r0["count"], r1["count"])]
                rich = {"w_min": args.rich_wmin, "steps": args.rich_steps, "ms_per_step": rm / args.rich_steps,
                        "particle_updates_per_s": args.rich_steps * sum(mc_r) / (rm * 1e-3),
                        "impact_ionizations_last_step": r1["impact_ionizations"],
                        "field_ionizations_last_step": r1["field_ionizations"],
                        "mg_cycles_per_step": (r1["mg_cycles_total"] - r0["mg_cycles_total"]) / args.rich_steps,
                        "max_face_field": r1["max_face_field"], "count_end": r1["count"],
                        "stage_ms": {k: round(r1["ms"][i] / args.rich_steps, 4) for i, k in
                                     enumerate(["emit", "push", "sort", "collide", "deposit", "solve", "heat"])},
                        "kernel_ms_per_step": {k: round(v[1] / args.rich_steps, 4) for k, v in kt_r.items()},
                        "roofline_particles": particle_roofline(kt_r, mc_r, nnode_, args.rich_steps,
                                                                peaks()[0].get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]),
                                                                peaks()[1])}
            except Exception as ex:   # a refused step (capacity, no convergence) is reported, not fatal
                rich = {"w_min": args.rich_wmin, "error": str(ex)}
            finally:
                if sim_r is not None:
                    sim_r.close()
    # max time over ranks, sum of work
    t_max, tot_updates, tot_e2e = reduce_over_ranks(dist, elapsed_ms, updates, e2e_updates / e2e_s, "cuda")
    times = [t_max]
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return None
    pk, pk_src = peaks()
    stages = ["emit", "push", "sort", "collide", "deposit", "solve", "heat"]
    stage_ms = {s: d1["ms"][i] / args.steps for i, s in enumerate(stages)}
    units = stage_units(cfg, d1["count"], d1["mg_cycles"], sim.nface, d1["emission_evals"])
    dom = max((s for s in units), key=lambda s: stage_ms[s])
    kind, amount = units[dom]
    t_s = stage_ms[dom] * 1e-3
    mean_counts = [0.5 * (a + b) for a, b in zip(d0["count"], d1["count"])]
    nnode = (cfg["nx"] + 1) * (cfg["ny"] + 1) * (cfg["nz"] + 1)
    roof = None
    if kt_dom:
        roof = kernel_roofline(dom_kernel, kt_dom, mean_counts, nnode, args.steps,
                               pk.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]), pk_src)
    if roof is not None:
        roof["traffic"] = NCU_TRAFFIC_PER_LAUNCH.get((args.config, dom_kernel))
        roof["kernel_share_of_step"] = round(kt_dom[1] / times[0], 4)
        roof["stage"] = {"stage": dom, "stage_ms": round(stage_ms[dom], 4)}
    elif kind == "hbm":
        peak = pk.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
        achieved = amount / t_s / 1e9
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None, "kernel_stage": dom,
                "peak_source": pk_src, "stage_ms": round(stage_ms[dom], 4)}
    else:
        achieved = amount / t_s / 1e12
        roof = {"bound": "alu", "achieved": round(achieved, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": round(achieved / FP64_PEAK_TFLOPS, 4), "traffic": None, "kernel_stage": dom,
                "peak_source": "nominal FP64 rate", "stage_ms": round(stage_ms[dom], 4)}
    roof_p = particle_roofline(kt_live, mean_counts, nnode, args.steps, pk.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]),
                               pk_src)
    kernel_ms = {k: round(v[1] / 2, 4) for k, v in sorted(kt_all.items(), key=lambda kv: -kv[1][1])[:20]}
    ms_step = times[0] / args.steps
    form = ("surrogate emission (FP32-Gamow integral where it falls back) + FP32 V-cycles with FP64 refinement"
            if args.form == "production" else "full FP64 emission integral + FP64 V-cycles")
    out = {
        "metric": METRIC, "value": tot_updates / (times[0] * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64+bf16", "data": "synthetic (seeded plasma, Philox)",
        "config": {"workload": workload_name(cfg, args.config), "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (2e7 SPs x 36 B SoA + 33.9M-node grids)",
                   "form": form, "poisson_tol": args.mg_tol,
                   "circuit": ({"R_ohm": 1e3, "C_F": 1e-12, "V_gap_end": d1["V_gap"], "I_gap_end": d1["I_gap"]}
                               if args.circuit else None),
                   "elastic": ({"e_Cu": d1["elastic_en"], "Cu_Cu": d1["elastic_nn"], "exchange": d1["charge_exchanges"]}
                               if args.elastic else None),
                   "coulomb": ({"e_e": d1["coulomb_ee"], "e_Cu+": d1["coulomb_ei"], "Cu+_Cu+": d1["coulomb_ii"]}
                               if args.coulomb else None),
                   "merge": ({"merge_max": args.merge, "merged_last_step": d1["merged"]} if args.merge > 0 else None),
                   "ion2": ({"double_ionizations_last_step": d1["double_ionizations"],
                             "cu1_ionizations_last_step": d1["ion_ionizations"], "count_cu2_end": d1["count"][3],
                             "coulomb_e_cu2_last_step": d1["coulomb_ej"], "coulomb_cu1_cu2_last_step": d1["coulomb_ij"],
                             "coulomb_cu2_cu2_last_step": d1["coulomb_jj"]} if args.ion2 else None),
                   "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()}, "mg_cycles": d1["mg_cycles"],
                   "mg_cycles_per_step": (d1["mg_cycles_total"] - d0["mg_cycles_total"]) / args.steps,
                   "kernel_ms_per_step": kernel_ms,
                   "surrogate": None if sur is None else {
                       "val_rms_dlog10J": round(sur["val_rms_dlog10J"], 4),
                       "valid_sample_fraction": round(sur["valid_sample_fraction"], 3),
                       "faces_served_per_step": round(sur_faces / max(sim.nface, 1), 4),
                       "fallback_faces_last_step": {"outside_range": d1["fallback_range"], "bin_not_validated": d1["fallback_bin"]},
                       "train_s": round((sur["ms_data"] + sur["ms_train"]) / 1e3, 2),
                       "data_s": round(sur["ms_data"] / 1e3, 2), "optimiser_steps": int(sur["steps"]),
                       "train_ms_per_optimiser_step": round(sur["ms_train"] / max(sur["steps"], 1), 4)},
                   "plain_form": plain, "graph_form": graph, "collision_rich": rich, "autotune": tune},
        "roofline": roof,
        "roofline_particles": roof_p,
        "clocks": clk.summary(),
        "e2e": {"value": tot_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(__import__("ctypes").sizeof(pic.Diag)),
                "phase_ms_per_step": {k: round(v / max(args.e2e_steps + 1, 1), 3) for k, v in e2e_phase.items()}},
        "gpu_launches": int(launches),
    }
    if args.cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(cfg, pop, args.cpu_sample, steps=1)
        out["cpu_baseline"]["nproc"] = os.cpu_count()
        if args.cpu_cores:
            # the same oracle on every host core and on 16 (the paper's thread count, Sec. 3.2)
            out["cpu_baseline_cores"] = [cpu_baseline(cfg, pop, args.cpu_sample // 2, steps=1, workers=w)
                                         for w in sorted({os.cpu_count() or 1, 16})]
    sim.close()
    if dist:
        dist.destroy_process_group()
    return out


# ---- the oracle on a bounded sample -----------------------------------------------------------
def _oracle_sample(pop, sample, seed):
    """A uniform sample of about `sample` SPs of the workload (each species in proportion)."""
    rng = np.random.default_rng(seed)
    n_tot = sum(len(pop[k]["x"]) for k in "eni")
    out = {}
    for k in "eni":
        n = len(pop[k]["x"])
        idx = np.sort(rng.choice(n, size=max(1, int(sample * n / n_tot)), replace=False))
        out[k] = {f: np.asarray(v)[idx] for f, v in pop[k].items()}
    return out


def _oracle_particle_steps(args):
    """The oracle's particle stages (push + boundary, stable sort, impact + field ionization,
    deposit) on one sample, on the full geometry with a uniform applied field: (SP updates timed,
    seconds).  Module level so that a spawned worker can run it."""
    cfg, sp0, steps, warmup = args
    sys.path.insert(0, ROOT)
    from oracle import collide, field, particles as P
    from oracle.grid import Grid
    from oracle import constants as OC
    g = Grid(cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["tip_radius"], cfg["tip_height"])
    phi = (cfg["apex_field"] / 5.0) * g.dx * np.arange(g.nz + 1, dtype=np.float64)[:, None, None] * np.ones((1, g.ny + 1, g.nx + 1))
    phi[g.dirichlet_mask() & (np.arange(g.nz + 1)[:, None, None] < g.nz)] = 0.0
    E = field.efield(g, phi)
    sp = {k: P.stable_sort(g, v)[0] for k, v in sp0.items()}
    prm = {"dt": cfg["dt"], "seed": cfg["seed"], "w_min": cfg["w_min"]}
    m = {"e": OC.M_E, "n": OC.M_CU, "i": OC.M_CU}
    z = {"e": -1, "n": 0, "i": 1}
    done, t_total = 0, 0.0
    for it in range(warmup + steps):
        t0 = time.perf_counter()
        count = sum(P.count(sp[k]) for k in "eni")
        offs = {}
        for k in "eni":
            qmdt = P.kick_factor(z[k], m[k], cfg["dt"]) if z[k] else 0.0
            new = P.push_f32(sp[k], E, qmdt, np.float32(cfg["dt"] / cfg["dx"]))
            alive, _ = P.boundary(g, sp[k], new, k == "i", m[k])
            for c, v in zip(("x", "y", "z", "vx", "vy", "vz"), new):
                sp[k][c] = v.astype(np.float32)
            sp[k], offs[k] = P.stable_sort(g, sp[k], alive)
        ids = collide.Counter(10 ** 12)
        ni, ne, _ = collide.impact_ionization(g, prm, sp["e"], offs["e"], sp["n"], offs["n"], it, ids)
        ni2, ne2, _ = collide.field_ionization(g, prm, sp["n"], E, it, ids)
        sp["i"] = P.concat(P.concat(sp["i"], ni), ni2)
        sp["e"] = P.concat(P.concat(sp["e"], ne), ne2)
        P.deposit(g, sp["i"], 1, Q=P.deposit(g, sp["e"], -1))
        dt_ = time.perf_counter() - t0
        if it >= warmup:
            done += count
            t_total += dt_
    return done, t_total


def cpu_baseline(cfg, pop, sample, steps=1, warmup=0, workers=1):
    """The oracle's particle-update rate as it stands, on host cores.  workers = 1: one process
    (single-threaded numpy).  workers > 1: that many spawned processes, each running the oracle on
    its own sample of the same size (the samples are independent, as the workload's cells are),
    the rate being all their SP updates over the slowest worker's time."""
    samples = [_oracle_sample(pop, sample, 1000 + w) for w in range(workers)]
    jobs = [(cfg, sp, steps, warmup) for sp in samples]
    if workers == 1:
        res = [_oracle_particle_steps(jobs[0])]
    else:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            res = pool.map(_oracle_particle_steps, jobs)
    done = sum(r[0] for r in res)
    t_max = max(r[1] for r in res)
    return {"value": done / t_max, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"{sample} SPs drawn uniformly from the workload per process ({workers} process(es)), the workload's full "
                      f"grid, uniform applied field; oracle particle stages (push+boundary, stable sort, "
                      f"MCC, DFI, deposit), {steps} step(s); numpy, one thread per process; the grid stages "
                      f"(33.9M-node CG, 75k-face integrals) are not sampled",
            "seconds": round(t_max, 3)}


def ensemble_share(n, world, rank):
    """The ensemble's instances that one rank steps: rank, rank + world, ...  Every instance
    belongs to exactly one rank (the instances are independent: no collective on the data path)."""
    return list(range(rank, n, world))


def gather_instances(dist, idx, rows, n, device):
    """Per-instance diagnostics of every rank, on every rank: rows (len(idx) x k) of this rank's
    instances idx -> an n x k table (NaN where no rank reported).  One all_gather of a small
    padded block after the timed region (dist None: one process)."""
    import torch
    rows = np.asarray(rows, dtype=np.float64).reshape(len(idx), -1)
    k = rows.shape[1]
    table = np.full((n, k), np.nan)
    if dist is None:
        table[idx] = rows
        return table
    world = dist.get_world_size()
    m = (n + world - 1) // world
    buf = torch.full((m, k + 1), float("nan"), dtype=torch.float64, device=device)
    if len(idx):
        buf[:len(idx), 0] = torch.tensor(idx, dtype=torch.float64, device=device)
        buf[:len(idx), 1:] = torch.tensor(rows, device=device)
    outs = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(outs, buf)
    for o in outs:
        for r in o.cpu().numpy():
            if not np.isnan(r[0]):
                table[int(r[0])] = r[1:]
    return table


def run_ensemble(args):
    """64 independent instances (apex fields 6-12 GV/m, grids 32x32x64 to 128x128x256) stepped by
    one CUDA-graph launch per step through pic_batch_step, against the same instances stepped one
    after another in the eager form.  With N ranks the one ensemble is partitioned: rank r steps
    instances r, r + N, ... (strong scaling: the job is fixed), and the per-instance diagnostics
    are gathered after the timed region.  Each rank trains the surrogate once on its first
    instance (the same seed everywhere, so the same network) and shares it; every instance is
    autotuned on its own grid."""
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2402_08404_gb300 import pic, synth
    cfgs_all = synth.ensemble_configs(n=args.ensemble_n, seed=7)
    mine = ensemble_share(len(cfgs_all), world, rank)
    cfgs = [cfgs_all[i] for i in mine]
    stream = torch.cuda.Stream()
    sims, tunes = [], []
    with torch.cuda.stream(stream):
        for i, cfg in enumerate(cfgs):
            n = cfg["n_sp"]
            # headroom for field emission: at 12 GV/m a small tip emits several thousand SPs per step
            cap = (int(0.4 * n * 2.5) + 400_000, int(0.4 * n * 1.5) + 100_000, int(0.2 * n * 4.0) + 100_000)
            sim = pic.Pic(cfg, capacity=cap, flags=pic.F_PRODUCTION, mg_tol=args.mg_tol, mg_max_cycles=60, stream=stream)
            pop = synth.plasma(cfg, seed=cfg["seed"])
            for s, k in enumerate("eni"):
                sim.load_particles(s, pop[k])
            sim.set_clock(0, n)
            sim.solve_field()
            if i == 0:
                sim.surrogate_train(nsamples=args.sur_samples, epochs=args.sur_epochs, batch=8192, lr=3e-3, seed=1)
            else:
                sim.surrogate_copy_from(sims[0])
            tunes.append(sim.autotune())
            sims.append(sim)
        # eager form, instances one after another
        for sim in sims:
            sim.step(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c0 = sum(sum(sim.diagnostics()["count"]) for sim in sims)
        for _ in range(args.ensemble_serial_steps):
            for sim in sims:
                sim.step(1)
        torch.cuda.synchronize()
        serial_s = (time.perf_counter() - t0) / max(args.ensemble_serial_steps, 1)
        batch = pic.Batch(sims)
        batch.step(max(args.warmup, 2))
        if dist:
            dist.barrier()
        with ClockSampler(local) as clk:
            d0 = [sim.diagnostics() for sim in sims]
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            batch.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
        if dist:
            dist.barrier()
        d1 = [sim.diagnostics() for sim in sims]
    updates = args.steps * 0.5 * sum(sum(a["count"]) + sum(b["count"]) for a, b in zip(d0, d1))
    t_max, tot_updates, tot_serial = reduce_over_ranks(dist, ms, updates, c0 / serial_s, "cuda")
    # per-instance diagnostics of the whole ensemble: step, SPs per species, mg cycles
    table = gather_instances(dist, mine, [[d["step"], *d["count"], d["mg_cycles"]] for d in d1], len(cfgs_all), "cuda")
    batch.close()
    for sim in sims:
        sim.close()
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return None
    grids = sorted({(c["nx"], c["ny"], c["nz"]) for c in cfgs_all})
    return {
        "metric": "ensemble PIC-MCC particle-updates/s (one graph launch per step)", "value": tot_updates / (t_max * 1e-3),
        "unit": "particle-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f32+f64+bf16", "data": "synthetic (seeded plasma, Philox)",
        "config": {"workload": f"ensemble: {len(cfgs_all)} instances, apex 6-12 GV/m, grids {grids[0]}..{grids[-1]}, "
                               f"dx 0.5-1 nm, {sum(c['n_sp'] for c in cfgs_all):.3g} SPs in all (1e4-2e6 each)",
                   "parallelism": f"instances partitioned over {world} rank(s) (rank r: r, r+{world}, ...)",
                   "form": "production (surrogate, FP32-Gamow fallback, mixed MG), graph per step",
                   "eager_serial_ms_per_step": round(serial_s * 1e3, 3),
                   "eager_serial_particle_updates_per_s": tot_serial,
                   "speedup_vs_eager_serial": round(serial_s * 1e3 / (ms / args.steps), 3),
                   "instances_stepped": int(np.sum(~np.isnan(table[:, 0]))),
                   "instance_steps": sorted(set(table[:, 0][~np.isnan(table[:, 0])].astype(int).tolist())),
                   "autotune_examples": tunes[:3],
                   "mg_cycles": [int(v) for v in table[:8, 4] if not np.isnan(v)]},
        "clocks": clk.summary(),
    }


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    from paper_2402_08404_gb300 import synth
    cfg = dict(synth.CONFIGS[args.config])
    pop = synth.plasma(cfg, seed=cfg["seed"])
    # each step a bounded sample, so that steps + warmup stay near a minute of CPU work
    sample = max(2000, int(args.cpu_sample * min(1.0, 20.0 / max(1, args.steps + args.warmup))))
    cb = cpu_baseline(cfg, pop, sample, steps=args.steps, warmup=args.warmup)
    return {"metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * cb["seconds"] / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded plasma, Philox)",
            "config": {"workload": workload_name(cfg, args.config), "parallelism": "cpu, 1 thread"},
            "impl": "reference", "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="production")
    ap.add_argument("--form", default="production", choices=["production", "plain"])
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--graph-steps", type=int, default=50)
    ap.add_argument("--ensemble-n", type=int, default=64)
    ap.add_argument("--ensemble-serial-steps", type=int, default=5)
    ap.add_argument("--sur-samples", type=int, default=2_000_000)
    ap.add_argument("--sur-epochs", type=int, default=150)
    ap.add_argument("--mg-tol", type=float, default=1e-6)
    ap.add_argument("--mg-sweeps", type=int, default=0, help="red-black sweeps per V-cycle side (0: library default)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--rich-steps", type=int, default=10, help="steps of the collision-rich form (0: skip)")
    ap.add_argument("--rich-wmin", type=float, default=1e-3, help="w_min of the collision-rich form")
    ap.add_argument("--cpu-sample", type=int, default=60000)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-cpu-cores", dest="cpu_cores", action="store_false",
                    help="skip the oracle timed on all host cores and on 16 processes")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--circuit", action="store_true", help="step with the RC circuit and Shockley-Ramo current")
    ap.add_argument("--elastic", action="store_true", help="step with elastic collisions and charge exchange")
    ap.add_argument("--extrapolate", action="store_true", help="start each solve from the time-extrapolated potential")
    ap.add_argument("--coulomb", action="store_true", help="step with Coulomb collisions between charged SPs")
    ap.add_argument("--ion2", action="store_true", help="step with Cu2+ and its channels (double ionization, Cu+ "
                                                         "ionization; with --coulomb its Coulomb pairs)")
    ap.add_argument("--merge", type=int, default=0, help="merge SPs in cells above this many SPs of a species (0: off)")
    args = ap.parse_args()
    if args.impl == "reference":
        out = run_reference(args)
    elif args.config == "ensemble":
        out = run_ensemble(args)
    else:
        out = run_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
