"""Seeded synthetic inputs (workload recipe).  Holds none of the step's arithmetic.

The paper runs no public dataset; its late-stage plasma (about 8e6 heavy particles dense
near the apex, ions drifting to the cathode at about 5000 m/s, Sec. 3.2) is stood in for by
a pre-seeded population around the tip:

  * Cu neutrals: density proportional to exp(-d/lambda), d the distance from the tip surface
    (capsule of radius r and height h), lambda = 2r; Maxwellian velocities at 3000 K;
  * Cu+: the same spatial law, velocities Gaussian (3000 K) with a 5000 m/s mean along -z;
  * electrons: half a beam above the apex (column of radius 2r, v along +z, 10-200 eV),
    half on the ions' positions with the ions' weights (a locally neutral cloud) and a 2 eV
    Maxwellian;
  * mix 40 % e- / 40 % Cu / 20 % Cu+ by SP count, weights uniform integers 1..8 (units of w_min);
  * w_min = 0.01 real particles per weight unit on the 1 nm grid and 1e-5 on the 0.5 nm
    grids: the net space charge of the seeded beam then stays below about 0.5 GV/m, well
    under the applied field (w_min = 1e-4 on the 0.5 nm grid screens the apex down to
    ~1 GV/m; 0.01 gives fields far above the barrier-suppression limit and ionizes every
    neutral in the first step);
  * ids 0..N-1 in the order electrons, neutrals, ions.

Points closer than one cell to the tip surface are redrawn, so no SP starts in a solid cell.
"""
import math

import numpy as np

KB = 1.380649e-23
QE = 1.602176634e-19
ME = 9.1093837015e-31
MCU = 63.546 * 1.66053906660e-27

# Workload configurations (grid cells, spacing, tip, field, SP count, time step).
CONFIGS = {
    "small": dict(nx=32, ny=32, nz=64, dx=1e-9, tip_radius=3e-9, tip_height=20e-9, apex_field=8e9,
                  n_sp=50_000, dt=5e-17, steps=100, T0=300.0, work_function=4.5, w_min=0.01,
                  w_max_units=1024, n_heat=1000, seed=1),
    "production": dict(nx=256, ny=256, nz=512, dx=0.5e-9, tip_radius=5e-9, tip_height=60e-9,
                       apex_field=10e9, n_sp=20_000_000, dt=5e-17, steps=10_000, T0=300.0,
                       work_function=4.5, w_min=1e-5, w_max_units=1024, n_heat=1000, seed=1),
    # a profiling case one eighth of production: arrays still larger than L2, ~1 GB on the device
    "medium": dict(nx=128, ny=128, nz=256, dx=0.5e-9, tip_radius=5e-9, tip_height=30e-9,
                   apex_field=10e9, n_sp=4_000_000, dt=5e-17, steps=10_000, T0=300.0,
                   work_function=4.5, w_min=1e-5, w_max_units=1024, n_heat=1000, seed=1),
    # the production grid with a tenth of its SPs: grid kernels at full size, ~3 GB on the device
    "production_grid": dict(nx=256, ny=256, nz=512, dx=0.5e-9, tip_radius=5e-9, tip_height=60e-9,
                            apex_field=10e9, n_sp=2_000_000, dt=5e-17, steps=10_000, T0=300.0,
                            work_function=4.5, w_min=1e-5, w_max_units=1024, n_heat=1000, seed=1),
    "large": dict(nx=512, ny=512, nz=1024, dx=0.5e-9, tip_radius=10e-9, tip_height=100e-9,
                  apex_field=12e9, n_sp=200_000_000, dt=5e-17, steps=5000, T0=300.0,
                  work_function=4.5, w_min=1e-5, w_max_units=1024, n_heat=1000, seed=1),
}


def _capsule_points(rng, n, cfg, lam_cells):
    """n points (cell units) with density ~ exp(-d/lambda) outside the tip capsule, d >= 1 cell."""
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    r = cfg["tip_radius"] / cfg["dx"]
    h = cfg["tip_height"] / cfg["dx"]
    zc = h - r
    ax, ay = nx / 2.0, ny / 2.0
    lam = lam_cells
    out = np.zeros((0, 3))
    side_vol = 2 * math.pi * zc * (r * lam + lam * lam)
    cap_vol = 2 * math.pi * (r * r * lam + 2 * r * lam * lam + 2 * lam ** 3)
    p_side = side_vol / (side_vol + cap_vol)
    while len(out) < n:
        m = int((n - len(out)) * 1.3) + 64
        side = rng.random(m) < p_side
        # distance: side ~ (r+d) e^{-d/lam}, cap ~ (r+d)^2 e^{-d/lam} (gamma mixtures)
        d = np.empty(m)
        ws = np.array([r, lam]); ws /= ws.sum()
        wc = np.array([r * r, 2 * r * lam, 2 * lam * lam]); wc /= wc.sum()
        ks = np.where(side, rng.choice(2, size=m, p=ws) + 1, rng.choice(3, size=m, p=wc) + 1)
        d = rng.gamma(ks, lam)
        psi = rng.random(m) * 2 * math.pi
        zs = rng.random(m) * zc
        ct = rng.random(m)                      # cap: uniform direction on the upper hemisphere
        stt = np.sqrt(1 - ct * ct)
        px = np.where(side, ax + (r + d) * np.cos(psi), ax + (r + d) * stt * np.cos(psi))
        py = np.where(side, ay + (r + d) * np.sin(psi), ay + (r + d) * stt * np.sin(psi))
        pz = np.where(side, zs, zc + (r + d) * ct)
        ok = (d >= 1.0) & (px >= 0) & (px < nx) & (py >= 0) & (py < ny) & (pz >= 0) & (pz < nz)
        out = np.concatenate([out, np.stack([px, py, pz], 1)[ok]])
    return out[:n]


def _pack(pos, vel, w, ids):
    return {"x": pos[:, 0].astype(np.float32), "y": pos[:, 1].astype(np.float32),
            "z": pos[:, 2].astype(np.float32), "vx": vel[:, 0].astype(np.float32),
            "vy": vel[:, 1].astype(np.float32), "vz": vel[:, 2].astype(np.float32),
            "w": w.astype(np.int32), "id": ids.astype(np.uint64)}


def _fix_f32(pos, cfg):
    """Keep positions inside the domain after rounding to float32."""
    for a, n in enumerate((cfg["nx"], cfg["ny"], cfg["nz"])):
        p = pos[:, a].astype(np.float32)
        p = np.minimum(p, np.nextafter(np.float32(n), np.float32(0)))
        pos[:, a] = p
    return pos


def plasma(cfg, n_sp=None, seed=1):
    """Seeded SoA population {e, n, i} for configuration dict cfg."""
    rng = np.random.default_rng(seed)
    n_sp = int(cfg["n_sp"] if n_sp is None else n_sp)
    ne, nn = int(0.4 * n_sp), int(0.4 * n_sp)
    ni = n_sp - ne - nn
    r = cfg["tip_radius"] / cfg["dx"]
    h = cfg["tip_height"] / cfg["dx"]
    lam = 2.0 * r
    pos_n = _fix_f32(_capsule_points(rng, nn, cfg, lam), cfg)
    pos_i = _fix_f32(_capsule_points(rng, ni, cfg, lam), cfg)
    s_cu = math.sqrt(KB * 3000.0 / MCU)
    vel_n = rng.normal(0.0, s_cu, size=(nn, 3))
    vel_i = rng.normal(0.0, s_cu, size=(ni, 3))
    vel_i[:, 2] -= 5000.0
    nc = ni
    nb = ne - nc
    # beam column above the apex
    rr = 2.0 * r * np.sqrt(rng.random(nb))
    ps = rng.random(nb) * 2 * math.pi
    zb = h + 1.0 + rng.random(nb) * (cfg["nz"] - h - 1.0)
    pos_b = np.stack([cfg["nx"] / 2 + rr * np.cos(ps), cfg["ny"] / 2 + rr * np.sin(ps), zb], 1)
    Eb = 10.0 + rng.random(nb) * 190.0
    vel_b = np.zeros((nb, 3))
    vel_b[:, 2] = np.sqrt(2.0 * Eb * QE / ME)
    # locally neutral cloud: one electron SP on every ion SP, same weight
    w_n = rng.integers(1, 9, size=nn)
    w_i = rng.integers(1, 9, size=ni)
    pos_c = pos_i.copy()
    s_e = math.sqrt(2.0 * QE / ME)
    vel_c = rng.normal(0.0, s_e, size=(nc, 3))
    pos_e = _fix_f32(np.concatenate([pos_b, pos_c]), cfg)
    vel_e = np.concatenate([vel_b, vel_c])
    w_e = np.concatenate([rng.integers(1, 9, size=nb), w_i])
    ids = np.arange(n_sp, dtype=np.uint64)
    return {"e": _pack(pos_e, vel_e, w_e, ids[:ne]),
            "n": _pack(pos_n, vel_n, w_n, ids[ne:ne + nn]),
            "i": _pack(pos_i, vel_i, w_i, ids[ne + nn:])}


def face_tuples(n, seed=1):
    """Emission-surrogate inputs: F log-uniform 1-15 GV/m, T uniform 300-4000 K,
    work function uniform 4.0-5.0 eV, radius log-uniform 1-20 nm."""
    rng = np.random.default_rng(seed)
    F = 10.0 ** rng.uniform(0.0, math.log10(15.0), n)
    T = rng.uniform(300.0, 4000.0, n)
    W = rng.uniform(4.0, 5.0, n)
    R = 10.0 ** rng.uniform(0.0, math.log10(20.0), n)
    return F, T, W, R


def potential_noise(shape, amplitude, seed=1):
    """Smooth-ish random potential perturbation [V] for field-gather tests."""
    rng = np.random.default_rng(seed)
    return amplitude * rng.standard_normal(shape)


def ensemble_configs(n=64, seed=7):
    """Independent tip instances of the ensemble workload: apex field uniform in 6-12 GV/m, grids
    nx = ny = nz/2 log-uniform between 32 and 128 cells (rounded to multiples of 32, so every
    multigrid level has even sizes), dx uniform in 0.5-1 nm, SPs log-uniform in 1e4-2e6
    (at most 2 per cell, about the production density; denser seeds charge the small grids past
    the barrier-suppression field), a 3 nm tip 20 nm high."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nx = int(32 * round(2.0 ** rng.uniform(5.0, 7.0) / 32.0))
        dx = rng.uniform(0.5, 1.0) * 1e-9
        n_sp = int(min(10.0 ** rng.uniform(4.0, math.log10(2e6)), 2 * nx * nx * 2 * nx))
        out.append(dict(nx=nx, ny=nx, nz=2 * nx, dx=dx, tip_radius=3e-9, tip_height=20e-9,
                        apex_field=rng.uniform(6.0, 12.0) * 1e9, n_sp=n_sp, dt=5e-17, steps=2000, T0=300.0,
                        work_function=4.5, w_min=1e-5, w_max_units=1024, n_heat=1000, seed=1000 + i))
    return out
