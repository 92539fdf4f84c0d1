"""Test helpers: oracle reference runs of single stages on seeded inputs (oracle side only)."""
import numpy as np

from oracle import field, particles as P
from oracle.grid import Grid
from oracle import constants as OC

SPECIES = (("e", -1, OC.M_E), ("n", 0, OC.M_CU), ("i", 1, OC.M_CU))


def small_cfg(**kw):
    from paper_2402_08404_gb300 import synth
    cfg = dict(synth.CONFIGS["small"])
    cfg.update(kw)
    return cfg


def fixed_phi(phi):
    """The potential on the library's fixed-point grid (steps of 2^-40 V, round half to even):
    tests that compare integer or bit-exact results hand both sides these representable values."""
    return np.round(np.asarray(phi, dtype=np.float64) * 2.0 ** 40) / 2.0 ** 40


def grid_of(cfg):
    return Grid(cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["tip_radius"], cfg["tip_height"])


def sorted_pop(g, pop):
    out = {}
    for k, _, _ in SPECIES:
        out[k], _ = P.stable_sort(g, {f: np.asarray(v).astype(P.DTYPES[f]) for f, v in pop[k].items()})
    return out


def oracle_push_sort(g, pop_sorted, E, dt):
    """Oracle a3 + a4 for every species from already cell-sorted SPs: returns (sorted SPs,
    offsets, impacts of ions)."""
    out, offs, imp = {}, {}, []
    dtdx = np.float32(dt / g.dx)
    for k, Z, m in SPECIES:
        sp_ = {f: v.copy() for f, v in pop_sorted[k].items()}
        qmdt = P.kick_factor(Z, m, dt) if Z else 0.0
        new = P.push_f32(sp_, E, qmdt, dtdx)
        alive, impacts = P.boundary(g, sp_, new, k == "i", m)
        if k == "i":
            imp = impacts
        for c, v in zip(("x", "y", "z", "vx", "vy", "vz"), new):
            sp_[c] = v.astype(np.float32)
        out[k], offs[k] = P.stable_sort(g, sp_, alive)
    return out, offs, imp


def assert_sp_equal(got, ref, fields=("x", "y", "z", "vx", "vy", "vz", "w", "id")):
    assert len(got["id"]) == len(ref["id"]), (len(got["id"]), len(ref["id"]))
    for f in fields:
        a, b = np.asarray(got[f]), np.asarray(ref[f])
        if not np.array_equal(a, b):
            bad = np.nonzero(a != b)[0]
            raise AssertionError(f"field {f}: {len(bad)} mismatches, first at {bad[:5]}: {a[bad[:5]]} vs {b[bad[:5]]}")


def colocated_population(cfg, seed):
    """Seeded plasma with the species brought together in cells: electrons and ions on neutral
    positions, half the neutrals on the other half's, electrons of 20-300 eV and ions of 1-50 eV
    in random directions (collision tests)."""
    from paper_2402_08404_gb300 import synth
    pop = synth.plasma(cfg, seed=seed)
    rng = np.random.default_rng(seed + 1)
    nn = len(pop["n"]["x"])
    half = nn // 2
    for c in ("x", "y", "z"):
        pop["n"][c][half:2 * half] = pop["n"][c][:half]
    for k, lo, hi, m in (("e", 20.0, 300.0, OC.M_E), ("i", 1.0, 50.0, OC.M_CU)):
        n = len(pop[k]["x"])
        src = rng.integers(0, nn, n)
        for c in ("x", "y", "z"):
            pop[k][c] = pop["n"][c][src].copy()
        speed = np.sqrt(2 * rng.uniform(lo, hi, n) * OC.E_CHARGE / m)
        u = rng.normal(size=(n, 3))
        u /= np.linalg.norm(u, axis=1)[:, None]
        for a, c in enumerate(("vx", "vy", "vz")):
            pop[k][c] = (speed * u[:, a]).astype(np.float32)
    return pop
