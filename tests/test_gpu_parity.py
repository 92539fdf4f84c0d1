"""Parity of the CUDA path (through the C ABI) with the oracle on seeded inputs.

Bars: integer work bit-exact (cell keys, order, weights, ids, decisions, fixed-point charge);
float32 push within 1e-5 relative of the float64 leapfrog; float64 fields within 1e-9 of the
oracle's solution scale; emission J within 1e-8 relative (P_N within 1e-6 of |P_N| + |J| 1 V).
"""
import math

import numpy as np
import pytest

from oracle import collide, emission as em, field, heat, particles as P, step as OS
from oracle import constants as OC
from paper_2402_08404_gb300 import synth

from _util import SPECIES, assert_sp_equal, fixed_phi, grid_of, oracle_push_sort, small_cfg, sorted_pop

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pic():
    import os
    from paper_2402_08404_gb300 import _build
    if not os.path.exists(_build.LIB):
        _build.build()
    from paper_2402_08404_gb300 import pic as m
    return m


def make(pic, cfg, cap=200_000, V0=0.0, flags=None, **kw):
    return pic.Pic(cfg, capacity=cap, V0=V0, flags=pic.F_ALL if flags is None else flags, **kw)


def load(sim, pop):
    for s, (k, _, _) in enumerate(SPECIES):
        sim.load_particles(s, pop[k])


def test_geometry_and_faces(pic):
    cfg = small_cfg()
    g = grid_of(cfg)
    sim = make(pic, cfg, cap=16, V0=10.0)
    v, d, o = sim.faces()
    assert sim.nface == g.nface and sim.nsolid == int(g.solid.sum())
    assert np.array_equal(v, g.face_vcell) and np.array_equal(d, g.face_dir) and np.array_equal(o, g.face_owner)
    sim.close()


def test_laplace_calibration(pic):
    cfg = small_cfg()
    g = grid_of(cfg)
    sim = make(pic, cfg, cap=16, V0=0.0, mg_tol=1e-11)
    V0 = field.calibrate_V0(g, cfg["apex_field"])
    d = sim.diagnostics()
    assert d["V0"] == pytest.approx(V0, rel=1e-8)
    phi_ref = field.solve_poisson(g, d["V0"])
    assert np.max(np.abs(sim.get_potential() - phi_ref)) <= 1e-9 * d["V0"]
    sim.close()


def test_efield_bit_exact(pic):
    cfg = small_cfg()
    g = grid_of(cfg)
    sim = make(pic, cfg, cap=16, V0=50.0)
    phi = fixed_phi(field.solve_poisson(g, 50.0) + synth.potential_noise((g.nz + 1, g.ny + 1, g.nx + 1), 0.3, seed=4))
    sim.set_potential(phi)
    assert np.array_equal(sim.get_efield(), field.efield(g, phi))
    sim.close()


def _pushed_case(pic, n_sp=20000, seed=2, V0=60.0):
    cfg = small_cfg(n_sp=n_sp)
    g = grid_of(cfg)
    sim = make(pic, cfg, V0=V0)
    pop = synth.plasma(cfg, seed=seed)
    phi = fixed_phi(field.solve_poisson(g, V0) + synth.potential_noise((g.nz + 1, g.ny + 1, g.nx + 1), 0.2, seed=seed))
    sim.set_potential(phi)
    load(sim, pop)
    sim.set_clock(3, n_sp)
    return cfg, g, sim, pop, phi


def test_load_sort_is_stable_cell_order(pic):
    cfg, g, sim, pop, phi = _pushed_case(pic)
    ref = sorted_pop(g, pop)
    for s, (k, _, _) in enumerate(SPECIES):
        assert_sp_equal(sim.get_particles(s), ref[k])
    sim.close()


def test_push_sort_bit_exact_and_f64_tolerance(pic):
    cfg, g, sim, pop, phi = _pushed_case(pic)
    E = field.efield(g, phi)
    start = sorted_pop(g, pop)
    ref, offs, impacts = oracle_push_sort(g, start, E, cfg["dt"])
    sim.push()
    sim.sort()
    for s, (k, Z, m) in enumerate(SPECIES):
        got = sim.get_particles(s)
        assert_sp_equal(got, ref[k])
        # float32 push vs the float64 leapfrog (same start state): 1e-5 of the local scale
        x64 = P.push_f64(start[k], E.astype(np.float64), Z * OC.E_CHARGE / m * cfg["dt"], cfg["dt"] / cfg["dx"])
        pos = dict(zip(start[k]["id"].tolist(), range(len(start[k]["id"]))))
        idx = np.array([pos[i] for i in got["id"].tolist()], dtype=np.int64)
        for c, arr in zip(("x", "y", "z", "vx", "vy", "vz"), x64):
            a = got[c].astype(np.float64)
            b = arr[idx]
            scale = max(1.0, float(np.max(np.abs(b)))) if c in "xyz" else float(np.max(np.abs(b))) + 1.0
            assert np.max(np.abs(a - b)) <= 1e-5 * scale, c
    d = sim.diagnostics()
    assert d["ion_impacts"] == len(impacts)
    acc = sim.face_accumulators()
    ref_Eb = np.zeros(g.nface, np.int64)
    for f, E_i, w in impacts:
        ref_Eb[f] += int(math.floor(w * cfg["w_min"] * E_i * 2.0 ** 20))
    assert np.array_equal(acc["Eb"], ref_Eb)
    sim.close()


def test_deposit_bit_exact_and_conserving(pic):
    cfg, g, sim, pop, phi = _pushed_case(pic)
    sim.deposit()
    ref = sorted_pop(g, pop)
    Q = P.deposit(g, ref["i"], 1, Q=P.deposit(g, ref["e"], -1))
    got = sim.get_charge()
    assert np.array_equal(got, Q)
    assert int(got.sum()) == (int(ref["i"]["w"].sum()) - int(ref["e"]["w"].sum())) << 30
    sim.close()


def test_collisions_match_oracle(pic):
    # energetic electrons mixed with the neutrals (impact ionization) and a strong applied
    # field (field ionization near the apex); w_min = 1 raises the per-pair probabilities
    n_sp = 30000
    cfg = small_cfg(n_sp=n_sp, w_min=1.0)
    g = grid_of(cfg)
    V0 = 420.0
    sim = make(pic, cfg, V0=V0)
    pop = synth.plasma(cfg, seed=5)
    rng = np.random.default_rng(6)
    ne = len(pop["e"]["x"])
    src = rng.integers(0, len(pop["n"]["x"]), ne)
    for c in ("x", "y", "z"):
        pop["e"][c] = pop["n"][c][src].copy()             # electrons on neutral positions
    speed = np.sqrt(2 * rng.uniform(20.0, 300.0, ne) * OC.E_CHARGE / OC.M_E)
    u = rng.normal(size=(ne, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    for a, c in enumerate(("vx", "vy", "vz")):
        pop["e"][c] = (speed * u[:, a]).astype(np.float32)
    phi = fixed_phi(field.solve_poisson(g, V0))
    sim.set_potential(phi)
    load(sim, pop)
    sim.set_clock(3, n_sp)
    E = field.efield(g, phi)
    st = sorted_pop(g, pop)
    offs = {k: P.stable_sort(g, st[k])[1] for k in "eni"}
    prm = {"dt": cfg["dt"], "seed": cfg["seed"], "w_min": cfg["w_min"]}
    ids = collide.Counter(cfg["n_sp"])
    ni, ne, ev = collide.impact_ionization(g, prm, st["e"], offs["e"], st["n"], offs["n"], 3, ids)
    ni2, ne2, ev2 = collide.field_ionization(g, prm, st["n"], E, 3, ids)
    ref = {"e": P.concat(P.concat(st["e"], ne), ne2), "n": st["n"], "i": P.concat(P.concat(st["i"], ni), ni2)}
    sim.collide()
    d = sim.diagnostics()
    assert ev > 20 and ev2 > 20, (ev, ev2)
    assert d["impact_ionizations"] == ev and d["field_ionizations"] == ev2
    assert d["next_id"] == ids.next_id
    for s, (k, _, _) in enumerate(SPECIES):
        got = sim.get_particles(s)
        assert_sp_equal(got, ref[k], fields=("x", "y", "z", "w", "id"))
        for c in ("vx", "vy", "vz"):
            a, b = got[c].astype(np.float64), ref[k][c].astype(np.float64)
            assert np.all(np.abs(a - b) <= 1e-6 * (np.abs(b) + 1.0)), (k, c)
    sim.close()


def test_emission_integral_matches_oracle(pic):
    cfg = small_cfg()
    sim = make(pic, cfg, cap=16, V0=10.0)
    F, T, W, R = synth.face_tuples(400, seed=7)
    R = np.where(np.arange(400) % 5 == 0, -1.0, R)          # some flat faces
    J, PN = sim.emission_eval(F * 1e9, T, W, np.where(R > 0, R * 1e-9, -1.0))
    Jr, Pr = em.current_density_fixed(F, T, W, np.where(R > 0, R, np.inf))
    assert np.all(np.isfinite(J)) and np.all(np.isfinite(PN)), np.nonzero(~(np.isfinite(J) & np.isfinite(PN)))
    ok = Jr > 1e-200
    bad = np.nonzero(ok & ~(np.abs(J / np.where(ok, Jr, 1.0) - 1) <= 1e-8))[0]
    assert len(bad) == 0, (bad[:5], F[bad[:5]], T[bad[:5]], W[bad[:5]], R[bad[:5]], J[bad[:5]], Jr[bad[:5]])
    tol = 1e-6 * (np.abs(Pr) + np.abs(Jr) * 1.0) + 1e-30
    bad = np.nonzero(~(np.abs(PN - Pr) <= tol))[0]
    assert len(bad) == 0, (bad[:5], F[bad[:5]], T[bad[:5]], W[bad[:5]], R[bad[:5]], PN[bad[:5]], Pr[bad[:5]])
    sim.close()


def test_fast_integral_matches_oracle(pic):
    """FP32 Gamow quadrature (PIC_F_FAST_INTEGRAL): J and P_N within 1e-4 relative of the oracle's
    FP64 integral wherever J is above 1e-5 A/m^2, and log10 J within 1e-3 everywhere it is finite."""
    cfg = small_cfg()
    sim = make(pic, cfg, cap=16, V0=10.0, flags=pic.F_ALL | pic.F_FAST_INTEGRAL)
    F, T, W, R = synth.face_tuples(400, seed=8)
    F = np.concatenate([F, np.full(40, 0.5), np.full(40, 14.0)])            # low and near-top fields
    T = np.concatenate([T, np.linspace(300, 4000, 40), np.linspace(300, 4000, 40)])
    W = np.concatenate([W, np.full(80, 4.5)])
    R = np.concatenate([R, np.full(80, 5.0)])
    R = np.where(np.arange(R.size) % 5 == 0, -1.0, R)
    J, PN = sim.emission_eval(F * 1e9, T, W, np.where(R > 0, R * 1e-9, -1.0))
    Jr, Pr = em.current_density_fixed(F, T, W, np.where(R > 0, R, np.inf))
    assert np.all(np.isfinite(J)) and np.all(np.isfinite(PN))
    rel = Jr > 1e-5
    assert rel.sum() > 100
    assert np.max(np.abs(J[rel] / Jr[rel] - 1)) <= 1e-4
    assert np.max(np.abs(PN[rel] - Pr[rel]) / (np.abs(Pr[rel]) + 0.05 * Jr[rel])) <= 1e-4
    tiny = (Jr > 1e-250) & ~rel
    assert np.max(np.abs(np.log10(J[tiny]) - np.log10(Jr[tiny]))) <= 1e-3
    sim.close()


def _emit_case(pic, T_tip):
    cfg = small_cfg(nx=16, ny=16, nz=32, tip_radius=2e-9, tip_height=10e-9, n_sp=3000, apex_field=9e9)
    g = grid_of(cfg)
    V0 = field.calibrate_V0(g, cfg["apex_field"])
    sim = make(pic, cfg, V0=V0)
    pop = synth.plasma(cfg, seed=8)
    phi = fixed_phi(field.solve_poisson(g, V0))
    sim.set_potential(phi)
    load(sim, pop)
    sim.set_clock(7, cfg["n_sp"])
    T = np.full(int(g.solid.sum()), T_tip)
    sim.set_temperature(T)
    prm = dict(cfg, V0=V0, step0=7, next_id=cfg["n_sp"])
    st = OS.State(g, prm, pop, phi, T=T)
    return cfg, g, sim, st


def test_emission_and_injection_match_oracle(pic):
    cfg, g, sim, st = _emit_case(pic, 3300.0)
    # a big evaporation accumulator on every face: injection happens this step
    acc = sim.face_accumulators()
    rng = np.random.default_rng(1)
    acc["evap"] = 1.0 + 0.05 * rng.random(g.nface)
    # and sputtered atoms waiting on a tenth of the faces (fractional SP weights drain them)
    atoms = np.where(rng.random(g.nface) < 0.1, rng.uniform(1.0, 1.6, g.nface), 0.0)
    acc["sput"] = np.floor(atoms * 2.0 ** 24).astype(np.int64)
    sim.set_face_accumulators(acc)
    st.acc_evap[:] = acc["evap"]
    st.acc_sput[:] = acc["sput"]
    sim.emit()
    Fv = field.face_field(g, st.phi)
    J, PN = em.current_density_fixed(Fv * 1e-9, OS.face_temperature(st), cfg["work_function"],
                                     OS.face_radius_nm(g, st.prm))
    F_got, J_got, P_got = sim.face_emission()
    assert np.array_equal(F_got, Fv)
    ok = J > 1e-200
    bad = np.nonzero(ok & ~(np.abs(J_got / np.where(ok, J, 1.0) - 1) <= 1e-8))[0]
    assert len(bad) == 0, (bad[:5], Fv[bad[:5]], J_got[bad[:5]], J[bad[:5]])
    N, new_e = OS.emit(st, J)
    st.acc_heat += PN * g.dx * g.dx * cfg["dt"]
    new_ev, new_sp = OS.inject(st)
    assert new_e["id"].size + new_ev["id"].size > 0
    ref_e = P.concat(st.sp["e"], new_e)
    ref_n = P.concat(P.concat(st.sp["n"], new_ev), new_sp)
    got_e = sim.get_particles(0)
    got_n = sim.get_particles(1)
    assert_sp_equal(got_e, ref_e)
    assert_sp_equal(got_n, ref_n, fields=("x", "y", "z", "w", "id"))
    for c in ("vx", "vy", "vz"):
        assert np.allclose(got_n[c], ref_n[c], rtol=1e-6, atol=1e-3)
    acc = sim.face_accumulators()
    assert np.allclose(acc["evap"], st.acc_evap, rtol=1e-12, atol=1e-12)
    assert np.array_equal(acc["sput"], st.acc_sput)
    assert new_sp["id"].size > 0
    assert np.allclose(acc["heat"], st.acc_heat, rtol=1e-6, atol=1e-30)
    sim.close()


def test_poisson_with_charge_matches_oracle(pic):
    for mixed in (True, False):
        cfg, g, sim, pop, phi = _pushed_case(pic, n_sp=20000, seed=9)
        sim.close()
        sim = make(pic, cfg, V0=60.0, mg_tol=1e-10,
                   flags=pic.F_ALL if mixed else pic.F_ALL & ~pic.F_MIXED_MG)
        load(sim, pop)
        sim.solve_field()
        ref = sorted_pop(g, pop)
        Q = P.deposit(g, ref["i"], 1, Q=P.deposit(g, ref["e"], -1))
        phi_ref = field.solve_poisson(g, 60.0, field.rhs_from_charge(g, Q, cfg["w_min"]))
        got = sim.get_potential()
        scale = np.max(np.abs(phi_ref))
        assert np.max(np.abs(got - phi_ref)) <= 1e-8 * scale
        d = sim.diagnostics()
        assert d["mg_residual"] <= 1e-10
        assert field.relative_residual(g, got, field.rhs_from_charge(g, Q, cfg["w_min"]), 60.0) <= 2e-10
        sim.close()


def test_heat_step_matches_oracle(pic):
    cfg = small_cfg(n_heat=1000)
    g = grid_of(cfg)
    sim = make(pic, cfg, cap=16, V0=50.0)
    rng = np.random.default_rng(3)
    T = 300.0 + 2000.0 * rng.random(sim.nsolid)
    sim.set_temperature(T)
    acc = sim.face_accumulators()
    tip = g.face_owner >= 0
    acc["heat"] = np.where(tip, rng.normal(0, 1e-16, g.nface), 0.0)
    acc["charge"] = np.where(tip, np.abs(rng.normal(0, 1e-21, g.nface)), 0.0)
    acc["Eb"] = np.where(tip, rng.integers(0, 1 << 30, g.nface), 0).astype(np.int64)
    acc["Es"] = np.where(tip, rng.integers(0, 1 << 28, g.nface), 0).astype(np.int64)
    sim.set_face_accumulators(acc)
    sim.heat()
    dth = cfg["dt"] * cfg["n_heat"]
    Eb = (acc["Eb"] - acc["Es"]).astype(np.float64) * 2.0 ** -20 * OC.E_CHARGE
    Tn, _ = heat.heat_step(g, T, (acc["heat"] + Eb) / dth, acc["charge"] / dth, dth, cfg["T0"])
    assert np.max(np.abs(sim.get_temperature() - Tn) / Tn) <= 1e-9
    acc2 = sim.face_accumulators()
    assert np.all(acc2["heat"] == 0) and np.all(acc2["Eb"] == 0)
    sim.close()


def test_full_steps_keep_the_books(pic):
    cfg = small_cfg(n_sp=20000, n_heat=3)
    g = grid_of(cfg)
    sim = make(pic, cfg, V0=0.0)
    pop = synth.plasma(cfg, seed=11)
    load(sim, pop)
    sim.set_clock(0, cfg["n_sp"])
    sim.solve_field()
    for _ in range(4):
        d0 = sim.diagnostics()
        sim.step(1)
        d = sim.diagnostics()
        created = d["next_id"] - d0["next_id"]
        removed = sum(d["removed"])
        zero_w = int((sim.get_particles(1)["w"] == 0).sum())
        assert sum(d["count"]) <= sum(d0["count"]) + created - removed + zero_w
        ids = np.concatenate([sim.get_particles(s)["id"] for s in range(3)])
        assert len(np.unique(ids)) == len(ids)
        for s in range(3):
            sp_ = sim.get_particles(s)
            c = P.cell_keys(g, sp_)
            assert np.all(~g.solid.ravel()[c])
        assert d["total_charge_fixed"] == (d["weight"][2] - d["weight"][0]) << 30
    assert d["step"] == 4
    sim.close()


def test_poisson_on_a_grid_above_the_cluster_tail_matches_oracle(pic):
    """A grid whose finest multigrid levels run as separate launches above the cluster-launched
    tail (65x65x129 nodes): the mixed-precision refinement reaches mg_tol = 1e-10 and matches the
    oracle's CG solution to 1e-8 of its scale."""
    cfg = small_cfg(nx=64, ny=64, nz=128, tip_radius=4e-9, tip_height=40e-9, n_sp=100_000)
    g = grid_of(cfg)
    pop = synth.plasma(cfg, seed=12)
    sim = make(pic, cfg, cap=400_000, V0=60.0, mg_tol=1e-10, mg_max_cycles=200)
    load(sim, pop)
    sim.solve_field()
    ref = sorted_pop(g, pop)
    Q = P.deposit(g, ref["i"], 1, Q=P.deposit(g, ref["e"], -1))
    assert np.array_equal(sim.get_charge(), Q)
    f = field.rhs_from_charge(g, Q, cfg["w_min"])
    phi_ref = field.solve_poisson(g, 60.0, f)
    got = sim.get_potential()
    assert np.max(np.abs(got - phi_ref)) <= 1e-8 * np.max(np.abs(phi_ref))
    d = sim.diagnostics()
    assert d["mg_residual"] <= 1e-10
    assert field.relative_residual(g, got, f, 60.0) <= 2e-10
    sim.close()
