"""Parity of the RC circuit and the Shockley-Ramo gap current (circuit passage of Sec. 2.3.1)
with the oracle, through the C ABI.

Bars.  I_gap: the library gathers E0 in float32 (E0 itself stored as float32) and forms v . E0
in float32, then sums in float64; a handful of roundings of 2^-24 per term bound the error by
4e-6 x sum_i |q_i| sum_c |v_c| <|E0_c|>_i (the cloud-in-cell average of |E0_c|), the bound the
test computes from the oracle's values.  V_gap: explicit Euler with the oracle's I_gap, so
|dV_n| <= sum_m (dt/C)|dI_m| + the float64 roundings of the update.  Potential with the anode at
V_gap: 1e-8 of the solution's scale, as for the Poisson solve without a circuit.
"""
import numpy as np
import pytest

from oracle import circuit as OC_, field, particles as P
from oracle import constants as OC
from paper_2402_08404_gb300 import synth

from _util import SPECIES, fixed_phi, grid_of, oracle_push_sort, small_cfg

pytestmark = pytest.mark.gpu

R_, C_ = 1e3, 1e-12   # the paper's circuit: 1 kOhm, 1 pF


@pytest.fixture(scope="module")
def pic():
    import os
    from paper_2402_08404_gb300 import _build
    if not os.path.exists(_build.LIB):
        _build.build()
    from paper_2402_08404_gb300 import pic as m
    return m


def _case(pic, n_sp=20000, seed=4, V0=60.0, flags=None):
    cfg = small_cfg(n_sp=n_sp, circuit_R=R_, circuit_C=C_)
    g = grid_of(cfg)
    f = pic.F_CIRCUIT if flags is None else flags
    sim = pic.Pic(cfg, capacity=200_000, V0=V0, flags=f, mg_tol=1e-11, mg_max_cycles=80)
    pop = synth.plasma(cfg, seed=seed)
    phi = fixed_phi(field.solve_poisson(g, V0) + synth.potential_noise((g.nz + 1, g.ny + 1, g.nx + 1), 0.2, seed=seed))
    sim.set_potential(phi)
    for s, (k, _, _) in enumerate(SPECIES):
        sim.load_particles(s, pop[k])
    sim.set_clock(0, n_sp)
    return cfg, g, sim, pop, phi


def _oracle_pushed(cfg, g, pop, phi):
    """The oracle's pushed SPs of e- and Cu+ that are still in the domain (from cell-sorted
    start states, as the library holds them after a load)."""
    E = field.efield(g, phi)
    dtdx = np.float32(cfg["dt"] / cfg["dx"])
    out = []
    for k, Z, m in SPECIES:
        if Z == 0:
            continue
        sp_, _ = P.stable_sort(g, {f: np.asarray(v).astype(P.DTYPES[f]) for f, v in pop[k].items()})
        new = P.push_f32(sp_, E, P.kick_factor(Z, m, cfg["dt"]), dtdx)
        alive, _ = P.boundary(g, sp_, new, k == "i", m)
        moved = {c: v.astype(np.float32)[alive] for c, v in zip(("x", "y", "z", "vx", "vy", "vz"), new)}
        moved["w"] = sp_["w"][alive]
        out.append((Z, moved))
    return out


def _bound(E0, species, w_min):
    """sum_i |q_i| sum_c |v_c| <|E0_c|>_i: the scale of the float32 rounding of I_gap."""
    tot = 0.0
    A = np.abs(E0)
    for Z, sp_ in species:
        a = OC_.gather64(A, sp_["x"], sp_["y"], sp_["z"])
        v = np.abs(np.stack([sp_[c].astype(np.float64) for c in ("vx", "vy", "vz")], 1))
        q = abs(Z) * OC.E_CHARGE * sp_["w"].astype(np.float64) * w_min
        tot += float(np.sum(q * np.sum(v * a, axis=1)))
    return tot


def test_gap_current_and_circuit_update_match_oracle(pic):
    cfg, g, sim, pop, phi = _case(pic)
    E0 = OC_.unit_field(g)
    species = _oracle_pushed(cfg, g, pop, phi)
    I_ref = OC_.gap_current(E0, species, cfg["w_min"])
    tol = 4e-6 * _bound(E0, species, cfg["w_min"])
    assert abs(I_ref) > 100 * tol            # the sum is not lost to cancellation
    sim.push()
    sim.circuit()
    d = sim.diagnostics()
    assert abs(d["I_gap"] - I_ref) <= tol, (d["I_gap"], I_ref, tol)
    # the first update starts from V_gap = V0: no circuit current, and the gap voltage falls by
    # dt/C I_gap
    V1, It = OC_.circuit_step(60.0, I_ref, 60.0, R_, C_, cfg["dt"])
    assert d["I_tot"] == 0.0 and It == 0.0
    assert abs(d["V_gap"] - V1) <= cfg["dt"] / C_ * tol + 4e-16 * 60.0
    assert d["V_gap"] < 60.0
    sim.close()


def test_anode_follows_gap_voltage(pic):
    """Repeated circuit updates from the same pushed SPs follow the Euler recursion; the next
    Poisson solve holds the anode plane at V_gap and matches the oracle's solve at that anode
    potential."""
    cfg, g, sim, pop, phi = _case(pic, seed=6)
    E0 = OC_.unit_field(g)
    species = _oracle_pushed(cfg, g, pop, phi)
    I_ref = OC_.gap_current(E0, species, cfg["w_min"])
    tol = 4e-6 * _bound(E0, species, cfg["w_min"])
    sim.push()
    V, bound = 60.0, 0.0
    for n in range(5):
        sim.circuit()
        V, It = OC_.circuit_step(V, I_ref, 60.0, R_, C_, cfg["dt"])
        bound += cfg["dt"] / C_ * (1 + cfg["dt"] / (R_ * C_)) ** n * tol + 4e-16 * 60.0
        d = sim.diagnostics()
        assert abs(d["V_gap"] - V) <= bound, (n, d["V_gap"], V, bound)
        assert d["I_tot"] == pytest.approx(It, rel=1e-6, abs=1e-6 * abs(I_ref))
    Vg = d["V_gap"]
    sim.sort()
    sim.deposit()
    sim.solve_field()
    got = sim.get_potential()
    top = got[-1]
    assert np.all(top == fixed_phi(np.full(top.shape, Vg)))
    # oracle: the same alive SPs, sorted and deposited, solved with the anode at V_gap
    ref, _, _ = oracle_push_sort(g, {k: P.stable_sort(g, {f: np.asarray(v).astype(P.DTYPES[f])
                                                          for f, v in pop[k].items()})[0]
                                     for k, _, _ in SPECIES}, field.efield(g, phi), cfg["dt"])
    Q = P.deposit(g, ref["i"], 1, Q=P.deposit(g, ref["e"], -1))
    assert np.array_equal(sim.get_charge(), Q)
    phi_ref = field.solve_poisson(g, Vg, field.rhs_from_charge(g, Q, cfg["w_min"]))
    assert np.max(np.abs(got - phi_ref)) <= 1e-8 * np.max(np.abs(phi_ref))
    sim.close()


def test_circuit_flag_and_errors(pic):
    cfg = small_cfg(n_sp=100)
    sim = pic.Pic(cfg, capacity=1000, V0=60.0, flags=pic.F_ALL)
    with pytest.raises(RuntimeError):
        sim.circuit()                         # created without R and C
    assert sim.diagnostics()["V_gap"] == 60.0
    sim.close()
    cfg, g, sim, pop, phi = _case(pic, n_sp=2000, flags=pic.F_ALL & ~pic.F_SURROGATE & ~pic.F_CIRCUIT)
    with pytest.raises(RuntimeError):
        sim.circuit()                         # R and C given, circuit switched off
    sim.close()


def _steps(pic, flags, calls, seed=8):
    cfg = small_cfg(n_sp=20000, n_heat=3, circuit_R=R_, circuit_C=C_)
    pop = synth.plasma(cfg, seed=seed)
    sim = pic.Pic(cfg, capacity=200_000, flags=flags, mg_tol=1e-10)
    for s, (k, _, _) in enumerate(SPECIES):
        sim.load_particles(s, pop[k])
    sim.set_clock(0, cfg["n_sp"])
    sim.solve_field()
    V0 = sim.diagnostics()["V0"]
    diags = []
    for n in calls:
        sim.step(n)
        diags.append(sim.diagnostics())
    out = {"sp": [sim.get_particles(s) for s in range(3)], "phi": sim.get_potential(), "diag": diags, "V0": V0,
           "dt": cfg["dt"]}
    sim.close()
    return out


def test_steps_with_circuit_graph_equals_eager(pic):
    """pic_step with the circuit: the graph form replays the eager form bit for bit (the gap
    voltage is device state read by the solve), every step's update follows the Euler
    recursion, and the anode plane holds the last V_gap."""
    base = (pic.F_ALL & ~pic.F_SURROGATE) | pic.F_CIRCUIT
    calls = (1, 1, 1, 2)
    ref = _steps(pic, base, calls)
    got = _steps(pic, base | pic.F_GRAPH, calls)
    for s in range(3):
        for f in ("x", "y", "z", "vx", "vy", "vz", "w", "id"):
            assert np.array_equal(ref["sp"][s][f], got["sp"][s][f]), (s, f)
    assert np.array_equal(ref["phi"], got["phi"])
    for a, b in zip(ref["diag"], got["diag"]):
        for k in ("V_gap", "I_gap", "I_tot", "step", "count"):
            assert a[k] == b[k], k
    V0, dt = ref["V0"], ref["dt"]
    Vp = V0
    for d in ref["diag"][:3]:                # one step per call: V_n = V_{n-1} + dt/C (I_tot - I_gap)
        assert d["I_tot"] == pytest.approx((V0 - Vp) / R_, rel=1e-12, abs=1e-18)
        assert d["V_gap"] == pytest.approx(Vp + dt / C_ * (d["I_tot"] - d["I_gap"]), rel=1e-14)
        Vp = d["V_gap"]
    assert ref["diag"][-1]["V_gap"] < V0
    assert np.all(ref["phi"][-1] == fixed_phi(np.full(ref["phi"][-1].shape, ref["diag"][-1]["V_gap"])))
