"""Pins of the RC circuit and the Shockley-Ramo gap current in the oracle (CPU only)."""
import math

import numpy as np

from oracle import circuit, constants as OC
from oracle.grid import Grid


def _plates(nx=8, ny=8, nz=16, dx=1e-9):
    return Grid(nx, ny, nz, dx, 0.0, 0.0)     # no tip: a parallel-plate gap


def test_unit_field_of_plates_is_uniform():
    g = _plates()
    E0 = circuit.unit_field(g)
    L = g.nz * g.dx
    assert np.allclose(E0[..., 2], -1.0 / L, rtol=1e-10, atol=0)
    assert np.allclose(E0[..., :2], 0.0, atol=1e-6 / L)


def test_ramo_current_between_plates():
    """Plates: E0 = -z/L, so I = -q v_z / L for any position; an electron (q = -e) drifting to the
    anode induces +e v_z / L, and the charge it induces crossing the whole gap is its own."""
    g = _plates()
    E0 = circuit.unit_field(g)
    L = g.nz * g.dx
    rng = np.random.default_rng(3)
    n = 50
    sp_ = {"x": rng.uniform(0, g.nx, n), "y": rng.uniform(0, g.ny, n), "z": rng.uniform(0, g.nz, n),
           "vx": rng.normal(0, 1e5, n), "vy": rng.normal(0, 1e5, n), "vz": rng.normal(0, 1e6, n),
           "w": rng.integers(1, 9, n)}
    w_min = 0.01
    I = circuit.gap_current(E0, [(-1, sp_)], w_min)
    ref = float(np.sum(OC.E_CHARGE * sp_["w"] * w_min * sp_["vz"])) / L
    assert I == np.float64(I) and abs(I - ref) <= 1e-10 * abs(ref)
    # one electron crossing the gap at constant speed: integral of I dt = e
    one = {"x": np.array([4.2]), "y": np.array([3.3]), "z": np.array([0.0]), "vx": np.zeros(1), "vy": np.zeros(1),
           "vz": np.array([2e6]), "w": np.array([1])}
    t_cross = L / 2e6
    Q = circuit.gap_current(E0, [(-1, one)], 1.0) * t_cross
    assert abs(Q - OC.E_CHARGE) <= 1e-12 * OC.E_CHARGE
    # neutrals induce nothing; an ion moving to the cathode induces the same sign as an electron
    assert circuit.gap_current(E0, [(0, sp_)], w_min) == 0.0
    ion = dict(sp_, vz=-sp_["vz"])
    assert abs(circuit.gap_current(E0, [(1, ion)], w_min) - ref) <= 1e-10 * abs(ref)


def test_circuit_euler_converges_to_the_rc_solution():
    """Constant gap current I: V(t) = V0 - I R (1 - exp(-t/RC)); explicit Euler is first order."""
    V0, R, Cg, I = 1000.0, 1e3, 1e-12, 0.05
    T = 3e-9
    errs = []
    for nsteps in (1000, 2000, 4000):
        dt = T / nsteps
        V = V0
        for _ in range(nsteps):
            V, _ = circuit.circuit_step(V, I, V0, R, Cg, dt)
        exact = V0 - I * R * (1 - math.exp(-T / (R * Cg)))
        errs.append(abs(V - exact))
    assert errs[0] < 0.5 and errs[1] < 0.6 * errs[0] and errs[2] < 0.6 * errs[1]
    # steady state: I_tot = I_gap at V = V0 - I R
    V, Itot = V0 - I * R, None
    Vn, Itot = circuit.circuit_step(V, I, V0, R, Cg, 1e-15)
    assert abs(Vn - V) <= 1e-12 * V0 and abs(Itot - I) <= 1e-12 * I
