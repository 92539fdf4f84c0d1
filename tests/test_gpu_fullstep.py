"""One full step with every process (emission, injection, push, circuit, sort, merging, impact
ionization, elastic and exchange passes, Coulomb passes, field ionization, deposit, solve) on
the GPU against the oracle's step from the same state.

The library deposits the step's charge inside the push and lets merging move the charge of its
pairs; the oracle deposits after the collisions.  Both must give the same int64 node charge bit
for bit (ionization puts its ion and electron on one point with one weight, splitting keeps
positions and weight sums, the elastic, exchange and Coulomb passes turn velocities only).  The
SPs' positions, weights and ids are bit-exact, their velocities within 1e-6 of the species'
largest speed (the collision products are FP64 rotations and FP32 turns).
"""
import numpy as np
import pytest

from oracle import field, step as OS
from oracle.grid import Grid

from _util import SPECIES, assert_sp_equal, colocated_population

pytestmark = pytest.mark.gpu

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


def test_full_step_with_every_process_matches_the_oracle(pic):
    g = Grid(CFG["nx"], CFG["ny"], CFG["nz"], CFG["dx"], CFG["tip_radius"], CFG["tip_height"])
    V0 = field.calibrate_V0(g, CFG["apex_field"])
    phi = np.round(field.solve_poisson(g, V0) * 2.0 ** 40) / 2.0 ** 40
    pop = colocated_population(CFG, seed=8)     # electrons and ions on neutrals: ionizations happen
    flags = ((pic.F_ALL & ~pic.F_SURROGATE & ~pic.F_HEAT) | pic.F_ELASTIC | pic.F_COULOMB | pic.F_MERGE |
             pic.F_CIRCUIT)
    sim = pic.Pic(CFG, capacity=100_000, flags=flags, V0=V0, mg_tol=1e-11, mg_max_cycles=100)
    sim.set_potential(phi)
    for s, (k, _, _) in enumerate(SPECIES):
        sim.load_particles(s, pop[k])
    sim.set_clock(0, CFG["n_sp"])
    prm = dict(CFG, V0=V0, next_id=CFG["n_sp"], elastic=True, coulomb=True)
    st = OS.State(g, prm, pop, phi)
    OS.step(st)
    sim.step(1)
    d = sim.diagnostics()
    for k in ("impact_ionizations", "field_ionizations", "elastic_en", "elastic_nn", "charge_exchanges",
              "coulomb_ee", "coulomb_ei", "coulomb_ii", "merged", "emitted", "evaporated"):
        assert d[k] == st.count.get(k, 0), (k, d[k], st.count.get(k))
    assert d["merged"] > 0 and d["impact_ionizations"] + d["elastic_en"] + d["charge_exchanges"] > 0
    assert d["next_id"] == st.next_id
    for s, (k, _, _) in enumerate(SPECIES):
        got = sim.get_particles(s)
        assert_sp_equal(got, st.sp[k], fields=("x", "y", "z", "w", "id"))
        vmax = max(np.abs(st.sp[k][c]).max() for c in ("vx", "vy", "vz")) if len(got["id"]) else 0.0
        for c in ("vx", "vy", "vz"):
            assert np.max(np.abs(got[c].astype(np.float64) - st.sp[k][c]), initial=0.0) <= 1e-6 * vmax + 1.0, (k, c)
    # the charge of the step, deposited by the push and moved by merging, equals the oracle's
    # deposit after the collisions, node by node
    assert np.array_equal(sim.get_charge().ravel(), st.Q.ravel().astype(np.int64))
    sim.close()
