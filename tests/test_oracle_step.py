"""Invariants of one full oracle step (counts, ids, charge, positions) on a small instance."""
import numpy as np
import pytest

from oracle import field, particles as P, step as S
from oracle.grid import Grid
from paper_2402_08404_gb300 import synth

CFG = dict(nx=16, ny=16, nz=32, dx=1e-9, tip_radius=2e-9, tip_height=10e-9, apex_field=8e9,
           n_sp=3000, dt=5e-17, T0=2900.0, work_function=4.5, w_min=0.01, w_max_units=1024,
           n_heat=2, seed=5)


@pytest.mark.slow
def test_two_steps_keep_the_books():
    g = Grid(CFG["nx"], CFG["ny"], CFG["nz"], CFG["dx"], CFG["tip_radius"], CFG["tip_height"])
    V0 = field.calibrate_V0(g, CFG["apex_field"])
    prm = dict(CFG, V0=V0, next_id=CFG["n_sp"])
    pop = synth.plasma(CFG, seed=2)
    phi = field.solve_poisson(g, V0)
    st = S.State(g, prm, pop, phi)
    for _ in range(2):
        before = {k: P.count(v) for k, v in st.sp.items()}
        id0 = st.next_id
        S.step(st)
        created = st.next_id - id0
        after = {k: P.count(v) for k, v in st.sp.items()}
        removed = sum(st.count["removed_" + k] for k in "eni")
        # neutrals fully ionized leave with w = 0 and are dropped at the next sort
        zero_w = int((st.sp["n"]["w"] == 0).sum())
        dropped_zero = sum(after.values()) - (sum(before.values()) + created - removed)
        assert dropped_zero <= 0 and -dropped_zero <= zero_w + before["n"]
        ids = np.concatenate([st.sp[k]["id"] for k in "eni"])
        assert len(np.unique(ids)) == len(ids)
        for k in "eni":
            sp_ = st.sp[k]
            c = P.cell_keys(g, sp_)
            assert np.all(~g.solid.ravel()[c])
        Qsum = int(st.Q.sum())
        assert Qsum == (int(st.sp["i"]["w"].sum()) - int(st.sp["e"]["w"].sum())) << 30
    # heat ran (n_heat = 2): the tip temperature changed and stays physical
    assert np.all(np.isfinite(st.T)) and np.any(st.T != CFG["T0"])
    # hot tip (2900 K) evaporates
    assert st.count["evaporated"] >= 0 and np.any(st.acc_evap > 0)
