"""Pins of the oracle's Cu2+ channels (Table colls): Cu + e -> Cu2+ + 3e inside the impact
ionization pass, Cu+ + e -> Cu2+ + 2e, the Coulomb passes with Cu2+, and the step's books with
a fourth species.  The cross sections are Lotz-form stand-ins (the paper's data is not
available): their shape is pinned, their values are parity unpinned against data."""
import math

import numpy as np
import pytest

from oracle import collide, constants as C, coulomb, particles as P, philox, step as OS
from oracle.grid import Grid


def _beam(g, n, w, vz, id0, seed, per_cell=False):
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) * np.array([g.nx, g.ny, g.nz])
    if per_cell:      # SP k in cell k mod ncell (then every cell holds n // ncell or one more)
        c = np.arange(n) % g.ncell
        pos = np.stack([c % g.nx, (c // g.nx) % g.ny, c // (g.nx * g.ny)], 1) + 0.1 + 0.8 * rng.random((n, 3))
    return {"x": pos[:, 0].astype(np.float32), "y": pos[:, 1].astype(np.float32), "z": pos[:, 2].astype(np.float32),
            "vx": np.zeros(n, np.float32), "vy": np.zeros(n, np.float32), "vz": np.full(n, vz, np.float32),
            "w": np.full(n, w, np.int32), "id": np.arange(id0, id0 + n, dtype=np.uint64)}


@pytest.mark.parametrize("fn,xi,a", [(collide.sigma_double, C.XI_CU_EV + C.XI2_CU_EV, collide.LOTZ_A / 10),
                                     (collide.sigma_ion2, C.XI2_CU_EV, collide.LOTZ_A * 10)])
def test_stand_in_cross_sections_have_the_lotz_shape(fn, xi, a):
    # zero up to the threshold; a ln(E/xi)/(E xi) rises to a/(e xi^2) at E = e xi, then falls as ln E / E
    assert fn(xi) == 0.0 and fn(0.9 * xi) == 0.0 and fn(xi * 1.0001) > 0.0
    E = np.linspace(xi * 1.001, 40 * xi, 40001)
    s = fn(E)
    assert E[np.argmax(s)] == pytest.approx(math.e * xi, rel=1e-3)
    assert s.max() == pytest.approx(a / (math.e * xi * xi), rel=1e-6)
    assert fn(1e6 * xi) * 1e6 * xi == pytest.approx(a * math.log(1e6) / xi, rel=1e-12)
    # the double channel is an order of magnitude below single ionization everywhere
    if fn is collide.sigma_double:
        assert np.all(s < 0.1 * collide.sigma_ion(E) + 1e-40)


def _mcc(double, E_beam, we, wn, ne, nn, seed, w_min=2.0, per_cell=False):
    g = Grid(4, 4, 4, 1e-9, 0.0, 0.0)
    v = math.sqrt(2 * E_beam * C.E_CHARGE / C.M_E)
    e, eo = P.stable_sort(g, _beam(g, ne, we, v, 0, seed, per_cell))
    n, no = P.stable_sort(g, _beam(g, nn, wn, 0.0, ne, seed + 1, per_cell))
    n["vz"][:] = 0
    prm = {"dt": 5e-17, "seed": 3 + seed, "w_min": w_min}
    e0, n0 = P.take(e, np.arange(ne)), P.take(n, np.arange(nn))
    ids = collide.Counter(ne + nn)
    out = collide.impact_ionization(g, prm, e, eo, n, no, seed, ids, double=double)
    return g, prm, (e0, eo, n0, no), (e, n), out, ids, v


def _expected(g, eo, no, we, wn, w_min, v, E_beam):
    """Binomial means and variances of single and double ionizations: per sub-particle of the
    projectile, P_T = 1 - exp(-u n_t sigma_T dt) split between the channels as sigma_c/sigma_T."""
    s1, s2 = float(collide.sigma_ion(E_beam)), float(collide.sigma_double(E_beam))
    out = np.zeros(4)
    cnt_e, cnt_n = np.diff(eo), np.diff(no)
    for c in range(g.ncell):
        if cnt_e[c] == 0 or cnt_n[c] == 0:
            continue
        if cnt_e[c] <= cnt_n[c]:      # electrons project: their sub-particles against n_t = N_n W_n
            trials, nt = cnt_e[c] * we, cnt_n[c] * wn * w_min / g.dx ** 3
        else:
            trials, nt = cnt_n[c] * wn, cnt_e[c] * we * w_min / g.dx ** 3
        PT = 1.0 - math.exp(-v * nt * (s1 + s2) * 5e-17)
        for k, p in enumerate((PT * s1 / (s1 + s2), PT * s2 / (s1 + s2))):
            out[2 * k] += trials * p
            out[2 * k + 1] += trials * p * (1 - p)
    return out


def test_double_channel_rates_are_n_sigma_v_per_sub_particle():
    # 200 eV electrons through Cu at P_T ~ 0.05: single and double ionizations per sub-particle in the
    # ratio of the cross sections, their sum 1 - exp(-u n sigma_T dt)
    E_beam = 200.0
    tot = np.zeros(2)
    ex = np.zeros(4)
    for seed in range(4):
        g, prm, (e0, eo, n0, no), (e, n), out, ids, v = _mcc(True, E_beam, 400, 400, 64, 64, seed, w_min=0.1)
        ni, ne_, ev, nj, ne2, ev2 = out
        tot += [int(ni["w"].sum()), int(nj["w"].sum())]
        ex += _expected(g, eo, no, 400, 400, 0.1, v, E_beam)
    assert ex[2] > 100 and ex[0] > 10 * ex[2]
    assert abs(tot[0] - ex[0]) < 4 * math.sqrt(ex[1]) and abs(tot[1] - ex[2]) < 4 * math.sqrt(ex[3])


def test_double_channel_windows_are_disjoint_at_high_probability():
    # P_T close to 1: n1 + n2 never exceeds the projectile's sub-particles and follows P_T; a
    # window for the double channel that overlapped the single one would count sub-particles twice
    E_beam = 300.0
    g, prm, (e0, eo, n0, no), (e, n), out, ids, v = _mcc(True, E_beam, 30, 2000, 64, 128, 5, w_min=1.0,
                                                          per_cell=True)
    ni, ne_, ev, nj, ne2, ev2 = out
    assert ev > 0 and ev2 > 0
    n1, n2 = int(ni["w"].sum()), int(nj["w"].sum())
    assert np.all(np.diff(eo) == 1) and np.all(np.diff(no) == 2)     # every electron projects
    assert n1 + n2 <= int(e0["w"].sum())
    ex = _expected(g, eo, no, 30, 2000, 1.0, v, E_beam)
    assert (ex[0] + ex[2]) > 0.5 * int(e0["w"].sum())
    assert abs((n1 + n2) - (ex[0] + ex[2])) < 4 * math.sqrt(ex[1] + ex[3]) + 1
    assert abs(n2 - ex[2]) < 4 * math.sqrt(ex[3]) + 1


def test_double_ionization_books_and_energy():
    E_beam = 250.0
    g, prm, (e0, eo, n0, no), (e, n), out, ids, v = _mcc(True, E_beam, 6, 9, 300, 200, 7, w_min=3e4)
    ni, ne_, ev, nj, ne2, ev2 = out
    assert ev > 0 and ev2 > 0
    wi, wj = int(ni["w"].sum()), int(nj["w"].sum())
    # Cu + Cu+ + Cu2+ conserved; the electrons gain one per Cu+ and two per Cu2+ (net charge 0)
    assert int(n["w"].sum()) + wi + wj == int(n0["w"].sum())
    assert int(e["w"].sum()) + int(ne_["w"].sum()) + int(ne2["w"].sum()) - int(e0["w"].sum()) == wi + 2 * wj
    assert -(int(e["w"].sum()) + int(ne_["w"].sum()) + int(ne2["w"].sum())) + wi + 2 * wj == -int(e0["w"].sum())
    # ids: the singles' products first, then the doubles', consecutive and unique
    ids1 = np.concatenate([ni["id"], ne_["id"]])
    ids2 = np.concatenate([nj["id"], ne2["id"]])
    assert ids1.max() < ids2.min()
    allid = np.concatenate([ids1, ids2])
    assert len(np.unique(allid)) == len(allid) == ids.next_id - 500
    # each of the three outgoing electrons of a double event carries (E0 - xi1 - xi2)/3 relative to the
    # (resting) neutral
    Ek = 0.5 * C.M_E * (ne2["vx"].astype(np.float64) ** 2 + ne2["vy"] ** 2 + ne2["vz"] ** 2) / C.E_CHARGE
    turned = e["vz"] != np.float32(v)
    Ek_t = 0.5 * C.M_E * (e["vx"][turned].astype(np.float64) ** 2 + e["vy"][turned] ** 2 + e["vz"][turned] ** 2) \
        / C.E_CHARGE
    third = (E_beam - C.XI_CU_EV - C.XI2_CU_EV) / 3.0
    half = (E_beam - C.XI_CU_EV) / 2.0
    for x in np.concatenate([Ek, Ek_t]):
        assert x == pytest.approx(third, rel=1e-5) or x == pytest.approx(half, rel=1e-5)
    assert np.sum(np.isclose(Ek, third, rtol=1e-5)) >= 2 * ev2
    # Cu2+ sit on their neutral with its velocity
    assert np.all(nj["vz"] == 0) and np.all(nj["w"] > 0)


def test_below_the_double_threshold_the_channel_changes_nothing():
    # 25 eV < xi_1 + xi_2: sigma_2 = 0, so the single decisions equal the one-process pass bit for
    # bit and no Cu2+ appears; above it the channel takes draws from single ionization
    a = _mcc(False, 25.0, 20, 30, 120, 90, 2, w_min=1e4)
    b = _mcc(True, 25.0, 20, 30, 120, 90, 2, w_min=1e4)
    assert a[4][2] > 0 and b[4][5] == 0 and len(b[4][3]["w"]) == 0
    for x, y in zip(a[4][:2] + a[3], b[4][:2] + b[3]):
        for k in P.FIELDS:
            assert np.array_equal(x[k], y[k]), k


def _ion_pop(E_beam, we, wi, ne, ni_, seed, w_min):
    g = Grid(4, 4, 4, 1e-9, 0.0, 0.0)
    v = math.sqrt(2 * E_beam * C.E_CHARGE / C.M_E)
    e, eo = P.stable_sort(g, _beam(g, ne, we, v, 0, seed))
    i, io = P.stable_sort(g, _beam(g, ni_, wi, 0.0, ne, seed + 1))
    return g, v, e, eo, i, io, {"dt": 5e-17, "seed": 11 + seed, "w_min": w_min}


def test_ion_ionization_rate_books_and_energy():
    E_beam = 150.0
    total = 0
    mean = var = 0.0
    for seed in range(3):
        g, v, e, eo, i, io, prm = _ion_pop(E_beam, 200, 200, 80, 64, seed, 0.05)
        e0w, i0w = int(e["w"].sum()), int(i["w"].sum())
        ids = collide.Counter(1000)
        nj, ne_, ev = collide.ion_ionization(g, prm, e, eo, i, io, seed, ids)
        wj = int(nj["w"].sum())
        total += wj
        assert int(i["w"].sum()) + wj == i0w                             # Cu+ + Cu2+ conserved
        assert int(e["w"].sum()) + int(ne_["w"].sum()) - e0w == wj        # one electron per Cu2+
        assert ids.next_id - 1000 == len(nj["id"]) + len(ne_["id"])
        Ek = 0.5 * C.M_E * (ne_["vx"].astype(np.float64) ** 2 + ne_["vy"] ** 2 + ne_["vz"] ** 2) / C.E_CHARGE
        assert np.allclose(Ek, 0.5 * (E_beam - C.XI2_CU_EV), rtol=1e-5)
        cnt_e, cnt_i = np.diff(eo), np.diff(io)
        for c in range(g.ncell):
            if cnt_e[c] == 0 or cnt_i[c] == 0:
                continue
            if cnt_e[c] <= cnt_i[c]:
                tr, dens = cnt_e[c] * 200, cnt_i[c] * 200 * prm["w_min"] / g.dx ** 3
            else:
                tr, dens = cnt_i[c] * 200, cnt_e[c] * 200 * prm["w_min"] / g.dx ** 3
            p = -math.expm1(-v * dens * float(collide.sigma_ion2(E_beam)) * prm["dt"])
            mean += tr * p; var += tr * p * (1 - p)
    assert mean > 200
    assert abs(total - mean) < 4 * math.sqrt(var)


def test_coulomb_with_cu2_scales_as_z_squared():
    # <delta^2> carries q_a^2 q_b^2: e-Cu2+ at the same density and speed deflects 4x e-Cu+ in variance
    u, n = 1e6, 1e25
    d1 = coulomb.delta2(-C.E_CHARGE, C.E_CHARGE, C.M_E, C.M_CU, n, 10.0, 5e-17, u)
    d2 = coulomb.delta2(-C.E_CHARGE, 2 * C.E_CHARGE, C.M_E, C.M_CU, n, 10.0, 5e-17, u)
    d3 = coulomb.delta2(2 * C.E_CHARGE, 2 * C.E_CHARGE, C.M_CU, C.M_CU, n, 10.0, 5e-17, u)
    d4 = coulomb.delta2(C.E_CHARGE, C.E_CHARGE, C.M_CU, C.M_CU, n, 10.0, 5e-17, u)
    assert d2 == pytest.approx(4 * d1, rel=1e-14) and d3 == pytest.approx(16 * d4, rel=1e-14)


def test_coulomb_cu2_passes_conserve_momentum_and_energy():
    g = Grid(4, 4, 4, 1e-9, 0.0, 0.0)
    rng = np.random.default_rng(3)

    def pop(nsp, m_scale, id0):
        p = _beam(g, nsp, 1, 0.0, id0, int(rng.integers(1 << 30)))
        for c in ("vx", "vy", "vz"):
            p[c] = (rng.normal(size=nsp) * m_scale).astype(np.float32)
        return P.stable_sort(g, p)

    prm = {"dt": 5e-17, "seed": 2, "w_min": 1e3, "coulomb_log": 10.0}
    i, io = pop(200, 2e3, 0)
    j, jo = pop(150, 2e3, 1000)

    def books(S, m):
        v = np.stack([S["vx"], S["vy"], S["vz"]], 1).astype(np.float64)
        return m * v.sum(0), 0.5 * m * (v ** 2).sum()
    p0 = books(i, C.M_CU)[0] + books(j, C.M_CU)[0]
    k0 = books(i, C.M_CU)[1] + books(j, C.M_CU)[1]
    ev = coulomb.coulomb_ij(g, prm, i, io, j, jo, 0) + coulomb.coulomb_jj(g, prm, j, jo, 0)
    assert ev > 100
    p1 = books(i, C.M_CU)[0] + books(j, C.M_CU)[0]
    k1 = books(i, C.M_CU)[1] + books(j, C.M_CU)[1]
    # equal weights: both members of every pair turn; momentum and energy conserved up to the f32 stores
    assert np.allclose(p1, p0, atol=1e-6 * C.M_CU * 2e3 * 350)
    assert k1 == pytest.approx(k0, rel=1e-5)


def test_step_with_cu2_keeps_the_books():
    # a collision-rich state stepped with every process and the Cu2+ channels: the deposited charge
    # equals sum(Z w) 2^30, Cu2+ appear, and turning the channels off removes every Cu2+ event
    from _util import colocated_population
    cfg = dict(nx=16, ny=16, nz=32, dx=1e-9, tip_radius=2e-9, tip_height=10e-9, apex_field=8e9, n_sp=3000, dt=5e-17,
               T0=2900.0, work_function=4.5, w_min=0.05, w_max_units=1024, n_heat=0, seed=5, merge_max=0,
               coulomb_log=10.0)
    from oracle import field
    g = Grid(cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["tip_radius"], cfg["tip_height"])
    V0 = field.calibrate_V0(g, cfg["apex_field"])
    phi = np.round(field.solve_poisson(g, V0) * 2.0 ** 40) / 2.0 ** 40
    pop = colocated_population(cfg, seed=8)
    for k in ("e",):
        pop[k]["vz"] = pop[k]["vz"] + np.float32(1.2e7)   # ~400 eV electrons: above every threshold
    prm = dict(cfg, V0=V0, next_id=cfg["n_sp"], coulomb=True, ion2=True, w_min=50.0)
    st = OS.State(g, prm, pop, phi)
    OS.step(st)
    assert st.count["double_ionizations"] > 0 and st.count["ion_ionizations"] > 0
    assert len(st.sp["j"]["w"]) > 0
    zw = sum(z * int(st.sp[k]["w"].astype(np.int64).sum()) for k, z in (("e", -1), ("i", 1), ("j", 2)))
    assert int(st.Q.sum()) == zw << 30
    ids = np.concatenate([st.sp[k]["id"] for k in "enij"])
    assert len(np.unique(ids)) == len(ids) and ids.max() < st.next_id
