"""Pins of the oracle's collisions: rotation of eq:du, MCC rate n sigma v, conservation,
ADK rate of eq:dfi against the ADK formula in atomic units."""
import math

import numpy as np
import pytest

from oracle import collide, constants as C, particles as P
from oracle.grid import Grid


def test_rotation_matrix_is_proper_and_maps_the_pole():
    rng = np.random.default_rng(0)
    for _ in range(50):
        th, ph = rng.random() * math.pi, rng.random() * 2 * math.pi
        R = np.stack([collide.rot_inv(th, ph, e) for e in np.eye(3)], 1).T   # R^-1 columns -> R
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-14)
        # R^-1(theta, phi) (0,0,u) is the vector of polar angles (theta, phi): eq:du gives
        # du = 0 for theta' = 0
        v = collide.rot_inv(th, ph, [0, 0, 2.0])
        assert np.allclose(v, 2.0 * np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)]))


def test_scattered_velocity_is_isotropic_with_given_speed():
    rng = np.random.default_rng(1)
    u = np.array([3.0, -1.0, 2.0])
    out = np.array([collide.scatter_velocity(u, 5.0, 2 * rng.random() - 1, 2 * math.pi * rng.random())
                    for _ in range(20000)])
    assert np.allclose(np.linalg.norm(out, axis=1), 5.0)
    assert np.all(np.abs(out.mean(axis=0)) < 5.0 * 4 / math.sqrt(3 * 20000))
    assert np.allclose((out ** 2).mean(axis=0), 25.0 / 3, rtol=0.03)


def test_cross_section_shape():
    xi = C.XI_CU_EV
    assert collide.sigma_ion(xi) == 0.0 and collide.sigma_ion(xi * 0.5) == 0.0
    E = np.linspace(xi * 1.001, 40 * xi, 20001)
    s = collide.sigma_ion(E)
    # a ln(E/xi)/(E xi) peaks at E = e xi with value a/(e xi^2)
    assert E[np.argmax(s)] == pytest.approx(math.e * xi, rel=1e-3)
    assert s.max() == pytest.approx(collide.LOTZ_A / (math.e * xi * xi), rel=1e-6)


def _uniform_cell_population(g, ne, nn, we, wn, v_e, seed):
    rng = np.random.default_rng(seed)
    def sp(n, w, vz, id0):
        pos = rng.random((n, 3)) * np.array([g.nx, g.ny, g.nz])
        return {"x": pos[:, 0].astype(np.float32), "y": pos[:, 1].astype(np.float32),
                "z": pos[:, 2].astype(np.float32), "vx": np.zeros(n, np.float32),
                "vy": np.zeros(n, np.float32), "vz": np.full(n, vz, np.float32),
                "w": np.full(n, w, np.int32), "id": np.arange(id0, id0 + n, dtype=np.uint64)}
    return sp(ne, we, v_e, 0), sp(nn, wn, 0.0, ne)


def test_ionization_rate_equals_n_sigma_v():
    # an electron beam through a uniform neutral background: ionizations per step must be
    # n sigma(v) v dt per electron (sub-particles counted), within 3 sigma binomial
    g = Grid(4, 4, 4, 1e-9, 0.0, 0.0)
    E_beam = 60.0
    v = math.sqrt(2 * E_beam * C.E_CHARGE / C.M_E)
    wn, we = 5, 3
    prm = {"dt": 5e-17, "seed": 9, "w_min": 2.0}
    total, expected, var = 0, 0.0, 0.0
    for step in range(6):
        e, n = _uniform_cell_population(g, 256, 640, we, wn, v, step)
        e, eo = P.stable_sort(g, e)
        n, no = P.stable_sort(g, n)
        ids = collide.Counter(10_000)
        _, ne_, _ = collide.impact_ionization(g, prm, e, eo, n, no, step, ids)
        # ionized real neutrals (units of w_min) = weight lost by the neutral background
        total += wn * 640 - int(n["w"].sum())
        cnt_n = np.diff(no)
        cnt_e = np.diff(eo)
        for c in range(g.ncell):
            if cnt_e[c] == 0 or cnt_n[c] == 0:
                continue
            n_real = cnt_n[c] * wn * prm["w_min"] / g.dx ** 3
            if cnt_e[c] <= cnt_n[c]:
                p = 1 - math.exp(-v * n_real * float(collide.sigma_ion(E_beam)) * prm["dt"])
                trials = cnt_e[c] * we
            else:
                ne_real = cnt_e[c] * we * prm["w_min"] / g.dx ** 3
                p = 1 - math.exp(-v * ne_real * float(collide.sigma_ion(E_beam)) * prm["dt"])
                trials = cnt_n[c] * wn
            expected += trials * p
            var += trials * p * (1 - p)
    assert expected > 200
    assert abs(total - expected) < 3 * math.sqrt(var)


def test_ionization_conserves_charge_and_heavy_weight():
    g = Grid(4, 4, 4, 1e-9, 0.0, 0.0)
    v = math.sqrt(2 * 80.0 * C.E_CHARGE / C.M_E)
    e, n = _uniform_cell_population(g, 300, 200, 4, 6, v, 3)
    e, eo = P.stable_sort(g, e)
    n, no = P.stable_sort(g, n)
    e0w, n0w = int(e["w"].sum()), int(n["w"].sum())
    ids = collide.Counter(500)
    ni, ne_, ev = collide.impact_ionization(g, {"dt": 5e-17, "seed": 4, "w_min": 3.0}, e, eo, n, no, 0, ids)
    assert ev > 0
    ions = int(ni["w"].sum())
    # Cu + Cu+ weight conserved; electrons gain exactly what ions gain (net charge 0)
    assert int(n["w"].sum()) + ions == n0w
    assert int(e["w"].sum()) + int(ne_["w"].sum()) - e0w == ions
    # new ids are consecutive and unique
    new_ids = np.concatenate([ni["id"], ne_["id"]])
    assert len(np.unique(new_ids)) == len(new_ids) and new_ids.min() == 500 and ids.next_id == 500 + len(new_ids)
    # energy: both outgoing electrons of an event carry (E0 - xi)/2 relative to the neutral
    sec = ne_["vx"] ** 2 + ne_["vy"] ** 2 + ne_["vz"] ** 2
    Ek = 0.5 * C.M_E * sec.astype(np.float64) / C.E_CHARGE
    assert np.allclose(Ek, 0.5 * (80.0 - C.XI_CU_EV), rtol=1e-5)


def adk_atomic_units(E_GV, Ip_eV, Z=1):
    """ADK tunnelling rate for an s-state (Ammosov, Delone, Krainov 1986) in atomic units:
    w = C^2 Ip (2 (2 Ip)^{3/2}/F)^{2n*-1} exp(-2 (2 Ip)^{3/2}/(3 F)),
    n* = Z/sqrt(2 Ip), C^2 = 2^{2n*}/(n* Gamma(n*+l*+1) Gamma(n*-l*)), l* = n* - 1."""
    hartree = 27.211386245988
    f_au = 514.220674763            # GV/m
    t_au = 2.4188843265857e-2      # fs
    Ip = Ip_eV / hartree
    F = E_GV / f_au
    ns = Z / math.sqrt(2 * Ip)
    C2 = 2 ** (2 * ns) / (ns * math.gamma(2 * ns) * math.gamma(1.0))
    k = (2 * Ip) ** 1.5
    w = C2 * Ip * (2 * k / F) ** (2 * ns - 1) * math.exp(-2 * k / (3 * F))
    return w / t_au


def test_dfi_rate_matches_adk_in_atomic_units():
    # eq:dfi is the ADK rate with its constants rounded to 3 digits: agree to 1 %
    for E in (6.0, 8.0, 10.0, 12.0, 15.0, 20.0, 30.0):
        assert float(collide.adk_rate_per_fs(E)) == pytest.approx(adk_atomic_units(E, C.XI_CU_EV), rel=0.01)
    assert collide.bsi_limit_GV() == pytest.approx(32.21, abs=0.01)


def test_dfi_fraction_and_barrier_suppression():
    g = Grid(4, 4, 4, 1e-9, 0.0, 0.0)
    rng = np.random.default_rng(2)
    n = 4000
    pos = rng.random((n, 3)) * 4
    def neutrals(w):
        return {"x": pos[:, 0].astype(np.float32), "y": pos[:, 1].astype(np.float32), "z": pos[:, 2].astype(np.float32),
                "vx": np.zeros(n, np.float32), "vy": np.zeros(n, np.float32), "vz": np.zeros(n, np.float32),
                "w": np.full(n, w, np.int32), "id": np.arange(n, dtype=np.uint64)}
    E = np.zeros((5, 5, 5, 3), np.float32)
    E[..., 2] = 15e9
    prm = {"dt": 5e-17, "seed": 3}
    nn = neutrals(6)
    ni, ne, ev = collide.field_ionization(g, prm, nn, E, 0, collide.Counter(0))
    p = float(collide.adk_rate_per_fs(15.0)) * 0.05
    got = int(ni["w"].sum())
    exp_ = n * 6 * p
    assert abs(got - exp_) < 3 * math.sqrt(n * 6 * p * (1 - p))
    assert np.array_equal(ni["w"], ne["w"]) and np.all(ne["vx"] == 0)
    # above the barrier-suppression limit every sub-particle ionizes
    E[..., 2] = 40e9
    nn = neutrals(3)
    ni, ne, ev = collide.field_ionization(g, prm, nn, E, 0, collide.Counter(0))
    assert ev == n and int(ni["w"].sum()) == 3 * n and np.all(nn["w"] == 0)
