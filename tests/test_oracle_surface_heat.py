"""Pins of the oracle's surface processes (Sec. 2.3.1-2.3.3), tip heat (eq:heat, eq:cont) and
the surrogate MLP's gradients."""
import math

import numpy as np
import pytest

from oracle import constants as C
from oracle import heat, mlp, surface
from oracle.grid import Grid


def test_evaporation_flux_is_kinetic_flux_at_boiling_point():
    # at T_b the vapour pressure is p_atm and the flux is the kinetic-theory n <v> / 4
    T = C.T_BOIL
    n = C.P_ATM / (C.K_B * T)
    vbar = math.sqrt(8 * C.K_B * T / (math.pi * C.M_CU))
    assert surface.evaporation_flux(T) == pytest.approx(n * vbar / 4, rel=1e-12)


def test_evaporation_obeys_clausius_clapeyron_slope():
    # d ln(phi sqrt(T)) / d(1/T) = -E_vap / k_B
    T1, T2 = 2000.0, 2001.0
    g = lambda T: math.log(float(surface.evaporation_flux(T)) * math.sqrt(T))
    slope = (g(T2) - g(T1)) / (1 / T2 - 1 / T1)
    assert slope == pytest.approx(-C.E_VAP_EV / C.K_B_EV, rel=1e-6)
    assert float(surface.evaporation_flux(300.0)) < 1e-20


def test_injection_weight_rule():
    wmin = 2.0
    # sparse cell, few atoms: the minimum weight
    assert surface.injection_weight_units(1e20, 3, wmin, 1024) == 1
    rng = np.random.default_rng(0)
    for _ in range(200):
        ncell = 10 ** rng.uniform(20, 30)
        N = int(10 ** rng.uniform(0, 6))
        w = surface.injection_weight_units(ncell, N, wmin, 64)
        assert isinstance(w, int) and 1 <= w <= 64
        r = ncell / C.N_MAX * N / wmin
        if w < 64:
            assert (w - 1) ** 2 < max(r, 1.0) <= w * w      # smallest integer with w^2 >= ratio


def test_thompson_energies_follow_truncated_law():
    rng = np.random.default_rng(1)
    prm = surface.SPUTTER
    E = np.array([surface.thompson_energy(u) for u in rng.random(40000)])
    assert E.max() <= prm["E_cap"] and E.min() >= 0
    Fc = (prm["E_cap"] / (prm["E_cap"] + prm["U_s"])) ** 2
    for e in (1.0, 3.43, 10.0, 50.0):
        cdf = (e / (e + prm["U_s"])) ** 2 / Fc
        assert np.mean(E <= e) == pytest.approx(cdf, abs=0.01)


def test_sputter_yield_stand_in():
    assert surface.sputter_yield(20.0) == 0.0 and surface.sputter_yield(25.0) == 0.0
    assert surface.sputter_yield(30.0) > 0.0
    assert surface.sputter_yield(1000.0) == pytest.approx(2.5, rel=0.05)
    ys = [surface.sputter_yield(E) for E in (50, 100, 300, 1000)]
    assert ys == sorted(ys)


def _column_grid(ncells):
    # a single column of solid cells on the axis (nx odd: a cell centre on the axis)
    return Grid(5, 5, ncells + 6, 1.0, 0.4, ncells)


def test_heat_rod_steady_state_is_linear():
    g = _column_grid(10)
    cells, index, pairs, base = heat.voxel_graph(g)
    assert len(cells) == 10 and base.sum() == 1
    T0 = 300.0
    T = np.full(len(cells), T0)
    P = 1e-9                                        # W into the top face
    fh = np.zeros(g.nface)
    top = [f for f in range(g.nface) if g.face_owner[f] == cells[-1] and g.face_dir[f] == 4][0]
    fh[top] = P
    Tn, _ = heat.heat_step(g, T, fh, np.zeros(g.nface), 1e6, T0)   # dt -> infinity: steady state
    kap = float(heat.kappa_of_T(T0))
    z = np.arange(10) + 0.5                          # cell centres above the base plane
    assert np.allclose(Tn, T0 + P * z * g.dx / (kap * g.dx ** 2), rtol=1e-8)


def test_joule_heat_of_uniform_current_and_energy_balance():
    g = _column_grid(8)
    cells, index, pairs, base = heat.voxel_graph(g)
    T0 = 500.0
    T = np.full(len(cells), T0)
    I = 2e-6
    fc = np.zeros(g.nface)
    top = [f for f in range(g.nface) if g.face_owner[f] == cells[-1] and g.face_dir[f] == 4][0]
    fc[top] = I
    dth = 5e-14
    Tn, joule = heat.heat_step(g, T, np.zeros(g.nface), fc, dth, T0)
    # uniform current through a column of length 7.5 cells + the half cell to the base: I^2 R
    sig = float(heat.sigma_of_T(T0))
    Rres = (len(cells) - 0.5) * g.dx / (sig * g.dx ** 2)
    assert joule.sum() == pytest.approx(I * I * Rres, rel=1e-9)
    # discrete energy balance: stored heat = (Joule - conduction into the base) dt
    kap = float(heat.kappa_of_T(T0))
    base_out = 2 * kap * g.dx * (Tn[base] - T0).sum()
    stored = heat.CV * g.dx ** 3 * (Tn - T).sum()
    assert stored == pytest.approx((joule.sum() - base_out) * dth, rel=1e-9)


def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    params = mlp.init_params(rng)
    x = rng.normal(size=(7, mlp.SIZES[0]))
    y = rng.normal(size=(7, 2))
    loss, grads = mlp.loss_and_grad(params, x, y)
    h = 1e-6
    for li in (0, 2, 3):
        W, b = params[li]
        for (r, c) in ((0, 0), (1, 3), (min(5, W.shape[0] - 1), 2)):
            Wp = W.copy(); Wp[r, c] += h
            Wm = W.copy(); Wm[r, c] -= h
            lp, _ = mlp.loss_and_grad([(Wp, b) if i == li else p for i, p in enumerate(params)], x, y)
            lm, _ = mlp.loss_and_grad([(Wm, b) if i == li else p for i, p in enumerate(params)], x, y)
            assert grads[li][0][r, c] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9)
        bp = b.copy(); bp[1] += h
        bm = b.copy(); bm[1] -= h
        lp, _ = mlp.loss_and_grad([(W, bp) if i == li else p for i, p in enumerate(params)], x, y)
        lm, _ = mlp.loss_and_grad([(W, bm) if i == li else p for i, p in enumerate(params)], x, y)
        assert grads[li][1][1] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert mlp.gelu(np.array([30.0]))[0] == pytest.approx(30.0)


def test_bf16_rounding_known_values():
    """Round to nearest even at 8 significand bits: 1 + 2^-9 -> 1; the tie 1 + 2^-8 -> 1 (even);
    the tie 1 + 3 2^-8 -> 1 + 2^-6 (even); 1 + 2^-7 is representable; signs are symmetric."""
    v = np.array([1 + 2.0 ** -9, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -7, -(1 + 3 * 2.0 ** -8), 0.0])
    assert list(mlp.bf16(v)) == [1.0, 1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7, -(1 + 2.0 ** -6), 0.0]
    assert mlp.near_bf16_tie(np.array([1 + 2.0 ** -8]))[0] and not mlp.near_bf16_tie(np.array([1.0]))[0]


def test_mlp_bf16_operands_stay_within_rounding_of_the_exact_network():
    """With BF16 operands the outputs and gradients differ from the float64 network by the
    rounding only: within a few BF16 steps (2^-8) of the scale of the summed terms, and the bias
    gradients of the BF16 layers sum the unrounded values."""
    rng = np.random.default_rng(3)
    params = [(W, rng.normal(0, 0.1, b.size)) for W, b in mlp.init_params(rng)]
    params = [(mlp.bf16(W) if li in mlp.BF16_LAYERS else W, b) for li, (W, b) in enumerate(params)]
    x = rng.normal(size=(64, mlp.SIZES[0]))
    y = rng.normal(size=(64, 2))
    o64, _ = mlp.forward(params, x)
    o16, _ = mlp.forward(params, x, bf16_operands=True)
    scale = np.abs(o64).max()
    assert 0 < np.abs(o16 - o64).max() <= 8 * 2.0 ** -8 * scale
    _, g64 = mlp.loss_and_grad(params, x, y)
    _, g16 = mlp.loss_and_grad(params, x, y, bf16_operands=True)
    for (gw, gb), (hw, hb) in zip(g64, g16):
        assert np.abs(gw - hw).max() <= 8 * 2.0 ** -8 * np.abs(gw).max()
        assert np.abs(gb - hb).max() <= 8 * 2.0 ** -8 * np.abs(gb).max()
    # the output layer's gradients see no rounded operand of their own
    assert not np.array_equal(g64[1][0], g16[1][0])
