"""Elastic collisions and resonant charge exchange (test infrastructure only).

Processes of Table colls that move no charge between SPs: e + Cu -> e + Cu and Cu + Cu ->
Cu + Cu (elastic, eq:newv with the velocity difference of eq:du), and Cu+ + Cu -> Cu + Cu+
(charge exchange).  Collision probability per pair from eq:colp, pairing as in Sec. 2.2.

Readings (the paper gives the equations, not these details):
  * Three passes run after impact ionization and before field ionization, in the order
    e-Cu elastic, Cu-Cu elastic, Cu+-Cu charge exchange, each on the cell-sorted SPs of the
    step (SPs created earlier in the step take no part).
  * Inter-species pairs (e-Cu, Cu+-Cu): as for impact ionization, the species with fewer SPs
    in the cell (tie: the charged one) is the projectile; projectile k meets target
    (k + o_c) mod N_t, o_c = floor(U(cell, step) N_t) from the pass's own pairing stream.
  * Like-species pairs (Cu-Cu): with N >= 2 neutral SPs in the cell and o_c = floor(U N),
    the SPs at shuffled places (o_c + 2m) mod N and (o_c + 2m + 1) mod N form pair m,
    m < floor(N/2) (with N odd one SP sits out); the first one is the projectile.
  * Whole SPs collide (no splitting; the paper splits SPs only where an ionization needs it,
    Sec. 2.3.2): one draw U_c per pair, collision iff U_c < P, P = 1 - exp(-u n_t W_t sigma dt)
    with n_t the target SP density in the cell and W_t the paired target's weight in real
    particles (the projectile view of the impact-ionization reading).  A pair in which either
    weight is 0 does not collide.
  * Weighted SPs (Nanbu-Yonemura rule): the SP with the smaller weight always takes its
    post-collision velocity; the other takes its own with probability w_small/w_large
    (equal weights: both), so momentum and energy are conserved on average, exactly when the
    weights are equal.  The test U_w < w_s/w_l is made in integers on the 24-bit draw.
  * Elastic velocities: du = R^-1(theta,phi) [R^-1(theta',phi') - I] (0,0,u) (eq:du), with
    (theta,phi) the polar angles of u = v_A - v_B, cos(theta') = 2U - 1, phi' = 2 pi U';
    v_A' = v_A + mu/m_A du, v_B' = v_B - mu/m_B du (eq:newv).
  * Charge exchange: the electron hops, so the ion continues with the neutral's velocity and
    the neutral with the ion's: the two SPs swap velocities (weights, positions and species
    unchanged).
  * Cross sections: the paper's data is not available, so constant stand-ins:
    e-Cu elastic 1e-19 m^2, Cu-Cu hard spheres pi (2 r)^2 with r = 128 pm, Cu+-Cu resonant
    charge exchange 5e-19 m^2 (each a parameter).
  * Draws per pair (Philox stream of the pass, keyed by the projectile's id and the step):
    word 0 U_c, word 1 cos(theta'), word 2 phi', word 3 U_w.
"""
import math

import numpy as np

from . import constants as C
from . import philox
from .collide import rot_inv

# Philox purposes of these passes (pairing offset per cell, draws per pair)
PAIR_EN, DRAW_EN, PAIR_NN, DRAW_NN, PAIR_CX, DRAW_CX = 8, 9, 10, 11, 12, 13

SIGMA_EN = 1.0e-19                          # m^2, e-Cu elastic (stand-in)
SIGMA_NN = math.pi * (2 * 128e-12) ** 2     # m^2, Cu-Cu hard spheres (r = 128 pm)
SIGMA_CX = 5.0e-19                          # m^2, Cu+-Cu resonant charge exchange (stand-in)

F32 = np.float32


def delta_u(u_vec, cos_tp, phi_p):
    """eq:du: R^-1(theta,phi) [R^-1(theta',phi') - I] (0,0,u), (theta,phi) the angles of u_vec."""
    u_vec = np.asarray(u_vec, dtype=np.float64)
    u = math.sqrt(float(u_vec[0] * u_vec[0] + u_vec[1] * u_vec[1] + u_vec[2] * u_vec[2]))
    theta = math.acos(max(-1.0, min(1.0, u_vec[2] / u))) if u > 0 else 0.0
    phi = math.atan2(u_vec[1], u_vec[0]) if u > 0 else 0.0
    pole = np.array([0.0, 0.0, u])
    return rot_inv(theta, phi, rot_inv(math.acos(cos_tp), phi_p, pole) - pole)


def elastic_velocities(vA, vB, mA, mB, cos_tp, phi_p):
    """eq:newv: (v_A', v_B') in float64."""
    vA, vB = np.asarray(vA, dtype=np.float64), np.asarray(vB, dtype=np.float64)
    du = delta_u(vA - vB, cos_tp, phi_p)
    mu = mA * mB / (mA + mB)
    return vA + mu / mA * du, vB - mu / mB * du


def collision_probability(vA, vB, Nt, V_cell, wt, w_min, sigma, dt):
    """eq:colp for one pair: 1 - exp(-u n_t W_t sigma dt) from float32 velocities, in float64."""
    d = [float(vA[c]) - float(vB[c]) for c in range(3)]
    u = math.sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2])
    return -math.expm1(-(u * (Nt / V_cell) * (wt * w_min) * sigma * dt))


def weight_keeps(word, w_small, w_large):
    """U_w < w_small / w_large for U_w = ((word >> 8) + 1/2) 2^-24, exactly in integers."""
    return (2 * (int(word) >> 8) + 1) * int(w_large) < int(w_small) << 25


def _vel(sp_, i):
    return np.array([sp_["vx"][i], sp_["vy"][i], sp_["vz"][i]], dtype=np.float64)


def _put(sp_, i, v):
    sp_["vx"][i], sp_["vy"][i], sp_["vz"][i] = F32(v[0]), F32(v[1]), F32(v[2])


def _collide_pair(A, ia, B, ib, mA, mB, Nt, V_cell, prm, sigma, purpose, step, kind):
    """One pair: decide, then update the velocities (elastic or exchange).  True if it collided."""
    wa, wb = int(A["w"][ia]), int(B["w"][ib])
    if wa <= 0 or wb <= 0:
        return False
    vA, vB = _vel(A, ia), _vel(B, ib)
    P = collision_probability(vA, vB, Nt, V_cell, wb, prm["w_min"], sigma, prm["dt"])
    w = philox.words(prm["seed"], purpose, int(A["id"][ia]), step, np.arange(4))
    U = ((int(w[0]) >> 8) + 0.5) * 2.0 ** -24
    if not U < P:
        return False
    if kind == "exchange":
        nA, nB = vB, vA
    else:
        cos_tp = 2.0 * (((int(w[1]) >> 8) + 0.5) * 2.0 ** -24) - 1.0
        phi_p = 2.0 * math.pi * (((int(w[2]) >> 8) + 0.5) * 2.0 ** -24)
        nA, nB = elastic_velocities(vA, vB, mA, mB, cos_tp, phi_p)
    if wa <= wb:
        _put(A, ia, nA)
        if weight_keeps(w[3], wa, wb):
            _put(B, ib, nB)
    else:
        _put(B, ib, nB)
        if weight_keeps(w[3], wb, wa):
            _put(A, ia, nA)
    return True


def _inter_species(grid, prm, P_, p_off, Q, q_off, mP, mQ, sigma, pair_purpose, draw_purpose, step, kind):
    """Pairs between species P_ (preferred projectile on ties) and Q in every cell."""
    seed = prm["seed"]
    V_cell = grid.dx ** 3
    cnt_p, cnt_q = np.diff(p_off), np.diff(q_off)
    events = 0
    for c in np.nonzero((cnt_p > 0) & (cnt_q > 0))[0]:
        Np, Nq = int(cnt_p[c]), int(cnt_q[c])
        if Np <= Nq:
            o = int(philox.uniform_index(seed, pair_purpose, c, step, 0, Nq))
            for k in range(Np):
                events += _collide_pair(P_, p_off[c] + k, Q, q_off[c] + (k + o) % Nq, mP, mQ, Nq, V_cell, prm, sigma,
                                        draw_purpose, step, kind)
        else:
            o = int(philox.uniform_index(seed, pair_purpose, c, step, 0, Np))
            for k in range(Nq):
                events += _collide_pair(Q, q_off[c] + k, P_, p_off[c] + (k + o) % Np, mQ, mP, Np, V_cell, prm, sigma,
                                        draw_purpose, step, kind)
    return events


def elastic_en(grid, prm, e, e_off, n, n_off, step):
    """e + Cu -> e + Cu on the cell-sorted SPs (velocities modified in place); returns events."""
    return _inter_species(grid, prm, e, e_off, n, n_off, C.M_E, C.M_CU, prm.get("sigma_el_en", SIGMA_EN),
                          PAIR_EN, DRAW_EN, step, "elastic")


def elastic_nn(grid, prm, n, n_off, step):
    """Cu + Cu -> Cu + Cu between the neutral SPs of each cell; returns events."""
    seed = prm["seed"]
    sigma = prm.get("sigma_el_nn", SIGMA_NN)
    V_cell = grid.dx ** 3
    cnt = np.diff(n_off)
    events = 0
    for c in np.nonzero(cnt >= 2)[0]:
        N = int(cnt[c])
        o = int(philox.uniform_index(seed, PAIR_NN, c, step, 0, N))
        for m in range(N // 2):
            a = n_off[c] + (o + 2 * m) % N
            b = n_off[c] + (o + 2 * m + 1) % N
            events += _collide_pair(n, a, n, b, C.M_CU, C.M_CU, N, V_cell, prm, sigma, DRAW_NN, step, "elastic")
    return events


def charge_exchange(grid, prm, i, i_off, n, n_off, step):
    """Cu+ + Cu -> Cu + Cu+ (velocity swap); returns events."""
    return _inter_species(grid, prm, i, i_off, n, n_off, C.M_CU, C.M_CU, prm.get("sigma_cx", SIGMA_CX),
                          PAIR_CX, DRAW_CX, step, "exchange")
