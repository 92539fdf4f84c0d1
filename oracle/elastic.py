"""Elastic collisions and resonant charge exchange (test infrastructure only).

Processes of Table colls that move no charge between species: e + Cu -> e + Cu and Cu + Cu ->
Cu + Cu (elastic, eq:newv with the velocity difference of eq:du), and Cu+ + Cu -> Cu + Cu+
(charge exchange).  Collision probability from eq:colp in the sub-particle form of Sec. 2.3.2,
pairing as in Sec. 2.2.

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
  * Splitting (Sec. 2.3.2, as for impact ionization): each of the w_p sub-particles of the
    projectile collides iff U_i < P, P = 1 - exp(-u n_t W_t sigma dt) with n_t the target SP
    density in the cell and W_t the paired target's weight in real particles; N_coll =
    #{i : U_i < P}, capped at the target weight.  A pair in which either weight is 0 does not
    collide.  The N_coll colliding sub-particles of each side leave their SP as a new SP of
    weight N_coll with the post-collision velocity (the whole SP turns when N_coll equals its
    weight); one pair of scattering angles serves the N_coll collisions.  Momentum is thus
    conserved exactly, and energy for elastic collisions.
  * Elastic velocities: du = R^-1(theta,phi) [R^-1(theta',phi') - I] (0,0,u) (eq:du), with
    (theta,phi) the polar angles of u = v_A - v_B, cos(theta') = 2U - 1, phi' = 2 pi U';
    v_A' = v_A + mu/m_A du, v_B' = v_B - mu/m_B du (eq:newv).
  * Charge exchange: the electron hops, so the ion continues with the neutral's velocity and
    the neutral with the ion's: the N_coll colliding sub-particles swap velocities.
  * Order of the new SPs (ids and slots): events of a pass in the order of the pair's member in
    the first species of the pass (e-, Cu+, or the projectile for Cu-Cu) in cell-sorted order;
    per event the projectile's new SP, then the target's.
  * Cross sections: the paper's data is not available, so constant stand-ins:
    e-Cu elastic 1e-19 m^2, Cu-Cu hard spheres pi (2 r)^2 with r = 128 pm, Cu+-Cu resonant
    charge exchange 5e-19 m^2 (each a parameter).
  * Draws (Philox streams of the pass, keyed by the projectile's id and the step): sub-particle
    i takes word i of the draw stream; the scattering angles take words 0 and 1 of the
    scatter stream.
"""
import math

import numpy as np

from . import constants as C
from . import particles as P
from . import philox
from .collide import rot_inv

# Philox purposes of these passes: pairing offset per cell, sub-particle draws, scattering angles
PAIR_EN, DRAW_EN, PAIR_NN, DRAW_NN, PAIR_CX, DRAW_CX, SCAT_EN, SCAT_NN = 8, 9, 10, 11, 12, 13, 14, 15

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
    """eq:colp per projectile sub-particle: 1 - exp(-u n_t W_t sigma dt) from float32 velocities."""
    d = [float(vA[c]) - float(vB[c]) for c in range(3)]
    u = math.sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2])
    return -math.expm1(-(u * (Nt / V_cell) * (wt * w_min) * sigma * dt))


def _vel(sp_, i):
    return np.array([sp_["vx"][i], sp_["vy"][i], sp_["vz"][i]], dtype=np.float64)


def _put(sp_, i, v):
    sp_["vx"][i], sp_["vy"][i], sp_["vz"][i] = F32(v[0]), F32(v[1]), F32(v[2])


class _Out:
    """New SPs of a pass per species and the id counter."""

    def __init__(self, ids):
        self.ids = ids
        self.new = {}

    def add(self, key, sp_, i, v, w):
        self.new.setdefault(key, []).append(
            {"x": sp_["x"][i], "y": sp_["y"][i], "z": sp_["z"][i], "vx": F32(v[0]), "vy": F32(v[1]), "vz": F32(v[2]),
             "w": np.int32(w), "id": np.uint64(self.ids.take())})

    def arrays(self, key):
        lst = self.new.get(key, [])
        if not lst:
            return P.empty()
        return {k: np.array([d[k] for d in lst], dtype=P.DTYPES[k]) for k in P.FIELDS}


def _collide_pair(A, ia, kA, B, ib, kB, mA, mB, Nt, V_cell, prm, sigma, draw, scat, step, kind, out):
    """One pair, A[ia] the projectile.  True if any sub-particle collided."""
    wa, wb = int(A["w"][ia]), int(B["w"][ib])
    if wa <= 0 or wb <= 0:
        return False
    vA, vB = _vel(A, ia), _vel(B, ib)
    Pc = collision_probability(vA, vB, Nt, V_cell, wb, prm["w_min"], sigma, prm["dt"])
    pid = int(A["id"][ia])
    U = philox.uniform(prm["seed"], draw, pid, step, np.arange(wa))
    n = min(int(np.sum(U < Pc)), wb)
    if n == 0:
        return False
    if kind == "exchange":
        nA, nB = vB, vA
    else:
        Us = philox.uniform(prm["seed"], scat, pid, step, np.arange(2))
        nA, nB = elastic_velocities(vA, vB, mA, mB, 2.0 * Us[0] - 1.0, 2.0 * math.pi * Us[1])
    for sp_, i, key, w, v in ((A, ia, kA, wa, nA), (B, ib, kB, wb, nB)):
        if n == w:
            _put(sp_, i, v)
        else:
            sp_["w"][i] = w - n
            out.add(key, sp_, i, v, n)
    return True


def _inter_species(grid, prm, P_, p_off, kP, Q, q_off, kQ, mP, mQ, sigma, pair_purpose, draw, scat, step, kind, out):
    """Pairs between species P_ (preferred projectile on ties) and Q in every cell, events in the
    order of their P_ member."""
    seed = prm["seed"]
    V_cell = grid.dx ** 3
    cnt_p, cnt_q = np.diff(p_off), np.diff(q_off)
    pairs = []   # (P_ index, projectile is P_, partner index, Nt)
    for c in np.nonzero((cnt_p > 0) & (cnt_q > 0))[0]:
        Np, Nq = int(cnt_p[c]), int(cnt_q[c])
        if Np <= Nq:
            o = int(philox.uniform_index(seed, pair_purpose, c, step, 0, Nq))
            for k in range(Np):
                pairs.append((p_off[c] + k, True, q_off[c] + (k + o) % Nq, Nq))
        else:
            o = int(philox.uniform_index(seed, pair_purpose, c, step, 0, Np))
            for k in range(Nq):
                pairs.append((p_off[c] + (k + o) % Np, False, q_off[c] + k, Np))
    pairs.sort(key=lambda t: t[0])
    events = 0
    for ip, p_proj, iq, Nt in pairs:
        if p_proj:
            events += _collide_pair(P_, ip, kP, Q, iq, kQ, mP, mQ, Nt, V_cell, prm, sigma, draw, scat, step, kind, out)
        else:
            events += _collide_pair(Q, iq, kQ, P_, ip, kP, mQ, mP, Nt, V_cell, prm, sigma, draw, scat, step, kind, out)
    return events


def elastic_en(grid, prm, e, e_off, n, n_off, step, ids):
    """e + Cu -> e + Cu on the cell-sorted SPs (modified in place); returns (new e-, new Cu,
    events)."""
    out = _Out(ids)
    ev = _inter_species(grid, prm, e, e_off, "e", n, n_off, "n", C.M_E, C.M_CU, prm.get("sigma_el_en", SIGMA_EN),
                        PAIR_EN, DRAW_EN, SCAT_EN, step, "elastic", out)
    return out.arrays("e"), out.arrays("n"), ev


def elastic_nn(grid, prm, n, n_off, step, ids):
    """Cu + Cu -> Cu + Cu between the neutral SPs of each cell; returns (new Cu, events)."""
    seed = prm["seed"]
    sigma = prm.get("sigma_el_nn", SIGMA_NN)
    V_cell = grid.dx ** 3
    cnt = np.diff(n_off)
    pairs = []
    for c in np.nonzero(cnt >= 2)[0]:
        N = int(cnt[c])
        o = int(philox.uniform_index(seed, PAIR_NN, c, step, 0, N))
        for m in range(N // 2):
            pairs.append((n_off[c] + (o + 2 * m) % N, n_off[c] + (o + 2 * m + 1) % N, N))
    pairs.sort(key=lambda t: t[0])
    out = _Out(ids)
    events = 0
    for a, b, N in pairs:
        events += _collide_pair(n, a, "n", n, b, "n", C.M_CU, C.M_CU, N, V_cell, prm, sigma, DRAW_NN, SCAT_NN, step,
                                "elastic", out)
    return out.arrays("n"), events


def charge_exchange(grid, prm, i, i_off, n, n_off, step, ids):
    """Cu+ + Cu -> Cu + Cu+ (velocity swap of the colliding sub-particles); returns (new Cu+,
    new Cu, events)."""
    out = _Out(ids)
    ev = _inter_species(grid, prm, i, i_off, "i", n, n_off, "n", C.M_CU, C.M_CU, prm.get("sigma_cx", SIGMA_CX),
                        PAIR_CX, DRAW_CX, None, step, "exchange", out)
    return out.arrays("i"), out.arrays("n"), ev
