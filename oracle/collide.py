"""Monte Carlo collisions of the step (test infrastructure only).

Impact ionization Cu + e -> Cu+ + 2e (Sec. 2.2, Table colls) with SP splitting (Sec. 2.3.2),
and direct field ionization of neutrals (Sec. 2.3.4, eq:dfi).

Readings where the paper is silent or ambiguous (each listed in the design notes):
  * Pairing (Sec. 2.2 cites Takizuka-Abe): in a cell with N_e electron SPs and N_n neutral
    SPs, the projectile species is the one with the lower SP density (tie: electrons).
    Projectile k (k-th in cell-sorted order) meets target (k + o_c) mod N_t, with the offset
    o_c = floor(U_PAIR(cell, step) * N_t).
  * Probability (eq:colp with the SP form of Sec. 2.3.2): for every sub-particle of the
    projectile, P = 1 - exp(-u * n_t * W_t * sigma(E0) * dt), n_t = N_t / V_cell the target
    SP density and W_t the paired target's weight in real particles.  A projectile
    sub-particle counts as one real particle, which makes the expected rate equal to the
    real-particle rate n * sigma(v) * v; N_coll = #{i : U_i < P} over the w_p sub-particles
    (the max(0, ceil(1 - U_i/P)) sum of Sec. 2.3.2), capped at the target weight.
  * Cross section: the paper's data (refs. bolcs, frecs, pincs, grecs) is not available; a
    Lotz-form stand-in sigma(E) = a ln(E/xi)/(E xi), a = 4.5e-14 cm^2 eV^2, xi = 7.726 eV.
  * Products: Cu+ of weight N_coll with the neutral's position and velocity; the electron SP
    is split (N_coll scattered, w_e - N_coll unchanged); a secondary electron of weight
    N_coll at the neutral's position.  E0 - xi is shared equally by the two outgoing
    electrons; each direction follows eq:du: u' = R^-1(theta,phi) R^-1(theta',phi') (0,0,u_k),
    with (theta,phi) the polar angles of u = v_e - v_n and cos(theta') ~ U(-1,1),
    phi' ~ U(0,2pi); v' = v_n + u' (neutral recoil neglected, m_e << m_Cu).
  * Field ionization: per sub-particle, ionized iff P_fs(E) * dt_fs > U (eq:dfi, linear
    criterion as printed).  Above the barrier-suppression limit E > 1.5 xi^{3/2} GV/m the
    paper "rejects" neutrals; read here as certain ionization.  Products as above with a new
    electron at rest.
"""
import math

import numpy as np

from . import constants as C
from . import particles as P
from . import philox

LOTZ_A = 4.5e-14 * 1e-4           # m^2 eV^2
F32 = np.float32


def sigma_ion(E_eV, xi=C.XI_CU_EV):
    """Lotz-form stand-in cross section [m^2]; 0 at or below threshold."""
    E = np.asarray(E_eV, dtype=np.float64)
    out = np.zeros_like(E)
    m = E > xi
    out[m] = LOTZ_A * np.log(E[m] / xi) / (E[m] * xi)
    return out


def rot_inv(theta, phi, vec):
    """R^-1(theta, phi) @ vec with R of Sec. 2.2 (orthogonal, so R^-1 = R^T)."""
    ct, st, cp, s_p = math.cos(theta), math.sin(theta), math.cos(phi), math.sin(phi)
    R = np.array([[ct * cp, ct * s_p, -st], [-s_p, cp, 0.0], [st * cp, st * s_p, ct]])
    return R.T @ np.asarray(vec, dtype=np.float64)


def scatter_velocity(u_vec, u_new, cos_tp, phi_p):
    """R^-1(theta,phi) R^-1(theta',phi') (0,0,u_new): eq:du with the outgoing speed u_new."""
    u = math.sqrt(float(u_vec @ u_vec))
    theta = math.acos(max(-1.0, min(1.0, u_vec[2] / u))) if u > 0 else 0.0
    phi = math.atan2(u_vec[1], u_vec[0]) if u > 0 else 0.0
    theta_p = math.acos(cos_tp)
    return rot_inv(theta, phi, rot_inv(theta_p, phi_p, np.array([0.0, 0.0, u_new])))


class Counter:
    """Global id counter: new SPs take consecutive ids in creation order."""

    def __init__(self, next_id):
        self.next_id = int(next_id)

    def take(self):
        v = self.next_id
        self.next_id += 1
        return v


def _new_sp(x, y, z, vx, vy, vz, w, ident):
    return {"x": F32(x), "y": F32(y), "z": F32(z), "vx": F32(vx), "vy": F32(vy), "vz": F32(vz),
            "w": np.int32(w), "id": np.uint64(ident)}


def _append(lst):
    out = P.empty()
    if not lst:
        return out
    return {k: np.array([d[k] for d in lst], dtype=P.DTYPES[k]) for k in P.FIELDS}


def impact_ionization(grid, prm, e, e_off, n, n_off, step, ids):
    """One MCC pass over all cells.  e, n: cell-sorted electron / neutral SPs (modified in
    place: weights and velocities); returns (new ions, new electrons, number of events)."""
    V_cell = grid.dx ** 3
    dt = prm["dt"]
    seed = prm["seed"]
    w_min = prm["w_min"]
    ncell = grid.ncell
    cnt_e = np.diff(e_off)
    cnt_n = np.diff(n_off)
    both = np.nonzero((cnt_e > 0) & (cnt_n > 0))[0]
    pairs_e, pairs_n = [], []          # (projectile index, target index)
    for c in both:
        Ne, Nn = int(cnt_e[c]), int(cnt_n[c])
        if Ne <= Nn:
            o = int(philox.uniform_index(seed, philox.PAIR, c, step, 0, Nn))
            for k in range(Ne):
                pairs_e.append((c, e_off[c] + k, n_off[c] + (k + o) % Nn, Nn))
        else:
            o = int(philox.uniform_index(seed, philox.PAIR, c, step, 0, Ne))
            for k in range(Nn):
                pairs_n.append((c, n_off[c] + k, e_off[c] + (k + o) % Ne, Ne))
    new_i, new_e = [], []
    events = 0
    for proj_is_e, plist in ((True, pairs_e), (False, pairs_n)):
        for (c, pi, ti, Nt) in plist:
            ie, inn = (pi, ti) if proj_is_e else (ti, pi)
            we, wn = int(e["w"][ie]), int(n["w"][inn])
            ve = np.array([e["vx"][ie], e["vy"][ie], e["vz"][ie]], dtype=np.float64)
            vn = np.array([n["vx"][inn], n["vy"][inn], n["vz"][inn]], dtype=np.float64)
            uvec = ve - vn
            u2 = uvec[0] * uvec[0] + uvec[1] * uvec[1] + uvec[2] * uvec[2]
            u = math.sqrt(u2)
            E0 = 0.5 * C.M_E * u2 / C.E_CHARGE
            sig = float(sigma_ion(E0))
            wt = wn if proj_is_e else we
            wp = we if proj_is_e else wn
            x = u * (Nt / V_cell) * (wt * w_min) * sig * dt
            prob = -math.expm1(-x)
            proj_id = int(e["id"][ie] if proj_is_e else n["id"][inn])
            U = philox.uniform(seed, philox.ION, proj_id, step, np.arange(wp))
            ncoll = int(np.sum(U < prob))
            ncoll = min(ncoll, wt)
            if ncoll == 0:
                continue
            events += 1
            # products: ion, scattered electron, secondary electron
            new_i.append(_new_sp(n["x"][inn], n["y"][inn], n["z"][inn], n["vx"][inn], n["vy"][inn],
                                 n["vz"][inn], ncoll, ids.take()))
            n["w"][inn] = wn - ncoll
            Ek = 0.5 * (E0 - C.XI_CU_EV)
            uk = math.sqrt(2.0 * Ek * C.E_CHARGE / C.M_E)
            Us = philox.uniform(seed, philox.SCAT, proj_id, step, np.arange(4))
            v1 = vn + scatter_velocity(uvec, uk, 2.0 * Us[0] - 1.0, 2.0 * math.pi * Us[1])
            v2 = vn + scatter_velocity(uvec, uk, 2.0 * Us[2] - 1.0, 2.0 * math.pi * Us[3])
            if ncoll == we:
                e["vx"][ie], e["vy"][ie], e["vz"][ie] = F32(v1[0]), F32(v1[1]), F32(v1[2])
            else:
                e["w"][ie] = we - ncoll
                new_e.append(_new_sp(e["x"][ie], e["y"][ie], e["z"][ie], v1[0], v1[1], v1[2], ncoll, ids.take()))
            new_e.append(_new_sp(n["x"][inn], n["y"][inn], n["z"][inn], v2[0], v2[1], v2[2], ncoll, ids.take()))
    return _append(new_i), _append(new_e), events


# --------------------------------------------------------------------------------------
# direct field ionization, eq:dfi
# --------------------------------------------------------------------------------------
def adk_rate_per_fs(E_GV, xi=C.XI_CU_EV, z=1):
    """P [1/fs] = 1.52 4^n xi / (n Gamma(2n)) (20.5 xi^{3/2}/E)^{2n-1} exp(-6.83 xi^{3/2}/E),
    n = 3.69 z xi^{-1/2}; E in GV/m, xi in eV (eq:dfi)."""
    E = np.asarray(E_GV, dtype=np.float64)
    n = 3.69 * z / math.sqrt(xi)
    pre = 1.52 * 4.0 ** n * xi / (n * math.gamma(2.0 * n))
    x15 = xi ** 1.5
    out = np.zeros_like(E)
    m = E > 0
    out[m] = pre * (20.5 * x15 / E[m]) ** (2.0 * n - 1.0) * np.exp(-6.83 * x15 / E[m])
    return out


def bsi_limit_GV(xi=C.XI_CU_EV):
    return 1.5 * xi ** 1.5


def field_ionization(grid, prm, n, E, step, ids):
    """ADK ionization of every neutral SP with w > 0 (cell-sorted order).  n modified in place;
    returns (new ions, new electrons, number of ionized SPs)."""
    dt_fs = prm["dt"] * 1e15
    seed = prm["seed"]
    new_i, new_e = [], []
    events = 0
    if P.count(n) == 0:
        return P.empty(), P.empty(), 0
    e = P.gather(E, n["x"], n["y"], n["z"])
    e64 = e.astype(np.float64)
    E2 = e64[:, 0] * e64[:, 0] + e64[:, 1] * e64[:, 1] + e64[:, 2] * e64[:, 2]
    lim = bsi_limit_GV() * 1e9
    for p in range(P.count(n)):
        wn = int(n["w"][p])
        if wn <= 0:
            continue
        if E2[p] > lim * lim:
            nion = wn
        else:
            prob = float(adk_rate_per_fs(math.sqrt(E2[p]) * 1e-9)) * dt_fs
            U = philox.uniform(seed, philox.DFI, int(n["id"][p]), step, np.arange(wn))
            nion = int(np.sum(U < prob))
        if nion == 0:
            continue
        events += 1
        new_i.append(_new_sp(n["x"][p], n["y"][p], n["z"][p], n["vx"][p], n["vy"][p], n["vz"][p], nion, ids.take()))
        new_e.append(_new_sp(n["x"][p], n["y"][p], n["z"][p], 0.0, 0.0, 0.0, nion, ids.take()))
        n["w"][p] = wn - nion
    return _append(new_i), _append(new_e), events
