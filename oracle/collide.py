"""Monte Carlo collisions of the step (test infrastructure only).

Impact ionization Cu + e -> Cu+ + 2e (Sec. 2.2, Table colls) with SP splitting (Sec. 2.3.2),
the Cu2+ channels of Table colls (Cu + e -> Cu2+ + 3e, Cu+ + e -> Cu2+ + 2e), and direct field
ionization of neutrals (Sec. 2.3.4, eq:dfi).

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
# Cu2+ channels (Table colls).  The paper's cross sections are not available; stand-ins of the
# same Lotz form: direct double ionization of Cu (threshold xi_1 + xi_2) with a tenth of the
# single-ionization constant (Sec. 2.2 expects these cross sections to be small), and
# ionization of Cu+ with the Lotz constant per electron times the 10 electrons of its 3d shell.
XI_DOUBLE = C.XI_CU_EV + C.XI2_CU_EV
LOTZ_A_DOUBLE = LOTZ_A / 10.0
LOTZ_Q_CU1 = 10


def sigma_ion(E_eV, xi=C.XI_CU_EV, a=LOTZ_A):
    """Lotz-form stand-in cross section a ln(E/xi) / (E xi) [m^2]; 0 at or below threshold."""
    E = np.asarray(E_eV, dtype=np.float64)
    out = np.zeros_like(E)
    m = E > xi
    out[m] = a * np.log(E[m] / xi) / (E[m] * xi)
    return out


def sigma_double(E_eV):
    """Cu + e -> Cu2+ + 3e stand-in [m^2]."""
    return sigma_ion(E_eV, XI_DOUBLE, LOTZ_A_DOUBLE)


def sigma_ion2(E_eV):
    """Cu+ + e -> Cu2+ + 2e stand-in [m^2]."""
    return sigma_ion(E_eV, C.XI2_CU_EV, LOTZ_A * LOTZ_Q_CU1)


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


def _pairs(seed, purpose, step, e_off, t_off):
    """Inter-species pairs of every cell holding both species, projectile species first in the
    order (pairs with an electron projectile in cell order, then the others): (projectile,
    target, target SPs in the cell) with the projectile the species with fewer SPs (tie: the
    electrons) and target (k + o_c) mod N_t."""
    cnt_e, cnt_t = np.diff(e_off), np.diff(t_off)
    pairs_e, pairs_t = [], []
    for c in np.nonzero((cnt_e > 0) & (cnt_t > 0))[0]:
        Ne, Nt = int(cnt_e[c]), int(cnt_t[c])
        if Ne <= Nt:
            o = int(philox.uniform_index(seed, purpose, c, step, 0, Nt))
            for k in range(Ne):
                pairs_e.append((e_off[c] + k, t_off[c] + (k + o) % Nt, Nt))
        else:
            o = int(philox.uniform_index(seed, purpose, c, step, 0, Ne))
            for k in range(Nt):
                pairs_t.append((t_off[c] + k, e_off[c] + (k + o) % Ne, Ne))
    return [(True, p) for p in pairs_e] + [(False, p) for p in pairs_t]


def _split_electron(e, ie, ncoll, v, ids, new_e):
    """The ncoll colliding sub-particles of electron SP ie take velocity v: the whole SP turns
    when ncoll is its weight, else they leave as a new SP (Sec. 2.3.2)."""
    we = int(e["w"][ie])
    if ncoll == we:
        e["vx"][ie], e["vy"][ie], e["vz"][ie] = F32(v[0]), F32(v[1]), F32(v[2])
    else:
        e["w"][ie] = we - ncoll
        new_e.append(_new_sp(e["x"][ie], e["y"][ie], e["z"][ie], v[0], v[1], v[2], ncoll, ids.take()))


def impact_ionization(grid, prm, e, e_off, n, n_off, step, ids, double=False):
    """One MCC pass over all cells.  e, n: cell-sorted electron / neutral SPs (modified in
    place: weights and velocities); returns (new ions, new electrons, number of events).

    double: the Cu2+ channel Cu + e -> Cu2+ + 3e competes for the same draws, by the total
    cross section (the paper gives eq:colp for one process): P_T = 1 - exp(-u n_t W_t
    (sigma_1 + sigma_2) dt), and sub-particle i ionizes once when U_i < P_T sigma_1/sigma_T and
    twice when P_T sigma_1/sigma_T <= U_i < P_T; N_1 capped at the target weight, N_2 at what
    is left of it.  Without the channel (or below its threshold) sigma_2 = 0 and the single
    decisions are those of the one-process pass.  The double events are applied after all
    single ones, in the same pair order (Cu2+, the scattered electron when the electron SP
    splits, two secondary electrons; E0 - xi_1 - xi_2 shared equally by the three outgoing
    electrons, directions by eq:du); returns then also (new Cu2+, new electrons, double
    events)."""
    V_cell = grid.dx ** 3
    dt = prm["dt"]
    seed = prm["seed"]
    w_min = prm["w_min"]
    new_i, new_e = [], []
    dbl = []
    events = 0
    for proj_is_e, (pi, ti, Nt) in _pairs(seed, philox.PAIR, step, e_off, n_off):
        ie, inn = (pi, ti) if proj_is_e else (ti, pi)
        we, wn = int(e["w"][ie]), int(n["w"][inn])
        ve = np.array([e["vx"][ie], e["vy"][ie], e["vz"][ie]], dtype=np.float64)
        vn = np.array([n["vx"][inn], n["vy"][inn], n["vz"][inn]], dtype=np.float64)
        uvec = ve - vn
        u2 = uvec[0] * uvec[0] + uvec[1] * uvec[1] + uvec[2] * uvec[2]
        u = math.sqrt(u2)
        E0 = 0.5 * C.M_E * u2 / C.E_CHARGE
        wt = wn if proj_is_e else we
        wp = we if proj_is_e else wn
        s1 = float(sigma_ion(E0))
        sT = s1 + float(sigma_double(E0)) if double else s1
        PT = -math.expm1(-(u * (Nt / V_cell) * (wt * w_min) * sT * dt))
        P1 = PT * (s1 / sT) if sT > 0 else 0.0
        proj_id = int(e["id"][ie] if proj_is_e else n["id"][inn])
        U = philox.uniform(seed, philox.ION, proj_id, step, np.arange(wp))
        ncoll = min(int(np.sum(U < P1)), wt)
        if double:
            n2 = min(int(np.sum((U >= P1) & (U < PT))), wt - ncoll)
            if n2 > 0:
                dbl.append((ie, inn, proj_id, n2, uvec, E0, vn))
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
        _split_electron(e, ie, ncoll, v1, ids, new_e)
        new_e.append(_new_sp(n["x"][inn], n["y"][inn], n["z"][inn], v2[0], v2[1], v2[2], ncoll, ids.take()))
    if not double:
        return _append(new_i), _append(new_e), events
    new_j, new_e2 = [], []
    for (ie, inn, proj_id, n2, uvec, E0, vn) in dbl:
        new_j.append(_new_sp(n["x"][inn], n["y"][inn], n["z"][inn], n["vx"][inn], n["vy"][inn], n["vz"][inn], n2,
                             ids.take()))
        n["w"][inn] = int(n["w"][inn]) - n2
        uk = math.sqrt(2.0 * (E0 - XI_DOUBLE) / 3.0 * C.E_CHARGE / C.M_E)
        Us = philox.uniform(seed, philox.SCAT2, proj_id, step, np.arange(6))
        vs = [vn + scatter_velocity(uvec, uk, 2.0 * Us[2 * q] - 1.0, 2.0 * math.pi * Us[2 * q + 1]) for q in range(3)]
        _split_electron(e, ie, n2, vs[0], ids, new_e2)
        for v in vs[1:]:
            new_e2.append(_new_sp(n["x"][inn], n["y"][inn], n["z"][inn], v[0], v[1], v[2], n2, ids.take()))
    return _append(new_i), _append(new_e), events, _append(new_j), _append(new_e2), len(dbl)


def ion_ionization(grid, prm, e, e_off, i, i_off, step, ids):
    """Cu+ + e -> Cu2+ + 2e (Table colls) on the cell-sorted electrons and Cu+, with the pairing,
    the per-sub-particle probability and the splitting of impact ionization (own Philox
    purposes): Cu2+ of weight N with the Cu+ SP's position and velocity, the Cu+ SP loses N, the
    electron SP splits, a secondary electron at the Cu+ position; E0 - xi_2 shared equally by the
    two outgoing electrons (eq:du about u = v_e - v_i).  e, i modified in place; returns (new Cu2+,
    new electrons, events)."""
    V_cell = grid.dx ** 3
    dt, seed, w_min = prm["dt"], prm["seed"], prm["w_min"]
    new_j, new_e = [], []
    events = 0
    for proj_is_e, (pi, ti, Nt) in _pairs(seed, philox.PAIR_IZ, step, e_off, i_off):
        ie, ii = (pi, ti) if proj_is_e else (ti, pi)
        we, wi = int(e["w"][ie]), int(i["w"][ii])
        if we <= 0 or wi <= 0:
            continue
        ve = np.array([e["vx"][ie], e["vy"][ie], e["vz"][ie]], dtype=np.float64)
        vi = np.array([i["vx"][ii], i["vy"][ii], i["vz"][ii]], dtype=np.float64)
        uvec = ve - vi
        u2 = uvec[0] * uvec[0] + uvec[1] * uvec[1] + uvec[2] * uvec[2]
        u = math.sqrt(u2)
        E0 = 0.5 * C.M_E * u2 / C.E_CHARGE
        wt = wi if proj_is_e else we
        wp = we if proj_is_e else wi
        prob = -math.expm1(-(u * (Nt / V_cell) * (wt * w_min) * float(sigma_ion2(E0)) * dt))
        proj_id = int(e["id"][ie] if proj_is_e else i["id"][ii])
        U = philox.uniform(seed, philox.ION_IZ, proj_id, step, np.arange(wp))
        ncoll = min(int(np.sum(U < prob)), wt)
        if ncoll == 0:
            continue
        events += 1
        new_j.append(_new_sp(i["x"][ii], i["y"][ii], i["z"][ii], i["vx"][ii], i["vy"][ii], i["vz"][ii], ncoll,
                             ids.take()))
        i["w"][ii] = wi - ncoll
        uk = math.sqrt(2.0 * 0.5 * (E0 - C.XI2_CU_EV) * C.E_CHARGE / C.M_E)
        Us = philox.uniform(seed, philox.SCAT_IZ, proj_id, step, np.arange(4))
        v1 = vi + scatter_velocity(uvec, uk, 2.0 * Us[0] - 1.0, 2.0 * math.pi * Us[1])
        v2 = vi + scatter_velocity(uvec, uk, 2.0 * Us[2] - 1.0, 2.0 * math.pi * Us[3])
        _split_electron(e, ie, ncoll, v1, ids, new_e)
        new_e.append(_new_sp(i["x"][ii], i["y"][ii], i["z"][ii], v2[0], v2[1], v2[2], ncoll, ids.take()))
    return _append(new_j), _append(new_e), events


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
