"""Coulomb collisions between charged SPs by the binary method the paper cites (Table colls:
e-e, Cu+-e, Cu+-Cu+, and with Cu2+ (Sec. 2.2: between all charged species) e-Cu2+, Cu+-Cu2+,
Cu2+-Cu2+; Takizuka and Abe, J. Comput. Phys. 25, 205 (1977)).  Test infrastructure only.

Every pair scatters every step by a small random angle theta: delta = tan(theta/2) is normal
with zero mean and variance
    <delta^2> = q_a^2 q_b^2 n lnL dt / (8 pi eps0^2 m_ab^2 u^3),    m_ab = m_a m_b / (m_a + m_b),
phi is uniform, and the relative velocity u = v_a - v_b turns by theta about its own direction,
i.e. the velocity difference is eq:du with (theta', phi') = (theta, phi); eq:newv then gives the
new velocities.

Readings (the paper names the method, not these details):
  * Three passes after the elastic passes (or impact ionization) and before field ionization:
    e-e, e-Cu+, Cu+-Cu+ (then e-Cu2+, Cu+-Cu2+, Cu2+-Cu2+ when Cu2+ is simulated), each on the
    cell-sorted SPs with the pairings of the elastic passes (inter-species: fewer SPs project,
    ties the first-named species; like-species: shuffled places (o + 2m, o + 2m + 1) mod N).
  * n is the target species' real density as the pair sees it, n_t W_t (the target SP
    density times the paired target's weight), as in eq:colp.
  * lnL is a constant parameter (default 10): the paper gives no plasma parameter for it.
  * Whole SPs scatter (there is no collision probability to split by): the SP with the smaller
    weight always takes its new velocity, the other with probability w_small / w_large
    (Nanbu-Yonemura), tested exactly in integers on a 24-bit draw; equal weights: both.
  * Draws per pair (Philox stream of the pass, keyed by the projectile's id and the step):
    delta = sqrt(<delta^2>) sqrt(-2 ln U0) cos(2 pi U1) (Box-Muller), phi = 2 pi U2, weight
    test on U3.  cos(theta) = (1 - delta^2) / (1 + delta^2); a pair with u = 0 does not turn.
"""
import math

import numpy as np

from . import constants as C
from . import philox
from .elastic import delta_u

PAIR_EE, DRAW_EE, PAIR_EI, DRAW_EI, PAIR_II, DRAW_II = 16, 17, 18, 19, 20, 21
PAIR_EJ, DRAW_EJ, PAIR_IJ, DRAW_IJ, PAIR_JJ, DRAW_JJ = 26, 27, 28, 29, 30, 31
COULOMB_LOG = 10.0
F32 = np.float32


def delta2(qa, qb, ma, mb, n, coulomb_log, dt, u):
    """<delta^2> of one pair: q_a^2 q_b^2 n lnL dt / (8 pi eps0^2 m_ab^2 u^3)."""
    mab = ma * mb / (ma + mb)
    return (qa * qa * qb * qb * n * coulomb_log * dt) / (8.0 * math.pi * C.EPS0 * C.EPS0 * mab * mab * u ** 3)


def weight_keeps(word, w_small, w_large):
    """U_w < w_small / w_large for U_w = ((word >> 8) + 1/2) 2^-24, exactly in integers."""
    return (2 * (int(word) >> 8) + 1) * int(w_large) < int(w_small) << 25


def _vel(sp_, i):
    return np.array([sp_["vx"][i], sp_["vy"][i], sp_["vz"][i]], dtype=np.float64)


def _put(sp_, i, v):
    sp_["vx"][i], sp_["vy"][i], sp_["vz"][i] = F32(v[0]), F32(v[1]), F32(v[2])


def scatter_pair(vA, vB, qa, qb, ma, mb, n, coulomb_log, dt, words):
    """(v_A', v_B') in float64 from the pair's four draws, or None when u = 0."""
    u_vec = vA - vB
    u = math.sqrt(float(u_vec[0] * u_vec[0] + u_vec[1] * u_vec[1] + u_vec[2] * u_vec[2]))
    if u == 0.0:
        return None
    U = [((int(w) >> 8) + 0.5) * 2.0 ** -24 for w in words]
    d = math.sqrt(delta2(qa, qb, ma, mb, n, coulomb_log, dt, u)) * math.sqrt(-2.0 * math.log(U[0])) \
        * math.cos(2.0 * math.pi * U[1])
    cos_t = (1.0 - d * d) / (1.0 + d * d)
    du = delta_u(u_vec, cos_t, 2.0 * math.pi * U[2])
    mab = ma * mb / (ma + mb)
    return vA + mab / ma * du, vB - mab / mb * du


def _pair(A, ia, B, ib, qa, qb, ma, mb, Nt, V_cell, prm, purpose, step):
    wa, wb = int(A["w"][ia]), int(B["w"][ib])
    if wa <= 0 or wb <= 0:
        return False
    n = Nt / V_cell * (wb * prm["w_min"])
    words = philox.words(prm["seed"], purpose, int(A["id"][ia]), step, np.arange(4))
    out = scatter_pair(_vel(A, ia), _vel(B, ib), qa, qb, ma, mb, n, prm.get("coulomb_log", COULOMB_LOG), prm["dt"],
                       words)
    if out is None:
        return False
    nA, nB = out
    if wa <= wb:
        _put(A, ia, nA)
        if weight_keeps(words[3], wa, wb):
            _put(B, ib, nB)
    else:
        _put(B, ib, nB)
        if weight_keeps(words[3], wb, wa):
            _put(A, ia, nA)
    return True


def _like(grid, prm, S, off, q, m, pair_purpose, draw, step):
    V_cell = grid.dx ** 3
    cnt = np.diff(off)
    events = 0
    for c in np.nonzero(cnt >= 2)[0]:
        N = int(cnt[c])
        o = int(philox.uniform_index(prm["seed"], pair_purpose, c, step, 0, N))
        for k in range(N // 2):
            a, b = off[c] + (o + 2 * k) % N, off[c] + (o + 2 * k + 1) % N
            events += _pair(S, a, S, b, q, q, m, m, N, V_cell, prm, draw, step)
    return events


def coulomb_ee(grid, prm, e, e_off, step):
    """e + e between the electron SPs of each cell (velocities in place); returns events."""
    return _like(grid, prm, e, e_off, -C.E_CHARGE, C.M_E, PAIR_EE, DRAW_EE, step)


def coulomb_ii(grid, prm, i, i_off, step):
    """Cu+ + Cu+ between the ion SPs of each cell; returns events."""
    return _like(grid, prm, i, i_off, C.E_CHARGE, C.M_CU, PAIR_II, DRAW_II, step)


def coulomb_jj(grid, prm, j, j_off, step):
    """Cu2+ + Cu2+ between the Cu2+ SPs of each cell; returns events."""
    return _like(grid, prm, j, j_off, 2.0 * C.E_CHARGE, C.M_CU, PAIR_JJ, DRAW_JJ, step)


def _inter(grid, prm, A, a_off, B, b_off, qa, qb, ma, mb, pair_purpose, draw, step):
    """A + B pairs of every cell holding both (fewer SPs project, ties A); returns events."""
    V_cell = grid.dx ** 3
    cnt_a, cnt_b = np.diff(a_off), np.diff(b_off)
    events = 0
    for c in np.nonzero((cnt_a > 0) & (cnt_b > 0))[0]:
        Na, Nb = int(cnt_a[c]), int(cnt_b[c])
        if Na <= Nb:
            o = int(philox.uniform_index(prm["seed"], pair_purpose, c, step, 0, Nb))
            for k in range(Na):
                events += _pair(A, a_off[c] + k, B, b_off[c] + (k + o) % Nb, qa, qb, ma, mb, Nb, V_cell, prm, draw, step)
        else:
            o = int(philox.uniform_index(prm["seed"], pair_purpose, c, step, 0, Na))
            for k in range(Nb):
                events += _pair(B, b_off[c] + k, A, a_off[c] + (k + o) % Na, qb, qa, mb, ma, Na, V_cell, prm, draw, step)
    return events


def coulomb_ei(grid, prm, e, e_off, i, i_off, step):
    """e + Cu+ pairs (fewer SPs project, ties the electrons); returns events."""
    return _inter(grid, prm, e, e_off, i, i_off, -C.E_CHARGE, C.E_CHARGE, C.M_E, C.M_CU, PAIR_EI, DRAW_EI, step)


def coulomb_ej(grid, prm, e, e_off, j, j_off, step):
    """e + Cu2+ pairs (fewer SPs project, ties the electrons); returns events."""
    return _inter(grid, prm, e, e_off, j, j_off, -C.E_CHARGE, 2.0 * C.E_CHARGE, C.M_E, C.M_CU, PAIR_EJ, DRAW_EJ,
                  step)


def coulomb_ij(grid, prm, i, i_off, j, j_off, step):
    """Cu+ + Cu2+ pairs (fewer SPs project, ties Cu+); returns events."""
    return _inter(grid, prm, i, i_off, j, j_off, C.E_CHARGE, 2.0 * C.E_CHARGE, C.M_CU, C.M_CU, PAIR_IJ, DRAW_IJ, step)
