"""Thermal-field electron emission (test infrastructure only), Sec. 2.3.1.

The paper computes the emitted current density J and the Nottingham heat P_N of each
surface location with the general thermal-field model through GETELEC; neither the code
nor its equations are in the paper, so this is the standard formulation written out
(energies in eV from the Fermi level, lengths in nm, fields in V/nm = GV/m):

  barrier   U(x) = phi - F R x / (R + x) - Q / (x (1 + x / (2R)))      (R = inf: phi - F x - Q/x)
            Q = e^2 / (16 pi eps0) = 0.35999 eV nm, R the local radius of curvature
  Gamow     G(W) = g * int_{x1}^{x2} sqrt(U(x) - W) dx,  g = 2 sqrt(2 m_e) / hbar,
            x1 < x2 the turning points U(x) = W
  transmission  D(W) = 1 / (1 + exp(G(W)))  below the barrier maximum U_m, D = 1 above it,
            D = 0 if the barrier never falls back to W (finite R, W <= phi - F R)
  current   J = z_S * int_{W_lo}^{inf} D(W) kT ln(1 + exp(-W/kT)) dW,  z_S = e m_e / (2 pi^2 hbar^3)
  Nottingham  P_N = z_S * int D(W) I(W) dW,  I(W) = int_W^inf (-E) f_FD(E) dE   [W/m^2]
            (energy deposited per unit area and time; > 0 heats the surface)
  W_lo = -7.0 eV, the bottom of the Cu conduction band (textbook Fermi energy).

`current_density_quad` is the definition evaluated by nested adaptive quadrature.
`current_density_fixed` evaluates the same integrals with fixed-order Gauss-Legendre rules
vectorised over many faces; it is pinned against the adaptive version in the tests.
"""
import math

import numpy as np
import scipy.integrate as si
import scipy.optimize as so
import scipy.special as ss

from . import constants as C

W_LO = -7.0
QI = C.Q_IMAGE_EVNM
G_CONST = C.GAMOW_G
Z_S = C.SOMMERFELD_Z


def barrier(x, F, phi, R):
    x = np.asarray(x, dtype=np.float64)
    if math.isinf(R):
        return phi - F * x - QI / x
    return phi - F * R * x / (R + x) - QI / (x * (1.0 + x / (2.0 * R)))


def barrier_slope(x, F, R):
    if math.isinf(R):
        return -F + QI / x ** 2
    return -F * R * R / (R + x) ** 2 + 2.0 * R * QI * (2.0 * R + 2.0 * x) / (x * x * (2.0 * R + x) ** 2)


def barrier_max(F, phi, R):
    """(x_m, U_m): the single maximum of U for F > 0."""
    lo, hi = 1e-9, 1.0
    while barrier_slope(hi, F, R) > 0:
        hi *= 2.0
    xm = so.brentq(lambda x: barrier_slope(x, F, R), lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    return xm, float(barrier(xm, F, phi, R))


def turning_points(W, F, phi, R, xm):
    """(x1, x2) with U = W on either side of x_m, or (x1, None) if U never returns to W."""
    f = lambda x: float(barrier(x, F, phi, R)) - W
    lo = xm
    while f(lo) > 0:
        lo *= 0.5
    x1 = so.brentq(f, lo, xm, xtol=1e-15, rtol=1e-15, maxiter=500)
    if not math.isinf(R) and phi - F * R >= W:
        return x1, None
    hi = xm * 2.0
    while f(hi) > 0:
        hi *= 2.0
    x2 = so.brentq(f, xm, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    return x1, x2


def gamow(W, F, phi, R, xm):
    x1, x2 = turning_points(W, F, phi, R, xm)
    if x2 is None:
        return math.inf
    val, _ = si.quad(lambda x: math.sqrt(max(float(barrier(x, F, phi, R)) - W, 0.0)), x1, x2,
                     epsabs=0.0, epsrel=1e-12, limit=200)
    return G_CONST * val


def transmission(W, F, phi, R, xm, Um):
    if W >= Um:
        return 1.0
    G = gamow(W, F, phi, R, xm)
    if math.isinf(G) or G > 700:
        return 0.0 if math.isinf(G) else math.exp(-G)
    return 1.0 / (1.0 + math.exp(G))


def supply(W, kT):
    """kT ln(1 + exp(-W/kT)) [eV], overflow-free."""
    w = np.asarray(W, dtype=np.float64) / kT
    return kT * (np.maximum(-w, 0.0) + np.log1p(np.exp(-np.abs(w))))


def _L(w):
    """L(w) = int_w^inf ln(1 + e^-t) dt = -Li2(-e^-w) = sum_k (-1)^(k+1) x^k / k^2, x = e^-w, w >= 0.
    The power series is used for x <= 1/2 (spence(1 + x) would lose x when 1 + x rounds to 1);
    scipy's spence (Li2(z) = spence(1 - z)) for 1/2 < x <= 1."""
    w = np.asarray(w, dtype=np.float64)
    x = np.exp(-w)
    k = np.arange(1, 61, dtype=np.float64)
    xs = np.minimum(x, 0.5)
    series = np.sum(((-1.0) ** (k + 1)) * xs[..., None] ** k / (k * k), axis=-1)
    return np.where(x <= 0.5, series, -ss.spence(1.0 + x))


def nottingham_inner(W, kT):
    """I(W) = int_W^inf (-E) / (1 + exp(E/kT)) dE [eV^2] in closed form through the dilogarithm:
    w >= 0:  -(kT)^2 [w ln(1+e^-w) + L(w)];   w < 0:  (kT)^2 [w^2/2 - pi^2/6 - w ln(1+e^w) + L(-w)].
    W and kT broadcast."""
    Wb, kTb = np.broadcast_arrays(np.asarray(W, dtype=np.float64), np.asarray(kT, dtype=np.float64))
    w = np.atleast_1d(Wb / kTb)
    k2 = np.atleast_1d(kTb) ** 2
    out = np.empty_like(w)
    p = w >= 0
    wp = w[p]
    out[p] = -k2[p] * (wp * np.log1p(np.exp(-wp)) + _L(wp))
    wn = w[~p]
    out[~p] = k2[~p] * (0.5 * wn * wn - math.pi ** 2 / 6.0 - wn * np.log1p(np.exp(wn)) + _L(-wn))
    return out if np.ndim(Wb) else out[0]


def nottingham_inner_quad(W, kT):
    """I(W) straight from its definition (used to pin the closed form)."""
    f = lambda E: -E / (1.0 + math.exp(min(E / kT, 700.0)))
    hi = max(W, 0.0) + 80.0 * kT
    pts = [0.0] if W < 0.0 < hi else None
    val, _ = si.quad(f, W, hi, epsabs=0.0, epsrel=1e-13, limit=400, points=pts)
    return val


def current_density_quad(F_GV, T, phi, R_nm):
    """(J [A/m^2], P_N [W/m^2]) by nested adaptive quadrature of the definitions above."""
    F = float(F_GV)
    if F <= 0.0:
        return 0.0, 0.0
    kT = C.K_B_EV * float(T)
    R = float(R_nm)
    xm, Um = barrier_max(F, phi, R)
    top = max(Um, W_LO)
    Jint, Pint = 0.0, 0.0
    if Um > W_LO:
        pts = [0.0] if W_LO < 0.0 < Um else None
        D = lambda W: transmission(W, F, phi, R, xm, Um)
        Jint += si.quad(lambda W: D(W) * float(supply(W, kT)), W_LO, Um, epsabs=0.0, epsrel=1e-10,
                        limit=400, points=pts)[0]
        Pint += si.quad(lambda W: D(W) * float(nottingham_inner(W, kT)), W_LO, Um, epsabs=0.0,
                        epsrel=1e-10, limit=400, points=pts)[0]
    # above the maximum D = 1; the integrands fall as exp(-W/kT), so 100 kT closes the tail
    Jint += si.quad(lambda W: float(supply(W, kT)), top, top + 100.0 * kT, epsabs=0.0, epsrel=1e-12,
                    limit=400)[0]
    Pint += si.quad(lambda W: float(nottingham_inner(W, kT)), top, top + 100.0 * kT, epsabs=0.0,
                    epsrel=1e-12, limit=400)[0]
    return Z_S * Jint, Z_S * Pint


# --------------------------------------------------------------------------------------
# vectorised fixed-order evaluation of the same integrals
# --------------------------------------------------------------------------------------
_GL8 = np.polynomial.legendre.leggauss(8)
_GL48 = np.polynomial.legendre.leggauss(48)


def _barrier_v(x, F, phi, R):
    finite = np.isfinite(R)
    Rs = np.where(finite, R, 1.0)
    curved = phi - F * Rs * x / (Rs + x) - QI / (x * (1.0 + x / (2.0 * Rs)))
    plane = phi - F * x - QI / x
    return np.where(finite, curved, plane)


def _slope_v(x, F, R):
    finite = np.isfinite(R)
    Rs = np.where(finite, R, 1.0)
    curved = -F * Rs * Rs / (Rs + x) ** 2 + 2.0 * Rs * QI * (2.0 * Rs + 2.0 * x) / (x * x * (2.0 * Rs + x) ** 2)
    plane = -F + QI / (x * x)
    return np.where(finite, curved, plane)


def _supply_v(W, kT):
    w = W / kT
    return kT * (np.maximum(-w, 0.0) + np.log1p(np.exp(-np.abs(w))))


def _bisect(fun, lo, hi, iters=200):
    """Vectorised bisection; fun(lo) and fun(hi) have opposite signs (sign of lo kept)."""
    slo = np.sign(fun(lo))
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        s = np.sign(fun(mid))
        same = s == slo
        lo = np.where(same, mid, lo)
        hi = np.where(same, hi, mid)
        if np.all(np.abs(hi - lo) <= 1e-15 * np.abs(hi)):
            break
    return 0.5 * (lo + hi)


def current_density_fixed(F_GV, T, phi, R_nm, panels=160):
    """Vectorised (J, P_N) for arrays of faces: 8-point Gauss-Legendre on the panels between
    breakpoints over [W_lo, U_m] -- `panels` equal panels, refined by geometric breakpoints
    toward the Fermi level (steps kT 2^j) and toward the barrier top (steps min(kT, hbar omega/2)
    2^j, omega the curvature frequency of the top) --, 48-point Gauss-Legendre in the
    Chebyshev-type angle for G(W), and 24 panels of 8 points over [U_m, U_m + 60 kT] for the
    part above the barrier."""
    F = np.atleast_1d(np.asarray(F_GV, dtype=np.float64))
    T = np.broadcast_to(np.asarray(T, dtype=np.float64), F.shape)
    phi = np.broadcast_to(np.asarray(phi, dtype=np.float64), F.shape)
    R = np.broadcast_to(np.asarray(R_nm, dtype=np.float64), F.shape)
    J = np.zeros(F.shape)
    PN = np.zeros(F.shape)
    act = F > 0
    if not np.any(act):
        return J, PN
    F, T, phi, R = F[act], T[act], phi[act], R[act]
    kT = C.K_B_EV * T
    # barrier maximum
    hi = np.ones_like(F)
    for _ in range(80):
        hi = np.where(_slope_v(hi, F, R) > 0, 2.0 * hi, hi)
    xm = _bisect(lambda x: _slope_v(x, F, R), np.full_like(F, 1e-9), hi)
    Um = _barrier_v(xm, F, phi, R)
    top = np.maximum(Um, W_LO)
    # below the barrier maximum: breakpoints (equal + graded), 8-point rule on every panel
    xg, wg = _GL8
    d = 1e-4 * xm
    d2U = (_slope_v(xm + d, F, R) - _slope_v(xm - d, F, R)) / (2 * d)
    hw = np.sqrt(8.0 * np.abs(d2U)) / G_CONST                  # hbar omega at the top [eV]
    steps = 2.0 ** np.arange(40) - 1.0
    span = (top - W_LO)[:, None]
    bp = np.concatenate([
        W_LO + span * np.linspace(0.0, 1.0, panels + 1)[None, :],
        top[:, None] - np.minimum(kT, 0.5 * hw)[:, None] * steps[None, :],
        kT[:, None] * steps[None, :],
        -kT[:, None] * steps[None, :]], axis=1)
    bp = np.sort(np.clip(bp, W_LO, top[:, None]), axis=1)
    a_, b_ = bp[:, :-1], bp[:, 1:]
    h = 0.5 * (b_ - a_)
    Wn = (0.5 * (a_ + b_))[:, :, None] + h[:, :, None] * xg[None, None, :]
    Wn = Wn.reshape(len(F), -1)
    Ww = (h[:, :, None] * wg[None, None, :]).reshape(len(F), -1)
    Fb, phib, Rb, xmb = (a[:, None] * np.ones_like(Wn) for a in (F, phi, R, xm))
    below = Wn < Um[:, None]
    # x1 in (0, xm]
    lo1 = xmb.copy()
    for _ in range(200):
        m = _barrier_v(lo1, Fb, phib, Rb) > Wn
        if not np.any(m):
            break
        lo1 = np.where(m, 0.5 * lo1, lo1)
    x1 = _bisect(lambda x: _barrier_v(x, Fb, phib, Rb) - Wn, lo1, xmb)
    finite = np.isfinite(Rb)
    open_ = ~finite | (phib - Fb * np.where(finite, Rb, 0.0) < Wn)
    hi2 = 2.0 * xmb
    for _ in range(200):
        m = open_ & (_barrier_v(hi2, Fb, phib, Rb) > Wn)
        if not np.any(m):
            break
        hi2 = np.where(m, 2.0 * hi2, hi2)
    x2 = _bisect(lambda x: _barrier_v(x, Fb, phib, Rb) - Wn, xmb, hi2)
    tg, tw = _GL48
    th = 0.5 * math.pi * (tg + 1.0)
    mid = 0.5 * (x1 + x2)
    half = 0.5 * (x2 - x1)
    xs = mid[..., None] - half[..., None] * np.cos(th)
    U = _barrier_v(xs, Fb[..., None], phib[..., None], Rb[..., None])
    integrand = np.sqrt(np.maximum(U - Wn[..., None], 0.0)) * half[..., None] * np.sin(th)
    G = G_CONST * 0.5 * math.pi * np.sum(integrand * tw, axis=-1)
    D = np.where(open_, 1.0 / (1.0 + np.exp(np.minimum(G, 700.0))), 0.0)
    D = np.where(below, D, 1.0)
    kTb = kT[:, None] * np.ones_like(Wn)
    Jint = np.sum(Ww * D * _supply_v(Wn, kTb), axis=1)
    Iw = nottingham_inner(Wn, kT[:, None])
    Pint = np.sum(Ww * D * Iw, axis=1)
    # above the barrier maximum (D = 1)
    npan = 24
    span = 60.0 * kT
    e2 = np.linspace(0.0, 1.0, npan + 1)
    h2 = span[:, None] / npan
    Wa = (top[:, None] + span[:, None] * e2[None, :-1])[:, :, None] + h2[:, :, None] * (0.5 * (xg + 1.0))[None, None, :]
    Wa = Wa.reshape(len(F), -1)
    Wwa = ((h2 * 0.5)[:, :, None] * wg[None, None, :] * np.ones((1, npan, 1))).reshape(len(F), -1)
    kTa = kT[:, None] * np.ones_like(Wa)
    Jint += np.sum(Wwa * _supply_v(Wa, kTa), axis=1)
    Pint += np.sum(Wwa * nottingham_inner(Wa, kT[:, None]), axis=1)
    J[act] = Z_S * Jint
    PN[act] = Z_S * Pint
    return J, PN
