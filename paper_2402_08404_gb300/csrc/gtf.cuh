// General thermal-field emission current density and Nottingham heat (Sec. 2.3.1; the paper
// uses GETELEC, whose equations it does not print, so this is the standard formulation).
// Energies in eV from the Fermi level, lengths in nm, fields in V/nm (= GV/m):
//   barrier  U(x) = phi - F R x/(R+x) - Q/(x (1 + x/(2R)))   (flat surface: phi - F x - Q/x)
//   Gamow    G(W) = g int_{x1}^{x2} sqrt(U - W) dx,  D(W) = 1/(1+exp G) below the barrier top, 1 above
//   J  = z_S int_{W_lo}^inf D(W) kT ln(1 + exp(-W/kT)) dW                         [A/m^2]
//   PN = z_S int D(W) I(W) dW,  I(W) = int_W^inf (-E) f_FD(E) dE                   [W/m^2]
// Numerical scheme (float64): turning points in closed form (flat) or by safeguarded Newton
// (curved); G by 32-point Gauss-Legendre in the angle of x = m - h cos(theta); W integrals by
// 16-point Gauss-Legendre panels graded geometrically away from the Fermi level (first width
// 4 kT), from the barrier top (first width min(4 kT, hbar omega/2), omega the curvature
// frequency of the top) and from phi - F R where a curved barrier stops closing; the below-E_F
// tail stops once a panel adds < 1e-18 relative.
// The part above the barrier top has J in closed form through the dilogarithm (Bernoulli
// series); I(W) likewise.
#pragma once
#include <math.h>

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

namespace gtf {

struct Consts {
  double Q;       // e^2/(16 pi eps0) [eV nm]
  double g;       // 2 sqrt(2 m_e)/hbar [eV^-1/2 nm^-1]
  double zS;      // e m_e/(2 pi^2 hbar^3) [A m^-2 eV^-2]
  double kB;      // eV/K
  double Wlo;     // bottom of the conduction band [eV]
};

struct Tables {
  const double *x16, *w16;   // Gauss-Legendre on [-1,1]
  const double *x32, *w32;
  const double *c32, *s32;   // cos and sin of the angles pi/2 (x32 + 1)
};

struct Barrier {
  double F, phi, R;
  bool flat;
  double Q;
};

__host__ __device__ inline double U(const Barrier &b, double x) {
  if (b.flat) return b.phi - b.F * x - b.Q / x;
  return b.phi - b.F * b.R * x / (b.R + x) - b.Q / (x * (1.0 + x / (2.0 * b.R)));
}

__host__ __device__ inline double dU(const Barrier &b, double x) {
  if (b.flat) return -b.F + b.Q / (x * x);
  const double rx = b.R + x, r2x = 2.0 * b.R + x;
  return -b.F * b.R * b.R / (rx * rx) + 2.0 * b.R * b.Q * (2.0 * b.R + 2.0 * x) / (x * x * r2x * r2x);
}

// Li2(-x) for 0 <= x <= 1: Bernoulli series in u = -ln(1+x), |u| <= ln 2.
__host__ __device__ inline double li2_neg(double x) {
  const double u = -log1p(x);
  const double u2 = u * u;
  // B_n/(n+1)! for n = 2, 4, ..., 18
  const double c[9] = {1.0 / 36.0, -1.0 / 3600.0, 1.0 / 211680.0, -1.0 / 10886400.0, 1.0 / 526901760.0,
                       -4.064761645144226e-11, 8.921691020456453e-13, -1.993929586072108e-14,
                       4.518980029619918e-16};
  double s = 0.0, p = u * u2;
  for (int k = 0; k < 9; ++k) { s += c[k] * p; p *= u2; }
  return u - 0.25 * u2 + s;
}

// L(w) = int_w^inf ln(1 + e^-t) dt = -Li2(-e^-w), w >= 0
__host__ __device__ inline double Lw(double w) { return -li2_neg(exp(-w)); }

__host__ __device__ inline double supply(double W, double kT) {
  const double w = W / kT;
  return kT * (fmax(-w, 0.0) + log1p(exp(-fabs(w))));
}

// I(W) = int_W^inf (-E)/(1+exp(E/kT)) dE [eV^2]
__host__ __device__ inline double inner(double W, double kT) {
  const double w = W / kT, k2 = kT * kT;
  if (w >= 0.0) return -k2 * (w * log1p(exp(-w)) + Lw(w));
  return k2 * (0.5 * w * w - 1.6449340668482264 - w * log1p(exp(w)) + Lw(-w));
}

// int_top^inf supply(W) dW, closed form
__host__ __device__ inline double supply_tail(double top, double kT) {
  const double wt = top / kT, k2 = kT * kT;
  if (wt >= 0.0) return k2 * Lw(wt);
  return k2 * (0.5 * wt * wt + 1.6449340668482264 - Lw(-wt));
}

// root of U(x) = W in [lo, hi] (U - W changes sign), safeguarded Newton from x0
__host__ __device__ inline double root(const Barrier &b, double W, double lo, double hi, double x0) {
  const double flo = U(b, lo) - W;
  double x = (x0 > lo && x0 < hi) ? x0 : 0.5 * (lo + hi);
  for (int it = 0; it < 100; ++it) {
    const double f = U(b, x) - W;
    if (f == 0.0) return x;
    if ((f < 0.0) == (flo < 0.0)) lo = x; else hi = x;
    const double d = dU(b, x);
    double xn = x - f / d;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    if (fabs(xn - x) <= 1e-15 * fabs(xn) || hi - lo <= 1e-15 * hi) return xn;
    x = xn;
  }
  return x;
}

// barrier maximum (x_m, U_m)
__host__ __device__ inline void barrier_top(const Barrier &b, double *xm, double *Um) {
  if (b.flat) {
    *xm = sqrt(b.Q / b.F);
  } else {
    double lo = 1e-9, hi = 1.0;
    for (int i = 0; i < 200 && dU(b, hi) > 0.0; ++i) hi *= 2.0;
    for (int i = 0; i < 200; ++i) {
      const double mid = 0.5 * (lo + hi);
      if (dU(b, mid) > 0.0) lo = mid; else hi = mid;
      if (hi - lo <= 1e-15 * hi) break;
    }
    *xm = 0.5 * (lo + hi);
  }
  *Um = U(b, *xm);
}

// transmission D(W) for W below the barrier top
__host__ __device__ inline double transmission(const Barrier &b, const Consts &C, const Tables &T, double W,
                                               double xm) {
  double x1, x2;
  const double a = b.phi - W;
  const double disc = a * a - 4.0 * b.Q * b.F;
  if (b.flat) {
    const double sq = sqrt(fmax(disc, 0.0));
    x1 = 2.0 * b.Q / (a + sq);
    x2 = (a + sq) / (2.0 * b.F);
  } else {
    if (b.phi - b.F * b.R >= W) return 0.0;          // the barrier never comes back down to W
    const double sq = sqrt(fmax(disc, 0.0));
    double lo = xm;
    for (int i = 0; i < 200 && U(b, lo) > W; ++i) lo *= 0.5;
    x1 = root(b, W, lo, xm, disc > 0 ? 2.0 * b.Q / (a + sq) : 0.5 * xm);
    const double s = a / (b.F * b.R);
    const double hi = 2.0 * s * b.R / (1.0 - s) + 2.0 * xm;
    x2 = root(b, W, xm, hi, disc > 0 ? (a + sq) / (2.0 * b.F) : 2.0 * xm);
  }
  const double m = 0.5 * (x1 + x2), h = 0.5 * (x2 - x1);
  double s = 0.0;
  for (int i = 0; i < 32; ++i) {
    const double x = m - h * T.c32[i];
    s += T.w32[i] * sqrt(fmax(U(b, x) - W, 0.0)) * T.s32[i];
  }
  const double G = C.g * 1.5707963267948966 * h * s;
  return G > 700.0 ? exp(-G) : 1.0 / (1.0 + exp(G));
}

struct Acc { double J, P; };

// panel [a, b] with 16-point Gauss-Legendre; below the barrier top
__host__ __device__ inline Acc panel_below(const Barrier &br, const Consts &C, const Tables &T, double a, double b,
                                           double kT, double xm) {
  Acc r = {0.0, 0.0};
  const double c = 0.5 * (a + b), hw = 0.5 * (b - a);
  for (int i = 0; i < 16; ++i) {
    const double W = c + hw * T.x16[i];
    const double D = transmission(br, C, T, W, xm);
    r.J += T.w16[i] * D * supply(W, kT);
    r.P += T.w16[i] * D * inner(W, kT);
  }
  r.J *= hw;
  r.P *= hw;
  return r;
}

// (J [A/m^2], PN [W/m^2]); F in V/nm, T in K, phi in eV, R in nm (R <= 0 or not finite: flat)
__host__ __device__ inline void current_density(const Consts &C, const Tables &T, double F, double Temp, double phi,
                                                double R, double *J_out, double *P_out, int *n_eval = nullptr) {
  if (!(F > 0.0)) { *J_out = 0.0; *P_out = 0.0; return; }
  Barrier b;
  b.F = F; b.phi = phi; b.Q = C.Q;
  b.flat = !(R > 0.0) || !isfinite(R);
  b.R = b.flat ? 1.0 : R;
  const double kT = C.kB * Temp;
  double xm, Um;
  barrier_top(b, &xm, &Um);
  const double top = fmax(Um, C.Wlo);
  // above the top (D = 1)
  double J = supply_tail(top, kT);
  double P = 0.0;
  {
    double lo = top, w = 4.0 * kT;
    for (int p = 0; p < 5; ++p) {     // 4, 8, 16, 32 kT panels and a last one to 64 kT past the top
      const double hi = lo + w;
      const double c = 0.5 * (lo + hi), hw = 0.5 * (hi - lo);
      double s = 0.0;
      for (int i = 0; i < 16; ++i) s += T.w16[i] * inner(c + hw * T.x16[i], kT);
      P += hw * s;
      lo = hi;
      w = p < 3 ? 2.0 * w : 4.0 * kT * 4.0;
    }
  }
  const double h0 = 4.0 * kT;
  // curvature of the top: hbar omega = sqrt(8 |U''|)/g  (hbar^2/2m = 4/g^2)
  const double dlt = 1e-4 * xm;
  const double d2U = (dU(b, xm + dlt) - dU(b, xm - dlt)) / (2.0 * dlt);
  const double htop = fmin(h0, 0.5 * sqrt(8.0 * fabs(d2U)) / C.g);
  // below W_cut a curved barrier never closes again (D = 0)
  const double Wcut = b.flat ? C.Wlo : fmax(C.Wlo, b.phi - b.F * b.R);
  // [max(0, W_cut), top]: graded from both ends toward the middle
  if (top > 0.0 && top > Wcut) {
    const double A = fmax(0.0, Wcut), B = top, M = 0.5 * (A + B);
    for (int side = 0; side < 2; ++side) {
      double w = side == 0 ? h0 : htop, pos = side == 0 ? A : B;
      for (int it = 0; it < 64; ++it) {
        const double nxt = side == 0 ? fmin(pos + w, M) : fmax(pos - w, M);
        const Acc r = side == 0 ? panel_below(b, C, T, pos, nxt, kT, xm) : panel_below(b, C, T, nxt, pos, kT, xm);
        J += r.J; P += r.P;
        if (n_eval) *n_eval += 16;
        pos = nxt;
        if (pos == M) break;
        w *= 2.0;
      }
    }
  }
  // [W_cut, min(0, top)]: graded downward from the upper end, stops when negligible
  {
    const double B = fmin(0.0, top);
    if (B > Wcut) {
      double w = B == top ? htop : h0, pos = B;
      for (int it = 0; it < 64; ++it) {
        const double nxt = fmax(pos - w, Wcut);
        const Acc r = panel_below(b, C, T, nxt, pos, kT, xm);
        J += r.J; P += r.P;
        if (n_eval) *n_eval += 16;
        pos = nxt;
        if (pos == Wcut) break;
        if (it >= 1 && fabs(r.J) <= 1e-18 * fabs(J) && fabs(r.P) <= 1e-18 * fabs(P)) break;
        w *= 2.0;
      }
    }
  }
  *J_out = C.zS * J;
  *P_out = C.zS * P;
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on the Legendre recurrence; host only).
inline void gauss_legendre(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(3.141592653589793 * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

}  // namespace gtf
