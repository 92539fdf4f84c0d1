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
  const float *w32f, *c32f, *s32f;   // the same in FP32 (transmission_f32)
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

// The same D(W) with the turning points and the Gamow quadrature in FP32 (the exponent and
// D itself in FP64).  U - W is formed as (phi - W) - (image and field terms) with phi - W taken
// in FP64 first, so the cancellation near the turning points costs ~1e-7 eV; relative error of
// G ~1e-6, of D ~1e-6 G.  On GB300 an FP32 operation is ~64x cheaper than an FP64 one.
__host__ __device__ inline float uw_f32(bool flat, float a, float F, float R, float Q, float x) {
  if (flat) return a - F * x - Q / x;
  return a - F * R * x / (R + x) - 2.0f * R * Q / (x * (2.0f * R + x));
}

__host__ __device__ inline float duw_f32(bool flat, float F, float R, float Q, float x) {
  if (flat) return -F + Q / (x * x);
  const float rx = R + x, r2x = 2.0f * R + x;
  return -F * R * R / (rx * rx) + 2.0f * R * Q * (2.0f * R + 2.0f * x) / (x * x * r2x * r2x);
}

// root of U(x) - W = 0 in [lo, hi], safeguarded Newton in FP32
__host__ __device__ inline float root_f32(bool flat, float a, float F, float R, float Q, float lo, float hi, float x0) {
  const float flo = uw_f32(flat, a, F, R, Q, lo);
  float x = (x0 > lo && x0 < hi) ? x0 : 0.5f * (lo + hi);
  for (int it = 0; it < 60; ++it) {
    const float f = uw_f32(flat, a, F, R, Q, x);
    if (f == 0.0f) return x;
    if ((f < 0.0f) == (flo < 0.0f)) lo = x; else hi = x;
    float xn = x - f / duw_f32(flat, F, R, Q, x);
    if (!(xn > lo && xn < hi)) xn = 0.5f * (lo + hi);
    if (fabsf(xn - x) <= 2e-7f * fabsf(xn) || hi - lo <= 2e-7f * hi) return xn;
    x = xn;
  }
  return x;
}

__host__ __device__ inline double transmission_f32(const Barrier &b, const Consts &C, const Tables &T, double W,
                                                   double xm) {
  const double a = b.phi - W;
  const double disc = a * a - 4.0 * b.Q * b.F;
  double x1, x2;
  const float af = (float)a, Ff = (float)b.F, Rf = (float)b.R, Qf = (float)b.Q;
  if (b.flat) {
    const double sq = sqrt(fmax(disc, 0.0));
    x1 = 2.0 * b.Q / (a + sq);
    x2 = (a + sq) / (2.0 * b.F);
  } else {
    if (b.phi - b.F * b.R >= W) return 0.0;
    const double sq = sqrt(fmax(disc, 0.0));
    float lo = (float)xm;
    for (int i = 0; i < 200 && uw_f32(false, af, Ff, Rf, Qf, lo) > 0.0f; ++i) lo *= 0.5f;
    x1 = root_f32(false, af, Ff, Rf, Qf, lo, (float)xm, disc > 0 ? (float)(2.0 * b.Q / (a + sq)) : 0.5f * (float)xm);
    const double s = a / (b.F * b.R);
    const double hi = 2.0 * s * b.R / (1.0 - s) + 2.0 * xm;
    x2 = root_f32(false, af, Ff, Rf, Qf, (float)xm, (float)hi, disc > 0 ? (float)((a + sq) / (2.0 * b.F)) : 2.0f * (float)xm);
  }
  const float m = (float)(0.5 * (x1 + x2)), h = (float)(0.5 * (x2 - x1));
  float s = 0.0f;
  for (int i = 0; i < 32; ++i) {
    const float x = m - h * T.c32f[i];
    s += T.w32f[i] * sqrtf(fmaxf(uw_f32(b.flat, af, Ff, Rf, Qf, x), 0.0f)) * T.s32f[i];
  }
  const double G = C.g * 1.5707963267948966 * (double)h * (double)s;
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

#ifdef __CUDACC__
__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP32 forms of the supply function and of I(W) for the FAST_INTEGRAL path: the same formulas
// with float transcendentals (~1e-7 relative per value; the panel sums stay in FP64).  On this
// part FP64 runs at 1/64 of the FP32 rate, and these two functions dominate an evaluation.
__host__ __device__ inline float li2_neg_f(float x) {
  const float u = -log1pf(x);
  const float u2 = u * u;
  // B_n/(n+1)! for n = 2, 4, 6, 8 (|u| <= ln 2: the next terms are below FP32 resolution)
  const float s = u * u2 * (1.0f / 36.0f + u2 * (-1.0f / 3600.0f + u2 * (1.0f / 211680.0f + u2 * (-1.0f / 10886400.0f))));
  return u - 0.25f * u2 + s;
}
__host__ __device__ inline float Lw_f(float w) { return -li2_neg_f(expf(-w)); }
__host__ __device__ inline float supply_f(float W, float kT) {
  const float w = W / kT;
  return kT * (fmaxf(-w, 0.0f) + log1pf(expf(-fabsf(w))));
}
__host__ __device__ inline float inner_f(float W, float kT) {
  const float w = W / kT, k2 = kT * kT;
  if (w >= 0.0f) return -k2 * (w * log1pf(expf(-w)) + Lw_f(w));
  return k2 * (0.5f * w * w - 1.6449340668f - w * log1pf(expf(w)) + Lw_f(-w));
}
// FP32 only where it cannot underflow: for W/kT > 80 both functions fall like e^{-W/kT} below
// the FP32 range, and those energies take the FP64 forms.
template <bool kFast>
__host__ __device__ __forceinline__ double supply_sel(double W, double kT) {
  return (kFast && W < 80.0 * kT) ? (double)supply_f((float)W, (float)kT) : supply(W, kT);
}
template <bool kFast>
__host__ __device__ __forceinline__ double inner_sel(double W, double kT) {
  return (kFast && W < 80.0 * kT) ? (double)inner_f((float)W, (float)kT) : inner(W, kT);
}


// The same integrals and panels as current_density, evaluated by a whole warp for one face: the
// 32 lanes split the (panel, node) work items and sum with a fixed butterfly, so a few faces
// still fill the FP64 pipes.  Every lane must call it with the same arguments; every lane gets
// the result.  The below-E_F tail is taken two panels per round with the same exit test.
template <bool kFast>
__device__ __forceinline__ double transmission_sel(const Barrier &b, const Consts &C, const Tables &T, double W,
                                                   double xm) {
  return kFast ? transmission_f32(b, C, T, W, xm) : transmission(b, C, T, W, xm);
}

// Barrier maximum for the fast path: bisection on dU in FP32 to ~1e-7 relative (the FP64
// bisection of barrier_top takes ~50 steps on a pipe 64x slower), then two FP64 Newton steps on
// dU = 0 with a central-difference second derivative.
__device__ inline void barrier_top_fast(const Barrier &b, double *xm, double *Um) {
  if (b.flat) {
    *xm = sqrt(b.Q / b.F);
    *Um = U(b, *xm);
    return;
  }
  const float Ff = (float)b.F, Rf = (float)b.R, Qf = (float)b.Q;
  float lo = 1e-9f, hi = 1.0f;
  for (int i = 0; i < 60 && duw_f32(false, Ff, Rf, Qf, hi) > 0.0f; ++i) hi *= 2.0f;
  for (int i = 0; i < 60; ++i) {
    const float mid = 0.5f * (lo + hi);
    if (duw_f32(false, Ff, Rf, Qf, mid) > 0.0f) lo = mid; else hi = mid;
    if (hi - lo <= 2e-7f * hi) break;
  }
  double x = 0.5 * ((double)lo + (double)hi);
  for (int it = 0; it < 2; ++it) {
    const double dl = 1e-4 * x;
    const double d2 = (dU(b, x + dl) - dU(b, x - dl)) / (2.0 * dl);
    if (d2 < 0.0) {
      const double xn = x - dU(b, x) / d2;
      if (xn > 0.5 * x && xn < 2.0 * x) x = xn;
    }
  }
  *xm = x;
  *Um = U(b, x);
}

// Fast path of one energy node: D(W) supply(W) and D(W) I(W) with the turning points, the Gamow
// quadrature, D and the two Fermi functions in FP32, and FP64 only where FP32 would underflow.
// G is the same FP32 Gamow exponent as transmission_f32's.  Where D or the Fermi factors fall
// below the FP32 range (G >= 80 or W >= 80 kT), the product is formed in log space with one
// FP64 exp: for W >= 80 kT, supply = kT e^{-w} and I = -(kT)^2 (w + 1) e^{-w} to within e^{-w}.
__device__ inline void eval_fast(const Barrier &b, const Consts &C, const Tables &T, double W, double xm, double kT,
                                 double inv_kT, double phimFR, double *DS, double *DI) {
  *DS = 0.0;
  *DI = 0.0;
  const double ad = b.phi - W;   // FP64 first: the cancellation near the turning points
  const float af = (float)ad, Ff = (float)b.F, Rf = (float)b.R, Qf = (float)b.Q;
  float x1, x2;
  const float disc = af * af - 4.0f * Qf * Ff;
  const float sq = sqrtf(fmaxf(disc, 0.0f));
  if (b.flat) {
    x1 = 2.0f * Qf / (af + sq);
    x2 = (af + sq) / (2.0f * Ff);
  } else {
    if (phimFR >= W) return;   // the barrier never comes back down to W
    const float xmf = (float)xm;
    float lo = xmf;
    for (int i = 0; i < 200 && uw_f32(false, af, Ff, Rf, Qf, lo) > 0.0f; ++i) lo *= 0.5f;
    x1 = root_f32(false, af, Ff, Rf, Qf, lo, xmf, disc > 0.0f ? 2.0f * Qf / (af + sq) : 0.5f * xmf);
    const float sr = af / (Ff * Rf);
    const float hi = 2.0f * sr * Rf / (1.0f - sr) + 2.0f * xmf;
    x2 = root_f32(false, af, Ff, Rf, Qf, xmf, hi, disc > 0.0f ? (af + sq) / (2.0f * Ff) : 2.0f * xmf);
  }
  const float m = 0.5f * (x1 + x2), h = 0.5f * (x2 - x1);
  float sg = 0.0f;
  for (int i = 0; i < 32; ++i) {
    const float x = m - h * T.c32f[i];
    sg += T.w32f[i] * sqrtf(fmaxf(uw_f32(b.flat, af, Ff, Rf, Qf, x), 0.0f)) * T.s32f[i];
  }
  const float G = (float)C.g * 1.5707963267948966f * h * sg;
  const double w = W * inv_kT;
  if (w < 80.0) {
    const float Wf = (float)W, kTf = (float)kT;
    const double S = (double)supply_f(Wf, kTf), I = (double)inner_f(Wf, kTf);
    const double D = G < 80.0f ? (double)(1.0f / (1.0f + expf(G))) : exp(-(double)G);
    *DS = D * S;
    *DI = D * I;
  } else {
    const double lnD = G < 80.0f ? -(double)log1pf(expf(G)) : -(double)G;
    const double e = exp(lnD - w);
    *DS = kT * e;
    *DI = -(kT * kT) * (w + 1.0) * e;
  }
}

// kFast: transmission_f32 at every node (J, P_N to ~1e-5 relative); else all FP64
template <bool kFast>
__device__ inline void current_density_warp(const Consts &C, const Tables &T, double F, double Temp, double phi,
                                            double R, double *J_out, double *P_out, int *n_eval = nullptr) {
  const int lane = threadIdx.x & 31;
  if (!(F > 0.0)) { *J_out = 0.0; *P_out = 0.0; return; }
  Barrier b;
  b.F = F; b.phi = phi; b.Q = C.Q;
  b.flat = !(R > 0.0) || !isfinite(R);
  b.R = b.flat ? 1.0 : R;
  const double kT = C.kB * Temp, inv_kT = 1.0 / kT;
  const double phimFR = b.flat ? -1e300 : b.phi - b.F * b.R;   // W at or below it: D = 0 (curved)
  double xm, Um;
  if (kFast) barrier_top_fast(b, &xm, &Um);
  else barrier_top(b, &xm, &Um);
  const double top = fmax(Um, C.Wlo);
  double J = supply_tail(top, kT);
  // above the top: panels of 4, 8, 16, 32, 16 kT, 16 nodes each
  double Pl = 0.0;
  for (int q = lane; q < 80; q += 32) {
    const int p = q >> 4, i = q & 15;
    const double lo = top + kT * (p == 0 ? 0.0 : p == 1 ? 4.0 : p == 2 ? 12.0 : p == 3 ? 28.0 : 60.0);
    const double wd = kT * (p == 0 ? 4.0 : p == 1 ? 8.0 : p == 2 ? 16.0 : p == 3 ? 32.0 : 16.0);
    const double c = lo + 0.5 * wd, hw = 0.5 * wd;
    Pl += hw * T.w16[i] * inner_sel<kFast>(c + hw * T.x16[i], kT);
  }
  double P = warp_sum_d(Pl);
  const double h0 = 4.0 * kT;
  const double dlt = 1e-4 * xm;
  const double d2U = (dU(b, xm + dlt) - dU(b, xm - dlt)) / (2.0 * dlt);
  const double htop = fmin(h0, 0.5 * sqrt(8.0 * fabs(d2U)) / C.g);
  const double Wcut = b.flat ? C.Wlo : fmax(C.Wlo, b.phi - b.F * b.R);
  int nev = 0;
  // [max(0, W_cut), top], graded from both ends toward the middle
  if (top > 0.0 && top > Wcut) {
    const double A = fmax(0.0, Wcut), B = top, M = 0.5 * (A + B);
    int nA = 0, nB = 0;
    for (double pos = A, w = h0; nA < 64; w *= 2.0) { ++nA; pos = fmin(pos + w, M); if (pos == M) break; }
    for (double pos = B, w = htop; nB < 64; w *= 2.0) { ++nB; pos = fmax(pos - w, M); if (pos == M) break; }
    double Jl = 0.0;
    Pl = 0.0;
    // A round covers two panels (16 nodes each). The bounds of a panel are the same on its 16
    // lanes, so lane L works out those of panel 32 g + L once per group g of 32 panels and
    // the lanes take theirs by shuffle: the FP64 pipe, the one this loop is bound by, sees one
    // bounds computation per 32 panels instead of one per round.
    double gmid = 0.0, ghw = 0.0;
    for (int base = 0; base < 16 * (nA + nB); base += 32) {
      const int q = base + lane, pnl = q >> 4, i = q & 15;
      if ((base & 511) == 0) {
        const int pg = (base >> 4) + lane;
        double a, c;
        if (pg < nA) {
          a = fmin(A + h0 * (ldexp(1.0, pg) - 1.0), M);
          c = fmin(A + h0 * (ldexp(1.0, pg + 1) - 1.0), M);
        } else {
          const int p2 = pg - nA;
          c = fmax(B - htop * (ldexp(1.0, p2) - 1.0), M);
          a = fmax(B - htop * (ldexp(1.0, p2 + 1) - 1.0), M);
        }
        gmid = 0.5 * (a + c);
        ghw = 0.5 * (c - a);
      }
      const double mid = __shfl_sync(0xffffffffu, gmid, pnl & 31), hw = __shfl_sync(0xffffffffu, ghw, pnl & 31);
      if (q >= 16 * (nA + nB)) continue;
      const double W = mid + hw * T.x16[i];
      if (kFast) {
        double DS, DI;
        eval_fast(b, C, T, W, xm, kT, inv_kT, phimFR, &DS, &DI);
        const double wt = hw * T.w16[i];
        Jl += wt * DS;
        Pl += wt * DI;
      } else {
        const double D = transmission_sel<kFast>(b, C, T, W, xm);
        Jl += hw * T.w16[i] * D * supply_sel<kFast>(W, kT);
        Pl += hw * T.w16[i] * D * inner_sel<kFast>(W, kT);
      }
    }
    J += warp_sum_d(Jl);
    P += warp_sum_d(Pl);
    nev += 16 * (nA + nB);
  }
  // [W_cut, min(0, top)], graded downward, two panels per round, stops when negligible
  {
    const double B = fmin(0.0, top);
    if (B > Wcut) {
      const double w0 = B == top ? htop : h0;
      const int half = lane >> 4, i = lane & 15;
      // panel bounds by shuffle, as above: lane L holds those of panel 32 g + L
      double ghi = 0.0, glo = 0.0;
      for (int r = 0; r < 32; ++r) {
        const int pnl = 2 * r + half;
        if ((r & 15) == 0) {
          const int pg = 2 * r + lane;
          ghi = fmax(B - w0 * (ldexp(1.0, pg) - 1.0), Wcut);
          glo = fmax(B - w0 * (ldexp(1.0, pg + 1) - 1.0), Wcut);
        }
        const double hi = __shfl_sync(0xffffffffu, ghi, pnl & 31), lo = __shfl_sync(0xffffffffu, glo, pnl & 31);
        const double last_lo = __shfl_sync(0xffffffffu, glo, (2 * r + 1) & 31);
        double Jl = 0.0;
        Pl = 0.0;
        if (hi > lo) {
          const double mid = 0.5 * (lo + hi), hw = 0.5 * (hi - lo);
          const double W = mid + hw * T.x16[i];
          if (kFast) {
            double DS, DI;
            eval_fast(b, C, T, W, xm, kT, inv_kT, phimFR, &DS, &DI);
            Jl = hw * T.w16[i] * DS;
            Pl = hw * T.w16[i] * DI;
          } else {
            const double D = transmission_sel<kFast>(b, C, T, W, xm);
            Jl = hw * T.w16[i] * D * supply_sel<kFast>(W, kT);
            Pl = hw * T.w16[i] * D * inner_sel<kFast>(W, kT);
          }
        }
        const double rJ = warp_sum_d(Jl), rP = warp_sum_d(Pl);
        J += rJ;
        P += rP;
        nev += 32;
        if (last_lo == Wcut) break;
        if (fabs(rJ) <= 1e-18 * fabs(J) && fabs(rP) <= 1e-18 * fabs(P)) break;
      }
    }
  }
  if (n_eval) *n_eval += nev;
  *J_out = C.zS * J;
  *P_out = C.zS * P;
}
#endif

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
