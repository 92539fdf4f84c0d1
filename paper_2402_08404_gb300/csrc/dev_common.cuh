// Device helpers shared by several kernel files (header-only, no relocatable device code).
#pragma once
#include "pic_internal.cuh"

namespace pic {

__device__ __forceinline__ float lerp_rn(float a, float b, float t) {
  return __fadd_rn(a, __fmul_rn(t, __fsub_rn(b, a)));
}

// E at a position (cell units) by nested lerps along x, then y, then z.
__device__ __forceinline__ float3 gather_E(const float4 *__restrict__ E, float x, float y, float z, int nx, int ny) {
  const float fi = floorf(x), fj = floorf(y), fk = floorf(z);
  const int i = (int)fi, j = (int)fj, k = (int)fk;
  const float fx = __fsub_rn(x, fi), fy = __fsub_rn(y, fj), fz = __fsub_rn(z, fk);
  const int64_t sy = nx + 1, sz = (int64_t)(nx + 1) * (ny + 1);
  const int64_t n000 = (int64_t)k * sz + (int64_t)j * sy + i;
  const float4 e000 = __ldg(E + n000), e100 = __ldg(E + n000 + 1);
  const float4 e010 = __ldg(E + n000 + sy), e110 = __ldg(E + n000 + sy + 1);
  const float4 e001 = __ldg(E + n000 + sz), e101 = __ldg(E + n000 + sz + 1);
  const float4 e011 = __ldg(E + n000 + sz + sy), e111 = __ldg(E + n000 + sz + sy + 1);
  float3 r;
  {
    float c00 = lerp_rn(e000.x, e100.x, fx), c10 = lerp_rn(e010.x, e110.x, fx);
    float c01 = lerp_rn(e001.x, e101.x, fx), c11 = lerp_rn(e011.x, e111.x, fx);
    r.x = lerp_rn(lerp_rn(c00, c10, fy), lerp_rn(c01, c11, fy), fz);
  }
  {
    float c00 = lerp_rn(e000.y, e100.y, fx), c10 = lerp_rn(e010.y, e110.y, fx);
    float c01 = lerp_rn(e001.y, e101.y, fx), c11 = lerp_rn(e011.y, e111.y, fx);
    r.y = lerp_rn(lerp_rn(c00, c10, fy), lerp_rn(c01, c11, fy), fz);
  }
  {
    float c00 = lerp_rn(e000.z, e100.z, fx), c10 = lerp_rn(e010.z, e110.z, fx);
    float c01 = lerp_rn(e001.z, e101.z, fx), c11 = lerp_rn(e011.z, e111.z, fx);
    r.z = lerp_rn(lerp_rn(c00, c10, fy), lerp_rn(c01, c11, fy), fz);
  }
  return r;
}

// Classical estimate the surrogate corrects: log10 of (Murphy-Good FN with Forbes' v(f), t(f),
// f capped at 1) + (Richardson-Dushman with Schottky lowering, barrier top capped at E_F);
// F in GV/m, T in K, phi in eV; clipped at the floor.
__device__ __forceinline__ double approx_log10J(double F, double T, double phi) {
  const double a = 1.541434e-6, b = 6.830890, c = 1.439964, ln10 = 2.302585092994046;
  const double f = fmin(c * F / (phi * phi), 1.0);
  const double lf = log(f);
  const double v = 1.0 - f + f / 6.0 * lf, t = 1.0 + f / 9.0 - f / 18.0 * lf;
  const double lfn = log10(a * F * F / (phi * t * t)) + 18.0 - v * b * phi * sqrt(phi) / F / ln10;
  const double kT = 8.617333262e-5 * T;
  const double lrd = log10(1.20173e6 * T * T) - fmax(phi - sqrt(c * F), 0.0) / kT / ln10;
  const double m = fmax(lfn, lrd);
  return fmax(m + log10(pow(10.0, lfn - m) + pow(10.0, lrd - m)), kSurLogJFloor);
}

// surrogate outputs of row i: J [A/m^2] and P_N [W/m^2]; 0 below the floor.
// log10 J = approx + y0 kSurY0s (approx from approx_log10J of the same tuple)
__device__ __forceinline__ void surrogate_out(const float *Y, int64_t i, double approx, double *J, double *P) {
  const double y0 = (double)Y[i * kSurOut];
  const double y1 = (double)Y[i * kSurOut + 1];
  const double lj = approx + y0 * kSurY0s;
  if (lj <= kSurLogJFloor + 1e-9) { *J = 0.0; *P = 0.0; return; }
  *J = pow(10.0, lj);
  *P = *J * (y1 * kSurY1s);
}

}  // namespace pic
