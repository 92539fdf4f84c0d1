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

}  // namespace pic
