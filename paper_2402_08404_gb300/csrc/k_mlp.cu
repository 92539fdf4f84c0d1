// Emission surrogate (no counterpart in the paper): an MLP 7 -> 128 -> 128 -> 128 -> 2 with GELU
// (exact erf form) mapping features of (F, T, work function, R | flat) to (log10 J - a classical
// estimate, eps_N = P_N / J in eV), trained on the full FP64 emission integral and used per face
// in the step wherever its inputs lie in the trained range and a held-out validation bin shows
// |delta log10 J| <= 0.015; elsewhere the step falls back to the full integral.
//
// Arithmetic: the two 128 x 128 hidden layers run on the fifth-generation tensor cores (tcgen05,
// TMEM accumulators) with BF16 operands and FP32 accumulation -- inference (the step's faces,
// pic_surrogate_eval, the validation map, forward calls without targets) in one fused kernel, and
// training, which keeps every layer's values for the backward pass, as separate products through
// one tiled GEMM kernel (k_mlp_tc.cu: forward, input gradients, and weight gradients split over
// the batch with a fixed-order sum).  The input layer
// (7 features) and the output layer (2 values)
// are FP32 on the CUDA cores, so the features and the last activations keep FP32 precision
// (in BF16 a feature step of 2^-9 moves log10 J by up to ~0.04 in the field-emission regime).
// FP32 master weights, Adam.  Weight gradients reduce over the batch with a fixed split order,
// so training is deterministic.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "pic_internal.cuh"
#include "gtf.cuh"
#include "dev_common.cuh"

namespace pic {

// ---- layout (public = master, row-major [out][in]) -------------------------------------------
constexpr int kH = 128, kIn = 7, kXld = 8, kOut = kSurOut;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kH, kOffW4 = kOffB3 + kH, kOffB4 = kOffW4 + kOut * kH,
              kNParam = kOffB4 + kOut;
static_assert(kNParam == 34306, "parameter count");
static_assert(kOffB1 == kOffW1 + kH * kIn && kOffB4 == kOffW4 + kOut * kH, "bias follows its weights");
static_assert(kH * kIn + kH <= 1024, "one thread per layer-1 gradient entry");

// input / output standardisation (fixed by the trained ranges)
constexpr double kF_lo = 0.001, kF_hi = 15.0;      // GV/m
constexpr double kF_mid = 0.05;                     // 70 % of the training tuples lie above
constexpr double kT_lo = 300.0, kT_hi = 4000.0;    // K
constexpr double kW_lo = 4.0, kW_hi = 5.0;         // eV
constexpr double kR_lo = 1.0, kR_hi = 20.0;        // nm
constexpr double kLogFlat = 3.0;                    // log10 R used for a flat surface
constexpr double kLogJFloor = kSurLogJFloor;       // log10 J below this carries no emission
constexpr double kY0s = kSurY0s, kY1s = kSurY1s;
constexpr int kBinF = 40, kBinT = 12, kBinW = 4, kBinR = 5, kNBin = kBinF * kBinT * kBinW * kBinR;
constexpr int kSplitMax = 64;

struct MlpState {
  bool ready = false, trained = false;
  float *master = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *w2 = nullptr, *w3 = nullptr;   // BF16 operand copies of the hidden layers
  int64_t cap_rows = 0;
  float *X = nullptr;                            // rows x kXld features (FP32)
  float *Z1 = nullptr, *Z2 = nullptr, *Z3 = nullptr, *A3 = nullptr, *Y = nullptr;
  __nv_bfloat16 *A1 = nullptr, *A2 = nullptr;
  float *dY = nullptr, *dZ = nullptr, *dA = nullptr;   // rows x 2, rows x kH, rows x kH
  __nv_bfloat16 *dZb = nullptr;
  float *part = nullptr;                         // split partials
  float *loss = nullptr;
  uint8_t *binok = nullptr;
  uint8_t *elig = nullptr;                       // per face (step)
};

static std::vector<std::pair<pic_t *, MlpState *>> &mlp_table() {
  static std::vector<std::pair<pic_t *, MlpState *>> table;
  return table;
}

static MlpState &mlp_of(pic_t *h) {
  auto &table = mlp_table();
  for (auto &e : table)
    if (e.first == h) return *e.second;
  table.push_back({h, new MlpState()});
  return *table.back().second;
}

// drop the surrogate state of a handle being destroyed (its device memory goes with the handle)
void mlp_forget(pic_t *h) {
  auto &table = mlp_table();
  for (size_t i = 0; i < table.size(); ++i)
    if (table[i].first == h) {
      delete table[i].second;
      table.erase(table.begin() + i);
      return;
    }
}

// ---- tensor-core GEMMs: C(M,128) = A(M,K) B(K,128), BF16 in, FP32 accumulate (tcgen05) -----------
// C(m,n) = sum_z partial[z](m,n) in fixed order
__global__ void k_reduce_splits(const float *part, int splits, int M, int N, float *C, int64_t scm, int64_t scn) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M * N; e += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += part[(int64_t)z * M * N + e];
    C[(int64_t)(e / N) * scm + (e % N) * scn] = s;
  }
}

// every training product has N = 128 (the hidden width); a product whose K is the batch is split
// over CTAs (splits partials in S.part, then the fixed-order sum)
static int gemm(pic_t *h, MlpState &S, const __nv_bfloat16 *A, int64_t sam, int64_t sak, const __nv_bfloat16 *B,
                int64_t sbk, int64_t sbn, float *C, int64_t scm, int64_t scn, int M, int N, int K, int splits) {
  if (N != kH) return pic_fail(h, PIC_E_INVALID, "training GEMM with N != 128");
  GemmTcArgs g{A, sam, sak, B, sbk, sbn, splits > 1 ? S.part : C, scm, scn, M, K, splits, 0};
  PIC_TRY(gemm_tc(h, g));
  if (splits > 1) {
    ++h->nlaunch;
    k_reduce_splits<<<std::max(1, (M * N + 255) / 256), 256, 0, h->stream>>>(S.part, splits, M, N, C, scm, scn);
  }
  return PIC_OK;
}

// ---- FP32 layers and elementwise ---------------------------------------------------------------
__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.3989422804014327f;
}

// input layer: Z1 = W1 x + b1 (FP32), A1 = bf16(gelu(Z1))
__global__ void k_layer1(const float *X, const float *W1, const float *b1, float *Z1, __nv_bfloat16 *A1, int64_t rows) {
  __shared__ float w[kH * kIn + kH];
  for (int e = threadIdx.x; e < kH * kIn + kH; e += blockDim.x) w[e] = W1[e];   // W1 then b1 (contiguous)
  __syncthreads();
  const int64_t n = rows * kH;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / kH;
    const int o = (int)(e - r * kH);
    float z = w[kH * kIn + o];
    for (int c = 0; c < kIn; ++c) z += w[o * kIn + c] * X[r * kXld + c];
    Z1[e] = z;
    A1[e] = __float2bfloat16(gelu_f(z));
  }
}

// Z += b (per column); A = bf16(gelu(Z)); Af = gelu(Z) in FP32 when given
__global__ void k_bias_gelu(float *Z, const float *b, __nv_bfloat16 *A, float *Af, int64_t rows) {
  const int64_t n = rows * kH;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float z = Z[e] + b[e % kH];
    Z[e] = z;
    const float a = gelu_f(z);
    if (A) A[e] = __float2bfloat16(a);
    if (Af) Af[e] = a;
  }
}

// output layer: one warp per row, Y = W4 A3 + b4 (FP32)
__global__ void k_layer4(const float *A3, const float *W4, const float *b4, float *Y, int64_t rows) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows; r += warps) {
    float y0 = 0.f, y1 = 0.f;
    for (int k = lane; k < kH; k += 32) {
      const float a = A3[r * kH + k];
      y0 += W4[k] * a;
      y1 += W4[kH + k] * a;
    }
    for (int o = 16; o > 0; o >>= 1) {
      y0 += __shfl_xor_sync(0xffffffffu, y0, o);
      y1 += __shfl_xor_sync(0xffffffffu, y1, o);
    }
    if (lane == 0) {
      Y[r * kOut] = y0 + b4[0];
      Y[r * kOut + 1] = y1 + b4[1];
    }
  }
}

// dY = (Y - T)/rows; loss partial sums (0.5 sum of squares) per block
__global__ void k_out_loss(const float *Y, const float *Tg, float *dY, int64_t rows, float *loss) {
  __shared__ float sh[32];
  float acc = 0.f;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
    for (int o = 0; o < kOut; ++o) {
      const float diff = Y[r * kOut + o] - Tg[r * 2 + o];
      acc += 0.5f * diff * diff;
      dY[r * kOut + o] = diff / (float)rows;
    }
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    loss[blockIdx.x] = s;
  }
}

// dA3 = dY W4 then dZ3 = dA3 gelu'(Z3) (FP32 and BF16 copies)
__global__ void k_layer4_bwd(const float *dY, const float *W4, const float *Z3, float *dZ, __nv_bfloat16 *dZb,
                             int64_t rows) {
  const int64_t n = rows * kH;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / kH;
    const int k = (int)(e - r * kH);
    const float da = dY[r * kOut] * W4[k] + dY[r * kOut + 1] * W4[kH + k];
    const float d = da * gelu_grad_f(Z3[e]);
    dZ[e] = d;
    dZb[e] = __float2bfloat16(d);
  }
}

// dZ = dA * gelu'(Z) (FP32, and BF16 when given)
__global__ void k_gelu_bwd(const float *dA, const float *Z, float *dZ, __nv_bfloat16 *dZb, int64_t rows) {
  const int64_t n = rows * kH;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float d = dA[e] * gelu_grad_f(Z[e]);
    dZ[e] = d;
    if (dZb) dZb[e] = __float2bfloat16(d);
  }
}

// Weight gradient of an FP32 layer, G[o][c] = sum_r D[r ldd + o] X[r ldx + c] (o < O, c < C), and
// with bias_out also sum_r D[r ldd + o]: block z sums its chunk of rows into partial z (one
// thread per (o, c) pair, O*C + O <= blockDim), k_reduce_splits adds the partials in order.
__global__ void k_wgrad32(const float *D, int ldd, const float *X, int ldx, int O, int C, int64_t rows, int chunks,
                          float *part) {
  const int t = threadIdx.x;
  const int nout = O * C + O;
  const int64_t per = (rows + chunks - 1) / chunks;
  const int64_t r0 = (int64_t)blockIdx.x * per, r1 = std::min<int64_t>(rows, r0 + per);
  if (t >= nout) return;
  const bool bias = t >= O * C;
  const int o = bias ? t - O * C : t / C, c = bias ? 0 : t - (t / C) * C;
  float s = 0.f;
  for (int64_t r = r0; r < r1; ++r) s += D[r * ldd + o] * (bias ? 1.f : X[r * ldx + c]);
  part[(int64_t)blockIdx.x * nout + t] = s;
}

// column sums of a rows x cols fp32 matrix (one block per column, fixed order)
__global__ void k_colsum(const float *X, int64_t rows, int ld, float *out) {
  __shared__ float sh[32];
  const int c = blockIdx.x;
  float s = 0.f;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) s += X[r * ld + c];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    out[c] = t;
  }
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, int n, float lr, float b1t, float b2t) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi, vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / b1t) / (sqrtf(vi / b2t) + 1e-8f);
  }
}

__global__ void k_to_bf16(const float *src, __nv_bfloat16 *dst, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = __float2bfloat16(src[i]);
}

// standardised features of one tuple: log10 F, T, phi_w, log10 R (flat: 3), 1/R (flat: 0),
// phi^1.5/F (the field-emission exponent scale, capped at 20), 1000/T
__device__ __forceinline__ void features(double F_GV, double T, double W, double R_nm, float x[kIn]) {
  const bool flat = !(R_nm > 0) || !isfinite(R_nm);
  x[0] = (float)((log10(F_GV) - (-0.912)) / 2.09);
  x[1] = (float)((T * 1e-3 - 2.15) / 1.85);
  x[2] = (float)((W - 4.5) / 0.5);
  x[3] = (float)((flat ? kLogFlat : log10(R_nm)) - 1.15);
  x[4] = (float)(flat ? -1.0 : 2.0 / R_nm - 1.0);
  x[5] = (float)(fmin(W * sqrt(W) / F_GV, 20.0) / 10.0 - 1.0);
  x[6] = (float)(1000.0 / T - 1.5);
}

__device__ __forceinline__ bool in_range(double F_GV, double T, double W, double R_nm) {
  const bool flat = !(R_nm > 0) || !isfinite(R_nm);
  return F_GV >= kF_lo && F_GV <= kF_hi && T >= kT_lo && T <= kT_hi && W >= kW_lo && W <= kW_hi &&
         (flat || (R_nm >= kR_lo && R_nm <= kR_hi));
}

__host__ __device__ inline int bin_of(double F_GV, double T, double W, double R_nm) {
  const bool flat = !(R_nm > 0) || !isfinite(R_nm);
  int bf = (int)((log10(F_GV) - log10(kF_lo)) / (log10(kF_hi) - log10(kF_lo)) * kBinF);
  int bt = (int)((T - kT_lo) / (kT_hi - kT_lo) * kBinT);
  int bw = (int)((W - kW_lo) / (kW_hi - kW_lo) * kBinW);
  int br = flat ? kBinR - 1 : (int)(log10(R_nm) / log10(kR_hi) * (kBinR - 1));
  bf = bf < 0 ? 0 : (bf > kBinF - 1 ? kBinF - 1 : bf);
  bt = bt < 0 ? 0 : (bt > kBinT - 1 ? kBinT - 1 : bt);
  bw = bw < 0 ? 0 : (bw > kBinW - 1 ? kBinW - 1 : bw);
  br = br < 0 ? 0 : (br > kBinR - 1 ? kBinR - 1 : br);
  return ((bf * kBinT + bt) * kBinW + bw) * kBinR + br;
}

// SI inputs (V/m, K, eV, m or <= 0 flat) -> feature rows
__global__ void k_features_rows(const double *F, const double *T, const double *W, const double *R, int64_t n,
                                float *X) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float x[kIn];
    features(F[i] * 1e-9, T[i], W[i], R[i] > 0 ? R[i] * 1e9 : -1.0, x);
    for (int c = 0; c < kXld; ++c) X[i * kXld + c] = c < kIn ? x[c] : 0.f;
  }
}

// training samples (SI units: V/m, K, eV, m; R <= 0 flat): Philox-drawn over the trained
// ranges, 20 % flat, 30 % of the fields below 0.05 GV/m
__global__ void k_samples(uint64_t seed, int64_t n, double *F, double *T, double *W, double *R) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const U4 r = rng_block(seed, 11u, (uint64_t)i, 0, 0);
    const U4 r2 = rng_block(seed, 11u, (uint64_t)i, 0, 1);
    const bool low = u01d(r2.v[1]) < 0.3;
    const double lo = low ? log10(kF_lo) : log10(kF_mid), hi = low ? log10(kF_mid) : log10(kF_hi);
    F[i] = 1e9 * pow(10.0, lo + u01d(r.v[0]) * (hi - lo));
    T[i] = kT_lo + u01d(r.v[1]) * (kT_hi - kT_lo);
    W[i] = kW_lo + u01d(r.v[2]) * (kW_hi - kW_lo);
    R[i] = u01d(r2.v[0]) < 0.2 ? -1.0 : 1e-9 * pow(10.0, u01d(r.v[3]) * log10(kR_hi));
  }
}

// targets: (clip(log10 J) - approx_log10J) / s0 and eps_N / s1 (SI tuples)
__global__ void k_targets(const double *F, const double *T, const double *W, const double *J, const double *P,
                          int64_t n, float *Tg, double *approx) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double lj = J[i] > 0 ? fmax(log10(J[i]), kLogJFloor) : kLogJFloor;
    const double ap = approx_log10J(F[i] * 1e-9, T[i], W[i]);
    const double eps = J[i] > 0 ? P[i] / J[i] : 0.0;
    Tg[2 * i] = (float)((lj - ap) / kY0s);
    Tg[2 * i + 1] = (float)(eps / kY1s);
    approx[i] = ap;
  }
}

// ---- host: forward / backward over `rows` rows of S.X -----------------------------------------
static int ensure(pic_t *h, MlpState &S, int64_t rows) {
  if (!S.ready) {
    S.master = (float *)dalloc(h, kNParam * 4);
    S.grad = (float *)dalloc(h, kNParam * 4);
    S.m = (float *)dalloc(h, kNParam * 4);
    S.v = (float *)dalloc(h, kNParam * 4);
    S.w2 = (__nv_bfloat16 *)dalloc(h, kH * kH * 2);
    S.w3 = (__nv_bfloat16 *)dalloc(h, kH * kH * 2);
    S.part = (float *)dalloc(h, (size_t)kSplitMax * kH * kH * 4);
    S.loss = (float *)dalloc(h, 4096 * 4);
    S.binok = (uint8_t *)dalloc(h, kNBin);
    if (!S.master || !S.grad || !S.m || !S.v || !S.w2 || !S.w3 || !S.part || !S.loss || !S.binok)
      return pic_fail(h, PIC_E_CUDA, "surrogate allocation failed");
    PIC_CUDA(h, cudaMemsetAsync(S.master, 0, kNParam * 4, h->stream));
    PIC_CUDA(h, cudaMemsetAsync(S.binok, 0, kNBin, h->stream));
    S.ready = true;
  }
  if (rows > S.cap_rows) {
    const int64_t r = std::max<int64_t>(rows, 1024);
    S.X = (float *)dalloc(h, r * kXld * 4);
    S.Z1 = (float *)dalloc(h, r * kH * 4); S.Z2 = (float *)dalloc(h, r * kH * 4); S.Z3 = (float *)dalloc(h, r * kH * 4);
    S.A3 = (float *)dalloc(h, r * kH * 4);
    S.Y = (float *)dalloc(h, r * kOut * 4);
    S.A1 = (__nv_bfloat16 *)dalloc(h, r * kH * 2); S.A2 = (__nv_bfloat16 *)dalloc(h, r * kH * 2);
    S.dY = (float *)dalloc(h, r * kOut * 4);
    S.dZ = (float *)dalloc(h, r * kH * 4);
    S.dA = (float *)dalloc(h, r * kH * 4);
    S.dZb = (__nv_bfloat16 *)dalloc(h, r * kH * 2);
    S.elig = (uint8_t *)dalloc(h, r);
    if (!S.X || !S.Z1 || !S.Z2 || !S.Z3 || !S.A3 || !S.Y || !S.A1 || !S.A2 || !S.dY || !S.dZ || !S.dA || !S.dZb ||
        !S.elig)
      return pic_fail(h, PIC_E_CUDA, "surrogate allocation failed");
    S.cap_rows = r;
  }
  return PIC_OK;
}

static void refresh_bf16(pic_t *h, MlpState &S) {
  h->nlaunch += 2;
  k_to_bf16<<<32, 256, 0, h->stream>>>(S.master + kOffW2, S.w2, kH * kH);
  k_to_bf16<<<32, 256, 0, h->stream>>>(S.master + kOffW3, S.w3, kH * kH);
}

static int eg(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }

// forward of feature rows X -> Y (rows x 2, bias included); keeps Z1..Z3, A1, A2, A3
static int forward(pic_t *h, MlpState &S, const float *X, int64_t rows) {
  const int M = (int)rows;
  ++h->nlaunch;
  k_layer1<<<eg(rows * kH), 256, 0, h->stream>>>(X, S.master + kOffW1, S.master + kOffB1, S.Z1, S.A1, rows);
  PIC_TRY(gemm(h, S, S.A1, kH, 1, S.w2, 1, kH, S.Z2, kH, 1, M, kH, kH, 1));
  ++h->nlaunch;
  k_bias_gelu<<<eg(rows * kH), 256, 0, h->stream>>>(S.Z2, S.master + kOffB2, S.A2, nullptr, rows);
  PIC_TRY(gemm(h, S, S.A2, kH, 1, S.w3, 1, kH, S.Z3, kH, 1, M, kH, kH, 1));
  ++h->nlaunch;
  k_bias_gelu<<<eg(rows * kH), 256, 0, h->stream>>>(S.Z3, S.master + kOffB3, nullptr, S.A3, rows);
  ++h->nlaunch;
  k_layer4<<<eg(rows * 32), 256, 0, h->stream>>>(S.A3, S.master + kOffW4, S.master + kOffB4, S.Y, rows);
  return PIC_OK;
}

// FP32 weight and bias gradient of a small layer into S.grad: the layouts keep b right after W
// (offB = offW + O C), so the partials [W | b] reduce straight into place
static void wgrad32(pic_t *h, MlpState &S, const float *D, int ldd, const float *X, int ldx, int O, int C, int64_t rows,
                    int offW) {
  const int nout = O * C + O;
  const int chunks = (int)std::min<int64_t>(kSplitMax, std::max<int64_t>(1, rows / 256));
  ++h->nlaunch;
  k_wgrad32<<<chunks, (nout + 31) / 32 * 32, 0, h->stream>>>(D, ldd, X, ldx, O, C, rows, chunks, S.part);
  ++h->nlaunch;
  k_reduce_splits<<<std::max(1, (nout + 255) / 256), 256, 0, h->stream>>>(S.part, chunks, 1, nout, S.grad + offW, 0, 1);
}

// loss and gradients (into S.grad) for targets Tg (rows x 2, fp32); loss partials in S.loss
static int backward(pic_t *h, MlpState &S, const float *X, const float *Tg, int64_t rows, int nloss_blocks) {
  const int M = (int)rows;
  ++h->nlaunch;
  k_out_loss<<<nloss_blocks, 256, 0, h->stream>>>(S.Y, Tg, S.dY, rows, S.loss);
  // weight gradients: the batch (K) split into ranges of 128 rows, one CTA each
  const int splits = (int)std::min<int64_t>(kSplitMax, std::max<int64_t>(1, (rows + 127) / 128));
  // layer 4 (FP32): dW4 = dY^T A3, db4; dZ3 = (dY W4) gelu'(Z3)
  wgrad32(h, S, S.dY, kOut, S.A3, kH, kOut, kH, rows, kOffW4);
  ++h->nlaunch;
  k_layer4_bwd<<<eg(rows * kH), 256, 0, h->stream>>>(S.dY, S.master + kOffW4, S.Z3, S.dZ, S.dZb, rows);
  // layer 3 (tensor cores): dW3 = dZ3^T A2, db3, dA2 = dZ3 W3
  PIC_TRY(gemm(h, S, S.dZb, 1, kH, S.A2, kH, 1, S.grad + kOffW3, kH, 1, kH, kH, M, splits));
  ++h->nlaunch;
  k_colsum<<<kH, 256, 0, h->stream>>>(S.dZ, rows, kH, S.grad + kOffB3);
  PIC_TRY(gemm(h, S, S.dZb, kH, 1, S.w3, kH, 1, S.dA, kH, 1, M, kH, kH, 1));
  ++h->nlaunch;
  k_gelu_bwd<<<eg(rows * kH), 256, 0, h->stream>>>(S.dA, S.Z2, S.dZ, S.dZb, rows);
  // layer 2 (tensor cores): dW2 = dZ2^T A1, db2, dA1 = dZ2 W2
  PIC_TRY(gemm(h, S, S.dZb, 1, kH, S.A1, kH, 1, S.grad + kOffW2, kH, 1, kH, kH, M, splits));
  ++h->nlaunch;
  k_colsum<<<kH, 256, 0, h->stream>>>(S.dZ, rows, kH, S.grad + kOffB2);
  PIC_TRY(gemm(h, S, S.dZb, kH, 1, S.w2, kH, 1, S.dA, kH, 1, M, kH, kH, 1));
  ++h->nlaunch;
  k_gelu_bwd<<<eg(rows * kH), 256, 0, h->stream>>>(S.dA, S.Z1, S.dZ, nullptr, rows);
  // layer 1 (FP32): dW1 = dZ1^T X, db1
  wgrad32(h, S, S.dZ, kH, X, kXld, kH, kIn, rows, kOffW1);
  return launch_check(h, "mlp backward");
}

// ---- step integration ---------------------------------------------------------------------------
__global__ void k_face_rows(const double *Fface, const int32_t *owner_vox, const double *Tvox, double T0, double phi_w,
                            double R_nm, int64_t nface, const uint8_t *binok, float *X, uint8_t *elig) {
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nface; f += (int64_t)gridDim.x * blockDim.x) {
    const int v = owner_vox[f];
    const double T = v >= 0 ? Tvox[v] : T0;
    const double R = v >= 0 ? R_nm : -1.0;
    const double F = Fface[f] * 1e-9;
    const bool inr = F > 0 && in_range(F, T, phi_w, R);
    float x[kIn] = {};
    if (inr) features(F, T, phi_w, R, x);
    for (int c = 0; c < kXld; ++c) X[f * kXld + c] = c < kIn ? x[c] : 0.f;
    // 1: inside the range and a validated bin; 2: inside the range only; 3: a pulling field
    // below the trained range (F < kF_lo); 0: otherwise
    elig[f] = inr ? (binok[bin_of(F, T, phi_w, R)] ? 1 : 2) : (F > 0 && F < kF_lo ? 3 : 0);
  }
}

}  // namespace pic

namespace pic {

__global__ void k_surrogate_apply(const float *Y, const uint8_t *elig, const double *F, const double *T,
                                  const double *W, int64_t n, double *J, double *P, uint8_t *valid) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double j = 0, p = 0;
    surrogate_out(Y, i, approx_log10J(F[i] * 1e-9, T[i], W[i]), &j, &p);
    J[i] = j;
    P[i] = p;
    if (valid) valid[i] = elig ? elig[i] : 1;
  }
}

__global__ void k_rows_eligible(const double *F, const double *T, const double *W, const double *R, int64_t n,
                                const uint8_t *binok, uint8_t *elig) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double Fg = F[i] * 1e-9, Rn = R[i] > 0 ? R[i] * 1e9 : -1.0;
    elig[i] = (Fg > 0 && in_range(Fg, T[i], W[i], Rn) && binok[bin_of(Fg, T[i], W[i], Rn)]) ? 1 : 0;
  }
}

// Surrogate forward for the step's faces: fills J, PN of eligible faces and the eligibility flag.
int surrogate_faces(pic_t *h, const uint8_t **elig_out, const float **Y_out) {
  MlpState &S = mlp_of(h);
  if (!S.trained) return pic_fail(h, PIC_E_INVALID, "surrogate not trained");
  PIC_TRY(ensure(h, S, h->faces.n));
  ++h->nlaunch;
  k_face_rows<<<grid_for(h->faces.n), kThreads, 0, h->stream>>>(h->faces.F, h->faces.owner_vox, h->heat.T, h->prm.T0,
                                                                 h->prm.work_function, h->geo.tip_radius * 1e9,
                                                                 h->faces.n, S.binok, S.X, S.elig);
  PIC_TRY(mlp_forward_tc(h, S.X, h->faces.n, S.master, S.w2, S.w3, S.Y));
  *elig_out = S.elig;
  *Y_out = S.Y;
  return launch_check(h, "surrogate faces");
}

bool surrogate_ready(pic_t *h) { return mlp_of(h).trained; }

}  // namespace pic

using namespace pic;

extern "C" {

int pic_mlp_num_params(void) { return kNParam; }

int pic_mlp_set_params(pic_t *h, const float *params) {
  if (h) graph_invalidate(h);   // its buffers may be reallocated
  if (!h || !params) return PIC_E_INVALID;
  MlpState &S = mlp_of(h);
  PIC_TRY(ensure(h, S, 1024));
  PIC_CUDA(h, cudaMemcpyAsync(S.master, params, kNParam * 4, cudaMemcpyHostToDevice, h->stream));
  refresh_bf16(h, S);
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  return launch_check(h, "mlp set");
}

int pic_mlp_get_params(pic_t *h, float *params) {
  if (!h || !params) return PIC_E_INVALID;
  MlpState &S = mlp_of(h);
  PIC_TRY(ensure(h, S, 1024));
  PIC_CUDA(h, cudaMemcpyAsync(params, S.master, kNParam * 4, cudaMemcpyDeviceToHost, h->stream));
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

// x: n x 7 standardised features (host, float); y: n x 2 outputs; optional t (n x 2 targets):
// then loss (mean over rows of sum 0.5 (y - t)^2) and grad (parameter layout) are returned too.
int pic_mlp_forward_backward(pic_t *h, const float *x, const float *t, int64_t n, float *y, float *loss, float *grad) {
  if (h) graph_invalidate(h);   // its buffers may be reallocated
  if (!h || !x || n <= 0 || n > (1 << 22)) return PIC_E_INVALID;
  MlpState &S = mlp_of(h);
  PIC_TRY(ensure(h, S, n));
  std::vector<float> X(n * kXld, 0.f);
  for (int64_t i = 0; i < n; ++i)
    for (int c = 0; c < kIn; ++c) X[i * kXld + c] = x[i * kIn + c];
  PIC_CUDA(h, cudaMemcpyAsync(S.X, X.data(), n * kXld * 4, cudaMemcpyHostToDevice, h->stream));
  if (t) PIC_TRY(forward(h, S, S.X, n));   // training: keeps the layer values the gradient needs
  else PIC_TRY(mlp_forward_tc(h, S.X, n, S.master, S.w2, S.w3, S.Y));   // inference (as in the step)
  if (t) {
    float *Tg = S.dA;   // scratch for targets (rows x 2 fits in rows x kH)
    PIC_CUDA(h, cudaMemcpyAsync(Tg, t, n * 2 * 4, cudaMemcpyHostToDevice, h->stream));
    PIC_TRY(backward(h, S, S.X, Tg, n, 64));
  }
  std::vector<float> Yh(n * kOut);
  PIC_CUDA(h, cudaMemcpyAsync(Yh.data(), S.Y, n * kOut * 4, cudaMemcpyDeviceToHost, h->stream));
  std::vector<float> lp(64), g(kNParam);
  if (t) {
    PIC_CUDA(h, cudaMemcpyAsync(lp.data(), S.loss, 64 * 4, cudaMemcpyDeviceToHost, h->stream));
    PIC_CUDA(h, cudaMemcpyAsync(g.data(), S.grad, kNParam * 4, cudaMemcpyDeviceToHost, h->stream));
  }
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  if (y)
    for (int64_t i = 0; i < n; ++i) { y[2 * i] = Yh[i * kOut]; y[2 * i + 1] = Yh[i * kOut + 1]; }
  if (t) {
    double l = 0;
    for (float v : lp) l += v;
    if (loss) *loss = (float)(l / n);
    if (grad) memcpy(grad, g.data(), kNParam * 4);
  }
  return launch_check(h, "mlp fwd/bwd");
}

// Train on nsamples tuples drawn over the trained ranges (targets from the FP64 integral),
// validate on nval held-out tuples, build the per-bin validity map and install the surrogate.
// stats (optional, 8 doubles): train loss, val RMS |dlog10 J|, val max |dlog10 J| (relevant),
// fraction of valid bins, fraction of valid held-out samples, ms data, ms train, steps.
int pic_surrogate_train(pic_t *h, int64_t nsamples, int epochs, int batch, double lr0, uint64_t seed, double *stats) {
  if (h) graph_invalidate(h);   // its buffers may be reallocated
  if (!h || nsamples < 1024 || epochs < 1 || batch < 256 || batch > 65536) return PIC_E_INVALID;
  MlpState &S = mlp_of(h);
  const int64_t nval = std::max<int64_t>(nsamples / 2, 4096);
  const int64_t ntot = nsamples + nval;
  PIC_TRY(ensure(h, S, std::max<int64_t>(batch, nval)));
  cudaStream_t st = h->stream;
  cudaEvent_t e0, e1, e2;
  cudaEventCreate(&e0); cudaEventCreate(&e1); cudaEventCreate(&e2);
  cudaEventRecord(e0, st);
  // data: tuples, FP64 integral, standardised features and targets
  double *buf = (double *)dalloc(h, (size_t)ntot * 6 * 8);
  float *Xall = (float *)dalloc(h, (size_t)ntot * kXld * 4);
  float *Tall = (float *)dalloc(h, (size_t)ntot * 2 * 4);
  if (!buf || !Xall || !Tall) return pic_fail(h, PIC_E_CUDA, "surrogate data allocation failed");
  double *F = buf, *T = buf + ntot, *W = buf + 2 * ntot, *R = buf + 3 * ntot, *J = buf + 4 * ntot, *P = buf + 5 * ntot;
  ++h->nlaunch;
  k_samples<<<grid_for(ntot), kThreads, 0, st>>>(seed, ntot, F, T, W, R);
  PIC_TRY(emission_eval_dev(h, F, T, W, R, J, P, ntot, false));   // targets from the FP64 integral
  ++h->nlaunch;
  k_features_rows<<<grid_for(ntot), kThreads, 0, st>>>(F, T, W, R, ntot, Xall);
  double *approx = (double *)dalloc(h, (size_t)ntot * 8);
  if (!approx) return pic_fail(h, PIC_E_CUDA, "surrogate data allocation failed");
  ++h->nlaunch;
  k_targets<<<grid_for(ntot), kThreads, 0, st>>>(F, T, W, J, P, ntot, Tall, approx);
  cudaEventRecord(e1, st);
  // init: He-normal weights from a fixed host generator, zero biases
  std::vector<float> pub(kNParam, 0.f);
  {
    uint64_t s = seed * 6364136223846793005ull + 1442695040888963407ull;
    auto nrm = [&]() {
      double u1, u2;
      s = s * 6364136223846793005ull + 1442695040888963407ull;
      u1 = ((s >> 11) + 0.5) * (1.0 / 9007199254740992.0);
      s = s * 6364136223846793005ull + 1442695040888963407ull;
      u2 = ((s >> 11) + 0.5) * (1.0 / 9007199254740992.0);
      return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2);
    };
    int q = 0;
    const int fan[4] = {kIn, kH, kH, kH}, outs[4] = {kH, kH, kH, kOut};
    for (int l = 0; l < 4; ++l) {
      const double sd = sqrt(2.0 / fan[l]);
      for (int e = 0; e < outs[l] * fan[l]; ++e) pub[q++] = (float)(sd * nrm());
      for (int e = 0; e < outs[l]; ++e) pub[q++] = 0.f;
    }
  }
  PIC_CUDA(h, cudaMemcpyAsync(S.master, pub.data(), kNParam * 4, cudaMemcpyHostToDevice, st));
  PIC_CUDA(h, cudaMemsetAsync(S.m, 0, kNParam * 4, st));
  PIC_CUDA(h, cudaMemsetAsync(S.v, 0, kNParam * 4, st));
  refresh_bf16(h, S);
  const int64_t steps_per_epoch = std::max<int64_t>(1, nsamples / batch);
  const int64_t total = steps_per_epoch * epochs;
  int64_t step = 0;
  double last_loss = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int64_t b = 0; b < steps_per_epoch; ++b, ++step) {
      const int64_t r0 = ((b + (int64_t)ep * 7919) % steps_per_epoch) * batch;
      const float *Xb = Xall + r0 * kXld;
      const float *Tb = Tall + r0 * 2;
      PIC_TRY(forward(h, S, Xb, batch));
      PIC_TRY(backward(h, S, Xb, Tb, batch, 16));
      const double lr = lr0 * (0.01 + 0.99 * 0.5 * (1.0 + cos(3.141592653589793 * (double)step / (double)total)));
      const int t = step + 1;
      ++h->nlaunch;
      k_adam<<<40, 256, 0, st>>>(S.master, S.grad, S.m, S.v, kNParam, (float)lr, (float)(1.0 - pow(0.9, t)),
                                 (float)(1.0 - pow(0.999, t)));
      refresh_bf16(h, S);
      if (ep == epochs - 1 && b == steps_per_epoch - 1) {
        std::vector<float> lp(16);
        PIC_CUDA(h, cudaMemcpyAsync(lp.data(), S.loss, 16 * 4, cudaMemcpyDeviceToHost, st));
        PIC_CUDA(h, cudaStreamSynchronize(st));
        double l = 0;
        for (float v : lp) l += v;
        last_loss = l / batch;
      }
    }
  }
  cudaEventRecord(e2, st);
  PIC_TRY(launch_check(h, "surrogate train"));
  // validation on the held-out tuples: per-bin max |dlog10 J| where either side is relevant
  const float *Xv = Xall + nsamples * kXld;
  PIC_TRY(mlp_forward_tc(h, Xv, nval, S.master, S.w2, S.w3, S.Y));   // the step's inference kernel
  std::vector<float> Yv(nval * kOut), Tv(nval * 2);
  std::vector<double> hF(nval), hT(nval), hW(nval), hR(nval), hA(nval);
  PIC_CUDA(h, cudaMemcpyAsync(hA.data(), approx + nsamples, nval * 8, cudaMemcpyDeviceToHost, st));
  PIC_CUDA(h, cudaMemcpyAsync(Yv.data(), S.Y, nval * kOut * 4, cudaMemcpyDeviceToHost, st));
  PIC_CUDA(h, cudaMemcpyAsync(Tv.data(), Tall + nsamples * 2, nval * 2 * 4, cudaMemcpyDeviceToHost, st));
  PIC_CUDA(h, cudaMemcpyAsync(hF.data(), F + nsamples, nval * 8, cudaMemcpyDeviceToHost, st));
  PIC_CUDA(h, cudaMemcpyAsync(hT.data(), T + nsamples, nval * 8, cudaMemcpyDeviceToHost, st));
  PIC_CUDA(h, cudaMemcpyAsync(hW.data(), W + nsamples, nval * 8, cudaMemcpyDeviceToHost, st));
  PIC_CUDA(h, cudaMemcpyAsync(hR.data(), R + nsamples, nval * 8, cudaMemcpyDeviceToHost, st));
  PIC_CUDA(h, cudaStreamSynchronize(st));
  std::vector<float> binerr(kNBin, 0.f);
  std::vector<int> binn(kNBin, 0);
  double se = 0, mx = 0;
  int64_t nrel = 0;
  const double relevant = -5.0;      // log10 J [A/m^2] below which no face ever emits an SP
  for (int64_t i = 0; i < nval; ++i) {
    const double lp = std::max(hA[i] + Yv[i * kOut] * kY0s, kLogJFloor), lt = hA[i] + Tv[i * 2] * kY0s;
    const double err = (std::max(lp, lt) >= relevant) ? fabs(lp - lt) : 0.0;
    const double Fg = hF[i] * 1e-9, Rn = hR[i] > 0 ? hR[i] * 1e9 : -1.0;
    const bool flat = !(Rn > 0);
    int bf = (int)((log10(Fg) - log10(kF_lo)) / (log10(kF_hi) - log10(kF_lo)) * kBinF);
    int bt = (int)((hT[i] - kT_lo) / (kT_hi - kT_lo) * kBinT);
    int bw = (int)((hW[i] - kW_lo) / (kW_hi - kW_lo) * kBinW);
    int br = flat ? kBinR - 1 : (int)(log10(Rn) / log10(kR_hi) * (kBinR - 1));
    bf = std::min(std::max(bf, 0), kBinF - 1); bt = std::min(std::max(bt, 0), kBinT - 1);
    bw = std::min(std::max(bw, 0), kBinW - 1); br = std::min(std::max(br, 0), kBinR - 1);
    const int bin = ((bf * kBinT + bt) * kBinW + bw) * kBinR + br;
    binerr[bin] = std::max(binerr[bin], (float)err);
    binn[bin] += 1;
    if (std::max(lp, lt) >= relevant) { se += err * err; mx = std::max(mx, err); ++nrel; }
  }
  std::vector<uint8_t> ok(kNBin);
  int nok = 0;
  // a bin is used when every held-out sample in it is within 0.015 (margin under the 0.02 bar)
  for (int b = 0; b < kNBin; ++b) { ok[b] = binn[b] >= 8 && binerr[b] <= 0.015f; nok += ok[b]; }
  int64_t nsok = 0;
  for (int b = 0; b < kNBin; ++b) nsok += ok[b] ? binn[b] : 0;
  PIC_CUDA(h, cudaMemcpyAsync(S.binok, ok.data(), kNBin, cudaMemcpyHostToDevice, st));
  PIC_CUDA(h, cudaStreamSynchronize(st));
  S.trained = true;
  float ms_data = 0, ms_train = 0;
  cudaEventElapsedTime(&ms_data, e0, e1);
  cudaEventElapsedTime(&ms_train, e1, e2);
  cudaEventDestroy(e0); cudaEventDestroy(e1); cudaEventDestroy(e2);
  if (stats) {
    stats[0] = last_loss;
    stats[1] = nrel ? sqrt(se / nrel) : 0.0;
    stats[2] = mx;
    stats[3] = (double)nok / kNBin;
    stats[4] = (double)nsok / nval;
    stats[5] = ms_data;
    stats[6] = ms_train;
    stats[7] = (double)total;
  }
  return PIC_OK;
}

// Install the trained surrogate of src (weights and validity map) in dst: one training serves
// every instance of an ensemble.  Both handles on the current device; PIC_E_INVALID if src has no
// trained surrogate.
int pic_surrogate_copy(pic_t *dst, pic_t *src) {
  if (!dst || !src || dst == src) return PIC_E_INVALID;
  graph_invalidate(dst);   // its buffers may be reallocated
  MlpState &A = mlp_of(src);
  if (!A.trained) return pic_fail(dst, PIC_E_INVALID, "source instance has no trained surrogate");
  MlpState &B = mlp_of(dst);
  PIC_TRY(ensure(dst, B, 1024));
  PIC_CUDA(dst, cudaStreamSynchronize(src->stream));
  PIC_CUDA(dst, cudaMemcpyAsync(B.master, A.master, kNParam * 4, cudaMemcpyDeviceToDevice, dst->stream));
  PIC_CUDA(dst, cudaMemcpyAsync(B.binok, A.binok, kNBin, cudaMemcpyDeviceToDevice, dst->stream));
  refresh_bf16(dst, B);
  PIC_CUDA(dst, cudaStreamSynchronize(dst->stream));
  B.trained = true;
  return launch_check(dst, "surrogate copy");
}

// Surrogate evaluation of n host tuples (F [V/m], T [K], phi_w [eV], R [m] or <= 0 flat):
// J, PN from the network; valid[i] = 1 where the tuple is inside the trained range and its
// validation bin passed (elsewhere the step uses the full integral).
int pic_surrogate_eval(pic_t *h, const double *F, const double *T, const double *phi_w, const double *R, double *J,
                       double *PN, uint8_t *valid, int64_t n) {
  if (h) graph_invalidate(h);   // its buffers may be reallocated
  if (!h || n <= 0 || !F || !T || !phi_w || !R || !J || !PN) return PIC_E_INVALID;
  MlpState &S = mlp_of(h);
  if (!S.trained) return pic_fail(h, PIC_E_INVALID, "surrogate not trained");
  PIC_TRY(ensure(h, S, n));
  double *buf = nullptr;
  PIC_CUDA(h, cudaMalloc(&buf, (size_t)n * 6 * 8));
  uint8_t *el = nullptr;
  PIC_CUDA(h, cudaMalloc(&el, (size_t)n));
  cudaStream_t st = h->stream;
  int rc = PIC_OK;
  double *dF = buf, *dT = buf + n, *dW = buf + 2 * n, *dR = buf + 3 * n, *dJ = buf + 4 * n, *dP = buf + 5 * n;
  if (cudaMemcpyAsync(dF, F, n * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dT, T, n * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dW, phi_w, n * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dR, R, n * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
    rc = pic_fail(h, PIC_E_CUDA, "surrogate eval upload");
  if (rc == PIC_OK) {
    ++h->nlaunch;
    k_rows_eligible<<<grid_for(n), kThreads, 0, st>>>(dF, dT, dW, dR, n, S.binok, el);
    ++h->nlaunch;
    k_features_rows<<<grid_for(n), kThreads, 0, st>>>(dF, dT, dW, dR, n, S.X);
    if (mlp_forward_tc(h, S.X, n, S.master, S.w2, S.w3, S.Y) != PIC_OK) rc = PIC_E_CUDA;
    ++h->nlaunch;
    k_surrogate_apply<<<grid_for(n), kThreads, 0, st>>>(S.Y, el, dF, dT, dW, n, dJ, dP, el);
    if (cudaMemcpyAsync(J, dJ, n * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(PN, dP, n * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        (valid && cudaMemcpyAsync(valid, el, n, cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = pic_fail(h, PIC_E_CUDA, "surrogate eval download");
  }
  cudaFree(buf);
  cudaFree(el);
  if (rc == PIC_OK) rc = launch_check(h, "surrogate eval");
  return rc;
}

}  // extern "C"

namespace pic {

// Surrogate state for pic_save / pic_load: the FP32 master weights (pic_mlp_num_params floats)
// and the per-bin validity map (surrogate_bins bytes); *trained says whether the step may use it.
int surrogate_bins() { return kNBin; }

int surrogate_export(pic_t *h, float *master, uint8_t *binok, int *trained) {
  MlpState &S = mlp_of(h);
  *trained = S.trained ? 1 : 0;
  if (!S.ready) {
    memset(master, 0, kNParam * 4);
    memset(binok, 0, kNBin);
    return PIC_OK;
  }
  PIC_CUDA(h, cudaMemcpyAsync(master, S.master, kNParam * 4, cudaMemcpyDeviceToHost, h->stream));
  PIC_CUDA(h, cudaMemcpyAsync(binok, S.binok, kNBin, cudaMemcpyDeviceToHost, h->stream));
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

int surrogate_import(pic_t *h, const float *master, const uint8_t *binok, int trained) {
  MlpState &S = mlp_of(h);
  PIC_TRY(ensure(h, S, 1024));
  PIC_CUDA(h, cudaMemcpyAsync(S.master, master, kNParam * 4, cudaMemcpyHostToDevice, h->stream));
  PIC_CUDA(h, cudaMemcpyAsync(S.binok, binok, kNBin, cudaMemcpyHostToDevice, h->stream));
  refresh_bf16(h, S);
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  S.trained = trained != 0;
  return launch_check(h, "surrogate import");
}

}  // namespace pic
