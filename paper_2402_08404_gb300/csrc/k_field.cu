// Poisson solve (eq:poi with eq:bcf1-3) by geometric multigrid and the node field E = -grad phi.
//
// Operator: (A u)_n = (6 u_n - sum of the 6 neighbours)/h^2 on free nodes, mirror images across
// the lateral walls (zero normal field), Dirichlet nodes on the z = 0 and z = nz planes and on
// every corner of a solid cell.  Charge density rho_n = Q_n e w_min 2^-30 / V_n with V_n = dx^3
// halved on each lateral wall the node lies on.
//
// Solve: refinement loop in float64 -- r = f - A phi, stop when ||r||/||f_lifted|| < tol, else
// one V-cycle on A e = r and phi += e.  The V-cycle runs in float32 (mixed form) or float64
// (plain form): red-black Gauss-Seidel 2+2 sweeps, full-weighting restriction, trilinear
// prolongation, a one-block smoother on the coarsest level.  Coarse Dirichlet masks are
// injected from the fine nodes they coincide with.
//
// Layout: phi (fixed point, 2^-40 V), the right-hand side, E and the fixed-point charge are
// node arrays in natural order.  The V-cycle levels keep their two colours apart: node (i, j, k) of colour
// c = (i + j + k) & 1 lives at c * nper + ((k (ny + 1) + j) Xh + (i >> 1)), Xh = (nx + 2) / 2.
// A colour sweep then reads the other colour and writes its own as contiguous rows, and its
// 6 neighbours of (i, j, k) sit at slots (i -+ 1) >> 1 of its own row and i >> 1 of the four
// rows around it, all in the other colour.
#include "pic_internal.cuh"

namespace pic {

// ---- natural-order helpers (phi, rhs) ---------------------------------------------------------
template <typename T>
__device__ __forceinline__ T nb_sum(const T *u, int i, int j, int k, int nx, int ny) {
  const int im = i > 0 ? i - 1 : 1, ip = i < nx ? i + 1 : nx - 1;
  const int jm = j > 0 ? j - 1 : 1, jp = j < ny ? j + 1 : ny - 1;
  const int64_t sy = nx + 1, sz = (int64_t)(nx + 1) * (ny + 1);
  const int64_t c = (int64_t)k * sz + (int64_t)j * sy;
  return u[c + im] + u[c + ip] + u[(int64_t)k * sz + (int64_t)jm * sy + i] + u[(int64_t)k * sz + (int64_t)jp * sy + i] +
         u[c - sz + i] + u[c + sz + i];
}

// Node kernels run on 3D grids: x over i (32 threads), y over j (8), z over k -- no index division.
__host__ __device__ inline dim3 node_block() { return dim3(32, 8, 1); }
inline dim3 node_grid3(int nx, int ny, int nz) { return dim3((nx + 1 + 31) / 32, (ny + 1 + 7) / 8, nz + 1); }
#define NODE_IJK(nx, ny)                                       \
  const int i = blockIdx.x * 32 + threadIdx.x;               \
  const int j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z; \
  if (i > (nx) || j > (ny)) return;                           \
  const int64_t n = node_index(i, j, k, nx, ny);

// ---- split-colour level geometry -------------------------------------------------------------
struct Lv {
  int nx, ny, nz, Xh;
  int64_t nper;
};

inline Lv lv_of(const MgLevel &L) { return Lv{L.nx, L.ny, L.nz, L.Xh, L.nper}; }

__host__ __device__ __forceinline__ int64_t srow(const Lv &L, int j, int k) {
  return ((int64_t)k * (L.ny + 1) + j) * L.Xh;
}

// split index of node (i, j, k)
__host__ __device__ __forceinline__ int64_t sidx(const Lv &L, int i, int j, int k) {
  return (int64_t)((i + j + k) & 1) * L.nper + srow(L, j, k) + (i >> 1);
}

// planes per thread in the level sweeps
constexpr int kKZ = 4;

// slot grid: x over slots (32), y over j (8), z over groups of kKZ planes (x colours)
inline dim3 slot_grid(const Lv &L, int colours) {
  return dim3((L.Xh + 31) / 32, (L.ny + 1 + 7) / 8, ((L.nz + kKZ) / kKZ) * colours);
}

// sum of the 6 neighbours of colour-c node i in row (j, k), read from the other colour uo
template <typename T>
__device__ __forceinline__ T nb_sum_s(const T *uo, const Lv &L, int i, int t, int j, int k) {
  const int im = i > 0 ? i - 1 : 1, ip = i < L.nx ? i + 1 : L.nx - 1;
  const int jm = j > 0 ? j - 1 : 1, jp = j < L.ny ? j + 1 : L.ny - 1;
  const int64_t row = srow(L, j, k);
  return uo[row + (im >> 1)] + uo[row + (ip >> 1)] + uo[srow(L, jm, k) + t] + uo[srow(L, jp, k) + t] +
         uo[srow(L, j, k - 1) + t] + uo[srow(L, j, k + 1) + t];
}

// The fine-level sweeps are bound by memory latency, not bandwidth, when a thread waits for its
// mask before loading the stencil: each thread therefore takes kKZ planes (k0 .. k0 + kKZ - 1)
// and issues every load of all of them (mask, right-hand side, neighbours) before the first
// store.  Within one colour pass no value read is written, so the order is free.

// one colour of red-black Gauss-Seidel on A u = f (grid z: plane groups of kKZ)
template <typename T>
__global__ void k_smooth(T *u, const T *f, const uint8_t *dirs, Lv L, T h2, int c) {
  const int t = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y, k0 = blockIdx.z * kKZ;
  if (t >= L.Xh || j > L.ny) return;
  const T *uo = u + (int64_t)(c ^ 1) * L.nper;
  T v[kKZ];
  int64_t m[kKZ];
  bool ok[kKZ];
#pragma unroll
  for (int q = 0; q < kKZ; ++q) {
    const int k = k0 + q;
    const int i = 2 * t + ((j + k + c) & 1);
    ok[q] = k > 0 && k < L.nz && i <= L.nx;   // the k = 0 and k = nz planes are Dirichlet
    m[q] = (int64_t)c * L.nper + srow(L, j, k) + t;
    v[q] = 0;
    if (ok[q]) {
      ok[q] = !dirs[m[q]];
      v[q] = nb_sum_s<T>(uo, L, i, t, j, k) + h2 * f[m[q]];
    }
  }
#pragma unroll
  for (int q = 0; q < kKZ; ++q)
    if (ok[q]) u[m[q]] = v[q] * (T)(1.0 / 6.0);
}

// r = f - A u at every node (grid z: plane groups of kKZ x 2 colours)
template <typename T>
__global__ void k_residual(const T *u, const T *f, T *r, const uint8_t *dirs, Lv L, T inv_h2) {
  const int t = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y, k0 = (blockIdx.z >> 1) * kKZ, c = blockIdx.z & 1;
  if (t >= L.Xh || j > L.ny) return;
  const T *uo = u + (int64_t)(c ^ 1) * L.nper;
  T v[kKZ];
  int64_t m[kKZ];
  bool ok[kKZ];
#pragma unroll
  for (int q = 0; q < kKZ; ++q) {
    const int k = k0 + q;
    const int i = 2 * t + ((j + k + c) & 1);
    ok[q] = k <= L.nz && i <= L.nx;
    m[q] = (int64_t)c * L.nper + srow(L, j, k) + t;
    v[q] = 0;
    if (ok[q] && k > 0 && k < L.nz) {
      const bool d = dirs[m[q]];
      const T rr = f[m[q]] - (6 * u[m[q]] - nb_sum_s<T>(uo, L, i, t, j, k)) * inv_h2;
      v[q] = d ? (T)0 : rr;
    }
  }
#pragma unroll
  for (int q = 0; q < kKZ; ++q)
    if (ok[q]) r[m[q]] = v[q];
}

__device__ __forceinline__ int mirror(int i, int n) { return i < 0 ? -i : (i > n ? 2 * n - i : i); }

// full weighting of a fine residual onto the coarse right-hand side; coarse u cleared
template <typename TF, typename TC>
__global__ void k_restrict(const TF *rf, Lv Fl, TC *fc, TC *uc, const uint8_t *dirsc, Lv Cl) {
  const int I = blockIdx.x * 32 + threadIdx.x;
  const int J = blockIdx.y * 8 + threadIdx.y, K = blockIdx.z;
  if (I > Cl.nx || J > Cl.ny) return;
  const int64_t n = sidx(Cl, I, J, K);
  uc[n] = 0;
  if (dirsc[n]) { fc[n] = 0; return; }
  // accumulate in the level's precision (float in the mixed form)
  TC s = 0;
  for (int dk = -1; dk <= 1; ++dk) {
    const TC wk = dk == 0 ? (TC)0.5 : (TC)0.25;
    const int k = 2 * K + dk;
    for (int dj = -1; dj <= 1; ++dj) {
      const TC wj = dj == 0 ? (TC)0.5 : (TC)0.25;
      const int j = mirror(2 * J + dj, Fl.ny);
      TC row = 0;
      for (int di = -1; di <= 1; ++di) {
        const TC wi = di == 0 ? (TC)0.5 : (TC)0.25;
        const int i = mirror(2 * I + di, Fl.nx);
        row += wi * (TC)rf[sidx(Fl, i, j, k)];
      }
      s += wk * wj * row;
    }
  }
  fc[n] = s;
}

// trilinear prolongation of the coarse correction, added on free fine nodes (fine slot grid,
// z: plane groups of kKZ x 2 colours; all loads before the stores)
template <typename TC, typename TF>
__global__ void k_prolong(const TC *uc, Lv Cl, TF *uf, const uint8_t *dirsf, Lv Fl) {
  const int t = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y, kb = (blockIdx.z >> 1) * kKZ, c = blockIdx.z & 1;
  if (t >= Fl.Xh || j > Fl.ny) return;
  TF v[kKZ];
  int64_t m[kKZ];
  bool ok[kKZ];
#pragma unroll
  for (int q = 0; q < kKZ; ++q) {
    const int k = kb + q;
    const int i = 2 * t + ((j + k + c) & 1);
    ok[q] = k > 0 && k < Fl.nz && i <= Fl.nx;
    m[q] = (int64_t)c * Fl.nper + srow(Fl, j, k) + t;
    v[q] = 0;
    if (ok[q]) {
      ok[q] = !dirsf[m[q]];
      const int i0 = i >> 1, j0 = j >> 1, k0 = k >> 1;
      const int i1 = i0 + (i & 1), j1 = j0 + (j & 1), k1 = k0 + (k & 1);
      const TC s = (TC)0.125 * (uc[sidx(Cl, i0, j0, k0)] + uc[sidx(Cl, i1, j0, k0)] + uc[sidx(Cl, i0, j1, k0)] +
                                uc[sidx(Cl, i1, j1, k0)] + uc[sidx(Cl, i0, j0, k1)] + uc[sidx(Cl, i1, j0, k1)] +
                                uc[sidx(Cl, i0, j1, k1)] + uc[sidx(Cl, i1, j1, k1)]);
      v[q] = uf[m[q]] + (TF)s;
    }
  }
#pragma unroll
  for (int q = 0; q < kKZ; ++q)
    if (ok[q]) uf[m[q]] = v[q];
}

// many red-black sweeps on the (small) coarsest level inside one block
template <typename T>
__global__ void k_coarse(T *u, const T *f, const uint8_t *dirs, Lv L, T h2, int sweeps) {
  const int64_t rows = (int64_t)(L.ny + 1) * (L.nz + 1);
  const int64_t slots = rows * L.Xh;
  for (int s = 0; s < sweeps; ++s)
    for (int c = 0; c < 2; ++c) {
      const T *uo = u + (int64_t)(c ^ 1) * L.nper;
      for (int64_t q = threadIdx.x; q < slots; q += blockDim.x) {
        const int t = (int)(q % L.Xh);
        const int64_t rw = q / L.Xh;
        const int j = (int)(rw % (L.ny + 1)), k = (int)(rw / (L.ny + 1));
        const int i = 2 * t + ((j + k + c) & 1);
        const int64_t n = (int64_t)c * L.nper + q;
        if (i > L.nx || dirs[n]) continue;
        u[n] = (nb_sum_s<T>(uo, L, i, t, j, k) + h2 * f[n]) * (T)(1.0 / 6.0);
      }
      __syncthreads();
    }
}

// coarse natural mask from the fine nodes it coincides with
__global__ void k_inject_mask(const uint8_t *dirf, int nxf, int nyf, uint8_t *dirc, int nxc, int nyc, int nzc) {
  const int I = blockIdx.x * 32 + threadIdx.x;
  const int J = blockIdx.y * 8 + threadIdx.y, K = blockIdx.z;
  if (I > nxc || J > nyc) return;
  dirc[node_index(I, J, K, nxc, nyc)] = dirf[node_index(2 * I, 2 * J, 2 * K, nxf, nyf)];
}

// split-colour copy of a level's natural mask (slots without a node stay 1: never updated)
__global__ void k_split_mask(const uint8_t *dir, uint8_t *dirs, Lv L) {
  NODE_IJK(L.nx, L.ny)
  dirs[sidx(L, i, j, k)] = dir[n];
}

// ---- fine level <-> FP64 refinement ---------------------------------------------------------------
// rho/eps0 from the fixed-point charge; Dirichlet values on the mask (V0 in fixed point)
__global__ void k_rhs(const unsigned long long *Q, double *f, long long *phi, const uint8_t *dir, int nx, int ny, int nz,
                      double unit, long long V0fx, int zero_charge) {
  NODE_IJK(nx, ny)
  // 1/V_n relative to dx^3: 2 per lateral wall the node lies on; a power of two, so folding it
  // into the unit leaves the one rounding of Q unit unchanged
  const double ku = unit * (i == 0 || i == nx ? 2.0 : 1.0) * (j == 0 || j == ny ? 2.0 : 1.0);
  f[n] = zero_charge ? 0.0 : (double)(long long)Q[n] * ku;
  if (dir[n]) phi[n] = k == nz ? V0fx : 0;
}

// Residual of the FP64 system r = f - A phi, handed straight to the finest V-cycle level as its
// right-hand side (rounded to the level's type T, split-colour layout) with a zero initial
// correction.  The stencil 6 phi_n - sum of neighbours is an exact int64 sum of fixed-point
// values; one FMA turns it into r (c = 2^-40 / h^2).  The squared norms of h^2 r and of h^2
// times the lifted right-hand side (f - A phi_D: only the plane below the anode carries a
// nonzero Dirichlet term) are accumulated in FP32 -- they only decide convergence -- so the
// FP64 pipe (1/64 of the FP32 rate on this part) runs three operations per node.  3D launch
// with blocks (32, 8); block partials land at the block's linear id.
__device__ __forceinline__ long long nb_sum_fx(const long long *u, int i, int j, int k, int nx, int ny) {
  const int im = i > 0 ? i - 1 : 1, ip = i < nx ? i + 1 : nx - 1;
  const int jm = j > 0 ? j - 1 : 1, jp = j < ny ? j + 1 : ny - 1;
  const int64_t sy = nx + 1, sz = (int64_t)(nx + 1) * (ny + 1);
  const int64_t c = (int64_t)k * sz + (int64_t)j * sy;
  return u[c + im] + u[c + ip] + u[(int64_t)k * sz + (int64_t)jm * sy + i] + u[(int64_t)k * sz + (int64_t)jp * sy + i] +
         u[c - sz + i] + u[c + sz + i];
}

template <typename T>
__global__ void k_residual64(const long long *phi, const double *f, T *fl, T *ul, const uint8_t *dir, Lv L,
                             double c_fx, float h2f, float V0f, double *part, int lift) {
  __shared__ float sh[2][8];
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
  float s = 0.f, sl = 0.f;
  if (i <= nx && j <= ny) {
    const int64_t n = node_index(i, j, k, nx, ny);
    const int64_t m = sidx(L, i, j, k);
    ul[m] = 0;
    if (dir[n]) {
      fl[m] = 0;
    } else {
      const double fn = f[n];
      const long long t = 6 * phi[n] - nb_sum_fx(phi, i, j, k, nx, ny);
      const double rr = fma(-(double)t, c_fx, fn);
      fl[m] = (T)rr;
      const float rs = (float)rr * h2f;
      s = rs * rs;
      if (lift) {
        const float l = (float)fn * h2f + (k == nz - 1 ? V0f : 0.f);
        sl = l * l;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    sl += __shfl_down_sync(0xffffffffu, sl, o);
  }
  if (threadIdx.x == 0) { sh[0][threadIdx.y] = s; sh[1][threadIdx.y] = sl; }
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    float a = 0.f, b = 0.f;
    for (int w = 0; w < 8; ++w) { a += sh[0][w]; b += sh[1][w]; }
    const int64_t bid = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    part[2 * bid] = (double)a;
    part[2 * bid + 1] = (double)b;
  }
}

// Fixed-order two-stage reduction of nb (a, b) block partials: block q of stage 1 sums the
// contiguous chunk q (thread t takes every 256th entry, then a tree), stage 2 one block the chunks.
constexpr int kSumChunks = 128;
__global__ void __launch_bounds__(256) k_sum_stage1(const double *part, int64_t nb, double *mid) {
  __shared__ double sa[256], sb[256];
  const int64_t per = (nb + kSumChunks - 1) / kSumChunks;
  const int64_t q0 = (int64_t)blockIdx.x * per, q1 = q0 + per < nb ? q0 + per : nb;
  double a = 0.0, b = 0.0;
  for (int64_t q = q0 + threadIdx.x; q < q1; q += 256) { a += part[2 * q]; b += part[2 * q + 1]; }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) { sa[threadIdx.x] += sa[threadIdx.x + w]; sb[threadIdx.x] += sb[threadIdx.x + w]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { mid[2 * blockIdx.x] = sa[0]; mid[2 * blockIdx.x + 1] = sb[0]; }
}

__global__ void __launch_bounds__(kSumChunks) k_sum_stage2(const double *mid, double *out) {
  __shared__ double sa[kSumChunks], sb[kSumChunks];
  sa[threadIdx.x] = mid[2 * threadIdx.x];
  sb[threadIdx.x] = mid[2 * threadIdx.x + 1];
  __syncthreads();
  for (int w = kSumChunks / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) { sa[threadIdx.x] += sa[threadIdx.x + w]; sb[threadIdx.x] += sb[threadIdx.x + w]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[0] = sa[0]; out[1] = sb[0]; }
}

// phi += e on free nodes, e (finest level, split layout) rounded to the fixed-point grid without
// FP64 work: e 2^40 is exact in T and converts straight to int64 (z: plane groups of kKZ)
__device__ __forceinline__ long long to_fx(float e) { return __float2ll_rn(e * 1099511627776.0f); }
__device__ __forceinline__ long long to_fx(double e) { return __double2ll_rn(e * kPhiScale); }

template <typename T>
__global__ void k_correct(long long *phi, const T *u, const uint8_t *dir, Lv L) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y, k0 = blockIdx.z * kKZ;
  if (i > L.nx || j > L.ny) return;
  long long v[kKZ];
  bool ok[kKZ];
#pragma unroll
  for (int q = 0; q < kKZ; ++q) {
    const int k = k0 + q;
    ok[q] = k > 0 && k < L.nz;
    v[q] = 0;
    if (ok[q]) {
      const int64_t n = node_index(i, j, k, L.nx, L.ny);
      ok[q] = !dir[n];
      v[q] = phi[n] + to_fx(u[sidx(L, i, j, k)]);
    }
  }
#pragma unroll
  for (int q = 0; q < kKZ; ++q)
    if (ok[q]) phi[node_index(i, j, k0 + q, L.nx, L.ny)] = v[q];
}

// E = -grad phi at every node: the node difference rounded to f32, times f32(1/(2 dx)) (or
// f32(1/dx) on the z planes) in f32.  The difference of two fixed-point values is an exact
// int64; its f32 rounding equals that of the exact FP64 difference, and the 2^-40 folds into the
// f32 factor exactly, so no FP64 operation is needed.
__global__ void k_efield(const long long *phi, float4 *E, int nx, int ny, int nz, float c2, float c1) {
  const int64_t sy = nx + 1, sz = (int64_t)(nx + 1) * (ny + 1);
  {
    NODE_IJK(nx, ny)
    const int im = i > 0 ? i - 1 : 1, ip = i < nx ? i + 1 : nx - 1;
    const int jm = j > 0 ? j - 1 : 1, jp = j < ny ? j + 1 : ny - 1;
    const int64_t row = (int64_t)k * sz + (int64_t)j * sy;
    float4 e;
    e.x = __fmul_rn(__ll2float_rn(phi[row + im] - phi[row + ip]), c2);
    e.y = __fmul_rn(__ll2float_rn(phi[(int64_t)k * sz + (int64_t)jm * sy + i] - phi[(int64_t)k * sz + (int64_t)jp * sy + i]), c2);
    if (k == 0) e.z = __fmul_rn(__ll2float_rn(phi[n] - phi[n + sz]), c1);
    else if (k == nz) e.z = __fmul_rn(__ll2float_rn(phi[n - sz] - phi[n]), c1);
    else e.z = __fmul_rn(__ll2float_rn(phi[n - sz] - phi[n + sz]), c2);
    e.w = 0.f;
    E[n] = e;
  }
}

template <typename T>
static T *lvl_u(MgLevel &L);
template <>
float *lvl_u<float>(MgLevel &L) { return L.u; }
template <>
double *lvl_u<double>(MgLevel &L) { return L.ud; }
template <typename T>
static T *lvl_f(MgLevel &L);
template <>
float *lvl_f<float>(MgLevel &L) { return L.f; }
template <>
double *lvl_f<double>(MgLevel &L) { return L.fd; }
template <typename T>
static T *lvl_r(MgLevel &L);
template <>
float *lvl_r<float>(MgLevel &L) { return L.r; }
template <>
double *lvl_r<double>(MgLevel &L) { return L.rd; }

template <typename T>
static void vcycle(pic_t *h, int l) {
  MgLevel &L = h->mg[l];
  const Lv lv = lv_of(L);
  const T h2 = (T)(L.h * L.h), inv_h2 = (T)(1.0 / (L.h * L.h));
  const int last = (int)h->mg.size() - 1;
  if (l == last) {
    ++h->nlaunch;
    k_coarse<T><<<1, 1024, 0, h->stream>>>(lvl_u<T>(L), lvl_f<T>(L), L.dirs, lv, h2, 60);
    return;
  }
  const dim3 sg = slot_grid(lv, 1), sg2 = slot_grid(lv, 2), bl = node_block();
  for (int s = 0; s < 2; ++s)
    for (int c = 0; c < 2; ++c) { ++h->nlaunch; k_smooth<T><<<sg, bl, 0, h->stream>>>(lvl_u<T>(L), lvl_f<T>(L), L.dirs, lv, h2, c); }
  ++h->nlaunch;
  k_residual<T><<<sg2, bl, 0, h->stream>>>(lvl_u<T>(L), lvl_f<T>(L), lvl_r<T>(L), L.dirs, lv, inv_h2);
  MgLevel &Cl = h->mg[l + 1];
  const Lv cv = lv_of(Cl);
  ++h->nlaunch;
  k_restrict<T, T><<<node_grid3(Cl.nx, Cl.ny, Cl.nz), bl, 0, h->stream>>>(lvl_r<T>(L), lv, lvl_f<T>(Cl), lvl_u<T>(Cl),
                                                                       Cl.dirs, cv);
  vcycle<T>(h, l + 1);
  ++h->nlaunch;
  k_prolong<T, T><<<sg2, bl, 0, h->stream>>>(lvl_u<T>(Cl), cv, lvl_u<T>(L), L.dirs, lv);
  for (int s = 0; s < 2; ++s)
    for (int c = 1; c >= 0; --c) { ++h->nlaunch; k_smooth<T><<<sg, bl, 0, h->stream>>>(lvl_u<T>(L), lvl_f<T>(L), L.dirs, lv, h2, c); }
}

// one V-cycle on A e = r (r already on the finest level, e = 0 there) and phi += e
template <typename T>
static void cycle_fine(pic_t *h) {
  MgLevel &L = h->mg[0];
  vcycle<T>(h, 0);
  ++h->nlaunch;
  const dim3 g((L.nx + 1 + 31) / 32, (L.ny + 1 + 7) / 8, (L.nz + 1 + kKZ - 1) / kKZ);
  k_correct<T><<<g, node_block(), 0, h->stream>>>(h->phi, lvl_u<T>(L), L.dir, lv_of(L));
}

int stage_efield(pic_t *h) {
  ++h->nlaunch;
  // f32(1/(2 dx)) 2^-40 and f32(1/dx) 2^-40: rounding then scaling by a power of two
  const float c2 = (float)(1.0 / (2.0 * h->dx)) * (float)kPhiUnit, c1 = (float)(1.0 / h->dx) * (float)kPhiUnit;
  k_efield<<<node_grid3(h->nx, h->ny, h->nz), node_block(), 0, h->stream>>>(h->phi, h->E, h->nx, h->ny, h->nz, c2, c1);
  return launch_check(h, "efield");
}

int mg_build_masks(pic_t *h) {
  for (size_t l = 1; l < h->mg.size(); ++l) {
    MgLevel &F = h->mg[l - 1], &Cl = h->mg[l];
    ++h->nlaunch;
    k_inject_mask<<<node_grid3(Cl.nx, Cl.ny, Cl.nz), node_block(), 0, h->stream>>>(F.dir, F.nx, F.ny, Cl.dir, Cl.nx, Cl.ny,
                                                                                  Cl.nz);
  }
  for (size_t l = 0; l < h->mg.size(); ++l) {
    MgLevel &L = h->mg[l];
    PIC_CUDA(h, cudaMemsetAsync(L.dirs, 1, (size_t)2 * L.nper, h->stream));
    ++h->nlaunch;
    k_split_mask<<<node_grid3(L.nx, L.ny, L.nz), node_block(), 0, h->stream>>>(L.dir, L.dirs, lv_of(L));
  }
  return launch_check(h, "mg_masks");
}

// Solve for phi with the current deposited charge (or none), anode at V0.
int stage_solve(pic_t *h, bool zero_charge, double V0) {
  MgLevel &L = h->mg[0];
  const Lv lv = lv_of(L);
  const double unit = kQe * h->prm.w_min / 1073741824.0 / (h->dx * h->dx * h->dx) / kEps0;
  ++h->nlaunch;
  const long long V0fx = llrint(V0 * kPhiScale);
  k_rhs<<<node_grid3(h->nx, h->ny, h->nz), node_block(), 0, h->stream>>>(h->Q, h->rhs, h->phi, L.dir, h->nx, h->ny, h->nz,
                                                                         unit, V0fx, zero_charge ? 1 : 0);
  const dim3 rg = node_grid3(h->nx, h->ny, h->nz);
  const int64_t nb = (int64_t)rg.x * rg.y * rg.z;
  const double inv_h2 = 1.0 / (h->dx * h->dx), c_fx = inv_h2 * kPhiUnit;
  const bool mixed = (h->prm.flags & PIC_F_MIXED_MG) != 0;
  double norms[2] = {0, 0};
  double lifted = 0.0;
  int cyc = 0;
  const float h2f = (float)(h->dx * h->dx), V0f = (float)V0;
  for (;; ++cyc) {
    ++h->nlaunch;
    if (mixed)
      k_residual64<float><<<rg, node_block(), 0, h->stream>>>(h->phi, h->rhs, L.f, L.u, L.dir, lv, c_fx, h2f, V0f,
                                                              h->red, cyc == 0 ? 1 : 0);
    else
      k_residual64<double><<<rg, node_block(), 0, h->stream>>>(h->phi, h->rhs, L.fd, L.ud, L.dir, lv, c_fx, h2f,
                                                               V0f, h->red, cyc == 0 ? 1 : 0);
    h->nlaunch += 2;
    k_sum_stage1<<<kSumChunks, 256, 0, h->stream>>>(h->red, nb, h->red_mid);
    k_sum_stage2<<<1, kSumChunks, 0, h->stream>>>(h->red_mid, h->red_out);
    PIC_CUDA(h, cudaMemcpyAsync(norms, h->red_out, sizeof norms, cudaMemcpyDeviceToHost, h->stream));
    PIC_CUDA(h, cudaStreamSynchronize(h->stream));
    if (cyc == 0) lifted = sqrt(norms[1]);
    const double rel = lifted > 0 ? sqrt(norms[0]) / lifted : sqrt(norms[0]);
    h->last_mg_res = rel;
    h->last_mg_cycles = cyc;
    if (rel <= h->prm.mg_tol) break;
    if (cyc >= h->prm.mg_max_cycles) {
      PIC_TRY(stage_efield(h));
      return pic_fail(h, PIC_E_NOCONV, "Poisson solve: relative residual " + std::to_string(rel) + " after " +
                                           std::to_string(cyc) + " cycles");
    }
    if (mixed) cycle_fine<float>(h);
    else cycle_fine<double>(h);
  }
  return stage_efield(h);
}

}  // namespace pic
