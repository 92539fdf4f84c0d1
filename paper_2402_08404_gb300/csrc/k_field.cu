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
#include "pic_internal.cuh"

namespace pic {

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
inline dim3 color_grid3(int nx, int ny, int nz) { return dim3(((nx + 2) / 2 + 31) / 32, (ny + 1 + 7) / 8, nz + 1); }
#define NODE_IJK(nx, ny)                                       \
  const int i = blockIdx.x * 32 + threadIdx.x;               \
  const int j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z; \
  if (i > (nx) || j > (ny)) return;                           \
  const int64_t n = node_index(i, j, k, nx, ny);

// one colour of red-black Gauss-Seidel on A u = f
template <typename T>
__global__ void k_smooth(T *u, const T *f, const uint8_t *dir, int nx, int ny, int nz, T h2, int color) {
  const int j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
  const int i = 2 * (blockIdx.x * 32 + threadIdx.x) + ((j + k + color) & 1);
  if (i > nx || j > ny) return;
  const int64_t n = node_index(i, j, k, nx, ny);
  if (dir[n]) return;
  u[n] = (nb_sum<T>(u, i, j, k, nx, ny) + h2 * f[n]) * (T)(1.0 / 6.0);
}

template <typename T>
__global__ void k_residual(const T *u, const T *f, T *r, const uint8_t *dir, int nx, int ny, int nz, T inv_h2) {
  NODE_IJK(nx, ny)
  if (dir[n]) { r[n] = 0; return; }
  r[n] = f[n] - (6 * u[n] - nb_sum<T>(u, i, j, k, nx, ny)) * inv_h2;
}

__device__ __forceinline__ int mirror(int i, int n) { return i < 0 ? -i : (i > n ? 2 * n - i : i); }

// full weighting of a fine residual onto the coarse right-hand side; coarse u cleared
template <typename TF, typename TC>
__global__ void k_restrict(const TF *rf, int nxf, int nyf, TC *fc, TC *uc, const uint8_t *dirc, int nxc, int nyc, int nzc) {
  {
    const int I = blockIdx.x * 32 + threadIdx.x;
    const int J = blockIdx.y * 8 + threadIdx.y, K = blockIdx.z;
    if (I > nxc || J > nyc) return;
    const int64_t n = node_index(I, J, K, nxc, nyc);
    uc[n] = 0;
    if (dirc[n]) { fc[n] = 0; return; }
    // accumulate in the level's precision (float in the mixed form)
    TC s = 0;
    for (int dk = -1; dk <= 1; ++dk) {
      const TC wk = dk == 0 ? (TC)0.5 : (TC)0.25;
      const int k = 2 * K + dk;
      for (int dj = -1; dj <= 1; ++dj) {
        const TC wj = dj == 0 ? (TC)0.5 : (TC)0.25;
        const int j = mirror(2 * J + dj, nyf);
        TC row = 0;
        for (int di = -1; di <= 1; ++di) {
          const TC wi = di == 0 ? (TC)0.5 : (TC)0.25;
          const int i = mirror(2 * I + di, nxf);
          row += wi * (TC)rf[node_index(i, j, k, nxf, nyf)];
        }
        s += wk * wj * row;
      }
    }
    fc[n] = s;
  }
}

// trilinear prolongation of the coarse correction, added on free fine nodes
template <typename TC, typename TF>
__global__ void k_prolong(const TC *uc, int nxc, int nyc, TF *uf, const uint8_t *dirf, int nxf, int nyf, int nzf) {
  {
    NODE_IJK(nxf, nyf)
    if (dirf[n]) return;
    const int i0 = i >> 1, j0 = j >> 1, k0 = k >> 1;
    const int i1 = i0 + (i & 1), j1 = j0 + (j & 1), k1 = k0 + (k & 1);
    const TC v = (TC)0.125 * (uc[node_index(i0, j0, k0, nxc, nyc)] + uc[node_index(i1, j0, k0, nxc, nyc)] +
                              uc[node_index(i0, j1, k0, nxc, nyc)] + uc[node_index(i1, j1, k0, nxc, nyc)] +
                              uc[node_index(i0, j0, k1, nxc, nyc)] + uc[node_index(i1, j0, k1, nxc, nyc)] +
                              uc[node_index(i0, j1, k1, nxc, nyc)] + uc[node_index(i1, j1, k1, nxc, nyc)]);
    uf[n] += (TF)v;
  }
}

// many red-black sweeps on the (small) coarsest level inside one block
template <typename T>
__global__ void k_coarse(T *u, const T *f, const uint8_t *dir, int nx, int ny, int nz, T h2, int sweeps) {
  const int64_t total = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  for (int s = 0; s < sweeps; ++s)
    for (int color = 0; color < 2; ++color) {
      for (int64_t n = threadIdx.x; n < total; n += blockDim.x) {
        const int i = (int)(n % (nx + 1));
        const int64_t q = n / (nx + 1);
        const int j = (int)(q % (ny + 1)), k = (int)(q / (ny + 1));
        if (((i + j + k) & 1) != color || dir[n]) continue;
        u[n] = (nb_sum<T>(u, i, j, k, nx, ny) + h2 * f[n]) * (T)(1.0 / 6.0);
      }
      __syncthreads();
    }
}

__global__ void k_inject_mask(const uint8_t *dirf, int nxf, int nyf, uint8_t *dirc, int nxc, int nyc, int nzc) {
  const int I = blockIdx.x * 32 + threadIdx.x;
  const int J = blockIdx.y * 8 + threadIdx.y, K = blockIdx.z;
  if (I > nxc || J > nyc) return;
  dirc[node_index(I, J, K, nxc, nyc)] = dirf[node_index(2 * I, 2 * J, 2 * K, nxf, nyf)];
}

// rho/eps0 from the fixed-point charge; Dirichlet values on the mask
__global__ void k_rhs(const unsigned long long *Q, double *f, double *phi, const uint8_t *dir, int nx, int ny, int nz,
                      double unit, double V0, int zero_charge) {
  NODE_IJK(nx, ny)
  // 1/V_n relative to dx^3: 2 per lateral wall the node lies on (exact powers of two)
  const double inv_vol = (i == 0 || i == nx ? 2.0 : 1.0) * (j == 0 || j == ny ? 2.0 : 1.0);
  f[n] = zero_charge ? 0.0 : (double)(long long)Q[n] * unit * inv_vol;
  if (dir[n]) phi[n] = k == nz ? V0 : 0.0;
}

// Residual of the FP64 system r = f - A phi, handed straight to the finest V-cycle level as its
// right-hand side (rounded to the level's type T) with a zero initial correction.  The squared
// norms of h^2 r and of h^2 times the lifted right-hand side (f - A phi_D: only the plane below
// the anode carries a nonzero Dirichlet term) are accumulated in FP32 -- they only decide
// convergence -- so the FP64 pipe (1/64 of the FP32 rate on this part) runs just the stencil.
// 3D launch with blocks (32, 8); block partials land at the block's linear id.
template <typename T>
__global__ void k_residual64(const double *phi, const double *f, T *fl, T *ul, const uint8_t *dir, int nx, int ny,
                             int nz, double inv_h2, float h2f, float V0f, double *part, int lift) {
  __shared__ float sh[2][8];
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
  float s = 0.f, sl = 0.f;
  if (i <= nx && j <= ny) {
    const int64_t n = node_index(i, j, k, nx, ny);
    ul[n] = 0;
    if (dir[n]) {
      fl[n] = 0;
    } else {
      const double fn = f[n];
      const double t = fma(6.0, phi[n], -nb_sum<double>(phi, i, j, k, nx, ny));
      const double rr = fma(-t, inv_h2, fn);
      fl[n] = (T)rr;
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

// fixed-order reduction of nb block partials: thread t sums blocks t, t+1024, ... then a tree
__global__ void __launch_bounds__(1024) k_sum_partials(const double *part, int64_t nb, double *out) {
  __shared__ double sa[1024], sb[1024];
  double a = 0.0, b = 0.0;
  for (int64_t q = threadIdx.x; q < nb; q += 1024) { a += part[2 * q]; b += part[2 * q + 1]; }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) { sa[threadIdx.x] += sa[threadIdx.x + w]; sb[threadIdx.x] += sb[threadIdx.x + w]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[0] = sa[0]; out[1] = sb[0]; }
}

template <typename T>
__global__ void k_correct(double *phi, const T *u, const uint8_t *dir, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!dir[i]) phi[i] += (double)u[i];
}

// E = -grad phi at every node, float64 differences rounded once to float32
__global__ void k_efield(const double *phi, float4 *E, int nx, int ny, int nz, double inv2dx, double invdx) {
  const int64_t sy = nx + 1, sz = (int64_t)(nx + 1) * (ny + 1);
  {
    NODE_IJK(nx, ny)
    const int im = i > 0 ? i - 1 : 1, ip = i < nx ? i + 1 : nx - 1;
    const int jm = j > 0 ? j - 1 : 1, jp = j < ny ? j + 1 : ny - 1;
    const int64_t row = (int64_t)k * sz + (int64_t)j * sy;
    float4 e;
    e.x = __double2float_rn(__dmul_rn(__dsub_rn(phi[row + im], phi[row + ip]), inv2dx));
    e.y = __double2float_rn(__dmul_rn(__dsub_rn(phi[(int64_t)k * sz + (int64_t)jm * sy + i], phi[(int64_t)k * sz + (int64_t)jp * sy + i]), inv2dx));
    if (k == 0) e.z = __double2float_rn(__dmul_rn(__dsub_rn(phi[n], phi[n + sz]), invdx));
    else if (k == nz) e.z = __double2float_rn(__dmul_rn(__dsub_rn(phi[n - sz], phi[n]), invdx));
    else e.z = __double2float_rn(__dmul_rn(__dsub_rn(phi[n - sz], phi[n + sz]), inv2dx));
    e.w = 0.f;
    E[n] = e;
  }
}

static int node_grid(pic_t *h, int64_t n) {
  int64_t g = (n + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)h->nsm * 16;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
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
  const T h2 = (T)(L.h * L.h), inv_h2 = (T)(1.0 / (L.h * L.h));
  const int last = (int)h->mg.size() - 1;
  if (l == last) {
    ++h->nlaunch;
    k_coarse<T><<<1, 1024, 0, h->stream>>>(lvl_u<T>(L), lvl_f<T>(L), L.dir, L.nx, L.ny, L.nz, h2, 60);
    return;
  }
  const dim3 cg = color_grid3(L.nx, L.ny, L.nz), bl = node_block();
  for (int s = 0; s < 2; ++s)
    for (int c = 0; c < 2; ++c) { ++h->nlaunch; k_smooth<T><<<cg, bl, 0, h->stream>>>(lvl_u<T>(L), lvl_f<T>(L), L.dir, L.nx, L.ny, L.nz, h2, c); }
  ++h->nlaunch;
  k_residual<T><<<node_grid3(L.nx, L.ny, L.nz), bl, 0, h->stream>>>(lvl_u<T>(L), lvl_f<T>(L), lvl_r<T>(L), L.dir, L.nx,
                                                                 L.ny, L.nz, inv_h2);
  MgLevel &Cl = h->mg[l + 1];
  ++h->nlaunch;
  k_restrict<T, T><<<node_grid3(Cl.nx, Cl.ny, Cl.nz), bl, 0, h->stream>>>(lvl_r<T>(L), L.nx, L.ny, lvl_f<T>(Cl), lvl_u<T>(Cl),
                                                                       Cl.dir, Cl.nx, Cl.ny, Cl.nz);
  vcycle<T>(h, l + 1);
  ++h->nlaunch;
  k_prolong<T, T><<<node_grid3(L.nx, L.ny, L.nz), bl, 0, h->stream>>>(lvl_u<T>(Cl), Cl.nx, Cl.ny, lvl_u<T>(L), L.dir, L.nx,
                                                                     L.ny, L.nz);
  for (int s = 0; s < 2; ++s)
    for (int c = 1; c >= 0; --c) { ++h->nlaunch; k_smooth<T><<<cg, bl, 0, h->stream>>>(lvl_u<T>(L), lvl_f<T>(L), L.dir, L.nx, L.ny, L.nz, h2, c); }
}

// one V-cycle on A e = r (r already on the finest level, e = 0 there) and phi += e
template <typename T>
static void cycle_fine(pic_t *h) {
  MgLevel &L = h->mg[0];
  vcycle<T>(h, 0);
  ++h->nlaunch;
  k_correct<T><<<node_grid(h, L.nnode), kThreads, 0, h->stream>>>(h->phi, lvl_u<T>(L), L.dir, L.nnode);
}

int stage_efield(pic_t *h) {
  ++h->nlaunch;
  k_efield<<<node_grid3(h->nx, h->ny, h->nz), node_block(), 0, h->stream>>>(h->phi, h->E, h->nx, h->ny, h->nz,
                                                                            1.0 / (2.0 * h->dx), 1.0 / h->dx);
  return launch_check(h, "efield");
}

int mg_build_masks(pic_t *h) {
  for (size_t l = 1; l < h->mg.size(); ++l) {
    MgLevel &F = h->mg[l - 1], &Cl = h->mg[l];
    ++h->nlaunch;
    k_inject_mask<<<node_grid3(Cl.nx, Cl.ny, Cl.nz), node_block(), 0, h->stream>>>(F.dir, F.nx, F.ny, Cl.dir, Cl.nx, Cl.ny,
                                                                                  Cl.nz);
  }
  return launch_check(h, "mg_masks");
}

// Solve for phi with the current deposited charge (or none), anode at V0.
int stage_solve(pic_t *h, bool zero_charge, double V0) {
  MgLevel &L = h->mg[0];
  const double unit = kQe * h->prm.w_min / 1073741824.0 / (h->dx * h->dx * h->dx) / kEps0;
  ++h->nlaunch;
  k_rhs<<<node_grid3(h->nx, h->ny, h->nz), node_block(), 0, h->stream>>>(h->Q, h->rhs, h->phi, L.dir, h->nx, h->ny, h->nz,
                                                                         unit, V0, zero_charge ? 1 : 0);
  const dim3 rg = node_grid3(h->nx, h->ny, h->nz);
  const int64_t nb = (int64_t)rg.x * rg.y * rg.z;
  const double inv_h2 = 1.0 / (h->dx * h->dx);
  const bool mixed = (h->prm.flags & PIC_F_MIXED_MG) != 0;
  double norms[2] = {0, 0};
  double lifted = 0.0;
  int cyc = 0;
  const float h2f = (float)(h->dx * h->dx), V0f = (float)V0;
  for (;; ++cyc) {
    ++h->nlaunch;
    if (mixed)
      k_residual64<float><<<rg, node_block(), 0, h->stream>>>(h->phi, h->rhs, L.f, L.u, L.dir, h->nx, h->ny, h->nz,
                                                              inv_h2, h2f, V0f, h->red, cyc == 0 ? 1 : 0);
    else
      k_residual64<double><<<rg, node_block(), 0, h->stream>>>(h->phi, h->rhs, L.fd, L.ud, L.dir, h->nx, h->ny,
                                                               h->nz, inv_h2, h2f, V0f, h->red, cyc == 0 ? 1 : 0);
    ++h->nlaunch;
    k_sum_partials<<<1, 1024, 0, h->stream>>>(h->red, nb, h->red_out);
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
