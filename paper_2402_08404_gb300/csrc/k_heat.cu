// Tip heat step (eq:heat with Wiedemann-Franz kappa = L T sigma) and current continuity
// (eq:cont) on the solid tip cells, every n_heat PIC steps (Sec. 2.1).
//
// Finite volumes: internal faces couple neighbouring tip cells with coefficients
// mean(p_a, p_b) dx^2/dx; the bottom faces of k = 0 cells are the bulk bottom (phi_J = 0,
// T = T_amb) at half a cell.  Surface heat (Nottingham + evaporation + bombardment, eq:bct1)
// and emitted current enter each tip face's owner cell.  Implicit Euler over dt_heat with
// kappa, sigma at the old temperature.  Joule power of a cell is half the dissipation
// I_f dphi_f of each of its internal faces plus its base faces.  Both SPD systems are solved
// by conjugate gradients inside one block (deterministic reduction order).
// Cu resistivity and heat capacity are not printed by the paper: stand-ins
// rho_e = 1.72e-8 T/293 Ohm m, C_v = 3.45e6 J m^-3 K^-1.
#include "pic_internal.cuh"

namespace pic {

constexpr double kCv = 3.45e6;
constexpr double kRho293 = 1.72e-8;

__global__ void k_heat_sources(const int32_t *owner_vox, int64_t nface, const double *acc_heat, const double *acc_charge,
                               const long long *Eb, const long long *Es, double dth, double *src, double *cur) {
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nface; f += (int64_t)gridDim.x * blockDim.x) {
    const int v = owner_vox[f];
    if (v < 0) continue;
    const double eb = (double)(Eb[f] - Es[f]) * 9.5367431640625e-07 * kQe;   // 2^-20 eV -> J
    atomicAdd(&src[v], (acc_heat[f] + eb) / dth);
    atomicAdd(&cur[v], acc_charge[f] / dth);
  }
}

__device__ double block_sum_d(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    sh[32] = s;
  }
  __syncthreads();
  const double s = sh[32];
  __syncthreads();
  return s;
}

struct HeatArgs {
  int64_t nvox;
  const int32_t *nbr;
  const uint8_t *base;
  double *T, *sig, *kap, *src, *cur, *phiJ, *joule, *p, *q, *r, *b;
  double A_over_dx, m, T_amb;
  int *status;
};

// y = K x with K from the per-cell property prop: internal faces mean(prop) A/dx, base faces
// 2 prop A/dx, plus a diagonal shift `shift`
__device__ void apply_K(const HeatArgs &a, const double *prop, double shift, const double *x, double *y) {
  for (int64_t v = threadIdx.x; v < a.nvox; v += blockDim.x) {
    double s = (shift + (a.base[v] ? 2.0 * prop[v] * a.A_over_dx : 0.0)) * x[v];
    for (int d = 0; d < 6; ++d) {
      const int u = a.nbr[6 * v + d];
      if (u >= 0) s += 0.5 * (prop[v] + prop[u]) * a.A_over_dx * (x[v] - x[u]);
    }
    y[v] = s;
  }
}

// CG on K x = b (x holds the initial guess); returns iterations or -1 on no convergence
__device__ int cg_solve(const HeatArgs &a, const double *prop, double shift, double *x, const double *b, double *sh) {
  apply_K(a, prop, shift, x, a.q);
  __syncthreads();
  double rr = 0.0, bb = 0.0;
  for (int64_t v = threadIdx.x; v < a.nvox; v += blockDim.x) {
    a.r[v] = b[v] - a.q[v];
    a.p[v] = a.r[v];
    rr += a.r[v] * a.r[v];
    bb += b[v] * b[v];
  }
  rr = block_sum_d(rr, sh);
  bb = block_sum_d(bb, sh);
  if (bb == 0.0) return 0;
  const double tol2 = 1e-26 * bb;
  for (int it = 0; it < 20000; ++it) {
    if (rr <= tol2) return it;
    apply_K(a, prop, shift, a.p, a.q);
    __syncthreads();
    double pq = 0.0;
    for (int64_t v = threadIdx.x; v < a.nvox; v += blockDim.x) pq += a.p[v] * a.q[v];
    pq = block_sum_d(pq, sh);
    const double alpha = rr / pq;
    double rn = 0.0;
    for (int64_t v = threadIdx.x; v < a.nvox; v += blockDim.x) {
      x[v] += alpha * a.p[v];
      a.r[v] -= alpha * a.q[v];
      rn += a.r[v] * a.r[v];
    }
    rn = block_sum_d(rn, sh);
    const double beta = rn / rr;
    rr = rn;
    for (int64_t v = threadIdx.x; v < a.nvox; v += blockDim.x) a.p[v] = a.r[v] + beta * a.p[v];
    __syncthreads();
  }
  return -1;
}

__global__ void __launch_bounds__(1024) k_heat_solve(HeatArgs a) {
  __shared__ double sh[33];
  bool any_cur = false;
  for (int64_t v = threadIdx.x; v < a.nvox; v += blockDim.x) {
    const double T = a.T[v];
    a.sig[v] = 1.0 / (kRho293 * T / 293.0);
    a.kap[v] = kLorentz * T * a.sig[v];
    a.phiJ[v] = 0.0;
    if (a.cur[v] != 0.0) any_cur = true;
  }
  any_cur = __syncthreads_or(any_cur);
  int st = 0;
  if (any_cur && cg_solve(a, a.sig, 0.0, a.phiJ, a.cur, sh) < 0) st = 1;
  __syncthreads();
  // Joule power per cell
  for (int64_t v = threadIdx.x; v < a.nvox; v += blockDim.x) {
    double jv = a.base[v] ? 2.0 * a.sig[v] * a.A_over_dx * a.phiJ[v] * a.phiJ[v] : 0.0;
    for (int d = 0; d < 6; ++d) {
      const int u = a.nbr[6 * v + d];
      if (u >= 0) {
        const double dphi = a.phiJ[v] - a.phiJ[u];
        jv += 0.5 * 0.5 * (a.sig[v] + a.sig[u]) * a.A_over_dx * dphi * dphi;
      }
    }
    a.joule[v] = jv;
  }
  __syncthreads();
  // implicit heat step: (K_th + m) T' = m T + base kappa T_amb + S + Joule
  for (int64_t v = threadIdx.x; v < a.nvox; v += blockDim.x) {
    a.b[v] = a.m * a.T[v] + (a.base[v] ? 2.0 * a.kap[v] * a.A_over_dx * a.T_amb : 0.0) + a.src[v] + a.joule[v];
  }
  __syncthreads();
  if (cg_solve(a, a.kap, a.m, a.T, a.b, sh) < 0) st |= 2;
  if (threadIdx.x == 0) *a.status = st;
}

int stage_heat(pic_t *h) {
  Heat &H = h->heat;
  if (H.nvox == 0) return PIC_OK;
  const double dth = h->prm.dt * (h->prm.n_heat > 0 ? h->prm.n_heat : 1);
  PIC_CUDA(h, cudaMemsetAsync(H.src, 0, H.nvox * sizeof(double), h->stream));
  PIC_CUDA(h, cudaMemsetAsync(H.cur, 0, H.nvox * sizeof(double), h->stream));
  Faces &fc = h->faces;
  ++h->nlaunch;
  k_heat_sources<<<grid_for(fc.n), kThreads, 0, h->stream>>>(fc.owner_vox, fc.n, fc.acc_heat, fc.acc_charge,
                                                             (const long long *)fc.acc_Eb, (const long long *)fc.acc_Es,
                                                             dth, H.src, H.cur);
  HeatArgs a;
  a.nvox = H.nvox; a.nbr = H.nbr; a.base = H.base; a.T = H.T; a.sig = H.sig; a.kap = H.kap; a.src = H.src;
  a.cur = H.cur; a.phiJ = H.phiJ; a.joule = H.joule; a.p = H.p; a.q = H.q; a.r = H.res; a.b = H.zv;
  a.A_over_dx = h->dx;
  a.m = kCv * h->dx * h->dx * h->dx / dth;
  a.T_amb = h->prm.T0;
  int *status = h->long_n + 7;
  a.status = status;
  ++h->nlaunch;
  k_heat_solve<<<1, 1024, 0, h->stream>>>(a);
  PIC_CUDA(h, cudaMemsetAsync(fc.acc_heat, 0, fc.n * sizeof(double), h->stream));
  PIC_CUDA(h, cudaMemsetAsync(fc.acc_charge, 0, fc.n * sizeof(double), h->stream));
  PIC_CUDA(h, cudaMemsetAsync(fc.acc_Eb, 0, fc.n * sizeof(int64_t), h->stream));
  PIC_CUDA(h, cudaMemsetAsync(fc.acc_Es, 0, fc.n * sizeof(int64_t), h->stream));
  return launch_check(h, "heat");
}

}  // namespace pic
