// Surface stage: local face field, thermal-field emission of electrons (Sec. 2.3.1),
// evaporation (Clausius-Clapeyron, Sec. 2.3.1) and sputter injection (Sec. 2.3.3) with the
// injection-weight rule of Sec. 2.3.2.
//
// Per face (one thread each): counts of new SPs; an exclusive scan in face order then gives
// every new SP its slot and its id, so creation is deterministic.
#include "pic_internal.cuh"
#include "gtf.cuh"
#include "dev_common.cuh"

namespace pic {

__constant__ double c_gl16x[16], c_gl16w[16], c_gl32x[32], c_gl32w[32], c_gl32c[32], c_gl32s[32];
__constant__ float c_gl32wf[32], c_gl32cf[32], c_gl32sf[32];
__constant__ gtf::Consts c_gtf;

struct FaceGeom {
  int axis, sign, plane;
  int ijk[3];
  int t0, t1;
};

__device__ __forceinline__ FaceGeom face_geom(int32_t vcell, int dir, int nx, int ny) {
  FaceGeom g;
  g.ijk[0] = vcell % nx;
  g.ijk[1] = (vcell / nx) % ny;
  g.ijk[2] = vcell / (nx * ny);
  g.axis = dir >> 1;
  if ((dir & 1) == 0) { g.plane = g.ijk[g.axis]; g.sign = 1; }
  else { g.plane = g.ijk[g.axis] + 1; g.sign = -1; }
  g.t0 = g.axis == 0 ? 1 : 0;
  g.t1 = g.axis == 2 ? 1 : 2;
  return g;
}

// A point on the face at tangential fractions (ua, ub), inside the vacuum cell.
__device__ __forceinline__ void face_point(const FaceGeom &g, float ua, float ub, float pos[3]) {
  const float pn = (float)g.plane;
  pos[g.axis] = g.sign > 0 ? pn : nextafterf(pn, -INFINITY);
  const float a = __fadd_rn((float)g.ijk[g.t0], ua), b = __fadd_rn((float)g.ijk[g.t1], ub);
  pos[g.t0] = fminf(a, nextafterf((float)(g.ijk[g.t0] + 1), -INFINITY));
  pos[g.t1] = fminf(b, nextafterf((float)(g.ijk[g.t1] + 1), -INFINITY));
}

// F_f = mean over the 4 corners of (phi one dx outward - phi at the corner) / dx
__global__ void k_face_field(const int32_t *vcell, const int8_t *dir, int64_t nface, const long long *phi, int nx,
                             int ny, double dx, double *F) {
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nface; f += (int64_t)gridDim.x * blockDim.x) {
    const FaceGeom g = face_geom(vcell[f], dir[f], nx, ny);
    double acc = 0.0;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        int c[3];
        c[g.axis] = g.plane;
        c[g.t0] = g.ijk[g.t0] + a;
        c[g.t1] = g.ijk[g.t1] + b;
        int o[3] = {c[0], c[1], c[2]};
        o[g.axis] = g.plane + g.sign;
        // the FP64 difference of two fixed-point values, exactly
        const long long d = phi[node_index(o[0], o[1], o[2], nx, ny)] - phi[node_index(c[0], c[1], c[2], nx, ny)];
        acc = __dadd_rn(acc, (double)d * kPhiUnit);
      }
    F[f] = acc / 4.0 / dx;
  }
}

__device__ __forceinline__ gtf::Tables dev_tables() {
  gtf::Tables t;
  t.x16 = c_gl16x; t.w16 = c_gl16w; t.x32 = c_gl32x; t.w32 = c_gl32w; t.c32 = c_gl32c; t.s32 = c_gl32s;
  t.w32f = c_gl32wf; t.c32f = c_gl32cf; t.s32f = c_gl32sf;
  return t;
}

template <bool kFast>
__global__ void k_emission_eval(const double *F, const double *T, const double *W, const double *R, double *J,
                                double *PN, int64_t n) {
  const gtf::Tables tb = dev_tables();
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    double j, p;
    gtf::current_density_warp<kFast>(c_gtf, tb, F[i] * 1e-9, T[i], W[i], R[i] > 0 ? R[i] * 1e9 : -1.0, &j, &p);
    if ((threadIdx.x & 31) == 0) {
      J[i] = j;
      PN[i] = p;
    }
  }
}

struct EmitArgs {
  const int32_t *vcell, *owner_vox;
  const int8_t *dir;
  int64_t nface;
  const double *F, *Tvox;
  double T0, phi_w, R_nm, A, dt, w_min;
  double *J, *PN, *acc_heat, *acc_charge;
  uint32_t *cnt;
  uint64_t seed;
  DevClock *clk;
  const uint8_t *elig;   // surrogate: eligible faces (null: full integral everywhere)
  const float *Y;
  int32_t *fb_list;      // surrogate pass: faces left for the integral (compacted, any order)
  int *fb_n;
};

// finish one face once (J, P) are known: accumulators and the emission count
__device__ __forceinline__ void emit_finish(const EmitArgs &a, int64_t f, int64_t step, double J, double P) {
  a.J[f] = J;
  a.PN[f] = P;
  a.acc_heat[f] += P * a.A * a.dt;
  a.acc_charge[f] += J * a.A * a.dt;
  const double lam = J * a.A * a.dt / (kQe * a.w_min);
  const double base = floor(lam);
  const U4 r = rng_block(a.seed, kEmit, (uint64_t)f, step, 0);
  const double U = u01d(r.v[0]);
  a.cnt[f] = (uint32_t)base + (U < lam - base ? 1u : 0u);
}

// surrogate pass: eligible faces and faces without a pulling field are finished here, the
// others are queued for k_emit_fallback (results do not depend on the queue order)
__global__ void k_emit_surrogate(EmitArgs a) {
  const int64_t step = a.clk->step;
  int served = 0;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < a.nface; f += (int64_t)gridDim.x * blockDim.x) {
    const int v = a.owner_vox[f];
    const double T = v >= 0 ? a.Tvox[v] : a.T0;
    double J = 0.0, P = 0.0;
    if (a.F[f] > 0.0) {
      const double ap = approx_log10J(a.F[f] * 1e-9, T, a.phi_w);
      // elig 1: inside a validated bin.  2: inside the range, bin not validated -- used only
      // when the network and the classical estimate both put J below 1e-3 A/m^2, where no
      // face emits an SP (probability < 1e-13 per step on these grids).  3: field below the
      // trained range -- tunnelling is nil there and Richardson-Dushman with flat Schottky
      // lowering bounds the current from above (a curved barrier's top is higher), so a bound
      // below 1e-3 A/m^2 means J = P_N = 0 for the step.
      const int e = a.elig[f];
      bool use = e == 1;
      if (e == 2) {
        surrogate_out(a.Y, f, ap, &J, &P);
        use = ap <= -3.0 && J <= 1e-3;
      } else if (e == 3 && ap <= -3.0) {
        J = 0.0;
        P = 0.0;
        emit_finish(a, f, step, J, P);
        ++served;
        continue;
      }
      if (!use) {
        a.fb_list[atomicAdd(a.fb_n, 1)] = (int32_t)f;
        // why the integral runs: outside the trained range, or in a bin that failed validation
        atomicAdd((unsigned long long *)&a.clk->ctr[e == 0 ? cFbRange : cFbBin], 1ull);
        continue;
      }
      surrogate_out(a.Y, f, ap, &J, &P);
      ++served;
    }
    emit_finish(a, f, step, J, P);
  }
  for (int o = 16; o > 0; o >>= 1) served += __shfl_down_sync(0xffffffffu, served, o);
  if ((threadIdx.x & 31) == 0 && served) atomicAdd((unsigned long long *)&a.clk->ctr[cSurFaces], (unsigned long long)served);
}

// the full integral over the queued faces: one warp per face
template <bool kFast>
__global__ void k_emit_fallback(EmitArgs a) {
  const gtf::Tables tb = dev_tables();
  const int64_t step = a.clk->step;
  const int nq = *a.fb_n;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nq; q += warps) {
    const int64_t f = a.fb_list[q];
    const int v = a.owner_vox[f];
    const double T = v >= 0 ? a.Tvox[v] : a.T0;
    const double R = v >= 0 ? a.R_nm : -1.0;
    double J, P;
    int nev = 0;
    gtf::current_density_warp<kFast>(c_gtf, tb, a.F[f] * 1e-9, T, a.phi_w, R, &J, &P, &nev);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd((unsigned long long *)&a.clk->ctr[cWevals], (unsigned long long)nev);
      emit_finish(a, f, step, J, P);
    }
  }
}

// every face by the full integral: one warp per face
template <bool kFast>
__global__ void k_emit_count(EmitArgs a) {
  const gtf::Tables tb = dev_tables();
  const int64_t step = a.clk->step;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t f = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; f < a.nface; f += warps) {
    const int v = a.owner_vox[f];
    const double T = v >= 0 ? a.Tvox[v] : a.T0;
    const double R = v >= 0 ? a.R_nm : -1.0;
    double J, P;
    int nev = 0;
    gtf::current_density_warp<kFast>(c_gtf, tb, a.F[f] * 1e-9, T, a.phi_w, R, &J, &P, &nev);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd((unsigned long long *)&a.clk->ctr[cWevals], (unsigned long long)nev);
      emit_finish(a, f, step, J, P);
    }
  }
}

__global__ void k_check_face_new(DevClock *clk, const uint32_t *total, const uint32_t *total2, int s, int64_t cap,
                                 int *go) {
  const int64_t add = (int64_t)*total + (total2 ? (int64_t)*total2 : 0);
  const bool ok = clk->n[s] + add <= cap;
  *go = ok ? 1 : 0;
  if (!ok) atomicOr(&clk->err, kErrCapacity);
}

__global__ void k_commit_face_new(DevClock *clk, const uint32_t *total, const uint32_t *total2, int s, const int *go,
                                  int ctr, int ctr2) {
  if (!*go) return;
  const int64_t a = *total, b = total2 ? (int64_t)*total2 : 0;
  clk->n[s] += a + b;
  clk->next_id += a + b;
  clk->ctr[ctr] += a;
  if (total2) clk->ctr[ctr2] += b;
}

__global__ void k_emit_write(SpeciesBuf e, const int32_t *vcell, const int8_t *dir, int64_t nface, const uint32_t *cnt,
                             const uint32_t *off, int nx, int ny, uint64_t seed, const DevClock *clk, const int *go) {
  if (!*go) return;
  const int64_t step = clk->step, base = clk->n[PIC_ELECTRON], id0 = clk->next_id;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nface; f += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t N = cnt[f];
    if (!N) continue;
    const FaceGeom g = face_geom(vcell[f], dir[f], nx, ny);
    for (uint32_t j = 0; j < N; ++j) {
      const uint32_t d0 = 1 + 2 * j, d1 = 2 + 2 * j;
      const float ua = u01f(rng_block(seed, kEmit, (uint64_t)f, step, d0 >> 2).v[d0 & 3]);
      const float ub = u01f(rng_block(seed, kEmit, (uint64_t)f, step, d1 >> 2).v[d1 & 3]);
      float pos[3];
      face_point(g, ua, ub, pos);
      const int64_t s = base + off[f] + j;
      e.x[s] = pos[0]; e.y[s] = pos[1]; e.z[s] = pos[2];
      e.vx[s] = 0.f; e.vy[s] = 0.f; e.vz[s] = 0.f;
      e.w[s] = 1;
      e.id[s] = (uint64_t)(id0 + off[f] + j);
    }
  }
}

// ---- evaporation and sputter injection ---------------------------------------------------------
__device__ __forceinline__ uint32_t inj_weight(double n_cell, double N_inj, double w_min, int w_max) {
  const double r = (n_cell / kNmax) * (N_inj / w_min);
  const double w = ceil(fmax(1.0, sqrt(r)));
  return (uint32_t)fmin(w, (double)w_max);
}

struct InjArgs {
  const int32_t *vcell, *owner_vox;
  const int8_t *dir;
  int64_t nface;
  const double *Tvox;
  double T0, A, dt, w_min, V_cell;
  int w_max;
  const uint32_t *off_e, *off_n, *off_i, *off_j;   // off_j: null without Cu2+
  double *acc_evap, *acc_heat;
  long long *acc_sput;
  uint32_t *cnt, *wu, *cnt2, *wu2;
  int evap, sput;
};

__global__ void k_inject_count(InjArgs a) {
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < a.nface; f += (int64_t)gridDim.x * blockDim.x) {
    const int v = a.owner_vox[f];
    const double T = v >= 0 ? a.Tvox[v] : a.T0;
    const int32_t c = a.vcell[f];
    const double nsp = (double)((a.off_e[c + 1] - a.off_e[c]) + (a.off_n[c + 1] - a.off_n[c]) + (a.off_i[c + 1] - a.off_i[c]) +
                                (a.off_j ? a.off_j[c + 1] - a.off_j[c] : 0u));
    const double ncell = nsp / a.V_cell;
    uint32_t n1 = 0, w1 = 0, n2 = 0, w2 = 0;
    if (a.evap) {
      const double pre = kPatm / sqrt(2.0 * kPi * kMcu * kKb * T);
      const double flux = pre * exp(kEvap / (kKb / kQe) * (1.0 / kTboil - 1.0 / T));
      double acc = a.acc_evap[f] + flux * a.A * a.dt;
      a.acc_heat[f] -= kEvap * kQe * flux * a.A * a.dt;
      const double Ninj = floor(acc);
      if (Ninj >= 1.0) {
        w1 = inj_weight(ncell, Ninj, a.w_min, a.w_max);
        n1 = (uint32_t)floor(acc / (w1 * a.w_min));
        acc -= n1 * w1 * a.w_min;
      }
      a.acc_evap[f] = acc;
    }
    if (a.sput) {
      const long long s = a.acc_sput[f];
      const double lam = (double)s * 5.9604644775390625e-8;   // 2^-24
      const double Ninj = floor(lam);
      if (Ninj >= 1.0) {
        w2 = inj_weight(ncell, Ninj, a.w_min, a.w_max);
        n2 = (uint32_t)floor(lam / (w2 * a.w_min));
        a.acc_sput[f] = s - (long long)floor(n2 * w2 * a.w_min * 16777216.0);
      }
    }
    a.cnt[f] = n1; a.wu[f] = w1; a.cnt2[f] = n2; a.wu2[f] = w2;
  }
}

struct InjWrite {
  SpeciesBuf n;
  const int32_t *vcell, *owner_vox;
  const int8_t *dir;
  int64_t nface;
  const double *Tvox;
  double T0, w_min;
  const uint32_t *cnt, *off, *wu, *cnt2, *off2, *wu2, *total1;
  unsigned long long *acc_Es;
  int nx, ny;
  uint64_t seed;
  const DevClock *clk;
  const int *go;
};

__global__ void k_inject_write(InjWrite a) {
  if (!*a.go) return;
  const int64_t step = a.clk->step, base = a.clk->n[PIC_NEUTRAL], id0 = a.clk->next_id;
  const uint32_t n_evap = *a.total1;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < a.nface; f += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t N1 = a.cnt[f], N2 = a.cnt2[f];
    if (!N1 && !N2) continue;
    const FaceGeom g = face_geom(a.vcell[f], a.dir[f], a.nx, a.ny);
    const int v = a.owner_vox[f];
    const double T = v >= 0 ? a.Tvox[v] : a.T0;
    for (uint32_t j = 0; j < N1; ++j) {
      const U4 r0 = rng_block(a.seed, kEvapP, (uint64_t)f, step, 2 * j);
      const U4 r1 = rng_block(a.seed, kEvapP, (uint64_t)f, step, 2 * j + 1);
      float pos[3];
      face_point(g, u01f(r0.v[0]), u01f(r0.v[1]), pos);
      const double vn = sqrt(-2.0 * kKb * T / kMcu * log(u01d(r0.v[2])));
      const double sig = sqrt(kKb * T / kMcu);
      const double rr = sig * sqrt(-2.0 * log(u01d(r0.v[3])));
      const double ph = 2.0 * kPi * u01d(r1.v[0]);
      double vel[3];
      vel[g.axis] = g.sign * vn;
      vel[g.t0] = rr * cos(ph);
      vel[g.t1] = rr * sin(ph);
      const int64_t s = base + a.off[f] + j;
      a.n.x[s] = pos[0]; a.n.y[s] = pos[1]; a.n.z[s] = pos[2];
      a.n.vx[s] = (float)vel[0]; a.n.vy[s] = (float)vel[1]; a.n.vz[s] = (float)vel[2];
      a.n.w[s] = (int32_t)a.wu[f];
      a.n.id[s] = (uint64_t)(id0 + a.off[f] + j);
    }
    const double Us = 3.43, Ec = 100.0;
    const double Fc = (Ec / (Ec + Us)) * (Ec / (Ec + Us));
    for (uint32_t j = 0; j < N2; ++j) {
      const U4 r0 = rng_block(a.seed, kSput, (uint64_t)f, step, 2 * j);
      const U4 r1 = rng_block(a.seed, kSput, (uint64_t)f, step, 2 * j + 1);
      float pos[3];
      face_point(g, u01f(r0.v[0]), u01f(r0.v[1]), pos);
      const double sq = sqrt(u01d(r0.v[2]) * Fc);
      const double Es = Us * sq / (1.0 - sq);
      const double vv = sqrt(2.0 * Es * kQe / kMcu);
      const double ct = u01d(r0.v[3]);
      const double st = sqrt(fmax(0.0, 1.0 - ct * ct));
      const double ph = 2.0 * kPi * u01d(r1.v[0]);
      double vel[3];
      vel[g.axis] = g.sign * vv * ct;
      vel[g.t0] = vv * st * cos(ph);
      vel[g.t1] = vv * st * sin(ph);
      const int64_t s = base + n_evap + a.off2[f] + j;
      a.n.x[s] = pos[0]; a.n.y[s] = pos[1]; a.n.z[s] = pos[2];
      a.n.vx[s] = (float)vel[0]; a.n.vy[s] = (float)vel[1]; a.n.vz[s] = (float)vel[2];
      a.n.w[s] = (int32_t)a.wu2[f];
      a.n.id[s] = (uint64_t)(id0 + n_evap + a.off2[f] + j);
      atomicAdd(&a.acc_Es[f], (unsigned long long)(long long)floor(a.wu2[f] * a.w_min * Es * 1048576.0));
    }
  }
}

static int face_grid(pic_t *h) { return grid_for(h->faces.n, 128); }

int stage_face_field(pic_t *h) {
  ++h->nlaunch;
  { KtScope kt_(h, kidFaceField, (double)h->faces.n); k_face_field<<<grid_for(h->faces.n), kThreads, 0, h->stream>>>(h->faces.vcell, h->faces.dir, h->faces.n, h->phi, h->nx,
                                                                 h->ny, h->dx, h->faces.F); }
  return launch_check(h, "face_field");
}

int emission_tables_upload(pic_t *h) {
  double x16[16], w16[16], x32[32], w32[32];
  gtf::gauss_legendre(16, x16, w16);
  gtf::gauss_legendre(32, x32, w32);
  gtf::Consts C;
  C.Q = kQe / (16.0 * kPi * kEps0) * 1e9;
  C.g = 2.0 / sqrt(kHbar * kHbar / (2.0 * kMe) / kQe * 1e18);
  C.zS = kQe * kQe * kQe * kMe / (2.0 * kPi * kPi * kHbar * kHbar * kHbar);
  C.kB = kKb / kQe;
  C.Wlo = -7.0;
  PIC_CUDA(h, cudaMemcpyToSymbol(c_gl16x, x16, sizeof x16));
  PIC_CUDA(h, cudaMemcpyToSymbol(c_gl16w, w16, sizeof w16));
  PIC_CUDA(h, cudaMemcpyToSymbol(c_gl32x, x32, sizeof x32));
  PIC_CUDA(h, cudaMemcpyToSymbol(c_gl32w, w32, sizeof w32));
  double c32[32], s32[32];
  for (int i = 0; i < 32; ++i) {
    c32[i] = cos(0.5 * kPi * (x32[i] + 1.0));
    s32[i] = sin(0.5 * kPi * (x32[i] + 1.0));
  }
  PIC_CUDA(h, cudaMemcpyToSymbol(c_gl32c, c32, sizeof c32));
  PIC_CUDA(h, cudaMemcpyToSymbol(c_gl32s, s32, sizeof s32));
  float w32f[32], c32f[32], s32f[32];
  for (int i = 0; i < 32; ++i) {
    w32f[i] = (float)w32[i];
    c32f[i] = (float)c32[i];
    s32f[i] = (float)s32[i];
  }
  PIC_CUDA(h, cudaMemcpyToSymbol(c_gl32wf, w32f, sizeof w32f));
  PIC_CUDA(h, cudaMemcpyToSymbol(c_gl32cf, c32f, sizeof c32f));
  PIC_CUDA(h, cudaMemcpyToSymbol(c_gl32sf, s32f, sizeof s32f));
  PIC_CUDA(h, cudaMemcpyToSymbol(c_gtf, &C, sizeof C));
  return PIC_OK;
}

int emission_eval_dev(pic_t *h, const double *F, const double *T, const double *W, const double *R, double *J,
                      double *PN, int64_t n, bool fast) {
  ++h->nlaunch;
  const int64_t blocks = std::min<int64_t>((n + 3) / 4, (int64_t)h->nsm * 16);
  if (fast)
    k_emission_eval<true><<<(int)blocks, 128, 0, h->stream>>>(F, T, W, R, J, PN, n);
  else
    k_emission_eval<false><<<(int)blocks, 128, 0, h->stream>>>(F, T, W, R, J, PN, n);
  return launch_check(h, "emission_eval");
}

int stage_emit(pic_t *h) {
  Faces &fc = h->faces;
  const double A = h->dx * h->dx;
  int *go = h->long_n + 5;
  uint32_t *tot1 = (uint32_t *)(h->tmp_len + 4);
  PIC_TRY(stage_face_field(h));
  if (h->prm.flags & PIC_F_EMISSION) {
    EmitArgs a;
    a.vcell = fc.vcell; a.owner_vox = fc.owner_vox; a.dir = fc.dir; a.nface = fc.n;
    a.F = fc.F; a.Tvox = h->heat.T; a.T0 = h->prm.T0; a.phi_w = h->prm.work_function;
    a.R_nm = h->geo.tip_radius * 1e9; a.A = A; a.dt = h->prm.dt; a.w_min = h->prm.w_min;
    a.J = fc.J; a.PN = fc.PN; a.acc_heat = fc.acc_heat; a.acc_charge = fc.acc_charge; a.cnt = fc.cnt;
    a.seed = h->prm.seed; a.clk = h->clock;
    a.elig = nullptr; a.Y = nullptr;
    const bool fast = (h->prm.flags & PIC_F_FAST_INTEGRAL) != 0;
    a.fb_list = (int32_t *)fc.cnt2;          // scratch: the injection pass rewrites it afterwards
    a.fb_n = h->long_n + 8;
    if ((h->prm.flags & PIC_F_SURROGATE) && surrogate_ready(h)) {
      {
        KtScope kt_(h, kidMlpForward, (double)fc.n);
        PIC_TRY(surrogate_faces(h, &a.elig, &a.Y));
      }
      PIC_CUDA(h, cudaMemsetAsync(a.fb_n, 0, sizeof(int), h->stream));
      ++h->nlaunch;
      { KtScope kt_(h, kidEmitSurrogate, (double)fc.n); k_emit_surrogate<<<grid_for(fc.n), kThreads, 0, h->stream>>>(a); }
      ++h->nlaunch;
      // one warp per block: the queued faces (a few thousand, each a long FP64-bound chain) then
      // spread over the SMs one warp at a time rather than four
      if (fast)
        { KtScope kt_(h, kidEmitFallback, (double)fc.n); k_emit_fallback<true><<<h->nsm * 32, 32, 0, h->stream>>>(a); }
      else
        { KtScope kt_(h, kidEmitFallback, (double)fc.n); k_emit_fallback<false><<<h->nsm * 32, 32, 0, h->stream>>>(a); }
    } else {
      ++h->nlaunch;
      const int blocks = (int)std::min<int64_t>((fc.n + 3) / 4, (int64_t)h->nsm * 16);
      if (fast)
        { KtScope kt_(h, kidEmitCount, (double)fc.n); k_emit_count<true><<<blocks, 128, 0, h->stream>>>(a); }
      else
        { KtScope kt_(h, kidEmitCount, (double)fc.n); k_emit_count<false><<<blocks, 128, 0, h->stream>>>(a); }
    }
    PIC_TRY(scan_u32(h, fc.cnt, fc.off, fc.n, nullptr, tot1));
    ++h->nlaunch;
    k_check_face_new<<<1, 1, 0, h->stream>>>(h->clock, tot1, nullptr, PIC_ELECTRON, h->sp[PIC_ELECTRON].cap, go);
    ++h->nlaunch;
    { KtScope kt_(h, kidEmitWrite, (double)fc.n); k_emit_write<<<grid_for(fc.n), kThreads, 0, h->stream>>>(h->sp[PIC_ELECTRON].a, fc.vcell, fc.dir, fc.n, fc.cnt,
                                                             fc.off, h->nx, h->ny, h->prm.seed, h->clock, go); }
    ++h->nlaunch;
    k_commit_face_new<<<1, 1, 0, h->stream>>>(h->clock, tot1, nullptr, PIC_ELECTRON, go, cEmitted, cEmitted);
    PIC_TRY(launch_check(h, "emit"));
  }
  return stage_inject(h);
}

int stage_inject(pic_t *h) {
  const uint32_t fl = h->prm.flags;
  if (!(fl & (PIC_F_EVAP | PIC_F_SPUTTER))) return PIC_OK;
  Faces &fc = h->faces;
  int *go = h->long_n + 6;
  uint32_t *tot1 = (uint32_t *)(h->tmp_len + 6), *tot2 = (uint32_t *)(h->tmp_len + 7);
  InjArgs a;
  a.vcell = fc.vcell; a.owner_vox = fc.owner_vox; a.dir = fc.dir; a.nface = fc.n;
  a.Tvox = h->heat.T; a.T0 = h->prm.T0; a.A = h->dx * h->dx; a.dt = h->prm.dt; a.w_min = h->prm.w_min;
  a.V_cell = h->dx * h->dx * h->dx; a.w_max = h->prm.w_max_units;
  a.off_e = h->sp[PIC_ELECTRON].off; a.off_n = h->sp[PIC_NEUTRAL].off; a.off_i = h->sp[PIC_ION].off;
  a.off_j = nsp_active(h) > PIC_ION2 ? h->sp[PIC_ION2].off : nullptr;
  a.acc_evap = fc.acc_evap; a.acc_heat = fc.acc_heat; a.acc_sput = (long long *)fc.acc_sput;
  a.cnt = fc.cnt; a.wu = fc.wu; a.cnt2 = fc.cnt2; a.wu2 = fc.wu2;
  a.evap = (fl & PIC_F_EVAP) != 0; a.sput = (fl & PIC_F_SPUTTER) != 0;
  ++h->nlaunch;
  { KtScope kt_(h, kidInjectCount, (double)fc.n); k_inject_count<<<grid_for(fc.n), kThreads, 0, h->stream>>>(a); }
  PIC_TRY(scan_u32(h, fc.cnt, fc.off, fc.n, nullptr, tot1));
  PIC_TRY(scan_u32(h, fc.cnt2, fc.off2, fc.n, nullptr, tot2));
  ++h->nlaunch;
  k_check_face_new<<<1, 1, 0, h->stream>>>(h->clock, tot1, tot2, PIC_NEUTRAL, h->sp[PIC_NEUTRAL].cap, go);
  InjWrite w;
  w.n = h->sp[PIC_NEUTRAL].a; w.vcell = fc.vcell; w.owner_vox = fc.owner_vox; w.dir = fc.dir; w.nface = fc.n;
  w.Tvox = h->heat.T; w.T0 = h->prm.T0; w.w_min = h->prm.w_min;
  w.cnt = fc.cnt; w.off = fc.off; w.wu = fc.wu; w.cnt2 = fc.cnt2; w.off2 = fc.off2; w.wu2 = fc.wu2; w.total1 = tot1;
  w.acc_Es = (unsigned long long *)fc.acc_Es; w.nx = h->nx; w.ny = h->ny; w.seed = h->prm.seed; w.clk = h->clock;
  w.go = go;
  ++h->nlaunch;
  { KtScope kt_(h, kidInjectWrite, (double)fc.n); k_inject_write<<<grid_for(fc.n), kThreads, 0, h->stream>>>(w); }
  ++h->nlaunch;
  k_commit_face_new<<<1, 1, 0, h->stream>>>(h->clock, tot1, tot2, PIC_NEUTRAL, go, cEvaporated, cSputtered);
  return launch_check(h, "inject");
}

}  // namespace pic
