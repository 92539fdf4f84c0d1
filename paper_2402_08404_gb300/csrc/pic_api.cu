// C ABI of libpic (declared in include/pic.h): handle creation, geometry and face list, state
// I/O, stage sequencing of the coupled step (Sec. 2.3.1, Fig. newpic) and diagnostics.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <unordered_map>
#include <vector>

#include "pic_internal.cuh"

int pic_fail(pic_t *h, int code, const std::string &msg) {
  if (h) h->last_error = msg;
  return code;
}

namespace pic {

int emission_tables_upload(pic_t *h);
int mg_build_masks(pic_t *h);

void *dalloc(pic_t *h, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void *p = nullptr;
  if (h->alloc) {
    p = h->alloc(bytes, (void *)h->stream, h->alloc_user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
  }
  if (p) h->allocations.push_back({p, bytes});
  return p;
}

// give back one allocation made by dalloc (stream-ordered when the caller's allocator is)
void dfree(pic_t *h, void *p) {
  if (!p) return;
  for (size_t i = 0; i < h->allocations.size(); ++i)
    if (h->allocations[i].first == p) {
      if (h->free_fn) h->free_fn(p, h->allocations[i].second, (void *)h->stream, h->alloc_user);
      else cudaFree(p);
      h->allocations.erase(h->allocations.begin() + i);
      return;
    }
}

static void dfree_all(pic_t *h) {
  for (auto &a : h->allocations) {
    if (h->free_fn) h->free_fn(a.first, a.second, (void *)h->stream, h->alloc_user);
    else cudaFree(a.first);
  }
  h->allocations.clear();
}

int launch_check(pic_t *h, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return pic_fail(h, PIC_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return PIC_OK;
}

int check_device(pic_t *h) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return pic_fail(h, PIC_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev != h->device)
    return pic_fail(h, PIC_E_INVALID, "the current device (" + std::to_string(dev) + ") is not the handle's device (" +
                                          std::to_string(h->device) + "); make it current first");
  return PIC_OK;
}

// ---- host geometry (same rules as the statement in pic.h) -----------------------------------
struct HostGeom {
  std::vector<uint8_t> solid, cheb, dir0;
  std::vector<int32_t> fvcell, fowner, fowner_vox;
  std::vector<int8_t> fdir;
  std::vector<int64_t> fkey;
  std::vector<int32_t> vox_cell, vox_nbr;
  std::vector<uint8_t> vox_base;
  std::vector<int64_t> apex;
};

static void build_geometry(pic_t *h, HostGeom &G) {
  const int nx = h->nx, ny = h->ny, nz = h->nz;
  const double rc = h->geo.tip_radius / h->dx, hc = h->geo.tip_height / h->dx;
  const double ax = nx / 2.0, ay = ny / 2.0, zc = hc - rc;
  G.solid.assign(h->ncell, 0);
  int kmax = std::min(nz, (int)ceil(hc) + 1);
  for (int k = 0; k < kmax; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const double cx = i + 0.5, cy = j + 0.5, cz = k + 0.5;
        const double rho2 = (cx - ax) * (cx - ax) + (cy - ay) * (cy - ay);
        const bool shaft = rho2 <= rc * rc && cz <= zc;
        const bool cap = rho2 + (cz - zc) * (cz - zc) <= rc * rc;
        if (shaft || cap) G.solid[cell_index(i, j, k, nx, ny)] = 1;
      }
  // voxels (solid cells in linear order)
  std::unordered_map<int64_t, int32_t> vid;
  for (int64_t c = 0; c < h->ncell; ++c)
    if (G.solid[c]) {
      vid[c] = (int32_t)G.vox_cell.size();
      G.vox_cell.push_back((int32_t)c);
    }
  const int D[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
  for (size_t v = 0; v < G.vox_cell.size(); ++v) {
    const int64_t c = G.vox_cell[v];
    const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((int64_t)nx * ny));
    G.vox_base.push_back(k == 0);
    for (int d = 0; d < 6; ++d) {
      const int a = i + D[d][0], b = j + D[d][1], e = k + D[d][2];
      int32_t u = -1;
      if (a >= 0 && a < nx && b >= 0 && b < ny && e >= 0 && e < nz) {
        auto it = vid.find(cell_index(a, b, e, nx, ny));
        if (it != vid.end()) u = it->second;
      }
      G.vox_nbr.push_back(u);
    }
  }
  // exposed faces: vacuum cells in linear order, directions -x,+x,-y,+y,-z,+z
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const int64_t c = cell_index(i, j, k, nx, ny);
        if (G.solid[c]) continue;
        for (int d = 0; d < 6; ++d) {
          const int a = i + D[d][0], b = j + D[d][1], e = k + D[d][2];
          int64_t own = -2;
          if (d == 4 && k == 0) own = -1;
          else if (a >= 0 && a < nx && b >= 0 && b < ny && e >= 0 && e < nz && G.solid[cell_index(a, b, e, nx, ny)])
            own = cell_index(a, b, e, nx, ny);
          if (own == -2) continue;
          G.fvcell.push_back((int32_t)c);
          G.fdir.push_back((int8_t)d);
          G.fowner.push_back((int32_t)own);
          G.fowner_vox.push_back(own >= 0 ? vid[own] : -1);
          G.fkey.push_back(c * 6 + d);
        }
      }
  // apex faces: +z tip faces of the highest owner cells touching the axis
  const int ai = (int)floor(ax), aj = (int)floor(ay);
  int top = -1;
  for (size_t f = 0; f < G.fvcell.size(); ++f) {
    if (G.fdir[f] != 4 || G.fowner[f] < 0) continue;
    const int64_t o = G.fowner[f];
    const int oi = (int)(o % nx), oj = (int)((o / nx) % ny), ok = (int)(o / ((int64_t)nx * ny));
    if ((oi == ai - 1 || oi == ai) && (oj == aj - 1 || oj == aj)) top = std::max(top, ok);
  }
  for (size_t f = 0; f < G.fvcell.size(); ++f) {
    if (G.fdir[f] != 4 || G.fowner[f] < 0) continue;
    const int64_t o = G.fowner[f];
    const int oi = (int)(o % nx), oj = (int)((o / nx) % ny), ok = (int)(o / ((int64_t)nx * ny));
    if ((oi == ai - 1 || oi == ai) && (oj == aj - 1 || oj == aj) && ok == top) G.apex.push_back((int64_t)f);
  }
  // Dirichlet nodes: z = 0, z = nz, corners of solid cells
  G.dir0.assign(h->nnode, 0);
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i <= nx; ++i) {
      G.dir0[node_index(i, j, 0, nx, ny)] = 1;
      G.dir0[node_index(i, j, nz, nx, ny)] = 1;
    }
  for (int32_t c : G.vox_cell) {
    const int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
    for (int dk = 0; dk < 2; ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) G.dir0[node_index(i + di, j + dj, k + dk, nx, ny)] = 1;
  }
  // Chebyshev distance to the nearest solid cell, capped at 8, by dilation inside the tip box
  const int cap = 8;
  G.cheb.assign(h->ncell, 255);
  if (!G.vox_cell.empty()) {
    int lo[3] = {nx, ny, nz}, hi[3] = {-1, -1, -1};
    for (int32_t c : G.vox_cell) {
      const int q[3] = {c % nx, (c / nx) % ny, c / (nx * ny)};
      for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], q[a]); hi[a] = std::max(hi[a], q[a]); }
    }
    const int n3[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a) { lo[a] = std::max(0, lo[a] - cap); hi[a] = std::min(n3[a] - 1, hi[a] + cap); }
    for (int32_t c : G.vox_cell) G.cheb[c] = 0;
    for (int r = 1; r <= cap; ++r)
      for (int k = lo[2]; k <= hi[2]; ++k)
        for (int j = lo[1]; j <= hi[1]; ++j)
          for (int i = lo[0]; i <= hi[0]; ++i) {
            const int64_t c = cell_index(i, j, k, nx, ny);
            if (G.cheb[c] != 255) continue;
            bool hit = false;
            for (int dk = -1; dk <= 1 && !hit; ++dk)
              for (int dj = -1; dj <= 1 && !hit; ++dj)
                for (int di = -1; di <= 1 && !hit; ++di) {
                  const int a = i + di, b = j + dj, e = k + dk;
                  if (a < 0 || a >= nx || b < 0 || b >= ny || e < 0 || e >= nz) continue;
                  if (G.cheb[cell_index(a, b, e, nx, ny)] == r - 1) hit = true;
                }
            if (hit) G.cheb[c] = (uint8_t)r;
          }
    // cells of the box left at 255 are farther than cap: keep 255 (> any cap test)
  }
}

template <typename T>
static T *alloc_n(pic_t *h, int64_t n) {
  return (T *)dalloc(h, (size_t)std::max<int64_t>(n, 1) * sizeof(T));
}

}  // namespace pic

// ---- kernel timing ----------------------------------------------------------------------------
namespace pic {
const char *const kKernelNames[kidNum] = {
    "k_push", "k_keys", "k_scatter", "k_fix_short", "k_fix_mid", "k_fix_long", "k_gather", "k_scan_partial",
    "k_scan_apply", "k_deposit", "k_mcc_count", "k_mcc_products", "k_elastic", "k_coulomb", "k_merge", "k_dfi_count", "k_dfi_products", "k_dirichlet",
    "k_residual64", "k_norm_sum", "k_smooth", "k_smooth_first", "k_residual", "k_restrict", "k_prolong", "k_coarse", "k_vcycle_tail", "k_ramo",
    "k_correct", "k_efield", "k_face_field", "k_emit_surrogate", "k_emit_fallback", "k_emit_count", "k_emit_write",
    "k_inject_count", "k_inject_write", "k_mlp_forward", "k_heat", "k_cross"};

KtScope::KtScope(pic_t *h_, int kid_, double units_) : h(h_), kid(kid_), units(units_) {
  on = h && (h->kt_mask >> kid & 1ull);
  if (!on) return;
  const size_t i = h->kt_pend.size();
  while (h->kt_ev.size() < 2 * (i + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) { on = false; return; }
    h->kt_ev.push_back(e);
  }
  cudaEventRecord(h->kt_ev[2 * i], h->stream);
}

KtScope::~KtScope() {
  if (!on) return;
  const size_t i = h->kt_pend.size();
  cudaEventRecord(h->kt_ev[2 * i + 1], h->stream);
  h->kt_pend.emplace_back(kid, units);
}

void kt_collect(pic_t *h) {
  for (size_t i = 0; i < h->kt_pend.size(); ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, h->kt_ev[2 * i], h->kt_ev[2 * i + 1]) != cudaSuccess) continue;
    const int k = h->kt_pend[i].first;
    h->kt_ms[k] += t;
    h->kt_units[k] += h->kt_pend[i].second;
    h->kt_n[k] += 1;
  }
  h->kt_pend.clear();
}
}  // namespace pic

using namespace pic;

static void graph_free(pic_t *h);

extern "C" {

const char *pic_last_error(pic_t *h) { return h ? h->last_error.c_str() : "null handle"; }

void pic_destroy(pic_t *h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  for (cudaEvent_t e : h->kt_ev) cudaEventDestroy(e);
  for (cudaEvent_t e : h->step_ev) cudaEventDestroy(e);
  graph_free(h);
  if (h->body_stream) cudaStreamDestroy(h->body_stream);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->copy_stream) {
    cudaStreamSynchronize(h->copy_stream);
    cudaStreamDestroy(h->copy_stream);
  }
  for (cudaEvent_t e : h->copy_ev)
    if (e) cudaEventDestroy(e);
  mlp_forget(h);
  dfree_all(h);
  delete h;
}

static int clock_sync(pic_t *h, DevClock *out) {
  PIC_CUDA(h, cudaMemcpyAsync(out, h->clock, sizeof(DevClock), cudaMemcpyDeviceToHost, h->stream));
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

static int check_err(pic_t *h) {
  DevClock c;
  PIC_TRY(clock_sync(h, &c));
  if (c.err) {
    const int e = c.err;
    int zero = 0;
    PIC_CUDA(h, cudaMemcpyAsync(&h->clock->err, &zero, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    PIC_CUDA(h, cudaStreamSynchronize(h->stream));
    if (e & kErrCapacity) return pic_fail(h, PIC_E_CAPACITY, "SP capacity exceeded: new SPs were not added");
    if (e & kErrSegment) return pic_fail(h, PIC_E_CAPACITY, "more SPs of one species in one cell than the sort handles");
    if (e & kErrNoconv) return pic_fail(h, PIC_E_NOCONV, "Poisson solve did not reach mg_tol within mg_max_cycles");
    return pic_fail(h, PIC_E_INVALID, "device error flag " + std::to_string(e));
  }
  return PIC_OK;
}

// phi *= s in fixed point (rounded to the nearest 2^-40 V)
__global__ void k_scale(long long *phi, int64_t n, double s) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    phi[i] = __double2ll_rn((double)phi[i] * s);
}

__global__ void k_phi_from_double(const double *src, long long *phi, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    phi[i] = __double2ll_rn(src[i] * kPhiScale);
}

__global__ void k_phi_to_double(const long long *phi, double *dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (double)phi[i] * kPhiUnit;
}

int pic_create(const pic_geometry_t *geometry, const pic_grid_t *grid, const pic_species_t *species, int nspecies,
               const pic_params_t *params, pic_alloc_fn alloc, pic_free_fn free_fn, void *alloc_user, void *stream,
               pic_t **out) {
  if (!geometry || !grid || !species || !params || !out || (nspecies != 3 && nspecies != PIC_NSPECIES))
    return PIC_E_INVALID;
  *out = nullptr;
  if (grid->nx < 8 || grid->ny < 8 || grid->nz < 8 || (grid->nx & 1) || (grid->ny & 1) || (grid->nz & 1) || !(grid->dx > 0))
    return PIC_E_INVALID;
  if ((int64_t)grid->nx * grid->ny * grid->nz >= (int64_t)0xFFFFFFF0u) return PIC_E_INVALID;
  // node arrays and the split-colour levels ((nx + 2) slots per row pair) are indexed in 32 bits
  if ((int64_t)(grid->nx + 2) * (grid->ny + 1) * (grid->nz + 1) >= (int64_t)0xFFFFFFFFu) return PIC_E_INVALID;
  if (!(params->dt > 0) || !(params->w_min > 0) || params->w_max_units < 1) return PIC_E_INVALID;
  // three species given: Cu2+ takes Cu+'s mass, charge 2 and room for one SP
  pic_species_t spc[PIC_NSPECIES];
  for (int s = 0; s < nspecies; ++s) spc[s] = species[s];
  if (nspecies == 3) { spc[PIC_ION2] = species[PIC_ION]; spc[PIC_ION2].charge_e = 2; spc[PIC_ION2].capacity = 1; }
  for (int s = 0; s < PIC_NSPECIES; ++s)
    if (spc[s].capacity < 1 || spc[s].capacity > 0x7FFFFFFF || !(spc[s].mass > 0)) return PIC_E_INVALID;
  pic_t *h = new pic_t();
  h->nx = grid->nx; h->ny = grid->ny; h->nz = grid->nz; h->dx = grid->dx;
  h->ncell = (int64_t)h->nx * h->ny * h->nz;
  h->nnode = (int64_t)(h->nx + 1) * (h->ny + 1) * (h->nz + 1);
  h->geo = *geometry; h->prm = *params;
  if (h->prm.mg_tol <= 0) h->prm.mg_tol = 1e-8;
  if (h->prm.mg_max_cycles <= 0) h->prm.mg_max_cycles = 50;
  // 3 + 3 sweeps: on the staircased tip a V-cycle contracts the error by ~0.4 with 2 + 2 and ~0.3
  // with 3 + 3, which reaches a 1e-6 step tolerance in one refinement cycle instead of two
  h->mg_sweeps = h->prm.mg_sweeps > 0 ? std::min(h->prm.mg_sweeps, 8) : 3;
  // constant stand-ins: e-Cu 1e-19 m^2, Cu-Cu hard spheres of radius 128 pm, Cu+-Cu 5e-19 m^2
  h->sigma_el_en = h->prm.sigma_el_en > 0 ? h->prm.sigma_el_en : 1.0e-19;
  h->sigma_el_nn = h->prm.sigma_el_nn > 0 ? h->prm.sigma_el_nn : kPi * ((2 * 128e-12) * (2 * 128e-12));
  h->sigma_cx = h->prm.sigma_cx > 0 ? h->prm.sigma_cx : 5.0e-19;
  h->stream = (cudaStream_t)stream;
  h->alloc = alloc; h->free_fn = free_fn; h->alloc_user = alloc_user;
  int dev = 0;
  cudaGetDevice(&dev);
  h->device = dev;
  cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (h->nsm <= 0) h->nsm = 148;
  auto fail = [&](int code, const std::string &m) {
    std::string msg = m;
    pic_destroy(h);
    (void)msg;
    return code;
  };
  HostGeom G;
  build_geometry(h, G);
  bool okalloc = true;
  auto A = [&](void *p) { if (!p) okalloc = false; };
  // grids
  h->solid = alloc_n<uint8_t>(h, h->ncell); A(h->solid);
  h->cheb = alloc_n<uint8_t>(h, h->ncell); A(h->cheb);
  h->phi = alloc_n<long long>(h, h->nnode); A(h->phi);
  h->E = alloc_n<float4>(h, h->nnode); A(h->E);
  h->Q = alloc_n<unsigned long long>(h, h->nnode); A(h->Q);
  // multigrid hierarchy
  {
    int lx = h->nx, ly = h->ny, lz = h->nz;
    double hh = h->dx;
    for (;;) {
      MgLevel L;
      L.nx = lx; L.ny = ly; L.nz = lz; L.h = hh;
      L.nnode = (int64_t)(lx + 1) * (ly + 1) * (lz + 1);
      L.Xh = (lx + 2) / 2;
      L.nper = (int64_t)(lz + 1) * (ly + 1) * L.Xh;
      const int64_t ns = 2 * L.nper;
      L.dir = alloc_n<uint8_t>(h, L.nnode); A(L.dir);
      L.dirs = alloc_n<uint8_t>(h, ns); A(L.dirs);
      L.u = alloc_n<float>(h, ns); A(L.u);
      L.f = alloc_n<float>(h, ns); A(L.f);
      L.r = alloc_n<float>(h, ns); A(L.r);
      L.ud = alloc_n<double>(h, ns); A(L.ud);
      L.fd = alloc_n<double>(h, ns); A(L.fd);
      L.rd = alloc_n<double>(h, ns); A(L.rd);
      h->mg.push_back(L);
      if ((lx & 1) || (ly & 1) || (lz & 1) || std::min(lx, std::min(ly, lz)) < 8) break;
      lx /= 2; ly /= 2; lz /= 2; hh *= 2.0;
    }
  }
  // species
  int64_t capsum = 0;
  for (int s = 0; s < PIC_NSPECIES; ++s) {
    Species &S = h->sp[s];
    S.Z = spc[s].charge_e;
    S.mass = spc[s].mass;
    S.cap = spc[s].capacity;
    S.qmdt = (float)((double)S.Z * kQe / S.mass * h->prm.dt);
    for (SpeciesBuf *B : {&S.a, &S.b}) {
      B->x = alloc_n<float>(h, S.cap); A(B->x);
      B->y = alloc_n<float>(h, S.cap); A(B->y);
      B->z = alloc_n<float>(h, S.cap); A(B->z);
      B->vx = alloc_n<float>(h, S.cap); A(B->vx);
      B->vy = alloc_n<float>(h, S.cap); A(B->vy);
      B->vz = alloc_n<float>(h, S.cap); A(B->vz);
      B->w = alloc_n<int32_t>(h, S.cap); A(B->w);
      B->id = alloc_n<uint64_t>(h, S.cap); A(B->id);
    }
    S.key = alloc_n<uint32_t>(h, S.cap); A(S.key);
    S.perm = alloc_n<uint32_t>(h, S.cap); A(S.perm);
    S.skey = alloc_n<uint32_t>(h, S.cap); A(S.skey);
    S.cnt = alloc_n<uint32_t>(h, h->ncell + 1); A(S.cnt);
    S.off = alloc_n<uint32_t>(h, h->ncell + 1); A(S.off);
  }
  // one staging slot per collision work item: impact ionization takes e- + Cu, the ionization of
  // Cu+ e- + Cu+, field ionization Cu, the elastic passes e-, Cu or Cu+ alone
  capsum = std::max(h->sp[PIC_ELECTRON].cap + h->sp[PIC_NEUTRAL].cap, h->sp[PIC_ELECTRON].cap + h->sp[PIC_ION].cap);
  h->pair_cnt = alloc_n<uint64_t>(h, capsum); A(h->pair_cnt);
  h->ev_hits = alloc_n<int>(h, capsum / 256 + 2); A(h->ev_hits);
  h->ev_cnt = alloc_n<uint64_t>(h, capsum / 256 + 2); A(h->ev_cnt);
  h->ev_off = alloc_n<uint64_t>(h, capsum / 256 + 2); A(h->ev_off);
  h->ev_cnt2 = alloc_n<uint64_t>(h, capsum / 256 + 2); A(h->ev_cnt2);
  h->ev_off2 = alloc_n<uint64_t>(h, capsum / 256 + 2); A(h->ev_off2);
  // faces
  Faces &fc = h->faces;
  fc.n = (int64_t)G.fvcell.size();
  fc.vcell = alloc_n<int32_t>(h, fc.n); A(fc.vcell);
  fc.dir = alloc_n<int8_t>(h, fc.n); A(fc.dir);
  fc.owner = alloc_n<int32_t>(h, fc.n); A(fc.owner);
  fc.owner_vox = alloc_n<int32_t>(h, fc.n); A(fc.owner_vox);
  fc.key = alloc_n<int64_t>(h, fc.n); A(fc.key);
  for (double **p : {&fc.F, &fc.J, &fc.PN, &fc.acc_evap, &fc.acc_heat, &fc.acc_charge}) { *p = alloc_n<double>(h, fc.n); A(*p); }
  for (int64_t **p : {&fc.acc_sput, &fc.acc_Eb, &fc.acc_Es}) { *p = alloc_n<int64_t>(h, fc.n); A(*p); }
  for (uint32_t **p : {&fc.cnt, &fc.off, &fc.cnt2, &fc.off2, &fc.wu, &fc.wu2}) { *p = alloc_n<uint32_t>(h, fc.n + 1); A(*p); }
  // heat
  Heat &H = h->heat;
  H.nvox = (int64_t)G.vox_cell.size();
  h->solid_count = H.nvox;
  H.cell = alloc_n<int32_t>(h, H.nvox); A(H.cell);
  H.nbr = alloc_n<int32_t>(h, 6 * H.nvox); A(H.nbr);
  H.base = alloc_n<uint8_t>(h, H.nvox); A(H.base);
  for (double **p : {&H.T, &H.Tn, &H.sig, &H.kap, &H.src, &H.cur, &H.phiJ, &H.joule, &H.p, &H.q, &H.res, &H.zv}) {
    *p = alloc_n<double>(h, H.nvox);
    A(*p);
  }
  // scratch
  h->scan_tmp = dalloc(h, (size_t)4 * h->nsm * sizeof(uint64_t)); A(h->scan_tmp);   // one partial per scan block
  // residual-norm partials: one pair per block of the 3D node grid (32 x 8 x 1 blocks)
  h->red = alloc_n<double>(h, (int64_t)2 * ((h->nx + 1 + 31) / 32) * ((h->ny + 1 + 7) / 8) * (h->nz + 1)); A(h->red);
  h->red_out = alloc_n<double>(h, 2); A(h->red_out);
  h->red_mid = alloc_n<double>(h, 2 * 128); A(h->red_mid);
  h->ramo_part = alloc_n<double>(h, kRamoBlocks); A(h->ramo_part);
  if (h->prm.circuit_R > 0 && h->prm.circuit_C > 0) { h->E0 = alloc_n<float4>(h, h->nnode); A(h->E0); }
  h->tmp_len = alloc_n<int64_t>(h, 24); A(h->tmp_len);
  h->long_list = alloc_n<int2>(h, kLongCap); A(h->long_list);
  {
    int64_t mc = 0;
    for (int s = 0; s < PIC_NSPECIES; ++s) mc = std::max<int64_t>(mc, h->sp[s].cap);
    h->mid_cap = std::min<int64_t>(mc / 5 + 1024, INT32_MAX);   // a queued segment holds >= 5 SPs
    h->mid_list = alloc_n<int2>(h, h->mid_cap); A(h->mid_list);
  }
  h->long_n = alloc_n<int>(h, 16); A(h->long_n);
  h->xq_n = alloc_n<int>(h, 4); A(h->xq_n);
  h->clock = alloc_n<DevClock>(h, 1); A(h->clock);
  if (!okalloc) return fail(PIC_E_CUDA, "device allocation failed");
  // uploads
  cudaStream_t st = h->stream;
  int rc = PIC_OK;
#define UP(dst, src, bytes) \
  if (rc == PIC_OK && cudaMemcpyAsync((dst), (src), (bytes), cudaMemcpyHostToDevice, st) != cudaSuccess) rc = PIC_E_CUDA
  UP(h->solid, G.solid.data(), h->ncell);
  UP(h->cheb, G.cheb.data(), h->ncell);
  UP(h->mg[0].dir, G.dir0.data(), h->nnode);
  if (fc.n) {
    UP(fc.vcell, G.fvcell.data(), fc.n * 4);
    UP(fc.dir, G.fdir.data(), fc.n);
    UP(fc.owner, G.fowner.data(), fc.n * 4);
    UP(fc.owner_vox, G.fowner_vox.data(), fc.n * 4);
    UP(fc.key, G.fkey.data(), fc.n * 8);
  }
  if (H.nvox) {
    UP(H.cell, G.vox_cell.data(), H.nvox * 4);
    UP(H.nbr, G.vox_nbr.data(), H.nvox * 24);
    UP(H.base, G.vox_base.data(), H.nvox);
    std::vector<double> T0(H.nvox, h->prm.T0);
    UP(H.T, T0.data(), H.nvox * 8);
    if (rc == PIC_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = PIC_E_CUDA;
  }
#undef UP
  if (rc != PIC_OK) return fail(rc, "upload failed");
  for (int s = 0; s < PIC_NSPECIES; ++s)
    for (uint32_t *p : {h->sp[s].cnt, h->sp[s].off})
      if (cudaMemsetAsync(p, 0, (h->ncell + 1) * 4, st) != cudaSuccess) rc = PIC_E_CUDA;
  for (double *p : {fc.acc_evap, fc.acc_heat, fc.acc_charge, fc.F, fc.J, fc.PN})
    if (cudaMemsetAsync(p, 0, std::max<int64_t>(fc.n, 1) * 8, st) != cudaSuccess) rc = PIC_E_CUDA;
  for (int64_t *p : {fc.acc_sput, fc.acc_Eb, fc.acc_Es})
    if (cudaMemsetAsync(p, 0, std::max<int64_t>(fc.n, 1) * 8, st) != cudaSuccess) rc = PIC_E_CUDA;
  if (cudaMemsetAsync(h->clock, 0, sizeof(DevClock), st) != cudaSuccess) rc = PIC_E_CUDA;
  if (cudaMemsetAsync(h->phi, 0, h->nnode * 8, st) != cudaSuccess) rc = PIC_E_CUDA;
  if (cudaMemsetAsync(h->Q, 0, h->nnode * 8, st) != cudaSuccess) rc = PIC_E_CUDA;
  // level corrections: Dirichlet slots stay 0 for good (the sweeps never write them)
  for (MgLevel &L : h->mg) {
    const size_t ns = (size_t)2 * L.nper;
    for (void *p : {(void *)L.u, (void *)L.f, (void *)L.r})
      if (cudaMemsetAsync(p, 0, ns * sizeof(float), st) != cudaSuccess) rc = PIC_E_CUDA;
    for (void *p : {(void *)L.ud, (void *)L.fd, (void *)L.rd})
      if (cudaMemsetAsync(p, 0, ns * sizeof(double), st) != cudaSuccess) rc = PIC_E_CUDA;
  }
  if (rc != PIC_OK) return fail(rc, "memset failed");
  if (mg_build_masks(h) != PIC_OK || mg_coarse_setup(h) != PIC_OK || emission_tables_upload(h) != PIC_OK)
    return fail(PIC_E_CUDA, "setup failed");
  // V0: calibrate from the apex field by a Laplace solve at a reference V_ref (phi is linear in
  // V0).  V_ref = 1024 V (a power of two, so the rescaling is exact up to the fixed-point
  // rounding) keeps the 2^-40 V steps of phi ~1e-15 of the solution.
  constexpr double kVref = 1024.0;
  if (h->prm.V0 >= kPhiMax) {
    pic_destroy(h);
    return PIC_E_INVALID;   // the fixed-point potential holds |phi| < 8192 V
  }
  if (h->prm.V0 > 0) {
    h->V0 = h->prm.V0;
    rc = stage_solve(h, true, h->V0);
    if (rc == PIC_OK && h->E0) rc = circuit_setup(h, h->V0);
  } else {
    rc = stage_solve(h, true, kVref);
    if (rc == PIC_OK && h->E0) rc = circuit_setup(h, kVref);
    if (rc == PIC_OK) rc = stage_face_field(h);
    double F1 = 0.0;
    if (rc == PIC_OK && !G.apex.empty()) {
      std::vector<double> F(fc.n);
      if (cudaMemcpyAsync(F.data(), fc.F, fc.n * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        rc = PIC_E_CUDA;
      for (int64_t f : G.apex) F1 += F[f];
      F1 /= (double)G.apex.size();
    }
    if (rc == PIC_OK) {
      h->V0 = (F1 > 0 && h->prm.apex_field > 0) ? h->prm.apex_field / F1 * kVref : kVref;
      if (!(h->V0 < kPhiMax)) rc = pic_fail(h, PIC_E_INVALID, "calibrated V0 is not below 8192 V");
    }
    if (rc == PIC_OK) {
      k_scale<<<grid_for(h->nnode), kThreads, 0, st>>>(h->phi, h->nnode, h->V0 / kVref);
      h->dirichlet_valid = false;
      rc = stage_efield(h);
    }
  }
  if (rc == PIC_OK && h->E0) rc = circuit_reset(h);
  if (rc != PIC_OK) {
    std::string m = h->last_error;
    pic_destroy(h);
    return rc;
  }
  *out = h;
  return PIC_OK;
}

int pic_set_clock(pic_t *h, int64_t step, int64_t next_id) {
  if (!h) return PIC_E_INVALID;
  int64_t v[2] = {step, next_id};
  PIC_CUDA(h, cudaMemcpyAsync(h->clock, v, sizeof v, cudaMemcpyHostToDevice, h->stream));
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  return PIC_OK;
}


int pic_load_particles(pic_t *h, int s, const float *x, const float *y, const float *z, const float *vx, const float *vy,
                       const float *vz, const int32_t *w, const uint64_t *id, int64_t n) {
  if (!h || s < 0 || s >= PIC_NSPECIES || n < 0) return PIC_E_INVALID;
  Species &S = h->sp[s];
  if (n > S.cap) return pic_fail(h, PIC_E_CAPACITY, "load exceeds the species capacity");
  if (n > 0 && (!x || !y || !z || !vx || !vy || !vz || !w || !id)) return PIC_E_INVALID;
  // the new SPs go to the scratch buffer first and replace the current ones only once the device
  // has checked that every one lies inside the domain and outside the tip
  cudaStream_t st = h->stream;
  if (n) {
    PIC_CUDA(h, cudaMemcpyAsync(S.b.x, x, n * 4, cudaMemcpyHostToDevice, st));
    PIC_CUDA(h, cudaMemcpyAsync(S.b.y, y, n * 4, cudaMemcpyHostToDevice, st));
    PIC_CUDA(h, cudaMemcpyAsync(S.b.z, z, n * 4, cudaMemcpyHostToDevice, st));
    PIC_CUDA(h, cudaMemcpyAsync(S.b.vx, vx, n * 4, cudaMemcpyHostToDevice, st));
    PIC_CUDA(h, cudaMemcpyAsync(S.b.vy, vy, n * 4, cudaMemcpyHostToDevice, st));
    PIC_CUDA(h, cudaMemcpyAsync(S.b.vz, vz, n * 4, cudaMemcpyHostToDevice, st));
    PIC_CUDA(h, cudaMemcpyAsync(S.b.w, w, n * 4, cudaMemcpyHostToDevice, st));
    PIC_CUDA(h, cudaMemcpyAsync(S.b.id, id, n * 8, cudaMemcpyHostToDevice, st));
    PIC_TRY(validate_loaded(h, S.b, n));
  }
  std::swap(S.a, S.b);
  PIC_CUDA(h, cudaMemcpyAsync(&h->clock->n[s], &n, 8, cudaMemcpyHostToDevice, st));
  PIC_CUDA(h, cudaStreamSynchronize(st));
  PIC_TRY(stage_keys(h, s));   // clears the counts a push may have left, then counts the new SPs
  PIC_TRY(sort_species(h, s));
  return check_err(h);
}

// Every species in one call: the copies of species s + 1 run on a second stream while species
// s is checked and sorted on the library stream.  A species is swapped in only after its own
// check has passed (the host waits for that check alone), so a failure leaves the species
// before it loaded and the rest unchanged, as the same sequence of pic_load_particles calls would.
int pic_load_all(pic_t *h, const pic_host_species_t *sp, int nspecies) {
  if (!h || !sp || nspecies < 1 || nspecies > PIC_NSPECIES) return PIC_E_INVALID;
  PIC_TRY(check_device(h));
  if (h->capturing) return pic_fail(h, PIC_E_INVALID, "pic_load_all during graph capture");
  for (int s = 0; s < nspecies; ++s) {
    const pic_host_species_t &a = sp[s];
    if (a.n < 0) return PIC_E_INVALID;
    if (a.n > h->sp[s].cap) return pic_fail(h, PIC_E_CAPACITY, "load exceeds the species capacity");
    if (a.n > 0 && (!a.x || !a.y || !a.z || !a.vx || !a.vy || !a.vz || !a.w || !a.id)) return PIC_E_INVALID;
  }
  if (!h->copy_stream) PIC_CUDA(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
  for (cudaEvent_t &e : h->copy_ev)
    if (!e) PIC_CUDA(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaStream_t cs = h->copy_stream, st = h->stream;
  // the copies overwrite the scratch buffers: after all work queued so far
  PIC_CUDA(h, cudaEventRecord(h->copy_ev[PIC_NSPECIES], st));
  PIC_CUDA(h, cudaStreamWaitEvent(cs, h->copy_ev[PIC_NSPECIES], 0));
  auto issue = [&](int s) -> int {
    const pic_host_species_t &a = sp[s];
    const SpeciesBuf &B = h->sp[s].b;
    const int64_t n = a.n;
    if (n) {
      PIC_CUDA(h, cudaMemcpyAsync(B.x, a.x, n * 4, cudaMemcpyHostToDevice, cs));
      PIC_CUDA(h, cudaMemcpyAsync(B.y, a.y, n * 4, cudaMemcpyHostToDevice, cs));
      PIC_CUDA(h, cudaMemcpyAsync(B.z, a.z, n * 4, cudaMemcpyHostToDevice, cs));
      PIC_CUDA(h, cudaMemcpyAsync(B.vx, a.vx, n * 4, cudaMemcpyHostToDevice, cs));
      PIC_CUDA(h, cudaMemcpyAsync(B.vy, a.vy, n * 4, cudaMemcpyHostToDevice, cs));
      PIC_CUDA(h, cudaMemcpyAsync(B.vz, a.vz, n * 4, cudaMemcpyHostToDevice, cs));
      PIC_CUDA(h, cudaMemcpyAsync(B.w, a.w, n * 4, cudaMemcpyHostToDevice, cs));
      PIC_CUDA(h, cudaMemcpyAsync(B.id, a.id, n * 8, cudaMemcpyHostToDevice, cs));
    }
    PIC_CUDA(h, cudaEventRecord(h->copy_ev[s], cs));
    return PIC_OK;
  };
  int rc = issue(0);
  for (int s = 0; s < nspecies && rc == PIC_OK; ++s) {
    if (s + 1 < nspecies) rc = issue(s + 1);
    if (rc != PIC_OK) break;
    Species &S = h->sp[s];
    const int64_t n = sp[s].n;
    if (cudaStreamWaitEvent(st, h->copy_ev[s], 0) != cudaSuccess) { rc = pic_fail(h, PIC_E_CUDA, "wait copy"); break; }
    if (n) {
      rc = validate_loaded(h, S.b, n);   // waits for this species' check only
      if (rc != PIC_OK) break;
    }
    std::swap(S.a, S.b);
    if (cudaMemcpyAsync(&h->clock->n[s], &sp[s].n, 8, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      rc = pic_fail(h, PIC_E_CUDA, "count upload");
      break;
    }
    rc = stage_keys(h, s);
    if (rc == PIC_OK) rc = sort_species(h, s);
  }
  cudaStreamSynchronize(cs);   // no copy outlives the call (the host arrays may go away)
  if (rc != PIC_OK) return rc;
  PIC_CUDA(h, cudaStreamSynchronize(st));
  return check_err(h);
}

int pic_get_particles(pic_t *h, int s, float *x, float *y, float *z, float *vx, float *vy, float *vz, int32_t *w,
                      uint64_t *id, int64_t cap, int64_t *n_out) {
  if (!h || s < 0 || s >= PIC_NSPECIES) return PIC_E_INVALID;
  DevClock c;
  PIC_TRY(clock_sync(h, &c));
  const int64_t n = c.n[s];
  if (n_out) *n_out = n;
  if (n > cap) return pic_fail(h, PIC_E_CAPACITY, "output arrays too short");
  Species &S = h->sp[s];
  cudaStream_t st = h->stream;
  if (n) {
    if (x) PIC_CUDA(h, cudaMemcpyAsync(x, S.a.x, n * 4, cudaMemcpyDeviceToHost, st));
    if (y) PIC_CUDA(h, cudaMemcpyAsync(y, S.a.y, n * 4, cudaMemcpyDeviceToHost, st));
    if (z) PIC_CUDA(h, cudaMemcpyAsync(z, S.a.z, n * 4, cudaMemcpyDeviceToHost, st));
    if (vx) PIC_CUDA(h, cudaMemcpyAsync(vx, S.a.vx, n * 4, cudaMemcpyDeviceToHost, st));
    if (vy) PIC_CUDA(h, cudaMemcpyAsync(vy, S.a.vy, n * 4, cudaMemcpyDeviceToHost, st));
    if (vz) PIC_CUDA(h, cudaMemcpyAsync(vz, S.a.vz, n * 4, cudaMemcpyDeviceToHost, st));
    if (w) PIC_CUDA(h, cudaMemcpyAsync(w, S.a.w, n * 4, cudaMemcpyDeviceToHost, st));
    if (id) PIC_CUDA(h, cudaMemcpyAsync(id, S.a.id, n * 8, cudaMemcpyDeviceToHost, st));
  }
  PIC_CUDA(h, cudaStreamSynchronize(st));
  return PIC_OK;
}

int pic_set_potential(pic_t *h, const double *phi) {
  if (!h || !phi) return PIC_E_INVALID;
  for (int64_t i = 0; i < h->nnode; ++i)
    if (!(fabs(phi[i]) < kPhiMax)) return pic_fail(h, PIC_E_INVALID, "potential outside (-8192, 8192) V or not finite");
  double *buf = (double *)dalloc(h, (size_t)h->nnode * 8);
  if (!buf) return pic_fail(h, PIC_E_CUDA, "staging allocation failed");
  int rc = PIC_OK;
  if (cudaMemcpyAsync(buf, phi, h->nnode * 8, cudaMemcpyHostToDevice, h->stream) != cudaSuccess) rc = PIC_E_CUDA;
  if (rc == PIC_OK) {
    ++h->nlaunch;
    k_phi_from_double<<<grid_for(h->nnode), kThreads, 0, h->stream>>>(buf, h->phi, h->nnode);
    h->dirichlet_valid = false;
    if (cudaMemsetAsync(&h->clock->phi_prev_ok, 0, sizeof(int), h->stream) != cudaSuccess) rc = PIC_E_CUDA;
    graph_free(h);
    rc = stage_efield(h);
  }
  if (rc == PIC_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = PIC_E_CUDA;
  dfree(h, buf);
  return rc == PIC_OK ? PIC_OK : pic_fail(h, rc, "set_potential failed");
}

static int d2h(pic_t *h, void *dst, const void *src, size_t bytes) {
  if (!dst) return pic_fail(h, PIC_E_INVALID, "null output");
  PIC_CUDA(h, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, h->stream));
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

int pic_get_potential(pic_t *h, double *phi) {
  if (!h) return PIC_E_INVALID;
  double *buf = (double *)dalloc(h, (size_t)h->nnode * 8);
  if (!buf) return pic_fail(h, PIC_E_CUDA, "staging allocation failed");
  ++h->nlaunch;
  k_phi_to_double<<<grid_for(h->nnode), kThreads, 0, h->stream>>>(h->phi, buf, h->nnode);
  const int rc = d2h(h, phi, buf, h->nnode * 8);
  dfree(h, buf);
  return rc;
}
int pic_get_charge(pic_t *h, int64_t *Q) { return h ? d2h(h, Q, h->Q, h->nnode * 8) : PIC_E_INVALID; }

int pic_get_efield(pic_t *h, float *E) {
  if (!h || !E) return PIC_E_INVALID;
  std::vector<float4> tmp(h->nnode);
  PIC_TRY(d2h(h, tmp.data(), h->E, h->nnode * sizeof(float4)));
  for (int64_t n = 0; n < h->nnode; ++n) { E[3 * n] = tmp[n].x; E[3 * n + 1] = tmp[n].y; E[3 * n + 2] = tmp[n].z; }
  return PIC_OK;
}

int pic_num_solid(pic_t *h, int64_t *n) {
  if (!h || !n) return PIC_E_INVALID;
  *n = h->heat.nvox;
  return PIC_OK;
}

int pic_set_temperature(pic_t *h, const double *T) {
  if (!h || !T) return PIC_E_INVALID;
  if (h->heat.nvox) {
    PIC_CUDA(h, cudaMemcpyAsync(h->heat.T, T, h->heat.nvox * 8, cudaMemcpyHostToDevice, h->stream));
    PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  return PIC_OK;
}

int pic_get_temperature(pic_t *h, double *T) {
  if (!h) return PIC_E_INVALID;
  return h->heat.nvox ? d2h(h, T, h->heat.T, h->heat.nvox * 8) : PIC_OK;
}

int pic_num_faces(pic_t *h, int64_t *n) {
  if (!h || !n) return PIC_E_INVALID;
  *n = h->faces.n;
  return PIC_OK;
}

int pic_get_faces(pic_t *h, int64_t *vcell, int32_t *dir, int64_t *owner) {
  if (!h) return PIC_E_INVALID;
  const int64_t n = h->faces.n;
  std::vector<int32_t> v(n), o(n);
  std::vector<int8_t> d(n);
  if (n) {
    PIC_TRY(d2h(h, v.data(), h->faces.vcell, n * 4));
    PIC_TRY(d2h(h, d.data(), h->faces.dir, n));
    PIC_TRY(d2h(h, o.data(), h->faces.owner, n * 4));
  }
  for (int64_t f = 0; f < n; ++f) {
    if (vcell) vcell[f] = v[f];
    if (dir) dir[f] = d[f];
    if (owner) owner[f] = o[f];
  }
  return PIC_OK;
}

int pic_get_face_emission(pic_t *h, double *F, double *J, double *PN) {
  if (!h) return PIC_E_INVALID;
  const size_t b = h->faces.n * 8;
  if (!h->faces.n) return PIC_OK;
  if (F) PIC_TRY(d2h(h, F, h->faces.F, b));
  if (J) PIC_TRY(d2h(h, J, h->faces.J, b));
  if (PN) PIC_TRY(d2h(h, PN, h->faces.PN, b));
  return PIC_OK;
}

int pic_get_face_accumulators(pic_t *h, double *evap, double *heat, double *charge, int64_t *sput, int64_t *Eb, int64_t *Es) {
  if (!h) return PIC_E_INVALID;
  const size_t b = h->faces.n * 8;
  if (!h->faces.n) return PIC_OK;
  if (evap) PIC_TRY(d2h(h, evap, h->faces.acc_evap, b));
  if (heat) PIC_TRY(d2h(h, heat, h->faces.acc_heat, b));
  if (charge) PIC_TRY(d2h(h, charge, h->faces.acc_charge, b));
  if (sput) PIC_TRY(d2h(h, sput, h->faces.acc_sput, b));
  if (Eb) PIC_TRY(d2h(h, Eb, h->faces.acc_Eb, b));
  if (Es) PIC_TRY(d2h(h, Es, h->faces.acc_Es, b));
  return PIC_OK;
}

int pic_set_face_accumulators(pic_t *h, const double *evap, const double *heat, const double *charge, const int64_t *sput,
                              const int64_t *Eb, const int64_t *Es) {
  if (!h) return PIC_E_INVALID;
  const size_t b = h->faces.n * 8;
  if (!h->faces.n) return PIC_OK;
  cudaStream_t st = h->stream;
  if (evap) PIC_CUDA(h, cudaMemcpyAsync(h->faces.acc_evap, evap, b, cudaMemcpyHostToDevice, st));
  if (heat) PIC_CUDA(h, cudaMemcpyAsync(h->faces.acc_heat, heat, b, cudaMemcpyHostToDevice, st));
  if (charge) PIC_CUDA(h, cudaMemcpyAsync(h->faces.acc_charge, charge, b, cudaMemcpyHostToDevice, st));
  if (sput) PIC_CUDA(h, cudaMemcpyAsync(h->faces.acc_sput, sput, b, cudaMemcpyHostToDevice, st));
  if (Eb) PIC_CUDA(h, cudaMemcpyAsync(h->faces.acc_Eb, Eb, b, cudaMemcpyHostToDevice, st));
  if (Es) PIC_CUDA(h, cudaMemcpyAsync(h->faces.acc_Es, Es, b, cudaMemcpyHostToDevice, st));
  PIC_CUDA(h, cudaStreamSynchronize(st));
  return PIC_OK;
}

// ---- stages -------------------------------------------------------------------------------
int pic_sort(pic_t *h);

int pic_set_flags(pic_t *h, uint32_t flags) {
  if (!h) return PIC_E_INVALID;
  // switching the extrapolation on: the stored previous potential may be many steps old
  if ((flags & PIC_F_EXTRAPOLATE) && !(h->prm.flags & PIC_F_EXTRAPOLATE) && h->phi_prev)
    PIC_CUDA(h, cudaMemsetAsync(&h->clock->phi_prev_ok, 0, sizeof(int), h->stream));
  h->prm.flags = flags;
  graph_free(h);
  return PIC_OK;
}

int pic_set_solver(pic_t *h, double mg_tol, int mg_max_cycles) {
  if (!h || !(mg_tol > 0) || mg_max_cycles < 1) return PIC_E_INVALID;
  h->prm.mg_tol = mg_tol;
  h->prm.mg_max_cycles = mg_max_cycles;
  graph_invalidate(h);   // the recorded convergence test holds the old values
  return PIC_OK;
}

int pic_emit(pic_t *h) {
  if (!h) return PIC_E_INVALID;
  PIC_TRY(stage_emit(h));
  return check_err(h);
}

int pic_push(pic_t *h) {
  if (!h) return PIC_E_INVALID;
  PIC_TRY(stage_push(h));
  return check_err(h);
}

int pic_sort(pic_t *h) {
  if (!h) return PIC_E_INVALID;
  PIC_TRY(stage_sort(h));
  return check_err(h);
}

int pic_merge(pic_t *h) {
  if (!h) return PIC_E_INVALID;
  if (!(h->prm.flags & PIC_F_MERGE)) return pic_fail(h, PIC_E_INVALID, "merging is off: set PIC_F_MERGE");
  PIC_TRY(stage_merge(h));
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  return check_err(h);
}


int pic_circuit(pic_t *h) {
  if (!h) return PIC_E_INVALID;
  if (!circuit_on(h)) return pic_fail(h, PIC_E_INVALID, "no circuit: set circuit_R, circuit_C and PIC_F_CIRCUIT");
  PIC_TRY(stage_circuit(h));
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  return launch_check(h, "circuit");
}

int pic_collide(pic_t *h) {
  if (!h) return PIC_E_INVALID;
  PIC_TRY(stage_collide(h));
  return check_err(h);
}

int pic_deposit(pic_t *h) {
  if (!h) return PIC_E_INVALID;
  PIC_TRY(stage_deposit(h));
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

int pic_solve_field(pic_t *h) {
  if (!h) return PIC_E_INVALID;
  PIC_TRY(stage_deposit(h));
  PIC_TRY(stage_solve(h, false, h->V0));
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

int pic_heat(pic_t *h) {
  if (!h) return PIC_E_INVALID;
  PIC_TRY(stage_heat(h));
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

int pic_num_kernels(void) { return kidNum; }

const char *pic_kernel_name(int k) { return k >= 0 && k < kidNum ? kKernelNames[k] : nullptr; }

int pic_set_kernel_timing(pic_t *h, uint64_t mask) {
  if (!h) return PIC_E_INVALID;
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  kt_collect(h);
  h->kt_mask = mask;
  for (int k = 0; k < 64; ++k) { h->kt_ms[k] = 0; h->kt_units[k] = 0; h->kt_n[k] = 0; }
  return PIC_OK;
}

int pic_get_kernel_timing(pic_t *h, int k, int64_t *launches, double *ms, double *units) {
  if (!h || k < 0 || k >= kidNum) return PIC_E_INVALID;
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  kt_collect(h);
  if (launches) *launches = h->kt_n[k];
  if (ms) *ms = h->kt_ms[k];
  if (units) *units = h->kt_units[k];
  return PIC_OK;
}

__global__ void k_begin_step(DevClock *clk) {
  for (int i = 0; i < cNum; ++i) clk->ctr[i] = 0;
}
__global__ void k_end_step(DevClock *clk) { clk->step += 1; }

}  // extern "C"

// ---- graph form of the step ---------------------------------------------------------------------
// One step recorded into the graph being captured on h->stream: the stages in their eager order,
// the Poisson loop as a conditional while node.  The heat stage is not part of it.
static int step_body_graph(pic_t *h) {
  ++h->nlaunch;
  k_begin_step<<<1, 1, 0, h->stream>>>(h->clock);
  PIC_TRY(stage_emit(h));
  PIC_TRY(stage_push(h, true));   // the charge deposit runs in the push (see pic_step_eager)
  PIC_TRY(stage_circuit(h));
  PIC_TRY(stage_sort(h));
  PIC_TRY(stage_merge(h, true));
  PIC_TRY(stage_collide(h));
  PIC_TRY(stage_extrapolate(h));
  PIC_TRY(stage_solve_graph(h, h->V0));
  ++h->nlaunch;
  k_end_step<<<1, 1, 0, h->stream>>>(h->clock);
  return launch_check(h, "step capture");
}


static void graph_free(pic_t *h) {
  for (int p = 0; p < 2; ++p)
    if (h->gexec[p]) {
      cudaGraphExecDestroy(h->gexec[p]);
      h->gexec[p] = nullptr;
    }
  h->graph_valid = false;
}

// Index of the graph whose particle buffers are the current ones, -1 if none
static int graph_index(pic_t *h) {
  for (int p = 0; p < 2; ++p) {
    bool ok = h->gexec[p] != nullptr;
    for (int s = 0; s < nsp_active(h); ++s) ok = ok && h->graph_a[p][s] == h->sp[s].a.x;
    if (ok) return p;
  }
  return -1;
}

namespace pic {
void graph_invalidate(pic_t *h) {
  graph_free(h);
  h->eager_flags = 0xFFFFFFFFu;
}

// Records one graph per parity of the particle double buffers (the sort swaps them every step,
// and a graph holds fixed addresses).  Nothing runs during the recording; the host-side buffer
// assignment is restored afterwards.  Lazily allocated buffers must exist already: a graph is
// built only after an eager step with the same flags (pic_step does that).
int graph_build_capture(pic_t *h) {
  graph_free(h);
  if (!h->body_stream) PIC_CUDA(h, cudaStreamCreateWithFlags(&h->body_stream, cudaStreamNonBlocking));
  if (!h->cap_stream) PIC_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  for (int s = 0; s < PIC_NSPECIES; ++s)
    if (h->keys_valid[s]) PIC_TRY(stage_sort(h));   // a step starts from sorted SPs
  SpeciesBuf saved[PIC_NSPECIES][2];
  for (int s = 0; s < PIC_NSPECIES; ++s) { saved[s][0] = h->sp[s].a; saved[s][1] = h->sp[s].b; }
  const uint64_t kt = h->kt_mask;
  h->kt_mask = 0;
  const int64_t n0 = h->nlaunch;
  int rc = PIC_OK;
  for (int p = 0; p < 2 && rc == PIC_OK; ++p) {
    for (int s = 0; s < PIC_NSPECIES; ++s) h->graph_a[p][s] = h->sp[s].a.x;
    // recorded on a private stream (the caller's may be the legacy stream, which cannot be
    // captured); the graph is launched on the caller's stream
    cudaGraph_t g = nullptr;
    cudaStream_t user = h->stream;
    h->stream = h->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
      h->stream = user;
      rc = pic_fail(h, PIC_E_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
      break;
    }
    h->capturing = true;
    const int64_t m0 = h->nlaunch;
    rc = step_body_graph(h);
    h->capturing = false;
    e = cudaStreamEndCapture(h->stream, &g);
    h->stream = user;
    if (rc == PIC_OK && e != cudaSuccess) rc = pic_fail(h, PIC_E_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
    if (rc == PIC_OK) {
      e = cudaGraphInstantiate(&h->gexec[p], g, 0);
      if (e != cudaSuccess) rc = pic_fail(h, PIC_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    if (g) cudaGraphDestroy(g);
    h->graph_outer_launches = h->nlaunch - m0 - h->graph_body_launches;
  }
  cudaGetLastError();
  h->nlaunch = n0;
  h->kt_mask = kt;
  for (int s = 0; s < PIC_NSPECIES; ++s) { h->sp[s].a = saved[s][0]; h->sp[s].b = saved[s][1]; h->keys_valid[s] = false; }
  if (rc != PIC_OK) { graph_free(h); return rc; }
  h->graph_valid = true;
  h->graph_flags = h->prm.flags;
  return PIC_OK;
}

// Launch the graph of the current parity (one step) and advance the host-side buffer assignment.
int graph_launch_step(pic_t *h) {
  const int p = graph_index(h);
  if (p < 0) return pic_fail(h, PIC_E_INVALID, "no step graph for the current particle buffers");
  PIC_CUDA(h, cudaGraphLaunch(h->gexec[p], h->stream));
  for (int s = 0; s < nsp_active(h); ++s) std::swap(h->sp[s].a, h->sp[s].b);
  h->nlaunch += h->graph_outer_launches;
  return PIC_OK;
}

}  // namespace pic

static int pic_step_graph(pic_t *h, int nsteps, int64_t step) {
  if (!h->graph_valid || h->graph_flags != h->prm.flags || graph_index(h) < 0) PIC_TRY(graph_build_capture(h));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, h->stream);
  int rc = PIC_OK;
  for (int it = 0; it < nsteps && rc == PIC_OK; ++it) {
    rc = graph_launch_step(h);
    ++step;
    if (rc == PIC_OK && (h->prm.flags & PIC_F_HEAT) && h->prm.n_heat > 0 && step % h->prm.n_heat == 0) rc = stage_heat(h);
  }
  cudaEventRecord(e1, h->stream);
  cudaEventSynchronize(e1);
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == PIC_OK && nsteps > 0) {
    for (int i = 0; i < 7; ++i) h->ms[i] = 0.f;   // the stages of a graph are not timed apart
    h->ms[7] = t;
  }
  if (rc != PIC_OK) return rc;
  PIC_TRY(launch_check(h, "graph step"));
  return check_err(h);
}

static int pic_step_eager(pic_t *h, int nsteps, int64_t step);

// ---- ensemble of independent instances -----------------------------------------------------------
constexpr int kNs = PIC_NSPECIES;   // species slots per instance in the batch tables

struct pic_batch_s {
  std::vector<pic_t *> inst;
  cudaStream_t stream = nullptr;       // the instances' common stream
  cudaStream_t cap = nullptr;          // private capture stream
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  std::vector<float *> graph_a[2];     // S.a.x of every instance and species at capture
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  bool valid = false;
  std::vector<uint32_t> flags;         // each instance's flags at capture
  float ms = 0.f;
  std::string err;
};

static void batch_free_graphs(pic_batch_t *b) {
  for (int p = 0; p < 2; ++p)
    if (b->gexec[p]) {
      cudaGraphExecDestroy(b->gexec[p]);
      b->gexec[p] = nullptr;
    }
  b->valid = false;
}

static int batch_index(pic_batch_t *b) {
  for (int p = 0; p < 2; ++p) {
    if (!b->gexec[p]) continue;
    bool ok = true;
    for (size_t i = 0; i < b->inst.size() && ok; ++i)
      for (int s = 0; s < nsp_active(b->inst[i]); ++s) ok = ok && b->graph_a[p][kNs * i + s] == b->inst[i]->sp[s].a.x;
    for (size_t i = 0; i < b->inst.size() && ok; ++i) ok = b->flags[i] == b->inst[i]->prm.flags;
    if (ok) return p;
  }
  return -1;
}

// One graph per buffer parity holding one step of every instance: the capture forks from the
// batch's private stream into each instance's own capture stream and joins back, so the
// instances form independent branches that the GPU runs concurrently; each branch holds its
// instance's Poisson loop as a device-side while node.
static int batch_capture(pic_batch_t *b) {
  batch_free_graphs(b);
  const size_t n = b->inst.size();
  for (pic_t *h : b->inst) {
    if (!h->body_stream && cudaStreamCreateWithFlags(&h->body_stream, cudaStreamNonBlocking) != cudaSuccess) return PIC_E_CUDA;
    if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return PIC_E_CUDA;
    for (int s = 0; s < PIC_NSPECIES; ++s)
      if (h->keys_valid[s]) PIC_TRY(stage_sort(h));
  }
  std::vector<SpeciesBuf> saved(2 * kNs * n);
  std::vector<uint64_t> kt(n);
  std::vector<int64_t> n0(n);
  for (size_t i = 0; i < n; ++i) {
    for (int s = 0; s < kNs; ++s) { saved[2 * (kNs * i + s)] = b->inst[i]->sp[s].a; saved[2 * (kNs * i + s) + 1] = b->inst[i]->sp[s].b; }
    kt[i] = b->inst[i]->kt_mask;
    b->inst[i]->kt_mask = 0;
    n0[i] = b->inst[i]->nlaunch;
  }
  int rc = PIC_OK;
  for (int p = 0; p < 2 && rc == PIC_OK; ++p) {
    b->graph_a[p].assign(kNs * n, nullptr);
    for (size_t i = 0; i < n; ++i)
      for (int s = 0; s < kNs; ++s) b->graph_a[p][kNs * i + s] = b->inst[i]->sp[s].a.x;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) { b->err = std::string("begin capture: ") + cudaGetErrorString(e); rc = PIC_E_CUDA; break; }
    if (cudaEventRecord(b->fork, b->cap) != cudaSuccess) rc = PIC_E_CUDA;
    for (size_t i = 0; i < n && rc == PIC_OK; ++i) {
      pic_t *h = b->inst[i];
      cudaStream_t user = h->stream;
      h->stream = h->cap_stream;
      if (cudaStreamWaitEvent(h->stream, b->fork, 0) != cudaSuccess) rc = PIC_E_CUDA;
      h->capturing = true;
      const int64_t m0 = h->nlaunch;
      if (rc == PIC_OK) rc = step_body_graph(h);
      h->capturing = false;
      h->graph_outer_launches = h->nlaunch - m0 - h->graph_body_launches;
      if (rc == PIC_OK && cudaEventRecord(b->join[i], h->stream) != cudaSuccess) rc = PIC_E_CUDA;
      if (rc == PIC_OK && cudaStreamWaitEvent(b->cap, b->join[i], 0) != cudaSuccess) rc = PIC_E_CUDA;
      if (rc != PIC_OK) b->err = "instance " + std::to_string(i) + ": " + h->last_error;
      h->stream = user;
    }
    e = cudaStreamEndCapture(b->cap, &g);
    if (rc == PIC_OK && e != cudaSuccess) { b->err = std::string("end capture: ") + cudaGetErrorString(e); rc = PIC_E_CUDA; }
    if (rc == PIC_OK && (e = cudaGraphInstantiate(&b->gexec[p], g, 0)) != cudaSuccess) {
      b->err = std::string("graph instantiate: ") + cudaGetErrorString(e);
      rc = PIC_E_CUDA;
    }
    if (g) cudaGraphDestroy(g);
  }
  cudaGetLastError();
  for (size_t i = 0; i < n; ++i) {
    pic_t *h = b->inst[i];
    for (int s = 0; s < kNs; ++s) {
      h->sp[s].a = saved[2 * (kNs * i + s)];
      h->sp[s].b = saved[2 * (kNs * i + s) + 1];
      h->keys_valid[s] = false;
    }
    h->kt_mask = kt[i];
    h->nlaunch = n0[i];
  }
  if (rc != PIC_OK) { batch_free_graphs(b); return rc; }
  b->flags.resize(n);
  for (size_t i = 0; i < n; ++i) b->flags[i] = b->inst[i]->prm.flags;
  b->valid = true;
  return PIC_OK;
}

extern "C" {

int pic_batch_create(pic_t *const *instances, int n, pic_batch_t **out) {
  if (!instances || n < 1 || !out) return PIC_E_INVALID;
  *out = nullptr;
  pic_batch_t *b = new pic_batch_t();
  for (int i = 0; i < n; ++i) {
    if (!instances[i]) { delete b; return PIC_E_INVALID; }
    for (pic_t *o : b->inst)
      if (o == instances[i]) { delete b; return PIC_E_INVALID; }   // each instance once
    b->inst.push_back(instances[i]);
  }
  b->stream = b->inst[0]->stream;
  for (pic_t *h : b->inst)
    if (h->stream != b->stream) { delete b; return PIC_E_INVALID; }   // one common stream
  bool ok = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  b->join.assign(n, nullptr);
  for (int i = 0; i < n && ok; ++i) ok = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) { pic_batch_destroy(b); return PIC_E_CUDA; }
  *out = b;
  return PIC_OK;
}

void pic_batch_destroy(pic_batch_t *b) {
  if (!b) return;
  if (b->stream || b->cap) cudaStreamSynchronize(b->stream);
  batch_free_graphs(b);
  if (b->fork) cudaEventDestroy(b->fork);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

const char *pic_batch_last_error(pic_batch_t *b) { return b ? b->err.c_str() : "null batch"; }

int pic_batch_step(pic_batch_t *b, int nsteps) {
  if (!b || nsteps < 0) return PIC_E_INVALID;
  if (nsteps == 0) return PIC_OK;
  const size_t n = b->inst.size();
  std::vector<int64_t> step(n);
  for (size_t i = 0; i < n; ++i) {
    DevClock c;
    PIC_TRY(clock_sync(b->inst[i], &c));
    step[i] = c.step;
  }
  // an instance records its graph only after an eager step with its current flags
  bool eager = false;
  for (pic_t *h : b->inst) {
    bool sorted = true;
    for (int s = 0; s < PIC_NSPECIES; ++s) sorted = sorted && !h->keys_valid[s];
    eager = eager || h->eager_flags != h->prm.flags || !sorted;
  }
  if (eager) {
    for (size_t i = 0; i < n; ++i) {
      const int rc = pic_step_eager(b->inst[i], 1, step[i]);
      if (rc != PIC_OK) { b->err = "instance " + std::to_string(i) + ": " + b->inst[i]->last_error; return rc; }
      ++step[i];
    }
    if (--nsteps == 0) return PIC_OK;
  }
  if (!b->valid || batch_index(b) < 0) PIC_TRY(batch_capture(b));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, b->stream);
  int rc = PIC_OK;
  for (int it = 0; it < nsteps && rc == PIC_OK; ++it) {
    const int p = batch_index(b);
    if (p < 0) { b->err = "no ensemble graph for the current particle buffers"; rc = PIC_E_INVALID; break; }
    if (cudaGraphLaunch(b->gexec[p], b->stream) != cudaSuccess) { b->err = "graph launch"; rc = PIC_E_CUDA; break; }
    for (size_t i = 0; i < n; ++i) {
      pic_t *h = b->inst[i];
      for (int s = 0; s < nsp_active(h); ++s) std::swap(h->sp[s].a, h->sp[s].b);
      h->nlaunch += h->graph_outer_launches;
      h->last_solve_graph = true;
      ++step[i];
      if ((h->prm.flags & PIC_F_HEAT) && h->prm.n_heat > 0 && step[i] % h->prm.n_heat == 0) {
        rc = stage_heat(h);
        if (rc != PIC_OK) { b->err = "instance " + std::to_string(i) + ": " + h->last_error; break; }
      }
    }
  }
  cudaEventRecord(e1, b->stream);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&b->ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != PIC_OK) return rc;
  for (size_t i = 0; i < n; ++i) {
    const int r = check_err(b->inst[i]);
    if (r != PIC_OK) { b->err = "instance " + std::to_string(i) + ": " + b->inst[i]->last_error; return r; }
  }
  return PIC_OK;
}

int pic_batch_ms(pic_batch_t *b, double *ms) {
  if (!b || !ms) return PIC_E_INVALID;
  *ms = b->ms;
  return PIC_OK;
}

// Autotuner: time the launch-shape candidates of the particle kernels, the fixed-point residual
// and the smoother on this instance's current state and keep the fastest; choices[0] receives the
// particle blocks per SM, choices[1] the residual's planes per thread, choices[2 + l] the
// smoother's planes per thread on level l.  Results do not depend on
// the choices.  Returns the number of values written (<= cap) or a negative error code.
int pic_autotune(pic_t *h, int *choices, int cap) {
  if (!h || (cap > 0 && !choices)) return PIC_E_INVALID;
  int bps = 0;
  PIC_TRY(tune_particles(h, &bps));
  int kz[16] = {0};
  PIC_TRY(tune_smoother(h, kz, 16));
  int rkz = 0;
  PIC_TRY(tune_residual(h, &rkz));
  graph_invalidate(h);
  int nw = 0;
  if (cap > 0) choices[nw++] = bps;
  if (cap > 1) choices[nw++] = rkz;
  const int nl = std::min<int>((int)h->mg.size() - 1, 16);
  for (int l = 0; l < nl && nw < cap; ++l) choices[nw++] = kz[l];
  return nw;
}

}  // extern "C"


extern "C" {

int pic_step(pic_t *h, int nsteps) {
  if (!h || nsteps < 0) return PIC_E_INVALID;
  DevClock c;
  PIC_TRY(clock_sync(h, &c));
  int64_t step = c.step;
  bool sorted = true;
  for (int s = 0; s < PIC_NSPECIES; ++s) sorted = sorted && !h->keys_valid[s];
  if ((h->prm.flags & PIC_F_GRAPH) && sorted && nsteps > 0) {
    // a graph is recorded only after an eager step with the same flags (lazily allocated buffers)
    if (h->eager_flags != h->prm.flags) {
      PIC_TRY(pic_step_eager(h, 1, step));
      ++step;
      --nsteps;
    }
    return nsteps > 0 ? pic_step_graph(h, nsteps, step) : PIC_OK;
  }
  return pic_step_eager(h, nsteps, step);
}

}  // extern "C"

// the step stage by stage from the host, with per-stage event timing
static int pic_step_eager(pic_t *h, int nsteps, int64_t step) {
  // eight events per step, read once after the last step: no host wait between steps beyond
  // the solve's own convergence checks
  const size_t need = (size_t)8 * std::max(nsteps, 0);
  while (h->step_ev.size() < need) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return pic_fail(h, PIC_E_CUDA, "event creation failed");
    h->step_ev.push_back(e);
  }
  int rc = PIC_OK;
  int done = 0;
  for (int it = 0; it < nsteps && rc == PIC_OK; ++it) {
    cudaEvent_t *ev = h->step_ev.data() + 8 * it;
    cudaEventRecord(ev[0], h->stream);
    ++h->nlaunch;
    k_begin_step<<<1, 1, 0, h->stream>>>(h->clock);
    rc = stage_emit(h);
    cudaEventRecord(ev[1], h->stream);
    // The charge of the step is deposited by the push, from the pushed positions of the charged
    // SPs that stay in the domain.  Nothing after it changes the charge on any node: impact and
    // field ionization put the new ion and its electron on the same position with the same weight
    // (their CIC charges cancel exactly), SP splitting keeps the position and the weight sum, the
    // elastic, exchange and Coulomb passes change velocities only, and merging moves its pairs'
    // charges itself.  The deposit stage of the step is therefore empty; its time is in the push.
    if (rc == PIC_OK) rc = stage_push(h, true);
    if (rc == PIC_OK) rc = stage_circuit(h);
    cudaEventRecord(ev[2], h->stream);
    if (rc == PIC_OK) rc = stage_sort(h);
    if (rc == PIC_OK) rc = stage_merge(h, true);
    cudaEventRecord(ev[3], h->stream);
    if (rc == PIC_OK) rc = stage_collide(h);
    cudaEventRecord(ev[4], h->stream);
    cudaEventRecord(ev[5], h->stream);
    if (rc == PIC_OK) rc = stage_extrapolate(h);
    if (rc == PIC_OK) rc = stage_solve(h, false, h->V0);
    cudaEventRecord(ev[6], h->stream);
    ++step;
    if (rc == PIC_OK && (h->prm.flags & PIC_F_HEAT) && h->prm.n_heat > 0 && step % h->prm.n_heat == 0) {
      KtScope kt_(h, kidHeat, (double)h->heat.nvox);
      rc = stage_heat(h);
    }
    ++h->nlaunch;
    k_end_step<<<1, 1, 0, h->stream>>>(h->clock);
    cudaEventRecord(ev[7], h->stream);
    ++done;
  }
  // per-stage times summed over the steps of this call (events on the library stream)
  float acc_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (done > 0) cudaEventSynchronize(h->step_ev[8 * (done - 1) + 7]);
  kt_collect(h);
  for (int it = 0; it < done; ++it) {
    cudaEvent_t *ev = h->step_ev.data() + 8 * it;
    float t;
    for (int i = 0; i < 7; ++i) {
      cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
      acc_ms[i] += t;
    }
    cudaEventElapsedTime(&t, ev[0], ev[7]);
    acc_ms[7] += t;
  }
  if (rc == PIC_OK && nsteps > 0)
    for (int i = 0; i < 8; ++i) h->ms[i] = acc_ms[i];
  if (rc != PIC_OK) return rc;
  PIC_TRY(launch_check(h, "step"));
  PIC_TRY(check_err(h));
  if (nsteps > 0) h->eager_flags = h->prm.flags;
  return PIC_OK;
}

extern "C" {

__global__ void k_sum_w(const int32_t *w, const DevClock *clk, int s, unsigned long long *out) {
  const int64_t n = clk->n[s];
  long long acc = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) acc += w[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, (unsigned long long)acc);
}

__global__ void k_sum_q(const unsigned long long *Q, int64_t n, unsigned long long *out) {
  long long acc = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += (long long)Q[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, (unsigned long long)acc);
}

int pic_diagnostics(pic_t *h, pic_diag_t *out) {
  if (!h || !out) return PIC_E_INVALID;
  memset(out, 0, sizeof *out);
  DevClock c;
  PIC_TRY(clock_sync(h, &c));
  out->step = c.step;
  out->next_id = c.next_id;
  unsigned long long *sums = (unsigned long long *)(h->tmp_len + 16);
  PIC_CUDA(h, cudaMemsetAsync(sums, 0, (PIC_NSPECIES + 1) * 8, h->stream));
  for (int s = 0; s < PIC_NSPECIES; ++s) {
    out->count[s] = c.n[s];
    ++h->nlaunch;
    k_sum_w<<<h->nsm * 4, kThreads, 0, h->stream>>>(h->sp[s].a.w, h->clock, s, sums + s);
    out->removed[s] = c.ctr[cRemovedE + s];
  }
  ++h->nlaunch;
  k_sum_q<<<h->nsm * 4, kThreads, 0, h->stream>>>(h->Q, h->nnode, sums + PIC_NSPECIES);
  unsigned long long hs[PIC_NSPECIES + 1];
  PIC_TRY(d2h(h, hs, sums, sizeof hs));
  for (int s = 0; s < PIC_NSPECIES; ++s) out->weight[s] = (int64_t)hs[s];
  out->total_charge_fixed = (int64_t)hs[PIC_NSPECIES];
  out->emitted = c.ctr[cEmitted];
  out->evaporated = c.ctr[cEvaporated];
  out->sputtered = c.ctr[cSputtered];
  out->impact_ionizations = c.ctr[cImpactIon];
  out->field_ionizations = c.ctr[cFieldIon];
  out->elastic_en = c.ctr[cElasticEn];
  out->elastic_nn = c.ctr[cElasticNn];
  out->charge_exchanges = c.ctr[cChargeEx];
  out->coulomb_ee = c.ctr[cCoulombEe];
  out->coulomb_ei = c.ctr[cCoulombEi];
  out->coulomb_ii = c.ctr[cCoulombIi];
  out->double_ionizations = c.ctr[cDoubleIon];
  out->ion_ionizations = c.ctr[cIonIon];
  out->coulomb_ej = c.ctr[cCoulombEj];
  out->coulomb_ij = c.ctr[cCoulombIj];
  out->coulomb_jj = c.ctr[cCoulombJj];
  out->merged = c.ctr[cMerged];
  out->fallback_range = c.ctr[cFbRange];
  out->fallback_bin = c.ctr[cFbBin];
  out->ion_impacts = c.ctr[cIonImpacts];
  out->mg_cycles = h->last_solve_graph ? c.mg_cycles_last : h->last_mg_cycles;
  out->mg_residual = h->last_solve_graph ? (double)c.mg_rel_last : h->last_mg_res;
  out->V0 = h->V0;
  const int64_t nf = h->faces.n;
  if (nf) {
    std::vector<double> F(nf), J(nf);
    PIC_TRY(d2h(h, F.data(), h->faces.F, nf * 8));
    PIC_TRY(d2h(h, J.data(), h->faces.J, nf * 8));
    double cur = 0;
    for (int64_t f = 0; f < nf; ++f) {
      out->max_face_field = std::max(out->max_face_field, F[f]);
      out->max_J = std::max(out->max_J, J[f]);
      cur += J[f] * h->dx * h->dx;
    }
    out->emitted_current = cur;
  }
  if (h->heat.nvox) {
    std::vector<double> T(h->heat.nvox);
    PIC_TRY(d2h(h, T.data(), h->heat.T, h->heat.nvox * 8));
    out->max_T = *std::max_element(T.begin(), T.end());
  }
  for (int i = 0; i < 8; ++i) out->ms[i] = h->ms[i];
  out->kernel_launches = h->nlaunch + c.mg_graph_cycles * h->graph_body_launches;
  out->mg_cycles_total = h->mg_cycles_host + c.mg_graph_cycles;
  out->emission_evals = c.ctr[cWevals];
  out->V_gap = h->E0 ? c.V_gap : h->V0;
  out->I_gap = c.I_gap;
  out->I_tot = c.I_tot;
  out->surrogate_faces = c.ctr[cSurFaces];
  return PIC_OK;
}

int pic_emission_eval(pic_t *h, const double *F, const double *T, const double *phi_w, const double *R, double *J,
                      double *PN, int64_t n) {
  if (!h || n < 0 || (n > 0 && (!F || !T || !phi_w || !R || !J || !PN))) return PIC_E_INVALID;
  PIC_TRY(check_device(h));
  if (n == 0) return PIC_OK;
  double *buf = nullptr;
  PIC_CUDA(h, cudaMalloc(&buf, (size_t)n * 6 * 8));
  cudaStream_t st = h->stream;
  int rc = PIC_OK;
  if (cudaMemcpyAsync(buf, F, n * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(buf + n, T, n * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(buf + 2 * n, phi_w, n * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(buf + 3 * n, R, n * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
    rc = pic_fail(h, PIC_E_CUDA, "emission_eval upload");
  if (rc == PIC_OK) rc = emission_eval_dev(h, buf, buf + n, buf + 2 * n, buf + 3 * n, buf + 4 * n, buf + 5 * n, n,
                                         (h->prm.flags & PIC_F_FAST_INTEGRAL) != 0);
  if (rc == PIC_OK && (cudaMemcpyAsync(J, buf + 4 * n, n * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                       cudaMemcpyAsync(PN, buf + 5 * n, n * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                       cudaStreamSynchronize(st) != cudaSuccess))
    rc = pic_fail(h, PIC_E_CUDA, "emission_eval download");
  cudaFree(buf);
  return rc;
}

}  // extern "C"
