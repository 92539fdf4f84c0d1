// Checkpoint and resume of one instance: pic_save writes the whole evolving state of a handle to
// a file, pic_load puts it into a handle created with the same geometry, grid, species and
// physical parameters.  Every random draw of the step is keyed by (seed, purpose, SP or face id,
// step), so a resumed run draws the same numbers as an uninterrupted one and repeats it bit for
// bit.
//
// What is state (everything else is rebuilt by pic_create or overwritten before it is read):
//   * the device clock: step, next id, per-species counts (held and covered by the last sort),
//     event counters, the circuit's V_gap / I_gap / I_tot, the extrapolation flag;
//   * per species, the SoA of the held SPs in their device order, the per-cell offsets of the
//     last sort (injection weights read them, Sec. 2.3.2) and the cell key of each sorted place;
//   * the fixed-point potential, the deposited charge, the previous potential when the
//     time extrapolation keeps one;
//   * per face, the last emission pass (F, J, P_N) and the six surface accumulators;
//   * the tip temperature per solid cell;
//   * the surrogate's master weights and validity map, and whether it is trained;
//   * the host-side anode potential V0 and the PIC_F_* flags.
// The node field E is recomputed from the potential on load (a pure function of it).
//
// File: the 8 bytes "PICSTATE", a version, a header of fixed layout (the creation inputs and
// sizes), the device clock, then tagged sections in a fixed order.  Native byte order and struct
// layout (LP64, little endian: the same on x86-64 and aarch64 Linux).
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "pic_internal.cuh"

namespace pic {

constexpr char kMagic[8] = {'P', 'I', 'C', 'S', 'T', 'A', 'T', 'E'};
constexpr uint32_t kVersion = 2;   // 2: four species (Cu2+)

struct SaveHeader {
  uint32_t version, endian, header_bytes, clock_bytes;
  pic_grid_t grid;
  pic_geometry_t geo;
  int32_t Z[PIC_NSPECIES];
  double mass[PIC_NSPECIES];
  pic_params_t prm;
  double V0;
  int64_t nface, nvox, nnode, ncell;
  int32_t has_prev, circuit_ready, has_mlp, mlp_trained;
  int32_t mlp_params, mlp_bins, last_mg_cycles, pad0;
  double last_mg_res;       // diagnostics of the last Poisson solve
  int64_t mg_cycles_host;   // refinement cycles of host-driven solves since create
};

enum Tag : uint32_t {
  tSpecies = 1, tOffsets = 2, tSortKeys = 3, tPhi = 4, tCharge = 5, tPhiPrev = 6, tFaces = 7, tTemp = 8, tMlp = 9,
  tEnd = 0x454E4421u
};

struct File {
  FILE *f = nullptr;
  ~File() { if (f) fclose(f); }
};

static int put(pic_t *h, FILE *f, const void *p, size_t bytes) {
  if (bytes && fwrite(p, 1, bytes, f) != bytes) return pic_fail(h, PIC_E_INVALID, "pic_save: write failed");
  return PIC_OK;
}

static int get(pic_t *h, FILE *f, void *p, size_t bytes) {
  if (bytes && fread(p, 1, bytes, f) != bytes) return pic_fail(h, PIC_E_INVALID, "pic_load: file is truncated");
  return PIC_OK;
}

static int put_tag(pic_t *h, FILE *f, uint32_t tag, uint64_t bytes) {
  const uint32_t t[2] = {tag, 0};
  PIC_TRY(put(h, f, t, sizeof t));
  return put(h, f, &bytes, sizeof bytes);
}

static int expect_tag(pic_t *h, FILE *f, uint32_t tag, uint64_t bytes) {
  uint32_t t[2];
  uint64_t b = 0;
  PIC_TRY(get(h, f, t, sizeof t));
  PIC_TRY(get(h, f, &b, sizeof b));
  if (t[0] != tag || b != bytes)
    return pic_fail(h, PIC_E_INVALID, "pic_load: section " + std::to_string(t[0]) + " of " + std::to_string(b) +
                                          " bytes where section " + std::to_string(tag) + " of " +
                                          std::to_string(bytes) + " bytes was expected");
  return PIC_OK;
}

// device -> file through a host buffer of at most kChunk bytes
constexpr size_t kChunk = (size_t)64 << 20;

static int dev_to_file(pic_t *h, FILE *f, const void *dev, size_t bytes, std::vector<char> &buf) {
  for (size_t o = 0; o < bytes; o += kChunk) {
    const size_t n = std::min(kChunk, bytes - o);
    buf.resize(std::max(buf.size(), n));
    PIC_CUDA(h, cudaMemcpyAsync(buf.data(), (const char *)dev + o, n, cudaMemcpyDeviceToHost, h->stream));
    PIC_CUDA(h, cudaStreamSynchronize(h->stream));
    PIC_TRY(put(h, f, buf.data(), n));
  }
  return PIC_OK;
}

static int file_to_dev(pic_t *h, FILE *f, void *dev, size_t bytes, std::vector<char> &buf) {
  for (size_t o = 0; o < bytes; o += kChunk) {
    const size_t n = std::min(kChunk, bytes - o);
    buf.resize(std::max(buf.size(), n));
    PIC_TRY(get(h, f, buf.data(), n));
    PIC_CUDA(h, cudaMemcpyAsync((char *)dev + o, buf.data(), n, cudaMemcpyHostToDevice, h->stream));
    PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  return PIC_OK;
}

static void fill_header(pic_t *h, SaveHeader &H) {
  memset(&H, 0, sizeof H);
  H.version = kVersion;
  H.endian = 0x01020304u;
  H.header_bytes = sizeof(SaveHeader);
  H.clock_bytes = sizeof(DevClock);
  H.grid.nx = h->nx; H.grid.ny = h->ny; H.grid.nz = h->nz; H.grid.dx = h->dx;
  H.geo = h->geo;
  for (int s = 0; s < PIC_NSPECIES; ++s) { H.Z[s] = h->sp[s].Z; H.mass[s] = h->sp[s].mass; }
  H.prm = h->prm;
  H.V0 = h->V0;
  H.nface = h->faces.n; H.nvox = h->heat.nvox; H.nnode = h->nnode; H.ncell = h->ncell;
  H.has_prev = h->phi_prev != nullptr;
  H.circuit_ready = h->circuit_ready;
  H.mlp_params = pic_mlp_num_params();
  H.mlp_bins = surrogate_bins();
}

// the last solve's cycles and residual as pic_diagnostics reports them
static void fill_solve_diag(pic_t *h, const DevClock &c, SaveHeader &H) {
  H.last_mg_cycles = h->last_solve_graph ? c.mg_cycles_last : h->last_mg_cycles;
  H.last_mg_res = h->last_solve_graph ? (double)c.mg_rel_last : h->last_mg_res;
  H.mg_cycles_host = h->mg_cycles_host;
}

// The creation inputs that shape the state must agree; the solver controls (mg_tol,
// mg_max_cycles, mg_sweeps) and the flags may differ (the flags are restored from the file).
static int compatible(pic_t *h, const SaveHeader &F, const SaveHeader &M) {
  auto bad = [&](const char *what) { return pic_fail(h, PIC_E_INVALID, std::string("pic_load: ") + what + " differs"); };
  if (F.grid.nx != M.grid.nx || F.grid.ny != M.grid.ny || F.grid.nz != M.grid.nz || F.grid.dx != M.grid.dx) return bad("grid");
  if (F.geo.tip_radius != M.geo.tip_radius || F.geo.tip_height != M.geo.tip_height) return bad("tip geometry");
  for (int s = 0; s < PIC_NSPECIES; ++s)
    if (F.Z[s] != M.Z[s] || F.mass[s] != M.mass[s]) return bad("species charge or mass");
  const pic_params_t &a = F.prm, &b = M.prm;
  if (a.dt != b.dt || a.apex_field != b.apex_field || a.V0 != b.V0 || a.T0 != b.T0 ||
      a.work_function != b.work_function || a.w_min != b.w_min || a.w_max_units != b.w_max_units ||
      a.n_heat != b.n_heat || a.seed != b.seed)
    return bad("a physical parameter (dt, apex_field, V0, T0, work_function, w_min, w_max_units, n_heat, seed)");
  if (a.circuit_R != b.circuit_R || a.circuit_C != b.circuit_C) return bad("the circuit (circuit_R, circuit_C)");
  if (a.sigma_el_en != b.sigma_el_en || a.sigma_el_nn != b.sigma_el_nn || a.sigma_cx != b.sigma_cx ||
      a.coulomb_log != b.coulomb_log || a.merge_max != b.merge_max)
    return bad("a collision parameter (sigma_el_en, sigma_el_nn, sigma_cx, coulomb_log, merge_max)");
  if (F.nface != M.nface || F.nvox != M.nvox || F.nnode != M.nnode || F.ncell != M.ncell) return bad("the face or voxel count");
  if (F.mlp_params != M.mlp_params || F.mlp_bins != M.mlp_bins) return bad("the surrogate layout");
  return PIC_OK;
}

}  // namespace pic

using namespace pic;

extern "C" {

int pic_save(pic_t *h, const char *path) {
  if (!h || !path) return PIC_E_INVALID;
  PIC_TRY(check_device(h));
  for (int s = 0; s < PIC_NSPECIES; ++s)
    if (h->keys_valid[s])
      return pic_fail(h, PIC_E_INVALID, "pic_save: SPs were pushed but not yet sorted; save between steps or after pic_sort");
  DevClock c;
  PIC_CUDA(h, cudaMemcpyAsync(&c, h->clock, sizeof c, cudaMemcpyDeviceToHost, h->stream));
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  if (c.err) return pic_fail(h, PIC_E_INVALID, "pic_save: the device error flag is set");
  SaveHeader H;
  fill_header(h, H);
  fill_solve_diag(h, c, H);
  std::vector<float> master(pic_mlp_num_params());
  std::vector<uint8_t> binok(surrogate_bins());
  int trained = 0;
  PIC_TRY(surrogate_export(h, master.data(), binok.data(), &trained));
  H.has_mlp = 1;
  H.mlp_trained = trained;
  File F;
  F.f = fopen(path, "wb");
  if (!F.f) return pic_fail(h, PIC_E_INVALID, std::string("pic_save: cannot open ") + path);
  std::vector<char> buf;
  PIC_TRY(put(h, F.f, kMagic, sizeof kMagic));
  PIC_TRY(put(h, F.f, &H, sizeof H));
  PIC_TRY(put(h, F.f, &c, sizeof c));
  for (int s = 0; s < PIC_NSPECIES; ++s) {
    const int64_t n = c.n[s];
    const SpeciesBuf &a = h->sp[s].a;
    PIC_TRY(put_tag(h, F.f, tSpecies, (uint64_t)n * 36));
    for (const void *p : {(const void *)a.x, (const void *)a.y, (const void *)a.z, (const void *)a.vx,
                          (const void *)a.vy, (const void *)a.vz, (const void *)a.w})
      PIC_TRY(dev_to_file(h, F.f, p, (size_t)n * 4, buf));
    PIC_TRY(dev_to_file(h, F.f, a.id, (size_t)n * 8, buf));
    PIC_TRY(put_tag(h, F.f, tOffsets, (uint64_t)(h->ncell + 1) * 4));
    PIC_TRY(dev_to_file(h, F.f, h->sp[s].off, (size_t)(h->ncell + 1) * 4, buf));
    PIC_TRY(put_tag(h, F.f, tSortKeys, (uint64_t)c.n_sorted[s] * 4));
    PIC_TRY(dev_to_file(h, F.f, h->sp[s].skey, (size_t)c.n_sorted[s] * 4, buf));
  }
  PIC_TRY(put_tag(h, F.f, tPhi, (uint64_t)h->nnode * 8));
  PIC_TRY(dev_to_file(h, F.f, h->phi, (size_t)h->nnode * 8, buf));
  PIC_TRY(put_tag(h, F.f, tCharge, (uint64_t)h->nnode * 8));
  PIC_TRY(dev_to_file(h, F.f, h->Q, (size_t)h->nnode * 8, buf));
  if (h->phi_prev) {
    PIC_TRY(put_tag(h, F.f, tPhiPrev, (uint64_t)h->nnode * 8));
    PIC_TRY(dev_to_file(h, F.f, h->phi_prev, (size_t)h->nnode * 8, buf));
  }
  const Faces &fc = h->faces;
  PIC_TRY(put_tag(h, F.f, tFaces, (uint64_t)fc.n * 8 * 9));
  for (const void *p : {(const void *)fc.F, (const void *)fc.J, (const void *)fc.PN, (const void *)fc.acc_evap,
                        (const void *)fc.acc_heat, (const void *)fc.acc_charge, (const void *)fc.acc_sput,
                        (const void *)fc.acc_Eb, (const void *)fc.acc_Es})
    PIC_TRY(dev_to_file(h, F.f, p, (size_t)fc.n * 8, buf));
  PIC_TRY(put_tag(h, F.f, tTemp, (uint64_t)h->heat.nvox * 8));
  PIC_TRY(dev_to_file(h, F.f, h->heat.T, (size_t)h->heat.nvox * 8, buf));
  PIC_TRY(put_tag(h, F.f, tMlp, (uint64_t)master.size() * 4 + binok.size()));
  PIC_TRY(put(h, F.f, master.data(), master.size() * 4));
  PIC_TRY(put(h, F.f, binok.data(), binok.size()));
  PIC_TRY(put_tag(h, F.f, tEnd, 0));
  if (fflush(F.f) != 0) return pic_fail(h, PIC_E_INVALID, "pic_save: write failed");
  return PIC_OK;
}

int pic_load(pic_t *h, const char *path) {
  if (!h || !path) return PIC_E_INVALID;
  PIC_TRY(check_device(h));
  File F;
  F.f = fopen(path, "rb");
  if (!F.f) return pic_fail(h, PIC_E_INVALID, std::string("pic_load: cannot open ") + path);
  char magic[8];
  PIC_TRY(get(h, F.f, magic, sizeof magic));
  if (memcmp(magic, kMagic, sizeof magic) != 0) return pic_fail(h, PIC_E_INVALID, "pic_load: not a libpic state file");
  SaveHeader H, M;
  PIC_TRY(get(h, F.f, &H, sizeof H));
  if (H.version != kVersion || H.endian != 0x01020304u || H.header_bytes != sizeof(SaveHeader) ||
      H.clock_bytes != sizeof(DevClock))
    return pic_fail(h, PIC_E_INVALID, "pic_load: file version or layout differs from this library's");
  fill_header(h, M);
  PIC_TRY(compatible(h, H, M));
  DevClock c;
  PIC_TRY(get(h, F.f, &c, sizeof c));
  for (int s = 0; s < PIC_NSPECIES; ++s)
    if (c.n[s] < 0 || c.n[s] > h->sp[s].cap || c.n_sorted[s] < 0 || c.n_sorted[s] > c.n[s])
      return pic_fail(h, PIC_E_CAPACITY, "pic_load: species " + std::to_string(s) + " holds " + std::to_string(c.n[s]) +
                                             " SPs, more than this handle's capacity " + std::to_string(h->sp[s].cap));
  // from here the handle's state is being replaced: any failure leaves it unusable for stepping
  graph_invalidate(h);
  std::vector<char> buf;
  for (int s = 0; s < PIC_NSPECIES; ++s) {
    const int64_t n = c.n[s];
    const SpeciesBuf &a = h->sp[s].a;
    PIC_TRY(expect_tag(h, F.f, tSpecies, (uint64_t)n * 36));
    for (void *p : {(void *)a.x, (void *)a.y, (void *)a.z, (void *)a.vx, (void *)a.vy, (void *)a.vz, (void *)a.w})
      PIC_TRY(file_to_dev(h, F.f, p, (size_t)n * 4, buf));
    PIC_TRY(file_to_dev(h, F.f, a.id, (size_t)n * 8, buf));
    PIC_TRY(expect_tag(h, F.f, tOffsets, (uint64_t)(h->ncell + 1) * 4));
    PIC_TRY(file_to_dev(h, F.f, h->sp[s].off, (size_t)(h->ncell + 1) * 4, buf));
    PIC_TRY(expect_tag(h, F.f, tSortKeys, (uint64_t)c.n_sorted[s] * 4));
    PIC_TRY(file_to_dev(h, F.f, h->sp[s].skey, (size_t)c.n_sorted[s] * 4, buf));
    // the per-cell count table is zero between sorts
    PIC_CUDA(h, cudaMemsetAsync(h->sp[s].cnt, 0, (size_t)(h->ncell + 1) * 4, h->stream));
    h->keys_valid[s] = false;
  }
  PIC_TRY(expect_tag(h, F.f, tPhi, (uint64_t)h->nnode * 8));
  PIC_TRY(file_to_dev(h, F.f, h->phi, (size_t)h->nnode * 8, buf));
  PIC_TRY(expect_tag(h, F.f, tCharge, (uint64_t)h->nnode * 8));
  PIC_TRY(file_to_dev(h, F.f, h->Q, (size_t)h->nnode * 8, buf));
  if (H.has_prev) {
    PIC_TRY(expect_tag(h, F.f, tPhiPrev, (uint64_t)h->nnode * 8));
    if (!h->phi_prev) {
      h->phi_prev = (long long *)dalloc(h, (size_t)h->nnode * sizeof(long long));
      if (!h->phi_prev) return pic_fail(h, PIC_E_CUDA, "pic_load: phi_prev allocation failed");
    }
    PIC_TRY(file_to_dev(h, F.f, h->phi_prev, (size_t)h->nnode * 8, buf));
  } else if (h->phi_prev) {
    c.phi_prev_ok = 0;   // this handle's previous potential belongs to another run
  }
  const Faces &fc = h->faces;
  PIC_TRY(expect_tag(h, F.f, tFaces, (uint64_t)fc.n * 8 * 9));
  for (void *p : {(void *)fc.F, (void *)fc.J, (void *)fc.PN, (void *)fc.acc_evap, (void *)fc.acc_heat,
                  (void *)fc.acc_charge, (void *)fc.acc_sput, (void *)fc.acc_Eb, (void *)fc.acc_Es})
    PIC_TRY(file_to_dev(h, F.f, p, (size_t)fc.n * 8, buf));
  PIC_TRY(expect_tag(h, F.f, tTemp, (uint64_t)h->heat.nvox * 8));
  PIC_TRY(file_to_dev(h, F.f, h->heat.T, (size_t)h->heat.nvox * 8, buf));
  std::vector<float> master(pic_mlp_num_params());
  std::vector<uint8_t> binok(surrogate_bins());
  PIC_TRY(expect_tag(h, F.f, tMlp, (uint64_t)master.size() * 4 + binok.size()));
  PIC_TRY(get(h, F.f, master.data(), master.size() * 4));
  PIC_TRY(get(h, F.f, binok.data(), binok.size()));
  PIC_TRY(expect_tag(h, F.f, tEnd, 0));
  if (H.mlp_trained || surrogate_ready(h)) PIC_TRY(surrogate_import(h, master.data(), binok.data(), H.mlp_trained));
  c.err = 0;
  PIC_CUDA(h, cudaMemcpyAsync(h->clock, &c, sizeof c, cudaMemcpyHostToDevice, h->stream));
  h->V0 = H.V0;
  h->prm.flags = H.prm.flags;
  h->circuit_ready = H.circuit_ready != 0 && h->E0 != nullptr;
  // the next solve rewrites the Dirichlet values (the loaded potential already holds them, so the
  // rewrite changes no bit) and the anode plane under a circuit
  h->dirichlet_valid = false;
  h->anode_dirty = true;
  h->last_solve_graph = false;
  h->last_mg_cycles = H.last_mg_cycles;
  h->last_mg_res = H.last_mg_res;
  h->mg_cycles_host = H.mg_cycles_host;
  PIC_TRY(stage_efield(h));
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  return launch_check(h, "pic_load");
}

}  // extern "C"
