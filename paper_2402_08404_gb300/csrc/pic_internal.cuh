// Internal declarations of libpic: device state, launch helpers, Philox4x32-10.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pic.h"

namespace pic {

// ---- physical constants (CODATA 2018) ------------------------------------------------------
constexpr double kQe = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kAmu = 1.66053906660e-27;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kKb = 1.380649e-23;
constexpr double kHbar = 1.054571817e-34;
constexpr double kPi = 3.141592653589793;
constexpr double kMcu = 63.546 * kAmu;
constexpr double kXiCu = 7.726;      // eV, first ionization energy of Cu
constexpr double kXi2Cu = 20.292;    // eV, second ionization energy of Cu (Cu+ -> Cu2+)
constexpr double kEvap = 3.43;       // eV (Sec. 2.3.1)
constexpr double kTboil = 2835.0;    // K
constexpr double kPatm = 101325.0;   // Pa
constexpr double kLorentz = 2.0e-8;  // W Ohm K^-2 (Sec. 2.1)
constexpr double kNmax = 1e24;       // m^-3 (1e-6 per cubic Angstrom, Sec. 2.3.2)

constexpr uint32_t kDead = 0xFFFFFFFFu;
constexpr int kRamoBlocks = 2048;   // blocks (and FP64 partial sums) of the Shockley-Ramo sum
constexpr int kFracBits = 10;         // CIC fixed-point fraction bits per axis
constexpr int kSputBits = 24;         // sputter accumulator: atoms * 2^24
constexpr int kEnergyBits = 20;       // energy accumulators: eV * 2^20
// The potential is held in fixed point, phi [V] = n 2^-40 (int64 n): the 7-point stencil of the
// FP64 refinement and the node differences of E are then exact integer sums, and on this part
// integer adds run at 32x the FP64 rate.  |phi| < 2^13 V keeps n within the 53-bit mantissa, so
// every value and every difference converts to FP64 exactly.
constexpr int kPhiShift = 40;
constexpr double kPhiScale = 1099511627776.0;                  // 2^40
constexpr double kPhiUnit = 1.0 / 1099511627776.0;             // 2^-40
constexpr double kPhiMax = 8192.0;                             // |phi| bound [V]
constexpr int kMaxSegment = 32768;    // SPs of one species in one cell (sort fix-up limit: a block's
                                      // bitonic sort of the segment in 128 KB of shared memory)
constexpr int kLongCap = 1 << 16;     // queued long segments per sort pass
// emission surrogate output decoding: log10 J = approx_log10J + y0 kSurY0s (floor
// kSurLogJFloor), eps_N = y1 kSurY1s [eV]; output rows are kSurOut floats (y0, y1)
constexpr double kSurY0c = 0.0, kSurY0s = 1.0, kSurY1s = 2.0, kSurLogJFloor = -8.0;
constexpr int kSurOut = 2;

// Philox purposes (one key per purpose)
enum Purpose : uint32_t {
  kEmit = 1, kPair = 2, kIon = 3, kScat = 4, kDfi = 5, kEvapP = 6, kSput = 7,
  kPairEn = 8, kDrawEn = 9, kPairNn = 10, kDrawNn = 11, kPairCx = 12, kDrawCx = 13,   // elastic e-Cu, Cu-Cu, exchange
  kScatEn = 14, kScatNn = 15,
  kPairEe = 16, kDrawEe = 17, kPairEi = 18, kDrawEi = 19, kPairIi = 20, kDrawIi = 21,  // Coulomb
  kScat2 = 22, kPairIz = 23, kIonIz = 24, kScatIz = 25,       // Cu2+: double ionization, Cu+ ionization
  kPairEj = 26, kDrawEj = 27, kPairIj = 28, kDrawIj = 29, kPairJj = 30, kDrawJj = 31   // Coulomb with Cu2+
};

// device counters (int64), indices
enum Ctr {
  cEmitted = 0, cEvaporated, cSputtered, cImpactIon, cFieldIon, cRemovedE, cRemovedN, cRemovedI, cRemovedJ,
  cIonImpacts, cWevals, cSurFaces, cElasticEn, cElasticNn, cChargeEx, cCoulombEe, cCoulombEi, cCoulombIi, cMerged, cFbRange,
  cFbBin, cDoubleIon, cIonIon, cCoulombEj, cCoulombIj, cCoulombJj, cNum
};

// error bits set by kernels
enum ErrBits : int { kErrCapacity = 1, kErrSegment = 2, kErrTimeout = 4, kErrNan = 8, kErrNoconv = 16 };

struct DevClock {
  int64_t step;
  int64_t next_id;
  int64_t n[PIC_NSPECIES];          // SPs held per species
  int64_t n_sorted[PIC_NSPECIES];   // leading SPs covered by the last cell sort (per-cell offsets valid)
  int64_t n_new[PIC_NSPECIES];      // scratch: SPs created by the current pass
  int64_t ctr[cNum];
  int err;
  int phi_prev_ok;       // phi_prev holds the previous step's potential (time extrapolation)
  // graph form of the Poisson loop (device-side convergence test)
  int mg_cycles_last;       // cycles of the last solve
  float mg_rel_last;        // its relative residual
  double mg_lifted;         // norm of the lifted right-hand side of the current solve
  int64_t mg_graph_cycles;  // cycles run inside graphs since create (launch accounting)
  double V_gap, I_gap, I_tot;  // RC circuit: gap voltage [V], Shockley-Ramo gap current, circuit current [A]
};

struct SpeciesBuf {
  float *x, *y, *z, *vx, *vy, *vz;
  int32_t *w;
  uint64_t *id;
};

struct Species {
  int Z = 0;
  double mass = 0;
  int64_t cap = 0;
  float qmdt = 0.f;
  SpeciesBuf a{}, b{};        // current and scratch SoA buffers
  uint32_t *key = nullptr;    // cell key per SP (kDead when removed)
  uint32_t *perm = nullptr;   // sort permutation
  uint32_t *skey = nullptr;   // cell key at each sorted position (written by the scatter)
  uint32_t *cnt = nullptr;    // per-cell counts (zero between sorts), ncell+1
  uint32_t *off = nullptr;    // per-cell offsets of the last sort, ncell+1
};

struct MgLevel {
  int nx, ny, nz;             // cells
  int64_t nnode;
  int Xh;                     // slots per row and colour, (nx + 2) / 2
  int64_t nper;               // slots per colour, (nz + 1) (ny + 1) Xh
  double h;
  uint8_t *dir = nullptr;     // Dirichlet mask per node (natural order)
  uint8_t *dirs = nullptr;    // the same in the split-colour layout (2 nper; unused slots 1)
  float *u = nullptr, *f = nullptr, *r = nullptr;        // split-colour, 2 nper each
  double *ud = nullptr, *fd = nullptr, *rd = nullptr;   // FP64 V-cycle storage (plain form)
};

struct Faces {
  int64_t n = 0;
  int32_t *vcell = nullptr;   // vacuum cell (linear)
  int8_t *dir = nullptr;      // 0..5
  int32_t *owner = nullptr;   // solid cell or -1
  int32_t *owner_vox = nullptr;  // index of the owner in the solid-cell list or -1
  int64_t *key = nullptr;     // vcell*6+dir, ascending
  double *F = nullptr, *J = nullptr, *PN = nullptr;
  double *acc_evap = nullptr, *acc_heat = nullptr, *acc_charge = nullptr;
  int64_t *acc_sput = nullptr, *acc_Eb = nullptr, *acc_Es = nullptr;
  uint32_t *cnt = nullptr, *off = nullptr;   // per-face creation counts / offsets (n+1)
  uint32_t *cnt2 = nullptr, *off2 = nullptr;
  uint32_t *wu = nullptr, *wu2 = nullptr;    // injection weights of this pass
};

struct Heat {
  int64_t nvox = 0;
  int32_t *cell = nullptr;     // solid cell of voxel v
  int32_t *nbr = nullptr;      // 6 neighbour voxels per voxel (-1 none)
  uint8_t *base = nullptr;     // voxel on the k = 0 layer
  double *T = nullptr, *Tn = nullptr, *sig = nullptr, *kap = nullptr;
  double *src = nullptr, *cur = nullptr, *phiJ = nullptr, *joule = nullptr;
  double *p = nullptr, *q = nullptr, *res = nullptr, *zv = nullptr;
};

}  // namespace pic

struct pic_s {
  // configuration
  int nx = 0, ny = 0, nz = 0;
  double dx = 0;
  int64_t ncell = 0, nnode = 0;
  pic_geometry_t geo{};
  pic_params_t prm{};
  double V0 = 0;
  cudaStream_t stream = nullptr;
  pic_alloc_fn alloc = nullptr;
  pic_free_fn free_fn = nullptr;
  void *alloc_user = nullptr;
  std::vector<std::pair<void *, size_t>> allocations;
  std::string last_error;
  int nsm = 148;
  int device = -1;               // CUDA device current at pic_create; every later call must run there

  // device state
  uint8_t *solid = nullptr;      // per cell
  uint8_t *cheb = nullptr;       // per cell: Chebyshev distance to the nearest solid cell (capped)
  long long *phi = nullptr;      // per node, fixed point: phi [V] = phi * 2^-kPhiShift
  bool anode_dirty = false;      // the anode plane holds a circuit's V_gap instead of V0
  bool circuit_ready = false;    // the circuit state holds V_gap = V0 (set once the unit field exists)
  bool dirichlet_valid = false;  // phi holds the Dirichlet values of dirichlet_V0fx on the mask
  long long dirichlet_V0fx = 0;
  float4 *E = nullptr;           // per node
  long long *phi_prev = nullptr;  // per node: potential of the previous step (PIC_F_EXTRAPOLATE)
  float4 *E0 = nullptr;          // per node: unit Laplace field [1/m] (circuit; null without one)
  double *ramo_part = nullptr;   // Shockley-Ramo partial sums
  unsigned long long *Q = nullptr;  // per node, int64 two's complement charge
  pic::Species sp[PIC_NSPECIES];
  pic::Faces faces;
  pic::Heat heat;
  std::vector<pic::MgLevel> mg;
  int coarse_n = 0;                 // free nodes of the coarsest level (0: sweeping coarse solver)
  float *coarse_inv_f = nullptr;    // its inverse operator times h^2, transposed (nf x nf)
  double *coarse_inv_d = nullptr;
  int32_t *coarse_slot = nullptr;   // split-layout slot of each free node
  int tail_start = -1;              // first level of the cluster-launched V-cycle tail (-1: none)
  int *ev_hits = nullptr;             // collision events staged per unit of 256 work items
  uint64_t *ev_cnt = nullptr, *ev_off = nullptr;
  uint64_t *ev_cnt2 = nullptr, *ev_off2 = nullptr;   // second product kind per unit (double ionization)
  double sigma_el_en = 0, sigma_el_nn = 0, sigma_cx = 0;   // m^2 (elastic and exchange passes)
  int mg_sweeps = 3;                // red-black sweeps before and after each coarse correction
  pic::DevClock *clock = nullptr;
  // scratch
  void *scan_tmp = nullptr;      // block partials for scans
  uint64_t *pair_cnt = nullptr;  // staged collision events (item | payload << 32), one slot per work item
  double *red = nullptr;         // reduction partials
  double *red_out = nullptr;
  double *red_mid = nullptr;     // first-stage sums of the partials (2 x 128)
  int64_t *tmp_len = nullptr;    // device-side lengths for scans
  int2 *long_list = nullptr;     // sort: long cell segments queued for the block-level fix-up
  int2 *mid_list = nullptr;      // sort: 5..32-SP cell segments queued for the warp-level fix-up
  int64_t mid_cap = 0;
  int *long_n = nullptr;
  int *xq_n = nullptr;           // push: lengths of the per-species crosser queues
  bool fix_long_smem_set = false;  // k_fix_long's dynamic shared memory limit raised on this handle
  // state flags and last diagnostics
  bool keys_valid[PIC_NSPECIES] = {false, false, false, false};
  int last_mg_cycles = 0;
  int64_t mg_cycles_host = 0;       // refinement cycles of host-driven solves since create
  double last_mg_res = 0;
  float ms[8] = {0};
  int64_t solid_count = 0;
  int64_t nlaunch = 0;           // kernels launched by the library since create
  // graph form of the step (PIC_F_GRAPH): one captured graph per double-buffer parity
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  float *graph_a[2][PIC_NSPECIES] = {};  // S.a.x at capture
  bool graph_valid = false;
  uint32_t graph_flags = 0;              // flags the graphs were recorded with
  uint32_t eager_flags = 0xFFFFFFFFu;   // flags of the last eager step (none yet)
  int64_t graph_outer_launches = 0, graph_body_launches = 0;
  cudaStream_t body_stream = nullptr;   // capture stream of the Poisson loop body
  cudaStream_t cap_stream = nullptr;    // capture stream of the step graphs
  cudaStream_t copy_stream = nullptr;   // pic_load_all: host-to-device copies beside the sorts
  cudaEvent_t copy_ev[PIC_NSPECIES + 1] = {};   // [s]: species s copied; [PIC_NSPECIES]: the call's start
  bool capturing = false;               // stage code is being recorded into a graph
  bool last_solve_graph = false;        // the last solve ran in a graph (its diagnostics are on the device)
  // autotuned launch shapes
  int tune_particle_bps = 8;            // blocks per SM of the particle kernels (sort, push, deposit)
  int tune_residual_kz = 4;            // planes per thread of the fixed-point residual
  int tune_smooth_kz[16] = {4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4};  // planes per thread, by level
  // kernel timing (diagnostics): launches of the kernels in kt_mask are bracketed by event pairs
  uint64_t kt_mask = 0;
  std::vector<cudaEvent_t> kt_ev;                   // 2 per recorded launch, reused
  std::vector<cudaEvent_t> step_ev;                 // 8 per step of an eager pic_step call, reused
  std::vector<std::pair<int, double>> kt_pend;      // (kernel, units) per recorded launch
  double kt_ms[64] = {0}, kt_units[64] = {0};
  int64_t kt_n[64] = {0};
};

// Species the step works on: Cu2+ only while PIC_F_ION2 is set (without it Cu2+ SPs are not made,
// and any held stay as they are)
inline int nsp_active(const pic_t *h) { return (h->prm.flags & PIC_F_ION2) ? PIC_NSPECIES : 3; }

namespace pic {

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from the published rounds ----
struct U4 { uint32_t v[4]; };

__host__ __device__ inline U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)M0 * c0;
    uint64_t p1 = (uint64_t)M1 * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0; k1 += W1;
  }
  U4 o; o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
  return o;
}

// Stream (seed, purpose, ident, step): the 4 words of draw block `blk` (draws 4*blk..4*blk+3)
__host__ __device__ inline U4 rng_block(uint64_t seed, uint32_t purpose, uint64_t ident, int64_t step, uint32_t blk) {
  uint32_t k0 = (uint32_t)seed;
  uint32_t k1 = (uint32_t)(((seed >> 32) << 8) | purpose);
  return philox((uint32_t)ident, (uint32_t)(ident >> 32), (uint32_t)step, blk, k0, k1);
}

// U = ((w >> 8) + 0.5) 2^-24, exact in float and double
__host__ __device__ inline float u01f(uint32_t w) { return ((float)(w >> 8) + 0.5f) * 5.9604644775390625e-8f; }
__host__ __device__ inline double u01d(uint32_t w) { return ((double)(w >> 8) + 0.5) * 5.9604644775390625e-8; }
// floor(U * n) exactly: ((2 (w>>8) + 1) n) >> 25
__host__ __device__ inline uint32_t u_index(uint32_t w, uint32_t n) {
  return (uint32_t)(((2ull * (w >> 8) + 1ull) * (uint64_t)n) >> 25);
}
__device__ inline double uniform_draw(uint64_t seed, uint32_t purpose, uint64_t ident, int64_t step, uint32_t d) {
  U4 b = rng_block(seed, purpose, ident, step, d >> 2);
  return u01d(b.v[d & 3]);
}

// ---- launch helpers -----------------------------------------------------------------------
constexpr int kThreads = 256;
inline int grid_for(int64_t n, int threads = kThreads) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 1 << 20) g = 1 << 20;
  return (int)g;
}

__host__ __device__ inline int64_t node_index(int i, int j, int k, int nx, int ny) {
  return ((int64_t)k * (ny + 1) + j) * (nx + 1) + i;
}
__host__ __device__ inline int64_t cell_index(int i, int j, int k, int nx, int ny) {
  return ((int64_t)k * ny + j) * nx + i;
}

}  // namespace pic

// ---- kernel timing (host) -------------------------------------------------------------------
namespace pic {
// Kernels whose launches can be timed one by one (pic_set_kernel_timing); the order is the ABI's.
enum Kid : int {
  kidPush = 0, kidKeys, kidScatter, kidFixShort, kidFixMid, kidFixLong, kidGather, kidScanPartial, kidScanApply,
  kidDeposit, kidMccCount, kidMccProducts, kidElastic, kidCoulomb, kidMerge, kidDfiCount, kidDfiProducts, kidDirichlet, kidResidual64, kidNormSum,
  kidSmooth, kidSmoothFirst, kidResidual, kidRestrict, kidProlong, kidCoarse, kidTail, kidRamo, kidCorrect, kidEfield, kidFaceField,
  kidEmitSurrogate, kidEmitFallback, kidEmitCount, kidEmitWrite, kidInjectCount, kidInjectWrite, kidMlpForward,
  kidHeat, kidCross, kidNum
};
extern const char *const kKernelNames[kidNum];
// Records an event before the launches of its scope and one after them, on the library stream,
// when kernel `kid` is selected; `units` is the work of the launch (nodes, slots or faces; 0
// for particle kernels, whose counts live on the device).
struct KtScope {
  pic_t *h;
  int kid;
  double units;
  bool on;
  KtScope(pic_t *h_, int kid_, double units_);
  ~KtScope();
};
// Fold the finished event pairs into the per-kernel sums (the stream must have been synchronised).
void kt_collect(pic_t *h);
}  // namespace pic

// ---- error plumbing (host) ------------------------------------------------------------------
int pic_fail(pic_t *h, int code, const std::string &msg);
#define PIC_CUDA(h, call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return pic_fail((h), PIC_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define PIC_TRY(expr)            \
  do {                           \
    int rc_ = (expr);            \
    if (rc_ != PIC_OK) return rc_; \
  } while (0)

// ---- stage entry points implemented in the kernel files --------------------------------------
namespace pic {
void *dalloc(pic_t *h, size_t bytes);
void dfree(pic_t *h, void *p);
int launch_check(pic_t *h, const char *what);
// PIC_E_INVALID when the calling thread's current device is not the handle's device
int check_device(pic_t *h);

// scans (k_scan.cu): exclusive scans of n values; n either a host size or a device int64
int scan_u32(pic_t *h, const uint32_t *in, uint32_t *out, int64_t n, const int64_t *n_dev, uint32_t *total);
int scan_u64(pic_t *h, const uint64_t *in, uint64_t *out, int64_t n, const int64_t *n_dev, uint64_t *total);

// particles (k_particles.cu)
int stage_keys(pic_t *h, int s);
// deposit: clear the charge and add the pushed SPs' CIC charges in the push (the step's form)
int stage_push(pic_t *h, bool deposit = false);
int stage_sort(pic_t *h);
int stage_deposit(pic_t *h);
// collisions (k_collide.cu)
int stage_collide(pic_t *h);
// surface (k_surface.cu)
int stage_face_field(pic_t *h);
int stage_emit(pic_t *h);
int stage_inject(pic_t *h);
int emission_eval_dev(pic_t *h, const double *F, const double *T, const double *W, const double *R,
                      double *J, double *PN, int64_t n, bool fast);
// field (k_field.cu)
int stage_efield(pic_t *h);
int stage_solve(pic_t *h, bool zero_charge, double V0);
int stage_solve_graph(pic_t *h, double V0);
int graph_build_capture(pic_t *h);
void graph_invalidate(pic_t *h);   // drop recorded step graphs (buffers they hold may change)
int graph_launch_step(pic_t *h);
// autotuner probes: time the launch-shape candidates on the current state, keep the fastest
int tune_particles(pic_t *h, int *best);
int tune_smoother(pic_t *h, int *best, int cap);
int tune_residual(pic_t *h, int *best);
int face_field_mean(pic_t *h, const int64_t *faces, int nf, double *out);
int mg_coarse_setup(pic_t *h);
// RC circuit and Shockley-Ramo current (k_field.cu)
bool circuit_on(pic_t *h);
int circuit_setup(pic_t *h, double V_L);
int circuit_reset(pic_t *h);
int stage_circuit(pic_t *h);
int stage_extrapolate(pic_t *h);
// fix_charge: the push deposited this step's charge, merged pairs move theirs
int stage_merge(pic_t *h, bool fix_charge = false);
int sort_species(pic_t *h, int s);
int validate_loaded(pic_t *h, const SpeciesBuf &p, int64_t n);
// heat (k_heat.cu)
int stage_heat(pic_t *h);
// emission surrogate (k_mlp.cu)
bool surrogate_ready(pic_t *h);
void mlp_forget(pic_t *h);
int surrogate_faces(pic_t *h, const uint8_t **elig, const float **Y);
int surrogate_bins();
int surrogate_export(pic_t *h, float *master, uint8_t *binok, int *trained);
int surrogate_import(pic_t *h, const float *master, const uint8_t *binok, int trained);
// training GEMM on the tcgen05 tensor cores (k_mlp_tc.cu): C(M x 128) = A(M x K) B(K x 128), BF16
// operands (A(m, k) = A[m sam + k sak], B(k, n) = B[k sbk + n sbn]), FP32 result C(m, n) =
// C[m scm + n scn]; with splits > 1 the K range is split over CTAs and CTA z writes its partial
// row-major at C + z M 128 (summed afterwards in a fixed order); kper is set by gemm_tc
struct GemmTcArgs {
  const void *A;
  int64_t sam, sak;
  const void *B;
  int64_t sbk, sbn;
  float *C;
  int64_t scm, scn;
  int M, K, splits, kper;
};
int gemm_tc(pic_t *h, const GemmTcArgs &g);
// fused surrogate forward pass on the tcgen05 tensor cores (k_mlp_tc.cu); __nv_bfloat16 passed as void
int mlp_forward_tc(pic_t *h, const float *X, int64_t rows, const float *master, const struct __nv_bfloat16 *w2,
                   const struct __nv_bfloat16 *w3, float *Y);
}  // namespace pic
