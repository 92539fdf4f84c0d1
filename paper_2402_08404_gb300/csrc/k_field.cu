// Poisson solve (eq:poi with eq:bcf1-3) by geometric multigrid and the node field E = -grad phi.
//
// Operator: (A u)_n = (6 u_n - sum of the 6 neighbours)/h^2 on free nodes, mirror images across
// the lateral walls (zero normal field), Dirichlet nodes on the z = 0 and z = nz planes and on
// every corner of a solid cell.  Charge density rho_n = Q_n e w_min 2^-30 / V_n with V_n = dx^3
// halved on each lateral wall the node lies on.
//
// Solve: refinement loop on the fixed-point potential -- t = h^2 (f - A phi) formed exactly in
// int64 (charge term Q K rounded once, see charge_fx), stop when ||r||/||f_lifted|| < tol, else
// one V-cycle on A e = r and phi += e rounded to the fixed-point grid.  The V-cycle runs in
// float32 (mixed form) or float64 (plain form): red-black Gauss-Seidel sweeps (3+3 by default), full-
// weighting restriction, trilinear prolongation, and a direct solve on the coarsest level (its
// inverse operator built at creation).  Coarse Dirichlet masks are injected from the fine nodes
// they coincide with.
//
// Layout: phi (fixed point, 2^-40 V), E and the fixed-point charge are node arrays in natural
// order.  The V-cycle levels keep their two colours apart: node (i, j, k) of colour
// c = (i + j + k) & 1 lives at c * nper + ((k (ny + 1) + j) Xh + (i >> 1)), Xh = (nx + 2) / 2.
// A colour sweep then reads the other colour and writes its own as contiguous rows, and its
// 6 neighbours of (i, j, k) sit at slots (i -+ 1) >> 1 of its own row and i >> 1 of the four
// rows around it, all in the other colour.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pic_internal.cuh"
#include "dev_common.cuh"

namespace pic {

// ---- natural-order helpers ---------------------------------------------------------
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
// Division by a fixed divisor d < 2^31 for numerators < 2^32: q = (umulhi(n, m) + n) >> s with
// s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1 (round-up reciprocal).
struct FastDiv {
  uint32_t m, s;
};
inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f{0, 0};
  while ((1ull << f.s) < d) ++f.s;
  f.m = (uint32_t)(((1ull << 32) * ((1ull << f.s) - d)) / d + 1);
  return f;
}
__device__ __forceinline__ uint32_t fdiv(uint32_t n, FastDiv f) {
  return (uint32_t)(((uint64_t)__umulhi(n, f.m) + n) >> f.s);
}

struct Lv {
  int nx, ny, nz, Xh;
  int64_t nper;
  uint32_t P;    // slots per plane and colour, (ny + 1) Xh
  FastDiv xd;    // division by Xh
  FastDiv pd;    // division by P
};

inline Lv lv_of(const MgLevel &L) {
  const uint32_t P = (uint32_t)((L.ny + 1) * L.Xh);
  return Lv{L.nx, L.ny, L.nz, L.Xh, L.nper, P, make_fastdiv((uint32_t)L.Xh), make_fastdiv(P)};
}

__host__ __device__ __forceinline__ int64_t srow(const Lv &L, int j, int k) {
  return ((int64_t)k * (L.ny + 1) + j) * L.Xh;
}

// split index of node (i, j, k)
__host__ __device__ __forceinline__ int64_t sidx(const Lv &L, int i, int j, int k) {
  return (int64_t)((i + j + k) & 1) * L.nper + srow(L, j, k) + (i >> 1);
}

// the same in 32-bit arithmetic (both colours of a level hold fewer than 2^32 slots, checked at
// creation): one index multiply-add chain instead of 64-bit ones
__device__ __forceinline__ uint32_t sidx32(const Lv &L, int i, int j, int k) {
  return (uint32_t)((i + j + k) & 1) * (uint32_t)L.nper + ((uint32_t)k * (uint32_t)(L.ny + 1) + (uint32_t)j) * (uint32_t)L.Xh +
         (uint32_t)(i >> 1);
}

// planes per thread in the level sweeps
constexpr int kKZ = 4;

// Level kernels index the slots of a plane flat (x: blocks of kSlotThreads slots, so no row
// tail leaves a warp mostly idle) and take kKZ planes per thread (y: plane groups x colours);
// j and t come from one division by Xh.
constexpr int kSlotThreads = 256;
inline dim3 flat_grid(const Lv &L, int colours, int planes_per_thread) {
  return dim3((L.P + kSlotThreads - 1) / kSlotThreads, ((L.nz + planes_per_thread) / planes_per_thread) * colours, 1);
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

// One colour of red-black Gauss-Seidel on A u = f.  Each thread takes slot q of KZ planes (chosen
// per level by the autotuner) and
// issues every load of all of them (right-hand side, mask, the six neighbours of the other
// colour) before its first store: nothing read in a colour pass is written in it, and every
// address is inside the level (mirrored at the lateral walls, unused slots clamp into the row),
// so the loads need not wait for the mask.  first = 1: the other colour is taken as zero (the
// first sweep after a new right-hand side), so the correction needs no clearing pass; Dirichlet
// slots of u hold 0 from creation and are never written.
template <typename T, bool first, int KZ>
__global__ void __launch_bounds__(kSlotThreads) k_smooth(T *u, const T *f, const uint8_t *dirs, Lv L, T h2, int c) {
  const uint32_t q = blockIdx.x * kSlotThreads + threadIdx.x;
  if (q >= L.P) return;
  const int j = (int)fdiv(q, L.xd), t = (int)(q - (uint32_t)j * (uint32_t)L.Xh);
  const int k0 = blockIdx.y * KZ;
  // one 64-bit base per array; every neighbour is a 32-bit offset from it (the integer pipe,
  // not the memory system, bounds this kernel once the loads are in flight)
  const size_t base = (size_t)k0 * L.P + q;
  const T *uo = u + (size_t)(c ^ 1) * L.nper + base;
  T *uc = u + (size_t)c * L.nper + base;
  const T *fc = f + (size_t)c * L.nper + base;
  const uint8_t *dc = dirs + (size_t)c * L.nper + base;
  const int P = (int)L.P;
  const int ojm = j > 0 ? -L.Xh : L.Xh, ojp = j < L.ny ? L.Xh : -L.Xh;
  // x-neighbour offsets (mirrored at the walls) for the two node parities along z; plane p has
  // parity par0 ^ (p & 1), known at compile time in the unrolled loop
  const int par0 = (j + k0 + c) & 1;
  int oxm[2], oxp[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int i = 2 * t + (par0 ^ e);
    const int im = i > 0 ? i - 1 : 1, ip = i < L.nx ? i + 1 : L.nx - 1;
    oxm[e] = (im >> 1) - t;
    oxp[e] = (ip >> 1) - t;
  }
  T v[KZ];
  uint8_t d[KZ];
#pragma unroll
  for (int p = 0; p < KZ; ++p) {
    const int k = k0 + p;
    v[p] = 0;
    d[p] = 1;
    if (k > 0 && k < L.nz) {   // the k = 0 and k = nz planes are Dirichlet
      const int o = p * P;
      d[p] = dc[o];
      if (first) {
        v[p] = h2 * fc[o];
      } else {
        v[p] = uo[o + oxm[p & 1]] + uo[o + oxp[p & 1]] + uo[o + ojm] + uo[o + ojp] + uo[o - P] + uo[o + P] +
               h2 * fc[o];
      }
    }
  }
#pragma unroll
  for (int p = 0; p < KZ; ++p)
    if (!d[p]) uc[p * P] = v[p] * (T)(1.0 / 6.0);
}

// r = f - A u at the colour-0 nodes.  The V-cycle's last pre-smoothing sweep updates colour 1,
// which leaves the colour-1 residual zero up to rounding (each colour-1 value solves its own row
// of A u = f), so colour 1 is neither evaluated nor stored: k_restrict reads colour 0 only.
// Grid y: plane groups of kKZ.
template <typename T>
__global__ void __launch_bounds__(kSlotThreads) k_residual(const T *u, const T *f, T *r, const uint8_t *dirs, Lv L,
                                                            T inv_h2) {
  const uint32_t q = blockIdx.x * kSlotThreads + threadIdx.x;
  if (q >= L.P) return;
  const int k0 = blockIdx.y * kKZ;
  const int j = (int)fdiv(q, L.xd), t = (int)(q - (uint32_t)j * (uint32_t)L.Xh);
  const T *uo = u + L.nper;
  const int64_t ojm = j > 0 ? -(int64_t)L.Xh : (int64_t)L.Xh, ojp = j < L.ny ? (int64_t)L.Xh : -(int64_t)L.Xh;
  // x-neighbour offsets of the two node parities along z (plane p: parity par0 ^ (p & 1))
  const int par0 = (j + k0) & 1;
  int oxm[2], oxp[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int i = 2 * t + (par0 ^ e);
    const int im = i > 0 ? i - 1 : 1, ip = i < L.nx ? i + 1 : L.nx - 1;
    oxm[e] = (im >> 1) - t;
    oxp[e] = (ip >> 1) - t;
  }
  T v[kKZ];
  uint8_t d[kKZ];
#pragma unroll
  for (int p = 0; p < kKZ; ++p) {
    const int k = k0 + p;
    v[p] = 0;
    d[p] = 1;
    if (k > 0 && k < L.nz) {
      const int64_t m = (int64_t)k * L.P + q;
      d[p] = dirs[m];
      const T nb = uo[m + oxm[p & 1]] + uo[m + oxp[p & 1]] + uo[m + ojm] + uo[m + ojp] + uo[m - L.P] + uo[m + L.P];
      v[p] = f[m] - (6 * u[m] - nb) * inv_h2;
    }
  }
#pragma unroll
  for (int p = 0; p < kKZ; ++p)
    if (k0 + p <= L.nz) r[(int64_t)(k0 + p) * L.P + q] = d[p] ? (T)0 : v[p];
}

__device__ __forceinline__ int mirror(int i, int n) { return i < 0 ? -i : (i > n ? 2 * n - i : i); }

// Full weighting of the fine residual onto the coarse right-hand side.  The fine residual is zero
// at colour-1 nodes (k_residual), and fine node (2I + di, 2J + dj, 2K + dk) has colour
// (di + dj + dk) & 1 (mirroring keeps parity), so only the 13 even offsets are read: the centre
// (weight 1/8) and the 12 with two nonzero components (1/32).  One coarse slot per thread, grid
// y: coarse planes x 2 colours.  Coarse Dirichlet nodes (all of the K = 0 and K = nz planes
// among them) return before any fine load.  The coarse correction needs no clearing.
template <typename TF, typename TC>
__global__ void __launch_bounds__(kSlotThreads) k_restrict(const TF *rf, Lv Fl, TC *fc, const uint8_t *dirsc, Lv Cl) {
  const uint32_t q = blockIdx.x * kSlotThreads + threadIdx.x;
  if (q >= Cl.P) return;
  const int cc = blockIdx.y & 1, K = blockIdx.y >> 1;
  const int J = (int)fdiv(q, Cl.xd), T = (int)(q - (uint32_t)J * (uint32_t)Cl.Xh);
  const int I = 2 * T + ((J + K + cc) & 1);
  if (I > Cl.nx) return;
  const int64_t n = (int64_t)cc * Cl.nper + (int64_t)K * Cl.P + q;
  if (dirsc[n]) { fc[n] = 0; return; }
  const int i0 = 2 * I, j0 = 2 * J, k0 = 2 * K;
  const int im = mirror(i0 - 1, Fl.nx), ip = mirror(i0 + 1, Fl.nx);
  const int jm = mirror(j0 - 1, Fl.ny), jp = mirror(j0 + 1, Fl.ny);
  // colour-0 fine values (all in the first half of the split layout)
#define RF(i, j, k) (TC) rf[srow(Fl, (j), (k)) + ((i) >> 1)]
  const TC ctr = RF(i0, j0, k0);
  const TC xy = RF(im, jm, k0) + RF(ip, jm, k0) + RF(im, jp, k0) + RF(ip, jp, k0);
  const TC xz = RF(im, j0, k0 - 1) + RF(ip, j0, k0 - 1) + RF(im, j0, k0 + 1) + RF(ip, j0, k0 + 1);
  const TC yz = RF(i0, jm, k0 - 1) + RF(i0, jp, k0 - 1) + RF(i0, jm, k0 + 1) + RF(i0, jp, k0 + 1);
#undef RF
  fc[n] = (TC)0.125 * ctr + (TC)0.03125 * ((xy + xz) + yz);
}

// Trilinear prolongation of the coarse correction, added on free fine nodes (flat fine slots,
// grid y: plane groups of kKZ x 2 colours).  Fine slot t of row j has i in {2t, 2t + 1}, so its
// coarse corners are columns t and t + 1 of rows j >> 1 and (j + 1) >> 1; the kKZ fine planes
// from an even kb share the coarse planes kb/2 .. kb/2 + 2.  The thread loads those 12 coarse
// values once (clamped into the level), then its fine values and masks, before any store.
template <typename TC, typename TF>
__global__ void __launch_bounds__(kSlotThreads) k_prolong(const TC *uc, Lv Cl, TF *uf, const uint8_t *dirsf, Lv Fl) {
  static_assert(kKZ == 4, "the plane pairing below assumes four fine planes per thread");
  const uint32_t q = blockIdx.x * kSlotThreads + threadIdx.x;
  if (q >= Fl.P) return;
  const int c = blockIdx.y & 1, kb = (blockIdx.y >> 1) * kKZ;
  const int j = (int)fdiv(q, Fl.xd), t = (int)(q - (uint32_t)j * (uint32_t)Fl.Xh);
  TF *ufc = uf + (int64_t)c * Fl.nper;
  const uint8_t *dc = dirsf + (int64_t)c * Fl.nper;
  const int t1 = min(t + 1, Cl.nx), j0 = j >> 1, j1 = j0 + (j & 1), Kb = kb >> 1;
  TC cv[3][4];   // coarse plane Kb + r: (t, j0), (t1, j0), (t, j1), (t1, j1)
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int K = min(Kb + r, Cl.nz);
    cv[r][0] = uc[sidx32(Cl, t, j0, K)];
    cv[r][1] = uc[sidx32(Cl, t1, j0, K)];
    cv[r][2] = uc[sidx32(Cl, t, j1, K)];
    cv[r][3] = uc[sidx32(Cl, t1, j1, K)];
  }
  TF v[kKZ];
  uint8_t d[kKZ];
#pragma unroll
  for (int p = 0; p < kKZ; ++p) {
    const int k = kb + p;
    d[p] = 1;
    v[p] = 0;
    if (k > 0 && k < Fl.nz) {
      const int64_t m = (int64_t)k * Fl.P + q;
      d[p] = dc[m];
      v[p] = ufc[m];
    }
  }
#pragma unroll
  for (int p = 0; p < kKZ; ++p) {
    const int k = kb + p;
    const bool odd = ((j + k + c) & 1) && 2 * t + 1 <= Fl.nx;   // fine i = 2t + 1: corners t and t + 1
    const int ra = p >> 1, rb = (p + 1) >> 1;                    // coarse planes k >> 1 and (k + 1) >> 1
    const TC a1 = odd ? cv[ra][1] : cv[ra][0], a3 = odd ? cv[ra][3] : cv[ra][2];
    const TC b1 = odd ? cv[rb][1] : cv[rb][0], b3 = odd ? cv[rb][3] : cv[rb][2];
    const TC s = (TC)0.125 * (cv[ra][0] + a1 + cv[ra][2] + a3 + cv[rb][0] + b1 + cv[rb][2] + b3);
    v[p] = v[p] + (TF)s;
  }
#pragma unroll
  for (int p = 0; p < kKZ; ++p)
    if (!d[p]) ufc[(int64_t)(kb + p) * Fl.P + q] = v[p];
}

// Direct solve on the coarsest level: u = A^-1 f over its free nodes, with the inverse (times
// h^2, transposed so that a warp reads consecutive rows of one column) built on the host at
// creation.  One block; f of the free nodes is staged in shared memory.
template <typename T>
__global__ void __launch_bounds__(1024) k_coarse_direct(T *u, const T *f, const T *ainvT, const int32_t *slot, int nf) {
  extern __shared__ unsigned char smem_raw[];
  T *fs = reinterpret_cast<T *>(smem_raw);
  for (int c = threadIdx.x; c < nf; c += blockDim.x) fs[c] = f[slot[c]];
  __syncthreads();
  for (int r = threadIdx.x; r < nf; r += blockDim.x) {
    T acc = 0;
    for (int c = 0; c < nf; ++c) acc += ainvT[(int64_t)c * nf + r] * fs[c];
    u[slot[r]] = acc;
  }
}

// ---- the coarse tail of the V-cycle in one thread-block cluster --------------------------------
// Levels from kTailNodes nodes down are too small to fill the GPU: each of their ~11 passes per
// V-cycle would be a short launch.  One cluster of kTailCtas CTAs runs the whole tail instead --
// pre-smoothing, residual and restriction level by level, the direct solve on the coarsest
// level, then prolongation and post-smoothing back up -- with the hardware cluster barrier
// (barrier.cluster arrive.release / wait.acquire, no spinning on flags) between passes, which
// also orders the global-memory writes of one pass before the reads of the next.  Each pass is
// the per-slot arithmetic of the level kernels above (k_smooth, k_residual, k_restrict,
// k_prolong) spread over the cluster's threads.
constexpr int kTailCtas = 8, kTailThreads = 1024, kMaxTail = 8;
constexpr int64_t kTailNodes = 80000;

template <typename T>
struct TailArgs {
  int nl;                           // levels in the tail; the last one is the coarsest
  int sweeps;                       // red-black sweeps before and after each coarse correction
  Lv lv[kMaxTail];
  T *u[kMaxTail], *f[kMaxTail], *r[kMaxTail];
  const uint8_t *dirs[kMaxTail];
  T h2[kMaxTail], inv_h2[kMaxTail];
  const T *ainv;                    // coarsest level: transposed inverse (times h^2), free slots
  const int32_t *cslot;
  int nf;
};

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}

// slot m (colour-array index over all planes) -> (t, j, k)
__device__ __forceinline__ void slot_tjk(const Lv &L, uint32_t m, int *t, int *j, int *k) {
  const uint32_t kk = fdiv(m, L.pd), q = m - kk * L.P;
  const uint32_t jj = fdiv(q, L.xd);
  *k = (int)kk;
  *j = (int)jj;
  *t = (int)(q - jj * (uint32_t)L.Xh);
}

template <typename T>
__device__ void tail_smooth(const TailArgs<T> &a, int l, int c, bool first, uint32_t g0, uint32_t gs) {
  const Lv &L = a.lv[l];
  T *u = a.u[l];
  const T *uo = u + (int64_t)(c ^ 1) * L.nper;
  const T *fc = a.f[l] + (int64_t)c * L.nper;
  const uint8_t *dc = a.dirs[l] + (int64_t)c * L.nper;
  const uint32_t n = (uint32_t)L.nper;
  for (uint32_t m = g0; m < n; m += gs) {
    int t, j, k;
    slot_tjk(L, m, &t, &j, &k);
    if (k == 0 || k == L.nz || dc[m]) continue;
    T v;
    if (first) {
      v = a.h2[l] * fc[m];
    } else {
      const int i = 2 * t + ((j + k + c) & 1);
      const int im = i > 0 ? i - 1 : 1, ip = i < L.nx ? i + 1 : L.nx - 1;
      const int64_t rb = (int64_t)m - t;
      const int64_t ojm = j > 0 ? -(int64_t)L.Xh : (int64_t)L.Xh, ojp = j < L.ny ? (int64_t)L.Xh : -(int64_t)L.Xh;
      v = uo[rb + (im >> 1)] + uo[rb + (ip >> 1)] + uo[m + ojm] + uo[m + ojp] + uo[m - L.P] + uo[m + L.P] +
          a.h2[l] * fc[m];
    }
    u[(int64_t)c * L.nper + m] = v * (T)(1.0 / 6.0);
  }
}

template <typename T>
__device__ void tail_residual(const TailArgs<T> &a, int l, uint32_t g0, uint32_t gs) {
  const Lv &L = a.lv[l];
  const T *u = a.u[l], *uo = u + L.nper, *f = a.f[l];
  T *r = a.r[l];
  const uint8_t *d = a.dirs[l];
  const uint32_t n = (uint32_t)L.nper;
  for (uint32_t m = g0; m < n; m += gs) {
    int t, j, k;
    slot_tjk(L, m, &t, &j, &k);
    T v = 0;
    if (k > 0 && k < L.nz && !d[m]) {
      const int i = 2 * t + ((j + k) & 1);
      const int im = i > 0 ? i - 1 : 1, ip = i < L.nx ? i + 1 : L.nx - 1;
      const int64_t rb = (int64_t)m - t;
      const int64_t ojm = j > 0 ? -(int64_t)L.Xh : (int64_t)L.Xh, ojp = j < L.ny ? (int64_t)L.Xh : -(int64_t)L.Xh;
      const T nb = uo[rb + (im >> 1)] + uo[rb + (ip >> 1)] + uo[m + ojm] + uo[m + ojp] + uo[m - L.P] + uo[m + L.P];
      v = f[m] - (6 * u[m] - nb) * a.inv_h2[l];
    }
    r[m] = v;
  }
}

template <typename T>
__device__ void tail_restrict(const TailArgs<T> &a, int l, uint32_t g0, uint32_t gs) {
  const Lv &Fl = a.lv[l], &Cl = a.lv[l + 1];
  const T *rf = a.r[l];
  T *fc = a.f[l + 1];
  const uint8_t *dc = a.dirs[l + 1];
  const uint32_t n = 2u * (uint32_t)Cl.nper;
  for (uint32_t m2 = g0; m2 < n; m2 += gs) {
    const int cc = m2 >= (uint32_t)Cl.nper ? 1 : 0;
    const uint32_t m = m2 - (cc ? (uint32_t)Cl.nper : 0u);
    int T_, J, K;
    slot_tjk(Cl, m, &T_, &J, &K);
    const int I = 2 * T_ + ((J + K + cc) & 1);
    if (I > Cl.nx) continue;
    if (dc[m2]) { fc[m2] = 0; continue; }
    const int i0 = 2 * I, j0 = 2 * J, k0 = 2 * K;
    const int im = mirror(i0 - 1, Fl.nx), ip = mirror(i0 + 1, Fl.nx);
    const int jm = mirror(j0 - 1, Fl.ny), jp = mirror(j0 + 1, Fl.ny);
#define RF(i, j, k) rf[srow(Fl, (j), (k)) + ((i) >> 1)]
    const T ctr = RF(i0, j0, k0);
    const T xy = RF(im, jm, k0) + RF(ip, jm, k0) + RF(im, jp, k0) + RF(ip, jp, k0);
    const T xz = RF(im, j0, k0 - 1) + RF(ip, j0, k0 - 1) + RF(im, j0, k0 + 1) + RF(ip, j0, k0 + 1);
    const T yz = RF(i0, jm, k0 - 1) + RF(i0, jp, k0 - 1) + RF(i0, jm, k0 + 1) + RF(i0, jp, k0 + 1);
#undef RF
    fc[m2] = (T)0.125 * ctr + (T)0.03125 * ((xy + xz) + yz);
  }
}

template <typename T>
__device__ void tail_prolong(const TailArgs<T> &a, int l, uint32_t g0, uint32_t gs) {
  const Lv &Fl = a.lv[l], &Cl = a.lv[l + 1];
  const T *uc = a.u[l + 1];
  T *uf = a.u[l];
  const uint8_t *df = a.dirs[l];
  const uint32_t n = 2u * (uint32_t)Fl.nper;
  for (uint32_t m2 = g0; m2 < n; m2 += gs) {
    const int c = m2 >= (uint32_t)Fl.nper ? 1 : 0;
    const uint32_t m = m2 - (c ? (uint32_t)Fl.nper : 0u);
    int t, j, k;
    slot_tjk(Fl, m, &t, &j, &k);
    if (k == 0 || k == Fl.nz || df[m2]) continue;
    const int i = min(2 * t + ((j + k + c) & 1), Fl.nx);
    const int i0 = i >> 1, j0 = j >> 1, k0 = k >> 1;
    const int i1 = i0 + (i & 1), j1 = j0 + (j & 1), k1 = k0 + (k & 1);
    const T s = (T)0.125 * (uc[sidx(Cl, i0, j0, k0)] + uc[sidx(Cl, i1, j0, k0)] + uc[sidx(Cl, i0, j1, k0)] +
                            uc[sidx(Cl, i1, j1, k0)] + uc[sidx(Cl, i0, j0, k1)] + uc[sidx(Cl, i1, j0, k1)] +
                            uc[sidx(Cl, i0, j1, k1)] + uc[sidx(Cl, i1, j1, k1)]);
    uf[m2] = uf[m2] + s;
  }
}

template <typename T>
__global__ void __cluster_dims__(kTailCtas, 1, 1) __launch_bounds__(kTailThreads, 1) k_vcycle_tail(TailArgs<T> a) {
  const uint32_t gs = kTailCtas * kTailThreads;
  const uint32_t g0 = cluster_rank() * kTailThreads + threadIdx.x;
  const int last = a.nl - 1;
  for (int l = 0; l < last; ++l) {
    for (int s = 0; s < a.sweeps; ++s)
      for (int c = 0; c < 2; ++c) {
        tail_smooth<T>(a, l, c, s == 0 && c == 0, g0, gs);
        cluster_sync_all();
      }
    tail_residual<T>(a, l, g0, gs);
    cluster_sync_all();
    tail_restrict<T>(a, l, g0, gs);
    cluster_sync_all();
  }
  // coarsest level: u = A^-1 f on its free nodes (rows spread over the cluster's threads)
  {
    const T *f = a.f[last];
    T *u = a.u[last];
    for (uint32_t rw = g0; rw < (uint32_t)a.nf; rw += gs) {
      T acc = 0;
      for (int c = 0; c < a.nf; ++c) acc += a.ainv[(int64_t)c * a.nf + rw] * f[a.cslot[c]];
      u[a.cslot[rw]] = acc;
    }
    cluster_sync_all();
  }
  for (int l = last - 1; l >= 0; --l) {
    tail_prolong<T>(a, l, g0, gs);
    cluster_sync_all();
    for (int s = 0; s < a.sweeps; ++s)
      for (int c = 1; c >= 0; --c) {
        tail_smooth<T>(a, l, c, false, g0, gs);
        cluster_sync_all();
      }
  }
}

// many red-black sweeps on the (small) coarsest level inside one block
template <typename T>
__global__ void k_coarse(T *u, const T *f, const uint8_t *dirs, Lv L, T h2, int sweeps) {
  const int64_t rows = (int64_t)(L.ny + 1) * (L.nz + 1);
  const int64_t slots = rows * L.Xh;
  for (int64_t q = threadIdx.x; q < 2 * L.nper; q += blockDim.x)
    if (!dirs[q]) u[q] = 0;
  __syncthreads();
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

// ---- fine level <-> fixed-point refinement ------------------------------------------------------
// Dirichlet values on the mask: phi = V0 on the anode plane, 0 elsewhere (V0 in fixed point)
__global__ void k_dirichlet(long long *phi, const uint8_t *dir, int nx, int ny, int nz, long long V0fx) {
  NODE_IJK(nx, ny)
  if (dir[n]) phi[n] = k == nz ? V0fx : 0;
}

// Anode plane (all Dirichlet nodes) at the circuit's gap voltage, rounded to the fixed-point grid.
__global__ void k_anode_plane(long long *phi, int nx, int ny, int nz, const double *V_gap) {
  const int64_t np = (int64_t)(nx + 1) * (ny + 1);
  const long long v = __double2ll_rn(*V_gap * kPhiScale);
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < np; q += (int64_t)gridDim.x * blockDim.x)
    phi[(int64_t)nz * np + q] = v;
}

// Unit Laplace field E0 = -grad(phi_L) / V_L of a zero-charge solution phi_L with the anode at
// V_L: central differences (one-sided on the z = 0 and z = nz planes, mirrored at the walls) in
// FP64 from the exact fixed-point differences, stored as float4 [1/m].
__global__ void k_unit_field(const long long *phi, float4 *E0, int nx, int ny, int nz, double c2, double c1) {
  NODE_IJK(nx, ny)
  const int64_t sy = nx + 1, sz = (int64_t)(nx + 1) * (ny + 1);
  const int im = i > 0 ? i - 1 : 1, ip = i < nx ? i + 1 : nx - 1;
  const int jm = j > 0 ? j - 1 : 1, jp = j < ny ? j + 1 : ny - 1;
  const int64_t row = (int64_t)k * sz + (int64_t)j * sy;
  float4 e;
  e.x = (float)((double)(phi[row + im] - phi[row + ip]) * c2);
  e.y = (float)((double)(phi[(int64_t)k * sz + (int64_t)jm * sy + i] - phi[(int64_t)k * sz + (int64_t)jp * sy + i]) * c2);
  if (k == 0) e.z = (float)((double)(phi[n] - phi[n + sz]) * c1);
  else if (k == nz) e.z = (float)((double)(phi[n - sz] - phi[n]) * c1);
  else e.z = (float)((double)(phi[n - sz] - phi[n + sz]) * c2);
  e.w = 0.f;
  E0[n] = e;
}

// Shockley-Ramo current of the charged SPs, I = sum Z e w w_min v . E0(x) (E0 gathered like E),
// over the SPs still in the domain (after a push: key != kDead; sorted SPs: w > 0).  Per-block
// partial sums in FP64 over a fixed grid of kRamoBlocks blocks (enough warps in flight to cover
// the gather latency on every SM), so the summation order, and with it every bit of the result,
// does not depend on anything but the SP order.
// Species in the order e-, Cu+, Cu2+ (nsp = 2 without Cu2+).
__global__ void __launch_bounds__(256) k_ramo_partial(SpeciesBuf e, SpeciesBuf ion, SpeciesBuf ion2,
                                                      const uint32_t *key_e, const uint32_t *key_i,
                                                      const uint32_t *key_j, int nsp, const float4 *E0, int nx, int ny,
                                                      const DevClock *clk, double qw, double *part) {
  __shared__ double sh[8];
  double acc = 0.0;
  for (int sp = 0; sp < nsp; ++sp) {
    const SpeciesBuf &p = sp == 0 ? e : (sp == 1 ? ion : ion2);
    const uint32_t *key = sp == 0 ? key_e : (sp == 1 ? key_i : key_j);
    const int64_t n = clk->n[sp == 0 ? PIC_ELECTRON : (sp == 1 ? PIC_ION : PIC_ION2)];
    const double z = sp == 0 ? -qw : (sp == 1 ? qw : 2.0 * qw);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      const int32_t w = p.w[i];
      if (w <= 0 || (key && key[i] == kDead)) continue;
      const float3 g = gather_E(E0, p.x[i], p.y[i], p.z[i], nx, ny);
      const float vdot = p.vx[i] * g.x + p.vy[i] * g.y + p.vz[i] * g.z;
      acc += z * (double)w * (double)vdot;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < 8; ++w) b += sh[w];
    part[blockIdx.x] = b;
  }
}

// I_gap from the partials (one block: runs of kRamoBlocks/256 partials, then a fixed tree), then
// one explicit Euler step of the RC circuit: I_tot = (V0 - V_gap)/R, V_gap += dt/C (I_tot - I_gap)
__global__ void __launch_bounds__(256) k_circuit(const double *part, DevClock *clk, double V0, double R, double Cg,
                                                 double dt) {
  __shared__ double sh[256];
  constexpr int kRun = kRamoBlocks / 256;
  double a = 0.0;
  for (int b = 0; b < kRun; ++b) a += part[threadIdx.x * kRun + b];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double I = sh[0];
  const double Itot = (V0 - clk->V_gap) / R;
  clk->I_gap = I;
  clk->I_tot = Itot;
  clk->V_gap = __dadd_rn(clk->V_gap, __dmul_rn(dt / Cg, Itot - I));   // no contraction: one rounding per operation
}

// Charge term of the right-hand side in the potential's fixed point: h^2 rho_n / eps0 in units
// of 2^-40 V equals Q_n K with K = e w_min 2^10 / (dx eps0) (2 per lateral wall the node lies
// on, from the halved node volume).  K is held as Kw = K 2^S (< 2^62) and the product is formed
// exactly in 128 bits and rounded once: (Q_n Kw + 2^(S-1)) >> S, 1 <= S <= 63.
__device__ __forceinline__ long long charge_fx(long long Qn, unsigned long long Kw, int S) {
  const unsigned long long lo = (unsigned long long)Qn * Kw;
  long long hi = __mul64hi(Qn, (long long)Kw);
  const unsigned long long r = lo + (1ull << (S - 1));
  hi += r < lo ? 1 : 0;
  return (long long)((r >> S) | ((unsigned long long)hi << (64 - S)));
}

// int64 -> float from its two 32-bit halves (the 32-bit conversions do not use the FP64 pipe):
// within 1.5 ulp of the correctly rounded value, all a V-cycle right-hand side or a norm needs.
__device__ __forceinline__ float fx_to_float(long long t) {
  return fmaf((float)(int)(t >> 32), 4294967296.0f, (float)(unsigned)t);
}
__device__ __forceinline__ float fx_to_level(long long t, float c) { return fx_to_float(t) * c; }   // CSE'd with tf
__device__ __forceinline__ double fx_to_level(long long t, double c) { return (double)t * c; }

// Residual of the discrete Poisson system in fixed point, t = h^2 (f - A phi) 2^40 = Q_n K -
// (6 phi_n - sum of neighbours): every term is an int64, so t is exact and no FP64 arithmetic is
// needed.  t 2^-40 / h^2 goes to the finest V-cycle level as its right-hand side (rounded to
// the level's type T, split-colour layout); the V-cycle starts from a zero correction (its first
// sweep).  The squared norms of h^2 r and of h^2 times the lifted right-hand side (only the
// plane below the anode carries a nonzero Dirichlet term) are accumulated in FP32 -- they only
// decide convergence.  3D launch with blocks (32, 8); block partials land at the block's
// linear id.
__device__ __forceinline__ long long nb_sum_fx(const long long *u, int i, int j, int k, int nx, int ny) {
  const int im = i > 0 ? i - 1 : 1, ip = i < nx ? i + 1 : nx - 1;
  const int jm = j > 0 ? j - 1 : 1, jp = j < ny ? j + 1 : ny - 1;
  const int64_t sy = nx + 1, sz = (int64_t)(nx + 1) * (ny + 1);
  const int64_t c = (int64_t)k * sz + (int64_t)j * sy;
  return u[c + im] + u[c + ip] + u[(int64_t)k * sz + (int64_t)jm * sy + i] + u[(int64_t)k * sz + (int64_t)jp * sy + i] +
         u[c - sz + i] + u[c + sz + i];
}

// kKZ planes per thread (grid z: plane groups): the centre column of phi is loaded once for the
// z differences of all of them, and every load is issued before the arithmetic (all addresses
// inside the grid; Dirichlet nodes, the k = 0 and k = nz planes among them, discard theirs).
// With E, the pass also writes the node field of this potential, by the arithmetic of k_efield
// from the same loads (the solve's last residual follows its last correction, so the field of
// the converged potential comes without another pass over phi).
template <typename T, int KZ, bool kE>
__global__ void __launch_bounds__(256) k_residual64(const long long *phi, const unsigned long long *Q,
                                                    unsigned long long Kfx, int S, int zero_charge, T *fl,
                                                    const uint8_t *dir, Lv L, T c_lvl, float V0f,
                                                    const double *V_anode, double *part,
                                                    int lift, float4 *E, float c2, float c1) {
  __shared__ float sh[2][8];
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y, k0 = blockIdx.z * KZ;
  if (V_anode) V0f = (float)*V_anode;   // the circuit's gap voltage
  float s = 0.f, sl = 0.f;
  if (i <= nx && j <= ny) {
    // 32-bit node offsets (a grid has fewer than 2^32 nodes, checked at creation)
    const int im = i > 0 ? i - 1 : 1, ip = i < nx ? i + 1 : nx - 1;
    const int jm = j > 0 ? j - 1 : 1, jp = j < ny ? j + 1 : ny - 1;
    const uint32_t sy = (uint32_t)(nx + 1), sz = (uint32_t)(nx + 1) * (uint32_t)(ny + 1);
    const uint32_t col = (uint32_t)j * sy + (uint32_t)i;
    const int32_t dxm = im - i, dxp = ip - i, dym = (jm - j) * (int32_t)sy, dyp = (jp - j) * (int32_t)sy;
    long long cz[KZ + 2];
#pragma unroll
    for (int p = 0; p < KZ + 2; ++p) cz[p] = phi[(uint32_t)min(max(k0 - 1 + p, 0), nz) * sz + col];
    long long side[KZ], exd[KZ], eyd[KZ];
    unsigned long long qv[KZ];
    uint8_t d[KZ];
#pragma unroll
    for (int p = 0; p < KZ; ++p) {
      const uint32_t c = (uint32_t)min(k0 + p, nz) * sz + col;
      d[p] = k0 + p <= nz ? dir[c] : 1;
      const long long pxm = phi[c + dxm], pxp = phi[c + dxp], pym = phi[c + dym], pyp = phi[c + dyp];
      side[p] = pxm + pxp + pym + pyp;
      if (kE) {
        exd[p] = pxm - pxp;
        eyd[p] = pym - pyp;
      }
      qv[p] = Q[c];
    }
    const int wall = (i == 0 || i == nx ? 1 : 0) + (j == 0 || j == ny ? 1 : 0);
    const unsigned long long Kw = Kfx << wall;
#pragma unroll
    for (int p = 0; p < KZ; ++p) {
      const int k = k0 + p;
      if (k > nz) break;
      long long t = 0, f = 0;
      if (!d[p]) {
        // most nodes carry no charge: the 128-bit product only where there is some
        f = (zero_charge || qv[p] == 0ull) ? 0 : charge_fx((long long)qv[p], Kw, S);
        t = f - (6 * cz[p + 1] - (side[p] + cz[p] + cz[p + 2]));
      }
      const float tf = fx_to_float(t);
      fl[sidx32(L, i, j, k)] = d[p] ? (T)0 : fx_to_level(t, c_lvl);
      if (kE) {
        const long long dz = k == 0 ? cz[p + 1] - cz[p + 2] : k == nz ? cz[p] - cz[p + 1] : cz[p] - cz[p + 2];
        float4 e;
        e.x = __fmul_rn(__ll2float_rn(exd[p]), c2);
        e.y = __fmul_rn(__ll2float_rn(eyd[p]), c2);
        e.z = __fmul_rn(__ll2float_rn(dz), k == 0 || k == nz ? c1 : c2);
        e.w = 0.f;
        E[(uint32_t)k * sz + col] = e;
      }
      const float rs = tf * 9.094947017729282e-13f;   // h^2 r = t 2^-40
      s += rs * rs;
      if (lift && !d[p]) {
        const float l = fx_to_float(f) * 9.094947017729282e-13f + (k == nz - 1 ? V0f : 0.f);
        sl += l * l;
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
__global__ void __launch_bounds__(256) k_efield(const long long *phi, float4 *E, int nx, int ny, int nz, float c2,
                                                float c1) {
  NODE_IJK(nx, ny)
  const int64_t sy = nx + 1, sz = (int64_t)(nx + 1) * (ny + 1);
  const int im = i > 0 ? i - 1 : 1, ip = i < nx ? i + 1 : nx - 1;
  const int jm = j > 0 ? j - 1 : 1, jp = j < ny ? j + 1 : ny - 1;
  const int64_t row = (int64_t)k * sz + (int64_t)j * sy;
  const long long dx = phi[row + im] - phi[row + ip];
  const long long dy = phi[(int64_t)k * sz + (int64_t)jm * sy + i] - phi[(int64_t)k * sz + (int64_t)jp * sy + i];
  const long long dz = k == 0 ? phi[n] - phi[n + sz] : k == nz ? phi[n - sz] - phi[n] : phi[n - sz] - phi[n + sz];
  float4 e;
  e.x = __fmul_rn(__ll2float_rn(dx), c2);
  e.y = __fmul_rn(__ll2float_rn(dy), c2);
  e.z = __fmul_rn(__ll2float_rn(dz), k == 0 || k == nz ? c1 : c2);
  e.w = 0.f;
  E[n] = e;
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
static const T *coarse_inv(pic_t *h);
template <>
const float *coarse_inv<float>(pic_t *h) { return h->coarse_inv_f; }
template <>
const double *coarse_inv<double>(pic_t *h) { return h->coarse_inv_d; }

template <typename T, int KZ>
static void smooth_kz(pic_t *h, MgLevel &L, const Lv &lv, T h2, int c, bool first) {
  const dim3 g = flat_grid(lv, 1, KZ);
  if (first) k_smooth<T, true, KZ><<<g, kSlotThreads, 0, h->stream>>>(lvl_u<T>(L), lvl_f<T>(L), L.dirs, lv, h2, c);
  else k_smooth<T, false, KZ><<<g, kSlotThreads, 0, h->stream>>>(lvl_u<T>(L), lvl_f<T>(L), L.dirs, lv, h2, c);
}

// one colour sweep on level l with its tuned planes per thread (1, 2, 4 or 8)
template <typename T>
static void smooth_launch(pic_t *h, MgLevel &L, const Lv &lv, T h2, int c, bool first, int kz) {
  switch (kz) {
    case 1: smooth_kz<T, 1>(h, L, lv, h2, c, first); break;
    case 2: smooth_kz<T, 2>(h, L, lv, h2, c, first); break;
    case 8: smooth_kz<T, 8>(h, L, lv, h2, c, first); break;
    default: smooth_kz<T, 4>(h, L, lv, h2, c, first); break;
  }
}

template <typename T>
static void smooth(pic_t *h, int l, MgLevel &L, const Lv &lv, T h2, int c, bool first) {
  ++h->nlaunch;
  KtScope kt_(h, first ? kidSmoothFirst : kidSmooth, (double)L.nper);
  smooth_launch<T>(h, L, lv, h2, c, first, h->tune_smooth_kz[l < 16 ? l : 15]);
}

// V-cycle on level l for A e = f_l, starting from e = 0: mg_sweeps red-black pre-sweeps (the
// first takes e = 0), residual, restriction, the coarser cycle, prolongation, mg_sweeps post-sweeps.
template <typename T>
static void vcycle(pic_t *h, int l) {
  MgLevel &L = h->mg[l];
  const Lv lv = lv_of(L);
  const T h2 = (T)(L.h * L.h), inv_h2 = (T)(1.0 / (L.h * L.h));
  const int last = (int)h->mg.size() - 1;
  if (l == h->tail_start && l < last) {   // the small levels in one cluster launch
    TailArgs<T> ta;
    ta.nl = last - l + 1;
    ta.sweeps = h->mg_sweeps;
    for (int q = 0; q < ta.nl; ++q) {
      MgLevel &M = h->mg[l + q];
      ta.lv[q] = lv_of(M);
      ta.u[q] = lvl_u<T>(M);
      ta.f[q] = lvl_f<T>(M);
      ta.r[q] = lvl_r<T>(M);
      ta.dirs[q] = M.dirs;
      ta.h2[q] = (T)(M.h * M.h);
      ta.inv_h2[q] = (T)(1.0 / (M.h * M.h));
    }
    ta.ainv = coarse_inv<T>(h);
    ta.cslot = h->coarse_slot;
    ta.nf = h->coarse_n;
    ++h->nlaunch;
    KtScope kt_(h, kidTail, (double)L.nnode);
    k_vcycle_tail<T><<<kTailCtas, kTailThreads, 0, h->stream>>>(ta);
    return;
  }
  if (l == last) {
    ++h->nlaunch;
    KtScope kt_(h, kidCoarse, (double)L.nnode);
    if (h->coarse_n > 0)
      k_coarse_direct<T><<<1, 1024, h->coarse_n * sizeof(T), h->stream>>>(lvl_u<T>(L), lvl_f<T>(L), coarse_inv<T>(h),
                                                                          h->coarse_slot, h->coarse_n);
    else
      k_coarse<T><<<1, 1024, 0, h->stream>>>(lvl_u<T>(L), lvl_f<T>(L), L.dirs, lv, h2, 60);
    return;
  }
  for (int s = 0; s < h->mg_sweeps; ++s)
    for (int c = 0; c < 2; ++c) smooth<T>(h, l, L, lv, h2, c, s == 0 && c == 0);
  ++h->nlaunch;
  { KtScope kt_(h, kidResidual, (double)L.nper); k_residual<T><<<flat_grid(lv, 1, kKZ), kSlotThreads, 0, h->stream>>>(lvl_u<T>(L), lvl_f<T>(L), lvl_r<T>(L), L.dirs, lv, inv_h2); }
  MgLevel &Cl = h->mg[l + 1];
  const Lv cv = lv_of(Cl);
  ++h->nlaunch;
  { KtScope kt_(h, kidRestrict, (double)Cl.nnode); k_restrict<T, T><<<flat_grid(cv, 2, 1), kSlotThreads, 0, h->stream>>>(lvl_r<T>(L), lv, lvl_f<T>(Cl), Cl.dirs, cv); }
  vcycle<T>(h, l + 1);
  ++h->nlaunch;
  { KtScope kt_(h, kidProlong, (double)L.nnode); k_prolong<T, T><<<flat_grid(lv, 2, kKZ), kSlotThreads, 0, h->stream>>>(lvl_u<T>(Cl), cv, lvl_u<T>(L), L.dirs, lv); }
  for (int s = 0; s < h->mg_sweeps; ++s)
    for (int c = 1; c >= 0; --c) smooth<T>(h, l, L, lv, h2, c, false);
}

// one V-cycle on A e = r (r already on the finest level) and phi += e
template <typename T>
static void cycle_fine(pic_t *h) {
  MgLevel &L = h->mg[0];
  vcycle<T>(h, 0);
  ++h->nlaunch;
  const dim3 g((L.nx + 1 + 31) / 32, (L.ny + 1 + 7) / 8, (L.nz + 1 + kKZ - 1) / kKZ);
  { KtScope kt_(h, kidCorrect, (double)L.nnode); k_correct<T><<<g, node_block(), 0, h->stream>>>(h->phi, lvl_u<T>(L), L.dir, lv_of(L)); }
}

static void efield_factors(const pic_t *h, float *c2, float *c1);

int stage_efield(pic_t *h) {
  ++h->nlaunch;
  float c2, c1;
  efield_factors(h, &c2, &c1);
  { KtScope kt_(h, kidEfield, (double)h->nnode); k_efield<<<node_grid3(h->nx, h->ny, h->nz), node_block(), 0, h->stream>>>(h->phi, h->E, h->nx, h->ny, h->nz, c2, c1); }
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

// The coarsest level's operator on its free nodes (6 on the diagonal, -1 per free neighbour,
// mirrored across the lateral walls, Dirichlet neighbours dropped), inverted on the host by
// Gauss-Jordan elimination with partial pivoting in FP64, for the direct coarse solve.  Levels
// with more than kCoarseDirectMax free nodes keep the sweeping solver.
constexpr int kCoarseDirectMax = 1024;
int mg_coarse_setup(pic_t *h) {
  MgLevel &L = h->mg.back();
  std::vector<uint8_t> dir(L.nnode);
  PIC_CUDA(h, cudaMemcpyAsync(dir.data(), L.dir, L.nnode, cudaMemcpyDeviceToHost, h->stream));
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  const Lv lv = lv_of(L);
  std::vector<int> id(L.nnode, -1);
  std::vector<int32_t> slot;
  for (int k = 0; k <= L.nz; ++k)
    for (int j = 0; j <= L.ny; ++j)
      for (int i = 0; i <= L.nx; ++i) {
        const int64_t n = node_index(i, j, k, L.nx, L.ny);
        if (dir[n]) continue;
        id[n] = (int)slot.size();
        slot.push_back((int32_t)sidx(lv, i, j, k));
      }
  const int nf = (int)slot.size();
  h->coarse_n = 0;
  if (nf == 0 || nf > kCoarseDirectMax) return PIC_OK;
  std::vector<double> A((size_t)nf * nf, 0.0), X((size_t)nf * nf, 0.0);
  for (int k = 0; k <= L.nz; ++k)
    for (int j = 0; j <= L.ny; ++j)
      for (int i = 0; i <= L.nx; ++i) {
        const int r = id[node_index(i, j, k, L.nx, L.ny)];
        if (r < 0) continue;   // free nodes have 0 < k < nz, so k -+ 1 stays inside
        A[(size_t)r * nf + r] = 6.0;
        const int nb[6][3] = {{i > 0 ? i - 1 : 1, j, k}, {i < L.nx ? i + 1 : L.nx - 1, j, k},
                              {i, j > 0 ? j - 1 : 1, k}, {i, j < L.ny ? j + 1 : L.ny - 1, k},
                              {i, j, k - 1}, {i, j, k + 1}};
        for (auto &q : nb) {
          const int c = id[node_index(q[0], q[1], q[2], L.nx, L.ny)];
          if (c >= 0) A[(size_t)r * nf + c] -= 1.0;
        }
      }
  for (int r = 0; r < nf; ++r) X[(size_t)r * nf + r] = 1.0;
  for (int col = 0; col < nf; ++col) {
    int piv = col;
    for (int r = col + 1; r < nf; ++r)
      if (fabs(A[(size_t)r * nf + col]) > fabs(A[(size_t)piv * nf + col])) piv = r;
    if (!(fabs(A[(size_t)piv * nf + col]) > 0)) return PIC_OK;   // singular: keep the sweeps
    if (piv != col)
      for (int c = 0; c < nf; ++c) {
        std::swap(A[(size_t)piv * nf + c], A[(size_t)col * nf + c]);
        std::swap(X[(size_t)piv * nf + c], X[(size_t)col * nf + c]);
      }
    const double inv = 1.0 / A[(size_t)col * nf + col];
    for (int c = 0; c < nf; ++c) { A[(size_t)col * nf + c] *= inv; X[(size_t)col * nf + c] *= inv; }
    for (int r = 0; r < nf; ++r) {
      if (r == col) continue;
      const double m = A[(size_t)r * nf + col];
      if (m == 0.0) continue;
      for (int c = 0; c < nf; ++c) {
        A[(size_t)r * nf + c] -= m * A[(size_t)col * nf + c];
        X[(size_t)r * nf + c] -= m * X[(size_t)col * nf + c];
      }
    }
  }
  // u = (A / h^2)^-1 f = h^2 A^-1 f, stored transposed
  const double h2 = L.h * L.h;
  std::vector<double> Td((size_t)nf * nf);
  std::vector<float> Tf((size_t)nf * nf);
  for (int r = 0; r < nf; ++r)
    for (int c = 0; c < nf; ++c) {
      Td[(size_t)c * nf + r] = h2 * X[(size_t)r * nf + c];
      Tf[(size_t)c * nf + r] = (float)Td[(size_t)c * nf + r];
    }
  h->coarse_inv_d = (double *)dalloc(h, Td.size() * sizeof(double));
  h->coarse_inv_f = (float *)dalloc(h, Tf.size() * sizeof(float));
  h->coarse_slot = (int32_t *)dalloc(h, slot.size() * sizeof(int32_t));
  if (!h->coarse_inv_d || !h->coarse_inv_f || !h->coarse_slot) return pic_fail(h, PIC_E_CUDA, "coarse solver allocation");
  PIC_CUDA(h, cudaMemcpyAsync(h->coarse_inv_d, Td.data(), Td.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  PIC_CUDA(h, cudaMemcpyAsync(h->coarse_inv_f, Tf.data(), Tf.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  PIC_CUDA(h, cudaMemcpyAsync(h->coarse_slot, slot.data(), slot.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                              h->stream));
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  h->coarse_n = nf;
  // the cluster tail takes every level from the first one of at most kTailNodes nodes down
  const int last = (int)h->mg.size() - 1;
  h->tail_start = -1;
  for (int l = 0; l < last; ++l)
    if (h->mg[l].nnode <= kTailNodes && last - l + 1 <= kMaxTail) { h->tail_start = l; break; }
  return PIC_OK;
}

// Autotuner probe for the smoother: on every level but the coarsest, time 4 colour sweeps of
// each planes-per-thread candidate (1, 2, 4, 8) on the level's FP32 arrays and keep the fastest.
// The sweeps only change the level's correction, which every solve rebuilds from zero.
int tune_smoother(pic_t *h, int *best, int cap) {
  const int cand[4] = {1, 2, 4, 8};
  cudaEvent_t e0, e1;
  PIC_CUDA(h, cudaEventCreate(&e0));
  PIC_CUDA(h, cudaEventCreate(&e1));
  const int nl = (int)h->mg.size() - 1;
  for (int l = 0; l < nl && l < 16; ++l) {
    MgLevel &L = h->mg[l];
    const Lv lv = lv_of(L);
    const float h2 = (float)(L.h * L.h);
    float best_ms = 1e30f;
    int pick = h->tune_smooth_kz[l];
    for (int kz : cand) {
      float t_min = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, h->stream);
        for (int c = 0; c < 4; ++c) smooth_launch<float>(h, L, lv, h2, c & 1, false, kz);
        cudaEventRecord(e1, h->stream);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        t_min = std::min(t_min, t);
      }
      if (t_min < best_ms) { best_ms = t_min; pick = kz; }
    }
    h->tune_smooth_kz[l] = pick;
    if (l < cap) best[l] = pick;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return launch_check(h, "tune smoother");
}

// Fixed-point charge scale and launch shape of the refinement (shared by both forms of the solve).
struct SolveSetup {
  unsigned long long Kfx;
  int S;
  double c_fx;
  bool mixed;
  float V0f;
  const double *V_anode;   // device gap voltage when the circuit drives the anode, else null
};

// Dirichlet values on phi for V0 (only when they changed) and the charge factor
// K = e w_min 2^10 / (dx eps0) as Kw = K 2^S in [2^59, 2^60].
static int solve_setup(pic_t *h, double V0, SolveSetup *ss) {
  MgLevel &L = h->mg[0];
  const long long V0fx = llrint(V0 * kPhiScale);
  const bool circ = circuit_on(h);
  if (!h->dirichlet_valid || h->dirichlet_V0fx != V0fx || (h->anode_dirty && !circ)) {
    if (h->capturing) return pic_fail(h, PIC_E_INVALID, "Dirichlet values must be set before graph capture");
    ++h->nlaunch;
    { KtScope kt_(h, kidDirichlet, (double)h->nnode); k_dirichlet<<<node_grid3(h->nx, h->ny, h->nz), node_block(), 0, h->stream>>>(h->phi, L.dir, h->nx, h->ny, h->nz, V0fx); }
    h->dirichlet_valid = true;
    h->dirichlet_V0fx = V0fx;
    h->anode_dirty = false;
  }
  if (circ) {   // the anode plane follows the circuit's gap voltage, every solve
    ++h->nlaunch;
    h->anode_dirty = true;
    k_anode_plane<<<grid_for((int64_t)(h->nx + 1) * (h->ny + 1)), kThreads, 0, h->stream>>>(h->phi, h->nx, h->ny, h->nz,
                                                                                           &h->clock->V_gap);
  }
  const double K = kQe * h->prm.w_min * 1024.0 / (h->dx * kEps0);
  const int S = 59 - (int)floor(log2(K));
  if (!(K > 0) || S < 1 || S > 63) return pic_fail(h, PIC_E_INVALID, "charge scale e w_min / (dx eps0) out of range");
  ss->Kfx = (unsigned long long)llround(ldexp(K, S));
  ss->S = S;
  ss->c_fx = 1.0 / (h->dx * h->dx) * kPhiUnit;
  ss->mixed = (h->prm.flags & PIC_F_MIXED_MG) != 0;
  ss->V0f = (float)V0;
  ss->V_anode = circ ? &h->clock->V_gap : nullptr;
  return PIC_OK;
}

// residual of the fixed-point system onto the finest level and its two norms in red_out (the
// planes per thread are the autotuner's, 1, 2 or 4)
// f32(1/(2 dx)) 2^-40 and f32(1/dx) 2^-40 of the node field: rounding then scaling by a power of two
static void efield_factors(const pic_t *h, float *c2, float *c1) {
  *c2 = (float)(1.0 / (2.0 * h->dx)) * (float)kPhiUnit;
  *c1 = (float)(1.0 / h->dx) * (float)kPhiUnit;
}

template <typename T, int KZ>
static void residual_kz(pic_t *h, const SolveSetup &ss, bool zero_charge, bool lift, bool efield, T *fl, T c_lvl,
                        double *part, int64_t *nb) {
  MgLevel &L = h->mg[0];
  const dim3 g((h->nx + 1 + 31) / 32, (h->ny + 1 + 7) / 8, (h->nz + KZ) / KZ);
  *nb = (int64_t)g.x * g.y * g.z;
  float c2, c1;
  efield_factors(h, &c2, &c1);
  if (efield)
    k_residual64<T, KZ, true><<<g, node_block(), 0, h->stream>>>(h->phi, h->Q, ss.Kfx, ss.S, zero_charge ? 1 : 0, fl,
                                                                 L.dir, lv_of(L), c_lvl, ss.V0f, ss.V_anode, part,
                                                                 lift ? 1 : 0, h->E, c2, c1);
  else
    k_residual64<T, KZ, false><<<g, node_block(), 0, h->stream>>>(h->phi, h->Q, ss.Kfx, ss.S, zero_charge ? 1 : 0, fl,
                                                                  L.dir, lv_of(L), c_lvl, ss.V0f, ss.V_anode, part,
                                                                  lift ? 1 : 0, nullptr, c2, c1);
}

template <typename T>
static int64_t residual_launch(pic_t *h, const SolveSetup &ss, bool zero_charge, bool lift, bool efield, T *fl,
                               T c_lvl) {
  int64_t nb = 0;
  // with the field, two planes per thread at most (four take ~95 registers)
  switch (efield ? std::min(h->tune_residual_kz, 2) : h->tune_residual_kz) {
    case 1: residual_kz<T, 1>(h, ss, zero_charge, lift, efield, fl, c_lvl, h->red, &nb); break;
    case 2: residual_kz<T, 2>(h, ss, zero_charge, lift, efield, fl, c_lvl, h->red, &nb); break;
    default: residual_kz<T, 4>(h, ss, zero_charge, lift, efield, fl, c_lvl, h->red, &nb); break;
  }
  return nb;
}

// efield: the pass also writes the node field of the current potential
static void residual_pass(pic_t *h, const SolveSetup &ss, bool zero_charge, bool lift, bool efield = false) {
  MgLevel &L = h->mg[0];
  ++h->nlaunch;
  int64_t nb;
  {
    KtScope kt_(h, kidResidual64, (double)h->nnode);
    nb = ss.mixed ? residual_launch<float>(h, ss, zero_charge, lift, efield, L.f, (float)ss.c_fx)
                  : residual_launch<double>(h, ss, zero_charge, lift, efield, L.fd, ss.c_fx);
  }
  h->nlaunch += 2;
  { KtScope kt_(h, kidNormSum, (double)nb); k_sum_stage1<<<kSumChunks, 256, 0, h->stream>>>(h->red, nb, h->red_mid); }
  k_sum_stage2<<<1, kSumChunks, 0, h->stream>>>(h->red_mid, h->red_out);
}

// Autotuner probe for the fixed-point residual: planes per thread 1, 2 or 4, each timed three
// times on the current potential and charge (it only rewrites the finest level's right-hand side
// and the norm partials, which every solve rebuilds); the fastest is kept.
int tune_residual(pic_t *h, int *best) {
  SolveSetup ss;
  PIC_TRY(solve_setup(h, h->V0, &ss));
  cudaEvent_t e0, e1;
  PIC_CUDA(h, cudaEventCreate(&e0));
  PIC_CUDA(h, cudaEventCreate(&e1));
  const int cand[3] = {1, 2, 4};
  float best_ms = 1e30f;
  int pick = h->tune_residual_kz;
  for (int kz : cand) {
    h->tune_residual_kz = kz;
    float t_min = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, h->stream);
      residual_pass(h, ss, false, false);
      cudaEventRecord(e1, h->stream);
      cudaEventSynchronize(e1);
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      t_min = std::min(t_min, t);
    }
    if (t_min < best_ms) { best_ms = t_min; pick = kz; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->tune_residual_kz = pick;
  *best = pick;
  return launch_check(h, "tune residual");
}

// Solve for phi with the current deposited charge (or none), anode at V0: refinement cycles
// until the relative residual reaches mg_tol, decided on the host after each residual.
int stage_solve(pic_t *h, bool zero_charge, double V0) {
  SolveSetup ss;
  PIC_TRY(solve_setup(h, V0, &ss));
  double norms[2] = {0, 0};
  double lifted = 0.0;
  // The residual pass after a correction also writes the field once this solve has run as many
  // cycles as the previous one (at least one): if the test then passes, that is the field of the
  // converged potential.  Earlier passes do not write it (a solve of many cycles would otherwise
  // write the field after each of them).
  const int field_from = std::max(h->last_mg_cycles, 1);
  for (int cyc = 0;; ++cyc) {
    const bool with_field = cyc >= field_from;
    residual_pass(h, ss, zero_charge, cyc == 0, with_field);
    PIC_CUDA(h, cudaMemcpyAsync(norms, h->red_out, sizeof norms, cudaMemcpyDeviceToHost, h->stream));
    PIC_CUDA(h, cudaStreamSynchronize(h->stream));
    if (cyc == 0) lifted = sqrt(norms[1]);
    const double rel = lifted > 0 ? sqrt(norms[0]) / lifted : sqrt(norms[0]);
    h->last_mg_res = rel;
    h->last_mg_cycles = cyc;
    h->last_solve_graph = false;
    if (rel <= h->prm.mg_tol) {
      h->mg_cycles_host += cyc;
      if (with_field) return launch_check(h, "solve");   // the field came with the last residual
      break;
    }
    if (cyc >= h->prm.mg_max_cycles) {
      PIC_TRY(stage_efield(h));
      return pic_fail(h, PIC_E_NOCONV, "Poisson solve: relative residual " + std::to_string(rel) + " after " +
                                           std::to_string(cyc) + " cycles");
    }
    if (ss.mixed) cycle_fine<float>(h);
    else cycle_fine<double>(h);
  }
  return stage_efield(h);
}

// Initial guess of a step's solve: phi <- 2 phi^n - phi^(n-1), exact in the fixed point (every
// |phi| < 2^53), and phi^(n-1) <- phi^n.  Without a previous potential it only records phi^n.
// Dirichlet values are unchanged by the extrapolation (the anode under a circuit is rewritten
// by the solve's set-up).
__global__ void k_extrapolate(long long *phi, long long *phi_prev, int64_t n, const DevClock *clk) {
  const bool ok = clk->phi_prev_ok != 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const long long p = phi[i];
    if (ok) phi[i] = 2 * p - phi_prev[i];
    phi_prev[i] = p;
  }
}

__global__ void k_set_prev_ok(DevClock *clk) { clk->phi_prev_ok = 1; }

int stage_extrapolate(pic_t *h) {
  if (!(h->prm.flags & PIC_F_EXTRAPOLATE)) return PIC_OK;
  if (!h->phi_prev) {
    if (h->capturing) return pic_fail(h, PIC_E_INVALID, "extrapolation buffer must exist before graph capture");
    h->phi_prev = (long long *)dalloc(h, (size_t)h->nnode * sizeof(long long));
    if (!h->phi_prev) return pic_fail(h, PIC_E_CUDA, "phi_prev allocation failed");
    PIC_CUDA(h, cudaMemsetAsync(&h->clock->phi_prev_ok, 0, sizeof(int), h->stream));
  }
  h->nlaunch += 2;
  k_extrapolate<<<h->nsm * 8, kThreads, 0, h->stream>>>(h->phi, h->phi_prev, h->nnode, h->clock);
  k_set_prev_ok<<<1, 1, 0, h->stream>>>(h->clock);
  return launch_check(h, "extrapolate");
}

bool circuit_on(pic_t *h) { return h->E0 != nullptr && h->circuit_ready && (h->prm.flags & PIC_F_CIRCUIT) != 0; }

// After a zero-charge solve with the anode at V_L: the unit Laplace field and the circuit's
// initial state (V_gap = V0, no current)
int circuit_setup(pic_t *h, double V_L) {
  const double c2 = kPhiUnit / (2.0 * h->dx * V_L), c1 = kPhiUnit / (h->dx * V_L);
  ++h->nlaunch;
  k_unit_field<<<node_grid3(h->nx, h->ny, h->nz), node_block(), 0, h->stream>>>(h->phi, h->E0, h->nx, h->ny, h->nz, c2, c1);
  return launch_check(h, "unit field");
}

int circuit_reset(pic_t *h) {
  const double st[3] = {h->V0, 0.0, 0.0};
  PIC_CUDA(h, cudaMemcpyAsync(&h->clock->V_gap, st, sizeof st, cudaMemcpyHostToDevice, h->stream));
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  h->circuit_ready = true;
  return PIC_OK;
}

// The circuit stage of a step: Shockley-Ramo current of the pushed SPs and the RC update.
int stage_circuit(pic_t *h) {
  if (!circuit_on(h)) return PIC_OK;
  const double qw = kQe * h->prm.w_min;
  h->nlaunch += 2;
  // after a push the keys mark the removed SPs; sorted SPs are all in the domain
  const uint32_t *ke = h->keys_valid[PIC_ELECTRON] ? h->sp[PIC_ELECTRON].key : nullptr;
  const uint32_t *ki = h->keys_valid[PIC_ION] ? h->sp[PIC_ION].key : nullptr;
  const uint32_t *kj = h->keys_valid[PIC_ION2] ? h->sp[PIC_ION2].key : nullptr;
  {
    KtScope kt_(h, kidRamo, 0);
    k_ramo_partial<<<kRamoBlocks, 256, 0, h->stream>>>(h->sp[PIC_ELECTRON].a, h->sp[PIC_ION].a, h->sp[PIC_ION2].a, ke, ki,
                                                       kj, nsp_active(h) > PIC_ION2 ? 3 : 2, h->E0, h->nx, h->ny,
                                                       h->clock, qw, h->ramo_part);
  }
  k_circuit<<<1, 256, 0, h->stream>>>(h->ramo_part, h->clock, h->V0, h->prm.circuit_R, h->prm.circuit_C, h->prm.dt);
  return launch_check(h, "circuit");
}

// Device-side convergence test of the graph form (one thread): first = 1 takes the lifted norm of
// this solve, otherwise one more cycle has run.  The graph's while node repeats (V-cycle,
// correction, residual, test) for as long as this sets its condition to 1; the cycle cap ends it
// with the no-convergence error bit.
__global__ void k_mg_check(const double *norms, DevClock *clk, double tol, int max_cycles, int first,
                           cudaGraphConditionalHandle cond) {
  if (first) {
    clk->mg_lifted = sqrt(norms[1]);
    clk->mg_cycles_last = 0;
  } else {
    clk->mg_cycles_last += 1;
    clk->mg_graph_cycles += 1;
  }
  const double Lf = clk->mg_lifted;
  const double rel = Lf > 0 ? sqrt(norms[0]) / Lf : sqrt(norms[0]);
  clk->mg_rel_last = (float)rel;
  bool more = !(rel <= tol);
  if (more && clk->mg_cycles_last >= max_cycles) {
    more = false;
    clk->err |= kErrNoconv;
  }
  cudaGraphSetConditional(cond, more ? 1u : 0u);
}

// The same solve recorded into the graph being captured on h->stream: residual and test, then a
// conditional while node whose body (captured on h->body_stream) is one refinement cycle and the
// next test.  The decision never leaves the device.
int stage_solve_graph(pic_t *h, double V0) {
  SolveSetup ss;
  PIC_TRY(solve_setup(h, V0, &ss));
  residual_pass(h, ss, false, true);
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  PIC_CUDA(h, cudaStreamGetCaptureInfo(h->stream, &st, nullptr, &g, &deps, nullptr, &nd));
  if (st != cudaStreamCaptureStatusActive) return pic_fail(h, PIC_E_INVALID, "graph solve outside a capture");
  cudaGraphConditionalHandle cond;
  PIC_CUDA(h, cudaGraphConditionalHandleCreate(&cond, g, 0, 0));
  ++h->nlaunch;
  k_mg_check<<<1, 1, 0, h->stream>>>(h->red_out, h->clock, h->prm.mg_tol, h->prm.mg_max_cycles, 1, cond);
  PIC_TRY(launch_check(h, "mg_check"));
  PIC_CUDA(h, cudaStreamGetCaptureInfo(h->stream, &st, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  PIC_CUDA(h, cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  PIC_CUDA(h, cudaStreamUpdateCaptureDependencies(h->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaStream_t outer = h->stream;
  h->stream = h->body_stream;
  const int64_t n0 = h->nlaunch;
  cudaError_t e = cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    if (ss.mixed) cycle_fine<float>(h);
    else cycle_fine<double>(h);
    residual_pass(h, ss, false, false);
    ++h->nlaunch;
    k_mg_check<<<1, 1, 0, h->stream>>>(h->red_out, h->clock, h->prm.mg_tol, h->prm.mg_max_cycles, 0, cond);
    cudaGraph_t tmp = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(h->stream, &tmp);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  h->graph_body_launches = h->nlaunch - n0;
  h->stream = outer;
  if (e != cudaSuccess) return pic_fail(h, PIC_E_CUDA, std::string("solve loop capture: ") + cudaGetErrorString(e));
  h->last_solve_graph = true;
  return stage_efield(h);
}

}  // namespace pic
