// Particle kernels: gather + leapfrog push + boundary test (Sec. 2.2), stable cell sort,
// fixed-point CIC charge deposit (density of eq:poi).
//
// Push arithmetic is float32 with every operation rounded on its own (no fused multiply-add),
// in a fixed order: the new cell keys, boundary events and deposits are integer decisions
// taken from the pushed positions, so the order is part of the definition.
#include <algorithm>

#include "pic_internal.cuh"
#include "dev_common.cuh"

namespace pic {

enum Event { kEvNone = 0, kEvSolid = 1, kEvCathode = 2, kEvAnode = 3, kEvLateral = 4 };

// First event along p0 -> p1 (FP64 traversal of the crossed cells, ties x < y < z).
__device__ int first_event(const double p0[3], const double p1[3], const uint8_t *__restrict__ solid,
                           int nx, int ny, int nz, int64_t *vcell_out, int *dcode_out) {
  int c[3] = {(int)floor(p0[0]), (int)floor(p0[1]), (int)floor(p0[2])};
  // end cell clamped to [-1, n]: leaving the domain is an event before any clamped cell
  const int ce[3] = {(int)fmin(fmax(floor(p1[0]), -1.0), (double)nx), (int)fmin(fmax(floor(p1[1]), -1.0), (double)ny),
                     (int)fmin(fmax(floor(p1[2]), -1.0), (double)nz)};
  double d[3];
  for (int a = 0; a < 3; ++a) d[a] = __dsub_rn(p1[a], p0[a]);
  const int n[3] = {nx, ny, nz};
  int guard = abs(ce[0] - c[0]) + abs(ce[1] - c[1]) + abs(ce[2] - c[2]) + 3;
  while ((c[0] != ce[0] || c[1] != ce[1] || c[2] != ce[2]) && guard-- > 0) {
    int best = -1;
    double bt = 0.0;
    for (int a = 0; a < 3; ++a) {
      if (c[a] == ce[a]) continue;
      const int bnd = ce[a] > c[a] ? c[a] + 1 : c[a];
      const double t = __ddiv_rn(__dsub_rn((double)bnd, p0[a]), d[a]);
      if (best < 0 || t < bt) { best = a; bt = t; }
    }
    const int step = ce[best] > c[best] ? 1 : -1;
    const int64_t vcell = cell_index(c[0], c[1], c[2], nx, ny);
    c[best] += step;
    const int dcode = 2 * best + (step > 0 ? 1 : 0);
    if (c[best] < 0 || c[best] >= n[best]) {
      *vcell_out = vcell; *dcode_out = dcode;
      if (best == 2) return step < 0 ? kEvCathode : kEvAnode;
      return kEvLateral;
    }
    if (solid[cell_index(c[0], c[1], c[2], nx, ny)]) {
      *vcell_out = vcell; *dcode_out = dcode;
      return kEvSolid;
    }
  }
  return kEvNone;
}

__device__ int64_t face_lookup(const int64_t *__restrict__ keys, int64_t n, int64_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (keys[mid] < key) lo = mid + 1; else hi = mid;
  }
  return (lo < n && keys[lo] == key) ? lo : -1;
}

// Yamamura-type stand-in sputtering yield (the paper's fitted data is not available).
__device__ double sputter_yield(double E) {
  const double Q = 10.7, ETF = 11.9e3, Eth = 25.0;
  if (E <= Eth) return 0.0;
  const double eps = E / ETF, se = sqrt(eps);
  const double sn = 3.441 * se * log(eps + 2.718) / (1.0 + 6.355 * se + eps * (6.882 * se - 1.708));
  const double t = 1.0 - sqrt(Eth / E);
  return Q * sn * (t * t * sqrt(t));
}

struct PushArgs {
  SpeciesBuf p;
  uint32_t *key, *cnt;
  const float4 *E;
  const uint8_t *solid, *cheb;
  int nx, ny, nz;
  float qmdt, dtdx;
  int charged, ion, species;
  double mass, w_min;
  const int64_t *face_key;
  int64_t nface;
  unsigned long long *acc_sput, *acc_Eb;
  DevClock *clk;
  unsigned long long *Q;   // charge deposit of the pushed SPs (null: no deposit)
  int Z;                   // charge number of the species
  uint32_t *xq;            // queue of SPs whose move may cross the tip or the domain boundary
  int *xq_n;               // its length
};

// The rare path of the push (an SP whose move may reach a solid cell or leave the domain): the
// FP64 cell traversal and, for an ion that hits the tip or the cathode, the sputter and
// bombardment accumulators of the face it hits.  Returns true when the SP is removed.
__device__ bool crosser_event(const PushArgs &a, float x, float y, float z, float x1, float y1, float z1,
                              float vx, float vy, float vz, int32_t w) {
  const double p0[3] = {(double)x, (double)y, (double)z};
  const double p1[3] = {(double)x1, (double)y1, (double)z1};
  int64_t vcell = -1;
  int dcode = -1;
  const int ev = first_event(p0, p1, a.solid, a.nx, a.ny, a.nz, &vcell, &dcode);
  if (ev == kEvNone) return false;
  if (a.ion && (ev == kEvSolid || ev == kEvCathode)) {
    const int64_t f = face_lookup(a.face_key, a.nface, vcell * 6 + dcode);
    if (f >= 0) {
      const double v2 = __dadd_rn(__dadd_rn(__dmul_rn((double)vx, (double)vx), __dmul_rn((double)vy, (double)vy)),
                                  __dmul_rn((double)vz, (double)vz));
      const double energy = 0.5 * a.mass * v2 / kQe;
      const double ww = (double)w * a.w_min;
      atomicAdd(&a.acc_sput[f], (unsigned long long)(int64_t)floor(ww * sputter_yield(energy) * 16777216.0));
      atomicAdd(&a.acc_Eb[f], (unsigned long long)(int64_t)floor(ww * energy * 1048576.0));
      atomicAdd((unsigned long long *)&a.clk->ctr[cIonImpacts], 1ull);
    }
  }
  return true;
}

// Cloud-in-cell weights of a position (cell units) with quantised fractions: the lower corner's
// node index and q = floor(frac 2^F) per axis, packed as qx | qy << 10 | qz << 20.
__device__ __forceinline__ uint32_t cic_corner(float x, float y, float z, int nx, int ny, uint32_t *qpack) {
  const float fi = floorf(x), fj = floorf(y), fk = floorf(z);
  const float one = (float)(1 << kFracBits);
  const uint32_t qx = (uint32_t)floorf(__fsub_rn(x, fi) * one);
  const uint32_t qy = (uint32_t)floorf(__fsub_rn(y, fj) * one);
  const uint32_t qz = (uint32_t)floorf(__fsub_rn(z, fk) * one);
  *qpack = qx | (qy << 10) | (qz << 20);
  return (uint32_t)node_index((int)fi, (int)fj, (int)fk, nx, ny);
}

// The 8 node charges Z w prod(W) of one SP (int64, exact): corner c = dx + 2 dy + 4 dz.
// The 8 weight products W = prod over the axes of (2^F - q) or q, corner c = dx + 2 dy + 4 dz
// (each below 2^30, exact in 32 bits).
__device__ __forceinline__ void cic_weights(uint32_t qpack, uint32_t W[8]) {
  const uint32_t one = 1u << kFracBits;
  const uint32_t qx = qpack & 1023u, qy = (qpack >> 10) & 1023u, qz = qpack >> 20;
  const uint32_t a00 = (one - qz) * (one - qy), a10 = (one - qz) * qy, a01 = qz * (one - qy), a11 = qz * qy;
  W[0] = a00 * (one - qx); W[1] = a00 * qx; W[2] = a10 * (one - qx); W[3] = a10 * qx;
  W[4] = a01 * (one - qx); W[5] = a01 * qx; W[6] = a11 * (one - qx); W[7] = a11 * qx;
}

// The 8 node charges Z w W of one SP (int64, exact).
__device__ __forceinline__ void cic_charges(uint32_t qpack, int32_t zw, long long c[8]) {
  uint32_t W[8];
  cic_weights(qpack, W);
#pragma unroll
  for (int q = 0; q < 8; ++q) c[q] = (long long)zw * (long long)W[q];
}

__device__ __forceinline__ void cic_global(unsigned long long *Q, uint32_t base, uint32_t qpack, int32_t zw, int nx,
                                           int ny) {
  long long c[8];
  cic_charges(qpack, zw, c);
  const int64_t sy = nx + 1, sz = (int64_t)(nx + 1) * (ny + 1);
#pragma unroll
  for (int q = 0; q < 8; ++q)
    if (c[q] != 0) atomicAdd(Q + base + (q & 1) + ((q >> 1) & 1) * sy + (q >> 2) * sz, (unsigned long long)c[q]);
}

// Leapfrog of one SP from its position and the (optional) field at x^n.
__device__ __forceinline__ void leapfrog(float qmdt, float dtdx, float3 e, bool charged, float &x, float &y, float &z,
                                         float &vx, float &vy, float &vz) {
  if (charged) {
    vx = __fadd_rn(vx, __fmul_rn(qmdt, e.x));
    vy = __fadd_rn(vy, __fmul_rn(qmdt, e.y));
    vz = __fadd_rn(vz, __fmul_rn(qmdt, e.z));
  }
  x = __fadd_rn(x, __fmul_rn(vx, dtdx));
  y = __fadd_rn(y, __fmul_rn(vy, dtdx));
  z = __fadd_rn(z, __fmul_rn(vz, dtdx));
}

// Cell of the pushed position and whether the move stays clear of the tip and the walls: an SP
// that stays in its cell, or moves m cells (Chebyshev) from a cell at Chebyshev distance > m from
// every solid cell while staying inside, cannot meet a boundary.  Returns 0 clear (cell in *c),
// 1 possible crosser, 2 non-finite position (removed).
__device__ __forceinline__ int move_class(const PushArgs &a, float x, float y, float z, float x1, float y1, float z1,
                                          uint32_t *c) {
  if (!(isfinite(x1) && isfinite(y1) && isfinite(z1))) return 2;
  const int i0 = (int)floorf(x), j0 = (int)floorf(y), k0 = (int)floorf(z);
  const int i1 = (int)fminf(fmaxf(floorf(x1), -1.f), (float)a.nx);
  const int j1 = (int)fminf(fmaxf(floorf(y1), -1.f), (float)a.ny);
  const int k1 = (int)fminf(fmaxf(floorf(z1), -1.f), (float)a.nz);
  if (i1 != i0 || j1 != j0 || k1 != k0) {
    const int m = max(abs(i1 - i0), max(abs(j1 - j0), abs(k1 - k0)));
    const bool inside = i1 >= 0 && i1 < a.nx && j1 >= 0 && j1 < a.ny && k1 >= 0 && k1 < a.nz;
    if (!(inside && (int)a.cheb[cell_index(i0, j0, k0, a.nx, a.ny)] > m)) return 1;
  }
  *c = (uint32_t)cell_index(i1, j1, k1, a.nx, a.ny);
  return 0;
}

// count of the SP's new cell: lanes of a warp with the same cell add their count with one atomic
__device__ __forceinline__ void count_cell(uint32_t *cnt, uint32_t c, bool on) {
  const unsigned grp = __match_any_sync(0xffffffffu, on ? c : kDead);
  if (on && (int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&cnt[c], (uint32_t)__popc(grp));
}

// append the lanes with `on` to the crosser queue (one atomic per warp)
__device__ __forceinline__ void enqueue(const PushArgs &a, int64_t i, bool on) {
  const unsigned bal = __ballot_sync(0xffffffffu, on);
  if (!bal) return;
  const int lane = threadIdx.x & 31, leader = __ffs(bal) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(a.xq_n, __popc(bal));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (on) a.xq[base + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)i;
}

// Push of the neutral species (ballistic, no field, no charge).
__global__ void __launch_bounds__(256) k_push_neutral(PushArgs a) {
  const int64_t n = a.clk->n[a.species];
  int removed = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {   // warp-uniform trip count
    const int64_t i = i0 + threadIdx.x;
    const int32_t w = i < n ? a.p.w[i] : 0;
    bool clear = false, cross = false;
    uint32_t c = kDead;
    if (w > 0) {
      float x = a.p.x[i], y = a.p.y[i], z = a.p.z[i];
      float vx = a.p.vx[i], vy = a.p.vy[i], vz = a.p.vz[i];
      const float x0 = x, y0 = y, z0 = z;
      leapfrog(0.f, a.dtdx, make_float3(0.f, 0.f, 0.f), false, x, y, z, vx, vy, vz);
      const int cls = move_class(a, x0, y0, z0, x, y, z, &c);
      clear = cls == 0;
      cross = cls == 1;
      if (!cross) { a.p.x[i] = x; a.p.y[i] = y; a.p.z[i] = z; }
      if (cls == 2) ++removed;
    }
    if (i < n && !clear && !cross) a.key[i] = kDead;
    if (clear) a.key[i] = c;
    count_cell(a.cnt, c, clear);
    enqueue(a, i, cross);
  }
  for (int o = 16; o > 0; o >>= 1) removed += __shfl_down_sync(0xffffffffu, removed, o);
  if ((threadIdx.x & 31) == 0 && removed)
    atomicAdd((unsigned long long *)&a.clk->ctr[cRemovedE + a.species], (unsigned long long)removed);
}

// Push of a charged species, one SP per thread in the SPs' device order (cell-sorted by the last
// sort, apart from the SPs created since): field gather at x^n, leapfrog, and the move's class.
// SPs whose move may meet the tip or a wall are left to k_cross (velocity written, position
// kept).  With kDep the CIC charges of the pushed SPs are added to a.Q: lanes of a warp whose new
// lower corner is the same node (neighbours in the cell order) sum their 8 charges with a
// segmented shuffle scan and the last lane of each run issues the atomics.  The charges are exact
// integers, so the grouping changes no bit.  (Per-run warp reductions on 21-bit limbs were
// measured twice as slow: the runs are reduced one after another.)  (Staging the field and the charge of a tile of SPs
// in shared-memory windows was measured slower: the barriers between the phases of a tile cost
// more than the L1 and L2 traffic they save.)
template <bool kDep>
__global__ void __launch_bounds__(256, 4) k_push_charged(PushArgs a) {
  const int64_t n = a.clk->n[a.species];
  const int lane = threadIdx.x & 31;
  int removed = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
    const int64_t i = i0 + threadIdx.x;
    const int32_t w = i < n ? a.p.w[i] : 0;
    bool clear = false, cross = false;
    uint32_t c = kDead, base = kDead, qp = 0;
    if (w > 0) {
      const float x = a.p.x[i], y = a.p.y[i], z = a.p.z[i];
      float vx = a.p.vx[i], vy = a.p.vy[i], vz = a.p.vz[i];
      const float3 e = gather_E(a.E, x, y, z, a.nx, a.ny);
      float x1 = x, y1 = y, z1 = z;
      leapfrog(a.qmdt, a.dtdx, e, true, x1, y1, z1, vx, vy, vz);
      a.p.vx[i] = vx; a.p.vy[i] = vy; a.p.vz[i] = vz;
      const int cls = move_class(a, x, y, z, x1, y1, z1, &c);
      clear = cls == 0;
      cross = cls == 1;
      if (!cross) { a.p.x[i] = x1; a.p.y[i] = y1; a.p.z[i] = z1; }
      if (cls == 2) ++removed;
      if (clear && kDep) base = cic_corner(x1, y1, z1, a.nx, a.ny, &qp);
    }
    if (i < n && !clear && !cross) a.key[i] = kDead;
    if (clear) a.key[i] = c;
    count_cell(a.cnt, c, clear);
    enqueue(a, i, cross);
    if (kDep) {
      long long cc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      if (base != kDead) cic_charges(qp, a.Z * w, cc);
      const uint32_t prev = __shfl_up_sync(0xffffffffu, base, 1);
      const uint32_t next = __shfl_down_sync(0xffffffffu, base, 1);
      const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != base);
      if (heads != 0xffffffffu) {   // segmented inclusive scan, as many rounds as the longest run needs
        const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
        const int maxrun = (int)__reduce_max_sync(0xffffffffu, (unsigned)(lane - start + 1));
        for (int off = 1; off < maxrun; off <<= 1) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const long long v = __shfl_up_sync(0xffffffffu, cc[q], off);
            if (lane - off >= start) cc[q] += v;
          }
        }
      }
      if (base != kDead && (lane == 31 || next != base)) {
        const int64_t sy = a.nx + 1, sz = (int64_t)(a.nx + 1) * (a.ny + 1);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (cc[q] != 0) atomicAdd(a.Q + base + (q & 1) + ((q >> 1) & 1) * sy + (q >> 2) * sz, (unsigned long long)cc[q]);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) removed += __shfl_down_sync(0xffffffffu, removed, o);
  if (lane == 0 && removed)
    atomicAdd((unsigned long long *)&a.clk->ctr[cRemovedE + a.species], (unsigned long long)removed);
}

// The queued crossers of a push: the same float32 move from the kept position and the pushed
// velocity, then the FP64 traversal decides removal (and records ion impacts); survivors get
// their key, count and (with a.Q) charge.
__global__ void __launch_bounds__(256) k_cross(PushArgs a) {
  const int nq = *a.xq_n;
  int removed = 0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    const uint32_t i = a.xq[q];
    const float x = a.p.x[i], y = a.p.y[i], z = a.p.z[i];
    const float vx = a.p.vx[i], vy = a.p.vy[i], vz = a.p.vz[i];
    const int32_t w = a.p.w[i];
    const float x1 = __fadd_rn(x, __fmul_rn(vx, a.dtdx));
    const float y1 = __fadd_rn(y, __fmul_rn(vy, a.dtdx));
    const float z1 = __fadd_rn(z, __fmul_rn(vz, a.dtdx));
    a.p.x[i] = x1; a.p.y[i] = y1; a.p.z[i] = z1;
    if (crosser_event(a, x, y, z, x1, y1, z1, vx, vy, vz, w)) {
      a.key[i] = kDead;
      ++removed;
      continue;
    }
    const uint32_t c = (uint32_t)cell_index((int)floorf(x1), (int)floorf(y1), (int)floorf(z1), a.nx, a.ny);
    a.key[i] = c;
    atomicAdd(&a.cnt[c], 1u);
    if (a.Q) {
      uint32_t qp;
      const uint32_t b = cic_corner(x1, y1, z1, a.nx, a.ny, &qp);
      cic_global(a.Q, b, qp, a.Z * w, a.nx, a.ny);
    }
  }
  for (int o = 16; o > 0; o >>= 1) removed += __shfl_down_sync(0xffffffffu, removed, o);
  if ((threadIdx.x & 31) == 0 && removed)
    atomicAdd((unsigned long long *)&a.clk->ctr[cRemovedE + a.species], (unsigned long long)removed);
}

// Keys without a push (after loading): cell of each SP, kDead for w <= 0.
__global__ void k_keys(SpeciesBuf p, uint32_t *key, uint32_t *cnt, int nx, int ny, const DevClock *clk, int s) {
  const int64_t n = clk->n[s];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (p.w[i] <= 0) { key[i] = kDead; continue; }
    const uint32_t c = (uint32_t)cell_index((int)floorf(p.x[i]), (int)floorf(p.y[i]), (int)floorf(p.z[i]), nx, ny);
    key[i] = c;
    atomicAdd(&cnt[c], 1u);
  }
}

// Counting-sort scatter.  Each warp takes 32 consecutive SPs; lanes with the same cell key form
// a group (__match_any_sync) whose leader reserves the group's places with one atomic, and the
// group fills them in input order.  The input is the previous step's sorted order (SPs rarely
// change cell), so most cells get all their SPs from one group and come out already in stable
// order; the fix-up below only sorts segments that did not.
__global__ void k_scatter(const uint32_t *__restrict__ key, uint32_t *cnt, const uint32_t *__restrict__ off,
                          uint32_t *perm, uint32_t *skey, const DevClock *clk, int s) {
  const int64_t n = clk->n[s];
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; i0 < n; i0 += warps * 32) {
    const int64_t i = i0 + lane;
    const uint32_t k = i < n ? key[i] : kDead;
    const unsigned grp = __match_any_sync(0xffffffffu, k);
    const int leader = __ffs(grp) - 1;
    const int size = __popc(grp), rank = __popc(grp & ((1u << lane) - 1u));
    uint32_t base = 0;
    if (lane == leader && k != kDead) base = atomicSub(&cnt[k], (uint32_t)size) - (uint32_t)size;
    base = __shfl_sync(0xffffffffu, base, leader);
    if (k != kDead) {
      const uint32_t pos = off[k] + base + (uint32_t)rank;
      perm[pos] = (uint32_t)i;
      skey[pos] = k;
    }
  }
}

// Restore source order inside every cell segment that the scatter left unsorted.  Segment heads
// come from the sorted keys (a position whose key differs from its left neighbour's); the
// length is found by reading on in the keys (off[] only past 32).  Unsorted segments of up to
// 4 SPs are sorted in registers by their head thread; 5 to 32 are queued for k_fix_mid (one
// warp each), longer ones for k_fix_long (one block each).
__global__ void k_fix_short(const uint32_t *__restrict__ skey, const uint32_t *__restrict__ off, uint32_t *perm,
                            int64_t ncell, int2 *mid_list, int *mid_n, int mid_cap, int2 *long_list, int *long_n,
                            int long_cap, DevClock *clk) {
  const int64_t n = off[ncell];
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = skey[s];
    if (s > 0 && skey[s - 1] == k) continue;
    int len = 1;
    while (len <= 32 && s + len < n && skey[s + len] == k) ++len;
    if (len > 32) len = (int)(off[k + 1] - (uint32_t)s);
    if (len <= 1) continue;
    if (len <= 4) {
      uint32_t v[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) v[a] = a < len ? perm[s + a] : 0xFFFFFFFFu;
      if (v[0] < v[1] && (len < 3 || v[1] < v[2]) && (len < 4 || v[2] < v[3])) continue;   // already in order
      // sorting network for 4 (pads sort last)
#define PIC_CSWAP(a, b) { const uint32_t lo = min(v[a], v[b]), hi = max(v[a], v[b]); v[a] = lo; v[b] = hi; }
      PIC_CSWAP(0, 1) PIC_CSWAP(2, 3) PIC_CSWAP(0, 2) PIC_CSWAP(1, 3) PIC_CSWAP(1, 2)
#undef PIC_CSWAP
#pragma unroll
      for (int a = 0; a < 4; ++a)
        if (a < len) perm[s + a] = v[a];
    } else if (len <= 32) {
      bool sorted = true;
      uint32_t prev = perm[s];
      for (int a = 1; a < len && sorted; ++a) {
        const uint32_t v = perm[s + a];
        sorted = prev < v;
        prev = v;
      }
      if (sorted) continue;
      const int q = atomicAdd(mid_n, 1);
      if (q < mid_cap) mid_list[q] = make_int2((int)s, len);
      else atomicOr(&clk->err, kErrSegment);
    } else if (len <= kMaxSegment) {
      const int q = atomicAdd(long_n, 1);
      if (q < long_cap) long_list[q] = make_int2((int)s, len);
      else atomicOr(&clk->err, kErrSegment);
    } else {
      atomicOr(&clk->err, kErrSegment);
    }
  }
}

// one warp per queued segment of 5..32 SPs: lane l holds element l, its rank is the number of
// smaller elements (the original indices are distinct), and it stores itself at that rank
__global__ void k_fix_mid(uint32_t *perm, const int2 *mid_list, const int *mid_n, int mid_cap) {
  const int lane = threadIdx.x & 31;
  const int nq = min(*mid_n, mid_cap);
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nq; q += warps) {
    const int2 seg = mid_list[q];
    const uint32_t v = lane < seg.y ? perm[seg.x + lane] : 0xFFFFFFFFu;
    int rank = 0;
    for (int m = 0; m < 32; ++m) {
      const uint32_t o = __shfl_sync(0xffffffffu, v, m);
      rank += o < v ? 1 : 0;
    }
    __syncwarp();
    if (lane < seg.y) perm[seg.x + rank] = v;
  }
}

// One block per queued segment (33..kMaxSegment SPs): bitonic sort of the permutation values in
// dynamic shared memory (kMaxSegment words).
__global__ void __launch_bounds__(1024) k_fix_long(uint32_t *perm, const int2 *long_list, const int *long_n, int long_cap) {
  extern __shared__ uint32_t sh[];
  const int nl = min(*long_n, long_cap);
  for (int q = blockIdx.x; q < nl; q += gridDim.x) {
    const int2 seg = long_list[q];
    int P = 1;
    while (P < seg.y) P <<= 1;
    for (int t = threadIdx.x; t < P; t += blockDim.x) sh[t] = t < seg.y ? perm[seg.x + t] : 0xFFFFFFFFu;
    __syncthreads();
    for (int kk = 2; kk <= P; kk <<= 1) {
      for (int jj = kk >> 1; jj > 0; jj >>= 1) {
        for (int t = threadIdx.x; t < P; t += blockDim.x) {
          const int ixj = t ^ jj;
          if (ixj > t) {
            const bool up = (t & kk) == 0;
            const uint32_t a = sh[t], b = sh[ixj];
            if ((a > b) == up) { sh[t] = b; sh[ixj] = a; }
          }
        }
        __syncthreads();
      }
    }
    for (int t = threadIdx.x; t < seg.y; t += blockDim.x) perm[seg.x + t] = sh[t];
    __syncthreads();
  }
}

// dst[s] = src[perm[s]] for every field; each thread takes kGatherItems positions spaced by the
// grid stride and issues all of their loads before the stores
constexpr int kGatherItems = 4;
__global__ void k_gather(SpeciesBuf src, SpeciesBuf dst, const uint32_t *__restrict__ perm, const uint32_t *off,
                         int64_t ncell) {
  const int64_t n = off[ncell];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s0 < n; s0 += stride * kGatherItems) {
    uint32_t q[kGatherItems];
#pragma unroll
    for (int u = 0; u < kGatherItems; ++u) q[u] = s0 + u * stride < n ? perm[s0 + u * stride] : 0u;
    float x[kGatherItems], y[kGatherItems], z[kGatherItems], vx[kGatherItems], vy[kGatherItems], vz[kGatherItems];
    int32_t w[kGatherItems];
    uint64_t id[kGatherItems];
#pragma unroll
    for (int u = 0; u < kGatherItems; ++u) {
      if (s0 + u * stride < n) {
        x[u] = src.x[q[u]]; y[u] = src.y[q[u]]; z[u] = src.z[q[u]];
        vx[u] = src.vx[q[u]]; vy[u] = src.vy[q[u]]; vz[u] = src.vz[q[u]];
        w[u] = src.w[q[u]]; id[u] = src.id[q[u]];
      }
    }
#pragma unroll
    for (int u = 0; u < kGatherItems; ++u) {
      const int64_t s = s0 + u * stride;
      if (s < n) {
        dst.x[s] = x[u]; dst.y[s] = y[u]; dst.z[s] = z[u];
        dst.vx[s] = vx[u]; dst.vy[s] = vy[u]; dst.vz[s] = vz[u];
        dst.w[s] = w[u]; dst.id[s] = id[u];
      }
    }
  }
}

__global__ void k_set_count(DevClock *clk, int s, const uint32_t *off, int64_t ncell) {
  clk->n[s] = off[ncell];
  clk->n_sorted[s] = off[ncell];
}

// Cloud-in-cell deposit with quantised fractions: q = floor(frac(x) 2^F), weights 2^F - q on
// the lower node and q on the upper node per axis; Z w prod(W) added as int64 (exact, order-free).
// The SPs are cell-sorted, so lanes of a warp that share a cell sit next to each other: such a
// run of lanes adds its 8 contributions up with a segmented shuffle scan and only its last lane
// issues the (nonzero) atomics -- the sums are exact integers, so the grouping changes no bit.
__global__ void __launch_bounds__(256) k_deposit(SpeciesBuf p, int Z, unsigned long long *Q, int nx, int ny,
                                                 const DevClock *clk, int s) {
  const int64_t n = clk->n[s];
  const int64_t sy = nx + 1, sz = (int64_t)(nx + 1) * (ny + 1);
  const int one = 1 << kFracBits;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < n; i0 += stride) {
    const int64_t i = i0 + lane;
    int64_t base = -1;
    long long c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int32_t w = i < n ? p.w[i] : 0;
    if (w > 0) {
      const float x = p.x[i], y = p.y[i], z = p.z[i];
      const float fi = floorf(x), fj = floorf(y), fk = floorf(z);
      const int qx = (int)floorf(__fsub_rn(x, fi) * (float)one);
      const int qy = (int)floorf(__fsub_rn(y, fj) * (float)one);
      const int qz = (int)floorf(__fsub_rn(z, fk) * (float)one);
      base = (int64_t)fk * sz + (int64_t)fj * sy + (int64_t)fi;
      const int64_t zw = (int64_t)Z * w;
      const int64_t wx0 = one - qx, wy0 = one - qy, wz0 = one - qz;
      const int64_t a00 = zw * wz0 * wy0, a10 = zw * wz0 * qy, a01 = zw * qz * wy0, a11 = zw * qz * qy;
      c[0] = a00 * wx0; c[1] = a00 * qx; c[2] = a10 * wx0; c[3] = a10 * qx;
      c[4] = a01 * wx0; c[5] = a01 * qx; c[6] = a11 * wx0; c[7] = a11 * qx;
    }
    const int64_t prev = __shfl_up_sync(0xffffffffu, base, 1);
    const int64_t next = __shfl_down_sync(0xffffffffu, base, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != base);
    if (heads != 0xffffffffu) {   // some cell holds several lanes: segmented sums
      const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const long long v = __shfl_up_sync(0xffffffffu, c[q], off);
          if (lane - off >= start) c[q] += v;
        }
      }
    }
    if (base >= 0 && (lane == 31 || next != base)) {
      const int64_t at[8] = {base, base + 1, base + sy, base + sy + 1, base + sz, base + sz + 1, base + sz + sy,
                             base + sz + sy + 1};
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (c[q] != 0) atomicAdd(Q + at[q], (unsigned long long)c[q]);
    }
  }
}

static int particle_grid(pic_t *h) { return h->nsm * h->tune_particle_bps; }

int stage_keys(pic_t *h, int s) {
  Species &S = h->sp[s];
  if (h->keys_valid[s]) PIC_CUDA(h, cudaMemsetAsync(S.cnt, 0, (h->ncell + 1) * sizeof(uint32_t), h->stream));
  ++h->nlaunch;
  { KtScope kt_(h, kidKeys, 0); k_keys<<<particle_grid(h), kThreads, 0, h->stream>>>(S.a, S.key, S.cnt, h->nx, h->ny, h->clock, s); }
  h->keys_valid[s] = true;
  return launch_check(h, "keys");
}

int stage_push(pic_t *h, bool deposit) {
  if (deposit) {   // timed with the push: clearing the charge is part of producing it
    KtScope kt_(h, kidPush, 0);
    PIC_CUDA(h, cudaMemsetAsync(h->Q, 0, h->nnode * sizeof(unsigned long long), h->stream));
  }
  PIC_CUDA(h, cudaMemsetAsync(h->xq_n, 0, PIC_NSPECIES * sizeof(int), h->stream));
  for (int s = 0; s < nsp_active(h); ++s) {
    Species &S = h->sp[s];
    if (h->keys_valid[s]) PIC_CUDA(h, cudaMemsetAsync(S.cnt, 0, (h->ncell + 1) * sizeof(uint32_t), h->stream));
    PushArgs a;
    a.p = S.a; a.key = S.key; a.cnt = S.cnt; a.E = h->E; a.solid = h->solid; a.cheb = h->cheb;
    a.nx = h->nx; a.ny = h->ny; a.nz = h->nz; a.qmdt = S.qmdt;
    a.dtdx = (float)(h->prm.dt / h->dx);
    a.charged = S.Z != 0; a.ion = s == PIC_ION || s == PIC_ION2; a.species = s;
    a.mass = S.mass; a.w_min = h->prm.w_min;
    a.face_key = h->faces.key; a.nface = h->faces.n;
    a.acc_sput = (unsigned long long *)h->faces.acc_sput; a.acc_Eb = (unsigned long long *)h->faces.acc_Eb;
    a.clk = h->clock;
    a.Q = deposit && S.Z != 0 ? h->Q : nullptr;
    a.Z = S.Z;
    a.xq = S.perm;   // free until the sort
    a.xq_n = h->xq_n + s;
    h->nlaunch += 2;
    {
      KtScope kt_(h, kidPush, 0);
      if (S.Z == 0) k_push_neutral<<<particle_grid(h), kThreads, 0, h->stream>>>(a);
      else if (a.Q) k_push_charged<true><<<particle_grid(h), kThreads, 0, h->stream>>>(a);
      else k_push_charged<false><<<particle_grid(h), kThreads, 0, h->stream>>>(a);
    }
    { KtScope kt_(h, kidCross, 0); k_cross<<<h->nsm * 2, 256, 0, h->stream>>>(a); }
    h->keys_valid[s] = true;
  }
  return launch_check(h, "push");
}

// ---- SP merging (Sec. 2.3.2) -------------------------------------------------------------------
// In a cell holding N > M SPs of a species, the SPs at cell-sorted places 2m and 2m + 1 merge for
// m < min(N - M, N/2): w = w1 + w2 and, with mu = w1 w2 / (w1 + w2), every position and velocity
// component a = a1 mu/w2 + a2 mu/w1 (the centre of mass), in FP64 with one rounding per
// operation in that order and one rounding to FP32.  Pairs holding a zero weight, or summing
// above the weight cap, stay.  The merged SP keeps the first place and its id; the second keeps
// weight 0 and leaves at the next sort.  The centre of mass lies in the cell, so the order and
// the offsets stay valid.
__device__ __forceinline__ float merge_comp(double q1, double q2, float a1, float a2) {   // q1 = mu/w2, q2 = mu/w1
  return (float)__dadd_rn(__dmul_rn((double)a1, q1), __dmul_rn((double)a2, q2));
}

// One work item per sorted SP (its cell from the sort's per-position key): the SP at an even
// place 2m of a cell above the cap merges with its successor when m < min(N - M, N/2), so the
// pairs of a dense cell spread over many threads.
// With Q (the push has deposited this step's charge), a merged pair of a charged species moves its
// charge: the two SPs' CIC charges are taken off and the merged SP's added (exact int64 sums).
__global__ void __launch_bounds__(256) k_merge(SpeciesBuf p, const uint32_t *off, const uint32_t *skey, int s, uint32_t M,
                                               int32_t wmax, DevClock *clk, unsigned long long *Q, int Z, int nx,
                                               int ny) {
  const int64_t n = clk->n_sorted[s];
  int done = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = skey[t];
    const uint32_t o = off[c], N = off[c + 1] - o;
    if (N <= M) continue;
    const uint32_t q = (uint32_t)(t - o);
    if ((q & 1u) || q / 2 >= min(N - M, N / 2)) continue;
    const int64_t a = t, b = t + 1;
    const int32_t w1 = p.w[a], w2 = p.w[b];
    if (w1 <= 0 || w2 <= 0 || (int64_t)w1 + w2 > wmax) continue;
    const double d1 = w1, d2 = w2;
    const double mu = __ddiv_rn(__dmul_rn(d1, d2), __dadd_rn(d1, d2));
    const double q1 = __ddiv_rn(mu, d2), q2 = __ddiv_rn(mu, d1);
    if (Q) {
      uint32_t qa, qb;
      const uint32_t ba = cic_corner(p.x[a], p.y[a], p.z[a], nx, ny, &qa);
      const uint32_t bb = cic_corner(p.x[b], p.y[b], p.z[b], nx, ny, &qb);
      cic_global(Q, ba, qa, -Z * w1, nx, ny);
      cic_global(Q, bb, qb, -Z * w2, nx, ny);
    }
    p.x[a] = merge_comp(q1, q2, p.x[a], p.x[b]);
    p.y[a] = merge_comp(q1, q2, p.y[a], p.y[b]);
    p.z[a] = merge_comp(q1, q2, p.z[a], p.z[b]);
    p.vx[a] = merge_comp(q1, q2, p.vx[a], p.vx[b]);
    p.vy[a] = merge_comp(q1, q2, p.vy[a], p.vy[b]);
    p.vz[a] = merge_comp(q1, q2, p.vz[a], p.vz[b]);
    p.w[a] = w1 + w2;
    p.w[b] = 0;
    if (Q) {
      uint32_t qm;
      const uint32_t bm = cic_corner(p.x[a], p.y[a], p.z[a], nx, ny, &qm);
      cic_global(Q, bm, qm, Z * (w1 + w2), nx, ny);
    }
    ++done;
  }
  for (int sh = 16; sh > 0; sh >>= 1) done += __shfl_down_sync(0xffffffffu, done, sh);
  if ((threadIdx.x & 31) == 0 && done) atomicAdd((unsigned long long *)&clk->ctr[cMerged], (unsigned long long)done);
}

int stage_merge(pic_t *h, bool fix_charge) {
  if (!(h->prm.flags & PIC_F_MERGE)) return PIC_OK;
  const int ns = nsp_active(h);
  for (int s = 0; s < ns; ++s) if (h->keys_valid[s]) return pic_fail(h, PIC_E_INVALID, "merging needs cell-sorted SPs");
  const uint32_t M = h->prm.merge_max > 0 ? (uint32_t)h->prm.merge_max : 32u;
  const int32_t wmax = h->prm.w_max_units > 0 ? h->prm.w_max_units : INT32_MAX;
  h->nlaunch += ns;
  KtScope kt_(h, kidMerge, 0);
  for (int s = 0; s < ns; ++s)
    k_merge<<<h->nsm * 8, kThreads, 0, h->stream>>>(h->sp[s].a, h->sp[s].off, h->sp[s].skey, s, M, wmax, h->clock,
                                                    fix_charge && h->sp[s].Z != 0 ? h->Q : nullptr, h->sp[s].Z,
                                                    h->nx, h->ny);
  return launch_check(h, "merge");
}

// Loaded SPs must lie inside the domain and outside the tip: the smallest offending index of
// each kind (bad[0]: outside, bad[1]: inside the tip; all ones when there is none).
__global__ void k_validate(SpeciesBuf p, int64_t n, const uint8_t *solid, int nx, int ny, int nz,
                           unsigned long long *bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float x = p.x[i], y = p.y[i], z = p.z[i];
    if (!(x >= 0.f && x < (float)nx && y >= 0.f && y < (float)ny && z >= 0.f && z < (float)nz))
      atomicMin(&bad[0], (unsigned long long)i);
    else if (solid[cell_index((int)floorf(x), (int)floorf(y), (int)floorf(z), nx, ny)])
      atomicMin(&bad[1], (unsigned long long)i);
  }
}

int validate_loaded(pic_t *h, const SpeciesBuf &p, int64_t n) {
  unsigned long long *bad = (unsigned long long *)(h->tmp_len + 14);
  PIC_CUDA(h, cudaMemsetAsync(bad, 0xff, 2 * sizeof(unsigned long long), h->stream));
  ++h->nlaunch;
  k_validate<<<particle_grid(h), kThreads, 0, h->stream>>>(p, n, h->solid, h->nx, h->ny, h->nz, bad);
  unsigned long long hb[2];
  PIC_CUDA(h, cudaMemcpyAsync(hb, bad, sizeof hb, cudaMemcpyDeviceToHost, h->stream));
  PIC_CUDA(h, cudaStreamSynchronize(h->stream));
  if (hb[0] != ~0ull) return pic_fail(h, PIC_E_INVALID, "SP " + std::to_string(hb[0]) + " outside the domain");
  if (hb[1] != ~0ull) return pic_fail(h, PIC_E_INVALID, "SP " + std::to_string(hb[1]) + " inside the tip");
  return PIC_OK;
}

// Counting sort of one species by cell: scan of the per-cell counts, scatter, the fix-ups that
// make the order stable, gather into the other buffer, swap.
int sort_species(pic_t *h, int s) {
  int2 *long_list = h->long_list;
  int *long_n = h->long_n;
  const int long_cap = kLongCap;
  Species &S = h->sp[s];
  if (!h->keys_valid[s]) PIC_TRY(stage_keys(h, s));
  PIC_TRY(scan_u32(h, S.cnt, S.off, h->ncell, nullptr, S.off + h->ncell));
  ++h->nlaunch;
  { KtScope kt_(h, kidScatter, 0); k_scatter<<<particle_grid(h), kThreads, 0, h->stream>>>(S.key, S.cnt, S.off, S.perm, S.skey, h->clock, s); }
  PIC_CUDA(h, cudaMemsetAsync(long_n, 0, 2 * sizeof(int), h->stream));   // long_n[0]: long, [1]: mid
  ++h->nlaunch;
  { KtScope kt_(h, kidFixShort, 0); k_fix_short<<<particle_grid(h), kThreads, 0, h->stream>>>(S.skey, S.off, S.perm, h->ncell, h->mid_list,
                                                            long_n + 1, (int)h->mid_cap, long_list, long_n,
                                                            long_cap, h->clock); }
  ++h->nlaunch;
  { KtScope kt_(h, kidFixMid, 0); k_fix_mid<<<particle_grid(h), kThreads, 0, h->stream>>>(S.perm, h->mid_list, long_n + 1, (int)h->mid_cap); }
  ++h->nlaunch;
  {
    static_assert(kMaxSegment * sizeof(uint32_t) <= 227 * 1024, "segment buffer above the shared memory of a block");
    if (!h->fix_long_smem_set) {
      PIC_CUDA(h, cudaFuncSetAttribute(k_fix_long, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(kMaxSegment * sizeof(uint32_t))));
      h->fix_long_smem_set = true;
    }
    KtScope kt_(h, kidFixLong, 0);
    k_fix_long<<<h->nsm, 1024, kMaxSegment * sizeof(uint32_t), h->stream>>>(S.perm, long_list, long_n, long_cap);
  }
  ++h->nlaunch;
  { KtScope kt_(h, kidGather, 0); k_gather<<<particle_grid(h), kThreads, 0, h->stream>>>(S.a, S.b, S.perm, S.off, h->ncell); }
  ++h->nlaunch;
  k_set_count<<<1, 1, 0, h->stream>>>(h->clock, s, S.off, h->ncell);
  std::swap(S.a, S.b);
  h->keys_valid[s] = false;
  return launch_check(h, "sort");
}

int stage_sort(pic_t *h) {
  for (int s = 0; s < nsp_active(h); ++s) PIC_TRY(sort_species(h, s));
  return PIC_OK;
}

int stage_deposit(pic_t *h) {
  PIC_CUDA(h, cudaMemsetAsync(h->Q, 0, h->nnode * sizeof(unsigned long long), h->stream));
  ++h->nlaunch;
  { KtScope kt_(h, kidDeposit, 0); k_deposit<<<particle_grid(h), kThreads, 0, h->stream>>>(h->sp[PIC_ELECTRON].a, -1, h->Q, h->nx, h->ny, h->clock,
                                                          PIC_ELECTRON); }
  ++h->nlaunch;
  { KtScope kt_(h, kidDeposit, 0); k_deposit<<<particle_grid(h), kThreads, 0, h->stream>>>(h->sp[PIC_ION].a, 1, h->Q, h->nx, h->ny, h->clock, PIC_ION); }
  if (nsp_active(h) > PIC_ION2) {
    ++h->nlaunch;
    KtScope kt_(h, kidDeposit, 0);
    k_deposit<<<particle_grid(h), kThreads, 0, h->stream>>>(h->sp[PIC_ION2].a, 2, h->Q, h->nx, h->ny, h->clock, PIC_ION2);
  }
  return launch_check(h, "deposit");
}

// Autotuner probe for the particle kernels' grid (blocks per SM): each candidate times the
// deposit (clear + e- and Cu+ launches; the fixed-point sums do not depend on the launch shape,
// so the probe leaves the charge as a deposit would) and the fastest is kept for every
// particle kernel.  All of them are grid-stride loops whose results do not depend on the grid.
int tune_particles(pic_t *h, int *best) {
  const int cand[5] = {2, 4, 8, 16, 32};
  cudaEvent_t e0, e1;
  PIC_CUDA(h, cudaEventCreate(&e0));
  PIC_CUDA(h, cudaEventCreate(&e1));
  const int keep = h->tune_particle_bps;
  float best_ms = 1e30f;
  int pick = keep;
  for (int c : cand) {
    h->tune_particle_bps = c;
    float t_min = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, h->stream);
      const int rc = stage_deposit(h);
      cudaEventRecord(e1, h->stream);
      if (rc != PIC_OK) { h->tune_particle_bps = keep; cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
      cudaEventSynchronize(e1);
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      t_min = std::min(t_min, t);
    }
    if (t_min < best_ms) { best_ms = t_min; pick = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->tune_particle_bps = pick;
  *best = pick;
  return launch_check(h, "tune particles");
}

}  // namespace pic
