// Monte Carlo collisions: impact ionization Cu + e -> Cu+ + 2e with SP splitting (Sec. 2.2,
// eq:colp, eq:du, Sec. 2.3.2) and direct field ionization of neutrals (eq:dfi, Sec. 2.3.4);
// with their flags, the Cu2+ channels of Table colls (Cu + e -> Cu2+ + 3e inside the impact
// ionization pass, then Cu+ + e -> Cu2+ + 2e), elastic e-Cu and Cu-Cu collisions and Cu+-Cu
// charge exchange (eq:newv, with splitting) and binary Coulomb collisions between charged SPs
// (Table colls), in the order impact ionization, Cu+ ionization, elastic passes, Coulomb passes,
// field ionization.
//
// Pairing in a cell with N_e electron SPs and N_t target SPs: the species with fewer SPs (tie:
// electrons) is the projectile; projectile k meets target (k + o_c) mod N_t, o_c =
// floor(U_PAIR(cell, step) N_t).  Each of the w_p sub-particles of a projectile collides iff
// U_i < P, P = 1 - exp(-u n_t W_t sigma(E0) dt), n_t the target SP density and W_t the paired
// target's weight in real particles; N_coll is capped at the target weight.  With the double
// channel the total cross section sets P_T and a sub-particle ionizes once below
// P_T sigma_1/sigma_T and twice between that and P_T.
//
// Decisions: P is evaluated in float32; any draw within a guard band of a threshold (2^-12
// relative to it plus the largest value this relative speed can reach) re-decides the whole
// pair in float64, so every decision equals the float64 decision.
//
// Products are written in a fixed order so ids and slots are deterministic: pairs with an
// electron projectile in cell-sorted electron order, then pairs with a target projectile in
// cell-sorted target order; per pair the ion, the scattered electron (when the electron SP
// is split) and the secondary electron take consecutive ids; the double events follow all single
// ones in the same pair order (Cu2+, scattered electron, two secondary electrons).
#include "pic_internal.cuh"
#include "dev_common.cuh"

namespace pic {

constexpr double kLotzA = 4.5e-18;     // m^2 eV^2  (4.5e-14 cm^2 eV^2), Cu + e -> Cu+ + 2e
// Stand-ins of the Cu2+ channels (same Lotz form): double ionization of Cu with a tenth of the
// single constant at xi_1 + xi_2, and ionization of Cu+ with ten times it (ten 3d electrons) at xi_2
constexpr double kLotzDouble = 4.5e-19, kXiDouble = 28.018;
constexpr double kLotzIz = 4.5e-17;
// The smallest uniform draw, 0.5 * 2^-24.  When P + guard band is below it, no draw can land
// under P or inside the band, so the decisions (none) are known without drawing.
constexpr float kUmin = 2.98023223876953125e-8f;

__device__ __forceinline__ double lotz64(double E, double xi, double a) {
  return E > xi ? a * log(E / xi) / (E * xi) : 0.0;
}
__device__ __forceinline__ float lotz32(float E, float xi, float a) {
  return E > xi ? a * logf(E / xi) / (E * xi) : 0.0f;
}

// One impact-ionization pass: electrons against a heavy target species (Cu, or Cu+ for the Cu+
// pass) producing an ion of the next charge.
struct McArgs {
  SpeciesBuf e, n;                   // electrons and the target species
  SpeciesBuf prod, j;                // single-channel products; Cu2+ (double channel)
  const uint32_t *off_e, *off_n;     // per-cell offsets of the last sort
  const uint32_t *skey_e, *skey_n;   // cell of each sorted position
  double V_cell, dt, w_min;
  double xi, lotz;                   // threshold [eV] and Lotz constant [m^2 eV^2] of the single channel
  float xi32, lotz32, sig_peak;      // the same in FP32; largest sigma_T (a/(e xi^2) summed over channels)
  uint32_t pur_pair, pur_draw, pur_scat;
  int sn, sprod;                     // species of the target and of the single products
  int dbl;                           // the double channel competes (Cu target)
  uint64_t seed;
  DevClock *clk;
  int *go;
  const uint64_t *total1;            // products kernel: totals of the single products (ions | e << 32)
};

// ---- ordered compaction of rare events ---------------------------------------------------------
// Work items are cut into units of kEvUnit consecutive items; warps take units round-robin (so
// dense regions spread over all warps) and stage each unit's items with an event, in item
// order, at rec[unit kEvUnit ...].  A scan of the units' product counts gives their offsets; the
// products kernel writes each unit's products in item order from its offset.  Slots and ids are
// thus those of an exclusive scan over all items in item order, without a scan over all items.
constexpr int kEvUnit = 256;
struct EvBlocks {
  uint64_t *rec;    // staged events: item | payload << 32
  int *hits;        // events per unit
  uint64_t *cnt;    // products per unit: ions | electrons << 32
  uint64_t *off;    // exclusive offsets of cnt
  uint64_t *cnt2;   // second product kind per unit (double ionization: Cu2+ | electrons << 32)
  uint64_t *off2;   // exclusive offsets of cnt2
};

__device__ __forceinline__ int ev_warp() { return (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); }
__device__ __forceinline__ int ev_nwarp() { return (int)((gridDim.x * blockDim.x) >> 5); }

// Units of work items: mode 0 sorted e- + sorted Cu (impact ionization), 1 all neutrals (DFI),
// 2 + s sorted species s (elastic passes), 6 sorted e- + sorted Cu+ (Cu+ ionization)
__global__ void k_ev_units(int64_t *out, const DevClock *clk, int mode) {
  const int64_t n = mode == 0   ? clk->n_sorted[PIC_ELECTRON] + clk->n_sorted[PIC_NEUTRAL]
                    : mode == 1 ? clk->n[PIC_NEUTRAL]
                    : mode == 6 ? clk->n_sorted[PIC_ELECTRON] + clk->n_sorted[PIC_ION]
                                : clk->n_sorted[mode - 2];
  *out = (n + kEvUnit - 1) / kEvUnit;
}

// capacity check + totals of a packed (ions | electrons << 32) scan
__global__ void k_check_new(DevClock *clk, const uint64_t *total, int64_t cap_i, int64_t cap_e, int *go) {
  const uint64_t t = *total;
  const int64_t ni = (int64_t)(t & 0xffffffffu), ne = (int64_t)(t >> 32);
  const bool ok = clk->n[PIC_ION] + ni <= cap_i && clk->n[PIC_ELECTRON] + ne <= cap_e;
  *go = ok ? 1 : 0;
  if (!ok) atomicOr(&clk->err, kErrCapacity);
}

// the same for an impact-ionization pass: single products (species sprod | e-) and, with
// total2, double products (Cu2+ | e-)
__global__ void k_mcc_check(DevClock *clk, const uint64_t *total1, const uint64_t *total2, int sprod, int64_t cap_p,
                            int64_t cap_e, int64_t cap_j, int *go) {
  const uint64_t t = *total1, u = total2 ? *total2 : 0ull;
  const int64_t np = (int64_t)(t & 0xffffffffu), ne = (int64_t)(t >> 32) + (int64_t)(u >> 32);
  const int64_t nj = (int64_t)(u & 0xffffffffu) + (sprod == PIC_ION2 ? np : 0);
  const bool ok = clk->n[sprod] + np <= cap_p && clk->n[PIC_ELECTRON] + ne <= cap_e && clk->n[PIC_ION2] + nj <= cap_j;
  *go = ok ? 1 : 0;
  if (!ok) atomicOr(&clk->err, kErrCapacity);
}

// Exclusive prefix of v over the warp in lane order, and the warp total.
__device__ __forceinline__ uint64_t warp_scan_u64(uint64_t v, uint64_t *total) {
  const int lane = threadIdx.x & 31;
  uint64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  *total = __shfl_sync(0xffffffffu, x, 31);
  return x - v;
}

// Stage this tile's events (payload != 0) in item order and add the tile's product count pc.
__device__ __forceinline__ void ev_stage(const EvBlocks &ev, int64_t lo, int64_t *run, uint64_t *prod, int64_t t,
                                         uint32_t payload, uint64_t pc) {
  const unsigned bal = __ballot_sync(0xffffffffu, payload != 0);
  const int lane = threadIdx.x & 31;
  if (payload) ev.rec[lo + *run + __popc(bal & ((1u << lane) - 1u))] = (uint64_t)t | ((uint64_t)payload << 32);
  *run += __popc(bal);
  if (__any_sync(0xffffffffu, pc != 0)) {   // most tiles have no event
    uint64_t p_tile;
    warp_scan_u64(pc, &p_tile);
    *prod += p_tile;
  }
}

// The leader of each run of adjacent lanes with the same cell draws the cell's pairing word once
// and shares it (every lane of the warp takes part).  Work items come cell-sorted, so a cell's
// lanes are adjacent; a cell split over two runs draws the same word twice.
__device__ __forceinline__ uint32_t cell_word(uint64_t seed, uint32_t purpose, uint32_t c, bool need, int64_t step) {
  const int lane = threadIdx.x & 31;
  const uint32_t key = need ? c : 0xffffffffu;
  const uint32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
  const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != key);
  const int leader = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
  uint32_t w = 0;
  if (need && lane == leader) w = rng_block(seed, purpose, c, step, 0).v[0];
  return __shfl_sync(0xffffffffu, w, leader);
}

struct Pair {
  int64_t ie, in;   // electron index, target index
  int proj_e;       // 1: electron is the projectile
  uint32_t Nt;
};

// Cell and counts of work item t (t < n_e: electron t; else target t - n_e); whether the item is
// the projectile of a pair.
struct McItem {
  uint32_t c, oe, Ne, on, Nn;
  bool proj;
};
__device__ __forceinline__ McItem mc_item(const McArgs &a, int64_t t, int64_t ne) {
  McItem m;
  const bool is_e = t < ne;
  m.c = is_e ? a.skey_e[t] : a.skey_n[t - ne];
  m.oe = a.off_e[m.c]; m.Ne = a.off_e[m.c + 1] - m.oe;
  m.on = a.off_n[m.c]; m.Nn = a.off_n[m.c + 1] - m.on;
  m.proj = m.Ne > 0 && m.Nn > 0 && (m.Ne <= m.Nn) == is_e;
  return m;
}

// The pair of projectile item t, from the cell's pairing word w.
__device__ __forceinline__ Pair mc_pair(const McItem &m, int64_t t, int64_t ne, uint32_t w) {
  Pair pr;
  const bool is_e = t < ne;
  const int64_t p = is_e ? t : t - ne;
  pr.Nt = is_e ? m.Nn : m.Ne;
  const uint32_t k = (uint32_t)(p - (is_e ? m.oe : m.on));
  const uint32_t tgt = (k + u_index(w, pr.Nt)) % pr.Nt;
  if (is_e) { pr.ie = p; pr.in = (int64_t)m.on + tgt; }
  else { pr.in = p; pr.ie = (int64_t)m.oe + tgt; }
  pr.proj_e = is_e;
  return pr;
}

// Sub-particle collisions of one pair: the single channel's count (0..min(w_p, w_t)) and, with
// the double channel, *n2 = #{P_1 <= U_i < P_T} capped at what the single ones leave of w_t.
__device__ int mcc_ncoll(const McArgs &a, const Pair &pr, int64_t step, int *n2) {
  const int we = a.e.w[pr.ie], wn = a.n.w[pr.in];
  const int wp = pr.proj_e ? we : wn, wt = pr.proj_e ? wn : we;
  const float dvx = a.e.vx[pr.ie] - a.n.vx[pr.in];
  const float dvy = a.e.vy[pr.ie] - a.n.vy[pr.in];
  const float dvz = a.e.vz[pr.ie] - a.n.vz[pr.in];
  const float u2 = dvx * dvx + dvy * dvy + dvz * dvz;
  const float u = sqrtf(u2);
  const float E0 = (float)(0.5 * kMe / kQe) * u2;
  const float nW = (float)((double)pr.Nt / a.V_cell * (double)wt * a.w_min * a.dt);
  const float s1 = lotz32(E0, a.xi32, a.lotz32);
  const float sT = a.dbl ? s1 + lotz32(E0, (float)kXiDouble, (float)kLotzDouble) : s1;
  const float PT = -expm1f(-(u * nW * sT));
  const float P1 = a.dbl ? (sT > 0.0f ? PT * (s1 / sT) : 0.0f) : PT;
  const float reach = u * nW * a.sig_peak;
  const float band1 = ldexpf(P1 + reach, -12), bandT = ldexpf(PT + reach, -12);
  const uint64_t pid = pr.proj_e ? a.e.id[pr.ie] : a.n.id[pr.in];
  int c1 = 0, c2 = 0;
  bool exact = false;
  for (int i = 0; i < wp && PT + bandT >= kUmin; i += 4) {
    const U4 r = rng_block(a.seed, a.pur_draw, pid, step, (uint32_t)(i >> 2));
    for (int j = 0; j < 4 && i + j < wp; ++j) {
      const float U = u01f(r.v[j]);
      if (fabsf(U - P1) <= band1 || (a.dbl && fabsf(U - PT) <= bandT)) exact = true;
      c1 += U < P1;
      c2 += U >= P1 && U < PT;
    }
  }
  if (exact) {   // the FP64 definition, in the oracle's order of operations
    const double ex = (double)a.e.vx[pr.ie] - (double)a.n.vx[pr.in];
    const double ey = (double)a.e.vy[pr.ie] - (double)a.n.vy[pr.in];
    const double ez = (double)a.e.vz[pr.ie] - (double)a.n.vz[pr.in];
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
    const double ud = sqrt(d2);
    const double E0d = 0.5 * kMe * d2 / kQe;
    const double s1d = lotz64(E0d, a.xi, a.lotz);
    const double sTd = a.dbl ? s1d + lotz64(E0d, kXiDouble, kLotzDouble) : s1d;
    const double PTd = -expm1(-(ud * ((double)pr.Nt / a.V_cell) * ((double)wt * a.w_min) * sTd * a.dt));
    const double P1d = sTd > 0.0 ? PTd * (s1d / sTd) : 0.0;
    c1 = 0;
    c2 = 0;
    for (int i = 0; i < wp; i += 4) {
      const U4 r = rng_block(a.seed, a.pur_draw, pid, step, (uint32_t)(i >> 2));
      for (int j = 0; j < 4 && i + j < wp; ++j) {
        const double U = u01d(r.v[j]);
        c1 += U < P1d;
        c2 += U >= P1d && U < PTd;
      }
    }
  }
  c1 = c1 > wt ? wt : c1;
  if (n2) *n2 = a.dbl ? (c2 > wt - c1 ? wt - c1 : c2) : 0;
  return c1;
}

// Work items: sorted electrons, then sorted targets; a pair with an event is staged with payload
// n1 (with the double channel: n1 | bit 31, so pairs with only double events are staged too).  A
// warp takes a unit of kEvUnit items in two passes: the first finds the unit's projectiles (the
// items of the species with fewer SPs in their cell) and queues their pairs in shared memory in
// item order; the second evaluates the queued pairs 32 at a time, so every lane works on a pair
// (the projectiles are a fraction of the items, and evaluating them in place left most lanes
// idle).
struct McQueued {
  uint32_t t;        // work item
  uint32_t ie, in;   // electron and target of the pair
  uint32_t nt;       // target SPs in the cell; bit 31: the electron is the projectile
};

__global__ void __launch_bounds__(256) k_mcc_count(McArgs a, EvBlocks ev) {
  __shared__ McQueued queue[256 / 32][kEvUnit];
  McQueued *qw = queue[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int64_t ne = a.clk->n_sorted[PIC_ELECTRON], nn = a.clk->n_sorted[a.sn];
  const int64_t step = a.clk->step;
  const int64_t total = ne + nn, nunit = (total + kEvUnit - 1) / kEvUnit;
  for (int64_t unit = ev_warp(); unit < nunit; unit += ev_nwarp()) {
    const int64_t lo = unit * kEvUnit, hi = min(total, lo + kEvUnit);
    int nq = 0;
    for (int64_t base = lo; base < hi; base += 32) {
      const int64_t t = base + lane;
      McItem m{};
      if (t < hi) m = mc_item(a, t, ne);
      const uint32_t w = cell_word(a.seed, a.pur_pair, m.c, m.proj, step);
      const unsigned bal = __ballot_sync(0xffffffffu, m.proj);
      if (m.proj) {
        const Pair pr = mc_pair(m, t, ne, w);
        McQueued e;
        e.t = (uint32_t)(t - lo);
        e.ie = (uint32_t)pr.ie;
        e.in = (uint32_t)pr.in;
        e.nt = pr.Nt | (pr.proj_e ? 0x80000000u : 0u);
        qw[nq + __popc(bal & ((1u << lane) - 1u))] = e;
      }
      nq += __popc(bal);
    }
    __syncwarp();
    int64_t run = 0;
    uint64_t prod = 0, prod2 = 0;
    for (int b = 0; b < nq; b += 32) {
      const int i = b + lane;
      int ncoll = 0, n2 = 0;
      uint64_t pc = 0, pc2 = 0;
      int64_t t = lo;
      if (i < nq) {
        const McQueued e = qw[i];
        Pair pr;
        pr.ie = e.ie;
        pr.in = e.in;
        pr.proj_e = (e.nt >> 31) & 1;
        pr.Nt = e.nt & 0x7fffffffu;
        t = lo + e.t;
        ncoll = mcc_ncoll(a, pr, step, &n2);
        const int we = a.e.w[pr.ie];
        if (ncoll > 0) pc = 1ull | ((uint64_t)(ncoll < we ? 2 : 1) << 32);
        if (n2 > 0) pc2 = 1ull | ((uint64_t)(n2 < we - ncoll ? 3 : 2) << 32);
      }
      const uint32_t payload = a.dbl ? ((ncoll > 0 || n2 > 0) ? (0x80000000u | (uint32_t)ncoll) : 0u) : (uint32_t)ncoll;
      ev_stage(ev, lo, &run, &prod, t, payload, pc);
      if (a.dbl && __any_sync(0xffffffffu, pc2 != 0)) {
        uint64_t t2;
        warp_scan_u64(pc2, &t2);
        prod2 += t2;
      }
    }
    __syncwarp();
    if (lane == 0) {
      ev.hits[unit] = (int)run;
      ev.cnt[unit] = prod;
      if (a.dbl) ev.cnt2[unit] = prod2;
    }
  }
}

__device__ void scatter_velocity(double ux, double uy, double uz, double uk, double cos_tp, double phi_p, double out[3]) {
  const double u = sqrt(ux * ux + uy * uy + uz * uz);
  double th = 0.0, ph = 0.0;
  if (u > 0) {
    double c = uz / u;
    c = c > 1.0 ? 1.0 : (c < -1.0 ? -1.0 : c);
    th = acos(c);
    ph = atan2(uy, ux);
  }
  const double tp = acos(cos_tp);
  const double a0 = uk * sin(tp) * cos(phi_p), a1 = uk * sin(tp) * sin(phi_p), a2 = uk * cos(tp);
  const double ct = cos(th), st = sin(th), cp = cos(ph), sp = sin(ph);
  // R^-1(theta, phi) = R^T with R rows (ct cp, ct sp, -st), (-sp, cp, 0), (st cp, st sp, ct)
  out[0] = ct * cp * a0 - sp * a1 + st * cp * a2;
  out[1] = ct * sp * a0 + cp * a1 + st * sp * a2;
  out[2] = -st * a0 + ct * a2;
}

__device__ __forceinline__ void put_sp(SpeciesBuf &B, int64_t s, float x, float y, float z, float vx, float vy, float vz,
                                       int32_t w, uint64_t id) {
  B.x[s] = x; B.y[s] = y; B.z[s] = z; B.vx[s] = vx; B.vy[s] = vy; B.vz[s] = vz; B.w[s] = w; B.id[s] = id;
}

__global__ void k_commit_new(DevClock *clk, const uint64_t *total, const int *go, int ctr) {
  if (!*go) return;
  const uint64_t t = *total;
  const int64_t ni = (int64_t)(t & 0xffffffffu), ne = (int64_t)(t >> 32);
  clk->n[PIC_ION] += ni;
  clk->n[PIC_ELECTRON] += ne;
  clk->next_id += ni + ne;
  clk->ctr[ctr] += ni;
}

// commit of an impact-ionization pass: single products (one ion per event) and double ones
__global__ void k_mcc_commit(DevClock *clk, const uint64_t *total1, const uint64_t *total2, const int *go, int sprod,
                             int ctr) {
  if (!*go) return;
  const uint64_t t = *total1, u = total2 ? *total2 : 0ull;
  const int64_t np = (int64_t)(t & 0xffffffffu), ne = (int64_t)(t >> 32);
  const int64_t nj = (int64_t)(u & 0xffffffffu), ne2 = (int64_t)(u >> 32);
  clk->n[sprod] += np;
  clk->n[PIC_ELECTRON] += ne + ne2;
  clk->n[PIC_ION2] += nj;
  clk->next_id += np + ne + nj + ne2;
  clk->ctr[ctr] += np;
  clk->ctr[cDoubleIon] += nj;
}

// Products of the staged pairs, warp by warp in item order from the warp's offsets.  Each
// thread's pair is its own (an SP belongs to one pair of a pass), so the pre-collision weights
// and velocities it reads are untouched until it writes them.
__global__ void __launch_bounds__(256) k_mcc_products(McArgs a, EvBlocks ev) {
  if (!*a.go) return;
  const int64_t ne = a.clk->n_sorted[PIC_ELECTRON], nn = a.clk->n_sorted[a.sn];
  const int64_t ne_all = a.clk->n[PIC_ELECTRON], np_all = a.clk->n[a.sprod], nj_all = a.clk->n[PIC_ION2];
  const int64_t step = a.clk->step, id_base = a.clk->next_id;
  const uint64_t t1 = *a.total1;
  const int64_t single_e = (int64_t)(t1 >> 32), single_all = (int64_t)(t1 & 0xffffffffu) + single_e;
  const int64_t nunit = (ne + nn + kEvUnit - 1) / kEvUnit;
  for (int64_t unit = ev_warp(); unit < nunit; unit += ev_nwarp()) {
    const int64_t lo = unit * kEvUnit;
    const int nh = ev.hits[unit];
    uint64_t run = ev.off[unit], run2 = a.dbl ? ev.off2[unit] : 0ull;
    for (int base = 0; base < nh; base += 32) {
      const int i = base + (threadIdx.x & 31);
      Pair pr{};
      int ncoll = 0, n2 = 0, we = 0;
      uint64_t pc = 0, pc2 = 0;
      if (i < nh) {
        const uint64_t rec = ev.rec[lo + i];
        const int64_t t = (int64_t)(uint32_t)rec;
        ncoll = (int)((rec >> 32) & 0x7fffffffu);
        const McItem m = mc_item(a, t, ne);
        pr = mc_pair(m, t, ne, rng_block(a.seed, a.pur_pair, m.c, step, 0).v[0]);
        if (a.dbl) mcc_ncoll(a, pr, step, &n2);
        we = a.e.w[pr.ie];
        if (ncoll > 0) pc = 1ull | ((uint64_t)(ncoll < we ? 2 : 1) << 32);
        if (n2 > 0) pc2 = 1ull | ((uint64_t)(n2 < we - ncoll ? 3 : 2) << 32);
      }
      uint64_t tile;
      const uint64_t off = run + warp_scan_u64(pc, &tile);
      run += tile;
      uint64_t off2 = 0;
      if (a.dbl) {
        off2 = run2 + warp_scan_u64(pc2, &tile);
        run2 += tile;
      }
      if (i >= nh) continue;
      const int64_t in = pr.in, ie = pr.ie;
      const int wn = a.n.w[in];
      const uint64_t pid = pr.proj_e ? a.e.id[ie] : a.n.id[in];
      const double vnx = a.n.vx[in], vny = a.n.vy[in], vnz = a.n.vz[in];
      const double ux = (double)a.e.vx[ie] - vnx, uy = (double)a.e.vy[ie] - vny, uz = (double)a.e.vz[ie] - vnz;
      const double u2 = __dadd_rn(__dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy)), __dmul_rn(uz, uz));
      const double E0 = 0.5 * kMe * u2 / kQe;
      const float tx = a.n.x[in], ty = a.n.y[in], tz = a.n.z[in];
      const float tvx = a.n.vx[in], tvy = a.n.vy[in], tvz = a.n.vz[in];
      if (ncoll > 0) {
        const int64_t ion_off = (int64_t)(off & 0xffffffffu), e_off = (int64_t)(off >> 32);
        int64_t id = id_base + ion_off + e_off;
        // ion of the next charge with the target's position and velocity
        put_sp(a.prod, np_all + ion_off, tx, ty, tz, tvx, tvy, tvz, ncoll, (uint64_t)id++);
        // outgoing electrons: (E0 - xi)/2 each, directions by eq:du about u = v_e - v_t
        const double Ek = 0.5 * (E0 - a.xi);
        const double uk = sqrt(2.0 * Ek * kQe / kMe);
        const U4 r = rng_block(a.seed, a.pur_scat, pid, step, 0);
        double v1[3], v2[3];
        scatter_velocity(ux, uy, uz, uk, 2.0 * u01d(r.v[0]) - 1.0, 2.0 * kPi * u01d(r.v[1]), v1);
        scatter_velocity(ux, uy, uz, uk, 2.0 * u01d(r.v[2]) - 1.0, 2.0 * kPi * u01d(r.v[3]), v2);
        int64_t slot = ne_all + e_off;
        if (ncoll == we) {
          a.e.vx[ie] = (float)(vnx + v1[0]); a.e.vy[ie] = (float)(vny + v1[1]); a.e.vz[ie] = (float)(vnz + v1[2]);
        } else {
          put_sp(a.e, slot++, a.e.x[ie], a.e.y[ie], a.e.z[ie], (float)(vnx + v1[0]), (float)(vny + v1[1]),
                 (float)(vnz + v1[2]), ncoll, (uint64_t)id++);
        }
        put_sp(a.e, slot, tx, ty, tz, (float)(vnx + v2[0]), (float)(vny + v2[1]), (float)(vnz + v2[2]), ncoll, (uint64_t)id);
      }
      if (n2 > 0) {
        // Cu2+ and three outgoing electrons of (E0 - xi_1 - xi_2)/3 each, after every single product
        const int64_t j_off = (int64_t)(off2 & 0xffffffffu), e_off = (int64_t)(off2 >> 32);
        int64_t id = id_base + single_all + j_off + e_off;
        put_sp(a.j, nj_all + j_off, tx, ty, tz, tvx, tvy, tvz, n2, (uint64_t)id++);
        const double uk = sqrt(2.0 * (E0 - kXiDouble) / 3.0 * kQe / kMe);
        const U4 r0 = rng_block(a.seed, kScat2, pid, step, 0), r1 = rng_block(a.seed, kScat2, pid, step, 1);
        double v[3][3];
        scatter_velocity(ux, uy, uz, uk, 2.0 * u01d(r0.v[0]) - 1.0, 2.0 * kPi * u01d(r0.v[1]), v[0]);
        scatter_velocity(ux, uy, uz, uk, 2.0 * u01d(r0.v[2]) - 1.0, 2.0 * kPi * u01d(r0.v[3]), v[1]);
        scatter_velocity(ux, uy, uz, uk, 2.0 * u01d(r1.v[0]) - 1.0, 2.0 * kPi * u01d(r1.v[1]), v[2]);
        const int we1 = we - ncoll;   // the electron SP's weight after the single channel
        int64_t slot = ne_all + single_e + e_off;
        if (n2 == we1) {
          a.e.vx[ie] = (float)(vnx + v[0][0]); a.e.vy[ie] = (float)(vny + v[0][1]); a.e.vz[ie] = (float)(vnz + v[0][2]);
        } else {
          put_sp(a.e, slot++, a.e.x[ie], a.e.y[ie], a.e.z[ie], (float)(vnx + v[0][0]), (float)(vny + v[0][1]),
                 (float)(vnz + v[0][2]), n2, (uint64_t)id++);
        }
        for (int q = 1; q < 3; ++q)
          put_sp(a.e, slot++, tx, ty, tz, (float)(vnx + v[q][0]), (float)(vny + v[q][1]), (float)(vnz + v[q][2]), n2,
                 (uint64_t)id++);
      }
      // weights last: the electron keeps we - n1 - n2 unless it turned whole, the target loses n1 + n2
      if (ncoll > 0 && ncoll < we) a.e.w[ie] = we - ncoll - (n2 > 0 && n2 < we - ncoll ? n2 : 0);
      else if (ncoll == 0 && n2 > 0 && n2 < we) a.e.w[ie] = we - n2;
      a.n.w[in] = wn - ncoll - n2;
    }
  }
}

// ---- elastic collisions and charge exchange ---------------------------------------------------
// e + Cu -> e + Cu and Cu + Cu -> Cu + Cu (eq:newv with the velocity difference of eq:du) and
// Cu+ + Cu -> Cu + Cu+ (the colliding sub-particles swap velocities), on the cell-sorted SPs of
// the step, with the splitting of Sec. 2.3.2: each of the projectile's w_p sub-particles collides
// iff U_i < P (eq:colp with the paired target's weight), N_coll is capped at the target weight,
// and the N_coll colliding sub-particles of each side leave their SP as a new SP with the
// post-collision velocity (the whole SP turns when N_coll is its weight).  The draws are decided
// in FP32 and re-decided in FP64 when one lies within the guard band of P, as for impact
// ionization.  Events are staged per unit of work items and their new SPs placed in item order,
// so ids and slots are deterministic: events of a pass in the order of the pair's member in the
// pass's first species (e-, Cu+, or the projectile for Cu-Cu), per event the projectile's new SP
// first.
struct ElArgs {
  double V_cell, dt, w_min;
  uint64_t seed;
  DevClock *clk;
  int *go;
};

struct ElPass {
  SpeciesBuf A, B;                          // like-species pass: A only (B = A)
  const uint32_t *off_a, *off_b;            // per-cell offsets of the last sort
  const uint32_t *skey_a, *skey_b;          // cell of each sorted position
  int sa, sb;                               // species indices; like-species pass: sb = sa
  double m_a, m_b, sigma;
  uint32_t pair_purpose, draw_purpose, scat_purpose;
  int exchange, like, ctr;
  float nWsd1;                              // w_min sigma dt / V_cell in FP32 (screening only)
};

__device__ __forceinline__ double rn3(double a0, double b0, double a1, double b1, double a2, double b2) {
  return __dadd_rn(__dadd_rn(__dmul_rn(a0, b0), __dmul_rn(a1, b1)), __dmul_rn(a2, b2));
}

// R^-1(theta, phi) v = R^T v, R rows (ct cp, ct sp, -st), (-sp, cp, 0), (st cp, st sp, ct)
__device__ void rot_inv(double th, double ph, const double v[3], double out[3]) {
  const double ct = cos(th), st = sin(th), cp = cos(ph), sp = sin(ph);
  out[0] = rn3(ct * cp, v[0], -sp, v[1], st * cp, v[2]);
  out[1] = rn3(ct * sp, v[0], cp, v[1], st * sp, v[2]);
  out[2] = rn3(-st, v[0], 0.0, v[1], ct, v[2]);
}

// eq:du: R^-1(theta,phi) [R^-1(theta',phi') - I] (0,0,u) for u = (ux,uy,uz)
__device__ void delta_u(double ux, double uy, double uz, double cos_tp, double phi_p, double du[3]) {
  const double u = sqrt(rn3(ux, ux, uy, uy, uz, uz));
  double th = 0.0, ph = 0.0;
  if (u > 0) {
    double c = uz / u;
    c = c > 1.0 ? 1.0 : (c < -1.0 ? -1.0 : c);
    th = acos(c);
    ph = atan2(uy, ux);
  }
  const double pole[3] = {0.0, 0.0, u};
  double t[3];
  rot_inv(acos(cos_tp), phi_p, pole, t);
  t[0] -= pole[0]; t[1] -= pole[1]; t[2] -= pole[2];
  rot_inv(th, ph, t, du);
}

// The pair of work item t of a pass (t a sorted SP of species A; for the like pass the
// projectile of its pair).  false if t has no pair.  For an inter-species pass with Na <= Nb
// (ties: A) the SP at place k is the projectile of target (k + o) mod Nb; otherwise it is the
// target of projectile j = (k - o) mod Na of B when j < Nb.  Like pass: places (o + 2m,
// o + 2m + 1) mod N form pair m, the first the projectile.
struct ElPair {
  int64_t ip, it;   // projectile and target index in their species
  bool proj_b;      // projectile in species B
  uint32_t Nt;
};

struct ElItem {
  uint32_t c, oa, Na, ob, Nb;
  bool need;
};

__device__ __forceinline__ ElItem el_item(const ElPass &ps, int64_t t, int64_t hi) {
  ElItem m{};
  if (t >= hi) return m;
  m.c = ps.skey_a[t];
  m.oa = ps.off_a[m.c]; m.Na = ps.off_a[m.c + 1] - m.oa;
  if (ps.like) {
    m.need = m.Na >= 2;
  } else {
    m.ob = ps.off_b[m.c]; m.Nb = ps.off_b[m.c + 1] - m.ob;
    m.need = m.Nb > 0;
  }
  return m;
}

__device__ __forceinline__ bool el_pair_of(const ElPass &ps, const ElItem &m, int64_t t, uint32_t w, ElPair *pr) {
  if (!m.need) return false;
  const uint32_t k = (uint32_t)(t - m.oa);
  if (ps.like) {
    const uint32_t q = (k + m.Na - u_index(w, m.Na)) % m.Na;   // shuffled place of this SP
    if ((q & 1u) || q + 1 >= m.Na) return false;
    pr->ip = t; pr->it = (int64_t)m.oa + (k + 1) % m.Na; pr->proj_b = false; pr->Nt = m.Na;
    return true;
  }
  if (m.Na <= m.Nb) {
    pr->ip = t; pr->it = (int64_t)m.ob + (k + u_index(w, m.Nb)) % m.Nb; pr->proj_b = false; pr->Nt = m.Nb;
    return true;
  }
  const uint32_t j = (k + m.Na - u_index(w, m.Na)) % m.Na;
  if (j >= m.Nb) return false;
  pr->ip = (int64_t)m.ob + j; pr->it = t; pr->proj_b = true; pr->Nt = m.Na;
  return true;
}

// Colliding sub-particles of a pair: #{i < w_p : U_i < P}, capped at w_t.
__device__ int el_ncoll(const ElArgs &a, const ElPass &ps, const ElPair &pr, int64_t step) {
  const SpeciesBuf &A = pr.proj_b ? ps.B : ps.A;
  const SpeciesBuf &B = pr.proj_b ? ps.A : ps.B;
  const int32_t wp = A.w[pr.ip], wt = B.w[pr.it];
  if (wp <= 0 || wt <= 0) return 0;
  const float ax = A.vx[pr.ip], ay = A.vy[pr.ip], az = A.vz[pr.ip];
  const float bx = B.vx[pr.it], by = B.vy[pr.it], bz = B.vz[pr.it];
  const float fx = ax - bx, fy = ay - by, fz = az - bz;
  const float x32 = sqrtf(fx * fx + fy * fy + fz * fz) * ((float)pr.Nt * (float)wt * ps.nWsd1);
  const float P32 = -expm1f(-x32);
  const float band = ldexpf(P32, -12);
  const uint64_t pid = A.id[pr.ip];
  int n = 0;
  bool exact = false;
  for (int i = 0; i < wp && P32 + band >= kUmin; i += 4) {
    const U4 r = rng_block(a.seed, ps.draw_purpose, pid, step, (uint32_t)(i >> 2));
    for (int j = 0; j < 4 && i + j < wp; ++j) {
      const float U = u01f(r.v[j]);
      if (fabsf(U - P32) <= band) exact = true;
      n += U < P32;
    }
  }
  if (exact) {   // the FP64 definition, in the oracle's order of operations
    const double dx = (double)ax - (double)bx, dy = (double)ay - (double)by, dz = (double)az - (double)bz;
    const double u = sqrt(rn3(dx, dx, dy, dy, dz, dz));
    const double P = -expm1(-(u * ((double)pr.Nt / a.V_cell) * ((double)wt * a.w_min) * ps.sigma * a.dt));
    n = 0;
    for (int i = 0; i < wp; i += 4) {
      const U4 r = rng_block(a.seed, ps.draw_purpose, pid, step, (uint32_t)(i >> 2));
      for (int j = 0; j < 4 && i + j < wp; ++j) n += u01d(r.v[j]) < P;
    }
  }
  return n < wt ? n : wt;
}

// New SPs of an event, packed per species of the pass: (in A) | (in B) << 32; the like pass
// counts both in the low half.
__device__ __forceinline__ uint64_t el_products(const ElPass &ps, const ElPair &pr, int n) {
  const SpeciesBuf &A = pr.proj_b ? ps.B : ps.A;
  const SpeciesBuf &B = pr.proj_b ? ps.A : ps.B;
  const uint64_t p_new = n < A.w[pr.ip] ? 1u : 0u, t_new = n < B.w[pr.it] ? 1u : 0u;
  if (ps.like) return p_new + t_new;
  const uint64_t in_a = pr.proj_b ? t_new : p_new, in_b = pr.proj_b ? p_new : t_new;
  return in_a | (in_b << 32);
}

// Work items: the sorted SPs of species A of the pass, in units of kEvUnit taken round-robin
// by warps; events staged with payload N_coll.
__global__ void __launch_bounds__(256) k_el_count(ElArgs a, ElPass ps, EvBlocks ev) {
  const int64_t total = a.clk->n_sorted[ps.sa];
  const int64_t step = a.clk->step;
  const int64_t nunit = (total + kEvUnit - 1) / kEvUnit;
  for (int64_t unit = ev_warp(); unit < nunit; unit += ev_nwarp()) {
    const int64_t lo = unit * kEvUnit, hi = min(total, lo + kEvUnit);
    int64_t run = 0;
    uint64_t prod = 0;
    for (int64_t base = lo; base < hi; base += 32) {
      const int64_t t = base + (threadIdx.x & 31);
      const ElItem m = el_item(ps, t, hi);
      const uint32_t w = cell_word(a.seed, ps.pair_purpose, m.c, m.need, step);
      ElPair pr;
      int n = 0;
      uint64_t pc = 0;
      if (el_pair_of(ps, m, t, w, &pr)) {
        n = el_ncoll(a, ps, pr, step);
        if (n > 0) pc = el_products(ps, pr, n);
      }
      ev_stage(ev, lo, &run, &prod, t, (uint32_t)n, pc);
    }
    if ((threadIdx.x & 31) == 0) {
      ev.hits[unit] = (int)run;
      ev.cnt[unit] = prod;
    }
  }
}

// capacity check of a pass's new SPs (packed as in el_products)
__global__ void k_el_check(DevClock *clk, const uint64_t *total, int sa, int sb, int like, int64_t cap_a, int64_t cap_b,
                           int *go) {
  const uint64_t t = *total;
  const int64_t na = (int64_t)(t & 0xffffffffu), nb = like ? 0 : (int64_t)(t >> 32);
  const bool ok = clk->n[sa] + na <= cap_a && (like || clk->n[sb] + nb <= cap_b);
  *go = ok ? 1 : 0;
  if (!ok) atomicOr(&clk->err, kErrCapacity);
}

__global__ void k_el_commit(DevClock *clk, const uint64_t *total, const int *go, int sa, int sb, int like) {
  if (!*go) return;
  const uint64_t t = *total;
  const int64_t na = (int64_t)(t & 0xffffffffu), nb = like ? 0 : (int64_t)(t >> 32);
  clk->n[sa] += na;
  if (!like) clk->n[sb] += nb;
  clk->next_id += na + nb;
}

// Events of the staged pairs, unit by unit in item order: the FP64 velocities, the turned or
// split SPs and the new ones.
__global__ void __launch_bounds__(256) k_el_products(ElArgs a, ElPass ps, EvBlocks ev) {
  if (!*a.go) return;
  const int64_t total = a.clk->n_sorted[ps.sa];
  const int64_t step = a.clk->step, id_base = a.clk->next_id;
  const int64_t n_a = a.clk->n[ps.sa], n_b = a.clk->n[ps.sb];
  const int64_t nunit = (total + kEvUnit - 1) / kEvUnit;
  int events = 0;
  for (int64_t unit = ev_warp(); unit < nunit; unit += ev_nwarp()) {
    const int64_t lo = unit * kEvUnit;
    const int nh = ev.hits[unit];
    uint64_t run = ev.off[unit];
    for (int base = 0; base < nh; base += 32) {
      const int i = base + (threadIdx.x & 31);
      ElPair pr{};
      int n = 0;
      uint64_t pc = 0;
      if (i < nh) {
        const uint64_t rec = ev.rec[lo + i];
        const int64_t t = (int64_t)(uint32_t)rec;
        n = (int)(rec >> 32);
        const ElItem m = el_item(ps, t, total);
        el_pair_of(ps, m, t, rng_block(a.seed, ps.pair_purpose, m.c, step, 0).v[0], &pr);
        pc = el_products(ps, pr, n);
      }
      uint64_t tile;
      const uint64_t off = run + warp_scan_u64(pc, &tile);
      run += tile;
      if (i >= nh) continue;
      ++events;
      SpeciesBuf &A = pr.proj_b ? ps.B : ps.A;
      SpeciesBuf &B = pr.proj_b ? ps.A : ps.B;
      const int64_t ip = pr.ip, it = pr.it;
      const float ax = A.vx[ip], ay = A.vy[ip], az = A.vz[ip];
      const float bx = B.vx[it], by = B.vy[it], bz = B.vz[it];
      float na[3], nb[3];
      if (ps.exchange) {
        na[0] = bx; na[1] = by; na[2] = bz;
        nb[0] = ax; nb[1] = ay; nb[2] = az;
      } else {
        const U4 r = rng_block(a.seed, ps.scat_purpose, A.id[ip], step, 0);
        const double mA = pr.proj_b ? ps.m_b : ps.m_a, mB = pr.proj_b ? ps.m_a : ps.m_b;
        double du[3];
        delta_u((double)ax - (double)bx, (double)ay - (double)by, (double)az - (double)bz, 2.0 * u01d(r.v[0]) - 1.0,
                2.0 * kPi * u01d(r.v[1]), du);
        const double mu = mA * mB / (mA + mB);
        const double ka = mu / mA, kb = mu / mB;
        na[0] = (float)((double)ax + ka * du[0]); na[1] = (float)((double)ay + ka * du[1]);
        na[2] = (float)((double)az + ka * du[2]);
        nb[0] = (float)((double)bx - kb * du[0]); nb[1] = (float)((double)by - kb * du[1]);
        nb[2] = (float)((double)bz - kb * du[2]);
      }
      // slots: the running offsets of species A (low half) and B (high half); the like pass
      // keeps both sides in the low half, projectile first
      int64_t off_a = (int64_t)(off & 0xffffffffu), off_b = (int64_t)(off >> 32);
      int64_t id = id_base + off_a + off_b;
      const int32_t wp = A.w[ip], wt = B.w[it];
      auto place = [&](SpeciesBuf &S, int64_t idx, int32_t w, const float v[3], bool in_b) {
        if (n == w) {
          S.vx[idx] = v[0]; S.vy[idx] = v[1]; S.vz[idx] = v[2];
          return;
        }
        S.w[idx] = w - n;
        const int64_t slot = in_b ? n_b + off_b++ : n_a + off_a++;
        put_sp(S, slot, S.x[idx], S.y[idx], S.z[idx], v[0], v[1], v[2], n, (uint64_t)id++);
      };
      const bool p_in_b = ps.like ? false : pr.proj_b, t_in_b = ps.like ? false : !pr.proj_b;
      place(A, ip, wp, na, p_in_b);
      place(B, it, wt, nb, t_in_b);
    }
  }
  for (int o = 16; o > 0; o >>= 1) events += __shfl_down_sync(0xffffffffu, events, o);
  if ((threadIdx.x & 31) == 0 && events) atomicAdd((unsigned long long *)&a.clk->ctr[ps.ctr], (unsigned long long)events);
}

// ---- Coulomb collisions ---------------------------------------------------------------------
// e-e, e-Cu+ and Cu+-Cu+ by the binary small-angle method the paper cites (Table colls): every
// pair turns its relative velocity u by theta, with delta = tan(theta/2) normal of variance
// <delta^2> = q_a^2 q_b^2 n lnL dt / (8 pi eps0^2 m_ab^2 u^3) (n the target density n_t W_t as in
// eq:colp) and a uniform azimuth; the velocity difference is eq:du and eq:newv gives the new
// velocities.  Whole SPs turn (the lighter always, the heavier with probability w_s/w_l, tested
// in integers).  No decision depends on floating point, so the turn is computed in FP32: sin and
// cos of theta from delta directly (no cancellation at small angles), the azimuth and the
// Box-Muller angle by sincospif.  Pairings as for the elastic passes.
struct CoPass {
  ElPass ps;        // species, offsets, sort keys, pairing purpose, like flag
  float K;          // q_a^2 q_b^2 lnL dt w_min / (8 pi eps0^2 m_ab^2 V_cell): <delta^2> = K Nt W_t / u^3
  float ka, kb;     // m_ab / m_a, m_ab / m_b of species A and B of the pass
  uint32_t draw_purpose;
};

__device__ __forceinline__ void co_turn(const CoPass &cp, const ElPair &pr, int64_t step, uint64_t seed, int *hits) {
  const ElPass &ps = cp.ps;
  SpeciesBuf A = pr.proj_b ? ps.B : ps.A;
  SpeciesBuf B = pr.proj_b ? ps.A : ps.B;
  const int32_t wa = A.w[pr.ip], wb = B.w[pr.it];
  if (wa <= 0 || wb <= 0) return;
  const float ax = A.vx[pr.ip], ay = A.vy[pr.ip], az = A.vz[pr.ip];
  const float bx = B.vx[pr.it], by = B.vy[pr.it], bz = B.vz[pr.it];
  const float ux = ax - bx, uy = ay - by, uz = az - bz;
  const float u2 = ux * ux + uy * uy + uz * uz;
  if (u2 == 0.0f) return;
  const float u = sqrtf(u2);
  float d2 = cp.K * (float)pr.Nt * (float)wb / (u2 * u);
  if (!(d2 < 1e30f)) d2 = 1e30f;
  const U4 r = rng_block(seed, cp.draw_purpose, A.id[pr.ip], step, 0);
  const float g = sqrtf(-2.0f * logf(u01f(r.v[0]))) * cospif(2.0f * u01f(r.v[1]));
  const float dd = d2 * g * g;                          // delta^2 of this pair
  const float sin_t = 2.0f * sqrtf(dd) / (1.0f + dd);   // |sin theta|
  const float cm1 = -2.0f * dd / (1.0f + dd);           // cos theta - 1
  float sp, cpf;
  sincospif(2.0f * u01f(r.v[2]), &sp, &cpf);
  // [R^-1(theta, phi) - I] (0, 0, u), then R^-1 of the angles of u
  const float v0 = u * sin_t * cpf, v1 = u * sin_t * sp, v2 = u * cm1;
  const float uperp = sqrtf(ux * ux + uy * uy);
  const float ct = uz / u, st = uperp / u;
  const float cph = uperp > 0.0f ? ux / uperp : 1.0f, sph = uperp > 0.0f ? uy / uperp : 0.0f;
  const float dux = ct * cph * v0 - sph * v1 + st * cph * v2;
  const float duy = ct * sph * v0 + cph * v1 + st * sph * v2;
  const float duz = -st * v0 + ct * v2;
  const float ka = pr.proj_b ? cp.kb : cp.ka, kb = pr.proj_b ? cp.ka : cp.kb;
  const bool a_small = wa <= wb;
  const uint64_t ws = (uint64_t)(a_small ? wa : wb), wl = (uint64_t)(a_small ? wb : wa);
  const bool large_too = (2ull * (r.v[3] >> 8) + 1ull) * wl < (ws << 25);
  if (a_small || large_too) { A.vx[pr.ip] = ax + ka * dux; A.vy[pr.ip] = ay + ka * duy; A.vz[pr.ip] = az + ka * duz; }
  if (!a_small || large_too) { B.vx[pr.it] = bx - kb * dux; B.vy[pr.it] = by - kb * duy; B.vz[pr.it] = bz - kb * duz; }
  ++*hits;
}

// One pass: one item per sorted SP of species A (whole warps: the cell's pairing word is shared).
__global__ void __launch_bounds__(256, 4) k_coulomb(CoPass cp, uint64_t seed, DevClock *clk, int ctr) {
  const ElPass &ps = cp.ps;
  const int64_t n = clk->n_sorted[ps.sa];
  const int64_t step = clk->step;
  const int64_t span = (n + 31) & ~31ll;
  int hits = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < span; t += (int64_t)gridDim.x * blockDim.x) {
    const ElItem m = el_item(ps, t, n);
    const uint32_t w = cell_word(seed, ps.pair_purpose, m.c, m.need, step);
    ElPair pr;
    if (el_pair_of(ps, m, t, w, &pr)) co_turn(cp, pr, step, seed, &hits);
  }
  for (int o = 16; o > 0; o >>= 1) hits += __shfl_down_sync(0xffffffffu, hits, o);
  if ((threadIdx.x & 31) == 0 && hits) atomicAdd((unsigned long long *)&clk->ctr[ctr], (unsigned long long)hits);
}

// ---- direct field ionization -----------------------------------------------------------------
struct DfiArgs {
  SpeciesBuf n, e, ions;
  const float4 *E;
  int nx, ny;
  double dt_fs, pre, c1, c2, expo, lim2;   // rate = pre (c1/E)^expo exp(-c2/E), E in GV/m
  float lim2f;                             // lim2 in FP32 (screening of the barrier-suppression test)
  float E2skip;                            // |E|^2 below which P dt < 2^-27: no draw can ionize
  uint64_t seed;
  DevClock *clk;
  int *go;
};

// Sub-particles of neutral t that ionize this step.
__device__ int dfi_nion(const DfiArgs &a, int64_t t, int64_t step) {
  const int w = a.n.w[t];
  if (w <= 0) return 0;
  const float3 e = gather_E(a.E, a.n.x[t], a.n.y[t], a.n.z[t], a.nx, a.ny);
  // |E|^2 is defined in FP64 (the oracle's sum of the three exact squares).  It is formed in
  // FP32 first (within a few ulp) and in FP64 only where the barrier-suppression decision is
  // close; P32 below only places the guard band, inside which the draw is re-decided from
  // the FP64 |E|^2.
  const float E2f = fmaf(e.x, e.x, fmaf(e.y, e.y, e.z * e.z));
  if (E2f < a.E2skip) return 0;
  const bool near_bsi = fabsf(E2f - a.lim2f) <= 1e-5f * a.lim2f;
  double E2 = (double)E2f;
  if (near_bsi)
    E2 = __dadd_rn(__dadd_rn(__dmul_rn((double)e.x, (double)e.x), __dmul_rn((double)e.y, (double)e.y)),
                   __dmul_rn((double)e.z, (double)e.z));
  if (E2 > a.lim2) return w;
  int k = 0;
  const float Eg = sqrtf(E2f) * 1e-9f;
  const float P32 = (float)a.pre * powf((float)a.c1 / Eg, (float)a.expo) * expf(-(float)a.c2 / Eg) * (float)a.dt_fs;
  const float band = ldexpf(P32, -12);
  const uint64_t id = a.n.id[t];
  bool exact = false;
  for (int i = 0; i < w && P32 + band >= kUmin; i += 4) {
    const U4 r = rng_block(a.seed, kDfi, id, step, (uint32_t)(i >> 2));
    for (int j = 0; j < 4 && i + j < w; ++j) {
      const float U = u01f(r.v[j]);
      if (fabsf(U - P32) <= band) exact = true;
      k += U < P32;
    }
  }
  if (exact) {
    const double E2d = __dadd_rn(__dadd_rn(__dmul_rn((double)e.x, (double)e.x), __dmul_rn((double)e.y, (double)e.y)),
                                 __dmul_rn((double)e.z, (double)e.z));
    const double Ed = sqrt(E2d) * 1e-9;
    const double P64 = a.pre * pow(a.c1 / Ed, a.expo) * exp(-a.c2 / Ed) * a.dt_fs;
    k = 0;
    for (int i = 0; i < w; i += 4) {
      const U4 r = rng_block(a.seed, kDfi, id, step, (uint32_t)(i >> 2));
      for (int j = 0; j < 4 && i + j < w; ++j) k += u01d(r.v[j]) < P64;
    }
  }
  return k;
}

__global__ void __launch_bounds__(256) k_dfi_count(DfiArgs a, EvBlocks ev) {
  const int64_t nn = a.clk->n[PIC_NEUTRAL];
  const int64_t step = a.clk->step;
  const int64_t nunit = (nn + kEvUnit - 1) / kEvUnit;
  for (int64_t unit = ev_warp(); unit < nunit; unit += ev_nwarp()) {
    const int64_t lo = unit * kEvUnit, hi = min(nn, lo + kEvUnit);
    int64_t run = 0;
    uint64_t prod = 0;
    for (int64_t base = lo; base < hi; base += 32) {
      const int64_t t = base + (threadIdx.x & 31);
      const int k = t < hi ? dfi_nion(a, t, step) : 0;
      ev_stage(ev, lo, &run, &prod, t, (uint32_t)k, k > 0 ? (1ull | (1ull << 32)) : 0ull);
    }
    if ((threadIdx.x & 31) == 0) {
      ev.hits[unit] = (int)run;
      ev.cnt[unit] = prod;
    }
  }
}

// Products: an ion with the neutral's state and an electron at rest, ion then electron id.
__global__ void __launch_bounds__(256) k_dfi_products(DfiArgs a, EvBlocks ev) {
  if (!*a.go) return;
  const int64_t nn = a.clk->n[PIC_NEUTRAL], ne = a.clk->n[PIC_ELECTRON], ni = a.clk->n[PIC_ION];
  const int64_t id_base = a.clk->next_id;
  const int64_t nunit = (nn + kEvUnit - 1) / kEvUnit;
  for (int64_t unit = ev_warp(); unit < nunit; unit += ev_nwarp()) {
    const int64_t lo = unit * kEvUnit;
    const int nh = ev.hits[unit];
    uint64_t run = ev.off[unit];
    for (int base = 0; base < nh; base += 32) {
      const int i = base + (threadIdx.x & 31);
      const uint64_t pc = i < nh ? (1ull | (1ull << 32)) : 0ull;
      uint64_t tile;
      const uint64_t off = run + warp_scan_u64(pc, &tile);
      run += tile;
      if (i >= nh) continue;
      const uint64_t rec = ev.rec[lo + i];
      const int64_t t = (int64_t)(uint32_t)rec;
      const int k = (int)(rec >> 32);
      const int64_t io = (int64_t)(off & 0xffffffffu), eo = (int64_t)(off >> 32);
      const int64_t id = id_base + io + eo;
      put_sp(a.ions, ni + io, a.n.x[t], a.n.y[t], a.n.z[t], a.n.vx[t], a.n.vy[t], a.n.vz[t], k, (uint64_t)id);
      put_sp(a.e, ne + eo, a.n.x[t], a.n.y[t], a.n.z[t], 0.f, 0.f, 0.f, k, (uint64_t)(id + 1));
      a.n.w[t] -= k;
    }
  }
}

// |E|^2 [V^2/m^2] below which the ADK probability per step is under 2^-27 (the rate rises with
// E below the barrier-suppression limit): there no 24-bit draw (>= 2^-25) can fall under P, so
// those neutrals are skipped without evaluating the rate.  FP64 bisection, rounded down.
static float dfi_skip_E2(const DfiArgs &d, double lim) {
  auto P = [&](double E) { const double Eg = E * 1e-9; return d.pre * pow(d.c1 / Eg, d.expo) * exp(-d.c2 / Eg) * d.dt_fs; };
  const double target = ldexp(1.0, -27);
  if (P(lim) <= target) return (float)(d.lim2 * (1.0 - 1e-4));
  double lo = 1e6, hi = lim;
  for (int it = 0; it < 200 && hi - lo > 1e-9 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    (P(mid) < target ? lo : hi) = mid;
  }
  return (float)(lo * lo * (1.0 - 1e-5));
}

int stage_collide(pic_t *h) {
  const uint32_t fl = h->prm.flags;
  int *go = h->long_n + 4;
  uint64_t *total = (uint64_t *)(h->tmp_len + 2);
  const int grid = h->nsm * 8;
  // events of the count kernels are staged per unit of 256 work items in the collision scratch
  const EvBlocks ev{h->pair_cnt, h->ev_hits, h->ev_cnt, h->ev_off, h->ev_cnt2, h->ev_off2};
  const bool ion2 = nsp_active(h) > PIC_ION2;
  uint64_t *total2 = (uint64_t *)(h->tmp_len + 3);
  // one impact-ionization pass: electrons on the target species sn, products of species sprod
  auto mcc_pass = [&](int sn, int sprod, double xi, double lotz, uint32_t pp, uint32_t pd, uint32_t ps, int dbl,
                      int ctr, int units_mode, int kid_count, int kid_products) -> int {
    McArgs a{};
    const Species &E = h->sp[PIC_ELECTRON], &N = h->sp[sn];
    a.e = E.a; a.n = N.a; a.prod = h->sp[sprod].a; a.j = h->sp[PIC_ION2].a;
    a.off_e = E.off; a.off_n = N.off; a.skey_e = E.skey; a.skey_n = N.skey;
    a.V_cell = h->dx * h->dx * h->dx; a.dt = h->prm.dt; a.w_min = h->prm.w_min; a.seed = h->prm.seed;
    a.xi = xi; a.lotz = lotz; a.xi32 = (float)xi; a.lotz32 = (float)lotz;
    double peak = lotz / (2.718281828459045 * xi * xi);
    if (dbl) peak += kLotzDouble / (2.718281828459045 * kXiDouble * kXiDouble);
    a.sig_peak = (float)peak;
    a.pur_pair = pp; a.pur_draw = pd; a.pur_scat = ps;
    a.sn = sn; a.sprod = sprod; a.dbl = dbl;
    a.clk = h->clock; a.go = go; a.total1 = total;
    h->nlaunch += 4;
    { KtScope kt_(h, kid_count, 0); k_mcc_count<<<grid, 256, 0, h->stream>>>(a, ev); }
    k_ev_units<<<1, 1, 0, h->stream>>>(h->tmp_len, h->clock, units_mode);
    PIC_TRY(scan_u64(h, ev.cnt, ev.off, 0, h->tmp_len, total));
    if (dbl) PIC_TRY(scan_u64(h, ev.cnt2, ev.off2, 0, h->tmp_len, total2));
    k_mcc_check<<<1, 1, 0, h->stream>>>(h->clock, total, dbl ? total2 : nullptr, sprod, h->sp[sprod].cap, E.cap,
                                        h->sp[PIC_ION2].cap, go);
    { KtScope kt_(h, kid_products, 0); k_mcc_products<<<grid, 256, 0, h->stream>>>(a, ev); }
    k_mcc_commit<<<1, 1, 0, h->stream>>>(h->clock, total, dbl ? total2 : nullptr, go, sprod, ctr);
    return launch_check(h, "mcc");
  };
  if (fl & PIC_F_IMPACT_ION) {
    PIC_TRY(mcc_pass(PIC_NEUTRAL, PIC_ION, kXiCu, kLotzA, kPair, kIon, kScat, ion2 ? 1 : 0, cImpactIon, 0, kidMccCount,
                     kidMccProducts));
    if (ion2)   // Cu+ + e -> Cu2+ + 2e on the Cu+ as the single pass left them
      PIC_TRY(mcc_pass(PIC_ION, PIC_ION2, kXi2Cu, kLotzIz, kPairIz, kIonIz, kScatIz, 0, cIonIon, 6, kidMccCount,
                       kidMccProducts));
  }
  if (fl & PIC_F_ELASTIC) {
    ElArgs a{};
    a.V_cell = h->dx * h->dx * h->dx; a.dt = h->prm.dt; a.w_min = h->prm.w_min; a.seed = h->prm.seed;
    a.clk = h->clock; a.go = go;
    const Species &E = h->sp[PIC_ELECTRON], &N = h->sp[PIC_NEUTRAL], &I = h->sp[PIC_ION];
    auto pass = [&](const Species &A, int sa, const Species &B, int sb, double sigma, uint32_t pp, uint32_t dp,
                    uint32_t sp_, int ex, int like, int ctr) {
      ElPass ps{};
      ps.A = A.a; ps.B = B.a; ps.off_a = A.off; ps.off_b = B.off; ps.skey_a = A.skey; ps.skey_b = B.skey;
      ps.sa = sa; ps.sb = sb; ps.m_a = A.mass; ps.m_b = B.mass; ps.sigma = sigma;
      ps.pair_purpose = pp; ps.draw_purpose = dp; ps.scat_purpose = sp_; ps.exchange = ex; ps.like = like; ps.ctr = ctr;
      ps.nWsd1 = (float)(h->prm.w_min * sigma * h->prm.dt / a.V_cell);
      return ps;
    };
    const ElPass passes[3] = {
        pass(E, PIC_ELECTRON, N, PIC_NEUTRAL, h->sigma_el_en, kPairEn, kDrawEn, kScatEn, 0, 0, cElasticEn),
        pass(N, PIC_NEUTRAL, N, PIC_NEUTRAL, h->sigma_el_nn, kPairNn, kDrawNn, kScatNn, 0, 1, cElasticNn),
        pass(I, PIC_ION, N, PIC_NEUTRAL, h->sigma_cx, kPairCx, kDrawCx, 0, 1, 0, cChargeEx)};
    for (int p = 0; p < 3; ++p) {
      const ElPass &ps = passes[p];
      h->nlaunch += 4;
      { KtScope kt_(h, kidElastic, 0); k_el_count<<<grid, 256, 0, h->stream>>>(a, ps, ev); }
      k_ev_units<<<1, 1, 0, h->stream>>>(h->tmp_len, h->clock, 2 + ps.sa);
      PIC_TRY(scan_u64(h, ev.cnt, ev.off, 0, h->tmp_len, total));
      k_el_check<<<1, 1, 0, h->stream>>>(h->clock, total, ps.sa, ps.sb, ps.like, h->sp[ps.sa].cap, h->sp[ps.sb].cap, go);
      { KtScope kt_(h, kidElastic, 0); k_el_products<<<grid, 256, 0, h->stream>>>(a, ps, ev); }
      k_el_commit<<<1, 1, 0, h->stream>>>(h->clock, total, go, ps.sa, ps.sb, ps.like);
    }
    PIC_TRY(launch_check(h, "elastic"));
  }
  if (fl & PIC_F_COULOMB) {
    const Species &E = h->sp[PIC_ELECTRON], &I = h->sp[PIC_ION];
    const double lnL = h->prm.coulomb_log > 0 ? h->prm.coulomb_log : 10.0;
    auto pass = [&](const Species &A, int sa, const Species &B, int sb, double qa, double qb, uint32_t pp, uint32_t dp,
                    int like) {
      CoPass cp{};
      ElPass &ps = cp.ps;
      ps.A = A.a; ps.B = B.a; ps.off_a = A.off; ps.off_b = B.off; ps.skey_a = A.skey; ps.skey_b = B.skey;
      ps.sa = sa; ps.sb = sb; ps.m_a = A.mass; ps.m_b = B.mass; ps.pair_purpose = pp; ps.like = like;
      const double mab = A.mass * B.mass / (A.mass + B.mass);
      const double V = h->dx * h->dx * h->dx;
      cp.K = (float)(qa * qa * qb * qb * lnL * h->prm.dt * h->prm.w_min / (8.0 * kPi * kEps0 * kEps0 * mab * mab * V));
      cp.ka = (float)(mab / A.mass); cp.kb = (float)(mab / B.mass);
      cp.draw_purpose = dp;
      return cp;
    };
    const CoPass ee = pass(E, PIC_ELECTRON, E, PIC_ELECTRON, kQe, kQe, kPairEe, kDrawEe, 1);
    const CoPass ei = pass(E, PIC_ELECTRON, I, PIC_ION, kQe, kQe, kPairEi, kDrawEi, 0);
    const CoPass ii = pass(I, PIC_ION, I, PIC_ION, kQe, kQe, kPairIi, kDrawIi, 1);
    h->nlaunch += 3;
    {
      KtScope kt_(h, kidCoulomb, 0);
      k_coulomb<<<grid, 256, 0, h->stream>>>(ee, h->prm.seed, h->clock, cCoulombEe);
      k_coulomb<<<grid, 256, 0, h->stream>>>(ei, h->prm.seed, h->clock, cCoulombEi);
      k_coulomb<<<grid, 256, 0, h->stream>>>(ii, h->prm.seed, h->clock, cCoulombIi);
    }
    if (ion2) {   // with Cu2+: e-Cu2+, Cu+-Cu2+, Cu2+-Cu2+ (Sec. 2.2: between all charged species)
      const Species &J = h->sp[PIC_ION2];
      const CoPass ej = pass(E, PIC_ELECTRON, J, PIC_ION2, kQe, 2.0 * kQe, kPairEj, kDrawEj, 0);
      const CoPass ij = pass(I, PIC_ION, J, PIC_ION2, kQe, 2.0 * kQe, kPairIj, kDrawIj, 0);
      const CoPass jj = pass(J, PIC_ION2, J, PIC_ION2, 2.0 * kQe, 2.0 * kQe, kPairJj, kDrawJj, 1);
      h->nlaunch += 3;
      KtScope kt_(h, kidCoulomb, 0);
      k_coulomb<<<grid, 256, 0, h->stream>>>(ej, h->prm.seed, h->clock, cCoulombEj);
      k_coulomb<<<grid, 256, 0, h->stream>>>(ij, h->prm.seed, h->clock, cCoulombIj);
      k_coulomb<<<grid, 256, 0, h->stream>>>(jj, h->prm.seed, h->clock, cCoulombJj);
    }
    PIC_TRY(launch_check(h, "coulomb"));
  }
  if (fl & PIC_F_DFI) {
    DfiArgs d;
    d.n = h->sp[PIC_NEUTRAL].a; d.e = h->sp[PIC_ELECTRON].a; d.ions = h->sp[PIC_ION].a;
    d.E = h->E; d.nx = h->nx; d.ny = h->ny;
    const double xi = kXiCu, nstar = 3.69 / sqrt(xi), x15 = pow(xi, 1.5);
    d.pre = 1.52 * pow(4.0, nstar) * xi / (nstar * tgamma(2.0 * nstar));
    d.c1 = 20.5 * x15; d.c2 = 6.83 * x15; d.expo = 2.0 * nstar - 1.0;
    const double lim = 1.5 * x15 * 1e9;
    d.lim2 = lim * lim;
    d.lim2f = (float)d.lim2;
    d.dt_fs = h->prm.dt * 1e15; d.seed = h->prm.seed; d.clk = h->clock; d.go = go;
    d.E2skip = dfi_skip_E2(d, lim);
    h->nlaunch += 4;
    { KtScope kt_(h, kidDfiCount, 0); k_dfi_count<<<grid, 256, 0, h->stream>>>(d, ev); }
    k_ev_units<<<1, 1, 0, h->stream>>>(h->tmp_len, h->clock, 1);
    PIC_TRY(scan_u64(h, ev.cnt, ev.off, 0, h->tmp_len, total));
    k_check_new<<<1, 1, 0, h->stream>>>(h->clock, total, h->sp[PIC_ION].cap, h->sp[PIC_ELECTRON].cap, go);
    { KtScope kt_(h, kidDfiProducts, 0); k_dfi_products<<<grid, 256, 0, h->stream>>>(d, ev); }
    k_commit_new<<<1, 1, 0, h->stream>>>(h->clock, total, go, cFieldIon);
    PIC_TRY(launch_check(h, "dfi"));
  }
  return PIC_OK;
}

}  // namespace pic
