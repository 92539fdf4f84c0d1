/*
 * pic.h -- C ABI of the GB300 vacuum-arc PIC-MCC step (libpic.so).
 *
 * The library advances the coupled plasma step of Koitermaa et al., "Simulating vacuum arc
 * initiation by coupling emission, heating and plasma processes" (arXiv:2402.08404): thermal-
 * field emission from every exposed cathode face (Sec. 2.3.1), evaporation and sputter
 * injection (Sec. 2.3.1-2.3.3), field gather and leapfrog push with boundary removal
 * (Sec. 2.2), cell sort, impact-ionization MCC with SP splitting (eq:colp, eq:du, Sec. 2.3.2),
 * direct field ionization (eq:dfi), charge deposition and the Poisson solve (eq:poi,
 * eq:bcf1-3), and the tip heat equation with Joule heating (eq:heat, eq:cont) every n_heat steps.
 * Equations are cited by their LaTeX labels in the paper.
 *
 * Geometry: an nx*ny*nz Cartesian grid of cells of size dx [m]; the cathode plane is z=0
 * (phi = 0), the anode plane z = nz*dx (phi = V0), the lateral walls carry zero normal field;
 * a Cu tip (cylinder + hemispherical cap on the axis x = nx/2, y = ny/2) is made of solid cells
 * whose centres lie inside it; all corners of solid cells are held at phi = 0.
 *
 * Species are indexed PIC_ELECTRON = 0, PIC_NEUTRAL = 1 (Cu), PIC_ION = 2 (Cu+), PIC_ION2 = 3
 * (Cu2+, present while PIC_F_ION2 is set: Table colls and Sec. 2.2).  Every SP has a
 * position in cell units (x/dx, float), a velocity [m/s] (float), a weight in units of w_min
 * (int32) and a 64-bit id that keys all its random draws (Philox4x32-10).
 *
 * Ownership.  The library owns all device state.  Device memory is taken through the
 * caller's allocator callbacks (pic_alloc_fn/pic_free_fn; NULL selects cudaMalloc/cudaFree),
 * kernels run on the caller's stream (a cudaStream_t passed as void*; NULL = legacy stream).
 * Unless stated otherwise, array arguments are HOST pointers owned by the caller; the call
 * copies them synchronously.
 *
 * Errors.  Every int-returning call returns PIC_OK (0) or a negative PIC_E_* code and records a
 * message readable through pic_last_error().  After PIC_E_CUDA the handle should be destroyed.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_OK 0
#define PIC_E_INVALID (-1)   /* bad argument or size */
#define PIC_E_CAPACITY (-2)  /* an SP count or a per-cell count would exceed its capacity */
#define PIC_E_NOCONV (-3)    /* Poisson solve did not reach mg_tol within mg_max_cycles */
#define PIC_E_TIMEOUT (-4)   /* a bounded device wait gave up */
#define PIC_E_CUDA (-5)      /* a CUDA runtime call failed */

#define PIC_ELECTRON 0
#define PIC_NEUTRAL 1
#define PIC_ION 2
#define PIC_ION2 3
#define PIC_NSPECIES 4

/* flags of pic_params_t */
#define PIC_F_EMISSION 0x01u    /* a1: thermal-field emission */
#define PIC_F_EVAP 0x02u        /* a2: evaporation */
#define PIC_F_SPUTTER 0x04u     /* a2: sputter injection from ion impacts */
#define PIC_F_IMPACT_ION 0x08u  /* a5: impact ionization MCC */
#define PIC_F_DFI 0x10u         /* a6: direct field ionization */
#define PIC_F_HEAT 0x20u        /* a10: heat + Joule every n_heat steps */
#define PIC_F_SURROGATE 0x40u   /* a1 uses the trained MLP where it is inside its validated range */
#define PIC_F_MIXED_MG 0x80u    /* a8: FP32 V-cycles with FP64 residual refinement (else FP64 V-cycles) */
#define PIC_F_FAST_INTEGRAL 0x100u  /* a1: Gamow quadrature and turning points in FP32 (J, P_N to ~1e-5
                                       relative) in the step and in pic_emission_eval; else all FP64 */
#define PIC_F_GRAPH 0x200u      /* pic_step replays a CUDA graph of one step (the Poisson loop a device-side
                                   while node); the first call with new flags runs one step eagerly and
                                   records the graph; results equal the eager form's bit for bit */
#define PIC_F_CIRCUIT 0x400u    /* the RC circuit drives the anode (needs circuit_R, circuit_C > 0 at create) */
#define PIC_F_ELASTIC 0x800u    /* a5: then elastic e-Cu and Cu-Cu collisions and Cu+-Cu charge exchange */
#define PIC_F_EXTRAPOLATE 0x1000u /* pic_step starts each solve from 2 phi^n - phi^(n-1) instead of phi^n */
#define PIC_F_COULOMB 0x2000u   /* a5: then e-e, e-Cu+, Cu+-Cu+ Coulomb collisions (binary small-angle method) */
#define PIC_F_MERGE 0x4000u     /* a4: after the sort, SP merging in cells above merge_max SPs of a species */
#define PIC_F_ION2 0x8000u      /* Cu2+ (species PIC_ION2) and the Cu2+ channels of Table colls: with
                                   PIC_F_IMPACT_ION double ionization Cu + e -> Cu2+ + 3e competing with
                                   single ionization by the total cross section, then Cu+ + e -> Cu2+ + 2e;
                                   with PIC_F_COULOMB also e-Cu2+, Cu+-Cu2+, Cu2+-Cu2+ Coulomb passes.
                                   Cu2+ SPs are pushed, sorted, merged, deposited (charge 2), counted in
                                   the gap current and sputter on impact like Cu+.  Stand-in Lotz cross
                                   sections: a = 4.5e-15 cm^2 eV^2 at xi_1 + xi_2 = 28.018 eV (double),
                                   a = 4.5e-13 cm^2 eV^2 at xi_2 = 20.292 eV (Cu+) */
#define PIC_F_ALL 0xFFu         /* every stage, surrogate and mixed-precision solve; not FAST_INTEGRAL and
                                   none of the opt-in flags 0x200-0x8000 */

typedef struct {
  double tip_radius; /* m */
  double tip_height; /* m, including the hemispherical cap */
} pic_geometry_t;

typedef struct {
  int nx, ny, nz; /* cells; nx, ny, nz must be even */
  double dx;      /* m */
} pic_grid_t;

typedef struct {
  int charge_e;     /* charge number: -1, 0, +1, +2 */
  double mass;      /* kg */
  int64_t capacity; /* maximum number of SPs held */
} pic_species_t;

typedef struct {
  double dt;            /* PIC time step [s] */
  double apex_field;    /* V/m: V0 is calibrated at create so the apex face field equals this */
  double V0;            /* V: if > 0, used as the anode potential and no calibration is done */
  double T0;            /* ambient / initial tip temperature [K] */
  double work_function; /* eV */
  double w_min;         /* real particles per weight unit (Sec. 2.3.2) */
  int w_max_units;      /* maximum injection weight in units of w_min */
  int n_heat;           /* heat step every n_heat PIC steps (dt_heat = n_heat dt); 0 = never */
  uint64_t seed;        /* Philox key */
  uint32_t flags;       /* PIC_F_* */
  double mg_tol;        /* relative residual target of the Poisson solve */
  int mg_max_cycles;    /* cap on refinement cycles per solve */
  int mg_sweeps;        /* red-black sweeps before and after each coarse-grid correction (<= 0: 3) */
  double circuit_R;     /* Ohm: external resistance of the RC circuit (with circuit_C > 0: allocates the
                           unit Laplace field; the circuit acts while PIC_F_CIRCUIT is set) */
  double circuit_C;     /* F: gap capacitance of the RC circuit */
  double sigma_el_en;   /* m^2: e-Cu elastic cross section (<= 0: 1e-19, a constant stand-in) */
  double sigma_el_nn;   /* m^2: Cu-Cu elastic cross section (<= 0: hard spheres pi (2 x 128 pm)^2) */
  double sigma_cx;      /* m^2: Cu+-Cu charge exchange cross section (<= 0: 5e-19, a constant stand-in) */
  double coulomb_log;   /* Coulomb logarithm of the Coulomb collisions (<= 0: 10) */
  int merge_max;        /* SPs of a species per cell above which pairs merge (PIC_F_MERGE; <= 0: 32) */
} pic_params_t;

typedef struct {
  int64_t step, next_id;
  int64_t count[PIC_NSPECIES];          /* SPs held per species */
  int64_t weight[PIC_NSPECIES];         /* sum of weights per species (units of w_min) */
  int64_t emitted, evaporated, sputtered;           /* SPs created this step */
  int64_t impact_ionizations, field_ionizations;    /* events this step */
  int64_t removed[PIC_NSPECIES], ion_impacts;       /* this step (impacts of Cu+ and Cu2+) */
  int64_t total_charge_fixed;           /* sum of deposited node charge (units e w_min 2^-30) */
  int mg_cycles;                        /* cycles of the last Poisson solve */
  double mg_residual;                   /* relative residual of the last Poisson solve */
  double V0;                            /* anode potential [V] */
  double max_face_field, max_J, max_T;  /* V/m, A/m^2, K */
  double emitted_current;               /* A, from the last emission pass */
  double ms[8]; /* ms of the last pic_step call, summed over its steps: emit+inject, push, sort,
                   collide, deposit, solve+E, heat, total (CUDA events on the library stream) */
  int64_t kernel_launches;  /* kernels launched by the library since create */
  int64_t emission_evals;   /* transmission evaluations of the emission integral this step */
  int64_t surrogate_faces;  /* faces whose emission came from the surrogate this step */
  double V_gap;             /* V: gap voltage (V0 without a circuit) */
  double I_gap, I_tot;      /* A: Shockley-Ramo gap current and circuit current of the last circuit stage */
  int64_t elastic_en, elastic_nn, charge_exchanges;  /* colliding pairs this step (PIC_F_ELASTIC) */
  int64_t mg_cycles_total;  /* Poisson refinement cycles since create (both forms) */
  int64_t coulomb_ee, coulomb_ei, coulomb_ii;  /* pairs turned this step (PIC_F_COULOMB) */
  int64_t merged;           /* SP pairs merged this step (PIC_F_MERGE) */
  int64_t fallback_range, fallback_bin;  /* faces the surrogate left to the integral this step:
                                            outside its trained range / in a bin that failed validation */
  int64_t double_ionizations, ion_ionizations;  /* Cu2+ events this step (PIC_F_ION2): Cu + e -> Cu2+ + 3e,
                                                   Cu+ + e -> Cu2+ + 2e */
  int64_t coulomb_ej, coulomb_ij, coulomb_jj;   /* Coulomb pairs with Cu2+ turned this step */
} pic_diag_t;

typedef struct pic_s pic_t;
typedef void *(*pic_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*pic_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

/* Create a handle (Sec. 2.1 statement of the problem): builds the staircased geometry, the
 * face list and the multigrid hierarchy on the device, then calibrates V0 from apex_field by a
 * Laplace solve (unless params->V0 > 0) and solves for the initial potential.
 * species: nspecies entries in the order electron, Cu, Cu+, Cu2+ (nspecies 4), or the first three
 * (nspecies 3: Cu2+ then holds at most one SP, and PIC_F_ION2 fails with PIC_E_CAPACITY as soon as a
 * Cu2+ channel produces more).  PIC_E_INVALID for any other nspecies. */
int pic_create(const pic_geometry_t *geometry, const pic_grid_t *grid, const pic_species_t *species,
               int nspecies, const pic_params_t *params, pic_alloc_fn alloc, pic_free_fn free_fn,
               void *alloc_user, void *stream, pic_t **out);
void pic_destroy(pic_t *h);
const char *pic_last_error(pic_t *h);

/* Replace all SPs of one species (host SoA arrays of length n) and cell-sort them.  Every SP
 * must lie inside the domain and outside the tip; PIC_E_INVALID otherwise, PIC_E_CAPACITY if
 * n exceeds the species capacity or a cell holds more than 32768 SPs of the species (the sort's
 * limit, which the step's sort reports the same way). */
int pic_load_particles(pic_t *h, int species, const float *x, const float *y, const float *z,
                       const float *vx, const float *vy, const float *vz, const int32_t *w,
                       const uint64_t *id, int64_t n);
/* The SPs of every species in one call: sp[s] for species s = 0 .. nspecies-1 (host SoA arrays
 * of length sp[s].n, pinned memory for full copy bandwidth).  Each species is checked and sorted
 * as by pic_load_particles, while the next species' host-to-device copies run on a second stream
 * of the library; the call returns once every species is in place.  Errors as for
 * pic_load_particles; on an error in species s the species before s are loaded and the others
 * unchanged (the same outcome as the sequence of pic_load_particles calls). */
typedef struct {
  const float *x, *y, *z, *vx, *vy, *vz;
  const int32_t *w;
  const uint64_t *id;
  int64_t n;
} pic_host_species_t;
int pic_load_all(pic_t *h, const pic_host_species_t *sp, int nspecies);
/* Copy out the SPs of one species in their current device order (cell-sorted part first, then
 * SPs created since the last sort); n_out receives the count.  PIC_E_CAPACITY if cap is short. */
int pic_get_particles(pic_t *h, int species, float *x, float *y, float *z, float *vx, float *vy,
                      float *vz, int32_t *w, uint64_t *id, int64_t cap, int64_t *n_out);
/* Step counter (keys the random draws) and the next id to hand out. */
int pic_set_clock(pic_t *h, int64_t step, int64_t next_id);

/* Checkpoint and resume (the paper runs each simulation to its end; this serves long runs).
 * pic_save writes the handle's whole evolving state to the file at `path` (created or
 * truncated): the device clock (step, next id, counts, counters, circuit state), every species'
 * SPs in their device order with the per-cell offsets and sorted-place cell keys of the last
 * sort, the fixed-point potential, the deposited charge, the previous potential when
 * PIC_F_EXTRAPOLATE keeps one, the per-face emission values and accumulators, the tip
 * temperature, the surrogate's weights and validity map, V0 and the flags.  It must be called
 * between steps or after pic_sort (PIC_E_INVALID while pushed SPs await their sort).
 * pic_load reads such a file into a handle created with the same grid, geometry, species charges
 * and masses and physical parameters (dt, apex_field, V0, T0, work_function, w_min, w_max_units,
 * n_heat, seed, circuit and collision parameters): PIC_E_INVALID names the first input that
 * differs; the solver controls (mg_tol, mg_max_cycles, mg_sweeps) may differ and the flags are
 * taken from the file.  PIC_E_CAPACITY if a species holds more SPs than this handle's capacity
 * (the handle is then unchanged).  After any other failure during the read the handle's state
 * is undefined and must be loaded again before stepping.  Every random draw is keyed by (seed,
 * purpose, id, step), so stepping a loaded handle repeats the uninterrupted run bit for bit, in
 * the eager and the graph form.  The file is in native byte order. */
int pic_save(pic_t *h, const char *path);
int pic_load(pic_t *h, const char *path);

/* Node arrays are (nz+1)*(ny+1)*(nx+1), index (k*(ny+1)+j)*(nx+1)+i.
 * The library holds the potential in fixed point, steps of 2^-40 V (~9.1e-13 V), so that the
 * Poisson stencil and the node differences of E are exact integer sums; pic_set_potential rounds
 * each value to that grid (half to even) and recomputes the node field; it returns PIC_E_INVALID
 * for a value that is not finite or not inside (-8192, 8192) V.  pic_get_potential returns the
 * held values exactly. */
int pic_set_potential(pic_t *h, const double *phi);
int pic_get_potential(pic_t *h, double *phi);
int pic_get_efield(pic_t *h, float *E);   /* 3 floats (Ex,Ey,Ez) [V/m] per node */
int pic_get_charge(pic_t *h, int64_t *Q); /* deposited charge, units e*w_min*2^-30 */
/* Tip temperature per solid cell, in linear cell order. */
int pic_set_temperature(pic_t *h, const double *T);
int pic_get_temperature(pic_t *h, double *T);
int pic_num_solid(pic_t *h, int64_t *n);

/* Exposed faces in their fixed order: vacuum cell, direction code (0..5 = -x,+x,-y,+y,-z,+z:
 * where the solid or the cathode plane lies) and owner solid cell (-1 for the cathode plane). */
int pic_num_faces(pic_t *h, int64_t *n);
int pic_get_faces(pic_t *h, int64_t *vcell, int32_t *dir, int64_t *owner);
/* Per-face state of the last emission pass: local field [V/m], J [A/m^2], P_N [W/m^2]. */
int pic_get_face_emission(pic_t *h, double *F, double *J, double *PN);
/* Per-face surface accumulators: evaporation [atoms], heat [J], emitted charge [C] (double) and
 * sputter [atoms 2^-24], bombardment energy E_b and sputtered energy E_s [eV 2^-20] (int64). */
int pic_get_face_accumulators(pic_t *h, double *evap, double *heat, double *charge, int64_t *sput,
                              int64_t *Eb, int64_t *Es);
int pic_set_face_accumulators(pic_t *h, const double *evap, const double *heat, const double *charge,
                              const int64_t *sput, const int64_t *Eb, const int64_t *Es);

/* Replace the PIC_F_* flags (e.g. switch the surrogate or the mixed-precision solve on or off
 * between steps of the same state). */
int pic_set_flags(pic_t *h, uint32_t flags);

/* Replace the Poisson solve's controls: relative residual target (> 0) and cap on refinement
 * cycles per solve (>= 1).  The next solve that cannot reach mg_tol within the cap returns
 * PIC_E_NOCONV. */
int pic_set_solver(pic_t *h, double mg_tol, int mg_max_cycles);

/* Stages of one step (each also usable alone; pic_step runs them all in this order). */
int pic_emit(pic_t *h);        /* a1 emission + a2 evaporation/sputter injection (appends SPs) */
int pic_push(pic_t *h);        /* a3 gather + leapfrog + boundary removal, ion impact records */
int pic_sort(pic_t *h);        /* a4 stable cell sort of every species, dropping removed SPs */
int pic_collide(pic_t *h);     /* a5 impact ionization MCC (with PIC_F_ION2 the Cu2+ channels), the elastic
                                  and Coulomb passes of their flags, then a6 field ionization (appends) */
/* SP merging (Sec. 2.3.2) on cell-sorted SPs: in a cell holding N > merge_max SPs of a species the
 * SPs at places 2m, 2m+1 merge for m < min(N - merge_max, N/2) into their centre of mass
 * (w = w1 + w2, a = a1 mu/w2 + a2 mu/w1, mu = w1 w2/(w1 + w2)); the second keeps weight 0 until the
 * next sort.  pic_step runs it after the sort when PIC_F_MERGE is set; PIC_E_INVALID without the
 * flag or on unsorted SPs. */
int pic_merge(pic_t *h);
/* RC circuit (the circuit passage of Sec. 2.3.1, after ArcPIC): I_gap = sum over e-, Cu+ (and Cu2+) SPs of
 * q v . E0(x) (Shockley-Ramo, E0 the Laplace field with the anode at unit potential, gathered like
 * E), then V_gap += dt/C ((V0 - V_gap)/R - I_gap).  pic_step runs it after the push; the following
 * Poisson solve holds the anode at V_gap.  PIC_E_INVALID without a circuit. */
int pic_circuit(pic_t *h);
int pic_deposit(pic_t *h);     /* a7 fixed-point CIC charge deposit of e-, Cu+ (and Cu2+, charge 2) */
int pic_solve_field(pic_t *h); /* a7 deposit, a8 Poisson solve, a9 node field */
int pic_heat(pic_t *h);        /* a10 continuity + heat on the tip cells from the accumulators */
/* nsteps full steps a1..a10 (heat every n_heat steps); the step counter advances by nsteps. */
int pic_step(pic_t *h, int nsteps);
int pic_diagnostics(pic_t *h, pic_diag_t *out);

/* Ensemble of independent instances (the paper has no counterpart; it runs one tip at a time).
 * pic_batch_create groups n distinct handles that share one stream (PIC_E_INVALID otherwise); the
 * handles stay owned by the caller and must outlive the batch.  pic_batch_step advances every
 * instance by nsteps full steps with ONE CUDA-graph launch per step: the graph holds one branch per
 * instance (independent, so the GPU runs them concurrently), each branch the instance's step with
 * its Poisson loop as a device-side while node.  The first call (and any call after an instance's
 * flags or buffers changed) runs one eager step per instance and records the graphs.  Each
 * instance's results equal those of pic_step on it alone, bit for bit.  The heat stage runs
 * between graph launches every n_heat steps of each instance.  Errors name the instance in
 * pic_batch_last_error.  pic_batch_ms returns the device time of the last pic_batch_step [ms]. */
typedef struct pic_batch_s pic_batch_t;
int pic_batch_create(pic_t *const *instances, int n, pic_batch_t **out);
int pic_batch_step(pic_batch_t *b, int nsteps);
int pic_batch_ms(pic_batch_t *b, double *ms);
const char *pic_batch_last_error(pic_batch_t *b);
void pic_batch_destroy(pic_batch_t *b);

/* Autotuner (no counterpart in the paper): times the launch-shape candidates on this instance's
 * current state and keeps the fastest -- blocks per SM of the particle kernels (2..32, probed on
 * the charge deposit, which it leaves as a deposit would), planes per thread of the fixed-point
 * residual (1, 2 or 4) and, per multigrid level, the smoother's planes per thread (1, 2, 4 or 8;
 * both probed on solver scratch that every solve rebuilds).  No result depends on the choices.
 * choices[0] receives the blocks per SM, choices[1] the residual's planes per thread and
 * choices[2 + l] the smoother's planes per thread on level l; returns the number of values
 * written (at most cap) or a negative PIC_E_* code. */
int pic_autotune(pic_t *h, int *choices, int cap);

/* Kernel timing (diagnostics of the library; the paper has no counterpart).  pic_num_kernels()
 * kernels are known by index (pic_kernel_name: "k_push", "k_smooth", ...).  pic_set_kernel_timing
 * selects kernels by bit mask (bit k = kernel k, 0 = none) and clears the sums; from then on every
 * launch of a selected kernel is bracketed by a pair of CUDA events on the library stream.
 * pic_get_kernel_timing synchronises the stream and returns, for kernel k, the launches timed,
 * their summed duration [ms] and their summed work units (nodes of the level a grid kernel
 * covers -- the swept colour's slots for k_smooth and k_smooth_first, colour-0 slots for
 * k_residual --, faces for face kernels, 0 for particle kernels, whose counts stay on the
 * device).  PIC_E_INVALID for a bad index.  Timing costs two event records per launch; keep the
 * mask 0 outside measurements. */
int pic_num_kernels(void);
const char *pic_kernel_name(int k);
int pic_set_kernel_timing(pic_t *h, uint64_t mask);
int pic_get_kernel_timing(pic_t *h, int k, int64_t *launches, double *ms, double *units);

/* Emission current density and Nottingham heat of n surface states (host arrays): F [V/m],
 * T [K], work function [eV], radius of curvature [m] (<= 0 or inf: flat); J [A/m^2], PN [W/m^2].
 * Evaluates the full FP64 thermal-field integral on the device (Sec. 2.3.1).  The handle's
 * device (current at pic_create) must be current: PIC_E_INVALID otherwise. */
int pic_emission_eval(pic_t *h, const double *F, const double *T, const double *phi_w,
                      const double *R, double *J, double *PN, int64_t n);

/* Emission surrogate (no counterpart in the paper): an MLP 7 -> 128 -> 128 -> 128 -> 2 with GELU.
 * The two 128 x 128 hidden layers run with BF16 operands and FP32 accumulation on the tensor
 * cores; the input and output layers are FP32.  Features (each standardised): log10 F, T, work
 * function, log10 R (flat: 3), 1/R (flat: 0), min(phi^1.5/F, 20), 1000/T.  Outputs: (log10 J -
 * log10 J_c, eps_N = P_N/J), J_c the classical estimate (Murphy-Good Fowler-Nordheim +
 * Richardson-Dushman with Schottky lowering).  Trained on tuples drawn over F 0.001-15 GV/m,
 * T 300-4000 K, phi_w 4-5 eV, R 1-20 nm or flat, with targets from the full FP64 integral; a
 * held-out set (half the training size) fills a validity map (bins whose every held-out sample has
 * |dlog10 J| <= 0.015 wherever log10 J >= -5, a margin under the 0.02 bar); log10 J is
 * clipped at -8 (no face emits below it).
 * With PIC_F_SURROGATE, pic_emit/pic_step use it on faces inside the range and a valid bin (and
 * on in-range faces of unvalidated bins where both it and J_c put J below 1e-3 A/m^2), and the
 * full integral elsewhere.  Parameters: W1 (128x7), b1, W2 (128x128), b2, W3 (128x128), b3,
 * W4 (2x128), b4 -- pic_mlp_num_params() floats, row-major [out][in]. */
int pic_mlp_num_params(void);
int pic_mlp_set_params(pic_t *h, const float *params);
int pic_mlp_get_params(pic_t *h, float *params);
/* Forward (and, with targets t, loss 0.5 mean sum (y - t)^2 and its gradient) on n host rows of
 * 7 standardised features; y: n x 2 standardised outputs. */
int pic_mlp_forward_backward(pic_t *h, const float *x, const float *t, int64_t n, float *y, float *loss, float *grad);
/* Train and install; stats (8 doubles, optional): train loss, validation RMS and max |dlog10 J|
 * over relevant samples, fraction of valid bins, fraction of valid held-out samples, ms of data
 * generation, ms of training, optimiser steps. */
int pic_surrogate_train(pic_t *h, int64_t nsamples, int epochs, int batch, double lr, uint64_t seed, double *stats);
/* Install src's trained surrogate (weights and validity map) in dst, so that one training serves
 * every instance of an ensemble; PIC_E_INVALID if src has none. */
int pic_surrogate_copy(pic_t *dst, pic_t *src);
/* Surrogate J [A/m^2], P_N [W/m^2] of n host tuples (F [V/m], T [K], phi_w [eV], R [m], <= 0 flat);
 * valid[i] = 1 where the step would use the surrogate for that tuple. */
int pic_surrogate_eval(pic_t *h, const double *F, const double *T, const double *phi_w, const double *R, double *J,
                       double *PN, uint8_t *valid, int64_t n);

/* Allocation-free form of pic_emission_eval, for callers that cannot take device memory: a
 * process whose device memory is fully reserved by another framework's pool, or a latency-bound
 * loop that cannot afford the device-wide synchronisation of cudaFree.  The paper has no
 * counterpart; this is a property of the library only.  Same arguments, units and results as
 * pic_emission_eval, for at most PIC_NOALLOC_MAX_TUPLES tuples per call (PIC_E_INVALID above
 * that, with a message).  The inputs and outputs are staged through one fixed device array
 * built into the library (1.5 MiB, held on every GPU that loads it until exit); no cudaMalloc,
 * cudaFree or allocating routine is called.  The first call on a device looks the array's
 * address up (cudaGetSymbolAddress) with that device current: make it before any stream
 * capture starts there.  The handle's device must be current (PIC_E_INVALID otherwise).  All
 * calls share the array, so calls whose work overlaps on the GPU race and must be serialised by
 * the caller. */
#define PIC_NOALLOC_MAX_TUPLES 32768
int pic_emission_eval_noalloc(pic_t *h, const double *F, const double *T, const double *phi_w,
                              const double *R, double *J, double *PN, int64_t n);

#ifdef __cplusplus
}
#endif
#endif
