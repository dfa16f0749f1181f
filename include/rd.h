/*
 * rd.h -- C ABI of the GB300 (sm_103a) Green's-function-corrected Brownian-dynamics
 * reaction-diffusion step of Pruestel & Meier-Schellersheim (arXiv:1107.0270).
 *
 * One call of rd_step advances every particle of every replica by one time step dt following the
 * paper's simulation algorithm (Section 3, steps 1-5):
 *   free Gaussian displacements (step 1, Eq. oLangevin), encounter detection for every interacting
 *   pair within the cut-off radius with the encounter probability p_enc = 1 - G_abs/G_free
 *   (Eq. bayes1D, Section 2.2.4 radial form), conflict resolution among several encounter
 *   candidates (Section 3, "Details"), propagation of encountered pairs by G_ref - G_abs
 *   (Eq. passage_prob), the reaction decision p_reac = (G_ref - G_rad)/(G_ref - G_abs)
 *   (Eq. psurv_radII), unimolecular decays 1 - exp(-k_d dt) (Eq. rad_prob) with reversible
 *   dissociation products placed at contact (Section 2.2.5), and compaction of the particle arrays.
 *
 * Every step runs as hand-written CUDA kernels on the caller's stream; there is no CPU fallback.
 * All functions return an rd_status code (never throw across the ABI).  Calls on one handle must
 * not run concurrently from several host threads.
 */
#ifndef RD_H
#define RD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RD_MAX_SPECIES 16
#define RD_MAX_PAIRS 32
#define RD_MAX_DECAYS 16

typedef enum {
  RD_OK = 0,
  RD_EINVAL = 1,     /* invalid argument or configuration (nothing was changed) */
  RD_ENOMEM = 2,     /* device allocation failed */
  RD_ECAPACITY = 3,  /* a device list or the particle array overflowed; the step was not committed */
  RD_ETIMEOUT = 4,   /* a bounded device-side iteration (conflict resolution) did not finish */
  RD_ECUDA = 5,      /* a CUDA runtime call failed; rd_last_cuda_error() gives the code */
  RD_ENOTREADY = 6   /* entry point not available for this configuration */
} rd_status;

/* Boundary condition at contact (Section 2.1): absorbing, reflective, radiation (Robin). */
typedef enum { RD_BC_NONE = 0, RD_BC_ABS = 1, RD_BC_REF = 2, RD_BC_RAD = 3 } rd_bc;

/* Arithmetic of the step.  RD_FP64: every stage in double precision.  RD_MIXED: positions stored
 * as float4; displacements, binning, the per-candidate p_enc (3D closed form; 2D per-run table),
 * the encounter and selection draws and the conflict keys in FP32; p_reac and the propagator
 * sample of an encountered pair from per-run FP32 tables (bicubic) built on the device in FP64 at
 * rd_init, the propagator sample refined by one FP32 Newton step; time and observable sums in
 * FP64 / int64.  Per-pair probability error against FP64: below 2e-6 absolute. */
typedef enum { RD_FP64 = 0, RD_MIXED = 1 } rd_precision;

/* Interaction of species s1 and s2 (unordered).  sigma: contact radius a_eff (length unit of the
 * box).  ka: intrinsic association rate kappa_a (volume/time in 3D, area/time in 2D), used by
 * RD_BC_RAD only.  product: species of the A+B->C product, or -1 for none. */
typedef struct {
  int32_t s1, s2;
  int32_t bc;
  int32_t product;
  double sigma;
  double ka;
} rd_pair_rule;

/* Unimolecular reaction parent -> products with rate kd (1/time).  n_products in {0,1,2}.  Two
 * products that form an interacting pair are placed at that pair's contact radius and propagated
 * by G_ref - G_abs (geminate recombination by p_reac); otherwise sigma_place apart. */
typedef struct {
  int32_t parent;
  int32_t n_products;
  int32_t products[2];
  double kd;
  double sigma_place;
} rd_decay;

/* One replica (independent periodic system) of a batched ensemble. */
typedef struct {
  double L;                           /* box edge */
  int64_t n_init[RD_MAX_SPECIES];     /* initial particles per species */
} rd_replica;

/* Device-memory provider.  When alloc is NULL the library uses cudaMallocAsync/cudaFreeAsync on
 * the handle's stream.  Bindings pass their framework's caching allocator here. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*release)(void* ptr, size_t bytes, void* stream, void* ctx);
  void* ctx;
} rd_allocator;

typedef struct {
  int32_t dim;                        /* 2 or 3 */
  int32_t precision;                  /* rd_precision */
  int32_t n_species, n_pairs, n_decays;
  int32_t n_replicas;                 /* >= 1; replicas points to n_replicas entries */
  double dt;                          /* time step */
  uint64_t seed;                      /* Philox key */
  double c_cut;                       /* cut-off r_cut = sigma + c_cut sqrt(2 (D_A+D_B) dt), default 5 */
  double tau_s;                       /* 2D: small-time series for tau <= tau_s (default 0.01) */
  double D[RD_MAX_SPECIES];           /* diffusion constants per species */
  rd_pair_rule pairs[RD_MAX_PAIRS];
  rd_decay decays[RD_MAX_DECAYS];
  const rd_replica* replicas;         /* read during rd_init only */
  double capacity_factor;             /* particle capacity = factor * initial total (default 2) */
  int64_t pair_capacity;              /* fired-pair list capacity (0: automatic) */
  int32_t cell_factor_x100;           /* cell edge = largest r_cut x factor/100; 0: density-based per
                                         replica (about 0.25 interacting particles per cell, edge between
                                         1 and 4 cut-offs); < 0: the fastest of four choices (fixed
                                         1.0, density rule x 0.7 / 1 / 1.5), timed by rd_init on the
                                         initial state */
  int32_t block_size;                 /* threads per block of the particle kernels: 0 (256) or a
                                         multiple of 32 in [32, 256]; RD_EINVAL otherwise */
  int32_t sweep_split;                /* cell sweep: 0 automatic (one thread per particle, or one per
                                         stencil row when the autotuner finds it faster), 1 one
                                         thread per particle, 2 one thread per (particle, row) */
  int32_t cell_reach;                 /* cell sweep stencil: 0 automatic (2 for dense 2D systems, else 1),
                                         1 cells of at least one cut-off, 2 (2D only) cells of at least
                                         half a cut-off with a stencil two cells wide */
  double drift[RD_MAX_SPECIES][3];    /* deterministic drift velocity per species (um/s); each step first
                                         moves every particle by drift * dt (periodic wrap), then the
                                         Brownian / reaction step runs from there with the pair
                                         probabilities taken from the Brownian end points.  All zero: no
                                         drift step */
  int32_t step_launch;                /* how a step is launched: 0 automatic (separate kernels under
                                         programmatic dependent launch; with the autotuner, and up
                                         to 2^22 particles of capacity, the faster of those and one
                                         fused cooperative launch), 1 always fused, 2 always
                                         separate kernels.  Both give bit-identical results;
                                         RD_EINVAL outside 0..2 */
  int32_t force_paths;                /* 0 normally.  Bit 0: conflict rounds on the whole cooperative
                                         grid for any number of conflict pairs (normally only above
                                         2048); bit 1: short conflict lists in global memory instead
                                         of shared memory.  For tests of the large-size code paths at
                                         small sizes; results are the same */
  int32_t angle_mode;                 /* direction of an encountered pair's new separation (Eq.
                                         passage_prob): 0 (default) drawn from the full propagator
                                         G_ref - G_abs, its angle to the start separation from the
                                         partial-wave series of Eqs. genericGF3D / genericGF (a draw
                                         needing more than 127 partial waves, kappa = R' R0 / 2 tau
                                         beyond ~53, keeps the free step's direction and is counted in
                                         RD_STAT_ANGLE_FALLBACK).  RD_FP64 evaluates the series per
                                         pair (about a millisecond of FP64 work each); RD_MIXED reads a
                                         per-rule table of the law built at rd_init (within 1e-4 in
                                         the law's CDF); 1 the free step's direction kept, only the
                                         length resampled */
  int32_t pad_angle;
  rd_allocator allocator;
} rd_config;

typedef struct rd_handle rd_handle;

/* Create a handle: validates cfg, allocates the device state through cfg->allocator on `stream`
 * (a cudaStream_t, NULL = legacy default stream), draws uniform initial positions from the Philox
 * INIT streams (ids 0..N-1 per replica, species in blocks of n_init) and enqueues nothing else.
 * *out receives the handle (NULL on error).  Errors: RD_EINVAL, RD_ENOMEM, RD_ECUDA. */
int rd_init(const rd_config* cfg, void* stream, rd_handle** out);

/* Advance all replicas by exactly one dt.  Asynchronous on the handle's stream; device-side
 * errors (RD_ECAPACITY, RD_ETIMEOUT) are latched in a device status word, leave the state of that
 * step uncommitted, and are returned by the next synchronising call (rd_observables, rd_sync,
 * rd_get_state). */
int rd_step(rd_handle* h);

/* Advance by nsteps >= 0 steps through captured CUDA graphs (two steps per graph launch).
 * Asynchronous like rd_step. */
int rd_run(rd_handle* h, int64_t nsteps);

/* Synchronise the handle's stream and return the latched device status. */
int rd_sync(rd_handle* h);

/* Observables after the last completed step; synchronises the stream.  counts: caller-owned
 * int64[n_replicas * n_species] (may be NULL), current particles per replica and species.
 * step/t (may be NULL): step index and simulated time (FP64 accumulation).  stats: caller-owned
 * int64[RD_NSTATS] (may be NULL), cumulative counters since rd_init (see RD_STAT_*). */
#define RD_NSTATS 13
enum {
  RD_STAT_CANDIDATES = 0, RD_STAT_FIRED = 1, RD_STAT_MATCHED = 2, RD_STAT_REACTIONS = 3,
  RD_STAT_RESAMPLED = 4, RD_STAT_DECAYS = 5, RD_STAT_RECOMBINED = 6, RD_STAT_NEAR_THRESHOLD = 7,
  RD_STAT_OVERLAPS = 8, RD_STAT_MATCH_ROUNDS = 9, RD_STAT_PARTICLE_STEPS = 10,
  RD_STAT_FIRED_HWM = 11,
  RD_STAT_ANGLE_FALLBACK = 12   /* exact-angle draws that needed more than 128 partial waves and kept
                                   the free step's direction instead (see rd_config.angle_mode) */
};
int rd_observables(rd_handle* h, int64_t* counts, int64_t* step, double* t, int64_t* stats);

/* Copy the current state to caller-owned HOST buffers (synchronises).  n_inout: in = capacity of
 * the buffers (particles), out = particles written; if the capacity is too small nothing is
 * copied, *n_inout is set to the required count and RD_EINVAL is returned.  x: double[n*3]
 * (z = 0 in 2D), species: int32[n], id: uint32[n], replica: int32[n] (any may be NULL), ordered by
 * (replica, id).  next_id: caller-owned uint32[n_replicas] or NULL. */
int rd_get_state(rd_handle* h, int64_t* n_inout, double* x, int32_t* species, uint32_t* id,
                 int32_t* replica, uint32_t* next_id, int64_t* step);

/* Replace the state from caller-owned HOST buffers (synchronises).  Particles must be grouped by
 * replica (ascending) and sorted by id inside a replica; positions must lie in [0, L).  step sets
 * the step counter (the random streams are keyed by it).  Errors: RD_EINVAL, RD_ECAPACITY. */
int rd_set_state(rd_handle* h, int64_t n, const double* x, const int32_t* species,
                 const uint32_t* id, const int32_t* replica, const uint32_t* next_id, int64_t step);

/* Per-pair probabilities for separations of species-pair rule `rule` (index into cfg->pairs):
 * for k < n, p_enc[k] = encounter probability for start separation r0[k] and end separation r[k]
 * (Eq. bayes1D with radial Green's functions), p_reac[k] = reaction probability for a pair that
 * met the boundary and ended at r[k] (Eq. psurv_radII).  r0, r, p_enc, p_reac are DEVICE pointers
 * (double, n entries each; p_enc or p_reac may be NULL), evaluated in the handle's precision
 * (RD_MIXED: p_enc in FP32 as the step evaluates it, p_reac from the same FP32 table as the step;
 * RD_FP64: both in FP64).  Asynchronous on the handle's stream. */
int rd_pair_probs(rd_handle* h, int32_t rule, const double* r0, const double* r, int64_t n,
                  double* p_enc, double* p_reac);

/* Resample separations of encountered pairs (Section 3 "Details", radial propagator
 * 4 pi R^2 (g_ref - g_abs)): for k < n, r_new[k] >= sigma solves T(r_new) = u[k] where T is the
 * normalised tail of the propagator started at r0[k].  DEVICE pointers, asynchronous. */
int rd_resample(rd_handle* h, int32_t rule, const double* r0, const double* u, int64_t n,
                double* r_new);

/* Propagation of encountered pairs (Eq. passage_prob with the full Green's functions of Eqs.
 * genericGF3D / genericGF): for k < n, a pair of rule `rule` (reflective or radiation boundary)
 * with start separation vector r0[3k .. 3k+2] gets the new separation vector r_out[3k .. 3k+2]
 * drawn from G_ref - G_abs: its length at tail fraction u[4k] of the radial law (as rd_resample),
 * the cosine of its angle to r0 (3D; in 2D the angle in [0, pi]) at CDF value u[4k+1] of the
 * partial-wave law given that length, its azimuth 2 pi u[4k+2] about r0 in the frame built from the
 * coordinate axis along r0's smallest component (2D: the angle's sign negative iff u[4k+2] < 1/2);
 * u[4k+3] is unused.  r0 = 0 uses the x axis.  A law needing more than 128 partial waves keeps r0's
 * direction.  In the handle's precision (RD_MIXED: FP32, the length from the per-run table).
 * DEVICE pointers (double; z = 0 in 2D); asynchronous.  Errors: RD_EINVAL. */
int rd_propagate(rd_handle* h, int32_t rule, const double* r0, const double* u, int64_t n, double* r_out);

/* First-passage refinement of encountered pairs (Appendix, "Relation to first-passage time
 * simulation algorithms"): for k < n, a pair of rule `rule` whose separation went from r0[k] to
 * r[k] in one step dt and that met the contact surface during it.  The step is halved `levels`
 * times (0..24); at each level the separation at the midpoint is drawn from the radial Brownian
 * bridge and the half holding the first contact is chosen with p_enc of the two halves, redrawn
 * until one half has an encounter (the encounter is known for the whole interval).
 * Outputs: bin[k] = j such that the first contact lies in [j, j + 1) dt / 2^levels; r_lo[k],
 * r_hi[k] = separations at that interval's ends; attempts[k] = midpoint draws used.  A pair whose
 * draws exceed max_attempts (0: RD_FPT_MAX_ATTEMPTS; the expected count is about 1/p_enc of the
 * whole step plus a few per level) gets bin = 0xFFFFFFFF and NaN separations.
 * Random numbers: Philox4x32-10 with the handle's seed, counter (stream[k] low word, high word,
 * attempt, 13 | word << 8).  Pointers are DEVICE pointers: r0, r (double, physical lengths),
 * stream (uint64), bin (uint32) required; r_lo, r_hi (double), attempts (uint32) may be NULL.
 * Precision: FP64, except on a mixed-precision handle in 3D, where every draw is evaluated in FP32
 * on contact distances R - 1 (the same Philox words; decisions agree with FP64 ones except within
 * about 1e-6 of their thresholds, separations to about 1e-6 relative).  Negative separations are
 * read as 0.
 * In 2D the half intervals longer than tau_s use Weber quadrature nodes built on the first call
 * for each (rule, levels) (allocation and a synchronisation then); accuracy holds for
 * separations up to the rule's cut-off plus 13 sqrt(D dt).  n < 2^32.  A call with more pairs than
 * any before on the handle allocates its work queues (136 bytes per pair, through the handle's
 * allocator) and releases the previous ones.  Asynchronous on the handle's stream.
 * Errors: RD_EINVAL (no handle, rule out of range or without a boundary condition, n < 0 or
 * n >= 2^32, levels outside 0..24, a required pointer NULL with n > 0), RD_ENOMEM (work queues or
 * Weber nodes), RD_ECUDA (launch).  A pair that hits the attempt bound is not an error (see
 * above). */
#define RD_FPT_MAX_ATTEMPTS (1u << 20)
int rd_first_passage(rd_handle* h, int32_t rule, const double* r0, const double* r,
                     const uint64_t* stream, int64_t n, int32_t levels, uint32_t max_attempts,
                     uint32_t* bin, double* r_lo, double* r_hi, uint32_t* attempts);

/* Diagnostics of the last step (synchronises): the fired (encounter) pairs as ids, their p_enc,
 * their selection key -ln(U_sel)/p_enc and whether the conflict resolution accepted them (the
 * accepted set is the greedy matching in ascending (key, id_a, id_b)).  cap: capacity of the
 * caller-owned HOST arrays; *n_out: pairs in the list (all copied when <= cap).  Any output array
 * may be NULL. */
int rd_last_fired(rd_handle* h, int64_t cap, int64_t* n_out, uint32_t* id_a, uint32_t* id_b,
                  double* p_enc, int32_t* accepted, int32_t* replica, double* key);

/* Number of particles currently alive (synchronises). */
int rd_num_particles(rd_handle* h, int64_t* n);

/* Per-step totals over replicas of every species, kept on the device for the last 65536 steps
 * without host synchronisation during rd_run (the A-count trajectory and, for an irreversible
 * reaction, the pair-survival histogram -dN_A per step).  Synchronises; out: caller-owned HOST
 * int64[n_steps * n_species], row k = step first_step + k (0 = initial state).  RD_EINVAL if a
 * requested step is in the future or no longer kept. */
int rd_count_history(rd_handle* h, int64_t first_step, int64_t n_steps, int64_t* out);

/* Failure-detection check (no counterpart in the paper): runs the cell scan of a step once with
 * its first tile withheld, so that the next tile's look-back waits on a flag that nothing sets.
 * With the device waits bounded by spin_limit polls (> 0) the kernel latches RD_ETIMEOUT and
 * returns instead of hanging.  Synchronises; *status_out (HOST int32[1]) receives the latched
 * status (RD_ETIMEOUT when the bound works); then the control block is restored, so the handle
 * keeps stepping from the same state.  Returns RD_OK, or the status already latched before the
 * call, or RD_EINVAL. */
int rd_check_bounded_wait(rd_handle* h, uint32_t spin_limit, int32_t* status_out);

/* Launch layout chosen at rd_init (no synchronisation): out[0] cell-edge choice (> 0: fixed factor
 * in units of the largest cut-off; < 0: per-replica density rule times -out[0]), out[1] total cells,
 * out[2] threads per block of the particle kernels, out[3] particle capacity, out[4] fired-pair
 * capacity, out[5] autotuned ms per step (0 if not tuned), out[6] largest cut-off radius, out[7]
 * threads per binned particle in the cell sweep (1, or one per stencil row), out[8] stencil reach
 * in cells (1, or 2 for 2D cells of half a cut-off), out[9] 1 if a step is one fused cooperative
 * launch (0: one launch per kernel), out[10] blocks of that launch.  Writes min(n, 11) values to the
 * caller-owned HOST array. */
int rd_info(rd_handle* h, double* out, int32_t n);

/* Kernel-level timing hook: rd_time_kernels enables timing of the next rd_step; rd_kernel_times
 * copies its (name, ms) pairs: with separate kernels the CUDA-event time of every kernel; with the
 * fused launch the device time of every phase (global-timer stamps taken at the phase barriers)
 * followed by "k_step_fused", the CUDA-event time of the whole launch. */
int rd_time_kernels(rd_handle* h, int32_t enable);
int rd_kernel_times(rd_handle* h, int32_t cap, int32_t* n_out, char* names /* cap*32 */,
                    float* ms);

/* ---------------------------------------------------------------------------------------------
 * Allocation-free single step (the paper has no counterpart; this is a library service).
 *
 * Some callers cannot allocate device memory: code running where a cudaMalloc would stall or be
 * refused (inside a larger application's memory budget, under an allocator that forbids
 * allocation after start-up, or in a real-time loop that must not synchronise on an allocation).
 * rd_step_static advances a small single-replica system (cfg->n_replicas == 1, box edge
 * cfg->replicas[0].L; n_init is ignored; 3D only: dim 2 returns RD_ENOTREADY) by one dt, exactly
 * as rd_step does, without calling
 * cudaMalloc, cudaFree or any allocating routine: every scratch buffer of the step lives in one
 * fixed device array of RD_STATIC_SCRATCH_BYTES that the library reserves on every GPU that loads
 * it, until the process exits.
 *
 * Limits: n <= RD_STATIC_MAX_PARTICLES, at most RD_STATIC_MAX_PAIRS encounter pairs per step (more
 * latch RD_ECAPACITY in *status_out and the outputs then hold the unchanged input state), the cell
 * grid is coarsened to RD_STATIC_MAX_CELLS cells.  With RD_MIXED the per-run FP32 tables of p_reac
 * and of the propagator sample are built inside the same array on every call (a fraction of a
 * millisecond); their size grows like (r_cut/sigma) (r_cut/sigma + 13 sqrt(tau)) / tau with
 * tau = (D_A + D_B) dt / sigma^2, so large steps do not fit: the 10 uM reversible system
 * (sigma = 0.005, D_A + D_B = 2) fits at dt = 1e-5 but not at dt = 1e-4 in RD_MIXED (RD_FP64 needs
 * no tables).  No table of the angle law is built: with angle_mode 0 an RD_MIXED call evaluates
 * that law per resampled pair in FP32 (about a millisecond of one warp each), where a handle reads
 * its table, so the two agree within the FP32 angle tolerance, not bit for bit.  Inputs beyond any
 * limit are rejected with RD_EINVAL before anything is enqueued, and the outputs are left
 * untouched.
 *
 * Inputs (DEVICE pointers, caller-owned): x_in double[n*3] (positions in [0,L)),
 * species_in int32[n], id_in uint32[n] sorted ascending; next_id = first id for new products;
 * step = step index that keys the random streams.  Outputs (DEVICE pointers, caller-owned):
 * x_out double[out_cap*3], species_out int32[out_cap], id_out uint32[out_cap] with
 * out_cap >= 2n; n_out int64[1], next_id_out uint32[1], status_out int32[1] (rd_status of the
 * step; each may be NULL).  Everything is enqueued on `stream`; the host returns without waiting.
 *
 * Sharing: all calls use the same scratch array, which keeps the previous call's contents (the
 * entry point clears what must start at zero).  Calls whose work overlaps on the GPU (different
 * streams, or several host threads) race on that array and give wrong results: serialise them.
 * Set-up: the first call on each device looks up the array's device address with that device
 * current; make that first call before any stream capture begins.  (This note is about that
 * set-up only.)
 * ------------------------------------------------------------------------------------------- */
#define RD_STATIC_MAX_PARTICLES 16384
#define RD_STATIC_MAX_CELLS 65536
#define RD_STATIC_MAX_PAIRS 65536
#define RD_STATIC_SCRATCH_BYTES (32u << 20)
int rd_step_static(const rd_config* cfg, void* stream, int64_t n, const double* x_in,
                   const int32_t* species_in, const uint32_t* id_in, uint32_t next_id, int64_t step,
                   int64_t out_cap, double* x_out, int32_t* species_out, uint32_t* id_out,
                   int64_t* n_out, uint32_t* next_id_out, int32_t* status_out);

/* Release all device memory of the handle (synchronises).  NULL is ignored. */
void rd_free(rd_handle* h);

const char* rd_strerror(int status);
int rd_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif
