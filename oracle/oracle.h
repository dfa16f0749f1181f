/*
 * Plain serial FP64 CPU oracle of the Green's-function-corrected Brownian-dynamics step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg may load or call this library.  It shares no code, header, table or helper with the CUDA
 * library; it is written from the paper (Sections 2-4 and the Appendix) and from the published
 * definitions of the algorithms it uses (Philox4x32-10, Box-Muller, the erfc continued fraction,
 * Best and Fisher's von Mises sampler).
 *
 * Units: lengths in the caller's unit (um), times in s.  Inside the Green's-function routines all
 * lengths are scaled by the contact radius a (R = r/a) and time by a^2/D (tau = D t / a^2), as in
 * Section 4.1 of the paper.
 */
#ifndef RD_ORACLE_H
#define RD_ORACLE_H
#include <stdint.h>

#define OR_MAX_SPECIES 16
#define OR_MAX_PAIRS 32
#define OR_MAX_DECAYS 16

enum { OR_BC_NONE = 0, OR_BC_ABS = 1, OR_BC_REF = 2, OR_BC_RAD = 3 };

/* Random-stream tags (counter word 3, low byte). */
enum {
  OR_TAG_INIT0 = 1, OR_TAG_INIT1 = 2, OR_TAG_UNI = 3, OR_TAG_DISP0 = 4, OR_TAG_DISP1 = 5,
  OR_TAG_ENC = 6, OR_TAG_RES = 7, OR_TAG_DIR = 8, OR_TAG_DISS0 = 9, OR_TAG_DISS1 = 10,
  OR_TAG_DISS2 = 11, OR_TAG_DISS3 = 12, OR_TAG_ANG = 14
};

typedef struct {
  int32_t s1, s2, bc, product;
  double sigma, ka;
} or_pair;

typedef struct {
  int32_t parent, n_products, p0, p1;
  double kd, sigma_place;
} or_decay;

typedef struct {
  int32_t dim, n_species, n_pairs, n_decays;
  double L, dt, c_cut, tau_s;
  uint64_t seed;
  uint32_t replica, pad_;
  double D[OR_MAX_SPECIES];
  or_pair pairs[OR_MAX_PAIRS];
  or_decay decays[OR_MAX_DECAYS];
  /* deterministic drift displacement per step and species (v dt), applied as a split step before
   * the Brownian step; has_drift = 0 skips it */
  double drift_dx[OR_MAX_SPECIES][3];
  int32_t has_drift;
  /* direction of an encountered pair's new separation: 0 = drawn from the full propagator
   * G_ref - G_abs (Eq. passage_prob with Eqs. genericGF3D / genericGF); 1 = the free step's
   * direction kept (only the length resampled) */
  int32_t angle_mode;
} or_system;

typedef struct {
  int64_t n, cap;
  double* x;          /* cap*3, z ignored in 2D */
  int32_t* sp;
  uint32_t* id;
  uint32_t step, next_id;
  double t;
} or_state;

typedef struct {
  int64_t candidates, fired, matched, reactions, resampled, decays, recombined, near_threshold,
      overlaps, products;
} or_stats;

/* Optional per-candidate record (NULL to skip).  One entry per candidate pair. */
typedef struct {
  int64_t cap, n;
  uint32_t *ida, *idb;
  double *p_enc, *u_enc;
  int32_t *fired, *matched;
} or_trace;

/* Philox4x32-10 and the derived uniforms / normals. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_u52(uint32_t hi, uint32_t lo);

/* erfcx(x) = exp(x^2) erfc(x) and the scaled repeated integral of erfc. */
double or_erfcx(double x);
double or_ierfc_scaled(int n, double z);

/* 3D radial Green's-function quantities (scaled units). */
double or_p_enc3(double R, double R0, double tau);
double or_p_reac3(double R, double R0, double tau, double h);
double or_tail3(double V, double R0, double tau);
double or_resample3(double U, double R0, double tau);
double or_S_abs3(double R0, double tau);
double or_S_rad3(double R0, double tau, double h);

/* 2D radial Green's-function quantities (scaled units). */
double or_gamma2(int k, int bc, double R, double R0, double h);
double or_gbc2_series(int bc, double R, double R0, double tau, double h, int nterms);
double or_gbc2_weber(int bc, double R, double R0, double tau, double h);
double or_gfree2(double R, double R0, double tau);
double or_p_enc2(double R, double R0, double tau, double tau_s);
double or_p_reac2(double R, double R0, double tau, double h, double tau_s);
double or_tail2(double V, double R0, double tau, double tau_s);
double or_resample2(double U, double R0, double tau, double tau_s);
double or_S_abs2(double R0, double tau);

/* First-passage refinement of an encountered pair (Appendix): bisects a step of length tau
 * (scaled units) `levels` times; *bin = index of the interval of length tau / 2^levels that holds
 * the first contact, *R_lo, *R_hi = separations at that interval's ends, *attempts = midpoint
 * draws used, *margin = min |U - p_enc| over the encounter decisions taken.  Returns 1 (bin =
 * 0xFFFFFFFF, R_lo = R_hi = NaN) when max_attempts draws did not suffice, else 0. */
int or_fpt_refine(int dim, double R0, double R, double tau, double tau_s, int levels, uint64_t seed,
                  uint64_t strm, uint32_t max_attempts, uint32_t* bin, double* R_lo, double* R_hi,
                  uint32_t* attempts, double* margin);

int or_fpt_direction(int dim, double kappa, uint64_t seed, uint64_t strm, uint32_t a, double* omc,
                     double* sn);

/* Exact angular propagation (partial waves of Eqs. genericGF3D / genericGF).  or_ang_coeffs: the
 * integrals D_n, n = 0..N, of the reflective minus absorbing products (which = 0), or of the
 * absorbing (1), reflective (2) or free (3) product alone; returns N (D holds N + 1 values, at most
 * cap).  or_ang_sample: the angle of r' to r0 at CDF value U (3D: cos(angle); 2D: the angle in
 * [0, pi]).  or_ang_density: its density. */
int or_ang_coeffs(int dim, int which, double R, double R0, double tau, double* D, int cap);
double or_ang_sample(int dim, double U, double R, double R0, double tau);
double or_ang_density(int dim, double v, double R, double R0, double tau);
double or_ang_cdf(int dim, double v, double R, double R0, double tau);
double or_gf_partial(int dim, int which, double v, double R, double R0, double tau);
/* One encountered pair's new separation vector (scaled units) from the start vector r0. */
void or_propagate(int dim, const double* r0, double tau, double tau_s, double u_res, double u_ang, double u_azi,
                  double* out);

/* Test hook of the negative controls (0: none; 1: key -ln(U) p; 2: descending greedy order;
 * 3: U_enc reused as U_sel; 4: the cylindrical Bessel derivative in the 3D boundary coefficients).
 * Never set outside a test. */
void or_set_fault(int fault);

/* Threads of a step's pair loop: omp_get_max_threads() in the OpenMP build, else 1. */
int or_threads(void);

/* Whole step and initial condition. */
int or_init_positions(const or_system* sys, const int64_t* n_init, or_state* st);
int or_step(const or_system* sys, const or_state* in, or_state* out, or_stats* stats, or_trace* trace);

#endif
