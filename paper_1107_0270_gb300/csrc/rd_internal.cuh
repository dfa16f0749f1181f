// Internal definitions of the GB300 GF-BD step: device-side parameter blocks, random streams and
// the 3D radial Green's-function quantities.  Included by the kernel and host translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rd.h"

namespace rd {

constexpr int kMaxSpecies = RD_MAX_SPECIES;
constexpr int kMaxPairs = RD_MAX_PAIRS;
constexpr int kMaxDecays = RD_MAX_DECAYS;
constexpr int kAngTabU = 64;       // intervals of the angle table's U axis
constexpr int kAngTabStride = kAngTabU + 4;   // floats per (R0, R') node of the angle table
constexpr uint32_t kNoCell = 0xFFFFFFFFu;
constexpr uint32_t kOneParticle = 0xFFFFFFFFu;   // id_b of one-particle random streams
constexpr int kSmemCounts = 6144;                // per-block histogram of (replica, species) counts

// Random-stream tags (counter word 3, low byte; replica index in the upper 24 bits).
enum Tag : uint32_t {
  TAG_INIT0 = 1, TAG_INIT1 = 2, TAG_UNI = 3, TAG_DISP0 = 4, TAG_DISP1 = 5, TAG_ENC = 6,
  TAG_RES = 7, TAG_DIR = 8, TAG_DISS0 = 9, TAG_DISS1 = 10, TAG_DISS2 = 11, TAG_DISS3 = 12,
  TAG_FPT = 13, TAG_ANG = 14
};

// Per-particle status word written every step.
enum : uint32_t {
  ST_DECAYED = 1u,         // bit 0: unimolecular decay drawn this step
  ST_CONSUMED = 2u,        // bit 1: removed at the end of the step (reacted or decayed)
  ST_NPROD_SHIFT = 2,      // bits 2-3: products owned (0..2)
  ST_CHANNEL_SHIFT = 4     // bits 4-7: decay channel
};

// Fired-pair state (low 2 bits), rule index (bits 2-7), replica (bits 8-31).
enum : uint32_t { FS_LIVE = 0u, FS_ACCEPTED = 1u, FS_DEAD = 2u };

struct __align__(32) d4 {
  double x, y, z, w;
};

struct WeberNode;
struct Series2D;

// Uniform 2D table over (d0, d) with spacing h; row/column 0 is a ghost point at -h and two ghost
// points follow the last grid point (n0 x n1 stored values).  Catmull-Rom bicubic lookup.
struct Tab2 {
  const float* v;             // n0 x n1 values on the grid (x0, x1) = (h (i-1), h1 (j-1))
  const float4* q;            // q[i n1 + j] = v[i n1 + j-1 .. j+2]: one aligned load per stencil row
  int32_t n0, n1;
  float inv_h, h;             // first axis
  float inv_h1, h1;           // second axis
};

// Tabulated conditional angle law of one pair rule (mixed step): for start and new separations
// R0 = 1 + (a - 1) h, R' = 1 + (b - 1) h (a < n0, b < n1; node 0 a ghost) and CDF values
// U = sin^2(pi w / 2), w = (k - 1) / kAngTabU (k < kAngTabU + 3, first and last ghosts), the
// CDF value s(U) of the exact angle under the reference law, then (k = kAngTabU + 3) the reference
// law's concentration (Catmull-Rom in all three axes); d0max, d1max: the largest R0 - 1 and R' - 1
// inside the table.
struct AngTab {
  const float* v;             // n0 x n1 x kAngTabStride values, null when not built
  int32_t n0, n1;
  float h, inv_h, d0max, d1max;
  float inv_2tau, pad;
};

struct PairDev {
  int32_t bc, product, s1, s2;
  double sigma, tau, inv_tau, s, h, alpha, rcut2, Drel;
  float sigma_f, inv_sigma_f, inv_tau_f, rcut2_f;
  float s_f, alpha_f, pad_f[2];
  // 2D: small-time series (series2d != 0) or Weber quadrature nodes
  int32_t series2d, n_nodes;
  int32_t series2d_rad, pad_s;   // p_reac from the series as well (else the Weber quadrature)
  const WeberNode* nodes;
  const Series2D* ser;
  // mixed step: FP32 tables of p_reac (2D and 3D), F = p_enc e^{d d0/tau} and -ln(tail) (2D)
  Tab2 tab_preac, tab_penc, tab_tail;
  Tab2 tab_inv;               // propagator sample V = R - 1 at (R0 - 1, sqrt(-ln U))
  AngTab tab_ang;             // conditional angle law of the exact propagation
};

struct DecayDev {
  int32_t parent, n_products, p0, p1;
  double kd, sigma_place;
};

struct DevParams {
  int32_t dim, n_species, precision, n_replicas;
  int32_t n_pairs, n_decays, match_max_rounds, pad0;
  uint32_t match_single_max;   // conflict pairs matched by one block (more: the whole grid)
  uint32_t match_smem_max;     // conflict pairs matched in shared memory by that block
  int32_t angle_mode;          // 0: exact propagator direction; 1: free-step direction
  int32_t pad_angle;
  double dt;
  uint32_t seed_lo, seed_hi;
  uint32_t binned_mask;        // species that appear in an interacting pair rule
  uint32_t pad1;
  int64_t cap_particles, cap_pairs;
  double D[kMaxSpecies];
  float D_f[kMaxSpecies];
  double ell[kMaxSpecies];     // sqrt(2 D dt)
  float ell_f[kMaxSpecies];
  double ktot[kMaxSpecies];    // total unimolecular rate per species
  double p_uni[kMaxSpecies];   // 1 - exp(-ktot dt)
  unsigned long long uni_thr[kMaxSpecies];   // decay iff (52-bit draw m) < uni_thr
  double gl16[32];             // 16-point Gauss-Legendre nodes then weights on [-1, 1]
  int8_t pair_of[kMaxSpecies][kMaxSpecies];   // index into pairs, -1 = no interaction
  PairDev pairs[kMaxPairs];
  DecayDev decays[kMaxDecays];
  double rcut2_max;            // largest squared cut-off over the pair rules
  float rcut2_max_f, pad2;
  int32_t has_drift, pad3;
  double drift_dx[kMaxSpecies][3];   // drift displacement per step (v dt) of the split step
  float drift_dx_f[kMaxSpecies][3];
};

struct RepDev {
  double L, half_L;
  double inv_edge[3];
  float Lf, half_Lf;
  float inv_edge_f[3];
  int32_t nc[3];
  int64_t cell_base;
  uint32_t beg, end, next_id, pad;
};

struct DevCtl {
  uint32_t step;
  int32_t status;
  uint32_t n;              // particles alive
  uint32_t fired;          // fired pairs this step
  uint32_t n_conflict;     // pairs left to the iterative matching
  uint32_t n_decay;        // decays this step
  uint32_t n_accept;       // trivially accepted pairs this step (final once the matching phase starts)
  uint32_t n_round_acc;    // pairs accepted by the conflict rounds (appended after the trivial ones)
  uint32_t n_ang;          // angle jobs of this step
  uint32_t epoch;          // incremented every step; tags the scan flags
  uint32_t tile_ctr[2];    // tile tickets of the two scans
  uint32_t done_blocks;    // blocks of the compaction that finished
  uint32_t last_fired;     // fired pairs of the last completed step
  uint32_t bar_count;      // grid barrier of the cooperative matching: arrivals, generation
  uint32_t bar_gen;
  uint32_t live[2];        // live conflict pairs after a matching round (by round parity)
  uint32_t done_res;       // blocks of the matching / resolution kernel that finished
  uint32_t n_new;          // particles after this step (set with the replica table)
  uint32_t spin_limit;     // bound of the device waits in polls (0: the built-in bounds)
  uint32_t ph_steps;       // steps timed by the fused step's phase clock
  unsigned long long ph_t[8];    // fused step: global-timer stamp at the start of each phase
  unsigned long long ph_acc[8];  // fused step: accumulated ns per phase
  double t;
  unsigned long long stats[RD_NSTATS];
};

// Per-replica placement of this step's compaction (built once the resolution is complete):
// products before the replica's first particle, survivors up to and including the replica, and
// the replica's survivors and products.
struct RepX {
  uint32_t p_beg, s_end, surv, prod;
};

// A conflict pair as the matching rounds read it (one coalesced 32-B load per pair and phase):
// its fired-list index, particle indices, round state (FS_*), key bits and (id_a << 32 | id_b).
struct ConflictRec {
  uint32_t e, ia, ib, st;
  unsigned long long key, pid;
};

// An encountered pair (kind 0) or a decay's product pair (kind 1) whose new separation direction is
// drawn from the full propagator in the angle pass (one warp per job); the resolution pass has
// already decided everything else (length, reaction, products).
struct AngJob {
  double c[3];              // centre of diffusion
  double u[3];              // axis: the start separation's direction (decay: the contact direction)
  double fb[3];             // direction kept if the law needs more partial waves than the device holds
  double len;               // new separation length R' sigma
  double Rn, R0, tau;       // scaled lengths and time of the law
  double ca, cb;            // D_a / D_rel, D_b / D_rel
  double U_ang, U_azi;      // the angle's CDF value and the azimuth (2D: the sign) uniform
  uint32_t kind, ia, ib;    // kind (low byte) 0: particles ia, ib -> x1; 1: parent ia -> prodpos[2 ia ..
                            // 2 ia + 1]; the pair rule in the bits above
  uint32_t wa, wb, r;       // species/replica bits of the two particles, replica
};

struct FiredPair {          // 32 B
  uint32_t ia, ib;          // particle indices of this step, id[ia] < id[ib]
  uint32_t ida, idb;        // their ids
  double p;                 // p_enc
  double key;               // -ln(U_sel)/p_enc
};

// ------------------------------------------------------------------------------------------------
// Philox4x32-10 counter-based generator (Salmon et al., SC'11).
// ------------------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
#ifdef __CUDA_ARCH__
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
#else
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
#endif
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

__device__ __forceinline__ uint4 draw(const DevParams& P, uint32_t c0, uint32_t ida, uint32_t idb,
                                      uint32_t tag, uint32_t replica) {
  return philox(make_uint4(c0, ida, idb, tag | (replica << 8)), P.seed_lo, P.seed_hi);
}

// 52-bit uniform in (0,1), exact: ((x >> 12) + 1/2) 2^-52 with x = hi:lo.
__host__ __device__ __forceinline__ double u52(uint32_t hi, uint32_t lo) {
  const uint64_t x = ((uint64_t)hi << 32) | lo;
  return ((double)(x >> 12) + 0.5) * 0x1p-52;
}

// 23-bit uniform in (0,1) for the FP32 path: ((w >> 9) + 1/2) 2^-23, exact in float.
__device__ __forceinline__ float u23(uint32_t w) { return ((float)(w >> 9) + 0.5f) * 0x1p-23f; }

__device__ __forceinline__ void box_muller(double u1, double u2, double& n0, double& n1) {
  const double rad = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  n0 = rad * cs;
  n1 = rad * sn;
}

__device__ __forceinline__ void box_muller_f(float u1, float u2, float& n0, float& n1) {
  const float rad = sqrtf(-2.0f * logf(u1));
  float sn, cs;
  sincospif(2.0f * u2, &sn, &cs);
  n0 = rad * cs;
  n1 = rad * sn;
}

// Up to four FP64 unit normals from one (dim 2) or two (dim 3) Philox calls, tags tag0, tag0+1.
__device__ __forceinline__ void normals64(const DevParams& P, uint32_t c0, uint32_t id, uint32_t tag0,
                                          uint32_t replica, int count, double n[4]) {
  uint4 w = draw(P, c0, id, kOneParticle, tag0, replica);
  box_muller(u52(w.x, w.y), u52(w.z, w.w), n[0], n[1]);
  n[2] = n[3] = 0.0;
  if (count > 2) {
    w = draw(P, c0, id, kOneParticle, tag0 + 1, replica);
    box_muller(u52(w.x, w.y), u52(w.z, w.w), n[2], n[3]);
  }
}

// ------------------------------------------------------------------------------------------------
// periodic geometry
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ double min_image(double d, double L, double half_L) {
  if (d > half_L)
    d -= L;
  else if (d < -half_L)
    d += L;
  return d;
}

__device__ __forceinline__ float min_image_f(float d, float L, float half_L) {
  if (d > half_L)
    d -= L;
  else if (d < -half_L)
    d += L;
  return d;
}

__device__ __forceinline__ double wrap(double x, double L) {
  if (x >= L) {
    x -= L;
  } else if (x < 0.0) {
    x += L;
    if (x >= L) x = 0.0;
  }
  return x;
}

__device__ __forceinline__ float wrap_f(float x, float L) {
  if (x >= L) {
    x -= L;
  } else if (x < 0.0f) {
    x += L;
    if (x >= L) x = 0.0f;
  }
  return x;
}

// squared length with explicit round-to-nearest (no contraction), summed x, y, z.
__device__ __forceinline__ double norm2_rn(double a, double b, double c, int dim) {
  double s = __dmul_rn(a, a);
  s = __dadd_rn(s, __dmul_rn(b, b));
  if (dim == 3) s = __dadd_rn(s, __dmul_rn(c, c));
  return s;
}

__device__ __forceinline__ uint32_t w_bits(double w) { return (uint32_t)__double_as_longlong(w); }
__device__ __forceinline__ uint32_t w_bits(float w) { return __float_as_uint(w); }
__device__ __forceinline__ double w_from_bits_d(uint32_t b) { return __longlong_as_double((long long)b); }
__device__ __forceinline__ float w_from_bits_f(uint32_t b) { return __uint_as_float(b); }
__host__ __device__ __forceinline__ uint32_t pack_sp(uint32_t species, uint32_t replica) {
  return species | (replica << 8);
}

// ------------------------------------------------------------------------------------------------
// 3D radial Green's-function quantities (a = 1, tau = D dt / a^2), Section 4.1 of the paper.
// ------------------------------------------------------------------------------------------------
constexpr double kSqrtPi = 1.7724538509055160273;
constexpr double kPi = 3.14159265358979323846;

// Encounter probability, Eq. (bayes1D) with the radial g_abs of Section 4.1 and the angle-averaged
// free Gaussian: p_enc = exp(-(R-1)(R0-1)/tau) (1 - exp(-(R+R0-1)/tau)) / (1 - exp(-R R0/tau)).
__device__ __forceinline__ double p_enc3(double R, double R0, double inv_tau) {
  if (R <= 1.0) return 1.0;
  if (R0 < 1.0) R0 = 1.0;
  const double d = R - 1.0, d0 = R0 - 1.0;
  return exp(-d * d0 * inv_tau) * (expm1(-(R + R0 - 1.0) * inv_tau) / expm1(-R * R0 * inv_tau));
}

// FP32 form from the contact distances d = R-1, d0 = R0-1 (absolute error <= 2e-6 for the
// configurations' tau; checked against the FP64 oracle).
__device__ __forceinline__ float p_enc3_f(float d, float d0, float inv_tau) {
  if (d <= 0.0f) return 1.0f;
  if (d0 < 0.0f) d0 = 0.0f;
  const float num = expm1f(-(d + d0 + 1.0f) * inv_tau);
  const float den = expm1f(-(d + 1.0f) * (d0 + 1.0f) * inv_tau);
  return expf(-d * d0 * inv_tau) * (num / den);
}

// q(y) = 1 - sqrt(pi) y erfcx(y) >= 0 given ey = erfcx(y): direct below y = 12, asymptotic series
// sum_{k>=1} (-1)^(k+1) (2k-1)!! / (2 y^2)^k (16 terms) above.
__device__ __forceinline__ double q_ierfc(double y, double ey) {
  if (y < 12.0) return 1.0 - kSqrtPi * y * ey;
  const double x = 1.0 / (2.0 * y * y);
  double term = x, sum = x;
#pragma unroll
  for (int k = 1; k < 16; ++k) {
    term *= -(2.0 * k + 1.0) * x;
    sum += term;
  }
  return sum;
}

// Reaction probability, Eq. (psurv_radII), after removing the common factor
// exp(-u^2/4tau)/(8 pi R R0 sqrt(pi tau)) (u = R+R0-2, s = sqrt(tau), y = s + u/2s):
//   p_reac = sqrt(pi tau) [alpha erfcx(alpha s + u/2s) - erfcx(y)] / [q(y) + sqrt(pi) (u/2s) erfcx(y)]
// The denominator, 1 - sqrt(pi tau) erfcx(y), is written as a sum of non-negative terms.
__device__ __forceinline__ double p_reac3(double R, double R0, double s, double alpha) {
  if (R < 1.0) R = 1.0;
  if (R0 < 1.0) R0 = 1.0;
  const double z = (R + R0 - 2.0) / (2.0 * s);
  const double y = s + z;
  const double ey = erfcx(y);
  const double num = kSqrtPi * s * (alpha * erfcx(alpha * s + z) - ey);
  const double den = q_ierfc(y, ey) + kSqrtPi * z * ey;
  double p = num / den;
  return p < 0.0 ? 0.0 : (p > 1.0 ? 1.0 : p);
}

// FP32 forms of q and p_reac, used only to pre-screen the FP64 step's reaction decisions: below
// y = 1.5 q = 1 - sqrt(pi) y erfcx(y) directly, above it through the Laplace continued fraction of
// erfc (24 terms, q = K/(y+K) with K = (1/2)/(y + 1/(y + (3/2)/(y + ...)))).
__device__ __forceinline__ float q_ierfc_f(float y, float ey) {
  if (y < 1.5f) return 1.0f - 1.7724538509f * y * ey;
  float K = 0.0f;
#pragma unroll
  for (int k = 24; k >= 1; --k) K = (0.5f * k) / (y + K);
  return K / (y + K);
}

__device__ __forceinline__ float p_reac3_f(float R, float R0, float s, float alpha) {
  if (R < 1.0f) R = 1.0f;
  if (R0 < 1.0f) R0 = 1.0f;
  const float z = ((R - 1.0f) + (R0 - 1.0f)) / (2.0f * s);
  const float y = s + z;
  const float ey = erfcxf(y);
  const float num = 1.7724538509f * s * (alpha * erfcxf(alpha * s + z) - ey);
  const float den = q_ierfc_f(y, ey) + 1.7724538509f * z * ey;
  const float p = num / den;
  return p < 0.0f ? 0.0f : (p > 1.0f ? 1.0f : p);
}

// Decision U < p evaluated in FP32 first; only draws within kFilter of the FP32 value (whose error
// stays below a few 1e-6) need the FP64 value, so every decision equals the FP64 one.
constexpr double kFilter = 1e-4;

// Propagator G_ref - G_abs of an encountered pair (radial density 4 pi R^2 (g_ref - g_abs)).
// With w = R0-1, z = (V+w)/2s, z0 = w/2s, the normalised tail beyond R = 1 + V is
//   T(V) = exp(z0^2 - z^2) [erfcx(z) + V erfcx(s+z)] / erfcx(z0),
//   d ln T / dV = -(1+V) [q(s+z) + sqrt(pi) z erfcx(s+z)] / (s sqrt(pi) [erfcx(z) + V erfcx(s+z)]).
__device__ __forceinline__ void lnT3(double V, double w, double s, double inv_4tau, double ln_ex0,
                                     double& f, double& df) {
  const double z = (V + w) / (2.0 * s);
  const double ez = erfcx(z), y = s + z, ey = erfcx(y);
  const double body = ez + V * ey;
  f = -V * (2.0 * w + V) * inv_4tau + log(body) - ln_ex0;
  df = -(1.0 + V) * (q_ierfc(y, ey) + kSqrtPi * z * ey) / (s * kSqrtPi * body);
}

// FP32 evaluation of ln T and its derivative (the FP64 solve's seed; the mixed step's Newton step).
__device__ __forceinline__ void lnT3_f(float V, float w, float s, float inv_4tau, float ln_ex0, float& f, float& df) {
  const float z = (V + w) / (2.0f * s);
  const float ez = erfcxf(z), y = s + z, ey = erfcxf(y);
  const float body = ez + V * ey;
  const float q = y < 12.0f ? 1.0f - 1.7724538509f * y * ey : 0.5f / (y * y) * (1.0f - 1.5f / (y * y));
  f = -V * (2.0f * w + V) * inv_4tau + logf(body) - ln_ex0;
  df = -(1.0f + V) * (q + 1.7724538509f * z * ey) / (s * 1.7724538509f * body);
}

// Solves ln T(V) = ln U.  A few FP32 Newton steps give a seed good to ~1e-5; FP64 Newton steps,
// each kept inside the bracket known so far (bisection / expansion otherwise), finish the solve.
// Once an FP64 Newton step is below 1e-10 of the length scale max(V, s), quadratic convergence
// makes the new iterate accurate to rounding.
__device__ __forceinline__ double resample3(double U, double R0, double s) {
  if (R0 < 1.0) R0 = 1.0;
  const double w = R0 - 1.0;
  const double inv_4tau = 1.0 / (4.0 * s * s);
  const double lnU = log(U);
  // FP32 seed
  float Vf = 0.0f;
  {
    const float wf = (float)w, sf = (float)s, i4f = (float)inv_4tau, lnUf = (float)lnU;
    const float lnx0f = logf(erfcxf(wf / (2.0f * sf)));
    float lo = 0.0f, hi = -1.0f;
    for (int it = 0; it < 24; ++it) {
      float f, df;
      lnT3_f(Vf, wf, sf, i4f, lnx0f, f, df);
      const float g = f - lnUf;
      if (g == 0.0f) break;
      if (g > 0.0f)
        lo = Vf;
      else
        hi = Vf;
      float Vn = Vf - g / df;
      const bool inside = Vn >= lo && (hi < 0.0f || Vn <= hi);
      if (!inside) Vn = hi < 0.0f ? lo + fmaxf(lo, sf) : 0.5f * (lo + hi);
      const float step = fabsf(Vn - Vf);
      Vf = Vn;
      if (inside && step <= 1e-5f * fmaxf(Vf, sf)) break;
    }
    if (!(Vf >= 0.0f) || !isfinite(Vf)) Vf = 0.0f;
  }
  const double ln_ex0 = log(erfcx(w / (2.0 * s)));
  double lo = 0.0, hi = -1.0;          // hi < 0: no upper bound yet
  double V = (double)Vf, f = 0.0, df;
  for (int it = 0; it < 200; ++it) {
    lnT3(V, w, s, inv_4tau, ln_ex0, f, df);
    const double g = f - lnU;
    if (g == 0.0) break;
    if (g > 0.0)
      lo = V;
    else
      hi = V;
    double Vn = V - g / df;
    const bool inside = Vn >= lo && (hi < 0.0 || Vn <= hi);
    if (!inside) Vn = hi < 0.0 ? lo + fmax(lo, s) : 0.5 * (lo + hi);
    const double step = fabs(Vn - V);
    V = Vn;
    if (inside && step <= 1e-10 * fmax(V, s)) break;
    if (hi >= 0.0 && hi - lo <= 4e-16 * fmax(hi, s)) break;
  }
  return 1.0 + V;
}

__device__ __forceinline__ void cr_w(float t, float w[4]) {
  const float t2 = t * t, t3 = t2 * t;
  w[0] = 0.5f * (-t3 + 2.0f * t2 - t);
  w[1] = 0.5f * (3.0f * t3 - 5.0f * t2 + 2.0f);
  w[2] = 0.5f * (-3.0f * t3 + 4.0f * t2 + t);
  w[3] = 0.5f * (t3 - t2);
}

// derivative of the Catmull-Rom weights with respect to t
__device__ __forceinline__ void cr_dw(float t, float w[4]) {
  const float t2 = t * t;
  w[0] = 0.5f * (-3.0f * t2 + 4.0f * t - 1.0f);
  w[1] = 0.5f * (9.0f * t2 - 10.0f * t);
  w[2] = 0.5f * (-9.0f * t2 + 8.0f * t + 1.0f);
  w[3] = 0.5f * (3.0f * t2 - 2.0f * t);
}

// bicubic Catmull-Rom value and its derivative along the second axis at (d0, d) >= 0
__device__ __forceinline__ float tab_eval_dd(const Tab2& T, float d0, float d, float& dval) {
  float x = d0 * T.inv_h + 1.0f, y = d * T.inv_h1 + 1.0f;
  x = fminf(fmaxf(x, 1.0f), (float)(T.n0 - 3) - 1e-3f);
  y = fminf(fmaxf(y, 1.0f), (float)(T.n1 - 3) - 1e-3f);
  const int i = (int)x, j = (int)y;
  float wx[4], wy[4], dwy[4];
  cr_w(x - i, wx);
  cr_w(y - j, wy);
  cr_dw(y - j, dwy);
  float4 v[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) v[a] = __ldg(T.q + (size_t)(i - 1 + a) * T.n1 + j);
  float acc = 0.0f, dacc = 0.0f;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    acc += wx[a] * (wy[0] * v[a].x + wy[1] * v[a].y + wy[2] * v[a].z + wy[3] * v[a].w);
    dacc += wx[a] * (dwy[0] * v[a].x + dwy[1] * v[a].y + dwy[2] * v[a].z + dwy[3] * v[a].w);
  }
  dval = dacc * T.inv_h1;
  return acc;
}

// bicubic Catmull-Rom value at (d0, d) >= 0 (clamped to the table)
__device__ __forceinline__ float tab_eval(const Tab2& T, float d0, float d) {
  float x = d0 * T.inv_h + 1.0f, y = d * T.inv_h1 + 1.0f;
  x = fminf(fmaxf(x, 1.0f), (float)(T.n0 - 3) - 1e-3f);
  y = fminf(fmaxf(y, 1.0f), (float)(T.n1 - 3) - 1e-3f);
  const int i = (int)x, j = (int)y;
  float wx[4], wy[4];
  cr_w(x - i, wx);
  cr_w(y - j, wy);
  float4 v[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) v[a] = __ldg(T.q + (size_t)(i - 1 + a) * T.n1 + j);
  float acc = 0.0f;
#pragma unroll
  for (int a = 0; a < 4; ++a) acc += wx[a] * (wy[0] * v[a].x + wy[1] * v[a].y + wy[2] * v[a].z + wy[3] * v[a].w);
  return acc;
}

// table p_reac (clamped to [0,1])
__device__ __forceinline__ float p_reac_tab(const PairDev& pr, float d, float d0) {
  const float p = tab_eval(pr.tab_preac, fmaxf(d0, 0.0f), fmaxf(d, 0.0f));
  return fminf(fmaxf(p, 0.0f), 1.0f);
}

}  // namespace rd
