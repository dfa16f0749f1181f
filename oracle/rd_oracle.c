/*
 * Plain serial FP64 CPU oracle of one Green's-function-corrected Brownian-dynamics step
 * (Pruestel & Meier-Schellersheim, "Coarse-grained stochastic particle-based reaction-diffusion
 * simulation algorithm", arXiv:1107.0270).
 *
 * TEST INFRASTRUCTURE ONLY: this file is the independent checker of the CUDA library.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load it.  It is slow on
 * purpose: an O(N^2) candidate search, a sort-based greedy matching and bisection root finding,
 * so that each step can be read against the paper.
 *
 * Conventions fixed where the paper is silent (they are the library's step specification too):
 *  - random numbers: Philox4x32-10 (Salmon et al., SC'11), key = (seed lo, seed hi), counter =
 *    (step, id_a, id_b, tag | replica << 8), id_b = 0xFFFFFFFF for one-particle streams;
 *    U = ((x >> 12) + 0.5) 2^-52 from x = (w_hi << 32) | w_lo, exactly representable, in (0,1);
 *    normals by Box-Muller.
 *  - candidate pairs: interacting species pairs whose minimum-image start-of-step distance is
 *    below r_cut = sigma + c sqrt(2 D dt) (Section 3, cut-off radius).
 *  - conflicts (Section 3, "Details"): key = -ln(U_sel)/p_enc per fired pair; fired pairs are
 *    accepted greedily in ascending (key, id_a, id_b); an exponential race gives each particle the
 *    paper's selection probability p_enc,j / sum p_enc among its own fired candidates.
 *  - unimolecular decays are drawn first from the start-of-step state; decaying particles neither
 *    move freely nor pair this step.  Products take no part in bimolecular reactions this step.
 *  - an encountered pair's new separation is drawn from the full propagator G_ref - G_abs
 *    (Eq. passage_prob): its length from the radial law, its angle to the start separation from
 *    the partial-wave series of Eqs. genericGF3D / genericGF (angle_mode 0); angle_mode 1 keeps
 *    the free step's direction instead.
 *  - products: a bimolecular product sits at the centre of diffusion (Eq. Rcoo) of the pair; ids
 *    are next_id + rank of the event ordered by its lower parent id; survivors keep their order
 *    and products are appended, so the particle array stays sorted by id.
 */
#define _DEFAULT_SOURCE
#include "oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846

/* Test hook for negative controls: plants one deliberate mistake so that a test can show its
 * statistic rejects it.  0 (default): the method as specified.
 *   1: conflict key = -ln(U_sel) * p_enc instead of -ln(U_sel) / p_enc
 *   2: fired pairs accepted greedily in DESCENDING key order
 *   3: the encounter draw U_enc reused as the selection draw
 *   4: the 3D boundary coefficients with the cylindrical derivative j_n' = j_{n-1} - n/z j_n */
static int g_fault = 0;
void or_set_fault(int fault) { g_fault = fault; }
#define SQRT_PI 1.77245385090551602730
#define NEAR_THRESHOLD 1e-9

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32->64 multiplies with  */
/* the published multipliers, key bumped by the two Weyl constants between rounds.              */
/* ------------------------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double or_u52(uint32_t hi, uint32_t lo) {
  uint64_t x = ((uint64_t)hi << 32) | (uint64_t)lo;
  return ((double)(x >> 12) + 0.5) * 0x1p-52;
}

static void stream(const or_system* sys, uint32_t c0, uint32_t ida, uint32_t idb, uint32_t tag,
                   uint32_t out[4]) {
  uint32_t ctr[4] = {c0, ida, idb, tag | (sys->replica << 8)};
  uint32_t key[2] = {(uint32_t)(sys->seed & 0xFFFFFFFFu), (uint32_t)(sys->seed >> 32)};
  or_philox4x32_10(ctr, key, out);
}

/* Box-Muller: two independent unit normals from two uniforms in (0,1). */
static void box_muller(double u1, double u2, double* n0, double* n1) {
  double rad = sqrt(-2.0 * log(u1));
  *n0 = rad * cos(2.0 * PI * u2);
  *n1 = rad * sin(2.0 * PI * u2);
}

/* Up to four unit normals from one or two Philox calls with consecutive tags. */
static void normals(const or_system* sys, uint32_t c0, uint32_t id, uint32_t tag0, int count,
                    double* n) {
  uint32_t w[4];
  stream(sys, c0, id, 0xFFFFFFFFu, tag0, w);
  box_muller(or_u52(w[0], w[1]), or_u52(w[2], w[3]), &n[0], &n[1]);
  if (count > 2) {
    double extra;
    stream(sys, c0, id, 0xFFFFFFFFu, tag0 + 1, w);
    box_muller(or_u52(w[0], w[1]), or_u52(w[2], w[3]), &n[2], &extra);
    if (count > 3) n[3] = extra;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* erfcx(x) = exp(x^2) erfc(x).  For x < 4 the product of libm's exp and erfc; for x >= 4 the    */
/* Laplace continued fraction of erfc (Abramowitz & Stegun 7.1.14),                             */
/*   sqrt(pi) erfcx(x) = 1/(x + (1/2)/(x + 1/(x + (3/2)/(x + 2/(x + ...))))),                   */
/* evaluated by the modified Lentz method.  cf_tail returns the tail K = (1/2)/(x + 1/(x + ...))  */
/* so that sqrt(pi) erfcx(x) = 1/(x + K).                                                         */
/* ------------------------------------------------------------------------------------------ */
static double cf_tail(double x) {
  /* Modified Lentz for f = b0 + a1/(b1 + a2/(b2 + ...)) with b0 = 0, a_n = n/2, b_n = x. */
  const double tiny = 1e-300;
  double f = tiny, C = f, Dv = 0.0;
  for (int n = 1; n < 5000; ++n) {
    double an = 0.5 * n;
    Dv = x + an * Dv;
    if (fabs(Dv) < tiny) Dv = tiny;
    Dv = 1.0 / Dv;
    C = x + an / C;
    if (fabs(C) < tiny) C = tiny;
    double delta = C * Dv;
    f *= delta;
    if (fabs(delta - 1.0) < 1e-16) break;
  }
  return f;
}

double or_erfcx(double x) {
  if (x < 0.0) return 2.0 * exp(x * x) - or_erfcx(-x);
  if (x < 4.0) return exp(x * x) * erfc(x);
  return 1.0 / (SQRT_PI * (x + cf_tail(x)));
}

/* ------------------------------------------------------------------------------------------ */
/* 3D, Section 4.1.  With a = 1, tau = D t / a^2, u = R + R0 - 2, s = sqrt(tau):                  */
/*  g_abs = [exp(-(R-R0)^2/4tau) - exp(-u^2/4tau)] / (8 pi R R0 sqrt(pi tau))                      */
/*  g_rad = [exp(-(R-R0)^2/4tau) + exp(-u^2/4tau)                                                  */
/*          - alpha sqrt(4 pi tau) exp(alpha^2 tau + alpha u) erfc(alpha s + u/2s)] / (same)       */
/*  g_ref = g_rad at kappa_a = 0, alpha = 1 + h (the paper's kappa := (kappa_a+4 pi a D)/(4 pi a D)) */
/* The radial free function is the angular average of the free Gaussian of Eq. (gaussian):       */
/*  g_free = [exp(-(R-R0)^2/4tau) - exp(-(R+R0)^2/4tau)] / (8 pi R R0 sqrt(pi tau)).               */
/* ------------------------------------------------------------------------------------------ */

/* Eq. (bayes1D) with radial Green's functions (Section 2.2.4): p_enc = 1 - g_abs/g_free.
 * Dividing numerator and denominator by exp(-(R-R0)^2/4tau) and using
 * (R+R0-2)^2 - (R-R0)^2 = 4 (R-1)(R0-1),  (R+R0)^2 - (R-R0)^2 = 4 R R0:
 *   g_abs/g_free = (1 - exp(-(R-1)(R0-1)/tau)) / (1 - exp(-R R0/tau)).
 * An overlapping end point (R <= 1) has certainly met the boundary (Section 3, step 2). */
double or_p_enc3(double R, double R0, double tau) {
  if (R <= 1.0) return 1.0;
  if (R0 < 1.0) R0 = 1.0;
  double ratio = (-expm1(-(R - 1.0) * (R0 - 1.0) / tau)) / (-expm1(-R * R0 / tau));
  return 1.0 - ratio;
}

/* Eq. (psurv_radII): p_reac = (g_ref - g_rad) / (g_ref - g_abs).
 * With E2 = exp(-u^2/4tau) and the identity exp(alpha^2 tau + alpha u) erfc(alpha s + u/2s)
 * = E2 erfcx(alpha s + u/2s) (because (alpha s + u/2s)^2 = alpha^2 tau + alpha u + u^2/4tau), the
 * common factor E2/(8 pi R R0 sqrt(pi tau)) cancels and the exp(-(R-R0)^2/4tau) terms drop out:
 *   g_ref - g_abs ~ 2 - sqrt(4 pi tau) erfcx(s + u/2s)
 *   g_ref - g_rad ~ sqrt(4 pi tau) [alpha erfcx(alpha s + u/2s) - erfcx(s + u/2s)]. */
double or_p_reac3(double R, double R0, double tau, double h) {
  if (R < 1.0) R = 1.0;
  if (R0 < 1.0) R0 = 1.0;
  double s = sqrt(tau), u = R + R0 - 2.0, alpha = 1.0 + h;
  double c = sqrt(4.0 * PI * tau);
  double ref_minus_abs = 2.0 - c * or_erfcx(s + u / (2.0 * s));
  double ref_minus_rad = c * (alpha * or_erfcx(alpha * s + u / (2.0 * s)) - or_erfcx(s + u / (2.0 * s)));
  double p = ref_minus_rad / ref_minus_abs;
  if (p < 0.0) p = 0.0;
  if (p > 1.0) p = 1.0;
  return p;
}

/* Radial propagator of an encountered pair (Section 3, "Details"): density 4 pi R^2 (g_ref - g_abs)
 * on R > 1.  Its integral over (1+V, inf) is, in closed form (w = R0 - 1, z = (V+w)/2s),
 *   [erfc(z) + V exp(-z^2) erfcx(s + z)] / R0,
 * (differentiate: d/dV gives -4 pi R^2 (g_ref - g_abs)), and over (1, inf) it is
 * 1 - S_abs = erfc(w/2s)/R0.  or_tail3 returns the normalised tail fraction T(V) in [0,1]. */
double or_tail3(double V, double R0, double tau) {
  if (R0 < 1.0) R0 = 1.0;
  double s = sqrt(tau), w = R0 - 1.0;
  double z = (V + w) / (2.0 * s), z0 = w / (2.0 * s);
  double num = erfc(z) + V * exp(-z * z) * or_erfcx(s + z);
  return num / erfc(z0);
}

/* Inverse of the tail fraction: the R' >= 1 with T(R'-1) = U, by plain bisection to the last bit
 * (T decreases monotonically from 1 at V = 0 to 0 as V grows). */
double or_resample3(double U, double R0, double tau) {
  double s = sqrt(tau);
  double lo = 0.0, hi = s;
  while (or_tail3(hi, R0, tau) > U) {
    lo = hi;
    hi *= 2.0;
  }
  for (int it = 0; it < 2000; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (or_tail3(mid, R0, tau) > U)
      lo = mid;
    else
      hi = mid;
  }
  return 1.0 + 0.5 * (lo + hi);
}

/* Survival probabilities, Eq. (SurvRad), by integrating the radial g's above over R > 1. */
double or_S_abs3(double R0, double tau) {
  double s = sqrt(tau);
  return 1.0 - erfc((R0 - 1.0) / (2.0 * s)) / R0;
}

double or_S_rad3(double R0, double tau, double h) {
  double s = sqrt(tau), w = R0 - 1.0, alpha = 1.0 + h;
  double z0 = w / (2.0 * s);
  return 1.0 - (h / alpha) / R0 * (erfc(z0) - exp(-z0 * z0) * or_erfcx(z0 + alpha * s));
}

/* ------------------------------------------------------------------------------------------ */
/* Adaptive Gauss-Legendre quadrature.  The 16-point nodes and weights are computed once by       */
/* Newton's method on the Legendre polynomial (three-term recurrence); an interval is accepted     */
/* when the rule on it and the rule on its two halves agree within the tolerance.               */
/* ------------------------------------------------------------------------------------------ */
#define GL_N 16
static double gl_x[GL_N], gl_w[GL_N];
static int gl_ready = 0;

static void gl_init(void) {
  if (gl_ready) return;
  for (int i = 0; i < GL_N; ++i) {
    double x = cos(PI * (i + 0.75) / (GL_N + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= GL_N; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = GL_N * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    gl_x[i] = x;
    gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  gl_ready = 1;
}

typedef double (*or_fn)(double, const void*);

static double gl_rule(or_fn f, const void* ctx, double a, double b) {
  double m = 0.5 * (a + b), h = 0.5 * (b - a), s = 0.0;
  for (int i = 0; i < GL_N; ++i) s += gl_w[i] * f(m + h * gl_x[i], ctx);
  return s * h;
}

static double gl_adapt(or_fn f, const void* ctx, double a, double b, double whole, double tol, int depth,
                       long* budget) {
  double m = 0.5 * (a + b);
  double left = gl_rule(f, ctx, a, m), right = gl_rule(f, ctx, m, b);
  *budget -= 2 * GL_N;
  if (depth <= 0 || *budget <= 0 || fabs(left + right - whole) <= tol) return left + right;
  return gl_adapt(f, ctx, a, m, left, 0.5 * tol, depth - 1, budget) +
         gl_adapt(f, ctx, m, b, right, 0.5 * tol, depth - 1, budget);
}

/* integral of f over [a,b]: `pieces` equal panels, each refined until halving changes it by less
 * than its share of rel * |first estimate| (at most 2e5 integrand evaluations in all) */
static double integrate(or_fn f, const void* ctx, double a, double b, int pieces, double rel) {
  gl_init();
  double hstep = (b - a) / pieces, first = 0.0, scale = 0.0;
  double est[4096];
  if (pieces > 4096) pieces = 4096;
  for (int k = 0; k < pieces; ++k) {
    est[k] = gl_rule(f, ctx, a + k * hstep, a + (k + 1) * hstep);
    first += est[k];
    scale += fabs(est[k]);
  }
  double tol = rel * (scale > 0.0 ? scale : 1.0) + 1e-300;
  long budget = 200000;
  double s = 0.0;
  for (int k = 0; k < pieces; ++k)
    s += gl_adapt(f, ctx, a + k * hstep, a + (k + 1) * hstep, est[k], tol / pieces, 30, &budget);
  (void)first;
  return s;
}

/* ------------------------------------------------------------------------------------------ */
/* 2D, Section 4.2.  Scaled units a = 1, tau = D t / a^2, h = kappa_a / (2 pi D) (Eq. 2Dh).        */
/* ------------------------------------------------------------------------------------------ */

/* e^{z^2} i^n erfc(z) for n >= -1, z >= 0, from the recursion 2n i^n erfc = i^{n-2} erfc -
 * 2z i^{n-1} erfc (Section 4.2) with i^{-1} erfc = (2/sqrt(pi)) e^{-z^2}, i^0 erfc = erfc.  Each
 * direction is used where it is stable: upward for z < 1, and for z >= 1 downward on the ratios
 * r_n = i^n erfc / i^{n-1} erfc, r_{n-1} = 1/(2z + 2n r_n), started at a high order from the
 * asymptotic ratio (Miller's backward recurrence). */
double or_ierfc_scaled(int n, double z) {
  if (n == -1) return 2.0 / SQRT_PI;
  double f = or_erfcx(z);
  if (n == 0) return f;
  if (z < 1.0) {
    double fm2 = 2.0 / SQRT_PI, fm1 = f;
    for (int k = 1; k <= n; ++k) {
      double fk = (fm2 - 2.0 * z * fm1) / (2.0 * k);
      fm2 = fm1;
      fm1 = fk;
    }
    return fm1;
  }
  int M = n + 120;
  double r = (-z + sqrt(z * z + 2.0 * M)) / (2.0 * M);
  double ratio[64];
  for (int k = M; k >= 1; --k) {
    if (k <= n) ratio[k] = r;
    r = 1.0 / (2.0 * z + 2.0 * k * r);
  }
  for (int k = 1; k <= n; ++k) f *= ratio[k];
  return f;
}

/* a_k(nu) of the large-argument expansions of I_nu and K_nu (Eq. coeffDef) */
static double a_coef(int k, double nu) {
  double v = 1.0;
  for (int j = 1; j <= k; ++j) v *= (4.0 * nu * nu - (2.0 * j - 1.0) * (2.0 * j - 1.0)) / (8.0 * j);
  return v;
}

/* power-series division c = a / b up to order n */
static void series_div(const double* a, const double* b, double* c, int n) {
  for (int k = 0; k <= n; ++k) {
    double v = a[k];
    for (int j = 1; j <= k; ++j) v -= b[j] * c[k - j];
    c[k] = v / b[0];
  }
}

static void series_mul(const double* a, const double* b, double* c, int n) {
  for (int k = 0; k <= n; ++k) {
    double v = 0.0;
    for (int j = 0; j <= k; ++j) v += a[j] * b[k - j];
    c[k] = v;
  }
}

/* gamma_k of the expansions (expansionLaplace): with y = 1/q~, the boundary quotient of Eqs.
 * (absPert), (refPert), (radPert) divided by its leading exponential is I0/K0 (abs), I1/K1 (ref)
 * or (I1 - h y I0)/(K1 + h y K0) (rad), expanded with the a_k series (I'_0 = I_1, K'_0 = -K_1), and
 * multiplied by the K_0(q~R0) K_0(q~R) series.  Returns gamma_k, k = 0..24. */
static void gamma_series(int bc, double R, double R0, double h, int n, double* g) {
  double A0[32], A0m[32], A1[32], A1m[32], num[32], den[32], ratio[32], k0a[32], k0b[32], kk[32];
  for (int k = 0; k <= n; ++k) {
    double sgn = (k & 1) ? -1.0 : 1.0;
    A0[k] = a_coef(k, 0.0);
    A0m[k] = sgn * A0[k];
    A1[k] = a_coef(k, 1.0);
    A1m[k] = sgn * A1[k];
    k0a[k] = A0[k] / pow(R0, k);
    k0b[k] = A0[k] / pow(R, k);
  }
  for (int k = 0; k <= n; ++k) {
    if (bc == OR_BC_ABS) {
      num[k] = A0m[k];
      den[k] = A0[k];
    } else {
      double hh = bc == OR_BC_RAD ? h : 0.0;
      num[k] = A1m[k] - (k > 0 ? hh * A0m[k - 1] : 0.0);
      den[k] = A1[k] + (k > 0 ? hh * A0[k - 1] : 0.0);
    }
  }
  series_div(num, den, ratio, n);
  series_mul(k0a, k0b, kk, n);
  series_mul(ratio, kk, g, n);
}

double or_gamma2(int k, int bc, double R, double R0, double h) {
  double g[32];
  if (k < 0 || k > 24) return NAN;
  gamma_series(bc, R, R0, h, k, g);
  return g[k];
}

/* bracket of Eqs. (smallTEabs)/(smallTEabsII) after factoring out e^{-z^2}:
 * pi^{-1/2} + (1/2) sum_{n=1}^{N} gamma_n e^{z^2} i^{n-1} erfc(z) (2 sqrt(tau))^n */
static double series_bracket(int bc, double R, double R0, double tau, double h, int N) {
  double g[32];
  gamma_series(bc, R, R0, h, N, g);
  double s = sqrt(tau), z = (R + R0 - 2.0) / (2.0 * s), sum = 1.0 / SQRT_PI, p = 1.0;
  for (int n = 1; n <= N; ++n) {
    p *= 2.0 * s;
    sum += 0.5 * g[n] * or_ierfc_scaled(n - 1, z) * p;
  }
  return sum;
}

/* boundary part g_bc of the radial Green's function, Eqs. (smallTEabs), (smallTEabsII) */
double or_gbc2_series(int bc, double R, double R0, double tau, double h, int nterms) {
  double s = sqrt(tau), z = (R + R0 - 2.0) / (2.0 * s);
  double pref = exp(-z * z) / (4.0 * PI * sqrt(tau * R * R0));
  double sign = bc == OR_BC_ABS ? -1.0 : 1.0;
  return sign * pref * series_bracket(bc, R, R0, tau, h, nterms);
}

/* e^{-x} I0(x): power series below x = 30, large-argument series above */
static double i0e(double x) {
  if (x < 30.0) {
    double t = 1.0, s = 1.0, q = 0.25 * x * x;
    for (int k = 1; k < 400; ++k) {
      t *= q / ((double)k * k);
      s += t;
      if (t < 1e-17 * s) break;
    }
    return s * exp(-x);
  }
  double s = 0.0, t = 1.0;
  for (int k = 0; k < 30; ++k) {
    if (k > 0) t *= (2.0 * k - 1.0) * (2.0 * k - 1.0) / (8.0 * k * x);
    s += t;
  }
  return s / sqrt(2.0 * PI * x);
}

/* radial free function: angular average of the free Gaussian of Section 2.1 in 2D */
double or_gfree2(double R, double R0, double tau) {
  return exp(-(R - R0) * (R - R0) / (4.0 * tau)) * i0e(R * R0 / (2.0 * tau)) / (4.0 * PI * tau);
}

/* C_0(R, x) of Eq. (fRad), with J_0' = -J_1, Y_0' = -Y_1:
 * C_0 = [Y0(Rx) alpha - J0(Rx) beta] / sqrt(alpha^2 + beta^2), alpha = x J1(x) + h J0(x),
 * beta = x Y1(x) + h Y0(x); absorbing is the h -> infinity limit (alpha = J0, beta = Y0). */
static void c0_coeffs(int bc, double x, double h, double* al, double* be, double* nrm) {
  if (bc == OR_BC_ABS) {
    *al = j0(x);
    *be = y0(x);
  } else {
    double hh = bc == OR_BC_RAD ? h : 0.0;
    *al = x * j1(x) + hh * j0(x);
    *be = x * y1(x) + hh * y0(x);
  }
  *nrm = sqrt((*al) * (*al) + (*be) * (*be));
}

typedef struct {
  double R, R0, tau, h;
  double coef[4];      /* weights of the abs, ref, rad products */
  int cdf;             /* 0: g; 1: integral of 2 pi R g over (1, R) */
} weber_ctx;

/* integrand in t with x = t^2 (dx = 2t dt) */
static double weber_integrand(double t, const void* vp) {
  const weber_ctx* c = (const weber_ctx*)vp;
  double x = t * t;
  if (x <= 0.0) return 0.0;
  double w = exp(-c->tau * x * x), s = 0.0;
  for (int bc = OR_BC_ABS; bc <= OR_BC_RAD; ++bc) {
    if (c->coef[bc] == 0.0) continue;
    double al, be, nr;
    c0_coeffs(bc, x, c->h, &al, &be, &nr);
    double c0r0 = (y0(c->R0 * x) * al - j0(c->R0 * x) * be) / nr;
    double other;
    if (!c->cdf) {
      other = (y0(c->R * x) * al - j0(c->R * x) * be) / nr;                    /* C_0(R, x) */
    } else {
      /* integral of R' C_0(R', x) over (1, R): R' Z_1(R' x) / x is an antiderivative of R' Z_0(R' x) */
      double hi = c->R * (y1(c->R * x) * al - j1(c->R * x) * be);
      double lo = y1(x) * al - j1(x) * be;
      other = (hi - lo) / (x * nr);
    }
    s += c->coef[bc] * c0r0 * other;
  }
  return w * s * x * 2.0 * t;
}

static double weber(weber_ctx* c) {
  double T = pow(60.0 / c->tau, 0.25);
  double rmax = c->R > c->R0 ? c->R : c->R0;
  int pieces = 8 + (int)(rmax * T * T / 3.0);
  double v = integrate(weber_integrand, c, 0.0, T, pieces, 1e-13);
  return c->cdf ? v : v / (2.0 * PI);
}

/* the exact radial Green's function from the n = 0 term of Eq. (genericGF):
 * g = (1/2pi) int_0^inf e^{-tau x^2} C_0(R,x) C_0(R0,x) x dx; returns the boundary part g - g_free */
double or_gbc2_weber(int bc, double R, double R0, double tau, double h) {
  weber_ctx c = {R, R0, tau, h, {0, 0, 0, 0}, 0};
  c.coef[bc] = 1.0;
  return weber(&c) - or_gfree2(R, R0, tau);
}

/* Eq. (bayes1D) in 2D: p_enc = 1 - g_abs/g_free = -g_abs^bc/g_free.  In the small-time regime
 * (tau <= tau_s) both g_abs^bc (Eq. smallTEabs, prefactor e^{-(R+R0-2)^2/4tau}/(4 pi sqrt(tau R R0)))
 * and g_free (prefactor e^{-(R-R0)^2/4tau}/(4 pi tau)) carry Gaussian factors whose ratio is
 * e^{-(R-1)(R0-1)/tau}, so p_enc = e^{-(R-1)(R0-1)/tau} sqrt(tau) B_abs / (sqrt(R R0) I0e(R R0/2tau))
 * with B_abs the bracket of Eq. (smallTEabs); otherwise the Weber integral. */
double or_p_enc2(double R, double R0, double tau, double tau_s) {
  if (R <= 1.0) return 1.0;
  if (R0 < 1.0) R0 = 1.0;
  if (R0 == 1.0) return 1.0;
  if (tau <= tau_s) {
    double b = series_bracket(OR_BC_ABS, R, R0, tau, 0.0, 12);
    return exp(-(R - 1.0) * (R0 - 1.0) / tau) * sqrt(tau) * b / (sqrt(R * R0) * i0e(R * R0 / (2.0 * tau)));
  }
  weber_ctx c = {R, R0, tau, 0.0, {0, 0, 0, 0}, 0};
  c.coef[OR_BC_ABS] = 1.0;
  return 1.0 - weber(&c) / or_gfree2(R, R0, tau);
}

/* Eq. (psurv_radII) in 2D; the free parts cancel (Section 4.2), and in the small-time regime so
 * does the common prefactor of Eqs. (smallTEabs)/(smallTEabsII): p_reac = (B_ref - B_rad)/(B_ref + B_abs)
 * with B the brackets (g_abs^bc carries the opposite sign). */
/* The radiation bracket's series coefficients grow like powers of h: the series is used only while
 * h sqrt(tau) <= OR_SERIES_H_SQRT_TAU (truncation error ~1e-8 there); beyond, the exact Weber
 * integral (strongly reactive pairs). */
#define OR_SERIES_H_SQRT_TAU 0.3
double or_p_reac2(double R, double R0, double tau, double h, double tau_s) {
  if (R < 1.0) R = 1.0;
  if (R0 < 1.0) R0 = 1.0;
  if (tau <= tau_s && h * sqrt(tau) <= OR_SERIES_H_SQRT_TAU) {
    double bref = series_bracket(OR_BC_REF, R, R0, tau, h, 12);
    double brad = series_bracket(OR_BC_RAD, R, R0, tau, h, 12);
    double babs = series_bracket(OR_BC_ABS, R, R0, tau, h, 12);
    double p = (bref - brad) / (bref + babs);
    return p < 0.0 ? 0.0 : (p > 1.0 ? 1.0 : p);
  }
  /* numerator and denominator of Eq. (psurv_radII) each integrated as one difference (the free
   * parts cancel inside the integrand, Section 4.2), so that the adaptive rule's tolerance is
   * relative to the difference itself, not to the much larger single Green's functions */
  weber_ctx num = {R, R0, tau, h, {0, 0, 0, 0}, 0}, den = {R, R0, tau, h, {0, 0, 0, 0}, 0};
  num.coef[OR_BC_REF] = 1.0;
  num.coef[OR_BC_RAD] = -1.0;
  den.coef[OR_BC_REF] = 1.0;
  den.coef[OR_BC_ABS] = -1.0;
  double p = weber(&num) / weber(&den);
  return p < 0.0 ? 0.0 : (p > 1.0 ? 1.0 : p);
}

/* density 2 pi R (g_ref - g_abs) of an encountered pair's new separation (small-time series) */
typedef struct { double R0, tau; } dens_ctx;
static double dens2_series(double R, const void* vp) {
  const dens_ctx* c = (const dens_ctx*)vp;
  return 2.0 * PI * R *
         (or_gbc2_series(OR_BC_REF, R, c->R0, c->tau, 0.0, 12) - or_gbc2_series(OR_BC_ABS, R, c->R0, c->tau, 0.0, 12));
}

/* normalised tail T(V) of the propagator G_ref - G_abs beyond R = 1 + V (Section 3, "Details");
 * the total over R > 1 is 1 - S_abs */
/* unnormalised CDF of the new separation over (1, 1 + V): integral of 2 pi R (g_ref - g_abs) */
static double cdf2(double V, double R0, double tau, double tau_s) {
  if (tau <= tau_s) {
    dens_ctx c = {R0, tau};
    return integrate(dens2_series, &c, 1.0, 1.0 + V, 8, 1e-12);
  }
  weber_ctx c = {1.0 + V, R0, tau, 0.0, {0, 0, 0, 0}, 1};
  c.coef[OR_BC_REF] = 1.0;
  c.coef[OR_BC_ABS] = -1.0;
  return weber(&c);
}

/* beyond 1 + vmax2 the density is below e^{-40} of its peak */
static double vmax2(double R0, double tau) { return R0 + 13.0 * sqrt(tau); }

double or_tail2(double V, double R0, double tau, double tau_s) {
  if (R0 < 1.0) R0 = 1.0;
  const double vmax = vmax2(R0, tau);
  if (V >= vmax) return 0.0;
  double t = 1.0 - cdf2(V, R0, tau, tau_s) / cdf2(vmax, R0, tau, tau_s);
  return t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
}

/* encountered fraction 1 - S_abs(tau | R0) = integral of 2 pi R (g_ref - g_abs) over R > 1 */
double or_S_abs2(double R0, double tau) {
  if (R0 < 1.0) R0 = 1.0;
  return 1.0 - cdf2(vmax2(R0, tau), R0, tau, 0.0);
}

double or_resample2(double U, double R0, double tau, double tau_s) {
  if (R0 < 1.0) R0 = 1.0;
  const double vmax = vmax2(R0, tau);
  const double tot = cdf2(vmax, R0, tau, tau_s);
  /* T(V) = 1 - cdf(V)/tot decreases from 1 to 0 on (0, vmax): bisection for T(V) = U */
  double lo = 0.0, hi = vmax;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi || hi - lo < 1e-14 * (1.0 + hi)) break;
    if (1.0 - cdf2(mid, R0, tau, tau_s) / tot > U)
      lo = mid;
    else
      hi = mid;
  }
  return 1.0 + 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------------------------ */
/* Exact propagation of an encountered pair (Eq. passage_prob with the full Green's functions of   */
/* Eqs. genericGF3D / genericGF): the new separation vector r' is drawn from G_ref - G_abs.  Its   */
/* length R' follows the radial law above (the n = 0 term); its angle to the start separation r0  */
/* follows, given R', the partial-wave series                                                      */
/*   3D: f(mu) = sum_n (2n+1) P_n(mu) D_n / (2 D_0),      mu = cos(angle),                         */
/*   2D: f(theta) = [D_0 + 2 sum_{n>=1} D_n cos(n theta)] / (2 pi D_0),                           */
/* with D_n the n-th Weber-type integral of the reflective minus the absorbing product,            */
/*   3D: D_n = int_0^inf e^{-tau x^2} x^2 [C^ref_n(R',x) C^ref_n(R0,x) - C^abs_n(R',x) C^abs_n(R0,x)] dx, */
/*   2D: the same with x instead of x^2 and the integer-order functions of Eq. fRad.               */
/* 3D: J_{n+1/2}(z) = sqrt(2z/pi) j_n(z) (spherical Bessel), so the paper's F_{n+1/2}(R, x) equals  */
/* sqrt(2Rx/pi) C_n(R, x) with C_n = [j_n(Rx) b_n(x) - y_n(Rx) a_n(x)] / sqrt(a_n^2 + b_n^2),        */
/* a_n = h j_n(x) - x j_n'(x), b_n = h y_n(x) - x y_n'(x) (h = 0 reflective; h -> infinity         */
/* absorbing: a_n = j_n, b_n = y_n), the sqrt(R R0) cancelling the prefactor of Eq. genericGF3D.    */
/* The Bessel functions come from the three-term recurrences (Eq. 3termBessel): the second kind   */
/* upward, the first kind downward from far above (Miller) normalised by its sum rule; Legendre    */
/* polynomials by their recurrence.                                                                */
/* ------------------------------------------------------------------------------------------ */
#define ANG_NMAX 1200
#define ANG_MMAX 8000     /* start order of the downward recurrences at most (z up to ~7000) */
#define ANG_Y_BIG 1e280

/* j_n(z), y_n(z), n = 0..N (3D; spherical Bessel functions of the first and second kind).  y_n
 * upward: y_{n+1} = ((2n+1)/z) y_n - y_{n-1}, y_0 = -cos z / z, y_1 = -cos z / z^2 - sin z / z; once
 * |y_n| passes ANG_Y_BIG the rest is set to -ANG_Y_BIG (such orders contribute nothing at that z).
 * j_n downward from M = N + 40 + z: j_{n-1} = ((2n+1)/z) j_n - j_{n+1}, scaled by the sum rule
 * sum_n (2n+1) j_n^2 = 1 with the sign of j_0 = sin z / z (or of j_1 near its zeros). */
static void sph_bessel(int N, double z, double* j, double* y) {
  double s = sin(z), c = cos(z);
  y[0] = -c / z;
  if (N >= 1) y[1] = -c / (z * z) - s / z;
  for (int n = 1; n < N; ++n) {
    if (fabs(y[n]) > ANG_Y_BIG) {
      for (int m = n + 1; m <= N; ++m) y[m] = -ANG_Y_BIG;
      break;
    }
    y[n + 1] = (2.0 * n + 1.0) / z * y[n] - y[n - 1];
  }
  int M = N + 40 + (int)z;
  if (M > ANG_MMAX) M = ANG_MMAX;
  double jp1 = 0.0, jn = 1e-30, sum = 0.0;
  double tmp[ANG_MMAX + 2];
  for (int n = M; n >= 0; --n) {
    tmp[n] = jn;
    sum += (2.0 * n + 1.0) * jn * jn;
    double jm1 = n > 0 ? (2.0 * n + 1.0) / z * jn - jp1 : 0.0;
    jp1 = jn;
    jn = jm1;
    if (fabs(jn) > 1e100) {           /* rescale the running values (and the sum) to stay finite */
      for (int m = n; m <= M; ++m) tmp[m] *= 1e-100;
      jn *= 1e-100;
      jp1 *= 1e-100;
      sum *= 1e-200;
    }
  }
  double scale = 1.0 / sqrt(sum);
  double j0 = s / z, j1 = s / (z * z) - c / z;
  if (fabs(j0) >= fabs(j1)) {
    if ((j0 < 0.0) != (tmp[0] < 0.0)) scale = -scale;
  } else {
    if ((j1 < 0.0) != (tmp[1] < 0.0)) scale = -scale;
  }
  for (int n = 0; n <= N; ++n) j[n] = tmp[n] * scale;
}

/* J_n(z), Y_n(z), n = 0..N (2D; integer order).  Y_n upward from libm's y0, y1:
 * Y_{n+1} = (2n/z) Y_n - Y_{n-1}; J_n downward from M = N + 40 + z (Miller) normalised by
 * J_0 + 2 sum_{k>=1} J_{2k} = 1. */
static void cyl_bessel(int N, double z, double* J, double* Y) {
  Y[0] = y0(z);
  if (N >= 1) Y[1] = y1(z);
  for (int n = 1; n < N; ++n) {
    if (fabs(Y[n]) > ANG_Y_BIG) {
      for (int m = n + 1; m <= N; ++m) Y[m] = -ANG_Y_BIG;
      break;
    }
    Y[n + 1] = 2.0 * n / z * Y[n] - Y[n - 1];
  }
  int M = N + 40 + (int)z;
  if (M > ANG_MMAX) M = ANG_MMAX;
  if (M & 1) M--;
  double jp1 = 0.0, jn = 1e-30, norm = 0.0;
  double tmp[ANG_MMAX + 2];
  for (int n = M; n >= 0; --n) {
    tmp[n] = jn;
    norm += (n == 0 ? 1.0 : (n % 2 == 0 ? 2.0 : 0.0)) * jn;
    double jm1 = n > 0 ? 2.0 * n / z * jn - jp1 : 0.0;
    jp1 = jn;
    jn = jm1;
    if (fabs(jn) > 1e150) {
      for (int m = n; m <= M; ++m) tmp[m] *= 1e-150;
      jn *= 1e-150;
      jp1 *= 1e-150;
      norm *= 1e-150;
    }
  }
  for (int n = 0; n <= N; ++n) J[n] = tmp[n] / norm;
}

/* Boundary coefficients of order n at the abscissa x for the reflective (h = 0) and absorbing
 * conditions, normalised: C_n(R, x) = Z1(Rx) cb - Z2(Rx) ca, with (ca, cb) = (a, b) / sqrt(a^2 + b^2).
 * 3D: a = -x j_n'(x), b = -x y_n'(x) (ref); a = j_n(x), b = y_n(x) (abs).
 * 2D (Eq. fRad): a = x J_n'(x), b = x Y_n'(x) (ref); a = J_n(x), b = Y_n(x) (abs).
 * Derivatives: j_n' = j_{n-1} - (n+1)/z j_n (j_0' = -j_1); J_n' = J_{n-1} - n/z J_n (J_0' = -J_1). */
static void bc_coeffs(int dim, int n, double x, const double* jx, const double* yx, double* ca_ref,
                      double* cb_ref, double* ca_abs, double* cb_abs) {
  double jd, yd;
  if (dim == 3 && g_fault != 4) {
    jd = n == 0 ? -jx[1] : jx[n - 1] - (n + 1.0) / x * jx[n];
    yd = n == 0 ? -yx[1] : yx[n - 1] - (n + 1.0) / x * yx[n];
  } else {
    jd = n == 0 ? -jx[1] : jx[n - 1] - (double)n / x * jx[n];
    yd = n == 0 ? -yx[1] : yx[n - 1] - (double)n / x * yx[n];
  }
  double a = -x * jd, b = -x * yd;
  double nr = hypot(a, b);
  *ca_ref = a / nr;
  *cb_ref = b / nr;
  nr = hypot(jx[n], yx[n]);
  *ca_abs = jx[n] / nr;
  *cb_abs = yx[n] / nr;
}

/* D_n, n = 0..N, for end separation R and start separation R0 (both > 0, scaled units), on a
 * composite 16-point Gauss-Legendre rule over x in [0, X], X = sqrt(46/tau) (e^{-46} ~ 1e-20), with
 * `panels` equal panels.  which = 0: G_ref - G_abs (the encountered propagator); which = 1: the
 * absorbing, 2: the reflective, 3: the free function alone (C_n = j_n(Rx) / J_n(Rx)) -- the last
 * three for the pins. */
static void ang_D_grid(int dim, int which, int N, double R, double R0, double tau, int panels, double* D) {
  gl_init();
  for (int n = 0; n <= N; ++n) D[n] = 0.0;
  /* 3D: panels in x on [0, X]; 2D: in t with x = t^2 on [0, sqrt(X)] (dx = 2t dt), which smooths
   * the logarithmic behaviour of the integer-order boundary coefficients at x -> 0 */
  double X = sqrt(46.0 / tau), hp = (dim == 3 ? X : sqrt(X)) / panels;
  double *jx = (double*)malloc(sizeof(double) * (N + 2)), *yx = (double*)malloc(sizeof(double) * (N + 2));
  double *jr = (double*)malloc(sizeof(double) * (N + 2)), *yr = (double*)malloc(sizeof(double) * (N + 2));
  double *j0_ = (double*)malloc(sizeof(double) * (N + 2)), *y0_ = (double*)malloc(sizeof(double) * (N + 2));
  for (int p = 0; p < panels; ++p) {
    double m = (p + 0.5) * hp;
    for (int i = 0; i < GL_N; ++i) {
      double t = m + 0.5 * hp * gl_x[i];
      double x = dim == 3 ? t : t * t;
      double w = 0.5 * hp * gl_w[i] * exp(-tau * x * x) * (dim == 3 ? x * x : x * 2.0 * t);
      int Nb = N + 1;
      if (dim == 3) {
        sph_bessel(Nb, x, jx, yx);
        sph_bessel(N, R * x, jr, yr);
        sph_bessel(N, R0 * x, j0_, y0_);
      } else {
        cyl_bessel(Nb, x, jx, yx);
        cyl_bessel(N, R * x, jr, yr);
        cyl_bessel(N, R0 * x, j0_, y0_);
      }
      for (int n = 0; n <= N; ++n) {
        if (which == 3) {
          D[n] += w * jr[n] * j0_[n];
          continue;
        }
        if (yr[n] == -ANG_Y_BIG || y0_[n] == -ANG_Y_BIG || yx[n + 1] == -ANG_Y_BIG) continue;
        double car, cbr, caa, cba;
        bc_coeffs(dim, n, x, jx, yx, &car, &cbr, &caa, &cba);
        double ref = (jr[n] * cbr - yr[n] * car) * (j0_[n] * cbr - y0_[n] * car);
        double abs_ = (jr[n] * cba - yr[n] * caa) * (j0_[n] * cba - y0_[n] * caa);
        D[n] += w * (which == 0 ? ref - abs_ : (which == 1 ? abs_ : ref));
      }
    }
  }
  free(jx); free(yx); free(jr); free(yr); free(j0_); free(y0_);
}

/* Number of partial waves kept: the free part's coefficients decay like I_{n+d/2-1}(kappa) with
 * kappa = R R0 / (2 tau), negligible for n well beyond kappa. */
static int ang_terms(double R, double R0, double tau) {
  double kappa = R * R0 / (2.0 * tau);
  int N = (int)ceil(kappa + 8.0 * sqrt(kappa + 1.0) + 14.0);
  return N > ANG_NMAX ? ANG_NMAX : N;
}

/* D_n with the panel count doubled until the coefficients D_n / D_0 change by less than 1e-12
 * (at most 4096 panels); returns the number of terms N (D has N + 1 entries). */
int or_ang_coeffs(int dim, int which, double R, double R0, double tau, double* D, int cap) {
  int N = ang_terms(R, R0, tau);
  if (N + 1 > cap) N = cap - 1;
  double X = sqrt(46.0 / tau);
  int panels = 8 + (int)ceil(X * (R + R0) / 1.5);
  double* prev = (double*)malloc(sizeof(double) * (N + 1));
  ang_D_grid(dim, which, N, R, R0, tau, panels, D);
  for (int it = 0; it < 8 && panels < 4096; ++it) {
    memcpy(prev, D, sizeof(double) * (N + 1));
    panels *= 2;
    ang_D_grid(dim, which, N, R, R0, tau, panels, D);
    double scale = fabs(D[0]) > 0.0 ? fabs(D[0]) : 1.0, diff = 0.0;
    for (int n = 0; n <= N; ++n) diff = fmax(diff, fabs(D[n] - prev[n]));
    if (diff <= 1e-12 * scale) break;
  }
  free(prev);
  return N;
}

/* CDF of the conditional angle.  3D: F(mu) = (1 + mu)/2 + sum_{n>=1} (D_n/D_0) [P_{n+1}(mu) -
 * P_{n-1}(mu)] / 2 (from the integral of P_n: [P_{n+1} - P_{n-1}] / (2n+1)); 2D, for theta in
 * [0, pi]: F(theta) = [theta + 2 sum_{n>=1} (D_n/D_0) sin(n theta)/n] / pi. */
static double ang_cdf(int dim, const double* D, int N, double v) {
  if (dim == 3) {
    double pm1 = 1.0, p = v, sum = 0.5 * (1.0 + v);       /* P_0, P_1 */
    for (int n = 1; n <= N; ++n) {
      double pp1 = ((2.0 * n + 1.0) * v * p - n * pm1) / (n + 1.0);
      sum += 0.5 * D[n] / D[0] * (pp1 - pm1);
      pm1 = p;
      p = pp1;
    }
    return sum;
  }
  double sum = v;
  for (int n = 1; n <= N; ++n) sum += 2.0 * D[n] / D[0] * sin(n * v) / n;
  return sum / PI;
}

/* The angle of r' to r0 at CDF value U (bisection to the last bit): 3D cos(angle) in [-1, 1],
 * 2D the angle in [0, pi]. */
double or_ang_sample(int dim, double U, double R, double R0, double tau) {
  double D[ANG_NMAX + 1];
  int N = or_ang_coeffs(dim, 0, R, R0, tau, D, ANG_NMAX + 1);
  double lo = dim == 3 ? -1.0 : 0.0, hi = dim == 3 ? 1.0 : PI;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (ang_cdf(dim, D, N, mid) < U)
      lo = mid;
    else
      hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* The CDF of the conditional angle at v (3D: the cosine; 2D: the angle in [0, pi]), the function
 * or_ang_sample inverts. */
double or_ang_cdf(int dim, double v, double R, double R0, double tau) {
  double D[ANG_NMAX + 1];
  int N = or_ang_coeffs(dim, 0, R, R0, tau, D, ANG_NMAX + 1);
  return ang_cdf(dim, D, N, v);
}

/* The full Green's function at (R, v) from its partial waves (for the pins; which as in
 * or_ang_coeffs): 3D (1/4pi)(2/pi) sum_n (2n+1) P_n(mu) D_n with mu = v, 2D (1/2pi)
 * [D_0 + 2 sum_{n>=1} D_n cos(n v)] (a = 1). */
double or_gf_partial(int dim, int which, double v, double R, double R0, double tau) {
  double D[ANG_NMAX + 1];
  int N = or_ang_coeffs(dim, which, R, R0, tau, D, ANG_NMAX + 1);
  if (dim == 3) {
    double pm1 = 1.0, p = v, sum = D[0];
    for (int n = 1; n <= N; ++n) {
      sum += (2.0 * n + 1.0) * D[n] * p;
      double pp1 = ((2.0 * n + 1.0) * v * p - n * pm1) / (n + 1.0);
      pm1 = p;
      p = pp1;
    }
    return sum / (4.0 * PI) * (2.0 / PI);
  }
  double sum = D[0];
  for (int n = 1; n <= N; ++n) sum += 2.0 * D[n] * cos(n * v);
  return sum / (2.0 * PI);
}

/* The conditional density of the angle (for the pins): 3D f(mu), 2D f(theta) on [0, pi] (twice
 * the density on (-pi, pi]). */
double or_ang_density(int dim, double v, double R, double R0, double tau) {
  double D[ANG_NMAX + 1];
  int N = or_ang_coeffs(dim, 0, R, R0, tau, D, ANG_NMAX + 1);
  if (dim == 3) {
    double pm1 = 1.0, p = v, sum = 0.5;
    for (int n = 1; n <= N; ++n) {
      sum += 0.5 * (2.0 * n + 1.0) * D[n] / D[0] * p;
      double pp1 = ((2.0 * n + 1.0) * v * p - n * pm1) / (n + 1.0);
      pm1 = p;
      p = pp1;
    }
    return sum;
  }
  double sum = 1.0;
  for (int n = 1; n <= N; ++n) sum += 2.0 * D[n] / D[0] * cos(n * v);
  return sum / PI;
}

/* A unit vector e1 perpendicular to the unit vector u (3D): the coordinate axis along u's
 * smallest component (the first such axis on ties), made perpendicular and normalised; e2 = u x e1. */
static void perp_frame(const double* u, double* e1, double* e2) {
  int k = 0;
  if (fabs(u[1]) < fabs(u[k])) k = 1;
  if (fabs(u[2]) < fabs(u[k])) k = 2;
  double a[3] = {0, 0, 0};
  a[k] = 1.0;
  double d = u[k];
  double v[3] = {a[0] - d * u[0], a[1] - d * u[1], a[2] - d * u[2]};
  double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  for (int i = 0; i < 3; ++i) e1[i] = v[i] / nv;
  e2[0] = u[1] * e1[2] - u[2] * e1[1];
  e2[1] = u[2] * e1[0] - u[0] * e1[2];
  e2[2] = u[0] * e1[1] - u[1] * e1[0];
}

/* Unit direction of the new separation: angle from or_ang_sample at U_ang about the axis u (the
 * start separation's direction), azimuth (3D) 2 pi U_azi, sign of the angle (2D) U_azi < 1/2.
 * The step evaluates the series only while at most ANG_NSTEP partial waves are needed (kappa =
 * R' R0 / 2 tau up to ~40); otherwise it returns 0 and the caller keeps the free step's direction. */
#define ANG_NSTEP 127
static int ang_direction(int dim, const double* u, double U_ang, double U_azi, double Rn, double R0, double tau,
                         double* dir) {
  if (ang_terms(Rn, R0, tau) > ANG_NSTEP) return 0;
  if (dim == 3) {
    double mu = or_ang_sample(3, U_ang, Rn, R0, tau);
    double st = sqrt(fmax(0.0, 1.0 - mu * mu)), ph = 2.0 * PI * U_azi;
    double e1[3], e2[3];
    perp_frame(u, e1, e2);
    double c = cos(ph), s = sin(ph);
    for (int i = 0; i < 3; ++i) dir[i] = mu * u[i] + st * (c * e1[i] + s * e2[i]);
  } else {
    double th = or_ang_sample(2, U_ang, Rn, R0, tau);
    if (U_azi < 0.5) th = -th;
    double c = cos(th), s = sin(th);
    dir[0] = c * u[0] - s * u[1];
    dir[1] = s * u[0] + c * u[1];
    dir[2] = 0.0;
  }
  return 1;
}

/* The whole propagation of one encountered pair (for the tests): start separation vector r0
 * (scaled by a), new length from the radial law at tail fraction u_res, direction from
 * ang_direction at (u_ang, u_azi); out = the new separation vector (scaled). */
void or_propagate(int dim, const double* r0, double tau, double tau_s, double u_res, double u_ang, double u_azi,
                  double* out) {
  double l0 = sqrt(r0[0] * r0[0] + r0[1] * r0[1] + (dim == 3 ? r0[2] * r0[2] : 0.0));
  double R0 = l0 < 1.0 ? 1.0 : l0;
  double Rn = dim == 3 ? or_resample3(u_res, R0, tau) : or_resample2(u_res, R0, tau, tau_s);
  double u[3] = {1.0, 0.0, 0.0}, dir[3];
  if (l0 > 0.0)
    for (int d = 0; d < dim; ++d) u[d] = r0[d] / l0;
  if (!ang_direction(dim, u, u_ang, u_azi, Rn, R0, tau, dir))
    for (int d = 0; d < 3; ++d) dir[d] = u[d];
  for (int d = 0; d < 3; ++d) out[d] = d < dim ? Rn * dir[d] : 0.0;
}

/* ------------------------------------------------------------------------------------------ */
/* Geometry in the periodic box.                                                                  */
/* ------------------------------------------------------------------------------------------ */
static double min_image(double d, double L) {
  if (d > 0.5 * L)
    d -= L;
  else if (d < -0.5 * L)
    d += L;
  return d;
}

static double wrap(double x, double L) {
  if (x >= L) {
    x -= L;
  } else if (x < 0.0) {
    x += L;
    if (x >= L) x = 0.0;
  }
  return x;
}

/* Squared length summed left to right (the build disables floating-point contraction). */
static double norm2(const double* v, int dim) {
  double s = v[0] * v[0];
  s = s + v[1] * v[1];
  if (dim == 3) s = s + v[2] * v[2];
  return s;
}

/* ------------------------------------------------------------------------------------------ */
/* Per-pair-type parameters.                                                                      */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  int rule;        /* index into sys->pairs, -1: no interaction */
  double sigma, Drel, tau, h, rcut2;
} pair_param;

static void pair_params(const or_system* sys, pair_param table[OR_MAX_SPECIES][OR_MAX_SPECIES]) {
  for (int a = 0; a < OR_MAX_SPECIES; ++a)
    for (int b = 0; b < OR_MAX_SPECIES; ++b) table[a][b].rule = -1;
  for (int k = 0; k < sys->n_pairs; ++k) {
    const or_pair* p = &sys->pairs[k];
    if (p->bc == OR_BC_NONE) continue;
    pair_param pp;
    pp.rule = k;
    pp.sigma = p->sigma;
    pp.Drel = sys->D[p->s1] + sys->D[p->s2];                 /* D_eff = D_A + D_B (Section 2.1) */
    pp.tau = pp.Drel * sys->dt / (p->sigma * p->sigma);
    if (sys->dim == 3)
      pp.h = p->ka / (4.0 * PI * p->sigma * pp.Drel);       /* h~3D = kappa_a / (4 pi a D) */
    else
      pp.h = p->ka / (2.0 * PI * pp.Drel);                  /* h~2D = kappa_a / (2 pi D) */
    double rc = p->sigma + sys->c_cut * sqrt(2.0 * pp.Drel * sys->dt);
    pp.rcut2 = rc * rc;
    table[p->s1][p->s2] = pp;
    table[p->s2][p->s1] = pp;
  }
}

static double p_enc_dim(const or_system* sys, double R, double R0, double tau) {
  return sys->dim == 3 ? or_p_enc3(R, R0, tau) : or_p_enc2(R, R0, tau, sys->tau_s);
}
static double p_reac_dim(const or_system* sys, double R, double R0, double tau, double h) {
  return sys->dim == 3 ? or_p_reac3(R, R0, tau, h) : or_p_reac2(R, R0, tau, h, sys->tau_s);
}
static double resample_dim(const or_system* sys, double U, double R0, double tau) {
  return sys->dim == 3 ? or_resample3(U, R0, tau) : or_resample2(U, R0, tau, sys->tau_s);
}

/* ------------------------------------------------------------------------------------------ */
/* Initial condition: uniform positions from the INIT streams, species in blocks of n_init.       */
/* ------------------------------------------------------------------------------------------ */
int or_init_positions(const or_system* sys, const int64_t* n_init, or_state* st) {
  int64_t n = 0;
  for (int s = 0; s < sys->n_species; ++s) n += n_init[s];
  if (n > st->cap) return -1;
  int64_t i = 0;
  for (int s = 0; s < sys->n_species; ++s) {
    for (int64_t k = 0; k < n_init[s]; ++k, ++i) {
      uint32_t w[4];
      stream(sys, 0u, (uint32_t)i, 0xFFFFFFFFu, OR_TAG_INIT0, w);
      double x = or_u52(w[0], w[1]) * sys->L, y = or_u52(w[2], w[3]) * sys->L, z = 0.0;
      if (sys->dim == 3) {
        stream(sys, 0u, (uint32_t)i, 0xFFFFFFFFu, OR_TAG_INIT1, w);
        z = or_u52(w[0], w[1]) * sys->L;
      }
      st->x[3 * i + 0] = x < sys->L ? x : 0.0;
      st->x[3 * i + 1] = y < sys->L ? y : 0.0;
      st->x[3 * i + 2] = z < sys->L ? z : 0.0;
      st->sp[i] = s;
      st->id[i] = (uint32_t)i;
    }
  }
  st->n = n;
  st->step = 0;
  st->next_id = (uint32_t)n;
  st->t = 0.0;
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* One step (Section 3, steps 1-5).                                                               */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  int64_t a, b;   /* particle indices, id[a] < id[b] */
  uint32_t ida, idb;
  double p, key;
  int rule;
  int64_t tidx;   /* trace entry or -1 */
} fired_pair;

/* total order (key, id_a, id_b) */
static int cmp_fired(const void* x, const void* y) {
  const fired_pair* e = (const fired_pair*)x;
  const fired_pair* f = (const fired_pair*)y;
  if (e->key != f->key) return e->key < f->key ? -1 : 1;
  if (e->ida != f->ida) return e->ida < f->ida ? -1 : 1;
  if (e->idb != f->idb) return e->idb < f->idb ? -1 : 1;
  return 0;
}


static int cmp_fired_faulty(const void* x, const void* y) {
  return g_fault == 2 ? -cmp_fired(x, y) : cmp_fired(x, y);
}

typedef struct {
  int n;             /* number of products (0..2) */
  int species[2];
  double x[2][3];
} products_t;

/* Steps 2-3 for the pair (i, j): returns -1 if it is not a candidate (decayed, non-interacting or
 * beyond the cut-off), 0 if it is a candidate that did not fire, 1 if it fired (*f filled).
 * Counts candidates, overlaps and near-threshold draws; appends the candidate to the trace. */
static int test_pair(const or_system* sys, const or_state* in, const pair_param pp[OR_MAX_SPECIES][OR_MAX_SPECIES],
                     const double* xstart, const double* x1, const int* decayed, uint32_t step, int64_t i,
                     int64_t j, fired_pair* f, int64_t* cand, int64_t* ovl, int64_t* near, or_trace* trace) {
  const int dim = sys->dim;
  const double L = sys->L;
  if (decayed[j]) return -1;
  const pair_param* q = &pp[in->sp[i]][in->sp[j]];
  if (q->rule < 0) return -1;
  int64_t a = in->id[i] < in->id[j] ? i : j;
  int64_t b = a == i ? j : i;
  double r0v[3] = {0, 0, 0}, rv[3] = {0, 0, 0};
  for (int d = 0; d < dim; ++d) {
    r0v[d] = min_image(xstart[3 * b + d] - xstart[3 * a + d], L);
    rv[d] = min_image(x1[3 * b + d] - x1[3 * a + d], L);
  }
  double r02 = norm2(r0v, dim);
  if (!(r02 < q->rcut2)) return -1;
  double R0 = sqrt(r02) / q->sigma;
  double R = sqrt(norm2(rv, dim)) / q->sigma;
  double p = p_enc_dim(sys, R, R0, q->tau);
  uint32_t w[4];
  stream(sys, step, in->id[a], in->id[b], OR_TAG_ENC, w);
  double u_enc = or_u52(w[0], w[1]), u_sel = or_u52(w[2], w[3]);
  int fires = u_enc < p;
  (*cand)++;
  if (R <= 1.0) (*ovl)++;
  if (fabs(u_enc - p) <= NEAR_THRESHOLD) (*near)++;
  int64_t tidx = -1;
  if (trace && trace->n < trace->cap) {
    tidx = trace->n;
    trace->ida[trace->n] = in->id[a];
    trace->idb[trace->n] = in->id[b];
    trace->p_enc[trace->n] = p;
    trace->u_enc[trace->n] = u_enc;
    trace->fired[trace->n] = fires;
    trace->matched[trace->n] = 0;
    trace->n++;
  }
  if (!fires) return 0;
  f->a = a;
  f->b = b;
  f->ida = in->id[a];
  f->idb = in->id[b];
  f->tidx = tidx;
  f->p = p;
  f->key = g_fault == 1 ? -log(u_sel) * p : (g_fault == 3 ? -log(u_enc) / p : -log(u_sel) / p);
  f->rule = q->rule;
  return 1;
}

int or_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int or_step(const or_system* sys, const or_state* in, or_state* out, or_stats* stats,
            or_trace* trace) {
  const int dim = sys->dim;
  const double L = sys->L, dt = sys->dt;
  const int64_t n = in->n;
  const uint32_t step = in->step;
  pair_param pp[OR_MAX_SPECIES][OR_MAX_SPECIES];
  pair_params(sys, pp);
  or_stats st;
  memset(&st, 0, sizeof st);
  if (trace) trace->n = 0;

  double* x1 = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  int* decayed = (int*)calloc((size_t)(n > 0 ? n : 1), sizeof(int));     /* 0, or channel+1 */
  int* consumed = (int*)calloc((size_t)(n > 0 ? n : 1), sizeof(int));
  int64_t* partner = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  products_t* prod = (products_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(products_t));
  for (int64_t i = 0; i < n; ++i) partner[i] = -1;

  /* Deterministic forces as a split step (Section 3 keeps them outside the Green's-function part):
   * every particle first moves by its species' drift displacement v dt (periodic wrap).  The
   * reaction-diffusion step below starts from these positions, so p_enc and p_reac see only the
   * Brownian end points. */
  double* xs = NULL;
  const double* xstart = in->x;
  if (sys->has_drift) {
    xs = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i)
      for (int d = 0; d < 3; ++d) {
        double v = in->x[3 * i + d];
        if (d < dim) v = wrap(v + sys->drift_dx[in->sp[i]][d], L);
        xs[3 * i + d] = v;
      }
    xstart = xs;
  }

  /* Step 4 of Section 3, drawn first (start-of-step state): Poisson decay with probability
   * 1 - exp(-k_d dt), Eq. (rad_prob); with several channels the total rate decides and a second
   * uniform picks the channel in proportion to its rate. */
  for (int64_t i = 0; i < n; ++i) {
    double ktot = 0.0;
    for (int c = 0; c < sys->n_decays; ++c)
      if (sys->decays[c].parent == in->sp[i]) ktot += sys->decays[c].kd;
    if (ktot <= 0.0) continue;
    uint32_t w[4];
    stream(sys, step, in->id[i], 0xFFFFFFFFu, OR_TAG_UNI, w);
    double u = or_u52(w[0], w[1]);
    double p_uni = -expm1(-ktot * dt);
    if (fabs(u - p_uni) <= NEAR_THRESHOLD) st.near_threshold++;
    if (!(u < p_uni)) continue;
    double target = or_u52(w[2], w[3]) * ktot, acc = 0.0;
    int chosen = -1, last = -1;
    for (int c = 0; c < sys->n_decays; ++c) {
      if (sys->decays[c].parent != in->sp[i]) continue;
      last = c;
      acc += sys->decays[c].kd;
      if (chosen < 0 && target < acc) chosen = c;
    }
    if (chosen < 0) chosen = last;
    decayed[i] = chosen + 1;
  }

  /* Step 1: free displacement sqrt(2 D dt) N(0,1) of every particle that did not decay. */
  for (int64_t i = 0; i < n; ++i) {
    double nrm[4] = {0, 0, 0, 0};
    if (!decayed[i]) normals(sys, step, in->id[i], OR_TAG_DISP0, dim, nrm);
    double ell = sqrt(2.0 * sys->D[in->sp[i]] * dt);
    for (int d = 0; d < 3; ++d) {
      double v = xstart[3 * i + d];
      if (d < dim && !decayed[i]) v = wrap(v + ell * nrm[d], L);
      x1[3 * i + d] = v;
    }
  }

  /* Steps 2-3: every interacting pair within the cut-off (start-of-step minimum image distance)
   * is tested with p_enc (overlap forces p_enc = 1) and a uniform draw. */
  int64_t fcap = 1024, fn = 0;
  fired_pair* fired = (fired_pair*)malloc(sizeof(fired_pair) * (size_t)fcap);
#ifdef _OPENMP
  /* The all-core CPU baseline build: rows of the pair loop on all threads, each with its own list;
   * the greedy matching sorts the fired pairs by (key, id_a, id_b), so the lists' order does not
   * matter and the result equals the serial loop's.  The per-candidate trace stays serial. */
  if (!trace) {
    int64_t cand = 0, ovl = 0, near = 0;
#pragma omp parallel reduction(+ : cand, ovl, near)
    {
      int64_t lcap = 256, ln = 0;
      fired_pair* loc = (fired_pair*)malloc(sizeof(fired_pair) * (size_t)lcap);
#pragma omp for schedule(dynamic, 16)
      for (int64_t i = 0; i < n; ++i) {
        if (decayed[i]) continue;
        for (int64_t j = i + 1; j < n; ++j) {
          fired_pair f;
          int rc = test_pair(sys, in, pp, xstart, x1, decayed, step, i, j, &f, &cand, &ovl, &near, NULL);
          if (rc <= 0) continue;
          if (ln == lcap) {
            lcap *= 2;
            loc = (fired_pair*)realloc(loc, sizeof(fired_pair) * (size_t)lcap);
          }
          loc[ln++] = f;
        }
      }
#pragma omp critical
      {
        while (fn + ln > fcap) fcap *= 2;
        fired = (fired_pair*)realloc(fired, sizeof(fired_pair) * (size_t)fcap);
        memcpy(fired + fn, loc, sizeof(fired_pair) * (size_t)ln);
        fn += ln;
      }
      free(loc);
    }
    st.candidates += cand;
    st.overlaps += ovl;
    st.near_threshold += near;
  } else
#endif
  {
    for (int64_t i = 0; i < n; ++i) {
      if (decayed[i]) continue;
      for (int64_t j = i + 1; j < n; ++j) {
        fired_pair f;
        int rc = test_pair(sys, in, pp, xstart, x1, decayed, step, i, j, &f, &st.candidates, &st.overlaps,
                           &st.near_threshold, trace);
        if (rc <= 0) continue;
        if (fn == fcap) {
          fcap *= 2;
          fired = (fired_pair*)realloc(fired, sizeof(fired_pair) * (size_t)fcap);
        }
        fired[fn++] = f;
      }
    }
  }
  st.fired = fn;

  /* Conflict resolution (Section 3, "Details"): greedy in ascending (key, id_a, id_b). */
  if (fn > 1) qsort(fired, (size_t)fn, sizeof(fired_pair), cmp_fired_faulty);
  for (int64_t e = 0; e < fn; ++e) {
    if (partner[fired[e].a] >= 0 || partner[fired[e].b] >= 0) continue;
    partner[fired[e].a] = fired[e].b;
    partner[fired[e].b] = fired[e].a;
    st.matched++;
    if (trace && fired[e].tidx >= 0) trace->matched[fired[e].tidx] = 1;
  }

  /* Steps 2(a)-(c) for each matched pair, all from their own free end points. */
  for (int64_t e = 0; e < fn; ++e) {
    int64_t a = fired[e].a, b = fired[e].b;
    if (partner[a] != b) continue;
    const or_pair* rule = &sys->pairs[fired[e].rule];
    const pair_param* q = &pp[in->sp[a]][in->sp[b]];
    double Da = sys->D[in->sp[a]], Db = sys->D[in->sp[b]];
    double wa = Da / q->Drel, wb = Db / q->Drel;
    double rv[3] = {0, 0, 0}, r0v[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) {
      rv[d] = min_image(x1[3 * b + d] - x1[3 * a + d], L);
      r0v[d] = min_image(xstart[3 * b + d] - xstart[3 * a + d], L);
    }
    /* centre of diffusion, Eq. (Rcoo): R = (D_B r_A + D_A r_B)/D_eff = r_A + (D_A/D_eff) r */
    double c[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) c[d] = x1[3 * a + d] + wa * rv[d];
    int react = 0;
    if (rule->bc == OR_BC_ABS) {
      react = 1;                                                   /* step 2(a) */
    } else {
      /* steps 2(b)-(c): new separation length from the radial propagator g_ref - g_abs, kept
       * along the free-step direction; centre of diffusion unchanged. */
      uint32_t w[4];
      stream(sys, step, in->id[a], in->id[b], OR_TAG_RES, w);
      double u_res = or_u52(w[0], w[1]), u_reac = or_u52(w[2], w[3]);
      double R0 = sqrt(norm2(r0v, dim)) / q->sigma;
      if (R0 < 1.0) R0 = 1.0;
      double Rn = resample_dim(sys, u_res, R0, q->tau);
      double dir[3] = {0, 0, 0};
      int exact = 0;
      if (sys->angle_mode == 0) {
        /* the direction from the full propagator: its angle to r0 from the partial-wave law
         * given R', uniform azimuth (start separation zero: the x axis) */
        double l0 = sqrt(norm2(r0v, dim)), u[3] = {1.0, 0.0, 0.0};
        if (l0 > 0.0)
          for (int d = 0; d < dim; ++d) u[d] = r0v[d] / l0;
        uint32_t wa[4];
        stream(sys, step, in->id[a], in->id[b], OR_TAG_ANG, wa);
        exact = ang_direction(dim, u, or_u52(wa[0], wa[1]), or_u52(wa[2], wa[3]), Rn, R0, q->tau, dir);
      }
      if (!exact) {
        double len = sqrt(norm2(rv, dim));
        if (len > 0.0) {
          for (int d = 0; d < dim; ++d) dir[d] = rv[d] / len;
        } else {
          double l0 = sqrt(norm2(r0v, dim));
          if (l0 > 0.0)
            for (int d = 0; d < dim; ++d) dir[d] = r0v[d] / l0;
          else
            dir[0] = 1.0;
        }
      }
      for (int d = 0; d < dim; ++d) {
        double nr = Rn * q->sigma * dir[d];
        x1[3 * a + d] = wrap(c[d] - wa * nr, L);
        x1[3 * b + d] = wrap(c[d] + wb * nr, L);
      }
      st.resampled++;
      if (rule->bc == OR_BC_RAD) {
        double p = p_reac_dim(sys, Rn, R0, q->tau, q->h);
        if (fabs(u_reac - p) <= NEAR_THRESHOLD) st.near_threshold++;
        react = u_reac < p;
      }
    }
    if (react) {
      consumed[a] = consumed[b] = 1;
      st.reactions++;
      if (rule->product >= 0) {
        prod[a].n = 1;
        prod[a].species[0] = rule->product;
        for (int d = 0; d < 3; ++d) prod[a].x[0][d] = d < dim ? wrap(c[d], L) : 0.0;
      }
    }
  }

  /* Unimolecular products (Section 2.2.5). */
  for (int64_t i = 0; i < n; ++i) {
    if (!decayed[i]) continue;
    const or_decay* dc = &sys->decays[decayed[i] - 1];
    consumed[i] = 1;
    st.decays++;
    const double* x0 = &xstart[3 * i];
    if (dc->n_products == 1) {
      double nrm[4] = {0, 0, 0, 0};
      normals(sys, step, in->id[i], OR_TAG_DISS0, dim, nrm);
      double ell = sqrt(2.0 * sys->D[dc->p0] * dt);
      prod[i].n = 1;
      prod[i].species[0] = dc->p0;
      for (int d = 0; d < 3; ++d) prod[i].x[0][d] = d < dim ? wrap(x0[d] + ell * nrm[d], L) : 0.0;
    } else if (dc->n_products == 2) {
      int sa = dc->p0, sb = dc->p1;
      const pair_param* q = &pp[sa][sb];
      double Drel = sys->D[sa] + sys->D[sb];
      double wa = sys->D[sa] / Drel, wb = sys->D[sb] / Drel;
      double DR = sys->D[sa] * sys->D[sb] / Drel;                 /* D_R, Section 2.1 */
      /* direction of the contact separation, uniform on the sphere / circle */
      uint32_t w[4];
      stream(sys, step, in->id[i], 0xFFFFFFFFu, OR_TAG_DIR, w);
      double dir[3] = {0, 0, 0};
      if (dim == 3) {
        double ct = 2.0 * or_u52(w[0], w[1]) - 1.0, ph = 2.0 * PI * or_u52(w[2], w[3]);
        double st_ = sqrt(fmax(0.0, 1.0 - ct * ct));
        dir[0] = st_ * cos(ph); dir[1] = st_ * sin(ph); dir[2] = ct;
      } else {
        double ph = 2.0 * PI * or_u52(w[0], w[1]);
        dir[0] = cos(ph); dir[1] = sin(ph);
      }
      /* centre of diffusion moves freely with D_R over dt */
      double nc[4] = {0, 0, 0, 0};
      normals(sys, step, in->id[i], OR_TAG_DISS0, dim, nc);
      double ellc = sqrt(2.0 * DR * dt);
      double c[3] = {0, 0, 0}, rv[3] = {0, 0, 0};
      for (int d = 0; d < dim; ++d) c[d] = x0[d] + ellc * nc[d];
      int recombine = 0;
      int product = -1;
      if (q->rule >= 0) {
        /* the pair starts at contact, |r0| = a: propagate by g_ref - g_abs with R0 = 1, then
         * Eq. (psurv_radII) decides escape or recombination (Section 2.2.5) */
        const or_pair* rule = &sys->pairs[q->rule];
        stream(sys, step, in->id[i], 0xFFFFFFFFu, OR_TAG_RES, w);
        double u_res = or_u52(w[0], w[1]), u_reac = or_u52(w[2], w[3]);
        double Rn = resample_dim(sys, u_res, 1.0, q->tau);
        if (sys->angle_mode == 0) {
          /* from contact along dir: the new direction from the full propagator about dir */
          double u[3] = {dir[0], dir[1], dir[2]}, nd[3];
          uint32_t wa[4];
          stream(sys, step, in->id[i], 0xFFFFFFFFu, OR_TAG_ANG, wa);
          if (ang_direction(dim, u, or_u52(wa[0], wa[1]), or_u52(wa[2], wa[3]), Rn, 1.0, q->tau, nd))
            for (int d = 0; d < 3; ++d) dir[d] = nd[d];
        }
        for (int d = 0; d < dim; ++d) rv[d] = Rn * q->sigma * dir[d];
        if (rule->bc == OR_BC_ABS) {
          recombine = 1;
        } else if (rule->bc == OR_BC_RAD) {
          double p = p_reac_dim(sys, Rn, 1.0, q->tau, q->h);
          if (fabs(u_reac - p) <= NEAR_THRESHOLD) st.near_threshold++;
          recombine = u_reac < p;
        }
        product = rule->product;
      } else {
        /* non-interacting products: start sigma_place apart, relative vector diffuses freely */
        double nr[4] = {0, 0, 0, 0};
        normals(sys, step, in->id[i], OR_TAG_DISS2, dim, nr);
        double ellr = sqrt(2.0 * Drel * dt);
        for (int d = 0; d < dim; ++d) rv[d] = dc->sigma_place * dir[d] + ellr * nr[d];
      }
      if (recombine) {
        st.recombined++;
        if (product >= 0) {
          prod[i].n = 1;
          prod[i].species[0] = product;
          for (int d = 0; d < 3; ++d) prod[i].x[0][d] = d < dim ? wrap(c[d], L) : 0.0;
        }
      } else {
        prod[i].n = 2;
        prod[i].species[0] = sa;
        prod[i].species[1] = sb;
        for (int d = 0; d < 3; ++d) {
          prod[i].x[0][d] = d < dim ? wrap(c[d] - wa * rv[d], L) : 0.0;
          prod[i].x[1][d] = d < dim ? wrap(c[d] + wb * rv[d], L) : 0.0;
        }
      }
    }
  }

  /* New state: survivors in their order, then products in event order (owner = lower parent id,
   * and the input is id-sorted, so array order is event order). */
  int64_t nsurv = 0, nprod = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (!consumed[i]) nsurv++;
    nprod += prod[i].n;
  }
  int status = 0;
  if (nsurv + nprod > out->cap) {
    status = -2;
  } else {
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
      if (consumed[i]) continue;
      for (int d = 0; d < 3; ++d) out->x[3 * k + d] = x1[3 * i + d];
      out->sp[k] = in->sp[i];
      out->id[k] = in->id[i];
      k++;
    }
    uint32_t next_id = in->next_id;
    for (int64_t i = 0; i < n; ++i) {
      for (int m = 0; m < prod[i].n; ++m) {
        for (int d = 0; d < 3; ++d) out->x[3 * k + d] = prod[i].x[m][d];
        out->sp[k] = prod[i].species[m];
        out->id[k] = next_id++;
        k++;
      }
    }
    out->n = k;
    out->next_id = next_id;
    out->step = step + 1;
    out->t = in->t + dt;
  }
  st.products = nprod;
  if (stats) *stats = st;
  free(x1); free(decayed); free(consumed); free(partner); free(prod); free(fired); free(xs);
  return status;
}

/* ------------------------------------------------------------------------------------------ */
/* First-passage refinement (Appendix, "Relation to first-passage time simulation algorithms"): */
/* a pair that went from separation R0 to R in a step of length tau (scaled units) and          */
/* encountered the contact surface on the way.  The step is halved `levels` times; at every      */
/* level the separation at the midpoint of the current interval is drawn from the bridge of the  */
/* radial process between the interval's end separations, and the half that holds the first     */
/* contact is chosen with p_enc of the two halves.  The encounter is known for the whole         */
/* interval, so the midpoint and the two halves' encounter decisions are redrawn until at least  */
/* one half has an encounter; the first contact then lies in the first half if that one has an  */
/* encounter, else in the second.                                                                */
/*                                                                                                */
/* Radial bridge midpoint (the paper states the 1D Gaussian law, Eq. midPGauss, mean half the    */
/* displacement, variance half of that of one half-interval step, and leaves the higher-         */
/* dimensional form to the reader): the end point's direction relative to the start is drawn    */
/* from the free Gaussian restricted to the sphere |r| = R_f, a von Mises-Fisher law with         */
/* concentration kappa = R_i R_f / (2 t) (3D: cos(theta) by inversion of its CDF; 2D: the von     */
/* Mises law by the rejection method of Best and Fisher, Appl. Stat. 28 (1979) 152); the         */
/* midpoint vector is then (r_i + r_f)/2 plus a Gaussian of variance t/2 per component, and its  */
/* length is the bridge midpoint of the radial process.  The azimuth of r_f about r_i and the    */
/* sign of the 2D angle do not change the law of |m| (the Gaussian is isotropic) and are fixed.  */
/*                                                                                                */
/* Random numbers: Philox4x32-10 with key (seed lo, seed hi) and counter (stream lo, stream hi,  */
/* a, OR_TAG_FPT | w << 8), a = the pair's attempt number counted over all levels, w = word:     */
/*   w = 0: U_dir (3D direction), U_e1 (encounter in the first half)                             */
/*   w = 1: two normals (Box-Muller);  w = 2: a third normal (3D)                                */
/*   w = 3: U_e2 (encounter in the second half)                                                  */
/*   w = 4 + j: the j-th von Mises trial (2D), j < 64                                            */
/* ------------------------------------------------------------------------------------------ */
#define OR_TAG_FPT 13
#define OR_VM_TRIALS 64

static void fpt_draw(uint64_t seed, uint64_t strm, uint32_t a, uint32_t w, double* u0, double* u1) {
  uint32_t ctr[4] = {(uint32_t)(strm & 0xFFFFFFFFu), (uint32_t)(strm >> 32), a, OR_TAG_FPT | (w << 8)};
  uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
  uint32_t o[4];
  or_philox4x32_10(ctr, key, o);
  *u0 = or_u52(o[0], o[1]);
  *u1 = or_u52(o[2], o[3]);
}

/* 3D: 1 - cos(theta) for a von Mises-Fisher direction with concentration kappa, from the CDF   */
/* F(w) = (e^{kappa w} - e^{-kappa}) / (e^{kappa} - e^{-kappa}) inverted at 1 - u:               */
/* 1 - w = -log(u + (1 - u) e^{-2 kappa}) / kappa, evaluated as written for u <= 1/2 and as       */
/* -log1p((1 - u) expm1(-2 kappa)) / kappa above (no cancellation in either range).               */
static double vmf3_one_minus_cos(double kappa, double u) {
  if (u <= 0.5) return -log(u + (1.0 - u) * exp(-2.0 * kappa)) / kappa;
  return -log1p((1.0 - u) * expm1(-2.0 * kappa)) / kappa;
}

/* 2D: von Mises angle with concentration kappa (Best & Fisher 1979), returned as (1 - cos, sin).*/
/* rho = 2 kappa / (t + sqrt(2 t)) with t = 1 + sqrt(1 + 4 kappa^2) and r = (1 + rho^2)/(2 rho); */
/* a trial takes z = cos(pi u1), f = (1 + r z)/(r + z), c = kappa (r - f) and accepts when        */
/* c (2 - c) > u2 or log(c / u2) + 1 - c >= 0; cos(theta) = f.  The differences r - f and 1 - f   */
/* are formed without cancellation: r - f = (r^2 - 1)/(r + z), 1 - f = (r - 1)(1 - z)/(r + z).  */
/* Returns 0 when all trials were rejected.                                                      */
static int vm2_draw(double kappa, uint64_t seed, uint64_t strm, uint32_t a, double* omc, double* sn) {
  const double s4 = sqrt(1.0 + 4.0 * kappa * kappa), t = 1.0 + s4;
  const double rho = 2.0 * kappa / (t + sqrt(2.0 * t));
  const double one_m_rho = (1.0 + 1.0 / (s4 + 2.0 * kappa) + sqrt(2.0 * t)) / (t + sqrt(2.0 * t));
  const double r = (1.0 + rho * rho) / (2.0 * rho);
  const double r_m1 = one_m_rho * one_m_rho / (2.0 * rho);
  const double r2_m1 = (one_m_rho * (1.0 + rho)) * (one_m_rho * (1.0 + rho)) / (4.0 * rho * rho);
  for (uint32_t j = 0; j < OR_VM_TRIALS; ++j) {
    double u1, u2;
    fpt_draw(seed, strm, a, 4 + j, &u1, &u2);
    const double sh = sin(0.5 * PI * u1), ch = cos(0.5 * PI * u1);
    const double one_m_z = 2.0 * sh * sh, one_p_z = 2.0 * ch * ch;
    const double r_p_z = r_m1 + one_p_z;            /* r + z */
    const double c = kappa * r2_m1 / r_p_z;         /* kappa (r - f) */
    if (c * (2.0 - c) > u2 || log(c / u2) + 1.0 - c >= 0.0) {
      const double omf = r_m1 * one_m_z / r_p_z;   /* 1 - f */
      const double opf = (r + 1.0) * one_p_z / r_p_z;
      *omc = omf;
      *sn = sqrt(omf * opf);
      return 1;
    }
  }
  return 0;
}

/* The direction draw alone (for the tests of the two samplers): 1 - cos(theta) and sin(theta)
 * of the end point relative to the start for concentration kappa, attempt a. */
int or_fpt_direction(int dim, double kappa, uint64_t seed, uint64_t strm, uint32_t a, double* omc,
                     double* sn) {
  if (dim == 3) {
    double u_dir, u_e1;
    fpt_draw(seed, strm, a, 0, &u_dir, &u_e1);
    *omc = vmf3_one_minus_cos(kappa, u_dir);
    *sn = sqrt(*omc * (2.0 - *omc));
    return 1;
  }
  return vm2_draw(kappa, seed, strm, a, omc, sn);
}

static double fpt_p_enc(int dim, double R, double R0, double tau, double tau_s) {
  return dim == 3 ? or_p_enc3(R, R0, tau) : or_p_enc2(R, R0, tau, tau_s);
}

int or_fpt_refine(int dim, double R0, double R, double tau, double tau_s, int levels, uint64_t seed,
                  uint64_t strm, uint32_t max_attempts, uint32_t* bin, double* R_lo, double* R_hi,
                  uint32_t* attempts, double* margin) {
  double Ri = R0, Rf = R, t = tau, mg = INFINITY;
  uint32_t b = 0, a = 0;
  int status = 0;
  for (int k = 0; k < levels && status == 0; ++k) {
    for (;;) {
      if (a >= max_attempts) { status = 1; break; }
      double u_dir, u_e1, u_e2, unused, xi[4];
      fpt_draw(seed, strm, a, 0, &u_dir, &u_e1);
      {
        double v0, v1;
        fpt_draw(seed, strm, a, 1, &v0, &v1);
        box_muller(v0, v1, &xi[0], &xi[1]);
        xi[2] = 0.0;
        if (dim == 3) {
          fpt_draw(seed, strm, a, 2, &v0, &v1);
          box_muller(v0, v1, &xi[2], &xi[3]);
        }
      }
      fpt_draw(seed, strm, a, 3, &u_e2, &unused);
      /* end point in the frame of the start point r_i = (R_i, 0, 0) */
      const double kappa = Ri * Rf / (2.0 * t);
      double omc, sn;
      if (dim == 3) {
        omc = vmf3_one_minus_cos(kappa, u_dir);
        sn = sqrt(omc * (2.0 - omc));
      } else if (!vm2_draw(kappa, seed, strm, a, &omc, &sn)) {
        status = 1;
        break;
      }
      const double sd = sqrt(0.5 * t);
      const double m0 = 0.5 * (Ri + Rf * (1.0 - omc)) + sd * xi[0];
      const double m1 = 0.5 * Rf * sn + sd * xi[1];
      const double m2 = dim == 3 ? sd * xi[2] : 0.0;
      const double Rm = sqrt(m0 * m0 + m1 * m1 + m2 * m2);
      a++;
      const double p1 = fpt_p_enc(dim, Rm, Ri, 0.5 * t, tau_s);
      if (fabs(u_e1 - p1) < mg) mg = fabs(u_e1 - p1);
      if (u_e1 < p1) {            /* first contact in the first half */
        Rf = Rm;
        b = 2 * b;
        break;
      }
      const double p2 = fpt_p_enc(dim, Rf, Rm, 0.5 * t, tau_s);
      if (fabs(u_e2 - p2) < mg) mg = fabs(u_e2 - p2);
      if (u_e2 < p2) {            /* no contact in the first half, so it is in the second */
        Ri = Rm;
        b = 2 * b + 1;
        break;
      }
    }
    t *= 0.5;
  }
  if (bin) *bin = status ? 0xFFFFFFFFu : b;
  if (R_lo) *R_lo = status ? NAN : Ri;
  if (R_hi) *R_hi = status ? NAN : Rf;
  if (attempts) *attempts = a;
  if (margin) *margin = mg;
  return status;
}
