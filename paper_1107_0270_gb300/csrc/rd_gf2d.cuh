// 2D radial Green's-function quantities on the device (Section 4.2 of the paper), scaled units
// a = 1, tau = D t / a^2, h = kappa_a / (2 pi D).
//
// Two regimes, as in the paper: tau <= tau_s uses the small-time series of Eqs. (smallTEabs) and
// (smallTEabsII) truncated at 12 terms; larger tau uses the exact n = 0 term of Eq. (genericGF),
//   g(R) = (1/2pi) int_0^inf e^{-tau x^2} C_0(R,x) C_0(R0,x) x dx,
// by composite Gauss-Legendre quadrature in t with x = t^2.  The Bessel values at the abscissas
// (x J1 + h J0, x Y1 + h Y0 and their norm for each boundary condition) are computed once per pair
// type on the host; the values at R x and R0 x are computed per pair.
#pragma once

#include "rd_internal.cuh"

namespace rd {

constexpr int kSeriesTerms = 12;

// Per-node record of the Weber quadrature (built by the host for one pair type).
struct WeberNode {
  double x;           // abscissa x = t^2
  double w;           // weight including dx = 2t dt, x and e^{-tau x^2} / (2 pi)
  double a[3], b[3];  // alpha/N, beta/N for abs, ref, rad: C_0(R,x) = Y0(Rx) a - J0(Rx) b
};

// Host-built per-pair-type series data: coefficients of the boundary quotient series in y = 1/q
// for abs, ref, rad (Eqs. absPert, refPert, radPert expanded with a_k(0), a_k(1)) and a_k(0).
struct Series2D {
  double ratio[3][kSeriesTerms + 1];
  double a0[kSeriesTerms + 1];
};

__device__ __forceinline__ int bc_slot(int bc) { return bc == RD_BC_ABS ? 0 : (bc == RD_BC_REF ? 1 : 2); }

// e^{x} I0(x) scaled: library I0 below 30, large-argument series above.
__device__ __forceinline__ double i0e_d(double x) {
  if (x < 30.0) return cyl_bessel_i0(x) * exp(-x);
  double s = 1.0, t = 1.0;
#pragma unroll 1
  for (int k = 1; k < 24; ++k) {
    t *= (2.0 * k - 1.0) * (2.0 * k - 1.0) / (8.0 * k * x);
    s += t;
  }
  return s * rsqrt(2.0 * kPi * x);
}

// e^{z^2} i^n erfc(z), n = 0..nmax-1 into out[0..nmax-1]: recursion upward for z < 1.5, downward on
// ratios from order nmax + 80 otherwise (i^{-1} erfc = (2/sqrt(pi)) e^{-z^2}, i^0 erfc = erfc).
__device__ __forceinline__ void ierfc_scaled_all(double z, int nmax, double out[kSeriesTerms]) {
  const double e0 = erfcx(z);
  out[0] = e0;
  if (z < 1.5) {
    double fm2 = 2.0 / kSqrtPi, fm1 = e0;
#pragma unroll 1
    for (int k = 1; k < nmax; ++k) {
      const double fk = (fm2 - 2.0 * z * fm1) / (2.0 * k);
      out[k] = fk;
      fm2 = fm1;
      fm1 = fk;
    }
  } else {
    const int M = nmax + 80;
    double r = (sqrt(z * z + 2.0 * M) - z) / (2.0 * M);
    double ratios[kSeriesTerms];
#pragma unroll 1
    for (int k = M; k >= 1; --k) {
      if (k < nmax) ratios[k] = r;
      r = 1.0 / (2.0 * z + 2.0 * k * r);
    }
    double f = e0;
#pragma unroll 1
    for (int k = 1; k < nmax; ++k) {
      f *= ratios[k];
      out[k] = f;
    }
  }
}

// bracket of Eqs. (smallTEabs)/(smallTEabsII) after removing e^{-z^2}: pi^{-1/2} +
// (1/2) sum_{n=1}^{12} gamma_n e^{z^2} i^{n-1} erfc(z) (2 sqrt tau)^n, gamma from the quotient
// series times the K0(q R0) K0(q R) series.
__device__ __forceinline__ double series_bracket2(const Series2D& S, int slot, double R, double R0, double s,
                                                  const double ie[kSeriesTerms]) {
  double k0[kSeriesTerms + 1], g[kSeriesTerms + 1];
  const double iR = 1.0 / R, iR0 = 1.0 / R0;
  // K0(q R0) K0(q R) series coefficients
#pragma unroll 1
  for (int k = 0; k <= kSeriesTerms; ++k) {
    double v = 0.0, pa = 1.0;
    for (int j = 0; j <= k; ++j) {
      // a0[j] R0^-j a0[k-j] R^-(k-j)
      double pb = 1.0;
      for (int m = 0; m < k - j; ++m) pb *= iR;
      v += S.a0[j] * pa * S.a0[k - j] * pb;
      pa *= iR0;
    }
    k0[k] = v;
  }
#pragma unroll 1
  for (int k = 0; k <= kSeriesTerms; ++k) {
    double v = 0.0;
    for (int j = 0; j <= k; ++j) v += S.ratio[slot][j] * k0[k - j];
    g[k] = v;
  }
  double sum = 1.0 / kSqrtPi, p = 1.0;
#pragma unroll 1
  for (int n = 1; n <= kSeriesTerms; ++n) {
    p *= 2.0 * s;
    sum += 0.5 * g[n] * ie[n - 1] * p;
  }
  return sum;
}

// Weber sums over the nodes for up to three boundary conditions at once: out[slot] =
// sum_i w_i C_slot(R, x_i) C_slot(R0, x_i) (= g_slot(R | R0), the full radial function).
__device__ __forceinline__ void weber_g(const WeberNode* __restrict__ nodes, int n, double R, double R0,
                                        unsigned mask, double out[3]) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll 1
  for (int i = 0; i < n; ++i) {
    const WeberNode& nd = nodes[i];
    const double jr = j0(R * nd.x), yr = y0(R * nd.x);
    const double jr0 = j0(R0 * nd.x), yr0 = y0(R0 * nd.x);
    if (mask & 1u) s0 += nd.w * (yr * nd.a[0] - jr * nd.b[0]) * (yr0 * nd.a[0] - jr0 * nd.b[0]);
    if (mask & 2u) s1 += nd.w * (yr * nd.a[1] - jr * nd.b[1]) * (yr0 * nd.a[1] - jr0 * nd.b[1]);
    if (mask & 4u) s2 += nd.w * (yr * nd.a[2] - jr * nd.b[2]) * (yr0 * nd.a[2] - jr0 * nd.b[2]);
  }
  out[0] = s0;
  out[1] = s1;
  out[2] = s2;
}

// Eq. (psurv_radII) numerator and denominator as single Weber sums of differences (the free parts
// cancel node by node, Section 4.2): num = sum_i w_i [C_ref C_ref - C_rad C_rad](R, R0; x_i),
// den = sum_i w_i [C_ref C_ref - C_abs C_abs](R, R0; x_i).
__device__ __forceinline__ void weber_reac_diffs(const WeberNode* __restrict__ nodes, int n, double R, double R0,
                                                 double& num, double& den) {
  double sn = 0.0, sd = 0.0;
#pragma unroll 1
  for (int i = 0; i < n; ++i) {
    const WeberNode& nd = nodes[i];
    const double jr = j0(R * nd.x), yr = y0(R * nd.x);
    const double jr0 = j0(R0 * nd.x), yr0 = y0(R0 * nd.x);
    const double ca = (yr * nd.a[0] - jr * nd.b[0]) * (yr0 * nd.a[0] - jr0 * nd.b[0]);
    const double cf = (yr * nd.a[1] - jr * nd.b[1]) * (yr0 * nd.a[1] - jr0 * nd.b[1]);
    const double cd = (yr * nd.a[2] - jr * nd.b[2]) * (yr0 * nd.a[2] - jr0 * nd.b[2]);
    sn += nd.w * (cf - cd);
    sd += nd.w * (cf - ca);
  }
  num = sn;
  den = sd;
}

// radial free function e^{-(R-R0)^2/4tau} I0e(R R0/2tau) / (4 pi tau)
__device__ __forceinline__ double gfree2_d(double R, double R0, double tau) {
  return exp(-(R - R0) * (R - R0) / (4.0 * tau)) * i0e_d(R * R0 / (2.0 * tau)) / (4.0 * kPi * tau);
}

struct Pair2D {
  bool series;           // tau <= tau_s
  bool series_rad;       // p_reac from the series too (tau <= tau_s and h sqrt(tau) small)
  double tau, s, h;
  const WeberNode* nodes;
  int n_nodes;
  const Series2D* ser;
};

// Eq. (bayes1D) in 2D.  Series: p_enc = e^{-(R-1)(R0-1)/tau} sqrt(tau) B_abs / (sqrt(R R0) I0e(R R0/2tau)).
__device__ __forceinline__ double p_enc2(const Pair2D& q, double R, double R0) {
  if (R <= 1.0) return 1.0;
  if (R0 <= 1.0) return 1.0;
  if (q.series) {
    double ie[kSeriesTerms];
    ierfc_scaled_all((R + R0 - 2.0) / (2.0 * q.s), kSeriesTerms, ie);
    const double b = series_bracket2(*q.ser, 0, R, R0, q.s, ie);
    return exp(-(R - 1.0) * (R0 - 1.0) / q.tau) * q.s * b / (sqrt(R * R0) * i0e_d(R * R0 / (2.0 * q.tau)));
  }
  double g[3];
  weber_g(q.nodes, q.n_nodes, R, R0, 1u, g);
  return 1.0 - g[0] / gfree2_d(R, R0, q.tau);
}

// Eq. (psurv_radII) in 2D (the free parts cancel; in the series so does the prefactor).
__device__ __forceinline__ double p_reac2(const Pair2D& q, double R, double R0) {
  if (R < 1.0) R = 1.0;
  if (R0 < 1.0) R0 = 1.0;
  double p;
  if (q.series_rad) {
    double ie[kSeriesTerms];
    ierfc_scaled_all((R + R0 - 2.0) / (2.0 * q.s), kSeriesTerms, ie);
    const double ba = series_bracket2(*q.ser, 0, R, R0, q.s, ie);
    const double bf = series_bracket2(*q.ser, 1, R, R0, q.s, ie);
    const double bd = series_bracket2(*q.ser, 2, R, R0, q.s, ie);
    p = (bf - bd) / (bf + ba);
  } else {
    double num, den;
    weber_reac_diffs(q.nodes, q.n_nodes, R, R0, num, den);
    p = num / den;
  }
  return p < 0.0 ? 0.0 : (p > 1.0 ? 1.0 : p);
}

// Unnormalised CDF of the encountered pair's new separation over (1, 1 + V):
// integral of 2 pi R (g_ref - g_abs).  Weber: the R-integral is analytic (R Z1(Rx)/x is an
// antiderivative of R Z0(Rx)); series: composite Gauss-Legendre in R.
__device__ __forceinline__ double cdf2(const Pair2D& q, double V, double R0, const double* __restrict__ gl16) {
  if (V <= 0.0) return 0.0;
  if (!q.series) {
    const double Rp = 1.0 + V;
    double s = 0.0;
#pragma unroll 1
    for (int i = 0; i < q.n_nodes; ++i) {
      const WeberNode& nd = q.nodes[i];
      const double x = nd.x;
      const double jr0 = j0(R0 * x), yr0 = y0(R0 * x);
      const double j1r = j1(Rp * x), y1r = y1(Rp * x), j11 = j1(x), y11 = y1(x);
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < 2; ++k) {      // ref (+) and abs (-)
        const int slot = k == 0 ? 1 : 0;
        const double c0r0 = yr0 * nd.a[slot] - jr0 * nd.b[slot];
        const double part = (Rp * (y1r * nd.a[slot] - j1r * nd.b[slot]) - (y11 * nd.a[slot] - j11 * nd.b[slot])) / x;
        acc += (k == 0 ? 1.0 : -1.0) * c0r0 * part;
      }
      s += nd.w * 2.0 * kPi * acc;     // nd.w carries 1/2pi
    }
    return s;
  }
  // series regime: panels of width ~ sqrt(tau), 16 Gauss-Legendre nodes each
  const int panels = 1 + (int)(V / q.s);
  const double hstep = V / panels;
  double s = 0.0;
  double ie[kSeriesTerms];
#pragma unroll 1
  for (int pnl = 0; pnl < panels; ++pnl) {
    const double a = 1.0 + pnl * hstep, m = a + 0.5 * hstep;
#pragma unroll 1
    for (int i = 0; i < 16; ++i) {
      const double R = m + 0.5 * hstep * gl16[i];
      const double z = (R + R0 - 2.0) / (2.0 * q.s);
      ierfc_scaled_all(z, kSeriesTerms, ie);
      const double pref = exp(-z * z) / (4.0 * kPi * sqrt(q.tau * R * R0));
      const double dens = 2.0 * kPi * R * pref *
                          (series_bracket2(*q.ser, 1, R, R0, q.s, ie) + series_bracket2(*q.ser, 0, R, R0, q.s, ie));
      s += gl16[16 + i] * dens;
    }
  }
  return s * 0.5 * hstep;
}

// density 2 pi R (g_ref - g_abs) at R (derivative of cdf2)
__device__ __forceinline__ double dens2(const Pair2D& q, double R, double R0) {
  if (q.series) {
    double ie[kSeriesTerms];
    const double z = (R + R0 - 2.0) / (2.0 * q.s);
    ierfc_scaled_all(z, kSeriesTerms, ie);
    const double pref = exp(-z * z) / (4.0 * kPi * sqrt(q.tau * R * R0));
    return 2.0 * kPi * R * pref * (series_bracket2(*q.ser, 1, R, R0, q.s, ie) + series_bracket2(*q.ser, 0, R, R0, q.s, ie));
  }
  double g[3];
  weber_g(q.nodes, q.n_nodes, R, R0, 3u, g);
  return 2.0 * kPi * R * (g[1] - g[0]);
}

// New separation R' >= 1 with tail fraction U (Newton on cdf2/tot = 1 - U within a bisection
// bracket on (0, vmax), vmax = R0 + 13 sqrt(tau) beyond which the density is below e^{-40}).
__device__ __forceinline__ double resample2(const Pair2D& q, double U, double R0, const double* __restrict__ gl16) {
  if (R0 < 1.0) R0 = 1.0;
  const double vmax = R0 + 13.0 * q.s;
  const double tot = cdf2(q, vmax, R0, gl16);
  const double target = (1.0 - U) * tot;
  double lo = 0.0, hi = vmax, V = fmin(q.s, 0.5 * vmax);
#pragma unroll 1
  for (int it = 0; it < 100; ++it) {
    const double f = cdf2(q, V, R0, gl16) - target;
    if (f < 0.0)
      lo = V;
    else
      hi = V;
    const double d = dens2(q, 1.0 + V, R0);
    double Vn = d > 0.0 ? V - f / d : 0.5 * (lo + hi);
    const bool inside = Vn > lo && Vn < hi;
    if (!inside) Vn = 0.5 * (lo + hi);
    const double step = fabs(Vn - V);
    V = Vn;
    if (inside && step <= 1e-10 * fmax(V, q.s)) break;
    if (hi - lo <= 4e-16 * fmax(hi, q.s)) break;
  }
  return 1.0 + V;
}

}  // namespace rd
