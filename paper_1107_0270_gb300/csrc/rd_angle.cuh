// Exact direction of an encountered pair's new separation on the device (Eq. passage_prob with the
// full Green's functions, Eqs. genericGF3D / genericGF).
//
// Given the new separation length R' (drawn from the radial law) and the start separation R0, the
// angle between the new and the start separation vectors follows the partial-wave series
//   3D: f(mu) = sum_n (2n+1) P_n(mu) D_n / (2 D_0),
//   2D: f(theta) = [D_0 + 2 sum_{n>=1} D_n cos(n theta)] / (2 pi D_0),
// D_n = int_0^inf e^{-tau x^2} x^{d-1} [C^ref_n(R',x) C^ref_n(R0,x) - C^abs_n(R',x) C^abs_n(R0,x)] dx,
// with C_n(R, x) = [Z1_n(Rx) b_n(x) - Z2_n(Rx) a_n(x)] / sqrt(a_n^2 + b_n^2) from the spherical (3D)
// or integer-order (2D, Eq. fRad) Bessel functions of the first and second kind; reflective:
// (a, b) = x times the derivatives of (Z1, Z2) at x; absorbing: (a, b) = (Z1, Z2) at x.  The
// functions come from their three-term recurrences (Eq. 3termBessel): the second kind upward, the
// first kind downward from far above, normalised by its sum rule.
//
// One warp evaluates one pair: the lanes share the quadrature nodes (composite 16-point
// Gauss-Legendre over x in [0, sqrt(46/tau)] in 3D, over t = sqrt(x) in 2D, with
// 8 + ceil(sqrt(46/tau)(R'+R0)/1.5) panels), the D_n are
// reduced across the warp and held distributed (lane l keeps D_l, D_{l+32}, ...), and the angle is
// found by bisection of the CDF, every lane evaluating its own orders' share of each CDF value.
// All 32 lanes must call with identical arguments.  T = double (FP64 step) or float (mixed step).
//
// Mixed step: the law is tabulated once per pair rule instead (FP64 build, one warp per node).  The
// table holds, on a grid of (R0, R') and of U, the CDF value s that the exact angle has under a
// reference law with closed-form CDF and the same concentration kappa = R' R0 / (2 tau): in 3D the
// free propagator's own angular law, exp(kappa mu) on mu in [-1, 1]; in 2D a normal law in theta
// of variance 1/kappa folded and truncated to [0, pi].  s(U) is smooth and equals U when the
// boundary does not matter, so a Catmull-Rom interpolation in the three axes followed by the
// reference law's inverse gives the angle in a few dozen loads per pair.
#pragma once

#include "rd_internal.cuh"

namespace rd {

constexpr int kAngNMax = 128;          // partial waves at most (kappa = R' R0 / 2 tau up to ~53)
constexpr int kAngSlots = kAngNMax / 32;
constexpr int kAngBuildSlots = 6;      // table nodes: up to 192 partial waves

template <class T> struct AngConst;
template <> struct AngConst<double> {
  static constexpr double big = 1e280, grow = 1e100, shrink = 1e-100, shrink2 = 1e-200, seed = 1e-30;
};
template <> struct AngConst<float> {
  static constexpr float big = 1e30f, grow = 1e15f, shrink = 1e-15f, shrink2 = 1e-30f, seed = 1e-10f;
};

__device__ __forceinline__ double ang_sin(double x) { return sin(x); }
__device__ __forceinline__ float ang_sin(float x) { return sinf(x); }
__device__ __forceinline__ double ang_cos(double x) { return cos(x); }
__device__ __forceinline__ float ang_cos(float x) { return cosf(x); }
__device__ __forceinline__ double ang_y0(double x) { return y0(x); }
__device__ __forceinline__ float ang_y0(float x) { return y0f(x); }
__device__ __forceinline__ double ang_y1(double x) { return y1(x); }
__device__ __forceinline__ float ang_y1(float x) { return y1f(x); }

// First kind, orders 0..N, by the downward recurrence from M = N + 40 + z (spherical: sum rule
// sum (2n+1) j_n^2 = 1, sign of j_0 or j_1; cylindrical: J_0 + 2 sum J_2k = 1).
template <class T>
__device__ __forceinline__ void bessel_first(int dim, int N, T z, T* __restrict__ j) {
  using C = AngConst<T>;
  int M = N + 40 + (int)z;
  if (dim == 2 && (M & 1)) ++M;
  T jp1 = T(0), jn = C::seed, sum = T(0);
  T scale_acc = T(1);   // product of rescalings applied to the stored values
  (void)scale_acc;
#pragma unroll 1
  for (int n = M; n >= 0; --n) {
    if (n <= N) j[n] = jn;
    sum += dim == 3 ? T(2 * n + 1) * jn * jn : (n == 0 ? jn : ((n & 1) ? T(0) : T(2) * jn));
    const T jm1 = n > 0 ? (dim == 3 ? T(2 * n + 1) : T(2 * n)) / z * jn - jp1 : T(0);
    jp1 = jn;
    jn = jm1;
    if (fabs(jn) > C::grow) {
      for (int m = n; m <= N; ++m) j[m] *= C::shrink;
      jn *= C::shrink;
      jp1 *= C::shrink;
      sum *= dim == 3 ? C::shrink2 : C::shrink;
    }
  }
  T scale;
  if (dim == 3) {
    scale = T(1) / sqrt(sum);
    const T s = ang_sin(z), c = ang_cos(z);
    const T j0 = s / z, j1 = s / (z * z) - c / z;
    const bool neg = fabs(j0) >= fabs(j1) ? ((j0 < T(0)) != (j[0] < T(0))) : ((j1 < T(0)) != (j[1] < T(0)));
    if (neg) scale = -scale;
  } else {
    scale = T(1) / sum;
  }
  for (int n = 0; n <= N; ++n) j[n] *= scale;
}

// Second kind of orders 0 and 1 at z.
template <class T>
__device__ __forceinline__ void bessel_second01(int dim, T z, T& y0v, T& y1v) {
  if (dim == 3) {
    const T s = ang_sin(z), c = ang_cos(z);
    y0v = -c / z;
    y1v = -c / (z * z) - s / z;
  } else {
    y0v = ang_y0(z);
    y1v = ang_y1(z);
  }
}

// lane-distributed value of slot k (k < S) of the partial-wave coefficients
template <class T, int S>
__device__ __forceinline__ T ang_slot(const T (&acc)[S], int k) {
  T v = acc[0];
#pragma unroll
  for (int s = 1; s < S; ++s)
    if (k == s) v = acc[s];
  return v;
}

// partial waves the law of concentration kappa needs (the series' terms beyond are below 1e-16)
template <class T>
__device__ __forceinline__ int ang_terms(T kappa) {
  return (int)ceil(kappa + T(8) * sqrt(kappa + T(1)) + T(14));
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

// CDF of the conditional angle at v from the distributed coefficients (every lane returns it).
template <class T, int S>
__device__ __forceinline__ T ang_cdf_warp(int dim, const T (&acc)[S], T inv_d0, int N, T v) {
  const int lane = threadIdx.x & 31;
  T part = T(0);
  if (dim == 3) {
    // sum_{n>=1} (D_n/D_0) [P_{n+1}(v) - P_{n-1}(v)] / 2 : every lane runs the recurrence and adds its orders
    T pm1 = T(1), p = v;   // P_{n-1}, P_n at n = 1
#pragma unroll 1
    for (int n = 1; n <= N; ++n) {
      const T pp1 = (T(2 * n + 1) * v * p - T(n) * pm1) / T(n + 1);
      if ((n & 31) == lane) part += ang_slot(acc, n >> 5) * (pp1 - pm1);
      pm1 = p;
      p = pp1;
    }
    return T(0.5) * (T(1) + v) + T(0.5) * inv_d0 * warp_sum(part);
  }
  // 2D: [theta + 2 sum_{n>=1} (D_n/D_0) sin(n theta)/n] / pi
#pragma unroll 1
  for (int n = lane; n <= N; n += 32)
    if (n >= 1) part += ang_slot(acc, n >> 5) * ang_sin(T(n) * v) / T(n);
  return (v + T(2) * inv_d0 * warp_sum(part)) / T(kPi);
}

// Partial-wave integrals D_0 .. D_N (N < 32 S) of the law at (R, R0, tau), lane-distributed: lane l
// holds D_{l + 32 s} in acc[s].  Warp-collective.
template <class T, int S>
__device__ __forceinline__ void ang_coeffs_warp(int dim, int N, T R, T R0, T tau, const double* __restrict__ gl16,
                                                T (&acc)[S]) {
  using C = AngConst<T>;
  const int lane = threadIdx.x & 31;
  const T X = sqrt(T(46) / tau);
  const int panels = 8 + (int)ceil(X * (R + R0) / T(1.5));
  const int nodes = 16 * panels;
  // 3D: panels in x on [0, X]; 2D: in t with x = t^2 on [0, sqrt(X)] (dx = 2t dt), which smooths the
  // logarithmic behaviour of the integer-order boundary coefficients at x -> 0
  const T hp = (dim == 3 ? X : sqrt(X)) / T(panels);
#pragma unroll
  for (int s = 0; s < S; ++s) acc[s] = T(0);
  T jx[32 * S + 2], jr[32 * S + 1], jq[32 * S + 1];
#pragma unroll 1
  for (int base = 0; base < nodes; base += 32) {
    const int k = base + lane;
    const bool on = k < nodes;
    T w = T(0), x = T(1);
    // second kind: (y_n, y_{n+1}) at x, R x, R0 x, and y_{n-1} at x
    T ax = T(0), bx = T(0), ar = T(0), br = T(0), aq = T(0), bq = T(0), px = T(0);
    if (on) {
      const int p = k >> 4, i = k & 15;
      const T t = (T(p) + T(0.5)) * hp + T(0.5) * hp * T(gl16[i]);
      x = dim == 3 ? t : t * t;
      w = T(0.5) * hp * T(gl16[16 + i]) * exp(-tau * x * x) * (dim == 3 ? x * x : x * T(2) * t);
      bessel_first<T>(dim, N + 1, x, jx);
      bessel_first<T>(dim, N, R * x, jr);
      bessel_first<T>(dim, N, R0 * x, jq);
      bessel_second01<T>(dim, x, ax, bx);
      bessel_second01<T>(dim, R * x, ar, br);
      bessel_second01<T>(dim, R0 * x, aq, bq);
    }
    bool dead = !on;
#pragma unroll 1
    for (int n = 0; n <= N; ++n) {
      T c = T(0);
      // an order whose second-kind values have grown past C::big contributes nothing here
      if (!dead && (fabs(bx) > C::big || fabs(ar) > C::big || fabs(aq) > C::big)) dead = true;
      if (!dead) {
        const T kd = dim == 3 ? T(n + 1) : T(n);
        const T jd = n == 0 ? -jx[1] : jx[n - 1] - kd / x * jx[n];
        const T yd = n == 0 ? -bx : px - kd / x * ax;
        T a = -x * jd, b = -x * yd;
        T nr = fabs(b) > fabs(a) ? fabs(b) * sqrt(T(1) + (a / b) * (a / b)) : fabs(a) * sqrt(T(1) + (b / a) * (b / a));
        const T car = a / nr, cbr = b / nr;
        a = jx[n];
        b = ax;
        nr = fabs(b) > fabs(a) ? fabs(b) * sqrt(T(1) + (a / b) * (a / b)) : fabs(a) * sqrt(T(1) + (b / a) * (b / a));
        const T caa = a / nr, cba = b / nr;
        const T ref = (jr[n] * cbr - ar * car) * (jq[n] * cbr - aq * car);
        const T abs_ = (jr[n] * cba - ar * caa) * (jq[n] * cba - aq * caa);
        c = w * (ref - abs_);
        // advance: Z_{n+2} = (k_{n+1} / z) Z_{n+1} - Z_n, k_m = 2m + 1 (3D) or 2m (2D)
        const T km = dim == 3 ? T(2 * n + 3) : T(2 * n + 2);
        const T nx = km / x * bx - ax, nrr = km / (R * x) * br - ar, nq = km / (R0 * x) * bq - aq;
        px = ax;
        ax = bx;
        bx = nx;
        ar = br;
        br = nrr;
        aq = bq;
        bq = nq;
      }
      c = warp_sum(c);
      if ((n & 31) == lane) {
#pragma unroll
        for (int s = 0; s < S; ++s)
          if ((n >> 5) == s) acc[s] += c;
      }
    }
  }
}

// Angle of the new separation to the start separation at CDF value U: 3D cos(angle) in [-1, 1],
// 2D the angle in [0, pi].  Returns NaN if the law needs more than kAngNMax partial waves.
template <class T>
__device__ __noinline__ T ang_sample_warp(int dim, T U, T R, T R0, T tau, const double* __restrict__ gl16) {
  const T kappa = R * R0 / (T(2) * tau);
  const int N = ang_terms(kappa);
  if (N > kAngNMax - 1) return T(NAN);
  T acc[kAngSlots];
  ang_coeffs_warp<T, kAngSlots>(dim, N, R, R0, tau, gl16, acc);
  const T d0 = __shfl_sync(0xFFFFFFFFu, acc[0], 0);
  const T inv_d0 = T(1) / d0;
  // bisection of the CDF to the last representable step
  T lo = dim == 3 ? T(-1) : T(0), hi = dim == 3 ? T(1) : T(kPi);
#pragma unroll 1
  for (int it = 0; it < 200; ++it) {
    const T mid = T(0.5) * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (ang_cdf_warp<T>(dim, acc, inv_d0, N, mid) < U)
      lo = mid;
    else
      hi = mid;
  }
  return T(0.5) * (lo + hi);
}

// A unit vector e1 perpendicular to the unit vector u (3D): the coordinate axis along u's smallest
// component (the first such axis on ties), made perpendicular and normalised; e2 = u x e1.
template <class T>
__device__ __forceinline__ void ang_perp_frame(const T* u, T* e1, T* e2) {
  int k = 0;
  if (fabs(u[1]) < fabs(u[k])) k = 1;
  if (fabs(u[2]) < fabs(u[k])) k = 2;
  const T d = u[k];
  T v[3] = {-d * u[0], -d * u[1], -d * u[2]};
  v[k] += T(1);
  const T nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  for (int i = 0; i < 3; ++i) e1[i] = v[i] / nv;
  e2[0] = u[1] * e1[2] - u[2] * e1[1];
  e2[1] = u[2] * e1[0] - u[0] * e1[2];
  e2[2] = u[0] * e1[1] - u[1] * e1[0];
}

// Unit direction of the new separation about the axis u (the start separation's direction) from
// the angle v (3D: its cosine; 2D: the angle in [0, pi]): azimuth 2 pi U_azi (3D) or the angle's
// sign from U_azi < 1/2 (2D).
template <class T>
__device__ __forceinline__ void ang_place(int dim, const T* u, T v, T U_azi, T* dir) {
  if (dim == 3) {
    const T st = sqrt(fmax(T(0), T(1) - v * v));
    T e1[3], e2[3];
    ang_perp_frame<T>(u, e1, e2);
    T sn, cs;
    if constexpr (sizeof(T) == 8)
      sincospi(T(2) * U_azi, &sn, &cs);
    else
      sincospif(T(2) * U_azi, &sn, &cs);
    for (int i = 0; i < 3; ++i) dir[i] = v * u[i] + st * (cs * e1[i] + sn * e2[i]);
  } else {
    const T th = U_azi < T(0.5) ? -v : v;
    const T c = ang_cos(th), s = ang_sin(th);
    dir[0] = c * u[0] - s * u[1];
    dir[1] = s * u[0] + c * u[1];
    dir[2] = T(0);
  }
}

// The direction from the exact law, warp-collective; returns false (dir untouched) when the law
// needs more partial waves than kAngNMax.
template <class T>
__device__ __forceinline__ bool ang_direction_warp(int dim, const T* u, T U_ang, T U_azi, T Rn, T R0, T tau,
                                                   const double* __restrict__ gl16, T* dir) {
  const T v = ang_sample_warp<T>(dim, U_ang, Rn, R0, tau, gl16);
  if (!(v == v)) return false;
  ang_place<T>(dim, u, v, U_azi, dir);
  return true;
}

// ------------------------------------------------------------------------------------------------
// Tabulated law (mixed step)
// ------------------------------------------------------------------------------------------------
// Reference law's CDF at v (3D: the cosine, density proportional to exp(kappa mu); 2D: the angle,
// normal of variance 1/kappa folded to [0, inf) and truncated to [0, pi]).
__device__ __forceinline__ double ang_ref_cdf(int dim, double v, double kappa) {
  if (dim == 3) return exp(kappa * (v - 1.0)) * expm1(-kappa * (v + 1.0)) / expm1(-2.0 * kappa);
  const double a = sqrt(0.5 * kappa);
  return erf(a * v) / erf(a * kPi);
}

// Inverse of the reference law's CDF at s in [0, 1].
__device__ __forceinline__ float ang_ref_inv(int dim, float s, float kappa) {
  if (dim == 3) return fminf(1.0f, fmaxf(-1.0f, 1.0f + log1pf((1.0f - s) * expm1f(-2.0f * kappa)) / kappa));
  const float a = sqrtf(0.5f * kappa);
  return fminf((float)kPi, fmaxf(0.0f, erfinvf(s * erff(a * (float)kPi)) / a));
}

// CDF of the exact law at v from the normalised coefficients Dn[n] = D_n / D_0 (n = 1..N), one
// thread (the table builder: every lane inverts its own U).
__device__ __forceinline__ double ang_cdf_thread(int dim, const double* Dn, int N, double v) {
  double acc = 0.0;
  if (dim == 3) {
    double pm1 = 1.0, p = v;   // P_{n-1}, P_n at n = 1
    for (int n = 1; n <= N; ++n) {
      const double pp1 = ((2 * n + 1) * v * p - n * pm1) / (n + 1);
      acc += Dn[n] * (pp1 - pm1);
      pm1 = p;
      p = pp1;
    }
    return 0.5 * (1.0 + v) + 0.5 * acc;
  }
  // sin(n v) by its recurrence sin((n+1) v) = 2 cos v sin(n v) - sin((n-1) v)
  const double c2 = 2.0 * cos(v);
  double sm1 = 0.0, sn = sin(v);
  for (int n = 1; n <= N; ++n) {
    acc += Dn[n] * sn / n;
    const double sp1 = c2 * sn - sm1;
    sm1 = sn;
    sn = sp1;
  }
  return (v + 2.0 * acc) / kPi;
}

// Concentration of the reference law whose median is v_med (bisection in ln kappa over
// [e^-12, e^8]; a median beyond the family's range takes the nearest end).
__device__ __forceinline__ double ang_ref_kappa(int dim, double v_med) {
  double lo = -12.0, hi = 8.0;
  for (int it = 0; it < 60; ++it) {
    const double m = 0.5 * (lo + hi), k = exp(m);
    // the reference median at k: 3D 1 + ln(1/2 + e^{-2k}/2)/k (rises with k), 2D falls with k
    const double vm = dim == 3 ? 1.0 + log1p(0.5 * expm1(-2.0 * k)) / k
                               : erfinv(0.5 * erf(sqrt(0.5 * k) * kPi)) / sqrt(0.5 * k);
    if (dim == 3 ? vm < v_med : vm > v_med)
      lo = m;
    else
      hi = m;
  }
  return exp(0.5 * (lo + hi));
}

// One node of the table (kAngTabStride floats at out): the reference-law CDF values s at
// w = (k - 1) / kAngTabU, k = 0 .. kAngTabU + 2, then the reference concentration.  The U axis is
// stretched towards both ends, U = sin^2(pi w / 2), where the exact law departs most from the
// reference (the backward direction); s is then an even function of w about w = 0 and about
// w = 1, which gives the ghosts.  The reference concentration is the one whose median is the exact
// law's: the encountered pairs' law is much broader than the free propagator's (its concentration
// R'R0/2tau), so matching it keeps s close to U.  Warp-collective; Dn: kAngBuildSlots * 32 doubles
// of this warp's shared memory.  A law needing more partial waves than the table build holds is
// stored as the free reference (s = U, concentration R'R0/2tau).
__device__ __forceinline__ void ang_table_node(int dim, double R, double R0, double tau,
                                               const double* __restrict__ gl16, double* Dn, float* out) {
  static_assert(kAngTabU == 64, "two interior U nodes per lane");
  const int lane = threadIdx.x & 31;
  const double kappa = R * R0 / (2.0 * tau);
  const int N = ang_terms(kappa);
  // lane l: the nodes j = l and j = l + 32 (interior nodes j = 1 .. 63; w = j / kAngTabU)
  double U2[2], v2[2], s2[2];
  for (int q = 0; q < 2; ++q) {
    const double sw = sin(0.5 * kPi * (lane + 32 * q) / kAngTabU);
    U2[q] = sw * sw;
    s2[q] = U2[q];
  }
  double kref = kappa;
  if (N <= 32 * kAngBuildSlots - 1) {
    double acc[kAngBuildSlots];
    ang_coeffs_warp<double, kAngBuildSlots>(dim, N, R, R0, tau, gl16, acc);
    const double inv_d0 = 1.0 / __shfl_sync(0xFFFFFFFFu, acc[0], 0);
#pragma unroll
    for (int k = 0; k < kAngBuildSlots; ++k) Dn[32 * k + lane] = acc[k] * inv_d0;
    __syncwarp();
    for (int q = 0; q < 2; ++q) {
      // bisection of the exact CDF to the last representable step (j = 0 is U = 0: no search)
      double lo = dim == 3 ? -1.0 : 0.0, hi = dim == 3 ? 1.0 : kPi;
      if (lane + 32 * q >= 1) {
        for (int it = 0; it < 80; ++it) {
          const double mid = 0.5 * (lo + hi);
          if (mid <= lo || mid >= hi) break;
          if (ang_cdf_thread(dim, Dn, N, mid) < U2[q])
            lo = mid;
          else
            hi = mid;
        }
      }
      v2[q] = 0.5 * (lo + hi);
    }
    __syncwarp();
    // the median: node j = 32 (U = 1/2) is lane 0's second node
    kref = ang_ref_kappa(dim, __shfl_sync(0xFFFFFFFFu, v2[1], 0));
    for (int q = 0; q < 2; ++q) s2[q] = ang_ref_cdf(dim, v2[q], kref);
  }
  const double s1 = __shfl_sync(0xFFFFFFFFu, s2[0], 1), slast = __shfl_sync(0xFFFFFFFFu, s2[1], 31);
  for (int q = 0; q < 2; ++q) {
    const int j = lane + 32 * q;
    if (j >= 1) out[j + 1] = (float)s2[q];
  }
  if (lane == 0) {
    out[0] = (float)s1;                     // ghost at w = -1 / kAngTabU
    out[1] = 0.0f;                          // U = 0
    out[kAngTabU + 1] = 1.0f;               // U = 1
    out[kAngTabU + 2] = (float)slast;       // ghost at w = 1 + 1 / kAngTabU
    out[kAngTabU + 3] = (float)kref;
  }
}

__device__ __forceinline__ void catmull_rom_w(float t, float w[4]) {
  const float t2 = t * t, t3 = t2 * t;
  w[0] = 0.5f * (-t3 + 2.0f * t2 - t);
  w[1] = 0.5f * (3.0f * t3 - 5.0f * t2 + 2.0f);
  w[2] = 0.5f * (-3.0f * t3 + 4.0f * t2 + t);
  w[3] = 0.5f * (t3 - t2);
}

// Angle from the table at (U, R', R0) (3D: its cosine; 2D: the angle in [0, pi]); NaN when the law
// needs more partial waves than kAngNMax (the exact evaluation's limit, so both precisions fall
// back on the same pairs).  Beyond the table (R' - 1 > d1max) the free reference law itself.
__device__ __forceinline__ float ang_table_sample(const AngTab& A, int dim, float U, float R, float R0) {
  const float kappa = R * R0 * A.inv_2tau;
  if (ang_terms(kappa) > kAngNMax - 1) return NAN;
  const float d0 = R0 - 1.0f, d1 = R - 1.0f;
  if (!(d1 <= A.d1max && d0 <= A.d0max)) return ang_ref_inv(dim, U, kappa);
  const float x0 = fmaxf(d0, 0.0f) * A.inv_h + 1.0f, x1 = fmaxf(d1, 0.0f) * A.inv_h + 1.0f;
  const float xu = asinf(sqrtf(U)) * (float)(2.0 / kPi) * kAngTabU + 1.0f;
  const int i0 = min((int)x0, A.n0 - 3), i1 = min((int)x1, A.n1 - 3), iu = min((int)xu, kAngTabU);
  float w0[4], w1[4], wu[4];
  catmull_rom_w(fminf(x0 - i0, 1.0f), w0);
  catmull_rom_w(fminf(x1 - i1, 1.0f), w1);
  catmull_rom_w(fminf(xu - iu, 1.0f), wu);
  float acc = 0.0f, kacc = 0.0f;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    float ra = 0.0f, ka = 0.0f;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float* node = A.v + ((size_t)(i0 - 1 + a) * A.n1 + (i1 - 1 + b)) * kAngTabStride;
      const float* row = node + (iu - 1);
      ra += w1[b] * (wu[0] * __ldg(row) + wu[1] * __ldg(row + 1) + wu[2] * __ldg(row + 2) + wu[3] * __ldg(row + 3));
      ka += w1[b] * __ldg(node + kAngTabU + 3);
    }
    acc += w0[a] * ra;
    kacc += w0[a] * ka;
  }
  return ang_ref_inv(dim, fminf(1.0f, fmaxf(0.0f, acc)), fmaxf(kacc, 1e-6f));
}

}  // namespace rd
