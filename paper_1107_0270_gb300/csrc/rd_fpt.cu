// First-passage refinement of encountered pairs (Appendix of the paper, "Relation to first-passage
// time simulation algorithms"): each pair's step is bisected `levels` times.
//
// At each level the separation at the midpoint of the current interval [t0, t0 + t] is drawn from
// the bridge of the radial process between the interval's end separations R_i, R_f, and the half
// holding the first contact is chosen with p_enc of the two halves (Eq. bayes1D in its radial
// form at time t/2).  The encounter is known for the whole interval, so the midpoint and the two
// decisions are redrawn until at least one half has an encounter; the first half wins when it has
// one.  Radial bridge midpoint: the end point's direction relative to the start follows the free
// Gaussian restricted to |r| = R_f (von Mises-Fisher with kappa = R_i R_f / 2t: 3D by inverting
// its CDF, 2D by Best and Fisher's rejection method), the midpoint vector is (r_i + r_f)/2 plus a
// Gaussian of variance t/2 per component (the paper's midpoint law, Eq. midPGauss, per component),
// and its length is the radial midpoint.
//
// Random numbers: Philox4x32-10, key = seed, counter (stream lo, stream hi, a, TAG_FPT | w << 8)
// with a the pair's attempt number over all levels and w: 0 = (U_dir, U_e1), 1 = two normals,
// 2 = a third normal (3D), 3 = U_e2, 4 + j = the j-th von Mises trial (2D, j < 64).
//
// The number of draws a pair needs is heavy-tailed (about 1/p_enc at the first level), so the
// attempts of a pair run in four tiers by count: a lane (phase 1), a warp (2), a block (3) and a
// group of blocks (4); since draws are indexed by the attempt number and the lowest-numbered
// decisive attempt always wins, every tier reproduces the serial loop.  On mixed-precision handles
// in 3D an attempt is evaluated in FP32 on contact distances (fpt_attempt_f), otherwise in FP64.
#include <type_traits>

#include "rd_gf2d.cuh"
#include "rd_kernels.h"

namespace rd {

constexpr uint32_t kVmTrials = 64;

__device__ __forceinline__ void fpt_draw(const FptArgs& A, uint64_t strm, uint32_t a, uint32_t w, double& u0,
                                         double& u1) {
  const uint4 o = philox(make_uint4((uint32_t)strm, (uint32_t)(strm >> 32), a, TAG_FPT | (w << 8)), A.seed_lo,
                         A.seed_hi);
  u0 = u52(o.x, o.y);
  u1 = u52(o.z, o.w);
}

// 3D von Mises-Fisher direction: 1 - cos(theta) = -log(u + (1 - u) e^{-2 kappa}) / kappa (the CDF
// inverted at 1 - u), as written for u <= 1/2 and through log1p/expm1 above, so that neither range
// cancels.
__device__ __forceinline__ double vmf3_omc(double kappa, double u) {
  if (u <= 0.5) return -log(u + (1.0 - u) * exp(-2.0 * kappa)) / kappa;
  return -log1p((1.0 - u) * expm1(-2.0 * kappa)) / kappa;
}

// von Mises angle (Best & Fisher 1979) as (1 - cos, sin), with the differences r - f and 1 - f
// formed from 1 - rho so that large kappa keeps its digits; false when all trials were rejected.
__device__ bool vm2_draw(const FptArgs& A, double kappa, uint64_t strm, uint32_t a, double& omc, double& sn) {
  const double s4 = sqrt(1.0 + 4.0 * kappa * kappa), t = 1.0 + s4, st = sqrt(2.0 * t);
  const double rho = 2.0 * kappa / (t + st);
  const double omr = (1.0 + 1.0 / (s4 + 2.0 * kappa) + st) / (t + st);     // 1 - rho
  const double r = (1.0 + rho * rho) / (2.0 * rho);
  const double r_m1 = omr * omr / (2.0 * rho);
  const double q = omr * (1.0 + rho);
  const double r2_m1 = q * q / (4.0 * rho * rho);
#pragma unroll 1
  for (uint32_t j = 0; j < kVmTrials; ++j) {
    double u1, u2;
    fpt_draw(A, strm, a, 4 + j, u1, u2);
    double sh, ch;
    sincospi(0.5 * u1, &sh, &ch);
    const double one_m_z = 2.0 * sh * sh, one_p_z = 2.0 * ch * ch;
    const double r_p_z = r_m1 + one_p_z;
    const double c = kappa * r2_m1 / r_p_z;
    if (c * (2.0 - c) > u2 || log(c / u2) + 1.0 - c >= 0.0) {
      const double omf = r_m1 * one_m_z / r_p_z;
      omc = omf;
      sn = sqrt(omf * ((r + 1.0) * one_p_z / r_p_z));
      return true;
    }
  }
  return false;
}

__device__ __noinline__ double fpt_p_enc2(const void* nodes, int n_nodes, const void* ser, double R, double R0,
                                          double tau) {
  if (R <= 1.0 || R0 <= 1.0) return 1.0;
  Pair2D q;
  q.series = nodes == nullptr;
  q.series_rad = false;
  q.tau = tau;
  q.s = sqrt(tau);
  q.h = 0.0;
  q.nodes = (const WeberNode*)nodes;
  q.n_nodes = n_nodes;
  q.ser = (const Series2D*)ser;
  return p_enc2(q, R, R0);
}

// 3D p_enc of a half interval.  Once (R + R0 - 1)/tau > 40 (so R R0 / tau > 40 too), both expm1
// terms of the closed form are -1 to within 5e-18 and p_enc = exp(-(R-1)(R0-1)/tau) to that
// accuracy; the deeper levels of the bisection are almost all in that range.
__device__ __forceinline__ double fpt_p_enc3(double R, double R0, double tau) {
  if (R <= 1.0) return 1.0;
  if (R0 < 1.0) R0 = 1.0;
  const double inv_tau = 1.0 / tau;
  if ((R + R0 - 1.0) * inv_tau > 40.0) return exp(-(R - 1.0) * (R0 - 1.0) * inv_tau);
  return p_enc3(R, R0, inv_tau);
}

__device__ __forceinline__ double fpt_p_enc(const FptArgs& A, int level, double R, double R0, double tau) {
  return A.dim == 3 ? fpt_p_enc3(R, R0, tau) : fpt_p_enc2(A.lv[level].nodes, A.lv[level].n_nodes, A.ser, R, R0, tau);
}

// One midpoint draw of attempt a on the interval (Ri, Rf, t) of level l: 0 = rejected (no
// encounter in either half), 1 = first contact in the first half, 2 = in the second half (no
// contact in the first), -1 = the von Mises trials ran out; *Rm = the midpoint separation.
__device__ __forceinline__ int fpt_attempt(const FptArgs& A, int l, uint64_t strm, uint32_t a, double Ri, double Rf,
                                           double t, double& Rm) {
  double u_dir, u_e1, u_e2, unused, v0, v1, x0, x1, x2 = 0.0, x3;
  fpt_draw(A, strm, a, 0, u_dir, u_e1);
  fpt_draw(A, strm, a, 1, v0, v1);
  box_muller(v0, v1, x0, x1);
  if (A.dim == 3) {
    fpt_draw(A, strm, a, 2, v0, v1);
    box_muller(v0, v1, x2, x3);
  }
  fpt_draw(A, strm, a, 3, u_e2, unused);
  const double kappa = Ri * Rf / (2.0 * t);
  double omc, sn;
  if (A.dim == 3) {
    omc = vmf3_omc(kappa, u_dir);
    sn = sqrt(omc * (2.0 - omc));
  } else if (!vm2_draw(A, kappa, strm, a, omc, sn)) {
    return -1;
  }
  const double sd = sqrt(0.5 * t);
  const double m0 = 0.5 * (Ri + Rf * (1.0 - omc)) + sd * x0;
  const double m1 = 0.5 * Rf * sn + sd * x1;
  const double m2 = sd * x2;
  Rm = sqrt(m0 * m0 + m1 * m1 + m2 * m2);
  if (u_e1 < fpt_p_enc(A, l, Rm, Ri, 0.5 * t)) return 1;
  if (u_e2 < fpt_p_enc(A, l, Rf, Rm, 0.5 * t)) return 2;
  return 0;
}

// FP32 form of one attempt (3D, mixed-precision handles).  It reads the same Philox words as the
// FP64 form (each uniform is the FP64 one rounded to FP32) and carries contact
// distances d = R - 1, so that separations near contact keep their digits: with the midpoint
// m = (1 + e0, m1, m2) in the frame of r_i, |m|^2 - 1 = e0 (2 + e0) + m1^2 + m2^2 and
// d_m = (|m|^2 - 1) / (|m| + 1).
// the FP64 uniform ((x >> 12) + 1/2) 2^-52 of x = hi:lo as hi 2^-32 + ((lo >> 12) + 1/2) 2^-52 in
// FP32 (32-bit conversions only; within one FP32 rounding of the FP64 value)
__device__ __forceinline__ float fpt_uf(uint32_t hi, uint32_t lo) {
  return fmaf(__uint2float_rn(hi), 0x1p-32f, (__uint2float_rn(lo >> 12) + 0.5f) * 0x1p-52f);
}

__device__ __forceinline__ void fpt_draw_f(const FptArgs& A, uint64_t strm, uint32_t a, uint32_t w, float& u0,
                                           float& u1) {
  const uint4 o = philox(make_uint4((uint32_t)strm, (uint32_t)(strm >> 32), a, TAG_FPT | (w << 8)), A.seed_lo,
                         A.seed_hi);
  u0 = fpt_uf(o.x, o.y);
  u1 = fpt_uf(o.z, o.w);
}

// p_enc in 3D from contact distances (FP32); the expm1 ratio is 1 to within 2e-9 once
// (d + d0 + 1) / tau > 20.
__device__ __forceinline__ float fpt_p_enc3_f(float d, float d0, float inv_tau) {
  if (d <= 0.0f) return 1.0f;
  if (d0 < 0.0f) d0 = 0.0f;
  if ((d + d0 + 1.0f) * inv_tau > 20.0f) return expf(-d * d0 * inv_tau);
  return p_enc3_f(d, d0, inv_tau);
}

__device__ __forceinline__ int fpt_attempt_f(const FptArgs& A, uint64_t strm, uint32_t a, float di, float df, float t,
                                             float& dm) {
  float u_dir, u_e1, u_e2, unused, v0, v1, x0, x1, x2, x3;
  fpt_draw_f(A, strm, a, 0, u_dir, u_e1);
  fpt_draw_f(A, strm, a, 1, v0, v1);
  box_muller_f(v0, v1, x0, x1);
  fpt_draw_f(A, strm, a, 2, v0, v1);
  box_muller_f(v0, v1, x2, x3);
  const float Rf = 1.0f + df;
  const float kappa = (1.0f + di) * Rf / (2.0f * t);
  const float omc = u_dir <= 0.5f ? -logf(u_dir + (1.0f - u_dir) * expf(-2.0f * kappa)) / kappa
                                  : -log1pf((1.0f - u_dir) * expm1f(-2.0f * kappa)) / kappa;
  const float sn = sqrtf(omc * (2.0f - omc));
  const float sd = sqrtf(0.5f * t);
  const float e0 = 0.5f * (di + df) - 0.5f * Rf * omc + sd * x0;
  const float m1 = 0.5f * Rf * sn + sd * x1;
  const float m2 = sd * x2;
  const float q = e0 * (2.0f + e0) + m1 * m1 + m2 * m2;
  dm = q / (sqrtf(1.0f + q) + 1.0f);
  const float inv_h = 2.0f / t;
  if (u_e1 < fpt_p_enc3_f(dm, di, inv_h)) return 1;
  fpt_draw_f(A, strm, a, 3, u_e2, unused);     // the second half's draw, needed only now
  if (u_e2 < fpt_p_enc3_f(df, dm, inv_h)) return 2;
  return 0;
}

// The precision dispatch: the FP64 form works on separations R, the FP32 form on d = R - 1; the
// interval state (Xi, Xf, t) is kept in the form's own type.
template <bool F32>
using fpt_real = typename std::conditional<F32, float, double>::type;

template <bool F32>
__device__ __forceinline__ int fpt_attempt_p(const FptArgs& A, int l, uint64_t strm, uint32_t a, fpt_real<F32> Xi,
                                             fpt_real<F32> Xf, fpt_real<F32> t, fpt_real<F32>& Xm) {
  if constexpr (F32)
    return fpt_attempt_f(A, strm, a, Xi, Xf, t, Xm);
  else
    return fpt_attempt(A, l, strm, a, Xi, Xf, t, Xm);
}

template <bool F32>
__device__ __forceinline__ void fpt_write(const FptArgs& A, int64_t k, bool ok, uint32_t b, uint32_t a, double Xi,
                                          double Xf, uint32_t* bin, double* r_lo, double* r_hi, uint32_t* attempts) {
  const double nan = __longlong_as_double(0x7FF8000000000000ll);
  const double Ri = F32 ? 1.0 + Xi : Xi, Rf = F32 ? 1.0 + Xf : Xf;
  bin[k] = ok ? b : 0xFFFFFFFFu;
  if (r_lo) r_lo[k] = ok ? Ri * A.sigma : nan;
  if (r_hi) r_hi[k] = ok ? Rf * A.sigma : nan;
  if (attempts) attempts[k] = a;
}

__device__ __forceinline__ FptItem fpt_item(double Ri, double Rf, double t, uint32_t k, uint32_t b, uint32_t a,
                                            int l) {
  FptItem it;
  it.Ri = Ri;
  it.Rf = Rf;
  it.t = t;
  it.k = k;
  it.b = b;
  it.a = a;
  it.l = (uint32_t)l;
  return it;
}

// Phase 1: persistent threads, one pair per lane, one draw per lane and iteration; a lane whose
// pair is done takes the next pair from a work counter (warp-aggregated), so the lanes of a warp
// stay busy whatever the draw counts of their pairs.  A pair that needs more than `budget` draws
// is queued with its state for phase 2.  The draws are indexed by the attempt number, so where an
// attempt runs does not change the result.
template <bool F32>
__global__ void __launch_bounds__(128) k_first_passage(const FptArgs A, const double* __restrict__ r0,
                                                       const double* __restrict__ r,
                                                       const uint64_t* __restrict__ stream, int64_t n,
                                                       uint32_t* __restrict__ bin, double* __restrict__ r_lo,
                                                       double* __restrict__ r_hi, uint32_t* __restrict__ attempts,
                                                       FptItem* __restrict__ queue, uint32_t* __restrict__ qctl,
                                                       uint32_t budget) {
  const uint32_t lane = threadIdx.x & 31u;
  const double inv_sigma = 1.0 / A.sigma;
  using real = fpt_real<F32>;
  int64_t k = 0;
  uint64_t strm = 0;
  real Ri = 0, Rf = 0, t = 0;
  uint32_t b = 0, a = 0;
  int l = 0;
  bool need = true, done = false;
#pragma unroll 1
  for (;;) {
    const unsigned nm = __ballot_sync(0xFFFFFFFFu, need);
    if (nm) {
      const int leader = __ffs(nm) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd((unsigned long long*)&qctl[kFptPairCtr], (unsigned long long)__popc(nm));
      base = __shfl_sync(0xFFFFFFFFu, base, leader);
      if (need) {
        const unsigned long long kk = base + __popc(nm & ((1u << lane) - 1u));
        need = false;
        if ((int64_t)kk < n) {
          k = (int64_t)kk;
          strm = stream[k];
          Ri = (real)(fmax(r0[k], 0.0) * inv_sigma - (F32 ? 1.0 : 0.0));     // a separation is not negative
          Rf = (real)(fmax(r[k], 0.0) * inv_sigma - (F32 ? 1.0 : 0.0));
          t = (real)A.tau;
          b = a = 0;
          l = 0;
        } else {
          done = true;
        }
      }
    }
    if (__all_sync(0xFFFFFFFFu, done)) break;
    if (done) continue;
    if (l >= A.levels) {
      fpt_write<F32>(A, k, true, b, a, Ri, Rf, bin, r_lo, r_hi, attempts);
      need = true;
      continue;
    }
    if (a >= A.max_attempts) {
      fpt_write<F32>(A, k, false, b, a, Ri, Rf, bin, r_lo, r_hi, attempts);
      need = true;
      continue;
    }
    if (a >= budget) {
      queue[atomicAdd(&qctl[kFptRound0 + kFptWarpIn], 1u)] = fpt_item(Ri, Rf, t, (uint32_t)k, b, a, l);
      need = true;
      continue;
    }
    real Rm;
    const int d = fpt_attempt_p<F32>(A, l, strm, a, Ri, Rf, t, Rm);
    if (d < 0) {                // the attempt that ran out of von Mises trials is not counted
      fpt_write<F32>(A, k, false, b, a, Ri, Rf, bin, r_lo, r_hi, attempts);
      need = true;
      continue;
    }
    ++a;
    if (d != 0) {
      if (d == 1) {
        Rf = Rm;
        b = 2 * b;
      } else {
        Ri = Rm;
        b = 2 * b + 1;
      }
      ++l;
      t *= (real)0.5;
      if (l >= A.levels) {      // done: the lane takes its next pair in the next iteration
        fpt_write<F32>(A, k, true, b, a, Ri, Rf, bin, r_lo, r_hi, attempts);
        need = true;
      }
    }
  }
}

// Phase 2: one warp per queued pair; each round the 32 lanes try the next 32 attempts and the
// lowest-numbered decisive one wins (the attempt the serial loop would stop at).  A pair that has
// drawn `budget` more times since it was queued moves on to queue_out (phase 3).
template <bool F32>
__global__ void __launch_bounds__(128) k_first_passage_warp(const FptArgs A, const uint64_t* __restrict__ stream,
                                                            uint32_t* __restrict__ bin, double* __restrict__ r_lo,
                                                            double* __restrict__ r_hi,
                                                            uint32_t* __restrict__ attempts,
                                                            const FptItem* __restrict__ queue, int count_word,
                                                            int next_word, FptItem* __restrict__ queue_out,
                                                            int out_word, uint32_t* __restrict__ qctl,
                                                            uint32_t budget) {
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll 1
  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(&qctl[next_word], 1u);
    item = __shfl_sync(0xFFFFFFFFu, item, 0);
    if (item >= *(volatile uint32_t*)&qctl[count_word]) break;
    using real = fpt_real<F32>;
    const FptItem it = queue[item];
    const uint64_t strm = stream[it.k];
    real Ri = (real)it.Ri, Rf = (real)it.Rf, t = (real)it.t;
    uint32_t b = it.b, a = it.a;
    bool ok = true, moved = false;
#pragma unroll 1
    for (int l = (int)it.l; l < A.levels && ok && !moved; ++l) {
#pragma unroll 1
      for (;;) {
        if (a >= A.max_attempts) {
          ok = false;
          break;
        }
        if (a - it.a >= budget) {
          if (lane == 0) queue_out[atomicAdd(&qctl[out_word], 1u)] = fpt_item(Ri, Rf, t, it.k, b, a, l);
          moved = true;
          break;
        }
        const unsigned long long mine = (unsigned long long)a + lane;
        real Rm = 0;
        int d = 0;
        if (mine < A.max_attempts) d = fpt_attempt_p<F32>(A, l, strm, (uint32_t)mine, Ri, Rf, t, Rm);
        const unsigned m = __ballot_sync(0xFFFFFFFFu, d != 0);
        if (m == 0) {
          const uint32_t room = A.max_attempts - a;
          a += room < 32u ? room : 32u;
          continue;
        }
        const int w = __ffs(m) - 1;
        const real rw = __shfl_sync(0xFFFFFFFFu, Rm, w);
        const int dw = __shfl_sync(0xFFFFFFFFu, d, w);
        a += dw < 0 ? (uint32_t)w : (uint32_t)w + 1u;
        if (dw < 0) {
          ok = false;
        } else if (dw == 1) {
          Rf = rw;
          b = 2 * b;
        } else {
          Ri = rw;
          b = 2 * b + 1;
        }
        break;
      }
      t *= (real)0.5;
    }
    if (!moved && lane == 0) fpt_write<F32>(A, it.k, ok, b, a, Ri, Rf, bin, r_lo, r_hi, attempts);
  }
}

// The levels from `l` on of one pair, by one block: the rounds of a level widen from 32 to
// blockDim.x attempts (a level that resolves quickly costs one warp's round) and the lowest-numbered
// decisive attempt of a round wins.  Stops after `budget` draws.  Shared scratch: s_win, s_rm, s_dec.
// Returns 0 (all levels done), 1 (failed: attempt bound or von Mises trials) or 2 (budget reached;
// the state is that of level l).
template <bool F32>
__device__ int block_levels(const FptArgs& A, uint64_t strm, int& l, fpt_real<F32>& Ri, fpt_real<F32>& Rf,
                            fpt_real<F32>& t, uint32_t& b, uint32_t& a, uint32_t budget, uint32_t* s_win, double* s_rm,
                            int* s_dec) {
  using real = fpt_real<F32>;
  const uint32_t tid = threadIdx.x, nt = blockDim.x, a0 = a;
#pragma unroll 1
  for (; l < A.levels; ++l) {
    uint32_t width = 32;
#pragma unroll 1
    for (;;) {
      if (a >= A.max_attempts) return 1;
      if (a - a0 >= budget) return 2;
      if (tid == 0) *s_win = 0xFFFFFFFFu;
      __syncthreads();
      const unsigned long long mine = (unsigned long long)a + tid;
      real Rm = 0;
      int d = 0;
      if (tid < width && mine < A.max_attempts) {
        d = fpt_attempt_p<F32>(A, l, strm, (uint32_t)mine, Ri, Rf, t, Rm);
        if (d != 0) atomicMin(s_win, tid);
      }
      __syncthreads();
      const uint32_t w = *s_win;
      if (w != 0xFFFFFFFFu && tid == w) {
        *s_rm = Rm;
        *s_dec = d;
      }
      __syncthreads();
      if (w == 0xFFFFFFFFu) {
        const uint32_t room = A.max_attempts - a;
        a += room < width ? room : width;
        width = width * 2 < nt ? width * 2 : nt;
        continue;
      }
      const int dw = *s_dec;
      a += dw < 0 ? w : w + 1;
      if (dw < 0) return 1;
      if (dw == 1) {
        Rf = (real)*s_rm;
        b = 2 * b;
      } else {
        Ri = (real)*s_rm;
        b = 2 * b + 1;
      }
      break;
    }
    t *= (real)0.5;
  }
  return 0;
}

// Phase 3: one block per pair that needs thousands of draws (work counter over the queue); a pair
// that has drawn `budget` more times since it was queued moves on to the grid phase with a fresh
// search record.
template <bool F32>
__global__ void __launch_bounds__(kFptBlockThreads) k_first_passage_block(
    const FptArgs A, const uint64_t* __restrict__ stream, uint32_t* __restrict__ bin, double* __restrict__ r_lo,
    double* __restrict__ r_hi, uint32_t* __restrict__ attempts, const FptItem* __restrict__ queue,
    FptItem* __restrict__ queue4, FptSearch* __restrict__ search, uint32_t* __restrict__ qctl, int words,
    uint32_t budget) {
  __shared__ uint32_t s_item, s_win;
  __shared__ double s_rm;
  __shared__ int s_dec;
  const uint32_t tid = threadIdx.x;
#pragma unroll 1
  for (;;) {
    if (tid == 0) s_item = atomicAdd(&qctl[words + kFptBlockNext], 1u);
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= *(volatile uint32_t*)&qctl[words + kFptBlockIn]) break;
    using real = fpt_real<F32>;
    const FptItem it = queue[item];
    const uint64_t strm = stream[it.k];
    real Ri = (real)it.Ri, Rf = (real)it.Rf, t = (real)it.t;
    uint32_t b = it.b, a = it.a;
    int l = (int)it.l;
    const int st = block_levels<F32>(A, strm, l, Ri, Rf, t, b, a, budget, &s_win, &s_rm, &s_dec);
    if (tid == 0) {
      if (st == 2) {
        const uint32_t j = atomicAdd(&qctl[words + kFptGridIn], 1u);
        queue4[j] = fpt_item(Ri, Rf, t, it.k, b, a, l);
        FptSearch z;
        z.next_chunk = 0;
        z.winner = 0xFFFFFFFFu;
        z.exited = 0;
        z.pad = 0;
        search[j] = z;
      } else {
        fpt_write<F32>(A, it.k, st == 0, b, a, Ri, Rf, bin, r_lo, r_hi, attempts);
      }
    }
    __syncthreads();
  }
}

// Phase 4: the very few pairs that need tens of thousands of draws at one level, each searched by
// a group of blocks (the grid split into kFptGridGroups groups).  Every block of a group visits the
// group's pairs in order; for a pair it takes chunks of blockDim.x
// consecutive attempts of the pair's current level from the pair's chunk counter and lowers the
// pair's winner (the lowest decisive attempt found) with atomicMin; it leaves the pair once a chunk
// starts at or past the winner.  Chunks are handed out in order, so when the last block leaves,
// every attempt below the winner has been tried and the winner is the attempt the serial loop
// would stop at; that block replays it and queues the pair's next level for the next round of
// phases 2-4.  No block waits for another.
template <bool F32>
__global__ void __launch_bounds__(kFptGridThreads) k_first_passage_grid(
    const FptArgs A, const uint64_t* __restrict__ stream, uint32_t* __restrict__ bin, double* __restrict__ r_lo,
    double* __restrict__ r_hi, uint32_t* __restrict__ attempts, const FptItem* __restrict__ queue,
    FptSearch* __restrict__ search, FptItem* __restrict__ queue_next, uint32_t* __restrict__ qctl, int words) {
  __shared__ uint32_t s_chunk, s_stop, s_last;
  const uint32_t tid = threadIdx.x, nt = blockDim.x;
  const uint32_t count = qctl[words + kFptGridIn];
  // the grid works in groups of blocks (block index mod groups); group g takes items g, g + groups, ...
  const uint32_t groups = gridDim.x >= 8 * kFptGridGroups ? kFptGridGroups : 1u;
  const uint32_t g = blockIdx.x % groups;
  const uint32_t gsize = gridDim.x / groups + (g < gridDim.x % groups ? 1u : 0u);
#pragma unroll 1
  for (uint32_t item = g; item < count; item += groups) {
    const FptItem it = queue[item];
    FptSearch* sr = &search[item];
    const uint64_t strm = stream[it.k];
#pragma unroll 1
    for (;;) {
      if (tid == 0) {
        const uint32_t c = atomicAdd(&sr->next_chunk, 1u);
        const unsigned long long st = (unsigned long long)it.a + (unsigned long long)c * nt;
        const uint32_t w = atomicAdd(&sr->winner, 0u);
        s_chunk = c;
        s_stop = (st >= w || st >= A.max_attempts) ? 1u : 0u;
      }
      __syncthreads();
      if (s_stop) break;
      const unsigned long long mine = (unsigned long long)it.a + (unsigned long long)s_chunk * nt + tid;
      if (mine < A.max_attempts) {
        fpt_real<F32> Rm;
        const int d = fpt_attempt_p<F32>(A, (int)it.l, strm, (uint32_t)mine, (fpt_real<F32>)it.Ri,
                                         (fpt_real<F32>)it.Rf, (fpt_real<F32>)it.t, Rm);
        if (d != 0) atomicMin(&sr->winner, (uint32_t)mine);
      }
      __syncthreads();
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(&sr->exited, 1u) == gsize - 1 ? 1u : 0u;
    __syncthreads();
    if (!s_last) continue;
    __threadfence();
    if (tid == 0) {
      const uint32_t win = *(volatile uint32_t*)&sr->winner;
      double Ri = it.Ri, Rf = it.Rf;
      uint32_t b = it.b, a = A.max_attempts;
      bool ok = false;
      if (win != 0xFFFFFFFFu) {           // replay the winning attempt
        fpt_real<F32> Rm;
        const int dw = fpt_attempt_p<F32>(A, (int)it.l, strm, win, (fpt_real<F32>)Ri, (fpt_real<F32>)Rf,
                                          (fpt_real<F32>)it.t, Rm);
        a = dw < 0 ? win : win + 1;
        ok = dw >= 0;
        if (dw == 1) {
          Rf = Rm;
          b = 2 * b;
        } else if (dw == 2) {
          Ri = Rm;
          b = 2 * b + 1;
        }
      }
      if (ok && (int)it.l + 1 < A.levels)
        queue_next[atomicAdd(&qctl[words + kFptRoundWords + kFptWarpIn], 1u)] =
            fpt_item(Ri, Rf, 0.5 * it.t, it.k, b, a, (int)it.l + 1);
      else
        fpt_write<F32>(A, it.k, ok, b, a, Ri, Rf, bin, r_lo, r_hi, attempts);
    }
    __syncthreads();
  }
}

template <bool F32>
static void launch_fpt(const FptArgs& A, const double* r0, const double* r, const uint64_t* stream, int64_t n,
                          uint32_t* bin, double* r_lo, double* r_hi, uint32_t* attempts, FptItem* warp_q[2],
                          FptItem* block_q, FptItem* grid_q, FptSearch* search, uint32_t* qctl, int device_sms,
                          cudaStream_t s) {
  auto clamp = [](int64_t g, int64_t gmax) { return (unsigned)(g > gmax ? gmax : (g < 1 ? 1 : g)); };
  const unsigned gw = clamp((n + 1023) / 1024, (int64_t)device_sms * 4);
  const unsigned gb = clamp((n + 4095) / 4096, (int64_t)device_sms * 2);
  cudaMemsetAsync(qctl, 0, kFptCtlWords * sizeof(uint32_t), s);
  // the FP32 lane phase needs 45 registers a thread, so it keeps twice the blocks resident
  k_first_passage<F32><<<clamp((n + 127) / 128, (int64_t)device_sms * (F32 ? 8 : 4)), 128, 0, s>>>(
      A, r0, r, stream, n, bin, r_lo, r_hi, attempts, warp_q[0], qctl, kFptBudget);
  // one round of phases 2-4 per level: a pair whose current level is hard goes through them once
  // more at a later level; a round with nothing queued ends at once
  for (int round = 0; round < A.levels; ++round) {
    const int w = kFptRound0 + round * kFptRoundWords;
    k_first_passage_warp<F32><<<gw, 128, 0, s>>>(A, stream, bin, r_lo, r_hi, attempts, warp_q[round & 1], w + kFptWarpIn,
                                            w + kFptWarpNext, block_q, w + kFptBlockIn, qctl, kFptWarpBudget);
    k_first_passage_block<F32><<<gb, kFptBlockThreads, 0, s>>>(A, stream, bin, r_lo, r_hi, attempts, block_q, grid_q,
                                                          search, qctl, w, kFptBlockBudget);
    k_first_passage_grid<F32><<<gb, kFptGridThreads, 0, s>>>(A, stream, bin, r_lo, r_hi, attempts, grid_q, search,
                                                        warp_q[(round + 1) & 1], qctl, w);
  }
}

void launch_first_passage(const FptArgs& A, const double* r0, const double* r, const uint64_t* stream, int64_t n,
                          uint32_t* bin, double* r_lo, double* r_hi, uint32_t* attempts, FptItem* warp_q[2],
                          FptItem* block_q, FptItem* grid_q, FptSearch* search, uint32_t* qctl, int device_sms,
                          cudaStream_t s) {
  if (A.f32)
    launch_fpt<true>(A, r0, r, stream, n, bin, r_lo, r_hi, attempts, warp_q, block_q, grid_q, search, qctl, device_sms, s);
  else
    launch_fpt<false>(A, r0, r, stream, n, bin, r_lo, r_hi, attempts, warp_q, block_q, grid_q, search, qctl, device_sms,
                      s);
}

}  // namespace rd
