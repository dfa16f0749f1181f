// First-passage refinement of encountered pairs (Appendix of the paper, "Relation to first-passage
// time simulation algorithms"): one thread per pair bisects the step `levels` times.
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

__device__ __forceinline__ double fpt_p_enc(const FptArgs& A, int level, double R, double R0, double tau) {
  return A.dim == 3 ? p_enc3(R, R0, 1.0 / tau) : fpt_p_enc2(A.lv[level].nodes, A.lv[level].n_nodes, A.ser, R, R0, tau);
}

__global__ void __launch_bounds__(128) k_first_passage(const FptArgs A, const double* __restrict__ r0,
                                                       const double* __restrict__ r,
                                                       const uint64_t* __restrict__ stream, int64_t n,
                                                       uint32_t* __restrict__ bin, double* __restrict__ r_lo,
                                                       double* __restrict__ r_hi, uint32_t* __restrict__ attempts) {
  const double inv_sigma = 1.0 / A.sigma;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t strm = stream[k];
    double Ri = r0[k] * inv_sigma, Rf = r[k] * inv_sigma, t = A.tau;
    uint32_t b = 0, a = 0;
    bool ok = true;
#pragma unroll 1
    for (int l = 0; l < A.levels && ok; ++l) {
#pragma unroll 1
      for (;;) {
        if (a >= A.max_attempts) {
          ok = false;
          break;
        }
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
          omc = -log1p((1.0 - u_dir) * expm1(-2.0 * kappa)) / kappa;
          sn = sqrt(omc * (2.0 - omc));
        } else if (!vm2_draw(A, kappa, strm, a, omc, sn)) {
          ok = false;
          break;
        }
        const double sd = sqrt(0.5 * t);
        const double m0 = 0.5 * (Ri + Rf * (1.0 - omc)) + sd * x0;
        const double m1 = 0.5 * Rf * sn + sd * x1;
        const double m2 = sd * x2;
        const double Rm = sqrt(m0 * m0 + m1 * m1 + m2 * m2);
        ++a;
        if (u_e1 < fpt_p_enc(A, l, Rm, Ri, 0.5 * t)) {
          Rf = Rm;
          b = 2 * b;
          break;
        }
        if (u_e2 < fpt_p_enc(A, l, Rf, Rm, 0.5 * t)) {
          Ri = Rm;
          b = 2 * b + 1;
          break;
        }
      }
      t *= 0.5;
    }
    bin[k] = ok ? b : 0xFFFFFFFFu;
    if (r_lo) r_lo[k] = ok ? Ri * A.sigma : __longlong_as_double(0x7FF8000000000000ll);
    if (r_hi) r_hi[k] = ok ? Rf * A.sigma : __longlong_as_double(0x7FF8000000000000ll);
    if (attempts) attempts[k] = a;
  }
}

void launch_first_passage(const FptArgs& A, const double* r0, const double* r, const uint64_t* stream, int64_t n,
                          uint32_t* bin, double* r_lo, double* r_hi, uint32_t* attempts, int max_grid,
                          cudaStream_t s) {
  int64_t g = (n + 127) / 128;
  if (g > max_grid) g = max_grid;
  if (g < 1) g = 1;
  k_first_passage<<<(unsigned)g, 128, 0, s>>>(A, r0, r, stream, n, bin, r_lo, r_hi, attempts);
}

}  // namespace rd
