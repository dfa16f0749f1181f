// Host runtime behind the C ABI of include/rd.h: configuration checks, derived per-pair
// parameters, cell grids, device buffers, CUDA-graph capture of two steps, state transfer.
#include <map>
#include <mutex>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "rd_gf2d.cuh"
#include "rd_kernels.h"

using namespace rd;

namespace {
thread_local int g_last_cuda_error = 0;

int cuda_fail(cudaError_t e) {
  g_last_cuda_error = (int)e;
  return RD_ECUDA;
}
}  // namespace

#define RD_CUDA(call)                        \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

constexpr int kHistoryLen = 1 << 16;   // steps kept by the per-step count history
// the autotuner tries the fused launch up to this particle capacity (at 2 resident blocks per SM
// the fused launch has fewer warps per SM than the separate sweep)
constexpr int64_t kFusedMaxCapacity = (int64_t)1 << 22;

struct rd_handle {
  rd_config cfg;
  std::vector<rd_replica> reps_host;
  std::vector<RepDev> reps_init;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  DevParams hp;
  StepLaunch L;
  void* xbuf[2] = {nullptr, nullptr};
  uint32_t* idbuf[2] = {nullptr, nullptr};
  int cur = 0;
  size_t vsize = 32;
  std::vector<std::pair<void*, size_t>> allocs;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  KernelTimer timer;
  bool time_next = false;
  std::vector<std::pair<std::string, float>> last_times;
  std::vector<double> factors;       // cell-edge factors (one, or the autotuner's candidates)
  double tuned_ms = 0.0;
  double factor = 1.0;               // cell-edge factor in use
  int reach = 1;                     // stencil reach of the cell sweep (2: 2D cells of half a cut-off)
  // staging of rd_set_state / rd_get_state (allocated on first use, capacity-sized)
  double* st_x = nullptr;
  int32_t* st_sp = nullptr;
  uint32_t* st_id = nullptr;
  int32_t* st_rep = nullptr;
  uint32_t* st_cnt = nullptr;        // per replica: particles, largest id + 1, next_id in
  uint32_t* st_maxid = nullptr;
  uint32_t* st_next = nullptr;
  int32_t* st_err = nullptr;
  // Weber nodes of the first-passage refinement's half intervals (2D), per rule and level
  std::vector<std::pair<const void*, int>> fpt_nodes[RD_MAX_PAIRS];
  // work queues of the refinement's later phases (capacity in pairs each), search records, counters
  FptItem* fpt_queue = nullptr;
  int64_t fpt_qcap = 0;
  uint32_t* fpt_qctl = nullptr;
};

static void* dev_alloc(rd_handle* h, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (h->cfg.allocator.alloc) {
    p = h->cfg.allocator.alloc(bytes, (void*)h->stream, h->cfg.allocator.ctx);
  } else if (cudaMallocAsync(&p, bytes, h->stream) != cudaSuccess) {
    p = nullptr;
  }
  if (p) h->allocs.emplace_back(p, bytes);
  return p;
}

// Returns one allocation of dev_alloc (stream-ordered: work already queued on the stream that uses
// it runs first).
static void dev_release(rd_handle* h, void* p) {
  for (size_t i = 0; i < h->allocs.size(); ++i) {
    if (h->allocs[i].first != p) continue;
    if (h->cfg.allocator.release)
      h->cfg.allocator.release(p, h->allocs[i].second, (void*)h->stream, h->cfg.allocator.ctx);
    else if (!h->cfg.allocator.alloc)
      cudaFreeAsync(p, h->stream);
    h->allocs.erase(h->allocs.begin() + i);
    return;
  }
}

static void free_all(rd_handle* h) {
  for (auto& a : h->allocs) {
    if (h->cfg.allocator.release)
      h->cfg.allocator.release(a.first, a.second, (void*)h->stream, h->cfg.allocator.ctx);
    else if (!h->cfg.allocator.alloc)
      cudaFreeAsync(a.first, h->stream);
  }
  h->allocs.clear();
}

// Streaming multiprocessors of the current device, cached per device (grid caps of the launches).
static int device_sms() {
  static std::mutex mu;
  static std::map<int, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
  cache[dev] = sms;
  return sms;
}

static StepLaunch launch_for(rd_handle* h, int cur) {
  StepLaunch L = h->L;
  L.x_cur = h->xbuf[cur];
  L.x_next = h->xbuf[1 - cur];
  L.id_cur = h->idbuf[cur];
  L.id_next = h->idbuf[1 - cur];
  return L;
}

static double max_cutoff(const rd_config& c) {
  double rc = 0.0;
  for (int k = 0; k < c.n_pairs; ++k) {
    const rd_pair_rule& p = c.pairs[k];
    if (p.bc == RD_BC_NONE) continue;
    rc = std::max(rc, p.sigma + c.c_cut * std::sqrt(2.0 * (c.D[p.s1] + c.D[p.s2]) * c.dt));
  }
  return rc;
}

static int validate(const rd_config* c) {
  if (!c || (c->dim != 2 && c->dim != 3)) return RD_EINVAL;
  if (c->precision != RD_FP64 && c->precision != RD_MIXED) return RD_EINVAL;
  if (c->n_species < 1 || c->n_species > RD_MAX_SPECIES) return RD_EINVAL;
  if (c->n_pairs < 0 || c->n_pairs > RD_MAX_PAIRS || c->n_decays < 0 || c->n_decays > RD_MAX_DECAYS) return RD_EINVAL;
  if (c->n_replicas < 1 || c->n_replicas >= (1 << 24) || !c->replicas) return RD_EINVAL;
  if (!(c->dt > 0.0) || !(c->c_cut >= 0.0)) return RD_EINVAL;
  if (c->block_size != 0 && (c->block_size < 32 || c->block_size > 256 || c->block_size % 32 != 0)) return RD_EINVAL;
  if (c->sweep_split < 0 || c->sweep_split > 2) return RD_EINVAL;
  if (c->cell_reach < 0 || c->cell_reach > 2 || (c->cell_reach == 2 && c->dim != 2)) return RD_EINVAL;
  if (c->step_launch < 0 || c->step_launch > 2 || (c->force_paths & ~3) != 0) return RD_EINVAL;
  if (c->angle_mode < 0 || c->angle_mode > 1) return RD_EINVAL;
  double L_min = 1e300;
  for (int r = 0; r < c->n_replicas; ++r) L_min = std::min(L_min, c->replicas[r].L);
  for (int s = 0; s < c->n_species; ++s) {
    if (!(c->D[s] >= 0.0)) return RD_EINVAL;
    // the drift step wraps once: its displacement per step stays below half a box
    for (int d = 0; d < 3; ++d)
      if (!std::isfinite(c->drift[s][d]) || !(std::fabs(c->drift[s][d] * c->dt) < 0.5 * L_min)) return RD_EINVAL;
  }
  for (int k = 0; k < c->n_pairs; ++k) {
    const rd_pair_rule& p = c->pairs[k];
    if (p.s1 < 0 || p.s1 >= c->n_species || p.s2 < 0 || p.s2 >= c->n_species) return RD_EINVAL;
    if (p.bc < RD_BC_NONE || p.bc > RD_BC_RAD) return RD_EINVAL;
    if (p.product < -1 || p.product >= c->n_species) return RD_EINVAL;
    if (p.bc != RD_BC_NONE && !(p.sigma > 0.0)) return RD_EINVAL;
    if (p.bc != RD_BC_NONE && !(c->D[p.s1] + c->D[p.s2] > 0.0)) return RD_EINVAL;
    if (p.bc == RD_BC_RAD && !(p.ka >= 0.0)) return RD_EINVAL;
    for (int q = 0; q < k; ++q) {
      const rd_pair_rule& o = c->pairs[q];
      if ((o.s1 == p.s1 && o.s2 == p.s2) || (o.s1 == p.s2 && o.s2 == p.s1)) return RD_EINVAL;
    }
  }
  for (int k = 0; k < c->n_decays; ++k) {
    const rd_decay& d = c->decays[k];
    if (d.parent < 0 || d.parent >= c->n_species || d.n_products < 0 || d.n_products > 2 || !(d.kd >= 0.0))
      return RD_EINVAL;
    for (int m = 0; m < d.n_products; ++m)
      if (d.products[m] < 0 || d.products[m] >= c->n_species) return RD_EINVAL;
  }
  const double rc = max_cutoff(*c);
  for (int r = 0; r < c->n_replicas; ++r) {
    if (!(c->replicas[r].L > 0.0)) return RD_EINVAL;
    if (rc > 0.0 && !(rc < 0.5 * c->replicas[r].L)) return RD_EINVAL;  // unique minimum image
    for (int s = 0; s < c->n_species; ++s)
      if (c->replicas[r].n_init[s] < 0) return RD_EINVAL;
  }
  return RD_OK;
}

static void gauss_legendre16(double* x, double* w);

static void derive_params(rd_handle* h) {
  const rd_config& c = h->cfg;
  DevParams& P = h->hp;
  std::memset(&P, 0, sizeof P);
  // 16-point Gauss-Legendre rule (2D quadratures and the exact angle law)
  double gx[16], gw[16];
  gauss_legendre16(gx, gw);
  for (int i = 0; i < 16; ++i) {
    P.gl16[i] = gx[i];
    P.gl16[16 + i] = gw[i];
  }
  P.dim = c.dim;
  P.n_species = c.n_species;
  P.precision = c.precision;
  P.n_replicas = c.n_replicas;
  P.n_pairs = c.n_pairs;
  P.n_decays = c.n_decays;
  P.match_max_rounds = 4096;
  P.match_single_max = (c.force_paths & 1) ? 0u : 2048u;
  P.match_smem_max = (c.force_paths & 2) ? 0u : 256u;
  P.angle_mode = c.angle_mode;
  P.dt = c.dt;
  P.seed_lo = (uint32_t)(c.seed & 0xFFFFFFFFu);
  P.seed_hi = (uint32_t)(c.seed >> 32);
  for (int s = 0; s < c.n_species; ++s) {
    P.D[s] = c.D[s];
    P.D_f[s] = (float)c.D[s];
    P.ell[s] = std::sqrt(2.0 * c.D[s] * c.dt);
    P.ell_f[s] = (float)P.ell[s];
  }
  for (int a = 0; a < kMaxSpecies; ++a)
    for (int b = 0; b < kMaxSpecies; ++b) P.pair_of[a][b] = -1;
  for (int k = 0; k < c.n_pairs; ++k) {
    const rd_pair_rule& p = c.pairs[k];
    PairDev& q = P.pairs[k];
    q.bc = p.bc;
    q.product = p.product;
    q.s1 = p.s1;
    q.s2 = p.s2;
    if (p.bc == RD_BC_NONE) continue;
    q.sigma = p.sigma;
    q.Drel = c.D[p.s1] + c.D[p.s2];
    q.tau = q.Drel * c.dt / (p.sigma * p.sigma);
    q.inv_tau = 1.0 / q.tau;
    q.s = std::sqrt(q.tau);
    q.h = c.dim == 3 ? p.ka / (4.0 * kPi * p.sigma * q.Drel) : p.ka / (2.0 * kPi * q.Drel);
    q.alpha = 1.0 + q.h;
    const double rc = p.sigma + c.c_cut * std::sqrt(2.0 * q.Drel * c.dt);
    q.rcut2 = rc * rc;
    q.sigma_f = (float)p.sigma;
    q.inv_sigma_f = (float)(1.0 / p.sigma);
    q.inv_tau_f = (float)q.inv_tau;
    q.rcut2_f = (float)q.rcut2;
    P.rcut2_max = std::max(P.rcut2_max, q.rcut2);
    P.rcut2_max_f = std::max(P.rcut2_max_f, q.rcut2_f);
    q.s_f = (float)q.s;
    q.alpha_f = (float)q.alpha;
    P.pair_of[p.s1][p.s2] = (int8_t)k;
    P.pair_of[p.s2][p.s1] = (int8_t)k;
    P.binned_mask |= (1u << p.s1) | (1u << p.s2);
  }
  for (int sp = 0; sp < c.n_species; ++sp)
    for (int d = 0; d < 3; ++d) {
      P.drift_dx[sp][d] = d < c.dim ? c.drift[sp][d] * c.dt : 0.0;
      P.drift_dx_f[sp][d] = (float)P.drift_dx[sp][d];
      if (P.drift_dx[sp][d] != 0.0) P.has_drift = 1;
    }
  for (int k = 0; k < c.n_decays; ++k) {
    const rd_decay& d = c.decays[k];
    DecayDev& q = P.decays[k];
    q.parent = d.parent;
    q.n_products = d.n_products;
    q.p0 = d.n_products > 0 ? d.products[0] : -1;
    q.p1 = d.n_products > 1 ? d.products[1] : -1;
    q.kd = d.kd;
    q.sigma_place = d.sigma_place;
  }
  for (int s = 0; s < c.n_species; ++s) {
    double kt = 0.0;
    for (int k = 0; k < c.n_decays; ++k)
      if (c.decays[k].parent == s) kt += c.decays[k].kd;
    P.ktot[s] = kt;
    P.p_uni[s] = -std::expm1(-kt * c.dt);
    // U = (m + 1/2) 2^-52 < p  <=>  m < ceil(p 2^52 - 1/2); p 2^52 - 1/2 is exact for p < 1
    const double T = std::ldexp(P.p_uni[s], 52) - 0.5;
    P.uni_thr[s] = T <= 0.0 ? 0ull : (unsigned long long)std::ceil(T);
  }
}


// ------------------------------------------------------------------------------------------------
// 2D tables: Gauss-Legendre nodes (Newton on the Legendre recurrence), the Weber quadrature nodes
// of each 2D pair type (Bessel values at the abscissas precomputed, as Section 4.1 suggests), and
// the coefficient series of the small-time expansion.
// ------------------------------------------------------------------------------------------------
static void gauss_legendre16(double* x, double* w) {
  const int n = 16;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), d = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      d = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / d;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * d * d);
  }
}

static std::vector<WeberNode> weber_nodes(double tau, double h, double Rmax) {
  double gx[16], gw[16];
  gauss_legendre16(gx, gw);
  const double T = std::pow(60.0 / tau, 0.25);           // e^{-tau x^2} < e^{-60} beyond x = T^2
  const int panels = 6 + (int)std::ceil(Rmax * T * T / 2.5);
  std::vector<WeberNode> nodes;
  nodes.reserve(panels * 16);
  const double hw = 0.5 * T / panels;
  for (int p = 0; p < panels; ++p) {
    const double mid = (2 * p + 1) * hw;
    for (int i = 0; i < 16; ++i) {
      const double t = mid + hw * gx[i], x = t * t;
      WeberNode nd;
      nd.x = x;
      nd.w = gw[i] * hw * 2.0 * t * x * std::exp(-tau * x * x) / (2.0 * kPi);
      const double J0 = ::j0(x), Y0 = ::y0(x), J1 = ::j1(x), Y1 = ::y1(x);
      const double al[3] = {J0, x * J1, x * J1 + h * J0};
      const double be[3] = {Y0, x * Y1, x * Y1 + h * Y0};
      for (int k = 0; k < 3; ++k) {
        const double nr = std::sqrt(al[k] * al[k] + be[k] * be[k]);
        nd.a[k] = al[k] / nr;
        nd.b[k] = be[k] / nr;
      }
      nodes.push_back(nd);
    }
  }
  return nodes;
}

// a_k(nu) of the large-argument expansions of I_nu, K_nu
static double ak_host(int k, double nu) {
  double v = 1.0;
  for (int j = 1; j <= k; ++j) v *= (4.0 * nu * nu - (2.0 * j - 1.0) * (2.0 * j - 1.0)) / (8.0 * j);
  return v;
}

static Series2D series_coeffs(double h) {
  Series2D S;
  const int n = kSeriesTerms;
  double A0[kSeriesTerms + 1], A0m[kSeriesTerms + 1], A1[kSeriesTerms + 1], A1m[kSeriesTerms + 1];
  for (int k = 0; k <= n; ++k) {
    const double sg = (k % 2) ? -1.0 : 1.0;
    A0[k] = ak_host(k, 0.0);
    A0m[k] = sg * A0[k];
    A1[k] = ak_host(k, 1.0);
    A1m[k] = sg * A1[k];
    S.a0[k] = A0[k];
  }
  for (int slot = 0; slot < 3; ++slot) {
    double num[kSeriesTerms + 1], den[kSeriesTerms + 1];
    for (int k = 0; k <= n; ++k) {
      if (slot == 0) {            // absorbing: I0/K0
        num[k] = A0m[k];
        den[k] = A0[k];
      } else {                    // reflective (h = 0) / radiation: (I1 - h y I0)/(K1 + h y K0)
        const double hh = slot == 2 ? h : 0.0;
        num[k] = A1m[k] - (k ? hh * A0m[k - 1] : 0.0);
        den[k] = A1[k] + (k ? hh * A0[k - 1] : 0.0);
      }
    }
    for (int k = 0; k <= n; ++k) {    // series division
      double v = num[k];
      for (int j = 1; j <= k; ++j) v -= den[j] * S.ratio[slot][k - j];
      S.ratio[slot][k] = v / den[0];
    }
  }
  return S;
}

// Builds the 2D data of every 2D pair type into device memory from `alloc`, patching hp.
constexpr double kSeriesHSqrtTau = 0.3;   // series limit of the radiation bracket in 2D

template <class Alloc>
static bool build_2d(const rd_config& c, DevParams& hp, Alloc alloc) {
  if (c.dim != 2) return true;
  for (int k = 0; k < c.n_pairs; ++k) {
    PairDev& q = hp.pairs[k];
    if (c.pairs[k].bc == RD_BC_NONE) continue;
    // small-time series for tau <= tau_s; for the radiation bracket only while h sqrt(tau) <= 0.3
    // (its coefficients grow like powers of h), else the exact Weber quadrature
    q.series2d = q.tau <= c.tau_s ? 1 : 0;
    q.series2d_rad = q.series2d && q.h * std::sqrt(q.tau) <= kSeriesHSqrtTau ? 1 : 0;
    Series2D S = series_coeffs(q.h);
    void* ds = alloc(sizeof(Series2D));
    if (!ds || cudaMemcpy(ds, &S, sizeof S, cudaMemcpyHostToDevice) != cudaSuccess) return false;
    q.ser = (const Series2D*)ds;
    if (!q.series2d || (c.pairs[k].bc == RD_BC_RAD && !q.series2d_rad)) {
      const double Rmax = std::sqrt(q.rcut2) / q.sigma + 13.0 * q.s + 3.0;
      std::vector<WeberNode> nodes = weber_nodes(q.tau, q.h, Rmax);
      void* dn = alloc(nodes.size() * sizeof(WeberNode));
      if (!dn || cudaMemcpy(dn, nodes.data(), nodes.size() * sizeof(WeberNode), cudaMemcpyHostToDevice) != cudaSuccess)
        return false;
      q.nodes = (const WeberNode*)dn;
      q.n_nodes = (int)nodes.size();
    }
  }
  return true;
}

// FP32 lookup tables of the mixed step (p_reac in 2D and 3D; F = p_enc e^{d d0/tau} and
// -ln(tail) in 2D), spacing 0.025 min(sqrt(tau), 1) over d0 up to the cut-off and d up to the propagator's
// support (d0 + 13 sqrt(tau)), built in FP64 on the device.
template <class Alloc>
static cudaError_t build_tables(rd_handle* h, Alloc alloc) {
  const rd_config& c = h->cfg;
  if (c.precision != RD_MIXED) return cudaSuccess;
  for (int k = 0; k < c.n_pairs; ++k) {
    PairDev& q = h->hp.pairs[k];
    if (c.pairs[k].bc == RD_BC_NONE) continue;
    const double hstep = 0.025 * std::min(q.s, 1.0);
    const double d0max = std::sqrt(q.rcut2) / q.sigma - 1.0 + hstep;
    const double dmax = d0max + 13.0 * q.s + 2.0 * hstep;
    const int n0 = (int)std::ceil(d0max / hstep) + 4, n1 = (int)std::ceil(dmax / hstep) + 4;
    // the inverse table's second axis: t = sqrt(-ln U) up to 4.2 (U >= 2^-24 needs t <= 4.08)
    const double hinv = 0.025;
    const int ninv = (int)std::ceil(4.2 / hinv) + 4;
    auto make = [&](int kind, Tab2& T, int m1, double h1, const Tab2* fwd) -> cudaError_t {
      const size_t bytes = (size_t)n0 * m1 * sizeof(float);
      float* t = (float*)alloc(bytes);
      float4* q4 = (float4*)alloc(4 * bytes);
      double* tot = (double*)alloc((size_t)n0 * sizeof(double));
      if (!t || !q4 || !tot) return cudaErrorMemoryAllocation;
      launch_build_table(h->L.P, k, kind, t, q4, n0, m1, hstep, h1, tot, fwd, device_sms(), h->stream);
      T.v = t;
      T.q = q4;
      T.n0 = n0;
      T.n1 = m1;
      T.h = (float)hstep;
      T.inv_h = (float)(1.0 / hstep);
      T.h1 = (float)h1;
      T.inv_h1 = (float)(1.0 / h1);
      return cudaGetLastError();
    };
    cudaError_t e = cudaSuccess;
    if (c.pairs[k].bc == RD_BC_RAD) e = make(0, q.tab_preac, n1, hstep, nullptr);
    if (e == cudaSuccess && c.dim == 2) e = make(1, q.tab_penc, n1, hstep, nullptr);
    if (e == cudaSuccess && c.dim == 2) e = make(2, q.tab_tail, n1, hstep, nullptr);
    if (e == cudaSuccess && c.pairs[k].bc != RD_BC_ABS)
      e = make(3, q.tab_inv, ninv, hinv, c.dim == 2 ? &q.tab_tail : nullptr);
    if (e == cudaSuccess && c.angle_mode == 0 && c.pairs[k].bc != RD_BC_ABS) {
      // conditional angle law of the exact propagation: spacing min(s, 1) / 10 in R0 and R' (the
      // law varies on the scale s, and near contact on the contact radius); R0 up to the cut-off,
      // R' up to 10 s beyond it (the radial law's tail at U = 2^-24 reaches about 8.2 s); at most
      // 150 000 nodes
      const double a0max = std::sqrt(q.rcut2) / q.sigma - 1.0, a1max = a0max + 10.0 * q.s;
      double ha = 0.1 * std::min(q.s, 1.0);
      int m0 = 0, m1 = 0;
      for (;;) {
        m0 = (int)std::ceil(a0max / ha) + 3;
        m1 = (int)std::ceil(a1max / ha) + 3;
        if ((int64_t)m0 * m1 <= 150000) break;
        ha *= 1.25;
      }
      float* t = (float*)alloc((size_t)m0 * m1 * kAngTabStride * sizeof(float));
      if (!t) return cudaErrorMemoryAllocation;
      launch_build_ang_table(h->L.P, c.dim, q.tau, ha, m0, m1, t, device_sms(), h->stream);
      AngTab& A = q.tab_ang;
      A.v = t;
      A.n0 = m0;
      A.n1 = m1;
      A.h = (float)ha;
      A.inv_h = (float)(1.0 / ha);
      A.d0max = (float)((m0 - 3) * ha);
      A.d1max = (float)((m1 - 3) * ha);
      A.inv_2tau = (float)(0.5 / q.tau);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return e;
  return cudaMemcpy((void*)h->L.P, &h->hp, sizeof(DevParams), cudaMemcpyHostToDevice);
}

// Blocks of the cooperative matching launch for the current device, cached per device.
static int match_grid_for_current_device() {
  static std::mutex mu;
  static std::map<int, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  const int g = match_grid_size(device_sms());
  cache[dev] = g;
  return g;
}

// Cell-edge factor for about 0.25 interacting particles per cell (between 1 and 4 cut-offs) at the
// given number density of binned particles.  The sweep walks five contiguous row ranges per
// particle whatever the cell size, so its cost grows with the particles those rows hold (15 cells
// x density) while the cell scan grows with the number of cells; 0.25 per cell balances the two.
static double density_edge_factor(double nb, double volume, int dim, double rc) {
  if (nb <= 0.0 || rc <= 0.0 || volume <= 0.0) return 1.0;
  const double per_cell = nb / volume * std::pow(rc, (double)dim);
  const double f = std::pow(0.25 / per_cell, 1.0 / dim);
  return std::min(4.0, std::max(1.0, f));
}

// Cell grid of every replica.  factor > 0: cell edge = factor x the largest cut-off / reach in every
// replica; factor < 0: each replica's own density-based edge factor times -factor (never below one
// cut-off), so that replicas of very different concentrations each get a suitable grid.  A grid is
// coarsened until it has at most 4 cells per interacting particle (+64).  Fills the grid fields of
// out[r].
static int64_t layout_cells(const rd_config& c, const std::vector<rd_replica>& reps, uint32_t binned_mask,
                            double rc, double factor, int reach, std::vector<RepDev>& out) {
  int64_t total = 0;
  for (size_t r = 0; r < reps.size(); ++r) {
    const rd_replica& rp = reps[r];
    RepDev& d = out[r];
    int64_t nb = 0;
    for (int s = 0; s < c.n_species; ++s)
      if ((binned_mask >> s) & 1u) nb += rp.n_init[s];
    double f = factor > 0.0 ? factor
                            : std::max(1.0, -factor * density_edge_factor((double)nb, std::pow(rp.L, (double)c.dim),
                                                                          c.dim, rc));
    int64_t cells = 1;
    for (int attempt = 0; attempt < 64; ++attempt) {
      cells = 1;
      for (int a = 0; a < 3; ++a) {
        int n = 1;
        if (a < c.dim && rc > 0.0) {
          // cell edge >= r_cut / reach; the stencil needs 2 reach + 1 distinct cells per axis
          const double m = std::floor(rp.L * reach / (rc * f * (1.0 + 1e-6)));
          n = m >= 2.0 * reach + 1.0 ? (int)std::min(m, 4096.0) : 1;
        }
        d.nc[a] = n;
        d.inv_edge[a] = n / rp.L;
        d.inv_edge_f[a] = (float)d.inv_edge[a];
        cells *= n;
      }
      if (cells <= 4 * nb + 64) break;
      f *= 1.25;
    }
    d.cell_base = total;
    total += cells;
  }
  return total;
}

// Cell-edge choice: a fixed factor (> 0) or the per-replica density rule with a multiplier (< 0).
static cudaError_t apply_factor(rd_handle* h, double factor) {
  const rd_config& c = h->cfg;
  std::vector<RepDev> reps(c.n_replicas);
  cudaError_t e = cudaMemcpy(reps.data(), h->L.reps, reps.size() * sizeof(RepDev), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  h->L.total_cells = layout_cells(c, h->reps_host, h->hp.binned_mask, max_cutoff(c), factor, h->reach, reps);
  return cudaMemcpy(h->L.reps, reps.data(), reps.size() * sizeof(RepDev), cudaMemcpyHostToDevice);
}

// Autotuner: times a few steps for each candidate cell-edge choice and resolution block size on
// the initial state, keeps the fastest, and restores the state (the scan epoch stays monotonic).
static cudaError_t autotune(rd_handle* h) {
  const size_t xbytes = (size_t)h->L.cap_particles * h->vsize, ibytes = (size_t)h->L.cap_particles * 4;
  const size_t rbytes = (size_t)h->cfg.n_replicas * sizeof(RepDev);
  void *sx = nullptr, *si = nullptr;
  cudaError_t e = cudaMalloc(&sx, xbytes);
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&si, ibytes);
  if (e != cudaSuccess) {
    cudaFree(sx);
    return e;
  }
  DevCtl ctl0;
  std::vector<RepDev> reps0(h->cfg.n_replicas);
  cudaMemcpy(&ctl0, h->L.ctl, sizeof ctl0, cudaMemcpyDeviceToHost);
  cudaMemcpy(reps0.data(), h->L.reps, rbytes, cudaMemcpyDeviceToHost);
  cudaMemcpy(sx, h->xbuf[0], xbytes, cudaMemcpyDeviceToDevice);
  cudaMemcpy(si, h->idbuf[0], ibytes, cudaMemcpyDeviceToDevice);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  auto restore = [&]() {
    DevCtl now;
    cudaMemcpy(&now, h->L.ctl, sizeof now, cudaMemcpyDeviceToHost);
    DevCtl back = ctl0;
    back.epoch = now.epoch;          // flags written by the trial steps must not look current later
    cudaMemcpy(h->L.ctl, &back, sizeof back, cudaMemcpyHostToDevice);
    // segments and ids go back to the saved state; the cell grid stays the one being timed, so
    // that it always matches L.total_cells
    std::vector<RepDev> cur(reps0.size());
    cudaMemcpy(cur.data(), h->L.reps, rbytes, cudaMemcpyDeviceToHost);
    for (size_t r = 0; r < cur.size(); ++r) {
      cur[r].beg = reps0[r].beg;
      cur[r].end = reps0[r].end;
      cur[r].next_id = reps0[r].next_id;
    }
    cudaMemcpy(h->L.reps, cur.data(), rbytes, cudaMemcpyHostToDevice);
    cudaMemcpy(h->xbuf[0], sx, xbytes, cudaMemcpyDeviceToDevice);
    cudaMemcpy(h->idbuf[0], si, ibytes, cudaMemcpyDeviceToDevice);
    h->cur = 0;
  };
  auto trial = [&]() -> float {
    StepLaunch L = launch_for(h, 0);
    launch_step(L, h->stream, nullptr);   // warm-up
    launch_step(launch_for(h, 1), h->stream, nullptr);
    cudaEventRecord(a, h->stream);
    for (int k = 0; k < 3; ++k) {
      launch_step(launch_for(h, 0), h->stream, nullptr);
      launch_step(launch_for(h, 1), h->stream, nullptr);
    }
    cudaEventRecord(b, h->stream);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    restore();
    return ms;
  };
  double best_f = h->factors[0];
  float best = 1e30f;
  const int block0 = h->L.block;
  for (double f : h->factors) {
    apply_factor(h, f);
    const float ms = std::min(trial(), trial());
    if (ms < best) {
      best = ms;
      best_f = f;
    }
  }
  apply_factor(h, best_f);
  h->factor = best_f;
  // threads per block of the particle-parallel kernels (prepare, scatter, compaction)
  int best_block = block0;
  for (int bs : {128, 256}) {
    if (bs == block0) continue;
    h->L.block = bs;
    const float ms = std::min(trial(), trial());
    if (ms < best) {
      best = ms;
      best_block = bs;
    }
  }
  h->L.block = best_block;
  // one thread per (particle, stencil row) in the sweep, for small systems
  const int rows = h->cfg.dim == 3 ? 5 : (h->reach == 2 ? 3 : 2);
  if (h->cfg.sweep_split == 0 && (double)h->L.cap_particles * rows < 4.0e9) {
    h->L.sweep_split = rows;
    const int g_split = fused_grid_size(h->L, device_sms());
    const int fused0 = h->L.fused;
    h->L.fused_grid = g_split;
    if (g_split < 1) h->L.fused = 0;
    const float ms = std::min(trial(), trial());
    if (ms < best) {
      best = ms;
    } else {
      h->L.sweep_split = 1;
      h->L.fused = fused0;
      h->L.fused_grid = fused_grid_size(h->L, device_sms());
    }
  }
  // one fused launch per step or one launch per kernel (bit-identical results either way)
  // (not with the FP64 step's exact angle pass, which can take far longer than a grid barrier
  // waits: about a millisecond of FP64 work per pair)
  if (h->cfg.step_launch == 0 && h->L.fused_grid >= 1 && h->L.cap_particles <= kFusedMaxCapacity &&
      !(h->cfg.angle_mode == 0 && h->cfg.precision == RD_FP64)) {
    h->L.fused = !h->L.fused;
    const float ms = std::min(trial(), trial());
    if (ms < best)
      best = ms;
    else
      h->L.fused = !h->L.fused;
  }
  h->tuned_ms = best / 6.0;
  restore();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sx);
  cudaFree(si);
  return cudaGetLastError();
}

extern "C" {

const char* rd_strerror(int status) {
  switch (status) {
    case RD_OK: return "ok";
    case RD_EINVAL: return "invalid argument";
    case RD_ENOMEM: return "device allocation failed";
    case RD_ECAPACITY: return "device list or particle capacity exceeded; step not committed";
    case RD_ETIMEOUT: return "conflict resolution did not finish within its iteration bound";
    case RD_ECUDA: return "CUDA runtime error";
    case RD_ENOTREADY: return "not available for this configuration";
    default: return "unknown status";
  }
}

int rd_last_cuda_error(void) { return g_last_cuda_error; }

int rd_init(const rd_config* cfg, void* stream, rd_handle** out) {
  if (!out) return RD_EINVAL;
  *out = nullptr;
  int v = validate(cfg);
  if (v != RD_OK) return v;
  rd_handle* h = new rd_handle();
  h->cfg = *cfg;
  if (h->cfg.c_cut == 0.0) h->cfg.c_cut = 5.0;
  if (h->cfg.tau_s == 0.0) h->cfg.tau_s = 0.01;
  const rd_config& c = h->cfg;
  h->reps_host.assign(cfg->replicas, cfg->replicas + cfg->n_replicas);
  h->cfg.replicas = nullptr;
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return cuda_fail(cudaGetLastError());
    }
    h->own_stream = true;
  }
  derive_params(h);
  const bool mixed = c.precision == RD_MIXED;
  h->vsize = mixed ? 16 : 32;

  // cell grids: edge >= the largest cut-off (with a relative margin against rounding); the edge
  // factor is explicit (cell_factor_x100 > 0), density-based (0) or autotuned (< 0)
  const double rc = max_cutoff(c);
  const uint32_t bmask = h->hp.binned_mask;
  // stencil reach: 2 (cells of half a cut-off) for dense 2D systems (>= 1.5 binned particles per
  // cut-off square), where it examines about a third fewer neighbours; else 1
  if (c.cell_reach > 0) {
    h->reach = c.cell_reach;
  } else if (c.dim == 2 && rc > 0.0) {
    double nb = 0.0, area = 0.0;
    for (const rd_replica& rp : h->reps_host) {
      for (int sp = 0; sp < c.n_species; ++sp)
        if ((bmask >> sp) & 1u) nb += (double)rp.n_init[sp];
      area += rp.L * rp.L;
    }
    h->reach = nb / area * rc * rc >= 1.5 ? 2 : 1;
  }
  // cell-edge choices: > 0 a fixed factor, < 0 the per-replica density rule times -value
  std::vector<double> factors;
  if (c.cell_factor_x100 > 0) {
    factors.push_back(c.cell_factor_x100 / 100.0);
  } else if (c.cell_factor_x100 == 0) {
    factors.push_back(-1.0);
  } else {
    for (double f : {-1.0, 1.0, -0.7, -1.5}) factors.push_back(f);
  }
  int64_t total_cells = 0, n_total = 0;
  h->reps_init.resize(c.n_replicas);
  for (int r = 0; r < c.n_replicas; ++r) {
    const rd_replica& rp = h->reps_host[r];
    RepDev& d = h->reps_init[r];
    std::memset(&d, 0, sizeof d);
    d.L = rp.L;
    d.half_L = 0.5 * rp.L;
    d.Lf = (float)rp.L;
    d.half_Lf = 0.5f * d.Lf;
    int64_t nr = 0;
    for (int s = 0; s < c.n_species; ++s) nr += rp.n_init[s];
    d.beg = (uint32_t)n_total;
    d.end = (uint32_t)(n_total + nr);
    d.next_id = (uint32_t)nr;
    n_total += nr;
  }
  int64_t max_cells = 0;
  {
    std::vector<RepDev> tmp = h->reps_init;
    for (double f : factors) max_cells = std::max(max_cells, layout_cells(c, h->reps_host, bmask, rc, f, h->reach, tmp));
  }
  total_cells = layout_cells(c, h->reps_host, bmask, rc, factors[0], h->reach, h->reps_init);
  h->factors = factors;
  h->factor = factors[0];
  if (max_cells >= (int64_t)0xFFFFFFF0) {
    delete h;
    return RD_EINVAL;
  }
  const double cf = c.capacity_factor > 0.0 ? c.capacity_factor : 2.0;
  int64_t cap = (int64_t)std::ceil(cf * (double)n_total) + 1024;
  if (cap >= (int64_t)0x7FFFFFF0) {
    delete h;
    return RD_EINVAL;
  }
  int64_t pair_cap = c.pair_capacity > 0 ? c.pair_capacity : std::max<int64_t>(65536, cap);
  h->hp.cap_particles = cap;
  h->hp.cap_pairs = pair_cap;

  StepLaunch& L = h->L;
  std::memset(&L, 0, sizeof L);
  L.pdl = true;
  L.reach = h->reach;
  const int rows = c.dim == 3 ? 5 : (h->reach == 2 ? 3 : 2);
  L.sweep_split = c.sweep_split == 2 && (double)cap * rows < 4.0e9 ? rows : 1;
  L.match_grid = match_grid_for_current_device();
  L.precision = c.precision;
  L.block = c.block_size > 0 ? c.block_size : 256;
  L.max_grid = device_sms() * 16;
  // automatic: separate kernels under programmatic dependent launch, which measured faster than
  // the fused launch on every workload timed (a grid barrier costs more than a kernel boundary the
  // next launch already overlaps); the autotuner tries the fused launch as well
  L.fused = c.step_launch == 1;
  L.scan_items = 8;
  L.cap_particles = cap;
  L.cap_pairs = pair_cap;
  L.total_cells = total_cells;
  L.n_counts = c.n_replicas * c.n_species;
  L.fused_grid = fused_grid_size(L, device_sms());
  if (L.fused_grid < 1) L.fused = 0;
  cudaGetLastError();   // a refused attribute or occupancy query leaves no error behind
  const int64_t chunk = 256 * (int64_t)L.scan_items;
  const int64_t nbc = (max_cells + chunk - 1) / chunk, nbp = (cap + chunk - 1) / chunk;
  L.flag_stride = std::max(nbc, nbp) + 1;

  bool ok = true;
  auto A = [&](size_t bytes) {
    void* p = dev_alloc(h, bytes);
    if (!p) ok = false;
    return p;
  };
  const size_t vs = h->vsize;
  h->xbuf[0] = A(cap * vs);
  h->xbuf[1] = A(cap * vs);
  h->idbuf[0] = (uint32_t*)A(cap * 4);
  h->idbuf[1] = (uint32_t*)A(cap * 4);
  L.x1 = A(cap * vs);
  // sorted start and end positions interleaved: record k's pair fills one 32-byte sector (mixed)
  L.sx0 = A(2 * cap * vs);
  L.sx1 = L.sx0 ? (void*)((char*)L.sx0 + vs) : nullptr;
  L.prodpos = A(2 * cap * vs);
  L.status = (uint32_t*)A(cap * 4);
  L.matched = (int32_t*)A(cap * 4);
  L.deg = (uint32_t*)A(cap * 4);
  L.cell_of = (uint32_t*)A(cap * 4);
  L.slot = (uint32_t*)A(cap * 4);
  L.sidx = (uint32_t*)A(cap * 4);
  L.decay_list = (uint32_t*)A(cap * 4);
  L.best_key = (unsigned long long*)A(cap * 8);
  L.best_pid = (unsigned long long*)A(cap * 8);
  L.x0d = h->hp.has_drift ? A(cap * vs) : nullptr;
  L.repx = (RepX*)A((size_t)c.n_replicas * sizeof(RepX));
  L.rep_cons = (uint32_t*)A((size_t)c.n_replicas * 4);
  L.rep_prod = (uint32_t*)A((size_t)c.n_replicas * 4);
  L.cell_count = (uint32_t*)A(max_cells * 4);
  L.cell_start = (uint32_t*)A((max_cells + 1) * 4);
  L.agg32 = (uint32_t*)A((nbc + 1) * 4);
  L.incl32 = (uint32_t*)A((nbc + 1) * 4);
  L.agg64 = (unsigned long long*)A((nbp + 1) * 8);
  L.incl64 = (unsigned long long*)A((nbp + 1) * 8);
  L.flags = (uint32_t*)A(2 * L.flag_stride * 4);
  L.accepted = (uint32_t*)A(pair_cap * 4);
  L.fired = (FiredPair*)A(pair_cap * sizeof(FiredPair));
  L.fstate = (uint32_t*)A(pair_cap * 4);
  L.conflict = (uint32_t*)A(pair_cap * 4);
  L.crec = (ConflictRec*)A(pair_cap * sizeof(ConflictRec));
  // angle jobs: one per accepted pair (two particles each) and one per decay with a product pair
  // (a decaying particle takes part in no pair), so never more than the particle capacity
  L.angles = c.angle_mode == 0;
  L.ang_cap = L.angles ? (uint32_t)cap : 1u;
  L.ang_jobs = (AngJob*)A((size_t)L.ang_cap * sizeof(AngJob));
  L.counts = (unsigned long long*)A((size_t)L.n_counts * 8);
  L.history_len = kHistoryLen;
  L.history = (long long*)A((size_t)kHistoryLen * c.n_species * 8);
  L.P = (const DevParams*)A(sizeof(DevParams));
  L.ctl = (DevCtl*)A(sizeof(DevCtl));
  L.reps = (RepDev*)A(c.n_replicas * sizeof(RepDev));
  if (!ok) {
    free_all(h);
    cudaStreamSynchronize(h->stream);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return RD_ENOMEM;
  }
  if (!build_2d(c, h->hp, [&](size_t bytes) { return dev_alloc(h, bytes); })) {
    free_all(h);
    cudaStreamSynchronize(h->stream);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return RD_ENOMEM;
  }
  auto fail = [&](cudaError_t e) {
    free_all(h);
    cudaStreamSynchronize(h->stream);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return cuda_fail(e);
  };
  cudaError_t e = cudaSuccess;
  e = cudaMemsetAsync(L.cell_count, 0, max_cells * 4, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.deg, 0, cap * 4, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.flags, 0, 2 * L.flag_stride * 4, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.status, 0, cap * 4, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.rep_cons, 0, (size_t)c.n_replicas * 4, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.rep_prod, 0, (size_t)c.n_replicas * 4, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync((void*)L.P, &h->hp, sizeof(DevParams), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(L.reps, h->reps_init.data(), c.n_replicas * sizeof(RepDev), cudaMemcpyHostToDevice, h->stream);
  DevCtl ctl;
  std::memset(&ctl, 0, sizeof ctl);
  ctl.n = (uint32_t)n_total;
  if (e == cudaSuccess) e = cudaMemcpyAsync(L.ctl, &ctl, sizeof ctl, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = build_tables(h, [&](size_t bytes) { return dev_alloc(h, bytes); });
  if (e != cudaSuccess) return fail(e);

  // initial positions: ids 0..N_r-1 per replica, species in blocks of n_init
  if (n_total > 0) {
    std::vector<int32_t> rep_of(n_total), sp_of(n_total);
    std::vector<uint32_t> id_of(n_total);
    int64_t i = 0;
    for (int r = 0; r < c.n_replicas; ++r) {
      uint32_t k = 0;
      for (int s = 0; s < c.n_species; ++s)
        for (int64_t m = 0; m < h->reps_host[r].n_init[s]; ++m, ++i, ++k) {
          rep_of[i] = r;
          sp_of[i] = s;
          id_of[i] = k;
        }
    }
    void* tmp = nullptr;
    const size_t bytes = (size_t)n_total * 12;
    e = cudaMallocAsync(&tmp, bytes, h->stream);
    if (e != cudaSuccess) return fail(e);
    int32_t* d_rep = (int32_t*)tmp;
    int32_t* d_sp = d_rep + n_total;
    uint32_t* d_id = (uint32_t*)(d_sp + n_total);
    e = cudaMemcpyAsync(d_rep, rep_of.data(), n_total * 4, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_sp, sp_of.data(), n_total * 4, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_id, id_of.data(), n_total * 4, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) {
      StepLaunch L0 = launch_for(h, 0);
      launch_init_positions(L0, d_rep, d_sp, d_id, (uint32_t)n_total, h->stream);
      e = cudaGetLastError();
    }
    cudaFreeAsync(tmp, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(e);
  }
  launch_count(launch_for(h, 0), h->stream);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(e);
  if (c.cell_factor_x100 < 0 && n_total > 0) {
    e = autotune(h);
    if (e != cudaSuccess) return fail(e);
  }
  *out = h;
  return RD_OK;
}

int rd_step(rd_handle* h) {
  if (!h) return RD_EINVAL;
  StepLaunch L = launch_for(h, h->cur);
  if (h->time_next && L.fused) {
    // per-phase device times from the phase clock of the fused launch, and the launch's event time
    DevCtl before, after;
    RD_CUDA(cudaStreamSynchronize(h->stream));
    RD_CUDA(cudaMemcpy(&before, h->L.ctl, sizeof before, cudaMemcpyDeviceToHost));
    h->timer.reset();
    h->timer.mark("begin", h->stream);
    launch_fused_steps(L, 1, h->stream);
    h->timer.mark("k_step_fused", h->stream);
    RD_CUDA(cudaGetLastError());
    RD_CUDA(cudaStreamSynchronize(h->stream));
    RD_CUDA(cudaMemcpy(&after, h->L.ctl, sizeof after, cudaMemcpyDeviceToHost));
    h->last_times.clear();
    for (int k = 0; k < kFusedPhases; ++k)
      h->last_times.emplace_back(kFusedPhaseNames[k], (float)((after.ph_acc[k] - before.ph_acc[k]) * 1e-6));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->timer.events[0], h->timer.events[1]);
    h->last_times.emplace_back("k_step_fused", ms);
    h->time_next = false;
    h->cur ^= 1;
    return RD_OK;
  }
  if (h->time_next) {
    h->timer.reset();
    launch_step(L, h->stream, &h->timer);
  } else {
    launch_step(L, h->stream, nullptr);
  }
  RD_CUDA(cudaGetLastError());
  if (h->time_next) {
    RD_CUDA(cudaStreamSynchronize(h->stream));
    h->last_times.clear();
    for (size_t k = 1; k < h->timer.used; ++k) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, h->timer.events[k - 1], h->timer.events[k]);
      h->last_times.emplace_back(h->timer.names[k], ms);
    }
    h->time_next = false;
  }
  h->cur ^= 1;
  return RD_OK;
}

static int capture_graph(rd_handle* h, int start) {
  cudaGraph_t g = nullptr;
  RD_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  if (h->L.fused) {
    launch_fused_steps(launch_for(h, start), 2, h->stream);     // both steps in one launch
  } else {
    launch_step(launch_for(h, start), h->stream, nullptr);
    launch_step(launch_for(h, 1 - start), h->stream, nullptr);
  }
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaGraphInstantiate(&h->graph[start], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->graph[start] = nullptr;
    return cuda_fail(e);
  }
  return RD_OK;
}

int rd_run(rd_handle* h, int64_t nsteps) {
  if (!h || nsteps < 0) return RD_EINVAL;
  int64_t pairs = nsteps / 2;
  if (pairs > 0) {
    if (!h->graph[h->cur]) {
      int rc = capture_graph(h, h->cur);
      if (rc != RD_OK) return rc;
    }
    for (int64_t k = 0; k < pairs; ++k) RD_CUDA(cudaGraphLaunch(h->graph[h->cur], h->stream));
  }
  if (nsteps & 1) return rd_step(h);
  return RD_OK;
}

int rd_sync(rd_handle* h) {
  if (!h) return RD_EINVAL;
  RD_CUDA(cudaStreamSynchronize(h->stream));
  int32_t st = 0;
  RD_CUDA(cudaMemcpy(&st, &h->L.ctl->status, sizeof st, cudaMemcpyDeviceToHost));
  return st;
}

int rd_observables(rd_handle* h, int64_t* counts, int64_t* step, double* t, int64_t* stats) {
  if (!h) return RD_EINVAL;
  RD_CUDA(cudaStreamSynchronize(h->stream));
  DevCtl ctl;
  RD_CUDA(cudaMemcpy(&ctl, h->L.ctl, sizeof ctl, cudaMemcpyDeviceToHost));
  if (counts)
    RD_CUDA(cudaMemcpy(counts, h->L.counts, (size_t)h->L.n_counts * 8, cudaMemcpyDeviceToHost));
  if (step) *step = ctl.step;
  if (t) *t = ctl.t;
  if (stats)
    for (int k = 0; k < RD_NSTATS; ++k) stats[k] = (int64_t)ctl.stats[k];
  return ctl.status;
}

int rd_num_particles(rd_handle* h, int64_t* n) {
  if (!h || !n) return RD_EINVAL;
  RD_CUDA(cudaStreamSynchronize(h->stream));
  uint32_t v = 0;
  RD_CUDA(cudaMemcpy(&v, &h->L.ctl->n, sizeof v, cudaMemcpyDeviceToHost));
  *n = v;
  return RD_OK;
}

static bool ensure_staging(rd_handle* h) {
  if (h->st_x) return true;
  const int64_t cap = h->L.cap_particles;
  const int R = h->cfg.n_replicas;
  h->st_x = (double*)dev_alloc(h, (size_t)cap * 24);
  h->st_sp = (int32_t*)dev_alloc(h, (size_t)cap * 4);
  h->st_id = (uint32_t*)dev_alloc(h, (size_t)cap * 4);
  h->st_rep = (int32_t*)dev_alloc(h, (size_t)cap * 4);
  h->st_cnt = (uint32_t*)dev_alloc(h, (size_t)R * 4);
  h->st_maxid = (uint32_t*)dev_alloc(h, (size_t)R * 4);
  h->st_next = (uint32_t*)dev_alloc(h, (size_t)R * 4);
  h->st_err = (int32_t*)dev_alloc(h, 16);
  return h->st_x && h->st_sp && h->st_id && h->st_rep && h->st_cnt && h->st_maxid && h->st_next && h->st_err;
}

int rd_get_state(rd_handle* h, int64_t* n_inout, double* x, int32_t* species, uint32_t* id, int32_t* replica,
                 uint32_t* next_id, int64_t* step) {
  if (!h || !n_inout) return RD_EINVAL;
  DevCtl ctl;
  RD_CUDA(cudaMemcpyAsync(&ctl, h->L.ctl, sizeof ctl, cudaMemcpyDeviceToHost, h->stream));
  RD_CUDA(cudaStreamSynchronize(h->stream));
  const int64_t n = ctl.n;
  if (*n_inout < n) {
    *n_inout = n;
    return RD_EINVAL;
  }
  *n_inout = n;
  if (step) *step = ctl.step;
  if (n > 0 && (x || species || replica)) {
    // unpacked on the device, then one copy per array (page-locked caller buffers take the copy
    // engines' direct path; a kernel writing host memory itself measured slower)
    if (!ensure_staging(h)) return RD_ENOMEM;
    launch_get_state(h->L, h->xbuf[h->cur], n, x ? h->st_x : nullptr, species ? h->st_sp : nullptr,
                     replica ? h->st_rep : nullptr, h->stream);
    RD_CUDA(cudaGetLastError());
    if (x) RD_CUDA(cudaMemcpyAsync(x, h->st_x, (size_t)n * 24, cudaMemcpyDeviceToHost, h->stream));
    if (species) RD_CUDA(cudaMemcpyAsync(species, h->st_sp, (size_t)n * 4, cudaMemcpyDeviceToHost, h->stream));
    if (replica) RD_CUDA(cudaMemcpyAsync(replica, h->st_rep, (size_t)n * 4, cudaMemcpyDeviceToHost, h->stream));
  }
  if (id && n > 0) RD_CUDA(cudaMemcpyAsync(id, h->idbuf[h->cur], (size_t)n * 4, cudaMemcpyDeviceToHost, h->stream));
  std::vector<RepDev> reps;
  if (next_id) {
    reps.resize(h->cfg.n_replicas);
    RD_CUDA(cudaMemcpyAsync(reps.data(), h->L.reps, reps.size() * sizeof(RepDev), cudaMemcpyDeviceToHost, h->stream));
  }
  RD_CUDA(cudaStreamSynchronize(h->stream));
  for (size_t r = 0; r < reps.size(); ++r) next_id[r] = reps[r].next_id;
  return ctl.status;
}

int rd_set_state(rd_handle* h, int64_t n, const double* x, const int32_t* species, const uint32_t* id,
                 const int32_t* replica, const uint32_t* next_id, int64_t step) {
  if (!h || n < 0 || (n > 0 && (!x || !species || !id))) return RD_EINVAL;
  if (n > h->L.cap_particles) return RD_ECAPACITY;
  if (step < 0 || step > 0xFFFFFFFFll) return RD_EINVAL;
  const rd_config& c = h->cfg;
  if (!ensure_staging(h)) return RD_ENOMEM;
  cudaStream_t s = h->stream;
  // raw inputs to the device, one copy per array; validation and packing there, into the spare
  // state buffer, so that a rejected state leaves the current one untouched
  if (n > 0) {
    RD_CUDA(cudaMemcpyAsync(h->st_x, x, (size_t)n * 24, cudaMemcpyHostToDevice, s));
    RD_CUDA(cudaMemcpyAsync(h->st_sp, species, (size_t)n * 4, cudaMemcpyHostToDevice, s));
    RD_CUDA(cudaMemcpyAsync(h->st_id, id, (size_t)n * 4, cudaMemcpyHostToDevice, s));
    if (replica) RD_CUDA(cudaMemcpyAsync(h->st_rep, replica, (size_t)n * 4, cudaMemcpyHostToDevice, s));
  }
  const double* dx = h->st_x;
  const int32_t* dsp = h->st_sp;
  const uint32_t* did = h->st_id;
  const int32_t* drep = replica ? h->st_rep : nullptr;
  if (next_id) RD_CUDA(cudaMemcpyAsync(h->st_next, next_id, (size_t)c.n_replicas * 4, cudaMemcpyHostToDevice, s));
  RD_CUDA(cudaMemsetAsync(h->st_cnt, 0, (size_t)c.n_replicas * 4, s));
  RD_CUDA(cudaMemsetAsync(h->st_maxid, 0, (size_t)c.n_replicas * 4, s));
  RD_CUDA(cudaMemsetAsync(h->st_err, 0, 4, s));
  const int spare = 1 - h->cur;
  launch_set_state(h->L, n, dx, dsp, did, drep, h->xbuf[spare], h->idbuf[spare], h->st_cnt, h->st_maxid,
                   next_id ? h->st_next : nullptr, h->st_err, step, s);
  RD_CUDA(cudaGetLastError());
  int32_t err = 0;
  RD_CUDA(cudaMemcpyAsync(&err, h->st_err, 4, cudaMemcpyDeviceToHost, s));
  RD_CUDA(cudaStreamSynchronize(s));
  if (err) return RD_EINVAL;
  h->cur = spare;
  // the counts of the new state follow in stream order (the next call that reads them synchronises)
  launch_count(launch_for(h, h->cur), s);
  RD_CUDA(cudaGetLastError());
  return RD_OK;
}

int rd_pair_probs(rd_handle* h, int32_t rule, const double* r0, const double* r, int64_t n, double* p_enc,
                  double* p_reac) {
  if (!h || rule < 0 || rule >= h->cfg.n_pairs || n < 0 || (n > 0 && (!r0 || !r))) return RD_EINVAL;
  if (h->cfg.pairs[rule].bc == RD_BC_NONE) return RD_EINVAL;
  if (n == 0) return RD_OK;
  launch_pair_probs(h->L.P, rule, r0, r, n, p_enc, p_reac, h->L.max_grid,
                    h->cfg.precision == RD_MIXED && h->cfg.dim == 3, h->stream);
  RD_CUDA(cudaGetLastError());
  return RD_OK;
}

int rd_resample(rd_handle* h, int32_t rule, const double* r0, const double* u, int64_t n, double* r_new) {
  if (!h || rule < 0 || rule >= h->cfg.n_pairs || n < 0 || (n > 0 && (!r0 || !u || !r_new))) return RD_EINVAL;
  if (h->cfg.pairs[rule].bc == RD_BC_NONE) return RD_EINVAL;
  if (n == 0) return RD_OK;
  launch_resample(h->L.P, rule, r0, u, n, r_new, h->L.max_grid, h->stream);
  RD_CUDA(cudaGetLastError());
  return RD_OK;
}

int rd_propagate(rd_handle* h, int32_t rule, const double* r0, const double* u, int64_t n, double* r_out) {
  if (!h || rule < 0 || rule >= h->cfg.n_pairs || n < 0 || (n > 0 && (!r0 || !u || !r_out))) return RD_EINVAL;
  const int bc = h->cfg.pairs[rule].bc;
  if (bc != RD_BC_REF && bc != RD_BC_RAD) return RD_EINVAL;
  if (n == 0) return RD_OK;
  launch_propagate(h->L.P, rule, r0, u, n, r_out, h->L.max_grid, h->stream);
  RD_CUDA(cudaGetLastError());
  return RD_OK;
}

int rd_first_passage(rd_handle* h, int32_t rule, const double* r0, const double* r, const uint64_t* stream,
                     int64_t n, int32_t levels, uint32_t max_attempts, uint32_t* bin, double* r_lo, double* r_hi,
                     uint32_t* attempts) {
  if (!h || rule < 0 || rule >= h->cfg.n_pairs || n < 0 || levels < 0 || levels > kFptMaxLevels) return RD_EINVAL;
  if (h->cfg.pairs[rule].bc == RD_BC_NONE) return RD_EINVAL;
  if (n > 0 && (!r0 || !r || !stream || !bin)) return RD_EINVAL;
  if (n > (int64_t)0xFFFFFFFFll) return RD_EINVAL;
  if (n == 0) return RD_OK;
  const PairDev& q = h->hp.pairs[rule];
  FptArgs A{};
  A.dim = h->cfg.dim;
  A.levels = levels;
  A.f32 = h->cfg.precision == RD_MIXED && h->cfg.dim == 3;
  A.max_attempts = max_attempts ? max_attempts : RD_FPT_MAX_ATTEMPTS;
  A.seed_lo = h->hp.seed_lo;
  A.seed_hi = h->hp.seed_hi;
  A.tau = q.tau;
  A.sigma = q.sigma;
  A.ser = q.ser;
  if (A.dim == 2) {
    auto& sets = h->fpt_nodes[rule];
    const double Rmax = std::sqrt(q.rcut2) / q.sigma + 13.0 * q.s + 3.0;
    for (int l = (int)sets.size(); l < levels; ++l) {
      const double tl = std::ldexp(q.tau, -(l + 1));
      if (tl <= h->cfg.tau_s) {
        sets.emplace_back(nullptr, 0);
        continue;
      }
      std::vector<WeberNode> nodes = weber_nodes(tl, q.h, Rmax);
      void* dn = dev_alloc(h, nodes.size() * sizeof(WeberNode));
      if (!dn) return RD_ENOMEM;
      RD_CUDA(cudaMemcpyAsync(dn, nodes.data(), nodes.size() * sizeof(WeberNode), cudaMemcpyHostToDevice, h->stream));
      RD_CUDA(cudaStreamSynchronize(h->stream));
      sets.emplace_back(dn, (int)nodes.size());
    }
    for (int l = 0; l < levels; ++l) {
      A.lv[l].nodes = sets[l].first;
      A.lv[l].n_nodes = sets[l].second;
    }
  }
  if (n > h->fpt_qcap) {
    // each queue holds a pair at most once per round, so n entries per queue suffice
    void* q = dev_alloc(h, 4 * (size_t)n * sizeof(FptItem) + (size_t)n * sizeof(FptSearch));
    if (!q) return RD_ENOMEM;
    if (h->fpt_queue) dev_release(h, h->fpt_queue);
    if (!h->fpt_qctl) {
      h->fpt_qctl = (uint32_t*)dev_alloc(h, kFptCtlWords * sizeof(uint32_t));
      if (!h->fpt_qctl) return RD_ENOMEM;
    }
    h->fpt_queue = (FptItem*)q;
    h->fpt_qcap = n;
  }
  FptItem* qb = h->fpt_queue;
  const int64_t qc = h->fpt_qcap;
  FptItem* warp_q[2] = {qb, qb + qc};
  launch_first_passage(A, r0, r, stream, n, bin, r_lo, r_hi, attempts, warp_q, qb + 2 * qc, qb + 3 * qc,
                       (FptSearch*)(qb + 4 * qc), h->fpt_qctl, h->L.max_grid / 16, h->stream);
  RD_CUDA(cudaGetLastError());
  return RD_OK;
}

int rd_last_fired(rd_handle* h, int64_t cap, int64_t* n_out, uint32_t* id_a, uint32_t* id_b, double* p_enc,
                  int32_t* accepted, int32_t* replica, double* key) {
  if (!h || !n_out || cap < 0) return RD_EINVAL;
  RD_CUDA(cudaStreamSynchronize(h->stream));
  DevCtl ctl;
  RD_CUDA(cudaMemcpy(&ctl, h->L.ctl, sizeof ctl, cudaMemcpyDeviceToHost));
  const int64_t n = std::min<int64_t>(ctl.last_fired, h->L.cap_pairs);
  *n_out = n;
  const int64_t m = std::min(n, cap);
  if (m > 0) {
    std::vector<FiredPair> f(m);
    std::vector<uint32_t> fs(m);
    RD_CUDA(cudaMemcpy(f.data(), h->L.fired, m * sizeof(FiredPair), cudaMemcpyDeviceToHost));
    RD_CUDA(cudaMemcpy(fs.data(), h->L.fstate, m * 4, cudaMemcpyDeviceToHost));
    for (int64_t k = 0; k < m; ++k) {
      if (id_a) id_a[k] = f[k].ida;
      if (id_b) id_b[k] = f[k].idb;
      if (p_enc) p_enc[k] = f[k].p;
      if (accepted) accepted[k] = (fs[k] & 3u) == FS_ACCEPTED;
      if (replica) replica[k] = (int32_t)(fs[k] >> 8);
      if (key) key[k] = f[k].key;
    }
  }
  return ctl.status;
}

int rd_check_bounded_wait(rd_handle* h, uint32_t spin_limit, int32_t* status_out) {
  if (!h || !status_out || spin_limit == 0) return RD_EINVAL;
  RD_CUDA(cudaStreamSynchronize(h->stream));
  DevCtl saved, probe;
  RD_CUDA(cudaMemcpy(&saved, h->L.ctl, sizeof saved, cudaMemcpyDeviceToHost));
  if (saved.status != 0) return saved.status;
  probe = saved;
  probe.epoch += 1;          // a scan epoch whose flags nobody has published yet
  probe.tile_ctr[0] = 1;     // tile 0 is never taken: tile 1 waits for a flag that nothing sets
  probe.spin_limit = spin_limit;
  RD_CUDA(cudaMemcpy(h->L.ctl, &probe, sizeof probe, cudaMemcpyHostToDevice));
  // the cell counts are all zero between steps; the scan rewrites the cell starts, which the next
  // step rebuilds
  launch_cell_scan(launch_for(h, h->cur), h->stream);
  RD_CUDA(cudaGetLastError());
  RD_CUDA(cudaStreamSynchronize(h->stream));
  DevCtl after;
  RD_CUDA(cudaMemcpy(&after, h->L.ctl, sizeof after, cudaMemcpyDeviceToHost));
  *status_out = after.status;
  DevCtl back = saved;
  back.epoch = after.epoch;  // flags written by the probe must not look current later
  RD_CUDA(cudaMemcpy(h->L.ctl, &back, sizeof back, cudaMemcpyHostToDevice));
  return RD_OK;
}

int rd_info(rd_handle* h, double* out, int32_t n) {
  if (!h || !out || n < 0) return RD_EINVAL;
  const double v[11] = {h->factor, (double)h->L.total_cells, (double)h->L.block,
                        (double)h->L.cap_particles, (double)h->L.cap_pairs, h->tuned_ms,
                        max_cutoff(h->cfg), (double)h->L.sweep_split, (double)h->reach,
                        (double)h->L.fused, (double)h->L.fused_grid};
  for (int k = 0; k < n && k < 11; ++k) out[k] = v[k];
  return RD_OK;
}

int rd_count_history(rd_handle* h, int64_t first_step, int64_t n_steps, int64_t* out) {
  if (!h || !out || first_step < 0 || n_steps < 0) return RD_EINVAL;
  RD_CUDA(cudaStreamSynchronize(h->stream));
  DevCtl ctl;
  RD_CUDA(cudaMemcpy(&ctl, h->L.ctl, sizeof ctl, cudaMemcpyDeviceToHost));
  const int64_t last = ctl.step;
  if (first_step + n_steps - 1 > last || (n_steps > 0 && last - first_step >= h->L.history_len)) return RD_EINVAL;
  const int ns = h->cfg.n_species;
  std::vector<long long> ring((size_t)h->L.history_len * ns);
  RD_CUDA(cudaMemcpy(ring.data(), h->L.history, ring.size() * sizeof(long long), cudaMemcpyDeviceToHost));
  for (int64_t k = 0; k < n_steps; ++k) {
    const int64_t slot = (first_step + k) % h->L.history_len;
    for (int sp = 0; sp < ns; ++sp) out[k * ns + sp] = ring[(size_t)slot * ns + sp];
  }
  return RD_OK;
}

int rd_time_kernels(rd_handle* h, int32_t enable) {
  if (!h) return RD_EINVAL;
  h->time_next = enable != 0;
  return RD_OK;
}

int rd_kernel_times(rd_handle* h, int32_t cap, int32_t* n_out, char* names, float* ms) {
  if (!h || !n_out) return RD_EINVAL;
  const int n = (int)h->last_times.size();
  *n_out = n;
  for (int k = 0; k < n && k < cap; ++k) {
    if (names) {
      std::memset(names + 32 * k, 0, 32);
      std::strncpy(names + 32 * k, h->last_times[k].first.c_str(), 31);
    }
    if (ms) ms[k] = h->last_times[k].second;
  }
  return RD_OK;
}

void rd_free(rd_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  for (int k = 0; k < 2; ++k)
    if (h->graph[k]) cudaGraphExecDestroy(h->graph[k]);
  h->timer.destroy();
  free_all(h);
  cudaStreamSynchronize(h->stream);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
}

}  // extern "C"

// ================================================================================================
// Allocation-free single step (rd_step_static).  Every scratch buffer of the step lives in one
// file-scope device array; the caller passes the state in and receives it out in device buffers.
// ================================================================================================

namespace {

constexpr size_t kStaticScratchBytes = (size_t)RD_STATIC_SCRATCH_BYTES;
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_addr[kStaticMaxDevices] = {};

// Device address of the static scratch for the current device, looked up once per device.
cudaError_t static_scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kStaticMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return cudaSuccess;
}

struct Bump {
  unsigned char* base;
  size_t used = 0;
  bool ok = true;
  void* take(size_t bytes) {
    size_t off = (used + 255) & ~(size_t)255;
    if (off + bytes > kStaticScratchBytes) {
      ok = false;
      return nullptr;
    }
    used = off + bytes;
    return base + off;
  }
};

template <class V>
__global__ void k_static_pack(int64_t n, int dim, double L, const double* __restrict__ x,
                              const int32_t* __restrict__ sp, const uint32_t* __restrict__ id,
                              V* __restrict__ xo, uint32_t* __restrict__ ido) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double p0 = x[3 * i], p1 = x[3 * i + 1], p2 = dim == 3 ? x[3 * i + 2] : 0.0;
    const uint32_t wb = pack_sp((uint32_t)sp[i], 0u);
    if constexpr (sizeof(V) == 32) {
      d4 v;
      v.x = p0; v.y = p1; v.z = p2; v.w = w_from_bits_d(wb);
      xo[i] = v;
    } else {
      float f[3] = {(float)p0, (float)p1, (float)p2};
      for (int d = 0; d < 3; ++d)
        if (!(f[d] < (float)L)) f[d] = 0.0f;
      xo[i] = make_float4(f[0], f[1], f[2], w_from_bits_f(wb));
    }
    ido[i] = id[i];
  }
}

template <class V>
__global__ void k_static_unpack(const DevCtl* __restrict__ ctl, const RepDev* __restrict__ rep,
                                const V* __restrict__ xs, const uint32_t* __restrict__ ids, double* __restrict__ x,
                                int32_t* __restrict__ sp, uint32_t* __restrict__ id, int64_t* __restrict__ n_out,
                                uint32_t* __restrict__ next_id_out, int32_t* __restrict__ status_out) {
  const uint32_t n = ctl->n;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const V v = xs[i];
    x[3 * i] = (double)v.x;
    x[3 * i + 1] = (double)v.y;
    x[3 * i + 2] = (double)v.z;
    sp[i] = (int32_t)(w_bits(v.w) & 0xFFu);
    id[i] = ids[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (n_out) *n_out = (int64_t)n;
    if (next_id_out) *next_id_out = rep->next_id;
    if (status_out) *status_out = ctl->status;
  }
}

}  // namespace

extern "C" int rd_step_static(const rd_config* cfg, void* stream, int64_t n, const double* x_in,
                              const int32_t* species_in, const uint32_t* id_in, uint32_t next_id, int64_t step,
                              int64_t out_cap, double* x_out, int32_t* species_out, uint32_t* id_out,
                              int64_t* n_out, uint32_t* next_id_out, int32_t* status_out) {
  if (!cfg || cfg->n_replicas != 1 || !cfg->replicas) return RD_EINVAL;
  if (cfg->dim != 3) return RD_ENOTREADY;
  if (n < 0 || n > RD_STATIC_MAX_PARTICLES || step < 0 || step > 0xFFFFFFFFll) return RD_EINVAL;
  if (n > 0 && (!x_in || !species_in || !id_in)) return RD_EINVAL;
  if (out_cap < 2 * n || !x_out || !species_out || !id_out) return RD_EINVAL;
  rd_config c = *cfg;
  if (c.c_cut == 0.0) c.c_cut = 5.0;
  if (c.tau_s == 0.0) c.tau_s = 0.01;
  const int v = validate(&c);
  if (v != RD_OK) return v;

  void* base = nullptr;
  cudaError_t e = static_scratch_address(&base);
  if (e != cudaSuccess) return cuda_fail(e);
  cudaStream_t s = (cudaStream_t)stream;

  // derived parameters and the single replica's cell grid (coarsened until it fits the maximum)
  rd_handle tmp;
  tmp.cfg = c;
  tmp.cfg.replicas = nullptr;
  derive_params(&tmp);
  const rd_replica& rp = cfg->replicas[0];
  const double rc = max_cutoff(c);
  RepDev rep;
  std::memset(&rep, 0, sizeof rep);
  rep.L = rp.L;
  rep.half_L = 0.5 * rp.L;
  rep.Lf = (float)rp.L;
  rep.half_Lf = 0.5f * rep.Lf;
  double factor = (c.cell_factor_x100 > 0 ? c.cell_factor_x100 : 100) / 100.0;
  int64_t cells = 1;
  for (int attempt = 0; attempt < 64; ++attempt) {
    cells = 1;
    for (int a = 0; a < 3; ++a) {
      int m = 1;
      if (a < c.dim && rc > 0.0) {
        const double q = std::floor(rp.L / (rc * factor * (1.0 + 1e-6)));
        m = q >= 3.0 ? (int)std::min(q, 2048.0) : 1;
      }
      rep.nc[a] = m;
      rep.inv_edge[a] = m / rp.L;
      rep.inv_edge_f[a] = (float)rep.inv_edge[a];
      cells *= m;
    }
    if (cells <= RD_STATIC_MAX_CELLS) break;
    factor *= 1.25;
  }
  if (cells > RD_STATIC_MAX_CELLS) return RD_EINVAL;
  rep.cell_base = 0;
  rep.beg = 0;
  rep.end = (uint32_t)n;
  rep.next_id = next_id;

  const int64_t cap = 2 * (int64_t)RD_STATIC_MAX_PARTICLES + 1024;
  const int64_t pair_cap = RD_STATIC_MAX_PAIRS;
  tmp.hp.cap_particles = cap;
  tmp.hp.cap_pairs = pair_cap;
  const size_t vs = c.precision == RD_MIXED ? 16 : 32;

  StepLaunch L;
  std::memset(&L, 0, sizeof L);
  L.pdl = true;
  L.sweep_split = 1;
  L.match_grid = match_grid_for_current_device();
  L.precision = c.precision;
  L.block = 256;
  L.max_grid = device_sms() * 16;
  L.scan_items = 8;
  L.cap_particles = cap;
  L.cap_pairs = pair_cap;
  L.total_cells = cells;
  L.n_counts = c.n_species;
  const int64_t chunk = 256 * (int64_t)L.scan_items;
  const int64_t nbc = (cells + chunk - 1) / chunk, nbp = (cap + chunk - 1) / chunk;
  Bump b{(unsigned char*)base};
  void* xb0 = b.take(cap * vs);
  void* xb1 = b.take(cap * vs);
  uint32_t* id0 = (uint32_t*)b.take(cap * 4);
  uint32_t* id1 = (uint32_t*)b.take(cap * 4);
  L.x1 = b.take(cap * vs);
  L.sx0 = b.take(2 * cap * vs);
  L.sx1 = (void*)((char*)L.sx0 + vs);
  L.prodpos = b.take(2 * cap * vs);
  L.status = (uint32_t*)b.take(cap * 4);
  L.matched = (int32_t*)b.take(cap * 4);
  L.deg = (uint32_t*)b.take(cap * 4);
  L.cell_of = (uint32_t*)b.take(cap * 4);
  L.slot = (uint32_t*)b.take(cap * 4);
  L.sidx = (uint32_t*)b.take(cap * 4);
  L.decay_list = (uint32_t*)b.take(cap * 4);
  L.best_key = (unsigned long long*)b.take(cap * 8);
  L.best_pid = (unsigned long long*)b.take(cap * 8);
  L.x0d = tmp.hp.has_drift ? b.take(cap * vs) : nullptr;
  L.repx = (RepX*)b.take(sizeof(RepX));
  L.rep_cons = (uint32_t*)b.take(4);
  L.rep_prod = (uint32_t*)b.take(4);
  L.cell_count = (uint32_t*)b.take(cells * 4);
  L.cell_start = (uint32_t*)b.take((cells + 1) * 4);
  L.flag_stride = std::max(nbc, nbp) + 1;
  L.agg32 = (uint32_t*)b.take((nbc + 1) * 4);
  L.incl32 = (uint32_t*)b.take((nbc + 1) * 4);
  L.agg64 = (unsigned long long*)b.take((nbp + 1) * 8);
  L.incl64 = (unsigned long long*)b.take((nbp + 1) * 8);
  L.flags = (uint32_t*)b.take(2 * L.flag_stride * 4);
  L.accepted = (uint32_t*)b.take(pair_cap * 4);
  L.fired = (FiredPair*)b.take(pair_cap * sizeof(FiredPair));
  L.fstate = (uint32_t*)b.take(pair_cap * 4);
  L.conflict = (uint32_t*)b.take(pair_cap * 4);
  L.crec = (ConflictRec*)b.take(pair_cap * sizeof(ConflictRec));
  L.angles = c.angle_mode == 0;
  L.ang_cap = RD_STATIC_MAX_PARTICLES;
  L.ang_jobs = (AngJob*)b.take((size_t)L.ang_cap * sizeof(AngJob));
  L.counts = (unsigned long long*)b.take((size_t)L.n_counts * 8);
  L.P = (const DevParams*)b.take(sizeof(DevParams));
  L.ctl = (DevCtl*)b.take(sizeof(DevCtl));
  L.reps = (RepDev*)b.take(sizeof(RepDev));
  if (!b.ok) return RD_EINVAL;
  L.x_cur = xb0;
  L.x_next = xb1;
  L.id_cur = id0;
  L.id_next = id1;

  // mixed precision: the step reads p_reac and the propagator sample from FP32 tables, built into
  // the scratch array on every call.  Their space is laid out here, before anything is enqueued,
  // so that a table that does not fit is rejected with the outputs untouched.
  struct TableJob {
    int rule, kind, m1;
    double hstep, h1;
    float* t;
    double* tot;
    float4* q4;
    int n0;
  };
  std::vector<TableJob> jobs;
  if (c.precision == RD_MIXED) {
    for (int k = 0; k < c.n_pairs; ++k) {
      if (c.pairs[k].bc == RD_BC_NONE || c.pairs[k].bc == RD_BC_ABS) continue;
      PairDev& q = tmp.hp.pairs[k];
      const double hstep = 0.025 * std::min(q.s, 1.0);
      const double d0max = std::sqrt(q.rcut2) / q.sigma - 1.0 + hstep;
      const double dmax = d0max + 13.0 * q.s + 2.0 * hstep;
      const int n0 = (int)std::ceil(d0max / hstep) + 4, n1 = (int)std::ceil(dmax / hstep) + 4;
      const double hinv = 0.025;
      const int ninv = (int)std::ceil(4.2 / hinv) + 4;
      // only the quad copies are read by the step; the scalar table and the totals are build
      // scratch shared by the tables of one rule (stream order keeps the builds apart)
      float* t = (float*)b.take((size_t)n0 * std::max(n1, ninv) * sizeof(float));
      double* tot = (double*)b.take((size_t)n0 * sizeof(double));
      auto plan = [&](int kind, Tab2& T, int m1, double h1) {
        float4* q4 = (float4*)b.take((size_t)n0 * m1 * sizeof(float4));
        jobs.push_back({k, kind, m1, hstep, h1, t, tot, q4, n0});
        T.v = nullptr;
        T.q = q4;
        T.n0 = n0;
        T.n1 = m1;
        T.h = (float)hstep;
        T.inv_h = (float)(1.0 / hstep);
        T.h1 = (float)h1;
        T.inv_h1 = (float)(1.0 / h1);
      };
      if (c.pairs[k].bc == RD_BC_RAD) plan(0, q.tab_preac, n1, hstep);
      plan(3, q.tab_inv, ninv, hinv);
    }
  }
  if (!b.ok) return RD_EINVAL;

  DevCtl ctl;
  std::memset(&ctl, 0, sizeof ctl);
  ctl.n = (uint32_t)n;
  ctl.step = (uint32_t)step;
  ctl.t = (double)step * c.dt;
  // the array keeps the previous call's contents: reset what the step expects to start at zero
  RD_CUDA(cudaMemsetAsync(L.cell_count, 0, (size_t)cells * 4, s));
  RD_CUDA(cudaMemsetAsync(L.flags, 0, (size_t)(2 * L.flag_stride) * 4, s));
  RD_CUDA(cudaMemsetAsync(L.deg, 0, (size_t)cap * 4, s));
  RD_CUDA(cudaMemsetAsync(L.counts, 0, (size_t)L.n_counts * 8, s));
  RD_CUDA(cudaMemsetAsync(L.rep_cons, 0, 4, s));
  RD_CUDA(cudaMemsetAsync(L.rep_prod, 0, 4, s));
  // the tables are built from the parameter block: first without the table pointers, then the
  // complete block once they are built
  DevParams hp0 = tmp.hp;
  for (int k = 0; k < c.n_pairs; ++k) {
    hp0.pairs[k].tab_preac = Tab2{};
    hp0.pairs[k].tab_inv = Tab2{};
  }
  RD_CUDA(cudaMemcpyAsync((void*)L.P, &hp0, sizeof(DevParams), cudaMemcpyHostToDevice, s));
  for (const TableJob& j : jobs)
    launch_build_table(L.P, j.rule, j.kind, j.t, j.q4, j.n0, j.m1, j.hstep, j.h1, j.tot, nullptr, device_sms(), s);
  if (!jobs.empty()) RD_CUDA(cudaMemcpyAsync((void*)L.P, &tmp.hp, sizeof(DevParams), cudaMemcpyHostToDevice, s));
  RD_CUDA(cudaMemcpyAsync(L.reps, &rep, sizeof rep, cudaMemcpyHostToDevice, s));
  RD_CUDA(cudaMemcpyAsync(L.ctl, &ctl, sizeof ctl, cudaMemcpyHostToDevice, s));
  const int G = (int)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), (int64_t)device_sms() * 8);
  if (n > 0) {
    if (vs == 32)
      k_static_pack<d4><<<G, 256, 0, s>>>(n, c.dim, rp.L, x_in, species_in, id_in, (d4*)xb0, id0);
    else
      k_static_pack<float4><<<G, 256, 0, s>>>(n, c.dim, rp.L, x_in, species_in, id_in, (float4*)xb0, id0);
  }
  launch_step(L, s, nullptr);
  const int Go = (int)std::min<int64_t>(std::max<int64_t>((2 * n + 255) / 256, 1), (int64_t)device_sms() * 8);
  if (vs == 32)
    k_static_unpack<d4><<<Go, 256, 0, s>>>(L.ctl, L.reps, (const d4*)xb1, id1, x_out, species_out, id_out, n_out,
                                           next_id_out, status_out);
  else
    k_static_unpack<float4><<<Go, 256, 0, s>>>(L.ctl, L.reps, (const float4*)xb1, id1, x_out, species_out, id_out,
                                               n_out, next_id_out, status_out);
  RD_CUDA(cudaGetLastError());
  return RD_OK;
}
