// Device kernels of one GF-BD step.  Positions are SoA vectors of 4 components (x, y, z, w) where
// w carries the bits of (species | replica << 8); T = double for the FP64 step, float for the
// mixed step.  Every kernel is a grid-stride loop so that CUDA graphs can be captured with grids
// sized for the capacity while the live particle count stays on the device.
#include <utility>
#include <cuda_runtime.h>

#include <algorithm>

#include "rd_angle.cuh"
#include "rd_gf2d.cuh"
#include "rd_kernels.h"

namespace rd {

// Programmatic dependent launch: a step kernel waits for the whole previous kernel (completion and
// memory visibility) before it touches memory, then lets the next kernel's blocks be scheduled while
// its own blocks run.  Both are no-ops for a launch without a programmatic dependency.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}


// Acquire load / release store of a 32-bit flag at GPU scope (the look-back's and the grid
// barrier's publication protocol: data written before a release store is visible to whoever
// acquires the flag value it stored).
__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <class T> struct V4;
template <> struct V4<double> { using type = d4; };
template <> struct V4<float> { using type = float4; };

__device__ __forceinline__ d4 make_v4(double x, double y, double z, uint32_t wb) {
  d4 v;
  v.x = x; v.y = y; v.z = z; v.w = w_from_bits_d(wb);
  return v;
}
__device__ __forceinline__ float4 make_v4f(float x, float y, float z, uint32_t wb) {
  return make_float4(x, y, z, w_from_bits_f(wb));
}

__device__ __forceinline__ void set_status(DevCtl* ctl, int code) { atomicCAS(&ctl->status, 0, code); }

// Warp-aggregated add of a per-thread value (all 32 lanes must be active).
__device__ __forceinline__ void warp_sum_add(unsigned long long* dst, unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

__device__ __forceinline__ int cell_coord(double x, double inv_edge, int n) {
  int c = (int)(x * inv_edge);
  return c < 0 ? 0 : (c >= n ? n - 1 : c);
}
__device__ __forceinline__ int cell_coord_f(float x, float inv_edge, int n) {
  int c = (int)(x * inv_edge);
  return c < 0 ? 0 : (c >= n ? n - 1 : c);
}


// ------------------------------------------------------------------------------------------------
// dimension dispatch of the pair quantities (2D evaluations are out-of-line: they are long loops)
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ Pair2D pair2d(const PairDev& pr) {
  Pair2D q;
  q.series = pr.series2d != 0;
  q.series_rad = pr.series2d_rad != 0;
  q.tau = pr.tau;
  q.s = pr.s;
  q.h = pr.h;
  q.nodes = pr.nodes;
  q.n_nodes = pr.n_nodes;
  q.ser = pr.ser;
  return q;
}
__device__ __noinline__ double p_enc2_call(const PairDev& pr, double R, double R0) { return p_enc2(pair2d(pr), R, R0); }
__device__ __noinline__ double p_reac2_call(const PairDev& pr, double R, double R0) { return p_reac2(pair2d(pr), R, R0); }
__device__ __noinline__ double resample2_call(const DevParams& P, const PairDev& pr, double U, double R0) {
  return resample2(pair2d(pr), U, R0, P.gl16);
}
__device__ __forceinline__ double p_enc_dim(const DevParams& P, const PairDev& pr, double R, double R0) {
  return P.dim == 3 ? p_enc3(R, R0, pr.inv_tau) : p_enc2_call(pr, R, R0);
}
__device__ __forceinline__ double p_reac_dim(const DevParams& P, const PairDev& pr, double R, double R0) {
  return P.dim == 3 ? p_reac3(R, R0, pr.s, pr.alpha) : p_reac2_call(pr, R, R0);
}
__device__ __forceinline__ double resample_dim(const DevParams& P, const PairDev& pr, double U, double R0) {
  return P.dim == 3 ? resample3(U, R0, pr.s) : resample2_call(P, pr, U, R0);
}

// ================================================================================================
// K0: drift step (deterministic forces, when configured), unimolecular decay draws (start-of-step
// state), free displacement of the other particles, and the first half of the counting sort by
// cell (start-of-step positions).
// ================================================================================================
template <class T>
__device__ __forceinline__ void ph_prepare(const DevParams* Pp, DevCtl* ctl,
                          const RepDev* reps, const typename V4<T>::type* x0,
                          const uint32_t* id, typename V4<T>::type* x1,
                          uint32_t* status, uint32_t* cell_of, uint32_t* slot,
                          uint32_t* cell_count, uint32_t* decay_list,
                          unsigned long long* counts, int n_counts,
                          typename V4<T>::type* x0d, const uint32_t bid, const uint32_t nblk) {
  const DevParams& P = *Pp;
  if (bid == 0) {
    // counters of the step's later kernels (the counters used by this kernel were reset at the
    // end of the previous step)
    for (int k = threadIdx.x; k < n_counts; k += blockDim.x) counts[k] = 0ull;
    if (threadIdx.x == 0) {
      ctl->epoch += 1u;
      ctl->tile_ctr[0] = 0u;
      ctl->tile_ctr[1] = 0u;
    }
  }
  if (ctl->status) return;
  const uint32_t n = ctl->n, step = ctl->step;
  const int dim = P.dim;
  for (uint32_t i = bid * blockDim.x + threadIdx.x; i < n; i += nblk * blockDim.x) {
    auto p = x0[i];
    const uint32_t wb = w_bits(p.w);
    const uint32_t sp = wb & 0xFFu, r = wb >> 8;
    const uint32_t pid = id[i];
    const RepDev& rep = reps[r];
    if (x0d) {
      // deterministic forces as a split step: the drift displacement first; the rest of the step
      // starts from the drifted position (kept in x0d for the later kernels)
      if constexpr (sizeof(T) == 8) {
        p.x = wrap(p.x + P.drift_dx[sp][0], rep.L);
        p.y = wrap(p.y + P.drift_dx[sp][1], rep.L);
        if (dim == 3) p.z = wrap(p.z + P.drift_dx[sp][2], rep.L);
      } else {
        p.x = wrap_f(p.x + P.drift_dx_f[sp][0], rep.Lf);
        p.y = wrap_f(p.y + P.drift_dx_f[sp][1], rep.Lf);
        if (dim == 3) p.z = wrap_f(p.z + P.drift_dx_f[sp][2], rep.Lf);
      }
      x0d[i] = p;
    }
    uint32_t st = 0;
    if (P.ktot[sp] > 0.0) {
      const uint4 w = draw(P, step, pid, kOneParticle, TAG_UNI, r);
      // U = (m + 1/2) 2^-52 < p_uni  <=>  m < ceil(p_uni 2^52 - 1/2), an exact integer test
      const unsigned long long m52 = ((((unsigned long long)w.x) << 32) | w.y) >> 12;
      if (m52 < P.uni_thr[sp]) {
        const double target = u52(w.z, w.w) * P.ktot[sp];
        double acc = 0.0;
        int chosen = -1, last = -1;
        for (int c = 0; c < P.n_decays; ++c) {
          if (P.decays[c].parent != (int)sp) continue;
          last = c;
          acc += P.decays[c].kd;
          if (chosen < 0 && target < acc) chosen = c;
        }
        if (chosen < 0) chosen = last;
        st = ST_DECAYED | ST_CONSUMED | ((uint32_t)chosen << ST_CHANNEL_SHIFT);
        const unsigned m = __activemask();
        const int leader = __ffs(m) - 1;
        uint32_t base = 0;
        if ((int)(threadIdx.x & 31) == leader) base = atomicAdd(&ctl->n_decay, (uint32_t)__popc(m));
        base = __shfl_sync(m, base, leader);
        decay_list[base + __popc(m & ((1u << (threadIdx.x & 31)) - 1u))] = i;
      }
    }
    status[i] = st;
    typename V4<T>::type q = p;
    if (!st) {
      if constexpr (sizeof(T) == 8) {
        double nr[4];
        normals64(P, step, pid, TAG_DISP0, r, dim, nr);
        const double ell = P.ell[sp];
        q.x = wrap(p.x + ell * nr[0], rep.L);
        q.y = wrap(p.y + ell * nr[1], rep.L);
        if (dim == 3) q.z = wrap(p.z + ell * nr[2], rep.L);
      } else {
        const uint4 w = draw(P, step, pid, kOneParticle, TAG_DISP0, r);
        float n0, n1, n2, n3;
        box_muller_f(u23(w.x), u23(w.y), n0, n1);
        const float ell = P.ell_f[sp];
        q.x = wrap_f(p.x + ell * n0, rep.Lf);
        q.y = wrap_f(p.y + ell * n1, rep.Lf);
        if (dim == 3) {
          box_muller_f(u23(w.z), u23(w.w), n2, n3);
          q.z = wrap_f(p.z + ell * n2, rep.Lf);
        }
      }
    }
    x1[i] = q;
    uint32_t cell = kNoCell;
    if (!st && ((P.binned_mask >> sp) & 1u)) {
      int cx, cy, cz = 0;
      if constexpr (sizeof(T) == 8) {
        cx = cell_coord(p.x, rep.inv_edge[0], rep.nc[0]);
        cy = cell_coord(p.y, rep.inv_edge[1], rep.nc[1]);
        if (dim == 3) cz = cell_coord(p.z, rep.inv_edge[2], rep.nc[2]);
      } else {
        cx = cell_coord_f(p.x, rep.inv_edge_f[0], rep.nc[0]);
        cy = cell_coord_f(p.y, rep.inv_edge_f[1], rep.nc[1]);
        if (dim == 3) cz = cell_coord_f(p.z, rep.inv_edge_f[2], rep.nc[2]);
      }
      cell = (uint32_t)(rep.cell_base + ((int64_t)cz * rep.nc[1] + cy) * rep.nc[0] + cx);
      slot[i] = atomicAdd(&cell_count[cell], 1u);
    }
    cell_of[i] = cell;
  }
}

template <class T>
__global__ void k_prepare(const DevParams* __restrict__ Pp, DevCtl* __restrict__ ctl,
                          const RepDev* __restrict__ reps, const typename V4<T>::type* __restrict__ x0,
                          const uint32_t* __restrict__ id, typename V4<T>::type* __restrict__ x1,
                          uint32_t* __restrict__ status, uint32_t* __restrict__ cell_of, uint32_t* __restrict__ slot,
                          uint32_t* __restrict__ cell_count, uint32_t* __restrict__ decay_list,
                          unsigned long long* __restrict__ counts, int n_counts,
                          typename V4<T>::type* __restrict__ x0d) {
  pdl_enter();
  ph_prepare<T>(Pp, ctl, reps, x0, id, x1, status, cell_of, slot, cell_count, decay_list, counts, n_counts, x0d,
                blockIdx.x, gridDim.x);
}

// ================================================================================================
// Block-level exclusive scan and the per-element loaders of the two scans of a step.
// ================================================================================================
template <class U, class Load>
__device__ __forceinline__ U block_exclusive_scan(U v, U* smem, U& total) {
  // smem: blockDim.x/32 entries
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  U x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const U y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem[wid] = x;
  __syncthreads();
  if (wid == 0) {
    U s = lane < nw ? smem[lane] : U(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const U y = __shfl_up_sync(0xFFFFFFFFu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) smem[lane] = s;
  }
  __syncthreads();
  total = smem[nw - 1];
  const U warp_off = wid ? smem[wid - 1] : U(0);
  __syncthreads();
  return warp_off + x - v;
}

struct LoadCellCount {
  const uint32_t* cnt;
  // 8 consecutive elements starting at i (i % 8 == 0); elements >= n read as 0
  __device__ __forceinline__ void load8(int64_t i, int64_t n, uint32_t v[8]) const {
    if (i + 8 <= n) {
      const uint4 a = __ldcg(reinterpret_cast<const uint4*>(cnt + i));
      const uint4 b = __ldcg(reinterpret_cast<const uint4*>(cnt + i) + 1);
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = i + k < n ? cnt[i + k] : 0u;
    }
  }
};

struct LoadCompact {
  const uint32_t* status;
  __device__ __forceinline__ static unsigned long long conv(uint32_t s) {
    const unsigned long long surv = (s & ST_CONSUMED) ? 0ull : 1ull;
    const unsigned long long np = (s >> ST_NPROD_SHIFT) & 3u;
    return (surv << 32) | np;
  }
  __device__ __forceinline__ void load8(int64_t i, int64_t n, unsigned long long v[8]) const {
    if (i + 8 <= n) {
      const uint4 a = __ldcg(reinterpret_cast<const uint4*>(status + i));
      const uint4 b = __ldcg(reinterpret_cast<const uint4*>(status + i) + 1);
      v[0] = conv(a.x); v[1] = conv(a.y); v[2] = conv(a.z); v[3] = conv(a.w);
      v[4] = conv(b.x); v[5] = conv(b.y); v[6] = conv(b.z); v[7] = conv(b.w);
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = i + k < n ? conv(status[i + k]) : 0ull;
    }
  }
};

constexpr int kScanItems = 8;
constexpr uint32_t kSpinLimit = 1u << 24;

// Decoupled look-back of one tile, run by warp 0 of its block: publishes the tile's aggregate, sums
// the predecessors' published values back to the nearest inclusive prefix (windows of 32 tiles at
// once; a predecessor that does not publish within kSpinLimit polls sets RD_ETIMEOUT), publishes
// the tile's inclusive prefix and returns the exclusive prefix (in every lane).  Flags carry an
// epoch that changes every scan, so nothing needs clearing.
template <class U>
__device__ __forceinline__ U tile_lookback(U tot, uint32_t tile, uint32_t epoch, U* agg,
                                           U* incl, uint32_t* flag, DevCtl* ctl) {
  const int lane = threadIdx.x & 31;
  U prefix = 0;
  if (tile > 0) {
    if (lane == 0) {
      agg[tile] = tot;
      st_release_gpu(&flag[tile], (epoch << 2) | 1u);
    }
    int64_t top = (int64_t)tile - 1;
    uint32_t spins = 0;
    const uint32_t limit = ctl->spin_limit ? ctl->spin_limit : kSpinLimit;
    for (;;) {
      const int64_t q = top - lane;
      // acquire: a flag seen set makes the value published before it visible
      const uint32_t f = q >= 0 ? ld_acquire_gpu(&flag[q]) : ((epoch << 2) | 2u);
      const bool ready = (f >> 2) == epoch && (f & 3u) != 0u;
      if (!__all_sync(0xFFFFFFFFu, ready)) {
        if (++spins > limit) {
          if (lane == 0) set_status(ctl, RD_ETIMEOUT);
          break;
        }
        continue;
      }
      const unsigned incl_mask = __ballot_sync(0xFFFFFFFFu, q >= 0 && (f & 3u) == 2u);
      const int stop = incl_mask ? __ffs(incl_mask) - 1 : 32;   // nearest inclusive predecessor
      U vv = 0;
      if (q >= 0 && lane <= stop) vv = lane == stop ? *(volatile U*)&incl[q] : *(volatile U*)&agg[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) vv += __shfl_xor_sync(0xFFFFFFFFu, vv, o);
      prefix += vv;
      if (incl_mask || top < 32) break;
      top -= 32;
    }
  }
  if (lane == 0) {
    incl[tile] = prefix + tot;
    st_release_gpu(&flag[tile], (epoch << 2) | 2u);
  }
  return prefix;
}

// Single-pass exclusive scan with decoupled look-back (Merrill & Garland, 2016).  Tiles of
// blockDim x kScanItems elements take tickets in launch order; each publishes its aggregate, then
// walks back over its predecessors' published values (bounded wait: a stalled predecessor sets
// RD_ETIMEOUT).  Flags carry an epoch that changes every scan, so nothing needs clearing.
// out[i] = exclusive prefix for i < n, out[n] = total; zero_after (optional) is cleared behind.

// One tile of the scan, taken by ticket (tile < ntiles).  Returns false when the tickets are used up.
template <class U, class Load>
__device__ __forceinline__ bool ph_scan_tile(Load load, int64_t n_const, const uint32_t* n_ptr,
                                             U* out, uint32_t* zero_after,
                                             U* agg, U* incl,
                                             uint32_t* flag, DevCtl* ctl, int which) {
  __shared__ U sm[32];
  __shared__ uint32_t s_tile;
  __shared__ U s_prefix;
  if (threadIdx.x == 0) s_tile = atomicAdd(&ctl->tile_ctr[which], 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  __syncthreads();
  const int64_t n = n_ptr ? (int64_t)*n_ptr : n_const;
  const int64_t tile_elems = (int64_t)blockDim.x * kScanItems;
  const int64_t ntiles = n > 0 ? (n + tile_elems - 1) / tile_elems : 1;
  if ((int64_t)tile >= ntiles) return false;
  const uint32_t epoch = (ctl->epoch * 2u + (uint32_t)which) & 0x3FFFFFFFu;
  const int64_t base = (int64_t)tile * tile_elems + (int64_t)threadIdx.x * kScanItems;
  // blocked arrangement: each thread owns kScanItems consecutive elements
  U v[kScanItems];
  load.load8(base, n, v);
  U ex[kScanItems];
  U run = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    ex[k] = run;
    run += v[k];
  }
  U tot;
  const U toff = block_exclusive_scan<U, Load>(run, sm, tot);
  if (threadIdx.x < 32) {
    const U prefix = tile_lookback<U>(tot, tile, epoch, agg, incl, flag, ctl);
    if (threadIdx.x == 0) s_prefix = prefix;
  }
  __syncthreads();
  const U prefix = s_prefix + toff;
  if (base + kScanItems <= n) {
    U o[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) o[k] = prefix + ex[k];
    uint4* dst = reinterpret_cast<uint4*>(out + base);
    const uint4* src = reinterpret_cast<const uint4*>(o);
#pragma unroll
    for (int k = 0; k < (int)(kScanItems * sizeof(U) / 16); ++k) dst[k] = src[k];
    if (zero_after) {
      uint4* z = reinterpret_cast<uint4*>(zero_after + base);
      z[0] = make_uint4(0u, 0u, 0u, 0u);
      z[1] = make_uint4(0u, 0u, 0u, 0u);
    }
  } else {
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const int64_t i = base + k;
      if (i < n) {
        out[i] = prefix + ex[k];
        if (zero_after) zero_after[i] = 0u;
      }
    }
  }
  if (threadIdx.x == 0 && (int64_t)tile == ntiles - 1) out[n > 0 ? n : 0] = s_prefix + tot;
  __syncthreads();
  return true;
}

template <class U, class Load>
__global__ void __launch_bounds__(256) k_scan1(Load load, int64_t n_const, const uint32_t* __restrict__ n_ptr,
                                               U* __restrict__ out, uint32_t* __restrict__ zero_after,
                                               U* __restrict__ agg, U* __restrict__ incl,
                                               uint32_t* __restrict__ flag, DevCtl* __restrict__ ctl, int which) {
  pdl_enter();
  ph_scan_tile<U, Load>(load, n_const, n_ptr, out, zero_after, agg, incl, flag, ctl, which);
}

// ================================================================================================
// K2: scatter of the binned particles into cell order: start-of-step position (w = species bits),
// end-of-free-step position (w = id bits) and the particle index.
// ================================================================================================
template <class T>
__device__ __forceinline__ void ph_scatter(const DevCtl* ctl, const typename V4<T>::type* x0,
                                const typename V4<T>::type* x1, const uint32_t* id,
                                const uint32_t* cell_of, const uint32_t* slot,
                                const uint32_t* cell_start,
                                typename V4<T>::type* sx0, typename V4<T>::type* sx1,
                                uint32_t* sidx, const uint32_t bid, const uint32_t nblk) {
  if (ctl->status) return;
  const uint32_t n = ctl->n;
  for (uint32_t i = bid * blockDim.x + threadIdx.x; i < n; i += nblk * blockDim.x) {
    const uint32_t c = cell_of[i];
    if (c == kNoCell) continue;
    const uint32_t k = cell_start[c] + slot[i];
    sx0[2 * (size_t)k] = x0[i];
    auto q = x1[i];
    if constexpr (sizeof(T) == 8)
      q.w = w_from_bits_d(id[i]);
    else
      q.w = w_from_bits_f(id[i]);
    sx1[2 * (size_t)k] = q;
    sidx[k] = i;
  }
}

template <class T>
__global__ void k_scatter_cells(const DevCtl* __restrict__ ctl, const typename V4<T>::type* __restrict__ x0,
                                const typename V4<T>::type* __restrict__ x1, const uint32_t* __restrict__ id,
                                const uint32_t* __restrict__ cell_of, const uint32_t* __restrict__ slot,
                                const uint32_t* __restrict__ cell_start,
                                typename V4<T>::type* __restrict__ sx0, typename V4<T>::type* __restrict__ sx1,
                                uint32_t* __restrict__ sidx) {
  pdl_enter();
  ph_scatter<T>(ctl, x0, x1, id, cell_of, slot, cell_start, sx0, sx1, sidx, blockIdx.x, gridDim.x);
}

// ================================================================================================
// K3: cell sweep.  One thread per binned particle (cell order) walks the forward half of the
// 27-cell (3D) / 9-cell (2D) neighbourhood; every pair (k, j > k) of an interacting species pair
// whose start-of-step minimum-image distance is below r_cut is a candidate: p_enc from the start and
// end separations, U_enc < p_enc fires and the pair is appended with a warp-aggregated atomic.
// In cell order the three cells x-1..x+1 of a row are one contiguous particle range, so the half
// stencil is five row ranges (3D: own row from k+1 through x+1, row y+1, the three rows of layer
// z+1; 2D: the first two), each split in two where the row wraps around x.
// ================================================================================================
constexpr int kSweepRanges = 10;

template <class T, bool kSplit, int kReach>
__device__ __forceinline__ void ph_sweep(const DevParams* Pp, DevCtl* ctl,
                                         const RepDev* reps,
                                         const typename V4<T>::type* sx0,
                                         const typename V4<T>::type* sx1,
                                         const uint32_t* sidx,
                                         const uint32_t* cell_start,
                                         const int64_t total_cells, FiredPair* fired,
                                         uint32_t* fstate, uint32_t* deg,
                                         int32_t* matched, const uint32_t cap_pairs,
                                         const uint32_t split, uint2 (*ranges)[256],
                                         const uint32_t bid, const uint32_t nblk) {
  using V = typename V4<T>::type;
  // per-warp queue of (particle, candidate) pairs that passed the cut-off test
  __shared__ uint2 s_queue[8][64];
  const DevParams& P = *Pp;
  if (ctl->status) return;
  const uint32_t nb = cell_start[total_cells];
  const uint32_t step = ctl->step;
  const int dim = P.dim;
  const int lane = threadIdx.x & 31;
  uint2* queue = s_queue[threadIdx.x >> 5];
  uint32_t qc = 0;   // entries in this warp's queue (the same in every lane)
  unsigned long long n_cand = 0, n_near = 0, n_overlap = 0;

  // One candidate pair (k, jj) within the cut-off: p_enc, the encounter draw, the append.
  auto process = [&](const uint32_t k, const uint32_t jj) {
    const auto a0 = sx0[2 * (size_t)k];
    const auto a1 = sx1[2 * (size_t)k];
    const uint32_t wa = w_bits(a0.w);
    const uint32_t spa = wa & 0xFFu, r = wa >> 8;
    const uint32_t ida = w_bits(a1.w);
    const RepDev& rep = reps[r];
    const auto b0 = sx0[2 * (size_t)jj];
        // start-of-step separation first (the norm does not depend on the pair's orientation),
        // against the largest cut-off; the species pair and its own cut-off after that
        double p, r02;
        float pf = 0.0f, r02f = 0.0f;
        if constexpr (sizeof(T) == 8) {
          const double r0x = min_image(b0.x - a0.x, rep.L, rep.half_L);
          const double r0y = min_image(b0.y - a0.y, rep.L, rep.half_L);
          const double r0z = dim == 3 ? min_image(b0.z - a0.z, rep.L, rep.half_L) : 0.0;
          r02 = norm2_rn(r0x, r0y, r0z, dim);
          if (!(r02 < P.rcut2_max)) return;
        } else {
          const float r0x = min_image_f(b0.x - a0.x, rep.Lf, rep.half_Lf);
          const float r0y = min_image_f(b0.y - a0.y, rep.Lf, rep.half_Lf);
          const float r0z = dim == 3 ? min_image_f(b0.z - a0.z, rep.Lf, rep.half_Lf) : 0.0f;
          r02f = r0x * r0x + r0y * r0y + r0z * r0z;
          if (!(r02f < P.rcut2_max_f)) return;
        }
        const uint32_t spb = w_bits(b0.w) & 0xFFu;
        const int rule = P.pair_of[spa][spb];
        if (rule < 0) return;
        const PairDev& pr = P.pairs[rule];
        if constexpr (sizeof(T) == 8) {
          if (!(r02 < pr.rcut2)) return;
        } else {
          if (!(r02f < pr.rcut2_f)) return;
        }
        const auto b1 = sx1[2 * (size_t)jj];
        const uint32_t idb = w_bits(b1.w);
        // orient the pair from the lower id to the higher id
        const bool swap = idb < ida;
        const uint32_t id_lo = swap ? idb : ida, id_hi = swap ? ida : idb;
        bool overlap;
        if constexpr (sizeof(T) == 8) {
          const double rx = min_image(b1.x - a1.x, rep.L, rep.half_L);
          const double ry = min_image(b1.y - a1.y, rep.L, rep.half_L);
          const double rz = dim == 3 ? min_image(b1.z - a1.z, rep.L, rep.half_L) : 0.0;
          const double R0 = sqrt(r02) / pr.sigma;
          const double R = sqrt(norm2_rn(rx, ry, rz, dim)) / pr.sigma;
          overlap = R <= 1.0;
          p = p_enc_dim(P, pr, R, R0);
        } else {
          const float rx = min_image_f(b1.x - a1.x, rep.Lf, rep.half_Lf);
          const float ry = min_image_f(b1.y - a1.y, rep.Lf, rep.half_Lf);
          const float rz = dim == 3 ? min_image_f(b1.z - a1.z, rep.Lf, rep.half_Lf) : 0.0f;
          const float d0 = (sqrtf(r02f) - pr.sigma_f) * pr.inv_sigma_f;
          const float d = (sqrtf(rx * rx + ry * ry + rz * rz) - pr.sigma_f) * pr.inv_sigma_f;
          overlap = d <= 0.0f;
          if (dim == 3) {
            pf = p_enc3_f(d, d0, pr.inv_tau_f);
          } else if (d <= 0.0f || d0 <= 0.0f) {
            pf = 1.0f;
          } else {
            const float xx = d * d0 * pr.inv_tau_f;
            pf = xx > 60.0f ? 0.0f : fminf(1.0f, fmaxf(0.0f, tab_eval(pr.tab_penc, d0, d) * expf(-xx)));
          }
          p = (double)pf;
        }
        ++n_cand;
        n_overlap += overlap;
        // mixed step: FP32 draw and comparison; the smallest FP32 uniform is 2^-24, so a smaller
        // p_enc cannot fire and needs no draw
        if constexpr (sizeof(T) == 4) {
          if (!(pf > 0x1p-24f)) return;
        }
        const uint4 w = draw(P, step, id_lo, id_hi, TAG_ENC, r);
        bool fires;
        if constexpr (sizeof(T) == 8) {
          const double u_enc = u52(w.x, w.y);
          n_near += fabs(u_enc - p) <= 1e-9;
          fires = u_enc < p;
        } else {
          fires = u23(w.x) < pf;
        }
        if (fires) {
          const unsigned m = __activemask();
          const int lane = threadIdx.x & 31;
          const int leader = __ffs(m) - 1;
          uint32_t base = 0;
          if (lane == leader) base = atomicAdd(&ctl->fired, (uint32_t)__popc(m));
          base = __shfl_sync(m, base, leader);
          const uint32_t pos = base + __popc(m & ((1u << lane) - 1u));
          if (pos < cap_pairs) {
            FiredPair f;
            const uint32_t ia = sidx[k], ib = sidx[jj];
            f.ia = swap ? ib : ia;
            f.ib = swap ? ia : ib;
            f.ida = id_lo;
            f.idb = id_hi;
            f.p = p;
            if constexpr (sizeof(T) == 8)
              f.key = -log(u52(w.z, w.w)) / p;
            else
              f.key = (double)(-logf(u23(w.z)) / pf);
            fired[pos] = f;
            fstate[pos] = FS_LIVE | ((uint32_t)rule << 2) | (r << 8);
            matched[f.ia] = -1;
            matched[f.ib] = -1;
            atomicAdd(&deg[f.ia], 1u);
            atomicAdd(&deg[f.ib], 1u);
          } else {
            set_status(ctl, RD_ECAPACITY);
          }
        }
  };

  // Walks one particle's candidates and queues those within the cut-off; whenever the warp's
  // queue holds 32 pairs, all lanes process one each.  (Examining a candidate is cheap, processing
  // one is not: processed where it is found, the expensive part would run once per loop iteration
  // in which any lane found one.)
  // split = 1: one thread walks all rows of a particle; split = number of rows: one thread per
  // (particle, row), more independent chains for small systems (the host keeps nb * split < 2^32)
  const uint32_t work = kSplit ? nb * split : nb;
  const uint32_t stride = nblk * blockDim.x;
  const uint32_t n_iter = (work + stride - 1) / stride;
  for (uint32_t it = 0; it < n_iter; ++it) {
    const uint32_t t = it * stride + bid * blockDim.x + threadIdx.x;
    int nr = 0;
    uint32_t k = 0;
    V a0{};
    float4 cut{};   // (L, half L, largest squared cut-off) of the particle's replica, FP32 step
    double Ld = 0.0, hLd = 0.0;
    uint32_t spa = 0;
    if (t < work) {
      k = kSplit ? t / split : t;
      const int row_lo = kSplit ? (int)(t - k * split) : 0;
      // rows of the half stencil: reach 1 (cell edge >= r_cut): 5 in 3D, 2 in 2D; reach 2 (2D only,
      // cell edge >= r_cut / 2): rows y, y+1, y+2, each x-2 .. x+2 (own row x .. x+2)
      constexpr int kRows = kReach == 2 ? 3 : kSweepRanges / 2;
      const int row_hi = kSplit ? row_lo + 1 : kRows;
      a0 = sx0[2 * (size_t)k];
      const uint32_t wa = w_bits(a0.w);
      spa = wa & 0xFFu;
      const uint32_t r = wa >> 8;
      const RepDev& rep = reps[r];
      int cx, cy, cz = 0;
      if constexpr (sizeof(T) == 8) {
        cx = cell_coord(a0.x, rep.inv_edge[0], rep.nc[0]);
        cy = cell_coord(a0.y, rep.inv_edge[1], rep.nc[1]);
        if (dim == 3) cz = cell_coord(a0.z, rep.inv_edge[2], rep.nc[2]);
      } else {
        cx = cell_coord_f(a0.x, rep.inv_edge_f[0], rep.nc[0]);
        cy = cell_coord_f(a0.y, rep.inv_edge_f[1], rep.nc[1]);
        if (dim == 3) cz = cell_coord_f(a0.z, rep.inv_edge_f[2], rep.nc[2]);
      }
      const int nc0 = rep.nc[0];
      // the grid has 1 or >= 2 kReach + 1 cells along each axis; with 1 only the own cell counts
      constexpr int kMinCells = 2 * kReach + 1;
      const bool ox = nc0 >= kMinCells, oy = rep.nc[1] >= kMinCells, oz = dim == 3 && rep.nc[2] >= kMinCells;
      // all row ranges first (independent loads in flight together), the non-empty ones kept in
      // order, then one flattened walk over them
#pragma unroll
      for (int row = 0; row < kRows; ++row) {
        const int dy = kReach == 2 ? row : (row == 0 ? 0 : (row == 1 ? 1 : row - 3));
        const int dz = (kReach == 2 || row < 2) ? 0 : 1;
        if (row >= row_lo && row < row_hi && (dy == 0 || oy) && (dz == 0 || oz)) {
          int yy = cy + dy, zz = cz + dz;
          yy = yy < 0 ? yy + rep.nc[1] : (yy >= rep.nc[1] ? yy - rep.nc[1] : yy);
          zz = zz >= rep.nc[2] ? zz - rep.nc[2] : zz;
          const int64_t rowc = rep.cell_base + ((int64_t)zz * rep.nc[1] + yy) * nc0;
          const int xl = (row == 0 || !ox) ? cx : max(cx - kReach, 0);
          const int xh = ox ? min(cx + kReach, nc0 - 1) : cx;
          const uint2 main_rg = make_uint2(row == 0 ? k + 1 : cell_start[rowc + xl], cell_start[rowc + xh + 1]);
          uint2 wrap_rg = make_uint2(0u, 0u);
          if (ox && row != 0 && cx - kReach < 0)          // cells nc0 + cx - kReach .. nc0 - 1
            wrap_rg = make_uint2(cell_start[rowc + nc0 + cx - kReach], cell_start[rowc + nc0]);
          else if (ox && cx + kReach >= nc0)               // cells 0 .. cx + kReach - nc0
            wrap_rg = make_uint2(cell_start[rowc], cell_start[rowc + cx + kReach - nc0 + 1]);
          if (main_rg.y > main_rg.x) ranges[nr++][threadIdx.x] = main_rg;
          if (wrap_rg.y > wrap_rg.x) ranges[nr++][threadIdx.x] = wrap_rg;
        }
      }
      Ld = rep.L;
      hLd = rep.half_L;
      cut = make_float4(rep.Lf, rep.half_Lf, 0.0f, 0.0f);
    }
    int rr = 0;
    uint2 rg = nr > 0 ? ranges[0][threadIdx.x] : make_uint2(0u, 0u);
    uint32_t j = rg.x;
    for (;;) {
      const bool more = rr < nr;
      if (!__any_sync(0xFFFFFFFFu, more)) break;
      bool push = false;
      uint32_t jj = 0;
      if (more) {
        jj = j++;
        if (j >= rg.y && ++rr < nr) {
          rg = ranges[rr][threadIdx.x];
          j = rg.x;
        }
        // the cut-off tests of process(), which repeats them
        const auto b0 = sx0[2 * (size_t)jj];
        bool in;
        if constexpr (sizeof(T) == 8) {
          const double r0x = min_image(b0.x - a0.x, Ld, hLd);
          const double r0y = min_image(b0.y - a0.y, Ld, hLd);
          const double r0z = dim == 3 ? min_image(b0.z - a0.z, Ld, hLd) : 0.0;
          const double r02 = norm2_rn(r0x, r0y, r0z, dim);
          in = r02 < P.rcut2_max;
          if (in) {
            const int rule = P.pair_of[spa][w_bits(b0.w) & 0xFFu];
            in = rule >= 0 && r02 < P.pairs[rule].rcut2;
          }
        } else {
          const float r0x = min_image_f(b0.x - a0.x, cut.x, cut.y);
          const float r0y = min_image_f(b0.y - a0.y, cut.x, cut.y);
          const float r0z = dim == 3 ? min_image_f(b0.z - a0.z, cut.x, cut.y) : 0.0f;
          const float r02f = r0x * r0x + r0y * r0y + r0z * r0z;
          in = r02f < P.rcut2_max_f;
          if (in) {
            const int rule = P.pair_of[spa][w_bits(b0.w) & 0xFFu];
            in = rule >= 0 && r02f < P.pairs[rule].rcut2_f;
          }
        }
        push = in;
      }
      const unsigned bal = __ballot_sync(0xFFFFFFFFu, push);
      if (push) queue[qc + __popc(bal & ((1u << lane) - 1u))] = make_uint2(k, jj);
      qc += __popc(bal);
      __syncwarp();
      if (qc >= 32) {
        const uint2 e = queue[lane];
        __syncwarp();
        if (lane + 32 < (int)qc) queue[lane] = queue[lane + 32];
        qc -= 32;
        __syncwarp();
        process(e.x, e.y);
      }
    }
  }
  // the rest of the queue
  __syncwarp();
  if (lane < (int)qc) {
    const uint2 e = queue[lane];
    process(e.x, e.y);
  }
  warp_sum_add(&ctl->stats[RD_STAT_CANDIDATES], n_cand);
  warp_sum_add(&ctl->stats[RD_STAT_NEAR_THRESHOLD], n_near);
  warp_sum_add(&ctl->stats[RD_STAT_OVERLAPS], n_overlap);
}

template <class T, bool kSplit, int kReach>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 4 : 5) k_sweep(const DevParams* __restrict__ Pp, DevCtl* __restrict__ ctl,
                                                  const RepDev* __restrict__ reps,
                                                  const typename V4<T>::type* __restrict__ sx0,
                                                  const typename V4<T>::type* __restrict__ sx1,
                                                  const uint32_t* __restrict__ sidx,
                                                  const uint32_t* __restrict__ cell_start,
                                                  const int64_t total_cells, FiredPair* __restrict__ fired,
                                                  uint32_t* __restrict__ fstate, uint32_t* __restrict__ deg,
                                                  int32_t* __restrict__ matched, const uint32_t cap_pairs,
                                                  const uint32_t split) {
  pdl_enter();
  __shared__ uint2 ranges[kSweepRanges][256];
  ph_sweep<T, kSplit, kReach>(Pp, ctl, reps, sx0, sx1, sidx, cell_start, total_cells, fired, fstate, deg, matched,
                              cap_pairs, split, ranges, blockIdx.x, gridDim.x);
}

// ================================================================================================
// K4: conflict resolution.  Pairs whose two particles fired with nobody else are accepted at once;
// the rest go through rounds of locally-dominant matching (a pair is accepted when its
// (key, id_a, id_b) is the smallest at both particles among the live pairs), which reproduces the
// greedy acceptance in ascending (key, id_a, id_b).
// ================================================================================================
__device__ __forceinline__ void append_accepted(DevCtl* ctl, uint32_t* accepted, uint32_t e) {
  const unsigned m = __activemask();
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(&ctl->n_accept, (uint32_t)__popc(m));
  base = __shfl_sync(m, base, leader);
  accepted[base + __popc(m & ((1u << lane) - 1u))] = e;
}

__device__ __forceinline__ void ph_match_trivial(DevCtl* ctl, const FiredPair* fired,
                                uint32_t* fstate, const uint32_t* deg,
                                int32_t* matched, uint32_t* conflict,
                                uint32_t* accepted,
                                unsigned long long* best_key,
                                unsigned long long* best_pid, uint32_t cap_pairs,
                                ConflictRec* crec, const uint32_t bid, const uint32_t nblk) {
  if (ctl->status) return;
  const uint32_t nf = min(ctl->fired, cap_pairs);
  unsigned long long acc = 0;
  const uint32_t stride = nblk * blockDim.x;
  const uint32_t n_iter = (nf + stride - 1) / stride;
  for (uint32_t it = 0; it < n_iter; ++it) {
    const uint32_t e = it * stride + bid * blockDim.x + threadIdx.x;
    if (e < nf) {
      const FiredPair f = fired[e];
      if (deg[f.ia] == 1u && deg[f.ib] == 1u) {
        matched[f.ia] = (int32_t)f.ib;
        matched[f.ib] = (int32_t)f.ia;
        fstate[e] = (fstate[e] & ~3u) | FS_ACCEPTED;
        append_accepted(ctl, accepted, e);
        ++acc;
      } else {
        const unsigned m = __activemask();
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(m) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(&ctl->n_conflict, (uint32_t)__popc(m));
        base = __shfl_sync(m, base, leader);
        const uint32_t q = base + __popc(m & ((1u << lane) - 1u));
        conflict[q] = e;
        ConflictRec c;
        c.e = e;
        c.ia = f.ia;
        c.ib = f.ib;
        c.st = FS_LIVE;
        c.key = (unsigned long long)__double_as_longlong(f.key);
        c.pid = ((unsigned long long)f.ida << 32) | f.idb;
        crec[q] = c;
        best_key[f.ia] = ~0ull;
        best_key[f.ib] = ~0ull;
        best_pid[f.ia] = ~0ull;
        best_pid[f.ib] = ~0ull;
      }
    }
  }
  warp_sum_add(&ctl->stats[RD_STAT_MATCHED], acc);
}

// Grid-wide barrier of the cooperative matching launch (every block resident).  Bounded: a block
// that waits longer than kBarrierSpin polls sets RD_ETIMEOUT and leaves; the caller then stops.
constexpr uint32_t kBarrierSpin = 1u << 22;

// check_status: also report a status latched by any block (the matching rounds stop on it); the
// fused step's barriers between phases report only their own timeout (a latched error still lets
// the step reach its compaction, which then keeps the old state).
// Arrival counts with acquire-release semantics instead of full fences: the __syncthreads before
// thread 0's arrival orders the block's writes before it, the release publishes them, the last
// arrival acquires every other block's arrival and releases the new generation, and each waiter
// acquires the generation before the closing __syncthreads hands the data to its block.  Waiters
// poll without sleeping for the first polls (the common wait is a few hundred nanoseconds).
__device__ __forceinline__ bool grid_barrier(DevCtl* ctl, bool check_status = true) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t g = ld_acquire_gpu(&ctl->bar_gen);
    int ok = 1;
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(&ctl->bar_count) : "memory");
    if (old == gridDim.x - 1) {
      asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(&ctl->bar_count) : "memory");
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&ctl->bar_gen) : "memory");
    } else {
      uint32_t spins = 0;
      const uint32_t limit = ctl->spin_limit ? ctl->spin_limit : kBarrierSpin;
      while (ld_acquire_gpu(&ctl->bar_gen) == g) {
        if (++spins > limit) {
          set_status(ctl, RD_ETIMEOUT);
          ok = 0;
          break;
        }
        if (spins > 64) __nanosleep(64);
        // a block that gave up at an earlier barrier never arrives: leave as soon as it is known
        if ((spins & 1023u) == 0 && *(volatile int32_t*)&ctl->status == RD_ETIMEOUT) {
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok && (!check_status || *(volatile int32_t*)&ctl->status == 0);
  }
  __syncthreads();
  return s_ok != 0;
}

// ================================================================================================

// Out-of-line copies of the random draw, the propagator samples, the normals and the p_reac
// table for the resolution path: its items are few and each runs a long straight code path once,
// so one shared copy of each keeps the instruction footprint small.  (The cell sweep keeps the
// inlined forms.)
__device__ __noinline__ uint4 draw_ni(const DevParams& P, uint32_t c0, uint32_t ida, uint32_t idb, uint32_t tag,
                                      uint32_t replica) {
  return draw(P, c0, ida, idb, tag, replica);
}
__device__ __noinline__ double resample_dim_ni(const DevParams& P, const PairDev& pr, double U, double R0) {
  return resample_dim(P, pr, U, R0);
}
__device__ __noinline__ float p_reac_tab_ni(const PairDev& pr, float d, float d0) { return p_reac_tab(pr, d, d0); }
__device__ __noinline__ void normals64_ni(const DevParams& P, uint32_t c0, uint32_t id, uint32_t tag0, uint32_t r,
                                          int dim, double n[4]) {
  normals64(P, c0, id, tag0, r, dim, n);
}

// Resolution of an accepted pair (device functions of K5; Section 3, steps 2(a)-(c)).  Absorbing:
// react.  Reflective / radiation: new separation length from the radial propagator G_ref - G_abs
// (direction of the free step kept, centre of diffusion unchanged); radiation reacts with p_reac
// (Eq. psurv_radII).  A product sits at the centre of diffusion (Eq. Rcoo).  FP64 step first, the
// mixed step's forms further down.
// ================================================================================================
template <class T>
__device__ __forceinline__ void load3(const typename V4<T>::type& v, double o[3]) {
  o[0] = (double)v.x; o[1] = (double)v.y; o[2] = (double)v.z;
}

// Stores one position record (x, y, z and the species/replica bits).  An FP64 record goes out as
// two 16-byte halves: built with nvcc 13.0 for sm_103a, a whole 32-byte record assignment in the
// out-of-line resolver kept only its x component in the separately launched resolution kernel
// (the same code inside the cooperative step launch stored all four).
template <class T>
__device__ __forceinline__ void put4(typename V4<T>::type* p, const double a[3], uint32_t wb) {
  if constexpr (sizeof(T) == 8) {
    double2* q = reinterpret_cast<double2*>(p);
    q[0] = make_double2(a[0], a[1]);
    q[1] = make_double2(a[2], w_from_bits_d(wb));
  } else {
    *p = make_v4f((float)a[0], (float)a[1], (float)a[2], wb);
  }
}

// Appends an angle job: the angle pass draws the pair's new direction and places its particles.
__device__ __forceinline__ void push_ang_job(DevCtl* ctl, AngJob* jobs, uint32_t cap,
                                             const AngJob& job) {
  const uint32_t k = atomicAdd(&ctl->n_ang, 1u);
  if (k < cap)
    jobs[k] = job;
  else
    set_status(ctl, RD_ECAPACITY);
}

template <class T>
__device__ __forceinline__ void resolve_pair(const DevParams& P, const RepDev* reps,
                                             const FiredPair* fired, const uint32_t* fstate,
                                             uint32_t e, uint32_t step, const typename V4<T>::type* x0,
                                             typename V4<T>::type* x1, uint32_t* status,
                                             typename V4<T>::type* prodpos, unsigned long long& n_react,
                                             unsigned long long& n_res, unsigned long long& n_near,
                                             DevCtl* ctl, AngJob* jobs, uint32_t job_cap) {
  const int dim = P.dim;
    const uint32_t fs = fstate[e];
    const FiredPair f = fired[e];
    const int rule = (fs >> 2) & 63u;
    const uint32_t r = fs >> 8;
    const PairDev& pr = P.pairs[rule];
    const RepDev& rep = reps[r];
    const auto pa1 = x1[f.ia], pb1 = x1[f.ib];
    const auto pa0 = x0[f.ia], pb0 = x0[f.ib];
    const uint32_t wa = w_bits(pa1.w), wb = w_bits(pb1.w);
    const int spa = wa & 0xFF, spb = wb & 0xFF;
    double a1[3], b1[3], a0[3], b0[3];
    load3<T>(pa1, a1); load3<T>(pb1, b1); load3<T>(pa0, a0); load3<T>(pb0, b0);
    const double Drel = P.D[spa] + P.D[spb];
    const double ca = P.D[spa] / Drel, cb = P.D[spb] / Drel;
    double rv[3] = {0, 0, 0}, r0v[3] = {0, 0, 0}, c[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) {
      rv[d] = min_image(b1[d] - a1[d], rep.L, rep.half_L);
      r0v[d] = min_image(b0[d] - a0[d], rep.L, rep.half_L);
      c[d] = a1[d] + ca * rv[d];
    }
    bool react = false, job = false;
    AngJob aj;
    if (pr.bc == RD_BC_ABS) {
      react = true;
    } else {
      const uint4 w = draw_ni(P, step, f.ida, f.idb, TAG_RES, r);
      const double u_res = u52(w.x, w.y), u_reac = u52(w.z, w.w);
      double R0 = sqrt(norm2_rn(r0v[0], r0v[1], r0v[2], dim)) / pr.sigma;
      if (R0 < 1.0) R0 = 1.0;
      const double Rn = resample_dim_ni(P, pr, u_res, R0);
      const double len = sqrt(norm2_rn(rv[0], rv[1], rv[2], dim));
      const double l0 = sqrt(norm2_rn(r0v[0], r0v[1], r0v[2], dim));
      // the free step's direction: the new direction itself (angle mode 1), or the one kept when
      // the exact law needs more partial waves than the device holds
      double dir[3] = {0, 0, 0};
      if (len > 0.0) {
        for (int d = 0; d < dim; ++d) dir[d] = rv[d] / len;
      } else if (l0 > 0.0) {
        for (int d = 0; d < dim; ++d) dir[d] = r0v[d] / l0;
      } else {
        dir[0] = 1.0;
      }
      if (P.angle_mode == 0) {
        // exact direction from the full propagator about the start separation (x axis if zero):
        // drawn in the angle pass
        job = true;
        const uint4 wg = draw_ni(P, step, f.ida, f.idb, TAG_ANG, r);
        for (int d = 0; d < 3; ++d) {
          aj.c[d] = c[d];
          aj.fb[d] = dir[d];
          aj.u[d] = d == 0 ? 1.0 : 0.0;
        }
        if (l0 > 0.0)
          for (int d = 0; d < 3; ++d) aj.u[d] = d < dim ? r0v[d] / l0 : 0.0;
        aj.len = Rn * pr.sigma;
        aj.Rn = Rn;
        aj.R0 = R0;
        aj.tau = pr.tau;
        aj.ca = ca;
        aj.cb = cb;
        aj.U_ang = u52(wg.x, wg.y);
        aj.U_azi = u52(wg.z, wg.w);
        aj.kind = 0u | ((uint32_t)rule << 8);
        aj.ia = f.ia;
        aj.ib = f.ib;
        aj.wa = wa;
        aj.wb = wb;
        aj.r = r;
      } else {
        for (int d = 0; d < dim; ++d) {
          const double nr = Rn * pr.sigma * dir[d];
          a1[d] = wrap(c[d] - ca * nr, rep.L);
          b1[d] = wrap(c[d] + cb * nr, rep.L);
        }
      }
      ++n_res;
      if (pr.bc == RD_BC_RAD) {
        const double pf = dim == 3 ? (double)p_reac3_f((float)Rn, (float)R0, pr.s_f, pr.alpha_f) : -1.0;
        if (dim == 3 && fabs(u_reac - pf) > kFilter) {
          react = u_reac < pf;
        } else {
          const double p = p_reac_dim(P, pr, Rn, R0);
          n_near += fabs(u_reac - p) <= 1e-9;
          react = u_reac < p;
        }
      }
    }
    if (react) {
      ++n_react;
      uint32_t np = 0;
      if (pr.product >= 0) {
        double cw[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) cw[d] = wrap(c[d], rep.L);
        put4<T>(&prodpos[2 * (size_t)f.ia], cw, pack_sp((uint32_t)pr.product, r));
        np = 1;
      }
      status[f.ia] |= ST_CONSUMED | (np << ST_NPROD_SHIFT);
      status[f.ib] |= ST_CONSUMED;
    } else if (job) {
      push_ang_job(ctl, jobs, job_cap, aj);
    } else {
      put4<T>(&x1[f.ia], a1, wa);
      put4<T>(&x1[f.ib], b1, wb);
    }
}

// ================================================================================================
// Unimolecular products (device functions of K5; Section 2.2.5).  One product: parent position plus a free step with
// the product's D.  Two products: centre of diffusion = parent position + free step with D_R;
// separation a n (n uniform) propagated by G_ref - G_abs from contact, geminate recombination by
// p_reac(R', 1); non-interacting products start sigma_place apart and separate freely.
// ================================================================================================
template <class T>
__device__ __forceinline__ void decay_products(const DevParams& P, const RepDev* reps, uint32_t i,
                                               uint32_t step, const typename V4<T>::type* x0,
                                               const uint32_t* id, uint32_t* status,
                                               typename V4<T>::type* prodpos, unsigned long long& n_rec,
                                               unsigned long long& n_near, DevCtl* ctl,
                                               AngJob* jobs, uint32_t job_cap) {
  const int dim = P.dim;
    const uint32_t st = status[i];
    const DecayDev& dc = P.decays[(st >> ST_CHANNEL_SHIFT) & 15u];
    const auto p0 = x0[i];
    const uint32_t r = w_bits(p0.w) >> 8;
    const RepDev& rep = reps[r];
    const uint32_t pid = id[i];
    double xp[3];
    load3<T>(p0, xp);
    uint32_t np = 0;
    if (dc.n_products == 1) {
      double nr[4];
      normals64_ni(P, step, pid, TAG_DISS0, r, dim, nr);
      const double ell = sqrt(2.0 * P.D[dc.p0] * P.dt);
      double q3[3] = {0, 0, 0};
      for (int d = 0; d < dim; ++d) q3[d] = wrap(xp[d] + ell * nr[d], rep.L);
      put4<T>(&prodpos[2 * (size_t)i], q3, pack_sp((uint32_t)dc.p0, r));
      np = 1;
    } else if (dc.n_products == 2) {
      const int sa = dc.p0, sb = dc.p1;
      const double Drel = P.D[sa] + P.D[sb];
      const double ca = P.D[sa] / Drel, cb = P.D[sb] / Drel;
      const double DR = P.D[sa] * P.D[sb] / Drel;
      uint4 w = draw_ni(P, step, pid, kOneParticle, TAG_DIR, r);
      double dir[3] = {0, 0, 0};
      if (dim == 3) {
        const double ct = 2.0 * u52(w.x, w.y) - 1.0;
        double sn, cs;
        sincospi(2.0 * u52(w.z, w.w), &sn, &cs);
        const double stt = sqrt(fmax(0.0, 1.0 - ct * ct));
        dir[0] = stt * cs; dir[1] = stt * sn; dir[2] = ct;
      } else {
        double sn, cs;
        sincospi(2.0 * u52(w.x, w.y), &sn, &cs);
        dir[0] = cs; dir[1] = sn;
      }
      double nc[4];
      normals64_ni(P, step, pid, TAG_DISS0, r, dim, nc);
      const double ellc = sqrt(2.0 * DR * P.dt);
      double c[3] = {0, 0, 0}, rv[3] = {0, 0, 0};
      for (int d = 0; d < dim; ++d) c[d] = xp[d] + ellc * nc[d];
      const int rule = P.pair_of[sa][sb];
      bool recombine = false, job = false;
      int product = -1;
      double Rn = 0.0;
      if (rule >= 0) {
        const PairDev& pr = P.pairs[rule];
        w = draw_ni(P, step, pid, kOneParticle, TAG_RES, r);
        const double u_res = u52(w.x, w.y), u_reac = u52(w.z, w.w);
        Rn = resample_dim_ni(P, pr, u_res, 1.0);
        for (int d = 0; d < dim; ++d) rv[d] = Rn * pr.sigma * dir[d];
        if (pr.bc == RD_BC_ABS) {
          recombine = true;
        } else if (pr.bc == RD_BC_RAD) {
          const double pf = dim == 3 ? (double)p_reac3_f((float)Rn, 1.0f, pr.s_f, pr.alpha_f) : -1.0;
          if (dim == 3 && fabs(u_reac - pf) > kFilter) {
            recombine = u_reac < pf;
          } else {
            const double p = p_reac_dim(P, pr, Rn, 1.0);
            n_near += fabs(u_reac - p) <= 1e-9;
            recombine = u_reac < p;
          }
        }
        product = pr.product;
        if (!recombine && P.angle_mode == 0) {
          // from contact along dir: the new direction from the full propagator, in the angle pass
          job = true;
          const uint4 wg = draw_ni(P, step, pid, kOneParticle, TAG_ANG, r);
          AngJob aj;
          for (int d = 0; d < 3; ++d) {
            aj.c[d] = c[d];
            aj.u[d] = dir[d];
            aj.fb[d] = dir[d];
          }
          aj.len = Rn * pr.sigma;
          aj.Rn = Rn;
          aj.R0 = 1.0;
          aj.tau = pr.tau;
          aj.ca = ca;
          aj.cb = cb;
          aj.U_ang = u52(wg.x, wg.y);
          aj.U_azi = u52(wg.z, wg.w);
          aj.kind = 1u | ((uint32_t)rule << 8);
          aj.ia = i;
          aj.ib = i;
          aj.wa = pack_sp((uint32_t)sa, r);
          aj.wb = pack_sp((uint32_t)sb, r);
          aj.r = r;
          push_ang_job(ctl, jobs, job_cap, aj);
        }
      } else {
        double nr[4];
        normals64_ni(P, step, pid, TAG_DISS2, r, dim, nr);
        const double ellr = sqrt(2.0 * Drel * P.dt);
        for (int d = 0; d < dim; ++d) rv[d] = dc.sigma_place * dir[d] + ellr * nr[d];
      }
      if (recombine) {
        ++n_rec;
        if (product >= 0) {
          double cw[3] = {0, 0, 0};
          for (int d = 0; d < dim; ++d) cw[d] = wrap(c[d], rep.L);
          put4<T>(&prodpos[2 * (size_t)i], cw, pack_sp((uint32_t)product, r));
          np = 1;
        }
      } else {
        if (!job) {
          double qa[3] = {0, 0, 0}, qb[3] = {0, 0, 0};
          for (int d = 0; d < dim; ++d) {
            qa[d] = wrap(c[d] - ca * rv[d], rep.L);
            qb[d] = wrap(c[d] + cb * rv[d], rep.L);
          }
          put4<T>(&prodpos[2 * (size_t)i], qa, pack_sp((uint32_t)sa, r));
          put4<T>(&prodpos[2 * (size_t)i + 1], qb, pack_sp((uint32_t)sb, r));
        }
        np = 2;
      }
    }
    status[i] = st | (np << ST_NPROD_SHIFT);
}

// ------------------------------------------------------------------------------------------------
// Mixed step: positions, displacements and the propagator sample in FP32; p_reac in FP64.
// ------------------------------------------------------------------------------------------------
// Mixed-step propagator samples from the inverse table V(R0 - 1, sqrt(-ln U)) and one Newton step
// on ln T: in 3D on the FP32 closed form, in 2D on the forward -ln(tail) table.
__device__ __forceinline__ float resample3_tab(const PairDev& pr, float U, float R0) {
  if (R0 < 1.0f) R0 = 1.0f;
  const float w = R0 - 1.0f, s = pr.s_f;
  const float lnU = logf(U);
  float V = fmaxf(tab_eval(pr.tab_inv, w, sqrtf(-lnU)), 0.0f);
  const float inv_4tau = 1.0f / (4.0f * s * s);
  const float ln_ex0 = logf(erfcxf(w / (2.0f * s)));
  float f, df;
  lnT3_f(V, w, s, inv_4tau, ln_ex0, f, df);
  if (df < 0.0f) V = fmaxf(V - (f - lnU) / df, 0.0f);
  return 1.0f + V;
}

__device__ __forceinline__ float resample2_tab(const PairDev& pr, float U, float R0) {
  const float d0 = fmaxf(R0 - 1.0f, 0.0f), target = -logf(U);
  float V = fmaxf(tab_eval(pr.tab_inv, d0, sqrtf(target)), 0.0f);
  float dF;
  const float F = tab_eval_dd(pr.tab_tail, d0, V, dF);
  if (dF > 0.0f) V = fmaxf(V - (F - target) / dF, 0.0f);
  return 1.0f + V;
}

__device__ __noinline__ float resample_tab_ni(const PairDev& pr, bool d3, float U, float R0) {
  return d3 ? resample3_tab(pr, U, R0) : resample2_tab(pr, U, R0);
}

__device__ __forceinline__ void resolve_pair_f(const DevParams& P, const RepDev* reps,
                                               const FiredPair* fired,
                                               const uint32_t* fstate, uint32_t e, uint32_t step,
                                               const float4* x0, float4* x1,
                                               uint32_t* status, float4* prodpos,
                                               unsigned long long& n_react, unsigned long long& n_res,
                                               DevCtl* ctl, AngJob* jobs, uint32_t job_cap) {
  const bool d3 = P.dim == 3;
  const uint32_t fs = fstate[e];
  const FiredPair f = fired[e];
  const int rule = (fs >> 2) & 63u;
  const uint32_t r = fs >> 8;
  const PairDev& pr = P.pairs[rule];
  const RepDev& rep = reps[r];
  const float4 a1 = x1[f.ia], b1 = x1[f.ib], a0 = x0[f.ia], b0 = x0[f.ib];
  const uint32_t wa = w_bits(a1.w), wb = w_bits(b1.w);
  const float Drel = P.D_f[wa & 0xFF] + P.D_f[wb & 0xFF];
  const float ca = P.D_f[wa & 0xFF] / Drel, cb = P.D_f[wb & 0xFF] / Drel;
  const float rx = min_image_f(b1.x - a1.x, rep.Lf, rep.half_Lf), ry = min_image_f(b1.y - a1.y, rep.Lf, rep.half_Lf);
  const float rz = d3 ? min_image_f(b1.z - a1.z, rep.Lf, rep.half_Lf) : 0.0f;
  const float cx = a1.x + ca * rx, cy = a1.y + ca * ry, cz = a1.z + ca * rz;
  bool react = true;
  if (pr.bc != RD_BC_ABS) {
    const float r0x = min_image_f(b0.x - a0.x, rep.Lf, rep.half_Lf), r0y = min_image_f(b0.y - a0.y, rep.Lf, rep.half_Lf);
    const float r0z = d3 ? min_image_f(b0.z - a0.z, rep.Lf, rep.half_Lf) : 0.0f;
    const uint4 w = draw_ni(P, step, f.ida, f.idb, TAG_RES, r);
    float R0 = sqrtf(r0x * r0x + r0y * r0y + r0z * r0z) * pr.inv_sigma_f;
    R0 = fmaxf(R0, 1.0f);
    const float Rn = resample_tab_ni(pr, d3, u23(w.x), R0);
    const float len = sqrtf(rx * rx + ry * ry + rz * rz);
    const float l0 = sqrtf(r0x * r0x + r0y * r0y + r0z * r0z);
    float dx, dy, dz;
    if (len > 0.0f) {
      dx = rx / len; dy = ry / len; dz = rz / len;
    } else if (l0 > 0.0f) {
      dx = r0x / l0; dy = r0y / l0; dz = r0z / l0;
    } else {
      dx = 1.0f; dy = 0.0f; dz = 0.0f;
    }
    const float ln = Rn * pr.sigma_f;
    ++n_res;
    react = pr.bc == RD_BC_RAD && u23(w.z) < p_reac_tab_ni(pr, Rn - 1.0f, R0 - 1.0f);
    if (!react) {
      if (P.angle_mode == 0) {
        // exact direction from the full propagator about the start separation, in the angle pass
        const uint4 wg = draw_ni(P, step, f.ida, f.idb, TAG_ANG, r);
        AngJob aj;
        aj.c[0] = cx; aj.c[1] = cy; aj.c[2] = cz;
        aj.fb[0] = dx; aj.fb[1] = dy; aj.fb[2] = dz;
        aj.u[0] = 1.0; aj.u[1] = 0.0; aj.u[2] = 0.0;
        if (l0 > 0.0f) {
          aj.u[0] = r0x / l0; aj.u[1] = r0y / l0; aj.u[2] = r0z / l0;
        }
        aj.len = ln;
        aj.Rn = Rn;
        aj.R0 = R0;
        aj.tau = pr.tau;
        aj.ca = ca;
        aj.cb = cb;
        aj.U_ang = u23(wg.x);
        aj.U_azi = u23(wg.z);
        aj.kind = 0u | ((uint32_t)rule << 8);
        aj.ia = f.ia;
        aj.ib = f.ib;
        aj.wa = wa;
        aj.wb = wb;
        aj.r = r;
        push_ang_job(ctl, jobs, job_cap, aj);
        return;
      }
      x1[f.ia] = make_float4(wrap_f(cx - ca * ln * dx, rep.Lf), wrap_f(cy - ca * ln * dy, rep.Lf),
                             d3 ? wrap_f(cz - ca * ln * dz, rep.Lf) : 0.0f, a1.w);
      x1[f.ib] = make_float4(wrap_f(cx + cb * ln * dx, rep.Lf), wrap_f(cy + cb * ln * dy, rep.Lf),
                             d3 ? wrap_f(cz + cb * ln * dz, rep.Lf) : 0.0f, b1.w);
      return;
    }
  }
  ++n_react;
  uint32_t np = 0;
  if (pr.product >= 0) {
    prodpos[2 * (size_t)f.ia] = make_float4(wrap_f(cx, rep.Lf), wrap_f(cy, rep.Lf), d3 ? wrap_f(cz, rep.Lf) : 0.0f,
                                            w_from_bits_f(pack_sp((uint32_t)pr.product, r)));
    np = 1;
  }
  status[f.ia] |= ST_CONSUMED | (np << ST_NPROD_SHIFT);
  status[f.ib] |= ST_CONSUMED;
}

__device__ __forceinline__ void normals_f(const DevParams& P, uint32_t c0, uint32_t id, uint32_t tag0, uint32_t r,
                                          bool d3, float n[4]) {
  const uint4 w = draw_ni(P, c0, id, kOneParticle, tag0, r);
  box_muller_f(u23(w.x), u23(w.y), n[0], n[1]);
  n[2] = n[3] = 0.0f;
  if (d3) box_muller_f(u23(w.z), u23(w.w), n[2], n[3]);
}

__device__ __forceinline__ void decay_products_f(const DevParams& P, const RepDev* reps, uint32_t i,
                                                 uint32_t step, const float4* x0,
                                                 const uint32_t* id, uint32_t* status,
                                                 float4* prodpos, unsigned long long& n_rec,
                                                 DevCtl* ctl, AngJob* jobs,
                                                 uint32_t job_cap) {
  const bool d3 = P.dim == 3;
  const uint32_t st = status[i];
  const DecayDev& dc = P.decays[(st >> ST_CHANNEL_SHIFT) & 15u];
  const float4 p0 = x0[i];
  const uint32_t r = w_bits(p0.w) >> 8;
  const RepDev& rep = reps[r];
  const uint32_t pid = id[i];
  const float dt = (float)P.dt;
  uint32_t np = 0;
  if (dc.n_products == 1) {
    float nr[4];
    normals_f(P, step, pid, TAG_DISS0, r, d3, nr);
    const float ell = sqrtf(2.0f * P.D_f[dc.p0] * dt);
    prodpos[2 * (size_t)i] = make_float4(wrap_f(p0.x + ell * nr[0], rep.Lf), wrap_f(p0.y + ell * nr[1], rep.Lf),
                                         d3 ? wrap_f(p0.z + ell * nr[2], rep.Lf) : 0.0f,
                                         w_from_bits_f(pack_sp((uint32_t)dc.p0, r)));
    np = 1;
  } else if (dc.n_products == 2) {
    const int sa = dc.p0, sb = dc.p1;
    const float Drel = P.D_f[sa] + P.D_f[sb];
    const float ca = P.D_f[sa] / Drel, cb = P.D_f[sb] / Drel;
    const float DR = P.D_f[sa] * P.D_f[sb] / Drel;
    uint4 w = draw_ni(P, step, pid, kOneParticle, TAG_DIR, r);
    float dx, dy, dz = 0.0f;
    if (d3) {
      const float ct = 2.0f * u23(w.x) - 1.0f;
      float sn, cs;
      sincospif(2.0f * u23(w.y), &sn, &cs);
      const float stt = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
      dx = stt * cs; dy = stt * sn; dz = ct;
    } else {
      sincospif(2.0f * u23(w.x), &dy, &dx);
    }
    float nc[4];
    normals_f(P, step, pid, TAG_DISS0, r, d3, nc);
    const float ellc = sqrtf(2.0f * DR * dt);
    const float cx = p0.x + ellc * nc[0], cy = p0.y + ellc * nc[1], cz = p0.z + ellc * nc[2];
    const int rule = P.pair_of[sa][sb];
    bool recombine = false, job = false;
    int product = -1;
    float rx, ry, rz;
    if (rule >= 0) {
      const PairDev& pr = P.pairs[rule];
      w = draw_ni(P, step, pid, kOneParticle, TAG_RES, r);
      const float Rn = resample_tab_ni(pr, d3, u23(w.x), 1.0f);
      const float ln = Rn * pr.sigma_f;
      rx = ln * dx; ry = ln * dy; rz = ln * dz;
      if (pr.bc == RD_BC_ABS)
        recombine = true;
      else if (pr.bc == RD_BC_RAD)
        recombine = u23(w.z) < p_reac_tab_ni(pr, Rn - 1.0f, 0.0f);
      product = pr.product;
      if (!recombine && P.angle_mode == 0) {
        // from contact along the drawn direction: the new direction in the angle pass
        job = true;
        const uint4 wg = draw_ni(P, step, pid, kOneParticle, TAG_ANG, r);
        AngJob aj;
        aj.c[0] = cx; aj.c[1] = cy; aj.c[2] = cz;
        aj.u[0] = dx; aj.u[1] = dy; aj.u[2] = dz;
        aj.fb[0] = dx; aj.fb[1] = dy; aj.fb[2] = dz;
        aj.len = ln;
        aj.Rn = Rn;
        aj.R0 = 1.0;
        aj.tau = pr.tau;
        aj.ca = ca;
        aj.cb = cb;
        aj.U_ang = u23(wg.x);
        aj.U_azi = u23(wg.z);
        aj.kind = 1u | ((uint32_t)rule << 8);
        aj.ia = i;
        aj.ib = i;
        aj.wa = pack_sp((uint32_t)sa, r);
        aj.wb = pack_sp((uint32_t)sb, r);
        aj.r = r;
        push_ang_job(ctl, jobs, job_cap, aj);
      }
    } else {
      float nr[4];
      normals_f(P, step, pid, TAG_DISS2, r, d3, nr);
      const float ellr = sqrtf(2.0f * Drel * dt);
      const float sp = (float)dc.sigma_place;
      rx = sp * dx + ellr * nr[0]; ry = sp * dy + ellr * nr[1]; rz = sp * dz + ellr * nr[2];
    }
    if (recombine) {
      ++n_rec;
      if (product >= 0) {
        prodpos[2 * (size_t)i] = make_float4(wrap_f(cx, rep.Lf), wrap_f(cy, rep.Lf), d3 ? wrap_f(cz, rep.Lf) : 0.0f,
                                             w_from_bits_f(pack_sp((uint32_t)product, r)));
        np = 1;
      }
    } else {
      if (!job) {
        prodpos[2 * (size_t)i] = make_float4(wrap_f(cx - ca * rx, rep.Lf), wrap_f(cy - ca * ry, rep.Lf),
                                             d3 ? wrap_f(cz - ca * rz, rep.Lf) : 0.0f,
                                             w_from_bits_f(pack_sp((uint32_t)sa, r)));
        prodpos[2 * (size_t)i + 1] = make_float4(wrap_f(cx + cb * rx, rep.Lf), wrap_f(cy + cb * ry, rep.Lf),
                                                 d3 ? wrap_f(cz + cb * rz, rep.Lf) : 0.0f,
                                                 w_from_bits_f(pack_sp((uint32_t)sb, r)));
      }
      np = 2;
    }
  }
  status[i] = st | (np << ST_NPROD_SHIFT);
}

// Rounds of locally-dominant matching for a short conflict list (at most kMatchSmemPairs pairs),
// by one block in shared memory: every particle of the list gets a local slot (open addressing on
// its index, load factor <= 1/2), so the per-round minima are shared-memory atomics.  Same rule as
// the global rounds: a pair is accepted when its (key, id_a, id_b) is the smallest at both of its
// particles among the live pairs.  Returns false if the round bound ran out.
constexpr int kMatchSmemPairs = 256, kMatchSmemSlots = 1024;

__device__ __noinline__ bool match_rounds_smem(const DevParams& P, DevCtl* ctl,
                                               const FiredPair* fired, uint32_t* fstate,
                                               int32_t* matched, const uint32_t* conflict,
                                               uint32_t* accepted, uint32_t nc, uint32_t n_triv) {
  __shared__ uint32_t s_e[kMatchSmemPairs];
  __shared__ unsigned long long s_key[kMatchSmemPairs], s_pid[kMatchSmemPairs];
  __shared__ uint16_t s_sa[kMatchSmemPairs], s_sb[kMatchSmemPairs];
  __shared__ uint8_t s_state[kMatchSmemPairs];     // 1 live, 2 accepted, 0 dead
  __shared__ uint32_t s_h[kMatchSmemSlots];
  __shared__ unsigned long long s_bk[kMatchSmemSlots], s_bp[kMatchSmemSlots];
  __shared__ uint8_t s_m[kMatchSmemSlots];
  __shared__ uint32_t s_live;
  __shared__ unsigned long long s_acc;
  __shared__ int s_err;
  for (int k = threadIdx.x; k < kMatchSmemSlots; k += blockDim.x) {
    s_h[k] = 0xFFFFFFFFu;
    s_bk[k] = ~0ull;
    s_bp[k] = ~0ull;
    s_m[k] = 0;
  }
  if (threadIdx.x == 0) {
    s_acc = 0ull;
    s_err = 0;
  }
  __syncthreads();
  auto slot_of = [&](uint32_t pidx) -> uint32_t {
    uint32_t h = (pidx * 2654435761u) >> (32 - 10);
    for (int probe = 0; probe < kMatchSmemSlots; ++probe) {
      const uint32_t prev = atomicCAS(&s_h[h], 0xFFFFFFFFu, pidx);
      if (prev == 0xFFFFFFFFu || prev == pidx) return h;
      h = (h + 1u) & (kMatchSmemSlots - 1);
    }
    s_err = 1;   // cannot happen at load factor <= 1/2
    return 0u;
  };
  for (uint32_t q = threadIdx.x; q < nc; q += blockDim.x) {
    const uint32_t e = conflict[q];
    const FiredPair f = fired[e];
    s_e[q] = e;
    s_key[q] = (unsigned long long)__double_as_longlong(f.key);
    s_pid[q] = ((unsigned long long)f.ida << 32) | f.idb;
    s_sa[q] = (uint16_t)slot_of(f.ia);
    s_sb[q] = (uint16_t)slot_of(f.ib);
    s_state[q] = 1;
  }
  __syncthreads();
  int rounds = 0;
  bool ok = s_err == 0;
  while (ok) {
    for (uint32_t q = threadIdx.x; q < nc; q += blockDim.x) {
      if (s_state[q] != 1) continue;
      atomicMin(&s_bk[s_sa[q]], s_key[q]);
      atomicMin(&s_bk[s_sb[q]], s_key[q]);
    }
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < nc; q += blockDim.x) {
      if (s_state[q] != 1) continue;
      if (s_bk[s_sa[q]] == s_key[q]) atomicMin(&s_bp[s_sa[q]], s_pid[q]);
      if (s_bk[s_sb[q]] == s_key[q]) atomicMin(&s_bp[s_sb[q]], s_pid[q]);
    }
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < nc; q += blockDim.x) {
      if (s_state[q] != 1) continue;
      const uint32_t a = s_sa[q], b = s_sb[q];
      if (s_bk[a] == s_key[q] && s_bk[b] == s_key[q] && s_bp[a] == s_pid[q] && s_bp[b] == s_pid[q]) {
        s_m[a] = 1;
        s_m[b] = 1;
        s_state[q] = 2;
        const uint32_t e = s_e[q];
        const FiredPair f = fired[e];
        matched[f.ia] = (int32_t)f.ib;
        matched[f.ib] = (int32_t)f.ia;
        fstate[e] = (fstate[e] & ~3u) | FS_ACCEPTED;
        accepted[n_triv + atomicAdd(&ctl->n_round_acc, 1u)] = e;
        atomicAdd(&s_acc, 1ull);
      }
    }
    if (threadIdx.x == 0) s_live = 0u;
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < nc; q += blockDim.x) {
      if (s_state[q] != 1) continue;
      const uint32_t a = s_sa[q], b = s_sb[q];
      if (s_m[a] || s_m[b]) {
        s_state[q] = 0;
        fstate[s_e[q]] = (fstate[s_e[q]] & ~3u) | FS_DEAD;
      } else {
        s_bk[a] = ~0ull;
        s_bk[b] = ~0ull;
        s_bp[a] = ~0ull;
        s_bp[b] = ~0ull;
        atomicAdd(&s_live, 1u);
      }
    }
    __syncthreads();
    ++rounds;
    if (s_live == 0u) break;
    if (rounds >= P.match_max_rounds) {
      ok = false;
      break;
    }
  }
  if (threadIdx.x == 0) {
    if (!ok) set_status(ctl, RD_ETIMEOUT);
    if (s_acc) atomicAdd(&ctl->stats[RD_STAT_MATCHED], s_acc);
    atomicAdd(&ctl->stats[RD_STAT_MATCH_ROUNDS], (unsigned long long)rounds);
  }
  __syncthreads();
  return ok;
}

// Compaction table over replicas, by one block: survivors = particles - consumed; exclusive
// prefixes of products and inclusive prefixes of survivors over the replicas; the new particle
// count.
__device__ __forceinline__ void replica_table(int n_replicas, const RepDev* reps,
                                              const uint32_t* rep_cons,
                                              const uint32_t* rep_prod, RepX* repx,
                                              DevCtl* ctl) {
  __shared__ unsigned long long sm[32];
  unsigned long long carry = 0;      // survivors << 32 | products of the replicas done so far
  for (int base = 0; base < n_replicas; base += blockDim.x) {
    const int r = base + (int)threadIdx.x;
    uint32_t surv = 0, prod = 0;
    if (r < n_replicas) {
      surv = reps[r].end - reps[r].beg - __ldcg(&rep_cons[r]);
      prod = __ldcg(&rep_prod[r]);
    }
    const unsigned long long v = ((unsigned long long)surv << 32) | prod;
    unsigned long long tot;
    const unsigned long long ex = carry + block_exclusive_scan<unsigned long long, int>(v, sm, tot);
    if (r < n_replicas) {
      RepX x;
      x.p_beg = (uint32_t)ex;
      x.s_end = (uint32_t)(ex >> 32) + surv;
      x.surv = surv;
      x.prod = prod;
      repx[r] = x;
    }
    carry += tot;
  }
  if (threadIdx.x == 0) ctl->n_new = (uint32_t)(carry >> 32) + (uint32_t)carry;
}

// One accepted pair or one decay of this step (item q of the combined list).
// One accepted pair or one decay of this step (item q of the combined list).
template <class T>
__device__ __noinline__ void resolve_item(const DevParams& P, const RepDev* reps,
                                             const FiredPair* fired, const uint32_t* fstate,
                                             bool pair, uint32_t idx, uint32_t step,
                                             const typename V4<T>::type* x0,
                                             typename V4<T>::type* x1, const uint32_t* id,
                                             uint32_t* status, typename V4<T>::type* prodpos,
                                             uint32_t* rep_cons, uint32_t* rep_prod,
                                             unsigned long long& n_react, unsigned long long& n_res,
                                             unsigned long long& n_rec, unsigned long long& n_near,
                                             DevCtl* ctl, AngJob* jobs, uint32_t job_cap) {
  if constexpr (sizeof(T) == 8) {
    if (pair)
      resolve_pair<T>(P, reps, fired, fstate, idx, step, x0, x1, status, prodpos, n_react, n_res, n_near, ctl, jobs,
                      job_cap);
    else
      decay_products<T>(P, reps, idx, step, x0, id, status, prodpos, n_rec, n_near, ctl, jobs, job_cap);
  } else {
    if (pair)
      resolve_pair_f(P, reps, fired, fstate, idx, step, x0, x1, status, prodpos, n_react, n_res, ctl, jobs, job_cap);
    else
      decay_products_f(P, reps, idx, step, x0, id, status, prodpos, n_rec, ctl, jobs, job_cap);
  }
  // per-replica tallies for the compaction: a reacting pair consumes both particles, a decay its
  // parent; the owner's status carries the number of products
  const uint32_t owner = pair ? fired[idx].ia : idx;
  const uint32_t st = status[owner];
  if (st & ST_CONSUMED) {
    const uint32_t r = pair ? (fstate[idx] >> 8) : (w_bits(x0[idx].w) >> 8);
    atomicAdd(&rep_cons[r], pair ? 2u : 1u);
    const uint32_t np = (st >> ST_NPROD_SHIFT) & 3u;
    if (np) atomicAdd(&rep_prod[r], np);
  }
}

// K5: rounds of locally-dominant matching over the conflict list, and the resolution of every
// accepted pair and every decay of the step (one cooperative launch).
//  - A short conflict list is matched by block 0 alone (block barriers); trivially accepted pairs
//    and decays involve no conflict pair, so blocks 1.. resolve them meanwhile.  A long list is
//    matched by the whole grid (grid barriers between the phases of a round), and everything is
//    resolved after the last round.
//  - Each round: every live pair offers its key to both particles (atomic min), then its
//    (id_a, id_b) among equal keys; a pair that is the minimum at both particles is accepted;
//    pairs touching an accepted particle die, the rest stay live.  The pairs accepted in the
//    rounds are resolved after the last round.
template <class T>
__device__ __forceinline__ void ph_match_resolve(
    const DevParams* Pp, DevCtl* ctl, const RepDev* reps,
    const FiredPair* fired, uint32_t* fstate, int32_t* matched,
    const uint32_t* conflict, uint32_t* accepted,
    unsigned long long* best_key, unsigned long long* best_pid,
    const uint32_t* decay_list, const typename V4<T>::type* x0,
    typename V4<T>::type* x1, const uint32_t* id, uint32_t* status,
    typename V4<T>::type* prodpos, uint32_t* deg, uint32_t cap_pairs,
    uint32_t* rep_cons, uint32_t* rep_prod, RepX* repx,
    ConflictRec* crec, AngJob* jobs, uint32_t job_cap) {
  __shared__ unsigned long long acc_s;
  __shared__ uint32_t live_s;
  const DevParams& P = *Pp;
  // the encounter degrees of this step go back to zero for the next one (the previous kernel made
  // the last reads of them)
  const uint32_t nf = min(ctl->fired, cap_pairs);
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < nf; e += gridDim.x * blockDim.x) {
    deg[fired[e].ia] = 0u;
    deg[fired[e].ib] = 0u;
  }
  if (ctl->status) return;
  // n_accept holds the trivially accepted pairs only: the rounds count theirs in n_round_acc, so
  // every block reads the same n_triv whenever it starts
  const uint32_t nc = ctl->n_conflict, n_triv = ctl->n_accept, nd = ctl->n_decay, step = ctl->step;
  const bool multi = nc > P.match_single_max && gridDim.x > 1;
  unsigned long long n_react = 0, n_res = 0, n_near = 0, n_rec = 0;
  if (!multi) {
    // block 0 runs the (short) rounds alone, the other blocks resolve meanwhile
    const bool skip0 = gridDim.x > 1 && nc > 0;
    const uint32_t nblk = skip0 ? gridDim.x - 1 : gridDim.x;
    if (!(skip0 && blockIdx.x == 0)) {
      const uint32_t b = skip0 ? blockIdx.x - 1 : blockIdx.x;
      for (uint32_t q = b * blockDim.x + threadIdx.x; q < n_triv + nd; q += nblk * blockDim.x) {
        const bool pair = q < n_triv;
        resolve_item<T>(P, reps, fired, fstate, pair, pair ? accepted[q] : decay_list[q - n_triv], step, x0, x1, id,
                        status, prodpos, rep_cons, rep_prod, n_react, n_res, n_rec, n_near, ctl, jobs, job_cap);
      }
    }
  }
  if (nc > 0 && !multi && nc <= min(P.match_smem_max, (uint32_t)kMatchSmemPairs) && blockIdx.x == 0) {
    // short list: block 0 matches in shared memory, then resolves the pairs it accepted
    if (match_rounds_smem(P, ctl, fired, fstate, matched, conflict, accepted, nc, n_triv)) {
      const uint32_t n_acc = n_triv + *(volatile uint32_t*)&ctl->n_round_acc;
      for (uint32_t q = n_triv + threadIdx.x; q < n_acc; q += blockDim.x)
        resolve_item<T>(P, reps, fired, fstate, true, accepted[q], step, x0, x1, id, status, prodpos, rep_cons,
                        rep_prod, n_react, n_res, n_rec, n_near, ctl, jobs, job_cap);
    }
  } else if (nc > 0 && (multi || blockIdx.x == 0)) {
    const uint32_t nthr = multi ? gridDim.x * blockDim.x : blockDim.x;
    const uint32_t tid = multi ? blockIdx.x * blockDim.x + threadIdx.x : threadIdx.x;
    auto sync = [&]() -> bool {
      if (multi) return grid_barrier(ctl);
      __syncthreads();
      return true;
    };
    if (threadIdx.x == 0) acc_s = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ctl->live[0] = 0u;
      ctl->live[1] = 0u;
    }
    // FP32 keys (mixed step) fit one 64-bit word with the partner's id: at a shared particle the
    // order (key, partner id) is the order (key, id_a, id_b) of its pairs, so the minimum takes
    // one atomic per endpoint; FP64 keys take the key and then the (id_a, id_b) minimum
    const bool packed = P.precision == RD_MIXED;
    int rounds = 0;
    bool ok = sync();
    while (ok) {
      for (uint32_t q = tid; q < nc; q += nthr) {
        const ConflictRec c = crec[q];
        if (c.st != FS_LIVE) continue;
        if (packed) {
          const unsigned long long kb = (unsigned long long)__float_as_uint((float)__longlong_as_double((long long)c.key)) << 32;
          atomicMin(&best_key[c.ia], kb | (uint32_t)c.pid);
          atomicMin(&best_key[c.ib], kb | (uint32_t)(c.pid >> 32));
        } else {
          atomicMin(&best_key[c.ia], c.key);
          atomicMin(&best_key[c.ib], c.key);
        }
      }
      if (!(ok = sync())) break;
      if (!packed) {
        for (uint32_t q = tid; q < nc; q += nthr) {
          const ConflictRec c = crec[q];
          if (c.st != FS_LIVE) continue;
          if (best_key[c.ia] == c.key) atomicMin(&best_pid[c.ia], c.pid);
          if (best_key[c.ib] == c.key) atomicMin(&best_pid[c.ib], c.pid);
        }
        if (!(ok = sync())) break;
      }
      for (uint32_t q = tid; q < nc; q += nthr) {
        const ConflictRec c = crec[q];
        if (c.st != FS_LIVE) continue;
        bool win;
        if (packed) {
          const unsigned long long kb = (unsigned long long)__float_as_uint((float)__longlong_as_double((long long)c.key)) << 32;
          win = best_key[c.ia] == (kb | (uint32_t)c.pid) && best_key[c.ib] == (kb | (uint32_t)(c.pid >> 32));
        } else {
          win = best_key[c.ia] == c.key && best_key[c.ib] == c.key && best_pid[c.ia] == c.pid &&
                best_pid[c.ib] == c.pid;
        }
        if (win) {
          matched[c.ia] = (int32_t)c.ib;
          matched[c.ib] = (int32_t)c.ia;
          fstate[c.e] = (fstate[c.e] & ~3u) | FS_ACCEPTED;
          crec[q].st = FS_ACCEPTED;
          accepted[n_triv + atomicAdd(&ctl->n_round_acc, 1u)] = c.e;
          atomicAdd(&acc_s, 1ull);
        }
      }
      if (threadIdx.x == 0) live_s = 0u;
      if (!(ok = sync())) break;
      for (uint32_t q = tid; q < nc; q += nthr) {
        const ConflictRec c = crec[q];
        if (c.st != FS_LIVE) continue;
        if (matched[c.ia] >= 0 || matched[c.ib] >= 0) {
          crec[q].st = FS_DEAD;
          fstate[c.e] = (fstate[c.e] & ~3u) | FS_DEAD;
        } else {
          best_key[c.ia] = ~0ull;
          best_key[c.ib] = ~0ull;
          best_pid[c.ia] = ~0ull;
          best_pid[c.ib] = ~0ull;
          atomicAdd(&live_s, 1u);
        }
      }
      __syncthreads();
      const int par = rounds & 1;
      if (threadIdx.x == 0 && live_s) atomicAdd(&ctl->live[par], live_s);
      if (!(ok = sync())) break;
      ++rounds;
      const uint32_t live = *(volatile uint32_t*)&ctl->live[par];
      if (live == 0) break;
      // the other parity was last read before this round's first barrier
      if (blockIdx.x == 0 && threadIdx.x == 0) ctl->live[par ^ 1] = 0u;
      if (rounds >= P.match_max_rounds) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(ctl, RD_ETIMEOUT);
        ok = false;
        break;
      }
    }
    if (threadIdx.x == 0) {
      if (acc_s) atomicAdd(&ctl->stats[RD_STAT_MATCHED], acc_s);
      if (blockIdx.x == 0) atomicAdd(&ctl->stats[RD_STAT_MATCH_ROUNDS], (unsigned long long)rounds);
    }
    // after the last barrier (all blocks of the rounds have passed it): the pairs accepted in the
    // rounds; with the whole grid in the rounds also the trivially accepted pairs and the decays,
    // kept out of the barrier-separated phases because a resolution can take long (FP64 2D)
    if (ok) {
      const uint32_t n_acc = n_triv + *(volatile uint32_t*)&ctl->n_round_acc;
      const uint32_t first = multi ? 0u : n_triv, last = multi ? n_acc + nd : n_acc;
      for (uint32_t q = first + tid; q < last; q += nthr) {
        const bool pair = q < n_acc;
        resolve_item<T>(P, reps, fired, fstate, pair, pair ? accepted[q] : decay_list[q - n_acc], step, x0, x1, id,
                        status, prodpos, rep_cons, rep_prod, n_react, n_res, n_rec, n_near, ctl, jobs, job_cap);
      }
    }
  }
  if (n_react) atomicAdd(&ctl->stats[RD_STAT_REACTIONS], n_react);
  if (n_res) atomicAdd(&ctl->stats[RD_STAT_RESAMPLED], n_res);
  if (n_rec) atomicAdd(&ctl->stats[RD_STAT_RECOMBINED], n_rec);
  if (n_near) atomicAdd(&ctl->stats[RD_STAT_NEAR_THRESHOLD], n_near);
  // with several replicas, the last block to finish (no block waits for it) builds the
  // compaction's replica table; a single replica needs none (the compaction reads its tallies)
  if (P.n_replicas == 1) return;
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&ctl->done_res, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  replica_table(P.n_replicas, reps, rep_cons, rep_prod, repx, ctl);
}

template <class T>
__global__ void __launch_bounds__(256, 2) k_match_resolve(
    const DevParams* __restrict__ Pp, DevCtl* __restrict__ ctl, const RepDev* __restrict__ reps,
    const FiredPair* __restrict__ fired, uint32_t* __restrict__ fstate, int32_t* __restrict__ matched,
    uint32_t* conflict, uint32_t* __restrict__ accepted,
    unsigned long long* __restrict__ best_key, unsigned long long* __restrict__ best_pid,
    const uint32_t* __restrict__ decay_list, const typename V4<T>::type* __restrict__ x0,
    typename V4<T>::type* __restrict__ x1, const uint32_t* __restrict__ id, uint32_t* __restrict__ status,
    typename V4<T>::type* __restrict__ prodpos, uint32_t* __restrict__ deg, uint32_t cap_pairs,
    uint32_t* __restrict__ rep_cons, uint32_t* __restrict__ rep_prod, RepX* __restrict__ repx,
    ConflictRec* __restrict__ crec, AngJob* __restrict__ jobs, uint32_t job_cap) {
  pdl_enter();
  // the degree-1 pairs accepted and the rest listed as conflicts first, then (every block past the
  // barrier) the rounds and the resolution: one launch for both stages
  ph_match_trivial(ctl, fired, fstate, deg, matched, conflict, accepted, best_key, best_pid,
                   cap_pairs, crec, blockIdx.x, gridDim.x);
  if (!grid_barrier(ctl, false)) return;
  ph_match_resolve<T>(Pp, ctl, reps, fired, fstate, matched, conflict, accepted, best_key, best_pid, decay_list, x0,
                      x1, id, status, prodpos, deg, cap_pairs, rep_cons, rep_prod, repx, crec, jobs, job_cap);
}

// Places the two particles of angle job j along dir (the new separation direction).
template <class T>
__device__ __forceinline__ void ang_job_place(const AngJob& j, const RepDev& rep, int dim, const T* dir,
                                              typename V4<T>::type* x1, typename V4<T>::type* prodpos) {
  double a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
  if constexpr (sizeof(T) == 8) {
    for (int d = 0; d < dim; ++d) {
      const double nr = j.len * dir[d];
      a[d] = wrap(j.c[d] - j.ca * nr, rep.L);
      b[d] = wrap(j.c[d] + j.cb * nr, rep.L);
    }
  } else {
    const float ln = (float)j.len, caf = (float)j.ca, cbf = (float)j.cb;
    for (int d = 0; d < dim; ++d) {
      const float cf = (float)j.c[d];
      a[d] = wrap_f(cf - caf * ln * dir[d], rep.Lf);
      b[d] = wrap_f(cf + cbf * ln * dir[d], rep.Lf);
    }
  }
  if ((j.kind & 0xFFu) == 0) {
    put4<T>(&x1[j.ia], a, j.wa);
    put4<T>(&x1[j.ib], b, j.wb);
  } else {
    put4<T>(&prodpos[2 * (size_t)j.ia], a, j.wa);
    put4<T>(&prodpos[2 * (size_t)j.ia + 1], b, j.wb);
  }
}

// Angle pass: the new separation direction of every encountered pair and every decay's product
// pair that the resolution left to it (angle mode 0), then the particles placed.  Mixed step: one
// thread per job from the rule's tabulated law; jobs of rules without a table (and every job of the
// FP64 step) one warp per job from the full propagator (the partial-wave evaluation is
// warp-collective).
template <class T>
__device__ __forceinline__ void ph_angles(const DevParams* Pp, DevCtl* ctl,
                                          const RepDev* reps, const AngJob* jobs,
                                          uint32_t job_cap, typename V4<T>::type* x1,
                                          typename V4<T>::type* prodpos, const uint32_t bid,
                                          const uint32_t nblk) {
  const DevParams& P = *Pp;
  if (ctl->status) return;
  const uint32_t nj = min(ctl->n_ang, job_cap);
  const int dim = P.dim;
  unsigned long long n_fb = 0;
  if constexpr (sizeof(T) == 4) {
    for (uint32_t q = bid * blockDim.x + threadIdx.x; q < nj; q += nblk * blockDim.x) {
      const AngJob& j = jobs[q];
      const AngTab& A = P.pairs[j.kind >> 8].tab_ang;
      if (!A.v) continue;
      float u[3] = {(float)j.u[0], (float)j.u[1], (float)j.u[2]}, dir[3];
      const float v = ang_table_sample(A, dim, (float)j.U_ang, (float)j.Rn, (float)j.R0);
      if (v == v) {
        ang_place<float>(dim, u, v, (float)j.U_azi, dir);
      } else {
        for (int d = 0; d < 3; ++d) dir[d] = (float)j.fb[d];
        ++n_fb;
      }
      ang_job_place<T>(j, reps[j.r], dim, dir, x1, prodpos);
    }
  }
  const uint32_t wpb = blockDim.x >> 5, nw = nblk * wpb;
  const bool lane0 = (threadIdx.x & 31) == 0;
  for (uint32_t q = bid * wpb + (threadIdx.x >> 5); q < nj; q += nw) {
    const AngJob& j = jobs[q];
    if (sizeof(T) == 4 && P.pairs[j.kind >> 8].tab_ang.v) continue;
    T u[3] = {(T)j.u[0], (T)j.u[1], (T)j.u[2]}, dir[3];
    if (!ang_direction_warp<T>(dim, u, (T)j.U_ang, (T)j.U_azi, (T)j.Rn, (T)j.R0, (T)j.tau, P.gl16, dir)) {
      for (int d = 0; d < 3; ++d) dir[d] = (T)j.fb[d];
      n_fb += lane0;
    }
    if (lane0) ang_job_place<T>(j, reps[j.r], dim, dir, x1, prodpos);
  }
  if (n_fb) atomicAdd(&ctl->stats[RD_STAT_ANGLE_FALLBACK], n_fb);
}

template <class T>
__global__ void __launch_bounds__(256, 2) k_angles(const DevParams* __restrict__ Pp, DevCtl* __restrict__ ctl,
                                                   const RepDev* __restrict__ reps, const AngJob* __restrict__ jobs,
                                                   uint32_t job_cap, typename V4<T>::type* __restrict__ x1,
                                                   typename V4<T>::type* __restrict__ prodpos) {
  pdl_enter();
  ph_angles<T>(Pp, ctl, reps, jobs, job_cap, x1, prodpos, blockIdx.x, gridDim.x);
}

// Per-warp aggregated count: lanes holding the same (replica, species) key add once.  Called by all
// 32 lanes of a converged warp; key kNoKey is skipped.
constexpr uint32_t kNoKey = 0xFFFFFFFFu;
__device__ __forceinline__ void count_key(uint32_t key, bool smem, uint32_t* hist, unsigned long long* counts) {
  const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
  if (key != kNoKey && (int)(threadIdx.x & 31) == __ffs(peers) - 1) {
    if (smem)
      atomicAdd(&hist[key], (uint32_t)__popc(peers));
    else
      atomicAdd(&counts[key], (unsigned long long)__popc(peers));
  }
}

// Species totals over all replicas of the (replica, species) counts, by one whole block.
__device__ __forceinline__ void species_totals(const unsigned long long* counts, int n_replicas, int ns,
                                               long long* out) {
  __shared__ unsigned long long tot[RD_MAX_SPECIES];
  for (int k = threadIdx.x; k < ns; k += blockDim.x) tot[k] = 0ull;
  __syncthreads();
  for (int k = 0; k < ns; ++k) {
    unsigned long long v = 0ull;
#pragma unroll 4
    for (int r = threadIdx.x; r < n_replicas; r += blockDim.x) v += counts[(size_t)r * ns + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&tot[k], v);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < ns; k += blockDim.x) out[k] = (long long)tot[k];
}

// ================================================================================================
// K7: compaction, one pass.  Tiles of 2048 particles scan (survivor, products) counts
// with a decoupled look-back, then place their own particles: survivors keep their order inside
// their replica, products follow the replica's survivors in owner order with ids next_id + rank
// (the per-replica offsets come from the table built at the end of the resolution).  An error
// latched during the step, or a particle count above capacity, turns this into a copy of the
// unchanged state.  The last block to finish commits the step.
// ================================================================================================
constexpr int kCompactTile = 2048;   // particles per tile (the look-back buffers are sized for it)

template <class T, int kCompactThreads>
__device__ __forceinline__ void ph_compact(const DevParams* Pp, DevCtl* ctl,
                          RepDev* reps, const RepX* repx,
                          uint32_t* rep_cons, uint32_t* rep_prod,
                          const typename V4<T>::type* x0,
                          const typename V4<T>::type* x1, const uint32_t* id,
                          const uint32_t* status, const typename V4<T>::type* prodpos,
                          unsigned long long* agg, unsigned long long* incl,
                          uint32_t* flag, typename V4<T>::type* xo,
                          uint32_t* ido, unsigned long long* counts, int n_counts,
                          long long* history, int history_len,
                          uint32_t* hist /* n_counts entries when n_counts <= kSmemCounts */,
                          unsigned long long* s_pre /* kCompactTile entries */,
                          const int stamp_phase = -1) {
  constexpr int kTile = kCompactTile, kCompactItems = kCompactTile / kCompactThreads;
  __shared__ unsigned long long sm[32];
  __shared__ uint32_t s_tile;
  __shared__ unsigned long long s_prefix;
  __shared__ bool s_last;
  const DevParams& P = *Pp;
  const int ns = P.n_species;
  const bool use_smem = n_counts <= kSmemCounts;
  if (use_smem)
    for (int k = threadIdx.x; k < n_counts; k += blockDim.x) hist[k] = 0u;
  const uint32_t n = ctl->n;
  // a single replica: its placement follows from the step's tallies directly
  const bool one = P.n_replicas == 1;
  RepX rx1 = {0u, 0u, 0u, 0u};
  if (one) {
    rx1.surv = n - __ldcg(&rep_cons[0]);
    rx1.prod = __ldcg(&rep_prod[0]);
    rx1.s_end = rx1.surv;
  }
  const uint32_t n_new = one ? rx1.surv + rx1.prod : ctl->n_new;
  const bool fail = ctl->status != 0 || (unsigned long long)n_new > (unsigned long long)P.cap_particles;
  const uint32_t ntiles = (uint32_t)(((int64_t)n + kTile - 1) / kTile);
  auto key_of = [&](uint32_t wb) { return (wb >> 8) * ns + (wb & 0xFFu); };
  // tiles by ticket, so that every tile's predecessors are taken before it (look-back order)
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_tile = atomicAdd(&ctl->tile_ctr[1], 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= ntiles) break;
    const int64_t t0 = (int64_t)tile * kTile;
    // with at most two placement passes per thread, the placement's loads go out before the scan,
    // so that their latency overlaps the scan and the look-back (more passes' worth of registers
    // cost occupancy: 512-thread tiles with four early passes ran at half the speed)
    constexpr int kPasses = kTile / kCompactThreads;
    constexpr bool kEarly = kPasses <= 2;
    typename V4<T>::type q_r[kEarly ? kPasses : 1];
    uint32_t st_r[kEarly ? kPasses : 1], id_r[kEarly ? kPasses : 1];
    if constexpr (kEarly) {
#pragma unroll
      for (int ps = 0; ps < kPasses; ++ps) {
        const int64_t i = t0 + threadIdx.x + ps * kCompactThreads;
        if (i < (int64_t)n) {
          q_r[ps] = fail ? x0[i] : x1[i];
          st_r[ps] = fail ? 0u : status[i];
          id_r[ps] = id[i];
        }
      }
    }
    if (!fail) {
      // blocked arrangement for the scan: each thread owns kCompactItems consecutive particles
      const int64_t base = t0 + (int64_t)threadIdx.x * kCompactItems;
      unsigned long long v[kCompactItems], ex[kCompactItems], run = 0;
      if constexpr (kCompactItems == 8) {
        LoadCompact{status}.load8(base, n, v);
      } else {
#pragma unroll
        for (int k = 0; k < kCompactItems; ++k) v[k] = base + k < (int64_t)n ? LoadCompact::conv(__ldcg(status + base + k)) : 0ull;
      }
#pragma unroll
      for (int k = 0; k < kCompactItems; ++k) {
        ex[k] = run;
        run += v[k];
      }
      unsigned long long tot;
      const unsigned long long toff = block_exclusive_scan<unsigned long long, int>(run, sm, tot);
      if (threadIdx.x < 32) {
        const uint32_t epoch = (ctl->epoch * 2u + 1u) & 0x3FFFFFFFu;
        const unsigned long long prefix = tile_lookback<unsigned long long>(tot, tile, epoch, agg, incl, flag, ctl);
        if (threadIdx.x == 0) s_prefix = prefix;
      }
      __syncthreads();
      const unsigned long long pre = s_prefix + toff;
#pragma unroll
      for (int k = 0; k < kCompactItems; ++k) s_pre[threadIdx.x * kCompactItems + k] = pre + ex[k];
      __syncthreads();
    }
    // striped placement (coalesced), one particle per thread per pass, warp-converged counting
#pragma unroll
    for (int ps = 0; ps < kPasses; ++ps) {
      const int j = threadIdx.x + ps * kCompactThreads;
      const int64_t i = t0 + j;
      uint32_t k0 = kNoKey, k1 = kNoKey, k2 = kNoKey;
      if (i < (int64_t)n) {
        if (fail) {
          const auto q0 = kEarly ? q_r[kEarly ? ps : 0] : x0[i];
          xo[i] = q0;
          ido[i] = kEarly ? id_r[kEarly ? ps : 0] : id[i];
          k0 = key_of(w_bits(q0.w));
        } else {
          const unsigned long long e = s_pre[j];
          const uint32_t S_i = (uint32_t)(e >> 32), P_i = (uint32_t)e;
          const uint32_t st = kEarly ? st_r[kEarly ? ps : 0] : status[i];
          const auto q = kEarly ? q_r[kEarly ? ps : 0] : x1[i];
          const uint32_t wb = w_bits(q.w);
          const uint32_t r = wb >> 8;
          const RepX rx = one ? rx1 : repx[r];
          if (!(st & ST_CONSUMED)) {
            const uint32_t o = S_i + rx.p_beg;
            xo[o] = q;
            ido[o] = kEarly ? id_r[kEarly ? ps : 0] : id[i];
            k0 = key_of(wb);
          }
          const uint32_t np = (st >> ST_NPROD_SHIFT) & 3u;
          for (uint32_t k = 0; k < np; ++k) {
            const uint32_t o = rx.s_end + P_i + k;
            const auto pp = prodpos[2 * (size_t)i + k];
            xo[o] = pp;
            ido[o] = reps[r].next_id + (P_i - rx.p_beg) + k;
            (k == 0 ? k1 : k2) = key_of(w_bits(pp.w));
          }
        }
      }
      count_key(k0, use_smem, hist, counts);
      if (__any_sync(0xFFFFFFFFu, k1 != kNoKey)) count_key(k1, use_smem, hist, counts);
      if (__any_sync(0xFFFFFFFFu, k2 != kNoKey)) count_key(k2, use_smem, hist, counts);
    }
  }
  if (use_smem) {
    __syncthreads();
    for (int k = threadIdx.x; k < n_counts; k += blockDim.x)
      if (hist[k]) atomicAdd(&counts[k], (unsigned long long)hist[k]);
  }
  __syncthreads();
  // the last block to finish commits the step: replica segments, ids, count, step, time
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&ctl->done_blocks, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int r = threadIdx.x; r < P.n_replicas; r += blockDim.x) {
    if (!fail) {
      const RepX rx = one ? rx1 : repx[r];
      const uint32_t beg = rx.s_end - rx.surv + rx.p_beg;
      reps[r].next_id += rx.prod;
      reps[r].beg = beg;
      reps[r].end = beg + rx.surv + rx.prod;
    }
    rep_cons[r] = 0u;
    rep_prod[r] = 0u;
  }
  // per-step totals over replicas of every species (ring buffer indexed by the new step)
  if (!fail && history_len > 0)
    species_totals(counts, P.n_replicas, ns, history + (size_t)((ctl->step + 1u) % (uint32_t)history_len) * ns);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (stamp_phase >= 0) {
      // fused step: the compaction phase ends with this commit
      unsigned long long now;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
      ctl->ph_acc[stamp_phase] += now - ctl->ph_t[stamp_phase];
      ctl->ph_steps += 1;
    }
    if (!fail) {
      ctl->stats[RD_STAT_PARTICLE_STEPS] += n;
      ctl->stats[RD_STAT_DECAYS] += ctl->n_decay;
      ctl->stats[RD_STAT_FIRED] += ctl->fired;
      if (ctl->fired > ctl->stats[RD_STAT_FIRED_HWM]) ctl->stats[RD_STAT_FIRED_HWM] = ctl->fired;
      ctl->n = n_new;
      ctl->step += 1;
      ctl->t += P.dt;
    } else if (ctl->status == 0) {
      ctl->status = RD_ECAPACITY;
    }
    ctl->last_fired = ctl->fired;
    ctl->fired = 0;
    ctl->n_conflict = 0;
    ctl->n_accept = 0;
    ctl->n_round_acc = 0;
    ctl->n_ang = 0;
    ctl->n_decay = 0;
    ctl->done_blocks = 0;
    ctl->done_res = 0;
  }
}

template <class T, int kCompactThreads>
__global__ void __launch_bounds__(kCompactThreads) k_compact(const DevParams* __restrict__ Pp, DevCtl* __restrict__ ctl,
                          RepDev* __restrict__ reps, const RepX* __restrict__ repx,
                          uint32_t* __restrict__ rep_cons, uint32_t* __restrict__ rep_prod,
                          const typename V4<T>::type* __restrict__ x0,
                          const typename V4<T>::type* __restrict__ x1, const uint32_t* __restrict__ id,
                          const uint32_t* __restrict__ status, const typename V4<T>::type* __restrict__ prodpos,
                          unsigned long long* __restrict__ agg, unsigned long long* __restrict__ incl,
                          uint32_t* __restrict__ flag, typename V4<T>::type* __restrict__ xo,
                          uint32_t* __restrict__ ido, unsigned long long* __restrict__ counts, int n_counts,
                          long long* __restrict__ history, int history_len) {
  pdl_enter();
  extern __shared__ uint32_t hist[];   // n_counts entries when n_counts <= kSmemCounts
  __shared__ unsigned long long s_pre[kCompactTile];
  ph_compact<T, kCompactThreads>(Pp, ctl, reps, repx, rep_cons, rep_prod, x0, x1, id, status, prodpos, agg, incl,
                                 flag, xo, ido, counts, n_counts, history, history_len, hist, s_pre);
}

// ================================================================================================
// Initial uniform positions (INIT streams) and helpers.
// ================================================================================================
template <class T>
__global__ void k_init_positions(const DevParams* __restrict__ Pp, const RepDev* __restrict__ reps,
                                 const int32_t* __restrict__ rep_of, const int32_t* __restrict__ sp_of,
                                 const uint32_t* __restrict__ id_of, uint32_t n,
                                 typename V4<T>::type* __restrict__ x, uint32_t* __restrict__ ido) {
  const DevParams& P = *Pp;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t r = (uint32_t)rep_of[i], pid = id_of[i];
    const double L = reps[r].L;
    uint4 w = draw(P, 0u, pid, kOneParticle, TAG_INIT0, r);
    double p[3];
    p[0] = u52(w.x, w.y) * L;
    p[1] = u52(w.z, w.w) * L;
    p[2] = 0.0;
    if (P.dim == 3) {
      w = draw(P, 0u, pid, kOneParticle, TAG_INIT1, r);
      p[2] = u52(w.x, w.y) * L;
    }
    for (int d = 0; d < 3; ++d)
      if (!(p[d] < L)) p[d] = 0.0;
    if constexpr (sizeof(T) == 8) {
      x[i] = make_v4(p[0], p[1], p[2], pack_sp((uint32_t)sp_of[i], r));
    } else {
      float f[3];
      for (int d = 0; d < 3; ++d) {
        f[d] = (float)p[d];
        if (!(f[d] < reps[r].Lf)) f[d] = 0.0f;
      }
      x[i] = make_v4f(f[0], f[1], f[2], pack_sp((uint32_t)sp_of[i], r));
    }
    ido[i] = pid;
  }
}

template <class T>
__global__ void k_count(const DevParams* __restrict__ Pp, const DevCtl* __restrict__ ctl,
                        const typename V4<T>::type* __restrict__ x, unsigned long long* __restrict__ counts) {
  const uint32_t n = ctl->n;
  const uint32_t stride = gridDim.x * blockDim.x;
  const uint32_t n_iter = (n + stride - 1) / stride;
  for (uint32_t it = 0; it < n_iter; ++it) {
    const uint32_t i = it * stride + blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t key = kNoKey;
    if (i < n) {
      const uint32_t wb = w_bits(x[i].w);
      key = (wb >> 8) * Pp->n_species + (wb & 0xFFu);
    }
    count_key(key, false, nullptr, counts);
  }
}

// Standalone per-pair probabilities (rd_pair_probs).
// p_enc and p_reac of one pair at start / end separations a, b (um); kMixed3D: the mixed step in
// 3D (no FP64 or 2D branch compiled, which keeps the streaming kernel's register count low).
template <bool kMixed3D>
__device__ __forceinline__ void pair_probs_one(const DevParams& P, const PairDev& pr, double a, double b, double& pe,
                                               double& prc, bool want_enc, bool want_reac) {
  // mixed: the separations rounded once to FP32 and scaled there (FP64 arithmetic runs at 1/64 of
  // the FP32 rate on this part)
  const float d0 = fmaf((float)a, pr.inv_sigma_f, -1.0f), d = fmaf((float)b, pr.inv_sigma_f, -1.0f);
  if (want_enc) {
    if (kMixed3D) {
      pe = (double)p_enc3_f(d, d0, pr.inv_tau_f);
    } else if (P.precision == RD_MIXED) {
      float pf;
      if (P.dim == 3) {
        pf = p_enc3_f(d, d0, pr.inv_tau_f);
      } else if (d <= 0.0f || d0 <= 0.0f) {
        pf = 1.0f;
      } else {
        const float xx = d * d0 * pr.inv_tau_f;
        pf = xx > 60.0f ? 0.0f : fminf(1.0f, fmaxf(0.0f, tab_eval(pr.tab_penc, d0, d) * expf(-xx)));
      }
      pe = (double)pf;
    } else {
      pe = p_enc_dim(P, pr, b / pr.sigma, a / pr.sigma);
    }
  }
  if (want_reac) {
    double v = pr.bc == RD_BC_ABS ? 1.0 : 0.0;
    if (pr.bc == RD_BC_RAD) {
      if (kMixed3D)
        v = (double)p_reac_tab(pr, d, d0);
      else
        v = P.precision == RD_MIXED ? (double)p_reac_tab(pr, d, d0) : p_reac_dim(P, pr, b / pr.sigma, a / pr.sigma);
    }
    prc = v;
  }
}

// Standalone pair probabilities (streaming).  With 16-byte aligned arrays each thread takes four
// consecutive pairs per pass through 16-byte loads and stores (more bytes in flight per thread);
// the remainder, or unaligned arrays, one pair per thread.
template <bool kMixed3D>
__global__ void k_pair_probs(const DevParams* __restrict__ Pp, int rule, const double* __restrict__ r0,
                             const double* __restrict__ r, int64_t n, double* __restrict__ p_enc,
                             double* __restrict__ p_reac) {
  const DevParams& P = *Pp;
  const PairDev& pr = P.pairs[rule];
  const bool we = p_enc != nullptr, wr = p_reac != nullptr;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
  const bool vec = (((uintptr_t)r0 | (uintptr_t)r | (uintptr_t)p_enc | (uintptr_t)p_reac) & 15u) == 0;
  int64_t done = 0;
  if (vec) {
    const int64_t n4 = n / 4;
    for (int64_t q = tid; q < n4; q += stride) {
      const double2 a01 = __ldcs(reinterpret_cast<const double2*>(r0) + 2 * q);
      const double2 a23 = __ldcs(reinterpret_cast<const double2*>(r0) + 2 * q + 1);
      const double2 b01 = __ldcs(reinterpret_cast<const double2*>(r) + 2 * q);
      const double2 b23 = __ldcs(reinterpret_cast<const double2*>(r) + 2 * q + 1);
      double e[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
      pair_probs_one<kMixed3D>(P, pr, a01.x, b01.x, e[0], c[0], we, wr);
      pair_probs_one<kMixed3D>(P, pr, a01.y, b01.y, e[1], c[1], we, wr);
      pair_probs_one<kMixed3D>(P, pr, a23.x, b23.x, e[2], c[2], we, wr);
      pair_probs_one<kMixed3D>(P, pr, a23.y, b23.y, e[3], c[3], we, wr);
      if (we) {
        __stcs(reinterpret_cast<double2*>(p_enc) + 2 * q, make_double2(e[0], e[1]));
        __stcs(reinterpret_cast<double2*>(p_enc) + 2 * q + 1, make_double2(e[2], e[3]));
      }
      if (wr) {
        __stcs(reinterpret_cast<double2*>(p_reac) + 2 * q, make_double2(c[0], c[1]));
        __stcs(reinterpret_cast<double2*>(p_reac) + 2 * q + 1, make_double2(c[2], c[3]));
      }
    }
    done = 4 * n4;
  }
  for (int64_t k = done + tid; k < n; k += stride) {
    double e = 0.0, c = 0.0;
    pair_probs_one<kMixed3D>(P, pr, r0[k], r[k], e, c, we, wr);
    if (we) p_enc[k] = e;
    if (wr) p_reac[k] = c;
  }
}

// Standalone propagation of encountered pairs (rd_propagate): one warp per pair, the same device
// functions as the step (length from the radial law, direction from the partial-wave law).
__global__ void k_propagate(const DevParams* __restrict__ Pp, int rule, const double* __restrict__ r0,
                            const double* __restrict__ u, int64_t n, double* __restrict__ out) {
  const DevParams& P = *Pp;
  const PairDev& pr = P.pairs[rule];
  const int dim = P.dim;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n; k += nw) {
    const double a0 = r0[3 * k] / pr.sigma, a1 = r0[3 * k + 1] / pr.sigma, a2 = dim == 3 ? r0[3 * k + 2] / pr.sigma : 0.0;
    const double l0 = sqrt(a0 * a0 + a1 * a1 + a2 * a2);
    const double R0 = l0 < 1.0 ? 1.0 : l0;
    double res[3] = {0.0, 0.0, 0.0};
    if (P.precision == RD_MIXED) {
      const float Rn = resample_tab_ni(pr, dim == 3, (float)u[4 * k], (float)R0);
      float uu[3] = {1.0f, 0.0f, 0.0f}, dir[3];
      if (l0 > 0.0) {
        uu[0] = (float)(a0 / l0); uu[1] = (float)(a1 / l0); uu[2] = (float)(a2 / l0);
      }
      bool ok;
      if (pr.tab_ang.v) {
        // the mixed step's tabulated law
        const float v = ang_table_sample(pr.tab_ang, dim, (float)u[4 * k + 1], Rn, (float)R0);
        ok = v == v;
        if (ok) ang_place<float>(dim, uu, v, (float)u[4 * k + 2], dir);
      } else {
        ok = ang_direction_warp<float>(dim, uu, (float)u[4 * k + 1], (float)u[4 * k + 2], Rn, (float)R0,
                                       (float)pr.tau, P.gl16, dir);
      }
      if (!ok) {
        dir[0] = uu[0]; dir[1] = uu[1]; dir[2] = uu[2];
      }
      for (int d = 0; d < dim; ++d) res[d] = (double)(Rn * dir[d]);
    } else {
      const double Rn = resample_dim_ni(P, pr, u[4 * k], R0);
      double uu[3] = {1.0, 0.0, 0.0}, dir[3];
      if (l0 > 0.0) {
        uu[0] = a0 / l0; uu[1] = a1 / l0; uu[2] = a2 / l0;
      }
      if (!ang_direction_warp<double>(dim, uu, u[4 * k + 1], u[4 * k + 2], Rn, R0, pr.tau, P.gl16, dir)) {
        dir[0] = uu[0]; dir[1] = uu[1]; dir[2] = uu[2];
      }
      for (int d = 0; d < dim; ++d) res[d] = Rn * dir[d];
    }
    if ((threadIdx.x & 31) == 0)
      for (int d = 0; d < 3; ++d) out[3 * k + d] = res[d] * pr.sigma;
  }
}

__global__ void k_resample(const DevParams* __restrict__ Pp, int rule, const double* __restrict__ r0,
                           const double* __restrict__ u, int64_t n, double* __restrict__ out) {
  const PairDev& pr = Pp->pairs[rule];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = (Pp->precision == RD_MIXED ? (double)resample_tab_ni(pr, Pp->dim == 3, (float)u[k], (float)(r0[k] / pr.sigma))
                                        : resample_dim(*Pp, pr, u[k], r0[k] / pr.sigma)) * pr.sigma;
}


// ================================================================================================
// Per-run FP32 tables for the mixed step, built in FP64 from the same pair functions.  Entry
// (i, j) sits at d0 = (i-1) h, d = (j-1) h; row/column 0 is a ghost filled by extrapolation.
// kind 0: p_reac; kind 1: F = p_enc e^{d d0/tau} (2D); kind 2: -ln(tail) of the propagator (2D);
// kind 3: the propagator sample V = R - 1 at U = exp(-t^2) (3D; second axis t with its own step).
// ================================================================================================
__global__ void k_tail_totals(const DevParams* __restrict__ Pp, int rule, int n0, double h, double* __restrict__ tot) {
  const PairDev& pr = Pp->pairs[rule];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n0; i += gridDim.x * blockDim.x) {
    const double R0 = 1.0 + fmax((i - 1) * h, 0.0);
    tot[i] = cdf2(pair2d(pr), R0 + 13.0 * pr.s, R0, Pp->gl16);
  }
}

__global__ void k_build_table(const DevParams* __restrict__ Pp, int rule, int kind, float* __restrict__ out, int n0,
                              int n1, double h, double h1, const double* __restrict__ tot) {
  const DevParams& P = *Pp;
  const PairDev& pr = P.pairs[rule];
  const int64_t total = (int64_t)n0 * n1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n1), j = (int)(e % n1);
    if (i == 0 || j == 0) continue;
    const double d0 = (i - 1) * h, d = (j - 1) * h;
    double v;
    if (kind == 0) {
      v = p_reac_dim(P, pr, 1.0 + d, 1.0 + d0);
    } else if (kind == 1) {
      const double x = d * d0 / pr.tau;
      v = x > 60.0 ? 1.0 : p_enc_dim(P, pr, 1.0 + d, 1.0 + d0) * exp(x);
      if (d <= 0.0 || d0 <= 0.0) v = 1.0;
    } else if (kind == 2) {
      const double t = 1.0 - cdf2(pair2d(pr), d, 1.0 + d0, P.gl16) / tot[i];
      v = t > 1e-30 ? -log(t) : 69.0;
    } else {
      // kind 3 (3D): V = R - 1 of the propagator sample at U = exp(-t^2), t on the second axis
      const double t = (j - 1) * h1;
      v = t > 0.0 ? resample3(exp(-t * t), 1.0 + d0, pr.s) - 1.0 : 0.0;
    }
    out[e] = (float)v;
  }
}

__global__ void k_table_ghosts(float* __restrict__ T, int n0, int n1) {
  // ghost column 0 of every row, then ghost row 0 (cubic extrapolation)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n0; i += gridDim.x * blockDim.x) {
    if (i == 0) continue;
    float* r = T + (size_t)i * n1;
    r[0] = 4.0f * r[1] - 6.0f * r[2] + 4.0f * r[3] - r[4];
  }
}

__global__ void k_table_ghost_row(float* __restrict__ T, int n1) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n1; j += gridDim.x * blockDim.x)
    T[j] = 4.0f * T[n1 + j] - 6.0f * T[2 * n1 + j] + 4.0f * T[3 * n1 + j] - T[4 * n1 + j];
}

// quad layout of a finished table: q[i n1 + j] = (v[i n1 + j-1], .., v[i n1 + j+2]), zero off the ends
__global__ void k_table_quads(const float* __restrict__ T, int n0, int n1, float4* __restrict__ Q) {
  const int64_t total = (int64_t)n0 * n1;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(k % n1);
    float4 q = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (j >= 1 && j + 2 < n1) q = make_float4(T[k - 1], T[k], T[k + 1], T[k + 2]);
    Q[k] = q;
  }
}

// 2D inverse table from a finished forward -ln(tail) table: at each node (d0, t) the V where the
// forward interpolant reaches t^2 (bisection on the interpolant, increasing in V).
__global__ void k_build_inverse2(Tab2 fwd, float* __restrict__ out, int n0, int n1, double h, double h1) {
  const int64_t total = (int64_t)n0 * n1;
  const float vmax = (float)(fwd.n1 - 4) * fwd.h1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n1), j = (int)(e % n1);
    if (i == 0 || j == 0) continue;
    const float d0 = (float)((i - 1) * h), t = (float)((j - 1) * h1), target = t * t;
    float lo = 0.0f, hi = vmax;
    for (int it = 0; it < 40; ++it) {
      const float mid = 0.5f * (lo + hi);
      if (tab_eval(fwd, d0, mid) < target)
        lo = mid;
      else
        hi = mid;
    }
    out[e] = j == 1 ? 0.0f : 0.5f * (lo + hi);
  }
}

void launch_build_table(const DevParams* P, int rule, int kind, float* out, float4* quad, int n0, int n1, double h,
                        double h1, double* tot, const Tab2* fwd, int device_sms, cudaStream_t s) {
  if (kind == 2) k_tail_totals<<<(n0 + 63) / 64, 64, 0, s>>>(P, rule, n0, h, tot);
  const int64_t total = (int64_t)n0 * n1;
  const int G = (int)std::min<int64_t>((total + 127) / 128, (int64_t)device_sms * 32);
  if (kind == 3 && fwd)
    k_build_inverse2<<<G, 128, 0, s>>>(*fwd, out, n0, n1, h, h1);
  else
    k_build_table<<<G, 128, 0, s>>>(P, rule, kind, out, n0, n1, h, h1, tot);
  k_table_ghosts<<<(n0 + 255) / 256, 256, 0, s>>>(out, n0, n1);
  k_table_ghost_row<<<(n1 + 255) / 256, 256, 0, s>>>(out, n1);
  k_table_quads<<<G, 128, 0, s>>>(out, n0, n1, quad);
}

// ================================================================================================
// The whole step as one cooperative launch (every block resident): the phases of the separate
// kernels above, in the same order and with the same device code, separated by bounded grid
// barriers instead of kernel boundaries; nsteps steps per launch with the state buffers
// alternating.  Block 0 stamps the global timer at each phase start (per-phase times).
// ================================================================================================
const char* const kFusedPhaseNames[kFusedPhases] = {"ph_prepare", "ph_scan_cells", "ph_scatter_cells", "ph_sweep",
                                                     "ph_match_trivial", "ph_match_resolve", "ph_angles",
                                                     "ph_compact"};

__device__ __forceinline__ void phase_stamp(DevCtl* ctl, int k) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned long long now;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
    if (k > 0) ctl->ph_acc[k - 1] += now - ctl->ph_t[k - 1];
    ctl->ph_t[k] = now;
  }
}

constexpr size_t kFusedSmemSweep = sizeof(uint2) * kSweepRanges * 256;

template <class T, bool kSplit, int kReach>
__global__ void __launch_bounds__(256, 2) k_step_fused(const StepLaunch L, const int nsteps) {
  using V = typename V4<T>::type;
  extern __shared__ __align__(16) unsigned char dsm[];
  DevCtl* ctl = L.ctl;
  const uint32_t split = L.sweep_split > 1 ? (uint32_t)L.sweep_split : 1u;
  for (int st = 0; st < nsteps; ++st) {
    const bool odd = st & 1;
    V* x0 = (V*)(odd ? L.x_next : L.x_cur);
    V* xo = (V*)(odd ? L.x_cur : L.x_next);
    uint32_t* id0 = odd ? L.id_next : L.id_cur;
    uint32_t* ido = odd ? L.id_cur : L.id_next;
    V* x0s = L.x0d ? (V*)L.x0d : x0;
    V* x1 = (V*)L.x1;
    V* sx0 = (V*)L.sx0;
    V* sx1 = (V*)L.sx1;
    V* prod = (V*)L.prodpos;
    phase_stamp(ctl, 0);
    ph_prepare<T>(L.P, ctl, L.reps, x0, id0, x1, L.status, L.cell_of, L.slot, L.cell_count, L.decay_list, L.counts,
                  L.n_counts, L.x0d ? x0s : (V*)nullptr, blockIdx.x, gridDim.x);
    if (!grid_barrier(ctl, false)) return;
    phase_stamp(ctl, 1);
    while (ph_scan_tile<uint32_t, LoadCellCount>(LoadCellCount{L.cell_count}, L.total_cells, nullptr, L.cell_start,
                                                 L.cell_count, L.agg32, L.incl32, L.flags, ctl, 0)) {
    }
    if (!grid_barrier(ctl, false)) return;
    phase_stamp(ctl, 2);
    ph_scatter<T>(ctl, x0s, x1, id0, L.cell_of, L.slot, L.cell_start, sx0, sx1, L.sidx, blockIdx.x, gridDim.x);
    if (!grid_barrier(ctl, false)) return;
    phase_stamp(ctl, 3);
    ph_sweep<T, kSplit, kReach>(L.P, ctl, L.reps, sx0, sx1, L.sidx, L.cell_start, L.total_cells, L.fired, L.fstate,
                                L.deg, L.matched, (uint32_t)L.cap_pairs, split, (uint2(*)[256])dsm, blockIdx.x,
                                gridDim.x);
    if (!grid_barrier(ctl, false)) return;
    phase_stamp(ctl, 4);
    ph_match_trivial(ctl, L.fired, L.fstate, L.deg, L.matched, L.conflict, L.accepted, L.best_key, L.best_pid,
                     (uint32_t)L.cap_pairs, L.crec, blockIdx.x, gridDim.x);
    if (!grid_barrier(ctl, false)) return;
    phase_stamp(ctl, 5);
    ph_match_resolve<T>(L.P, ctl, L.reps, L.fired, L.fstate, L.matched, L.conflict, L.accepted, L.best_key,
                        L.best_pid, L.decay_list, x0s, x1, id0, L.status, prod, L.deg, (uint32_t)L.cap_pairs,
                        L.rep_cons, L.rep_prod, L.repx, L.crec, L.ang_jobs, L.ang_cap);
    if (!grid_barrier(ctl, false)) return;
    phase_stamp(ctl, 6);
    if (L.angles) {
      ph_angles<T>(L.P, ctl, L.reps, L.ang_jobs, L.ang_cap, x1, prod, blockIdx.x, gridDim.x);
      if (!grid_barrier(ctl, false)) return;
    }
    phase_stamp(ctl, 7);
    ph_compact<T, 256>(L.P, ctl, L.reps, (const RepX*)L.repx, L.rep_cons, L.rep_prod, x0, x1, id0, L.status, prod,
                       L.agg64, L.incl64, L.flags + L.flag_stride, xo, ido, L.counts, L.n_counts, L.history,
                       L.history_len, (uint32_t*)(dsm + sizeof(unsigned long long) * kCompactTile),
                       (unsigned long long*)dsm, 7);
    if (st + 1 < nsteps) {
      // the next step starts from the committed state; after an error the state is kept and the
      // remaining steps are not taken
      if (!grid_barrier(ctl, false)) return;
      if (*(volatile int32_t*)&ctl->status != 0) return;
    }
  }
}

static size_t fused_smem_bytes(const StepLaunch& L) {
  const size_t hist = L.n_counts <= kSmemCounts ? (size_t)L.n_counts * 4 : 0;
  return std::max(kFusedSmemSweep, sizeof(unsigned long long) * kCompactTile + hist);
}

template <class T>
static void* fused_kernel_for(const StepLaunch& L) {
  const bool split = L.sweep_split > 1;
  if (L.reach == 2)
    return split ? (void*)k_step_fused<T, true, 2> : (void*)k_step_fused<T, false, 2>;
  return split ? (void*)k_step_fused<T, true, 1> : (void*)k_step_fused<T, false, 1>;
}

static void* fused_kernel(const StepLaunch& L) {
  return L.precision == RD_MIXED ? fused_kernel_for<float>(L) : fused_kernel_for<double>(L);
}

int fused_grid_size(const StepLaunch& L, int device_sms) {
  int per_sm = 0;
  // static (conflict rounds, ~28 KB) plus dynamic shared memory exceeds the default 48 KB per
  // block: opt in to the larger dynamic size (per kernel, per device)
  if (cudaFuncSetAttribute(fused_kernel(L), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_smem_bytes(L)) !=
      cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_kernel(L), 256, fused_smem_bytes(L)) !=
      cudaSuccess)
    return 0;
  per_sm = std::min(per_sm, 2);
  return per_sm >= 1 ? device_sms * per_sm : 0;
}

void launch_fused_steps(const StepLaunch& L, int nsteps, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)std::max(L.fused_grid, 1));
  cfg.blockDim = dim3(256u);
  cfg.dynamicSmemBytes = fused_smem_bytes(L);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {(void*)&L, (void*)&nsteps};
  cudaLaunchKernelExC(&cfg, fused_kernel(L), args);
}

// ================================================================================================
// host-side launchers
// ================================================================================================
static inline int grid_for(int64_t n, int block, int max_grid) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > max_grid) g = max_grid;
  return (int)g;
}

// Kernel launch with the programmatic-stream-serialization attribute (see pdl_enter).
template <typename... KArgs, typename... Args>
static void launch_k(bool pdl, void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                     Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Cooperative launch (all blocks resident at once, as the grid barrier requires; a grid larger
// than the device can hold is refused by the runtime), optionally with programmatic dependent
// launch: the kernel's blocks wait for the previous kernel before their first grid barrier.
template <typename... KArgs, typename... Args>
static void launch_coop(bool pdl, void (*kernel)(KArgs...), int grid, int block, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 2 : 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

int match_grid_size(int device_sms) {
  int a = 0, b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_match_resolve<float>, 256, 0) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_match_resolve<double>, 256, 0) != cudaSuccess)
    return 1;
  const int per_sm = std::min(std::min(a, b), 2);
  return per_sm >= 1 ? device_sms * per_sm : 1;
}

template <class T>
static void step_impl(const StepLaunch& L, cudaStream_t s, KernelTimer* timer) {
  using V = typename V4<T>::type;
  const int B = L.block;
  const int Gp = grid_for(L.cap_particles, B, L.max_grid);
  auto mark = [&](const char* name) {
    if (timer) timer->mark(name, s);
  };
  V* x0 = (V*)L.x_cur;
  V* xo = (V*)L.x_next;
  V* x1 = (V*)L.x1;
  V* sx0 = (V*)L.sx0;
  V* sx1 = (V*)L.sx1;
  V* prod = (V*)L.prodpos;
  const int64_t tile = 256 * (int64_t)kScanItems;

  mark("begin");
  const bool pdl = L.pdl;
  // start-of-step positions of the step proper: drifted copies when there is a drift step
  V* x0s = L.x0d ? (V*)L.x0d : x0;
  launch_k(pdl, k_prepare<T>, Gp, B, 0, s, L.P, L.ctl, L.reps, x0, L.id_cur, x1, L.status, L.cell_of, L.slot,
           L.cell_count, L.decay_list, L.counts, L.n_counts, L.x0d ? x0s : (V*)nullptr);
  mark("k_prepare");
  const int nbc = (int)((L.total_cells + tile - 1) / tile);
  launch_k(pdl, k_scan1<uint32_t, LoadCellCount>, nbc, 256, 0, s, LoadCellCount{L.cell_count}, L.total_cells,
           (const uint32_t*)nullptr, L.cell_start, L.cell_count, L.agg32, L.incl32, L.flags, L.ctl, 0);
  mark("k_scan_cells");
  launch_k(pdl, k_scatter_cells<T>, Gp, B, 0, s, L.ctl, x0s, x1, L.id_cur, L.cell_of, L.slot, L.cell_start, sx0,
           sx1, L.sidx);
  mark("k_scatter_cells");
  const uint32_t split = L.sweep_split > 1 ? (uint32_t)L.sweep_split : 1u;
  const int Gs = grid_for(L.cap_particles * (int64_t)split, 256, L.max_grid);
  auto sweep = [&](auto kernel) {
    launch_k(pdl, kernel, Gs, 256, 0, s, L.P, L.ctl, L.reps, sx0, sx1, L.sidx, L.cell_start, L.total_cells, L.fired,
             L.fstate, L.deg, L.matched, (uint32_t)L.cap_pairs, split);
  };
  if (L.reach == 2)
    split > 1 ? sweep(k_sweep<T, true, 2>) : sweep(k_sweep<T, false, 2>);
  else
    split > 1 ? sweep(k_sweep<T, true, 1>) : sweep(k_sweep<T, false, 1>);
  mark("k_sweep");
  launch_coop(pdl, k_match_resolve<T>, L.match_grid > 0 ? L.match_grid : 1, 256, s, L.P, L.ctl, L.reps, L.fired, L.fstate,
              L.matched, L.conflict, L.accepted, L.best_key, L.best_pid, L.decay_list, x0s, x1, L.id_cur, L.status,
              prod, L.deg, (uint32_t)L.cap_pairs, L.rep_cons, L.rep_prod, L.repx, L.crec, L.ang_jobs, L.ang_cap);
  mark("k_match_resolve");
  if (L.angles) {
    launch_k(pdl, k_angles<T>, L.match_grid > 0 ? L.match_grid : 1, 256, 0, s, L.P, L.ctl, (const RepDev*)L.reps,
             (const AngJob*)L.ang_jobs, L.ang_cap, x1, prod);
    mark("k_angles");
  }
  const int nbp = (int)((L.cap_particles + kCompactTile - 1) / kCompactTile);
  const size_t hist_bytes = L.n_counts <= kSmemCounts ? (size_t)L.n_counts * 4 : 0;
  // small systems: 1024 threads per tile (more independent placements per tile); large ones 256
  if (L.cap_particles <= (int64_t)1 << 20)
    launch_k(pdl, k_compact<T, 1024>, nbp, 1024, hist_bytes, s, L.P, L.ctl, L.reps, (const RepX*)L.repx, L.rep_cons,
             L.rep_prod, x0, x1, L.id_cur, L.status, prod, L.agg64, L.incl64, L.flags + L.flag_stride, xo, L.id_next,
             L.counts, L.n_counts, L.history, L.history_len);
  else
    launch_k(pdl, k_compact<T, 256>, nbp, 256, hist_bytes, s, L.P, L.ctl, L.reps, (const RepX*)L.repx, L.rep_cons,
             L.rep_prod, x0, x1, L.id_cur, L.status, prod, L.agg64, L.incl64, L.flags + L.flag_stride, xo, L.id_next,
             L.counts, L.n_counts, L.history, L.history_len);
  mark("k_compact");
}

// ================================================================================================
// State transfer on the device: validation + packing of a caller's state, and unpacking.
// ================================================================================================
// Validates element i of a caller's state (replica and species in range, (replica, id) strictly
// increasing, position inside the box) and packs it into out / ido; counts particles and the
// largest id per replica.  Any failure sets *err.
template <class V>
__global__ void k_set_state(const DevParams* __restrict__ Pp, const RepDev* __restrict__ reps, int64_t n,
                            const double* __restrict__ x, const int32_t* __restrict__ sp,
                            const uint32_t* __restrict__ id, const int32_t* __restrict__ rep, V* __restrict__ out,
                            uint32_t* __restrict__ ido, uint32_t* __restrict__ cnt, uint32_t* __restrict__ maxid,
                            int32_t* __restrict__ err) {
  const DevParams& P = *Pp;
  // every lane runs the same number of iterations so that the per-replica tallies can be reduced
  // across the warp (one atomic per replica present in the warp, not one per particle)
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n_iter = (n + stride - 1) / stride;
  for (int64_t it = 0; it < n_iter; ++it) {
    const int64_t i = it * stride + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool ok = i < n;
    int r = 0;
    if (ok) {
      r = rep ? rep[i] : 0;
      const int s = sp[i];
      ok = r >= 0 && r < P.n_replicas && s >= 0 && s < P.n_species;
      if (ok && i > 0) {
        const int rp = rep ? rep[i - 1] : 0;
        ok = r > rp || (r == rp && id[i] > id[i - 1]);
      }
      if (ok) {
        const RepDev& rd = reps[r];
        const double px = x[3 * i], py = x[3 * i + 1], pz = P.dim == 3 ? x[3 * i + 2] : 0.0;
        ok = px >= 0.0 && px < rd.L && py >= 0.0 && py < rd.L && (P.dim == 2 || (pz >= 0.0 && pz < rd.L));
        if (ok) {
          const uint32_t wb = ((uint32_t)r << 8) | (uint32_t)s;
          V v;
          if constexpr (sizeof(V) == 32) {
            v.x = px; v.y = py; v.z = pz;
            v.w = w_from_bits_d(wb);
          } else {
            float f[3] = {(float)px, (float)py, (float)pz};
            for (int d = 0; d < 3; ++d)
              if (!(f[d] < rd.Lf)) f[d] = 0.0f;
            v = make_float4(f[0], f[1], f[2], w_from_bits_f(wb));
          }
          out[i] = v;
          ido[i] = id[i];
        }
      }
      if (!ok) atomicOr(err, 1);
    }
    // lanes with a valid particle of the same replica add once
    const uint32_t key = ok ? (uint32_t)r : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
    const uint32_t mx = __reduce_max_sync(peers, ok ? id[i] + 1u : 0u);
    if (ok && (int)(threadIdx.x & 31) == __ffs(peers) - 1) {
      atomicAdd(&cnt[r], (uint32_t)__popc(peers));
      atomicMax(&maxid[r], mx);
    }
  }
}

// Replica segments and control words of an accepted state (one block; nothing if *err).
__global__ void k_set_state_finish(const DevParams* __restrict__ Pp, RepDev* __restrict__ reps, DevCtl* __restrict__ ctl,
                                   const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ maxid,
                                   const uint32_t* __restrict__ next_id_in, const int32_t* __restrict__ err, int64_t n,
                                   int64_t step) {
  __shared__ unsigned long long sm[32];
  if (*err) return;
  const DevParams& P = *Pp;
  unsigned long long carry = 0;
  for (int base = 0; base < P.n_replicas; base += blockDim.x) {
    const int r = base + (int)threadIdx.x;
    const unsigned long long c = r < P.n_replicas ? cnt[r] : 0ull;
    unsigned long long tot;
    const unsigned long long ex = carry + block_exclusive_scan<unsigned long long, int>(c, sm, tot);
    if (r < P.n_replicas) {
      reps[r].beg = (uint32_t)ex;
      reps[r].end = (uint32_t)(ex + c);
      reps[r].next_id = next_id_in ? max(next_id_in[r], maxid[r]) : maxid[r];
    }
    carry += tot;
  }
  if (threadIdx.x == 0) {
    ctl->n = (uint32_t)n;
    ctl->step = (uint32_t)step;
    ctl->t = (double)step * P.dt;
    ctl->status = 0;
  }
}

// Unpacks n records into positions (n x 3 doubles), species and replica (each optional).
template <class V>
__global__ void k_get_state(const V* __restrict__ in, int64_t n, double* __restrict__ x, int32_t* __restrict__ sp,
                            int32_t* __restrict__ rep) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const V v = in[i];
    const uint32_t wb = w_bits(v.w);
    if (x) {
      x[3 * i] = (double)v.x;
      x[3 * i + 1] = (double)v.y;
      x[3 * i + 2] = (double)v.z;
    }
    if (sp) sp[i] = (int32_t)(wb & 0xFFu);
    if (rep) rep[i] = (int32_t)(wb >> 8);
  }
}

void launch_set_state(const StepLaunch& L, int64_t n, const double* x, const int32_t* sp, const uint32_t* id,
                      const int32_t* rep, void* out, uint32_t* ido, uint32_t* cnt, uint32_t* maxid,
                      const uint32_t* next_id_in, int32_t* err, int64_t step, cudaStream_t s) {
  const int G = grid_for(n, 256, L.max_grid);
  if (n > 0) {
    if (L.precision == RD_MIXED)
      k_set_state<float4><<<G, 256, 0, s>>>(L.P, L.reps, n, x, sp, id, rep, (float4*)out, ido, cnt, maxid, err);
    else
      k_set_state<d4><<<G, 256, 0, s>>>(L.P, L.reps, n, x, sp, id, rep, (d4*)out, ido, cnt, maxid, err);
  }
  k_set_state_finish<<<1, 256, 0, s>>>(L.P, L.reps, L.ctl, cnt, maxid, next_id_in, err, n, step);
}

void launch_get_state(const StepLaunch& L, const void* in, int64_t n, double* x, int32_t* sp, int32_t* rep,
                      cudaStream_t s) {
  if (n <= 0) return;
  const int G = grid_for(n, 256, L.max_grid);
  if (L.precision == RD_MIXED)
    k_get_state<float4><<<G, 256, 0, s>>>((const float4*)in, n, x, sp, rep);
  else
    k_get_state<d4><<<G, 256, 0, s>>>((const d4*)in, n, x, sp, rep);
}

void launch_cell_scan(const StepLaunch& L, cudaStream_t s) {
  const int64_t tile = 256 * (int64_t)kScanItems;
  const int nbc = (int)((L.total_cells + tile - 1) / tile);
  k_scan1<uint32_t, LoadCellCount><<<nbc, 256, 0, s>>>(LoadCellCount{L.cell_count}, L.total_cells, nullptr,
                                                       L.cell_start, L.cell_count, L.agg32, L.incl32, L.flags,
                                                       L.ctl, 0);
}

void launch_step(const StepLaunch& L, cudaStream_t s, KernelTimer* timer) {
  if (L.fused && !timer) {
    launch_fused_steps(L, 1, s);
    return;
  }
  if (L.precision == RD_MIXED)
    step_impl<float>(L, s, timer);
  else
    step_impl<double>(L, s, timer);
}

void launch_init_positions(const StepLaunch& L, const int32_t* rep_of, const int32_t* sp_of, const uint32_t* id_of,
                           uint32_t n, cudaStream_t s) {
  const int G = grid_for(n, 256, L.max_grid);
  if (L.precision == RD_MIXED)
    k_init_positions<float><<<G, 256, 0, s>>>(L.P, L.reps, rep_of, sp_of, id_of, n, (float4*)L.x_cur, L.id_cur);
  else
    k_init_positions<double><<<G, 256, 0, s>>>(L.P, L.reps, rep_of, sp_of, id_of, n, (d4*)L.x_cur, L.id_cur);
}

__global__ void k_zero_counts(unsigned long long* __restrict__ counts, int n_counts) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_counts; i += gridDim.x * blockDim.x) counts[i] = 0;
}

// history entry of the current step from the counts (after initialisation or a state upload)
__global__ void k_history_now(const DevParams* __restrict__ Pp, const DevCtl* __restrict__ ctl,
                              const unsigned long long* __restrict__ counts, long long* __restrict__ history,
                              int history_len) {
  const int ns = Pp->n_species;
  species_totals(counts, Pp->n_replicas, ns, history + (size_t)(ctl->step % (uint32_t)history_len) * ns);
}

void launch_count(const StepLaunch& L, cudaStream_t s) {
  k_zero_counts<<<grid_for(L.n_counts, 256, 64), 256, 0, s>>>(L.counts, L.n_counts);
  const int G = grid_for(L.cap_particles, 256, L.max_grid);
  if (L.precision == RD_MIXED)
    k_count<float><<<G, 256, 0, s>>>(L.P, L.ctl, (const float4*)L.x_cur, L.counts);
  else
    k_count<double><<<G, 256, 0, s>>>(L.P, L.ctl, (const d4*)L.x_cur, L.counts);
  if (L.history && L.history_len > 0) k_history_now<<<1, 256, 0, s>>>(L.P, L.ctl, L.counts, L.history, L.history_len);
}

void launch_pair_probs(const DevParams* P, int rule, const double* r0, const double* r, int64_t n, double* pe,
                       double* pr, int max_grid, bool mixed3d, cudaStream_t s) {
  if (mixed3d)
    k_pair_probs<true><<<grid_for(n, 256, max_grid), 256, 0, s>>>(P, rule, r0, r, n, pe, pr);
  else
    k_pair_probs<false><<<grid_for(n, 256, max_grid), 256, 0, s>>>(P, rule, r0, r, n, pe, pr);
}

void launch_propagate(const DevParams* P, int rule, const double* r0, const double* u, int64_t n, double* out,
                      int max_grid, cudaStream_t s) {
  k_propagate<<<grid_for(n * 32, 128, max_grid), 128, 0, s>>>(P, rule, r0, u, n, out);
}

void launch_resample(const DevParams* P, int rule, const double* r0, const double* u, int64_t n, double* out,
                     int max_grid, cudaStream_t s) {
  k_resample<<<grid_for(n, 128, max_grid), 128, 0, s>>>(P, rule, r0, u, n, out);
}

// Angle table of one pair rule (mixed step): one warp per node (a, b) of the law at
// R0 = 1 + (a - 1) h, R' = 1 + (b - 1) h, FP64.  The ghost row and column (a = 0, b = 0: R0 or R'
// = 1 - h) hold the law's own continuation below contact, which keeps the interpolation's first
// interval as accurate as the others (a linear extrapolation there cost a factor ten).
__global__ void __launch_bounds__(128) k_ang_table(const DevParams* __restrict__ Pp, int dim, double tau, double h,
                                                   int n0, int n1, float* __restrict__ out) {
  __shared__ double dn[4][32 * kAngBuildSlots];
  const int w = threadIdx.x >> 5;
  const int64_t nodes = (int64_t)n0 * n1;
  for (int64_t q = (int64_t)blockIdx.x * 4 + w; q < nodes; q += (int64_t)gridDim.x * 4) {
    const int a = (int)(q / n1), b = (int)(q % n1);
    ang_table_node(dim, 1.0 + (b - 1) * h, 1.0 + (a - 1) * h, tau, Pp->gl16, dn[w],
                   out + ((size_t)a * n1 + b) * kAngTabStride);
  }
}

void launch_build_ang_table(const DevParams* P, int dim, double tau, double h, int n0, int n1, float* out,
                            int device_sms, cudaStream_t s) {
  const int64_t nodes = (int64_t)n0 * n1;
  const int G = (int)std::min<int64_t>((nodes + 3) / 4, (int64_t)device_sms * 16);
  k_ang_table<<<G, 128, 0, s>>>(P, dim, tau, h, n0, n1, out);
}

}  // namespace rd
