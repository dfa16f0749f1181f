// Launch interface between the host runtime and the step kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "rd_internal.cuh"

namespace rd {

// Device buffers and sizes of one step (pointers are device addresses).
struct StepLaunch {
  int precision;
  int block;
  int max_grid;
  int scan_items;
  bool pdl;                    // programmatic dependent launch between the step kernels
  int match_grid;              // blocks of the cooperative matching launch (all resident)
  int fused;                   // 1: the whole step as one cooperative launch (k_step_fused)
  int fused_grid;              // blocks of that launch (all resident)
  int angles;                  // 1: exact directions of encountered pairs (angle pass after the resolution)
  AngJob* ang_jobs;            // angle jobs of a step (ang_cap entries)
  uint32_t ang_cap;
  void* x0d;                   // drifted start positions (drift step only; nullptr without drift)
  ConflictRec* crec;           // conflict pairs of the matching rounds (fired-pair capacity)
  RepX* repx;                  // per-replica placement of the compaction
  uint32_t* rep_cons;          // per-replica particles consumed this step
  uint32_t* rep_prod;          // per-replica products formed this step
  int sweep_split;             // threads per binned particle in the sweep: 1 or the stencil rows
  int reach;                   // stencil reach in cells: 1 (cell edge >= r_cut) or 2 (2D, >= r_cut / 2)
  int64_t cap_particles, cap_pairs, total_cells;
  int n_counts;
  const DevParams* P;
  DevCtl* ctl;
  RepDev* reps;
  void* x_cur;
  void* x_next;
  uint32_t* id_cur;
  uint32_t* id_next;
  void* x1;
  void* sx0;                 // cell-ordered start / end positions, interleaved: record k at sx0[2k],
  void* sx1;                 // sx1[2k] (sx1 = sx0 + one record)
  void* prodpos;
  uint32_t* status;
  int32_t* matched;
  uint32_t* deg;
  uint32_t* cell_of;
  uint32_t* slot;
  uint32_t* cell_count;
  uint32_t* cell_start;
  uint32_t* sidx;
  uint32_t* decay_list;
  uint32_t* agg32;             // per-tile aggregates / inclusive prefixes of the cell scan
  uint32_t* incl32;
  unsigned long long* agg64;   // ... of the compaction scan
  unsigned long long* incl64;
  uint32_t* flags;             // 2 x flag_stride tile flags
  int64_t flag_stride;
  uint32_t* accepted;          // accepted pair list
  FiredPair* fired;
  uint32_t* fstate;
  uint32_t* conflict;
  unsigned long long* best_key;
  unsigned long long* best_pid;
  unsigned long long* counts;
  long long* history;          // history_len x n_species totals per step (ring), may be null
  int history_len;
};

// CUDA-event marks between kernel groups of one (non-graph) step.
struct KernelTimer {
  std::vector<cudaEvent_t> events;
  std::vector<std::string> names;
  size_t used = 0;
  void reset() { used = 0; names.clear(); }
  void mark(const char* name, cudaStream_t s) {
    if (used == events.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      events.push_back(e);
    }
    cudaEventRecord(events[used++], s);
    names.push_back(name);
  }
  void destroy() {
    for (auto e : events) cudaEventDestroy(e);
    events.clear();
    names.clear();
    used = 0;
  }
};

// blocks of the cooperative matching launch that fit on the device at once (>= 1)
int match_grid_size(int device_sms);
// blocks of the fused step launch for L's precision, sweep split and reach that fit on the device
// at once (at most 2 per SM); 0 if the kernel cannot be made resident (the step then uses separate
// kernels)
int fused_grid_size(const StepLaunch& L, int device_sms);
// one step; with L.fused and no timer, the fused single-launch step
void launch_step(const StepLaunch& L, cudaStream_t s, KernelTimer* timer);
// nsteps steps as ONE fused cooperative launch (buffers alternate inside; L.x_cur holds the state
// at the start and, for even nsteps, at the end)
void launch_fused_steps(const StepLaunch& L, int nsteps, cudaStream_t s);
// names of the fused step's phases (index k of DevCtl::ph_acc)
constexpr int kFusedPhases = 8;
extern const char* const kFusedPhaseNames[kFusedPhases];
// device-side state transfer (validation + packing into out / ido; unpacking)
void launch_set_state(const StepLaunch& L, int64_t n, const double* x, const int32_t* sp, const uint32_t* id,
                      const int32_t* rep, void* out, uint32_t* ido, uint32_t* cnt, uint32_t* maxid,
                      const uint32_t* next_id_in, int32_t* err, int64_t step, cudaStream_t s);
void launch_get_state(const StepLaunch& L, const void* in, int64_t n, double* x, int32_t* sp, int32_t* rep,
                      cudaStream_t s);
// the cell scan of a step on its own (bounded-wait check)
void launch_cell_scan(const StepLaunch& L, cudaStream_t s);
void launch_init_positions(const StepLaunch& L, const int32_t* rep_of, const int32_t* sp_of, const uint32_t* id_of,
                           uint32_t n, cudaStream_t s);
void launch_count(const StepLaunch& L, cudaStream_t s);
void launch_pair_probs(const DevParams* P, int rule, const double* r0, const double* r, int64_t n, double* pe,
                       double* pr, int max_grid, bool mixed3d, cudaStream_t s);
// kind 3 with fwd != nullptr: the 2D inverse table from the forward -ln(tail) table fwd
void launch_build_table(const DevParams* P, int rule, int kind, float* out, float4* quad, int n0, int n1, double h,
                        double h1, double* tot, const Tab2* fwd, int device_sms, cudaStream_t s);
void launch_resample(const DevParams* P, int rule, const double* r0, const double* u, int64_t n, double* out,
                     int max_grid, cudaStream_t s);
// Angle table of one pair rule into out (n0 x n1 x (kAngTabU + 3) floats), on stream s.
void launch_build_ang_table(const DevParams* P, int dim, double tau, double h, int n0, int n1, float* out,
                            int device_sms, cudaStream_t s);
void launch_propagate(const DevParams* P, int rule, const double* r0, const double* u, int64_t n, double* out,
                      int max_grid, cudaStream_t s);

// First-passage refinement of encountered pairs (one pair rule, one step length).
constexpr int kFptMaxLevels = 24;
struct FptLevel {              // p_enc data of the half intervals of level l (2D)
  const void* nodes;           // Weber nodes for tau / 2^(l+1) (nullptr: small-time series)
  int n_nodes;
};
struct FptArgs {
  int dim, levels;
  int f32;                     // 3D in FP32 on contact distances (mixed-precision handles)
  uint32_t max_attempts;
  uint32_t seed_lo, seed_hi;
  double tau;                  // D dt / sigma^2 of the rule
  double sigma;
  const void* ser;             // 2D small-time series coefficients of the rule
  FptLevel lv[kFptMaxLevels];
};
constexpr uint32_t kFptBudget = 256;        // draws per pair in the lane-per-pair phase
constexpr uint32_t kFptWarpBudget = 4352;   // draws per pair before the block-per-pair phase
constexpr uint32_t kFptBlockBudget = 32768; // draws per pair before the grid phase
constexpr int kFptBlockThreads = 512;       // threads per pair in the block-per-pair phase
constexpr int kFptGridThreads = 256;        // threads per block (and attempts per chunk) of the grid phase
constexpr uint32_t kFptGridGroups = 4;      // block groups of the grid phase, each searching its own pairs
// control words of one refinement launch: a 64-bit pair counter, then per round of phases 2-4 the
// queue lengths and work counters of the warp, block and grid phases
enum : int {
  kFptPairCtr = 0, kFptRound0 = 8, kFptRoundWords = 8,
  kFptWarpIn = 0, kFptWarpNext = 1, kFptBlockIn = 2, kFptBlockNext = 3, kFptGridIn = 4,
  kFptCtlWords = kFptRound0 + kFptRoundWords * (kFptMaxLevels + 1)
};
struct FptItem {                            // a pair's state when it moves to a later phase
  double Ri, Rf, t;
  uint32_t k, b, a, l;
};
struct FptSearch {                          // the grid phase's search state of one pair
  uint32_t next_chunk, winner, exited, pad;
};
void launch_first_passage(const FptArgs& A, const double* r0, const double* r, const uint64_t* stream, int64_t n,
                          uint32_t* bin, double* r_lo, double* r_hi, uint32_t* attempts, FptItem* warp_q[2],
                          FptItem* block_q, FptItem* grid_q, FptSearch* search, uint32_t* qctl, int device_sms,
                          cudaStream_t s);

}  // namespace rd
