// Engine: device memory, launch sequence and CUDA-graph replay for one packed
// set of periodic DPD boxes.  The single-box context, the multi-box batch and
// the request queue all drive an Engine.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dpd_device.cuh"
#include "kernels.h"

namespace dpd {

// NVTX range over a host call: its launches and copies appear under this
// name in a profiler's timeline (Nsight Systems, ncu --nvtx).  Header-only
// NVTX; without a tool attached a range costs a few nanoseconds.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Capacity of one packed set: particle slots are 26-bit indices in the pair
// lists, and the cell starts (cells + 1 entries) fit one scan.
constexpr long long kMaxSlots = 1LL << 26;
constexpr long long kMaxCellEntries = (long long)kScanMaxTiles * kScanTile - 1;

// Records a message for dpd_last_error() and returns `code`.
int set_error(int code, const char *fmt, ...);
void clear_error();

#define DPD_CUDA_TRY(expr)                                                                  \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return ::dpd::set_error(e_ == cudaErrorMemoryAllocation ? -2 : -3, "%s: %s (%s:%d)", \
                              #expr, cudaGetErrorString(e_), __FILE__, __LINE__);           \
  } while (0)

// Host description of one box.
struct BoxParams {
  double L[3];
  double a, gamma, kT, rc, dt, mass, kexp;
  double fb;        // body force magnitude
  int fb_mode;      // 0 none, 1 constant, 2 periodic Poiseuille
  int fb_flow, fb_grad;
  uint64_t seed;
  int noise;        // 0 uniform, 1 Gaussian
  // several species: nspec 2..4 with symmetric tables at [4 s + t]
  // (1: one species with a, gamma, rc above)
  int nspec = 1;
  double sa[16] = {}, sg[16] = {}, src[16] = {};
};

// Validates the parameters and derives the cell grid; returns DPD_OK or DPD_ERR_ARG.
int check_params(const BoxParams &bp, int n_out[3]);

BoxDev make_box_dev(const BoxParams &bp, int cellBase, int pbase, int np);

struct DeviceArrays {
  float4 *pos = nullptr, *vel = nullptr, *frc = nullptr, *pos2 = nullptr, *vel2 = nullptr;
  int *cellOf = nullptr, *slotIn = nullptr, *keyTmp = nullptr;
  int *count = nullptr, *start = nullptr, *bsum = nullptr;
  BoxDev *boxes = nullptr;
  int *pbase = nullptr;
  BoxState *st = nullptr;
  unsigned *err = nullptr;
  StatsWork *work = nullptr;
  double *part = nullptr;
  size_t capP = 0, capC = 0, capB = 0, capW = 0;
};

class Engine {
 public:
  Engine();
  ~Engine();
  Engine(const Engine &) = delete;
  Engine &operator=(const Engine &) = delete;

  int init();                       // binds the current device, prepares kernels
  int set_stream(cudaStream_t s);
  int set_stencil(int stencil);
  // Force-kernel tiling: use_tiles = 0 selects one thread per particle reading
  // neighbours from global memory; tc / stage_cap > 0 override the choice by
  // density (cells per tile, staged particles per block).
  int set_tiling(int use_tiles, int tc, int stage_cap);
  // Direct force-kernel variant: -1 (default) picks per box from the tuning
  // table by density; 0..kNumForceVariants-1 forces one for every box.
  int set_variant(int variant);
  // Fuse each full-stencil step's next kick/drift/bin into its force kernel.
  int set_fuse(bool on);
  bool fuse() const { return fuse_; }
  int variant_override() const { return variant_override_; }
  // Re-derive the per-band variants (after the tuning table changed).
  int refresh_bands();
  const StepConfig &step_config() const { return cfg_; }

  // Lay out boxes: particle counts per box decide the slot ranges.  Allocates
  // (or grows) device memory and uploads descriptors.  Box state is reset.
  int layout(const std::vector<BoxParams> &params, const std::vector<int64_t> &np);
  // Re-upload descriptors after a parameter change (same layout).
  int update_params(const std::vector<BoxParams> &params);
  // A new state with the same particle counts and parameters: the packing,
  // the tables and the captured graphs stay, and the box states are reset
  // as layout() resets them.  Returns false (nothing changed) when the
  // counts differ or sampling is on, and layout() is needed.
  bool restart_same_layout(const std::vector<int64_t> &np);

  // Load particles of one box (n x 3 host or device arrays).
  int load_box(int box, const float *pos, const float *vel, bool device_ptr,
               const int32_t *species = nullptr);
  // Host mirror of a box's step state; takes effect at the next rebuild().
  void set_box_state(int box, uint64_t step0, int64_t remaining);
  // Cell-list build and force at each box's current step, without moving
  // particles (used after loading).  Boxes that were not reloaded keep their
  // order and get the same force again.
  int rebuild();
  const BoxState &box_state(int b) const { return st_host_[b]; }
  // Change how many steps a box may still take (0 freezes it); uploads at once.
  int set_remaining(int box, int64_t remaining);

  int step(int64_t nsteps);         // enqueue nsteps steps (graph chunks + direct launches)
  // Run nsteps steps with per-stage CUDA events (synchronising after each
  // step); adds the mean milliseconds of each stage to stage_ms[kNumStages].
  int profile(int64_t nsteps, double *stage_ms);
  int sync();
  int check_error();                // reads and clears the device error word
  // The same in two halves, so that a read-out that synchronises anyway
  // brings the error word back with its data: fetch_error() enqueues the
  // copy to pinned memory, take_error() (after a synchronisation) reads and
  // clears it.  gather() and box_sums() fetch; their callers take.
  int fetch_error();
  int take_error();

  int gather(int box, float *pos, float *vel, float *frc, bool device_ptr);
  // Raw slot-order copies of one box's pos / vel / frc (float4) to or from
  // host memory, for checkpoints.  Synchronises the stream.
  int copy_box_raw(int box, float4 *pos, float4 *vel, float4 *frc, bool to_host);
  void set_box_state_raw(int box, const BoxState &s) { st_host_[box] = s; }

  // ---- served form
  // Statistics sampling every `every` box steps into per-box FP64
  // accumulators {samples, sum v^2, sum frc.w, slab sums, slab counts};
  // every = 0 turns it off.
  int enable_sampling(int every, int nbins);
  int sample_fields() const { return 3 + 2 * nbins_; }
  // Boxes sample only at steps > from (host mirror; uploaded at rebuild).
  void set_sample_from(int box, long long from) { from_h_[box] = from; }
  int zero_acc(int box);
  int read_acc(int box, double *out);  // synchronises the stream
  // Draw a box's initial state on the device (uniform positions, Maxwellian
  // velocities of variance kT/m, zero mean momentum).
  int init_box(int box, uint64_t seed);
  // New packing: box k of `params` is old box src[k] (its particles, step
  // state and accumulators are kept) or new (src[k] < 0, to be loaded or
  // initialised).  Call rebuild() before stepping.
  int repack(const std::vector<BoxParams> &params, const std::vector<int64_t> &np,
             const std::vector<int> &src);
  // FP64 partial sums per box: {sum v (3), sum v^2, sum frc.w, count}.
  int box_sums(std::vector<double> &sums);

  int nbox() const { return (int)boxes_.size(); }
  int ntot() const { return ntot_; }
  int ncell() const { return ncell_; }
  int64_t box_n(int b) const { return pbase_[b + 1] - pbase_[b]; }
  const BoxParams &params(int b) const { return params_[b]; }
  cudaStream_t stream() const { return stream_; }
  size_t device_bytes() const;
  int graph_chunk = 32;             // steps per captured graph

 private:
  Packed packed() const;
  int reserve(size_t np, size_t nc, size_t nb);
  int free_all();
  int capture_graph(int nsteps, cudaGraphExec_t *out);
  void drop_graph();

  int device_ = -1;
  cudaStream_t stream_ = nullptr;   // caller's stream (nullptr: legacy default)
  cudaStream_t cap_ = nullptr;      // private stream used to capture graphs
  StepConfig cfg_{};
  int tile_tc_override_ = 0;      // cells per tile forced by set_tiling (0: by density)
  int stage_cap_override_ = 0;    // staging capacity forced by set_tiling (0: by density)
  std::vector<int4> tiles_h_;
  int4 *d_tiles_ = nullptr;
  int *d_mixed_ = nullptr;        // first slots of the bands' two-box warps
  size_t cap_mixed_ = 0;
  size_t cap_tiles_ = 0;
  int build_tiles();
  int build_bands();
  // Work items of the brick force kernel for every box (brick_beg_[b] ..
  // brick_beg_[b + 1] are box b's).
  int build_bricks();
  std::vector<int4> bricks_h_;
  std::vector<int> brick_beg_;
  int4 *d_bricks_ = nullptr;
  size_t cap_bricks_ = 0;
  int variant_override_ = -1;
  bool fuse_ = true;
  bool fused_steps() const;  // fusion applies to this engine's steps now
  std::vector<BoxParams> params_;
  std::vector<BoxDev> boxes_;
  std::vector<int> pbase_;
  std::vector<BoxState> st_host_;   // host mirror of the device box states
  int ntot_ = 0, ncell_ = 0;
  DeviceArrays d_;
  std::vector<StatsWork> work_;
  std::vector<int> wbeg_;            // first work item of each box (nbox + 1)
  int *d_wbeg_ = nullptr;
  double *h_sum_ = nullptr;  // pinned per-box statistics totals
  unsigned *h_err_ = nullptr;  // pinned copy of the device error word
  size_t cap_hsum_ = 0;
  size_t cap_wbeg_ = 0;
  bool work_dirty_ = true;
  int build_work();
  int sample_every_ = 0, nbins_ = 0;
  std::vector<long long> from_h_;
  long long *d_from_ = nullptr;
  double *d_acc_ = nullptr, *d_spart_ = nullptr;
  size_t cap_from_ = 0, cap_acc_ = 0, cap_spart_ = 0;
  int ensure_sampling_buffers();
  int launch_extra(const Packed &P, cudaStream_t s);
  cudaGraphExec_t graph_ = nullptr;   // graph_chunk steps
  cudaGraphExec_t graph1_ = nullptr;  // one step (calls that end with a single step)
};

}  // namespace dpd
