// Host-side launchers of the DPD kernels (kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "dpd_device.cuh"

namespace dpd {

// Device pointers and sizes of one packed set of boxes.  Passed by value to
// every kernel.  `single` duplicates boxes[0] when nbox == 1 so that the
// single-box kernels read box constants from the parameter bank.
struct Packed {
  float4 *pos, *vel, *frc;     // primary arrays, cell order
  float4 *pos2, *vel2;         // integrated copies before the reorder; staging
  int *cellOf;                 // packed global cell of each slot (pre-reorder order)
  int *slotIn;                 // arrival rank of each slot inside its cell
  int *keyTmp;                 // old slot index at each arrival position
  int *count;                  // particles per cell (zeroed by the scan)
  int *start;                  // exclusive scan of count, ncell + 1 entries
  int *bsum;                   // per-tile sums of the scan
  const BoxDev *boxes;
  const int *pbase;            // nbox + 1 entries
  BoxState *st;
  unsigned *err;
  int ntot, ncell, nbox;
  BoxDev single;
};

// Tiling of the staged force kernel.  Single box: tiles are computed from
// the block index (tc cells per tile, tpr tiles per row).  Packed boxes:
// `list` holds one int4 {box, cy, cz, cx0 | nc << 16} per tile.
constexpr int kTileThreads = 128;
constexpr int kTileMaxCells = 64;
struct TileGrid {
  const int4 *list;
  int ntiles;
  int tc;         // cells per tile
  int tpr;        // tiles per row
  int stage_cap;  // staged particles per block (positions + velocities)
};

// Brick force kernel (half stencil, brick.cu): one block per work item
// {box, y0 | by << 16, z0 | bz << 16, s0 | s1 << 16}, target rows y0 .. y0+by-1
// and z0 .. z0+bz-1 over x slices [s0, s1), staged through shared memory
// in chunks of at most kBrickWMax slices.
constexpr int kBrickThreads = 256;
constexpr int kBrickMaxBY = 4, kBrickMaxBZ = 4;
constexpr int kBrickMaxRows = (kBrickMaxBY + 2) * (kBrickMaxBZ + 1);
constexpr int kBrickWMax = 32;
constexpr int kBrickListCap = 24;
constexpr int kBrickMaxCaps = 1024;  // staged particles per block, at most
constexpr int kBrickCaps = 896;      // staged particles per block used
constexpr int kBrickVariant = 13;    // the force variant that selects it
struct BrickGrid {
  const int4 *items;  // device, ordered by box
  int nitems;
  int caps;           // staged particles per block
};
size_t brick_smem_bytes(int caps);
cudaError_t prepare_brick();
cudaError_t launch_force_brick(const Packed &P, const BrickGrid &G, int i0, int i1,
                               cudaStream_t s);

// A contiguous slot range whose force kernel uses one variant.
struct ForceBand {
  int slot0, slot1, variant;
  int gauss;  // 1: the band needs the general kernel (Gaussian noise or several species)
  // packed sets: the band's warps whose slots span two boxes (first slots at
  // StepConfig::mixed_warps[mw_off ..]); warp-cooperative variants skip them
  // and a second launch runs them with the per-lane drain
  int mw_off, mw_count;
  int item0, item1;  // the band's brick work items (brick variant)
  int box0, box1;    // the band's boxes (whole boxes, slots slot0 .. slot1)
};

// Box-grouped launches (group.cu), packed sets with the half stencil:
// every block takes slots of one box only, and the constants of up to
// kGroupBoxes boxes travel in the kernel parameters, so each block reads
// its box's constants as block-uniform values, as the single-box kernels
// read theirs.  BoxHot holds the constants the half stencil's direct force
// routine reads for uniform noise and one species.
struct BoxHot {
  float L[3];
  float invh[3];
  int n[3];
  float xwin;
  int cellBase, pbase, np;
  float a, gamma, sig, rc2, inv_rc, kexp;
  float fb, fb_half;
  int fb_mode, fb_flow, fb_grad;
  uint32_t seed_lo, seed_hi;
};
constexpr int kGroupBoxes = 240;
struct BoxGroup {
  int nbox;                  // boxes in this launch
  int blk[kGroupBoxes + 1];  // first block of each box; blk[nbox] = blocks launched
  int box[kGroupBoxes];      // each box's index in the packed set
  BoxHot hot[kGroupBoxes];
};
// kernel parameters are limited to 32764 bytes
static_assert(sizeof(BoxGroup) + sizeof(Packed) + 64 <= 32764, "grouped launch parameters");
BoxHot box_hot(const BoxDev &B);
// Whether the grouped launch serves this band's kernel: the half stencil's
// spread-drain variants (10-12) for uniform noise and one species.
inline bool grouped_variant(int v, bool general, bool half) {
  return half && !general && v >= 10 && v <= 12;
}
// The force stage of boxes [box0, box1) of a packed set (host copies of the
// box constants in hboxes), in launches of at most kGroupBoxes boxes.
cudaError_t launch_force_group(const Packed &P, const BoxDev *hboxes, int box0, int box1,
                               int variant, cudaStream_t s);
constexpr int kMaxBands = 8;
constexpr int kNumForceVariants = 14;

// How a step is launched.
struct StepConfig {
  int stencil = 0;       // 0 full, 1 half
  bool tiles = false;    // full stencil: staged tiles (true) or one thread per particle
  TileGrid grid{};
  int nbands = 0;        // 0: one band over every slot with variant 0
  ForceBand band[kMaxBands]{};
  const int *mixed_warps = nullptr;  // device: first slots of the bands' two-box warps
  BrickGrid bricks{};                // work items of the brick force kernel
  const BoxDev *hboxes = nullptr;    // host copies of the box constants (grouped launches)
  bool grouped = true;               // packed half stencil: box-grouped launches
};
// Whether the variant drains over the whole warp (balanced or spread): such
// kernels evaluate other lanes' entries with their own box's parameters.
inline bool cooperative_variant(int v, bool general, bool half) {
  if (general) return half;  // the half stencil's general kernel drains spread
  return (v >= 7 && v <= 9) || (half && v >= 10 && v <= 12);
}
size_t tile_smem_bytes(int stage_cap);
// fuse: full stencil only; the kernel also performs the next step's row a1
// (integrate_one) for every slot and stores no force.
cudaError_t launch_force(const Packed &P, const StepConfig &cfg, cudaStream_t s,
                         bool fuse = false);

// Direct force-kernel variants (threads per block, pair-list capacity).
int force_variant_info(int v, int *threads, int *cap);
// Process-wide tuning table: density band -> variant, per stencil.
int tuning_set(int table, int n, const double *upper, const int *variant);
int tuning_get(int table, int max, double *upper, int *variant);
int tuned_band(int table, double rho);
int tuned_variant(int table, double rho);

#ifdef __CUDACC__
// Full periodic fold for a coordinate that left [0, L) by more than one edge.
__device__ __forceinline__ float refold(float x, float L) {
  if (x >= 0.0f && x < L) return x;
  x = x - L * floorf(x / L);
  return (x >= 0.0f && x < L) ? x : 0.0f;
}

// Cell entries of particles that keep their slot through the reorder
// (bit 31 of cellOf): the particles of a stopped box, which did not move,
// so that their slots, and with them the forces held there, stay as they
// are (the half stencil's reorder otherwise clears the forces).
constexpr int kKeepSlot = (int)0x80000000u;

// Row a1 for the particle in slot p (Sec. 3.1 item 5, Eq. 1; Sec. 3.2): if
// `move`, the second half kick of the previous step (when `pending`), this
// step's first half kick with the force (fx, fy, fz), the drift and the
// periodic wrap; then the cell of the position, its arrival rank by an
// atomic count, and the copies the reorder reads.  `keep`: the particle's
// box is stopped and the particle keeps its slot.  The integrate kernel and
// the full stencil's fused force epilogue both call it, so they give the
// same bits.
template <typename BX>
__device__ __forceinline__ void integrate_one(const Packed &P, const BX &B, int p, float4 x,
                                              float4 v, float fx, float fy, float fz, bool move,
                                              bool pending, bool keep = false) {
  if (move) {
    const float h = B.hdt_m;
    if (pending) {  // second half kick of the previous step
      v.x = fmaf(h, fx, v.x);
      v.y = fmaf(h, fy, v.y);
      v.z = fmaf(h, fz, v.z);
    }
    v.x = fmaf(h, fx, v.x);  // first half kick of this step
    v.y = fmaf(h, fy, v.y);
    v.z = fmaf(h, fz, v.z);
    x.x = wrap_coord(fmaf(B.dt, v.x, x.x), B.L[0]);
    x.y = wrap_coord(fmaf(B.dt, v.y, x.y), B.L[1]);
    x.z = wrap_coord(fmaf(B.dt, v.z, x.z), B.L[2]);
    const bool finite = isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(v.x) &&
                        isfinite(v.y) && isfinite(v.z);
    if (!finite) {
      atomicOr(P.err, kErrNonFinite);
      x.x = isfinite(x.x) ? x.x : 0.0f;
      x.y = isfinite(x.y) ? x.y : 0.0f;
      x.z = isfinite(x.z) ? x.z : 0.0f;
    }
    if (!(x.x >= 0.0f && x.x < B.L[0] && x.y >= 0.0f && x.y < B.L[1] && x.z >= 0.0f &&
          x.z < B.L[2])) {
      atomicOr(P.err, kErrRunaway);  // moved more than one edge in a step
      x.x = refold(x.x, B.L[0]);
      x.y = refold(x.y, B.L[1]);
      x.z = refold(x.z, B.L[2]);
    }
  }
  const int cx = cell_axis(x.x, B.invh[0], B.n[0]);
  const int cy = cell_axis(x.y, B.invh[1], B.n[1]);
  const int cz = cell_axis(x.z, B.invh[2], B.n[2]);
  const int c = B.cellBase + (cz * B.n[1] + cy) * B.n[0] + cx;
  v.w = __int_as_float(pack_cell(cx, cy, cz));
  P.pos2[p] = x;
  P.vel2[p] = v;
  if (!DPD_IN_BOUNDS(c >= 0 && c < P.ncell, P.err)) return;
  P.cellOf[p] = keep ? (c | kKeepSlot) : c;
  P.slotIn[p] = atomicAdd(P.count + c, 1);
}

// Box constants: the kernel parameter copy for a single box, else from memory.
template <bool SINGLE>
__device__ __forceinline__ BoxDev box_of(const Packed &P, int b) {
  if constexpr (SINGLE) {
    return P.single;
  } else {
    return P.boxes[b];
  }
}
#endif

struct StatsWork {  // one block of the statistics reduction
  int box, begin, end, pad;
};
constexpr int kStatsFields = 6;  // sum v (3), sum v^2, sum frc.w, count

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;  // cells per scan tile
constexpr int kScanMaxTiles = 1024 * 16;              // one block scans up to this many tile sums

inline int scan_tiles(int ncell) { return (ncell + 1 + kScanTile - 1) / kScanTile; }

// Set per-function launch attributes on the current device (once per device,
// before any capture).
cudaError_t prepare_device();

// Convert n x 3 inputs of one box into float4 slots (ids 0..n-1, wrapped).
// species: n species 0..nspec-1 (device memory), or null for all 0.
cudaError_t launch_load(const Packed &P, int box_slot0, int n, const float *pos3, const float *vel3,
                        float Lx, float Ly, float Lz, cudaStream_t s,
                        const int32_t *species = nullptr, int nspec = 1);

// One step (move = true) or the initial rebuild (move = false):
// kick/drift/wrap + cell count, scan, reorder, force.  fused_in: the previous
// step's force kernel already did this step's kick/drift/wrap + count, so the
// step starts at the scan; fuse_out: this step's force kernel does the next
// step's (full stencil).
cudaError_t launch_step(const Packed &P, bool move, bool advance, const StepConfig &cfg,
                        cudaStream_t s, bool fused_in = false, bool fuse_out = false);

// One step with events recorded around its stages: ev[0] before the
// integrate/count kernel, then after it, after the scan, after the key pass,
// after the reorder and after the force kernel (6 events).
cudaError_t launch_step_timed(const Packed &P, const StepConfig &cfg, cudaStream_t s,
                              cudaEvent_t *ev);
constexpr int kNumStages = 5;
constexpr int kKernelsPerStep = 7;

// Per-work-item FP64 partial sums for box statistics.
// With box_out: also the per-box totals (nbox x kStatsFields, a fixed order per box).
cudaError_t launch_stats(const Packed &P, const StatsWork *work, int nwork, double *out,
                         cudaStream_t s, const int *wbeg = nullptr, int nbox = 0,
                         double *box_out = nullptr);

// Write slots [slot0, slot0 + n) to id order as n x 3 arrays (any may be null);
// velocities are full-step (pending half kick applied).
cudaError_t launch_gather(const Packed &P, int box, int slot0, int n, float *pos3, float *vel3,
                          float *frc3, cudaStream_t s);

// Served form: device-drawn initial state of a box (uniform positions,
// Maxwellian velocities with variance vscale^2, zero mean momentum).
cudaError_t launch_init_box(const Packed &P, int slot0, int n, float Lx, float Ly, float Lz,
                            float vscale, uint64_t seed, cudaStream_t s);
// Copy surviving boxes' particles into a new packing.
cudaError_t launch_repack(const float4 *opos, const float4 *ovel, float4 *npos, float4 *nvel,
                          const int *newbase, const int *src0, int nbox, int ntot, cudaStream_t s);
// Statistics sample (boxes whose step is a multiple of `every` past from[b]).
cudaError_t launch_sample(const Packed &P, const StatsWork *work, int nwork, const int *wbeg,
                          const long long *from, int every, int nbins, double *part, double *acc,
                          cudaStream_t s);

cudaError_t launch_debug_rng(const uint32_t *lo, const uint32_t *hi, long long n, uint64_t step,
                             uint64_t seed, int noise, uint32_t *out, uint32_t *out1, float *xi,
                             cudaStream_t s);

}  // namespace dpd
