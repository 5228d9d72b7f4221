// Device-side definitions of the DPD fluid step: per-box descriptors, the
// pair-noise generator and small geometry helpers.
//
// Data layout in HBM (one packed set of boxes; a single box is the case
// nbox = 1):
//   pos[p]  float4 (x, y, z, id)     id = box-local particle id as int bits
//   vel[p]  float4 (vx, vy, vz, cell) cell = packed local cell coordinates
//   frc[p]  float4 (fx, fy, fz, vir)  vir = sum over this particle's pairs of
//                                     r . F^C (both members count the pair)
// Particles of box b occupy slots [pbase[b], pbase[b+1]) and, after every
// rebuild, appear in cell order (cell = cellBase[b] + (cz*ny + cy)*nx + cx).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dpd {

// Pair noise: Philox-4x32-R (Salmon, Moraes, Dror, Shaw, SC'11).
#ifndef DPD_PHILOX_ROUNDS
#define DPD_PHILOX_ROUNDS 10
#endif
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;  // round multipliers
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;  // Weyl key increments
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// A particle's id and species share pos.w: id in the low 30 bits (the pair
// noise uses the id alone), species 0..3 in the top two.
constexpr int kSpeciesShift = 30;
constexpr uint32_t kIdMask = (1u << kSpeciesShift) - 1u;
constexpr int kMaxSpecies = 4;
// Cells: floor(L_d / rc) per axis, each cut into kSlicesX slices along x
// (the cell list's x resolution: a row is scanned only over the slices
// within rc of the particle's x).
constexpr int kSlicesX = 2;
constexpr int kCellBits = 10;                 // packed cell coords: 10 bits for y and z,
constexpr int kSliceBits = 12;                // 12 for the x slice
constexpr int kMaxCellsPerAxis = (1 << kCellBits) - 1;
static_assert(kSlicesX >= 2 && kSlicesX * kMaxCellsPerAxis < (1 << kSliceBits),
              "an x window must not cover a slice twice; slices must fit the packed field");

// Error bits raised by kernels into the context's device error word.
constexpr unsigned kErrNonFinite = 1u;        // a position or velocity is NaN/Inf
constexpr unsigned kErrRunaway = 2u;          // a particle moved more than one box edge
constexpr unsigned kErrSpecies = 4u;          // a loaded species outside 0..nspec-1
constexpr unsigned kErrBounds = 8u;           // checked build: an index check failed
constexpr unsigned kErrCapacity = 16u;        // brick force kernel: one cell row's stencil
                                              // holds more particles than its staging

// Checked build (-DDPD_CHECKED=1, libdpd_checked.so): the kernels test the
// indices they derive from device data (cell indices, cell starts, list
// entries, scatter targets) before using them; a failed test records
// kErrBounds in the error word and the access is skipped, so nothing faults.
// In the normal build DPD_IN_BOUNDS is the constant true and the tests
// compile away.
#if defined(DPD_CHECKED) && DPD_CHECKED
#define DPD_IN_BOUNDS(cond, err) ((cond) || (atomicOr((err), ::dpd::kErrBounds), false))
#else
#define DPD_IN_BOUNDS(cond, err) true
#endif

// Constants of one periodic box (read-only during a step).
struct BoxDev {
  float L[3];       // box edges
  float invh[3];    // cells (x: slices) per unit length, n_d / L_d
  int n[3];         // x: slices, kSlicesX floor(L_x / rc); y, z: cells, floor(L_d / rc) >= 3
  float xwin;       // half-width of the x window: rc plus a margin of several ulp of L
  int cellBase;     // first packed cell index of this box
  int pbase;        // first particle slot of this box
  int np;           // particles in this box
  float a;          // conservative coefficient (Eq. 3)
  float gamma;      // dissipative coefficient (Eq. 5)
  float sig;        // sigma * sqrt(3) * 2^-24 / sqrt(dt): multiplies the integer noise
  float rc2;        // rc^2
  float inv_rc;     // 1 / rc
  float kexp;       // weight exponent k, w_R = w^k
  float hdt_m;      // dt / (2 m)
  float dt;         // time step
  float fb;         // body-force magnitude
  int fb_mode;      // 0 none, 1 constant, 2 periodic Poiseuille (Sec. 4.2)
  int fb_flow;      // axis of the body force
  int fb_grad;      // axis on which the Poiseuille force switches sign
  float fb_half;    // L[fb_grad] / 2
  uint32_t seed_lo; // noise key
  uint32_t seed_hi;
  int noise;        // 0: uniform xi of unit variance, 1: Gaussian xi (Box-Muller)
  float sig_g;      // sigma / sqrt(dt): multiplies a Gaussian xi
  // Several species (nspec 2..4; 1 uses the scalars above): the interaction
  // of species s with t at [kMaxSpecies s + t].  rc_st <= rc, the cells' cut-off.
  int nspec;
  float sp_a[kMaxSpecies * kMaxSpecies];
  float sp_gamma[kMaxSpecies * kMaxSpecies];
  float sp_sig[kMaxSpecies * kMaxSpecies];    // as sig, from gamma_st
  float sp_sig_g[kMaxSpecies * kMaxSpecies];  // as sig_g, from gamma_st
  float sp_rc2[kMaxSpecies * kMaxSpecies];
  float sp_inv_rc[kMaxSpecies * kMaxSpecies];
};

// Mutable per-box step state (device resident so that graphs can replay it).
struct BoxState {
  unsigned long long step;  // noise step index of the force held in frc
  long long remaining;      // steps still to take; 0 freezes the box
  int pending;              // 1: vel holds v(n - 1/2); the full-step velocity is vel + hdt_m f
  int adv;                  // 1: the box is being advanced / needs its force this step
};

// ---------------------------------------------------------------- noise
// Word 0 of Philox-4x32-R on counter (c0, c1, c2, c3) and key (k0, k1).
__device__ __forceinline__ uint32_t philox_word0(uint32_t c0, uint32_t c1, uint32_t c2,
                                                 uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < DPD_PHILOX_ROUNDS; ++r) {
    if (r > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    const uint64_t p0 = (uint64_t)kPhiloxM0 * c0;  // one wide multiply each
    const uint64_t p1 = (uint64_t)kPhiloxM1 * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c0 = n0;
    c1 = (uint32_t)p1;
    c2 = n2;
    c3 = (uint32_t)p0;
  }
  return c0;
}

// Words 0 and 1 of Philox-4x32-R (word 1 is the low half of the last
// round's second product).
__device__ __forceinline__ uint2 philox_word01(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < DPD_PHILOX_ROUNDS; ++r) {
    if (r > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    const uint64_t p0 = (uint64_t)kPhiloxM0 * c0;
    const uint64_t p1 = (uint64_t)kPhiloxM1 * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c0 = n0;
    c1 = (uint32_t)p1;
    c2 = n2;
    c3 = (uint32_t)p0;
  }
  return make_uint2(c0, c1);
}

// Signed odd integer t = 2 (u >> 8) + 1 - 2^24, exactly representable in FP32;
// xi = sqrt(3) (2U - 1) = sqrt(3) t 2^-24 with U = ((u >> 8) + 1/2) 2^-24.
__device__ __forceinline__ float noise_int(uint32_t u) {
  const int t = (int)((u >> 8) * 2u + 1u) - (1 << 24);
  return __int2float_rn(t);
}

__device__ __forceinline__ uint32_t pair_word(uint32_t ida, uint32_t idb, uint32_t step_lo,
                                              uint32_t step_hi, uint32_t seed_lo,
                                              uint32_t seed_hi) {
  const uint32_t lo = min(ida, idb), hi = max(ida, idb);
  return philox_word0(lo, hi, step_lo, step_hi, seed_lo, seed_hi);
}

__device__ __forceinline__ uint2 pair_words(uint32_t ida, uint32_t idb, uint32_t step_lo,
                                            uint32_t step_hi, uint32_t seed_lo, uint32_t seed_hi) {
  const uint32_t lo = min(ida, idb), hi = max(ida, idb);
  return philox_word01(lo, hi, step_lo, step_hi, seed_lo, seed_hi);
}

// Gaussian xi from two words by the Box-Muller transform:
// sqrt(-2 ln U1) cos(2 pi U2), U_k = ((u_k >> 8) + 1/2) 2^-24.
__device__ __forceinline__ float gauss_xi(uint32_t u0, uint32_t u1) {
  const float U1 = fmaf((float)(u0 >> 8), 5.9604645e-08f, 2.9802322e-08f);
  const float U2 = fmaf((float)(u1 >> 8), 5.9604645e-08f, 2.9802322e-08f);
  return sqrtf(-2.0f * logf(U1)) * cospif(2.0f * U2);
}

// ---------------------------------------------------------------- geometry
// Fold a coordinate that moved by less than one edge back into [0, L).
__device__ __forceinline__ float wrap_coord(float x, float L) {
  if (x < 0.0f) {
    x += L;
  } else if (x >= L) {
    x -= L;
  }
  if (x >= L) x = 0.0f;  // a tiny negative x + L can round up to L
  return x;
}

__device__ __forceinline__ int cell_axis(float x, float invh, int n) {
  int c = __float2int_rz(__fmul_rn(x, invh));
  return min(max(c, 0), n - 1);
}

__device__ __forceinline__ int pack_cell(int cx, int cy, int cz) {
  return (int)((uint32_t)cx | ((uint32_t)cy << kSliceBits) |
               ((uint32_t)cz << (kSliceBits + kCellBits)));
}

__device__ __forceinline__ void unpack_cell(int c, int &cx, int &cy, int &cz) {
  const uint32_t u = (uint32_t)c;
  cx = (int)(u & ((1u << kSliceBits) - 1u));
  cy = (int)((u >> kSliceBits) & kMaxCellsPerAxis);
  cz = (int)((u >> (kSliceBits + kCellBits)) & kMaxCellsPerAxis);
}

// Largest b with pbase[b] <= p (pbase has nbox + 1 entries, non-decreasing).
__device__ __forceinline__ int find_box(const int *__restrict__ pbase, int nbox, int p) {
  int lo = 0, hi = nbox - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(pbase + mid) <= p)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// find_box for a warp of consecutive slots: one search for the warp's first
// slot, a per-lane search only for lanes past that box's end.  All lanes of
// the warp must call it.
__device__ __forceinline__ int find_box_warp(const int *__restrict__ pbase, int nbox, int p) {
  const int p0 = __shfl_sync(0xffffffffu, p, 0);
  int b0 = 0;
  if ((threadIdx.x & 31) == 0) b0 = find_box(pbase, nbox, p0);
  b0 = __shfl_sync(0xffffffffu, b0, 0);
  const int end0 = __ldg(pbase + b0 + 1);
  return (p >= p0 && p < end0) ? b0 : find_box(pbase, nbox, p);
}

}  // namespace dpd
