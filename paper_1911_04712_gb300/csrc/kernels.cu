// CUDA kernels of the DPD fluid step for sm_103a.
//
// One step, every stage a kernel over the packed particle slots (the force
// kernels are in force.cu):
//   1. integrate_bin  kick (completing the previous step), kick, drift, wrap
//                     (Sec. 3.1 item 5, Eq. 1); cell (x slice) of the new
//                     position and its arrival rank by an atomic count
//                     (Sec. 3.2); with the full stencil the previous step's
//                     force kernel can do this instead (fused);
//   2. scan           exclusive scan of the cell counts into cell starts
//                     (three passes: tile sums, scan of the tile sums, apply);
//   3. bin_keys       full stencil: record each slot's old index at its
//                     arrival position;
//   4. bin_scatter    move position and velocity to the new slot: full
//                     stencil ranked by old index inside the cell (a stable
//                     counting sort), half stencil by arrival rank;
//   5. force          pair forces of Eqs. 2-5 over the 27 neighbouring cells
//                     (full stencil) or 13 cells + own cell with Newton's third
//                     law (half stencil, Sec. 3.2), plus the body force.
// All arithmetic is FP32; statistics sum in FP64 above each thread.
#include <cuda_runtime.h>

#include <cstdint>

#include "dpd_device.cuh"
#include "kernels.h"

namespace dpd {

constexpr int kBinThreads = 256;
static inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }
constexpr float kSqrt3Scale = (float)(1.7320508075688772 / 16777216.0);  // sqrt(3) 2^-24


// ------------------------------------------------------------------ load
__global__ void k_load(Packed P, int slot0, int n, const float *__restrict__ pos3,
                       const float *__restrict__ vel3, float Lx, float Ly, float Lz,
                       const int32_t *__restrict__ species, int nspec) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x[3] = {pos3[3 * i], pos3[3 * i + 1], pos3[3 * i + 2]};
  const float L[3] = {Lx, Ly, Lz};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float y = x[k];
    if (!(y >= 0.0f && y < L[k])) {
      y = y - L[k] * floorf(y / L[k]);
      if (y >= L[k]) y = 0.0f;
      if (!(y >= 0.0f)) {  // NaN or still negative after rounding
        if (!(y == y)) atomicOr(P.err, kErrNonFinite);
        y = 0.0f;
      }
    }
    x[k] = y;
  }
  int s = species ? species[i] : 0;
  if (s < 0 || s >= nspec) {
    atomicOr(P.err, kErrSpecies);
    s = 0;
  }
  P.pos[slot0 + i] =
      make_float4(x[0], x[1], x[2], __uint_as_float((uint32_t)i | ((uint32_t)s << kSpeciesShift)));
  P.vel[slot0 + i] = make_float4(vel3[3 * i], vel3[3 * i + 1], vel3[3 * i + 2], 0.0f);
}

// ------------------------------------------------------- integrate + count
template <bool SINGLE>
__global__ void __launch_bounds__(kBinThreads) k_integrate_bin(Packed P, bool move) {
  const int p = blockIdx.x * kBinThreads + threadIdx.x;
  int b = 0;
  if constexpr (!SINGLE) b = find_box_warp(P.pbase, P.nbox, min(p, P.ntot - 1));
  if (p >= P.ntot) return;
  const BoxDev B = box_of<SINGLE>(P, b);
  const bool mv = move && P.st[b].remaining > 0;
  const float4 f = mv ? P.frc[p] : make_float4(0.f, 0.f, 0.f, 0.f);
  // a stopped box (a step with nothing left to take) keeps its slots and forces
  integrate_one(P, B, p, P.pos[p], P.vel[p], f.x, f.y, f.z, mv, P.st[b].pending != 0,
                move && !mv);
}

// ------------------------------------------------------------------ scan
__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive block scan of one value per thread; returns the block total in *total.
template <int NT>
__device__ __forceinline__ int block_excl_scan(int v, int *total) {
  __shared__ int wsum[NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int incl = warp_incl_scan(v);
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int s = (lane < NT / 32) ? wsum[lane] : 0;
    s = warp_incl_scan(s);
    if (lane < NT / 32) wsum[lane] = s;
  }
  __syncthreads();
  const int before = (warp > 0) ? wsum[warp - 1] : 0;
  *total = wsum[NT / 32 - 1];
  __syncthreads();
  return before + incl - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int *__restrict__ count,
                                                              int *__restrict__ bsum) {
  const int4 *c4 = reinterpret_cast<const int4 *>(count) +
                   (size_t)blockIdx.x * (kScanTile / 4) + threadIdx.x * (kScanItems / 4);
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems / 4; ++k) {
    const int4 q = c4[k];
    s += q.x + q.y + q.z + q.w;
  }
  int total;
  block_excl_scan<kScanThreads>(s, &total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// Exclusive scan of the tile sums in place (one block).
__global__ void __launch_bounds__(1024) k_scan_bsum(int *__restrict__ bsum, int ntile) {
  const int per = (ntile + 1023) / 1024;
  const int b0 = threadIdx.x * per;
  int s = 0;
  for (int k = 0; k < per; ++k)
    if (b0 + k < ntile) s += bsum[b0 + k];
  int total;
  int run = block_excl_scan<1024>(s, &total);
  for (int k = 0; k < per; ++k)
    if (b0 + k < ntile) {
      const int v = bsum[b0 + k];
      bsum[b0 + k] = run;
      run += v;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(Packed P, bool advance) {
  int4 *c4 = reinterpret_cast<int4 *>(P.count) + (size_t)blockIdx.x * (kScanTile / 4) +
             threadIdx.x * (kScanItems / 4);
  int4 *s4 = reinterpret_cast<int4 *>(P.start) + (size_t)blockIdx.x * (kScanTile / 4) +
             threadIdx.x * (kScanItems / 4);
  int v[kScanItems];
#pragma unroll
  for (int k = 0; k < kScanItems / 4; ++k) {
    const int4 q = c4[k];
    v[4 * k] = q.x;
    v[4 * k + 1] = q.y;
    v[4 * k + 2] = q.z;
    v[4 * k + 3] = q.w;
    c4[k] = make_int4(0, 0, 0, 0);  // counts start from zero at the next rebuild
  }
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) s += v[k];
  int total;
  int run = block_excl_scan<kScanThreads>(s, &total) + P.bsum[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems / 4; ++k) {
    int4 o;
    o.x = run;
    run += v[4 * k];
    o.y = run;
    run += v[4 * k + 1];
    o.z = run;
    run += v[4 * k + 2];
    o.w = run;
    run += v[4 * k + 3];
    s4[k] = o;
  }
  if (advance && blockIdx.x == 0) {
    for (int b = threadIdx.x; b < P.nbox; b += kScanThreads) {
      BoxState st = P.st[b];
      if (st.remaining > 0) {
        st.step += 1;
        st.remaining -= 1;
        st.pending = 1;
        st.adv = 1;
      } else {
        st.adv = 0;
      }
      P.st[b] = st;
    }
  }
}

// ---------------------------------------------------------------- reorder
__global__ void __launch_bounds__(kBinThreads) k_bin_keys(Packed P) {
  const int p = blockIdx.x * kBinThreads + threadIdx.x;
  if (p >= P.ntot) return;
  const int c = P.cellOf[p];
  if (c < 0) return;  // keeps its slot (stopped box): every particle of its cell does
  if (!DPD_IN_BOUNDS(c >= 0 && c < P.ncell, P.err)) return;
  const int k = P.start[c] + P.slotIn[p];
  if (!DPD_IN_BOUNDS(k >= 0 && k < P.ntot, P.err)) return;
  P.keyTmp[k] = p;
}

// STABLE: a particle's place in its cell is its rank by previous slot among
// the cell's particles (listed by k_bin_keys), so the order, and with it the
// full stencil's sums, are reproducible.  Otherwise (half stencil, whose sums
// are atomic anyway) it is its arrival rank from the count, as in Sec. 3.2.
// A particle of a stopped box keeps its slot, and its force (which the half
// stencil's reorder otherwise clears for the atomic sums): it did not move,
// so its cell's slot range is the one it was placed in.
template <bool STABLE>
__global__ void __launch_bounds__(kBinThreads) k_bin_scatter(Packed P, bool zero_frc) {
  const int p = blockIdx.x * kBinThreads + threadIdx.x;
  if (p >= P.ntot) return;
  const int ce = P.cellOf[p];
  const bool keep = ce < 0;
  const int c = ce & ~kKeepSlot;
  if (!DPD_IN_BOUNDS(c >= 0 && c < P.ncell, P.err)) return;
  const int s0 = P.start[c];
  int dst = p;
  if (!keep) {
    int rank = P.slotIn[p];
    if constexpr (STABLE) {
      const int s1 = P.start[c + 1];
      if (!DPD_IN_BOUNDS(s0 >= 0 && s0 <= s1 && s1 <= P.ntot, P.err)) return;
      rank = 0;
      for (int t = s0; t < s1; ++t) rank += (P.keyTmp[t] < p) ? 1 : 0;
    }
    dst = s0 + rank;
  }
  if (!DPD_IN_BOUNDS(dst >= s0 && dst < P.start[c + 1] && dst < P.ntot, P.err)) return;
  P.pos[dst] = P.pos2[p];
  P.vel[dst] = P.vel2[p];
  if (zero_frc && !keep) P.frc[dst] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ------------------------------------------------------------------ stats
constexpr int kStatsThreads = 256;

// Sum of two unevaluated pairs hi + lo of FP32 numbers, as such a pair: the
// high parts are added error-free (TwoSum), the low parts and that error go
// into the new low part, then the pair is renormalised (Dekker's Fast2Sum).
// The result carries about 2^-44 of the operands' magnitude as error.
__device__ __forceinline__ void pair_add(float &hi, float &lo, float bh, float bl) {
  const float s = hi + bh;
  const float bv = s - hi;
  float e = (hi - (s - bv)) + (bh - bv);
  e += lo + bl;
  hi = s + e;
  lo = e - (hi - s);
}

__global__ void __launch_bounds__(kStatsThreads) k_stats(Packed P, const StatsWork *__restrict__ work,
                                                         double *__restrict__ out) {
  const StatsWork w = work[blockIdx.x];
  const BoxDev &B = P.boxes[w.box];
  const BoxState S = P.st[w.box];
  const float h = S.pending ? B.hdt_m : 0.0f;
  // Each thread sums its particles' FP32 values as unevaluated pairs
  // hi + lo of FP32 numbers (the error-free TwoSum transformation: each
  // addition's rounding error is carried in lo).  The warp and the block
  // combine those pairs as pairs, and only the block's total is converted
  // to FP64: every FP64 operation per particle or per lane is avoided,
  // since FP64 runs at a small fraction of the FP32 rate on this part.
  // Everything above the block (work items, boxes) is summed in FP64.
  constexpr int F = kStatsFields - 1;
  float hi[F] = {0.f, 0.f, 0.f, 0.f, 0.f};
  float lo[F] = {0.f, 0.f, 0.f, 0.f, 0.f};
  auto two_sum = [&](int k, float x) {
    const float t = hi[k] + x;
    const float xv = t - hi[k];
    lo[k] += (hi[k] - (t - xv)) + (x - xv);
    hi[k] = t;
  };
#pragma unroll 4
  for (int p = w.begin + threadIdx.x; p < w.end; p += kStatsThreads) {
    float4 v = P.vel[p];
    const float4 f = P.frc[p];
    v.x = fmaf(h, f.x, v.x);
    v.y = fmaf(h, f.y, v.y);
    v.z = fmaf(h, f.z, v.z);
    two_sum(0, v.x);
    two_sum(1, v.y);
    two_sum(2, v.z);
    two_sum(3, fmaf(v.x, v.x, fmaf(v.y, v.y, v.z * v.z)));
    two_sum(4, f.w);
  }
#pragma unroll
  for (int k = 0; k < F; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      pair_add(hi[k], lo[k], __shfl_down_sync(0xffffffffu, hi[k], o),
               __shfl_down_sync(0xffffffffu, lo[k], o));
  constexpr int NW = kStatsThreads / 32;
  static_assert(NW <= 32 && (NW & (NW - 1)) == 0, "block of 1 to 32 warps, a power of two");
  __shared__ float2 red[F][NW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < F; ++k) red[k][warp] = make_float2(hi[k], lo[k]);
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < F; ++k) {
      float2 r = (lane < NW) ? red[k][lane] : make_float2(0.f, 0.f);
#pragma unroll
      for (int o = NW / 2; o > 0; o >>= 1)
        pair_add(r.x, r.y, __shfl_down_sync(0xffffffffu, r.x, o),
                 __shfl_down_sync(0xffffffffu, r.y, o));
      if (lane == 0) out[(size_t)blockIdx.x * kStatsFields + k] = (double)r.x + (double)r.y;
    }
    if (lane == 0) out[(size_t)blockIdx.x * kStatsFields + F] = (double)(w.end - w.begin);
  }
}

// ----------------------------------------------------------------- gather
__global__ void k_gather(Packed P, int box, int slot0, int n, float *__restrict__ pos3,
                         float *__restrict__ vel3, float *__restrict__ frc3) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int p = slot0 + k;
  const float4 x = P.pos[p];
  const int id = (int)(__float_as_uint(x.w) & kIdMask);
  if (id >= n) {
    atomicOr(P.err, kErrNonFinite);
    return;
  }
  const float4 f = P.frc[p];
  if (pos3) {
    pos3[3 * id] = x.x;
    pos3[3 * id + 1] = x.y;
    pos3[3 * id + 2] = x.z;
  }
  if (vel3) {
    const float h = P.st[box].pending ? P.boxes[box].hdt_m : 0.0f;
    const float4 v = P.vel[p];
    vel3[3 * id] = fmaf(h, f.x, v.x);
    vel3[3 * id + 1] = fmaf(h, f.y, v.y);
    vel3[3 * id + 2] = fmaf(h, f.z, v.z);
  }
  if (frc3) {
    frc3[3 * id] = f.x;
    frc3[3 * id + 1] = f.y;
    frc3[3 * id + 2] = f.z;
  }
}

// -------------------------------------------------------------- debug rng
__global__ void k_debug_rng(const uint32_t *__restrict__ lo, const uint32_t *__restrict__ hi,
                            long long n, uint32_t slo, uint32_t shi, uint32_t klo, uint32_t khi,
                            int noise, uint32_t *__restrict__ out, uint32_t *__restrict__ out1,
                            float *__restrict__ xi) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint2 u = pair_words(lo[k], hi[k], slo, shi, klo, khi);
  out[k] = u.x;
  if (out1) out1[k] = u.y;
  if (xi) xi[k] = noise ? gauss_xi(u.x, u.y) : __fmul_rn(noise_int(u.x), kSqrt3Scale);
}

// ------------------------------------------------------ served-form kernels
// Initial state of a new box drawn on the device from its seed: positions
// uniform in [0, L), velocities Maxwellian (Box-Muller) with variance kT/m.
// Philox-4x32-10 with key (seed lo, seed hi ^ 0x5EED0001) on counters
// (id, 0, 0, 0) and (id, 1, 0, 0); this only samples an initial condition.
__device__ __forceinline__ void philox4(uint32_t c0, uint32_t c1, uint32_t k0, uint32_t k1,
                                        uint32_t out[4]) {
  uint32_t c2 = 0u, c3 = 0u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    const uint32_t hi0 = __umulhi(kPhiloxM0, c0), lo0 = kPhiloxM0 * c0;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c2), lo1 = kPhiloxM1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

__device__ __forceinline__ float unit_open(uint32_t u) {  // (0, 1)
  return ((float)(u >> 8) + 0.5f) * (1.0f / 16777216.0f);
}

__global__ void k_init_box(Packed P, int slot0, int n, float Lx, float Ly, float Lz, float vscale,
                           uint32_t seed_lo, uint32_t seed_hi) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t a[4], b[4];
  philox4((uint32_t)i, 0u, seed_lo, seed_hi ^ 0x5EED0001u, a);
  philox4((uint32_t)i, 1u, seed_lo, seed_hi ^ 0x5EED0001u, b);
  float x = unit_open(a[0]) * Lx, y = unit_open(a[1]) * Ly, z = unit_open(a[2]) * Lz;
  x = x < Lx ? x : 0.f;
  y = y < Ly ? y : 0.f;
  z = z < Lz ? z : 0.f;
  const float r1 = sqrtf(-2.0f * logf(unit_open(b[0])));
  const float r2 = sqrtf(-2.0f * logf(unit_open(b[2])));
  float s1, c1, s2, c2;
  sincospif(2.0f * unit_open(b[1]), &s1, &c1);
  sincospif(2.0f * unit_open(b[3]), &s2, &c2);
  P.pos[slot0 + i] = make_float4(x, y, z, __int_as_float(i));
  P.vel[slot0 + i] = make_float4(vscale * r1 * c1, vscale * r1 * s1, vscale * r2 * c2, 0.f);
}

// Remove the mean velocity of one box: one block sums in a fixed order (FP64),
// then every thread subtracts.
__global__ void __launch_bounds__(1024) k_zero_momentum(Packed P, int slot0, int n) {
  __shared__ double red[3][32];
  __shared__ float mean[3];
  double s[3] = {0, 0, 0};
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float4 v = P.vel[slot0 + i];
    s[0] += v.x;
    s[1] += v.y;
    s[2] += v.z;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double t = s[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) red[k][warp] = t;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[threadIdx.x][w];
    mean[threadIdx.x] = (float)(n > 0 ? t / n : 0.0);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float4 v = P.vel[slot0 + i];
    v.x -= mean[0];
    v.y -= mean[1];
    v.z -= mean[2];
    P.vel[slot0 + i] = v;
  }
}

// Move surviving boxes to their new slot ranges: new slot q of new box b
// takes old slot src0[b] + (q - newbase[b]) (src0 < 0: a new box, skipped).
__global__ void k_repack(const float4 *__restrict__ opos, const float4 *__restrict__ ovel,
                         float4 *__restrict__ npos, float4 *__restrict__ nvel,
                         const int *__restrict__ newbase, const int *__restrict__ src0, int nbox,
                         int ntot) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ntot) return;
  const int b = find_box(newbase, nbox, q);
  const int s0 = src0[b];
  if (s0 < 0) return;
  const int src = s0 + (q - newbase[b]);
  npos[q] = opos[src];
  nvel[q] = ovel[src];
}

// Statistics sample of every box whose step is a multiple of `every` and
// past its window start: per work item FP64 partials of sum v^2, sum r.F^C
// (frc.w, each pair counted twice) and per-slab sums of the flow-axis
// velocity with their counts.
__global__ void __launch_bounds__(256) k_sample(Packed P, const StatsWork *__restrict__ work,
                                                const long long *__restrict__ from, int every,
                                                int nbins, double *__restrict__ part) {
  extern __shared__ double sbin[];  // 2 * nbins: sums then counts
  const StatsWork w = work[blockIdx.x];
  const BoxState S = P.st[w.box];
  const int fields = 3 + 2 * nbins;
  double *out = part + (size_t)blockIdx.x * fields;
  const bool take = S.adv && every > 0 && (long long)S.step > from[w.box] &&
                    (S.step % (unsigned long long)every) == 0ull;
  if (!take) {
    if (threadIdx.x == 0) out[0] = 0.0;  // marks "no sample"
    return;
  }
  for (int k = threadIdx.x; k < 2 * nbins; k += blockDim.x) sbin[k] = 0.0;
  __syncthreads();
  const BoxDev B = P.boxes[w.box];
  const float h = S.pending ? B.hdt_m : 0.0f;
  const float Lg = B.L[B.fb_grad];
  double v2 = 0.0, vir = 0.0;
  for (int p = w.begin + threadIdx.x; p < w.end; p += blockDim.x) {
    const float4 x = P.pos[p];
    float4 v = P.vel[p];
    const float4 f = P.frc[p];
    v.x = fmaf(h, f.x, v.x);
    v.y = fmaf(h, f.y, v.y);
    v.z = fmaf(h, f.z, v.z);
    v2 += (double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z;
    vir += (double)f.w;
    if (nbins > 0) {
      const float xg = (B.fb_grad == 0) ? x.x : (B.fb_grad == 1) ? x.y : x.z;
      const float vf = (B.fb_flow == 0) ? v.x : (B.fb_flow == 1) ? v.y : v.z;
      int bin = (int)(xg / Lg * nbins);
      bin = min(max(bin, 0), nbins - 1);
      atomicAdd(&sbin[bin], (double)vf);
      atomicAdd(&sbin[nbins + bin], 1.0);
    }
  }
  __shared__ double red[2][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v2 += __shfl_down_sync(0xffffffffu, v2, o);
    vir += __shfl_down_sync(0xffffffffu, vir, o);
  }
  if (lane == 0) {
    red[0][warp] = v2;
    red[1][warp] = vir;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int q = 0; q < (int)(blockDim.x / 32); ++q) {
      a += red[0][q];
      c += red[1][q];
    }
    out[0] = 1.0;
    out[1] = a;
    out[2] = c;
  }
  for (int k = threadIdx.x; k < 2 * nbins; k += blockDim.x) out[3 + k] = sbin[k];
}

// Add each box's work-item partials (in work order) to its accumulators:
// acc[b] = {samples, sum v^2, sum frc.w, slab sums[nbins], slab counts[nbins]}.
__global__ void k_sample_acc(const StatsWork *__restrict__ work, const int *__restrict__ wbeg,
                             int nbox, int nbins, const double *__restrict__ part,
                             double *__restrict__ acc) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  const int fields = 3 + 2 * nbins;
  const int w0 = wbeg[b], w1 = wbeg[b + 1];
  if (w1 <= w0 || part[(size_t)w0 * fields] == 0.0) return;
  double *a = acc + (size_t)b * fields;
  a[0] += 1.0;
  for (int k = 1; k < fields; ++k) {
    double s = 0.0;
    for (int w = w0; w < w1; ++w) s += part[(size_t)w * fields + k];
    a[k] += s;
  }
}

// ================================================================ launchers

cudaError_t launch_load(const Packed &P, int slot0, int n, const float *pos3, const float *vel3,
                        float Lx, float Ly, float Lz, cudaStream_t s, const int32_t *species,
                        int nspec) {
  if (n <= 0) return cudaSuccess;
  k_load<<<blocks_for(n, 256), 256, 0, s>>>(P, slot0, n, pos3, vel3, Lx, Ly, Lz, species, nspec);
  return cudaGetLastError();
}

cudaError_t launch_step(const Packed &P, bool move, bool advance, const StepConfig &cfg,
                        cudaStream_t s, bool fused_in, bool fuse_out) {
  if (P.ntot <= 0) return cudaSuccess;
  const bool single = (P.nbox == 1);
  const int gb = blocks_for(P.ntot, kBinThreads);
  if (fused_in) {
    // row a1 of this step ran in the previous step's force kernel
  } else if (single) {
    k_integrate_bin<true><<<gb, kBinThreads, 0, s>>>(P, move);
  } else {
    k_integrate_bin<false><<<gb, kBinThreads, 0, s>>>(P, move);
  }
  const int nt = scan_tiles(P.ncell);
  k_scan_reduce<<<nt, kScanThreads, 0, s>>>(P.count, P.bsum);
  k_scan_bsum<<<1, 1024, 0, s>>>(P.bsum, nt);
  k_scan_apply<<<nt, kScanThreads, 0, s>>>(P, advance);
  if (cfg.stencil == 1) {
    k_bin_scatter<false><<<gb, kBinThreads, 0, s>>>(P, true);
  } else {
    k_bin_keys<<<gb, kBinThreads, 0, s>>>(P);
    k_bin_scatter<true><<<gb, kBinThreads, 0, s>>>(P, false);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_force(P, cfg, s, fuse_out && cfg.stencil == 0);
}

cudaError_t launch_step_timed(const Packed &P, const StepConfig &cfg, cudaStream_t s,
                              cudaEvent_t *ev) {
  if (P.ntot <= 0) return cudaSuccess;
  const bool single = (P.nbox == 1);
  const int gb = blocks_for(P.ntot, kBinThreads);
  cudaError_t e;
  if ((e = cudaEventRecord(ev[0], s)) != cudaSuccess) return e;
  if (single)
    k_integrate_bin<true><<<gb, kBinThreads, 0, s>>>(P, true);
  else
    k_integrate_bin<false><<<gb, kBinThreads, 0, s>>>(P, true);
  if ((e = cudaEventRecord(ev[1], s)) != cudaSuccess) return e;
  const int nt = scan_tiles(P.ncell);
  k_scan_reduce<<<nt, kScanThreads, 0, s>>>(P.count, P.bsum);
  k_scan_bsum<<<1, 1024, 0, s>>>(P.bsum, nt);
  k_scan_apply<<<nt, kScanThreads, 0, s>>>(P, true);
  if ((e = cudaEventRecord(ev[2], s)) != cudaSuccess) return e;
  if (cfg.stencil != 1) k_bin_keys<<<gb, kBinThreads, 0, s>>>(P);
  if ((e = cudaEventRecord(ev[3], s)) != cudaSuccess) return e;
  if (cfg.stencil == 1)
    k_bin_scatter<false><<<gb, kBinThreads, 0, s>>>(P, true);
  else
    k_bin_scatter<true><<<gb, kBinThreads, 0, s>>>(P, false);
  if ((e = cudaEventRecord(ev[4], s)) != cudaSuccess) return e;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_force(P, cfg, s)) != cudaSuccess) return e;
  return cudaEventRecord(ev[5], s);
}

// Per-box totals of the work items' partial sums (work items of a box are
// contiguous, wbeg[b] .. wbeg[b + 1]): one block per box, each thread a
// strided sum, then a tree in a fixed order, so a box's totals do not
// depend on the other boxes packed with it.
constexpr int kBoxSumThreads = 512;
__global__ void __launch_bounds__(kBoxSumThreads)
    k_stats_boxes(const double *__restrict__ part, const int *__restrict__ wbeg,
                  double *__restrict__ out) {
  __shared__ double red[kStatsFields][kBoxSumThreads];
  const int b = blockIdx.x, t = threadIdx.x;
  double acc[kStatsFields] = {0, 0, 0, 0, 0, 0};
#pragma unroll 4
  for (int w = wbeg[b] + t; w < wbeg[b + 1]; w += kBoxSumThreads)
#pragma unroll
    for (int k = 0; k < kStatsFields; ++k) acc[k] += part[(size_t)w * kStatsFields + k];
#pragma unroll
  for (int k = 0; k < kStatsFields; ++k) red[k][t] = acc[k];
  __syncthreads();
  for (int h = kBoxSumThreads / 2; h > 0; h >>= 1) {
    if (t < h)
#pragma unroll
      for (int k = 0; k < kStatsFields; ++k) red[k][t] += red[k][t + h];
    __syncthreads();
  }
  if (t < kStatsFields) out[(size_t)b * kStatsFields + t] = red[t][0];
}

cudaError_t launch_stats(const Packed &P, const StatsWork *work, int nwork, double *out,
                         cudaStream_t s, const int *wbeg, int nbox, double *box_out) {
  if (nwork <= 0) return cudaSuccess;
  k_stats<<<nwork, kStatsThreads, 0, s>>>(P, work, out);
  if (box_out && nbox > 0) k_stats_boxes<<<nbox, kBoxSumThreads, 0, s>>>(out, wbeg, box_out);
  return cudaGetLastError();
}

cudaError_t launch_gather(const Packed &P, int box, int slot0, int n, float *pos3, float *vel3,
                          float *frc3, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_gather<<<blocks_for(n, 256), 256, 0, s>>>(P, box, slot0, n, pos3, vel3, frc3);
  return cudaGetLastError();
}

cudaError_t launch_debug_rng(const uint32_t *lo, const uint32_t *hi, long long n, uint64_t step,
                             uint64_t seed, int noise, uint32_t *out, uint32_t *out1, float *xi,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_debug_rng<<<blocks_for(n, 256), 256, 0, s>>>(lo, hi, n, (uint32_t)step,
                                                 (uint32_t)(step >> 32), (uint32_t)seed,
                                                 (uint32_t)(seed >> 32), noise, out, out1, xi);
  return cudaGetLastError();
}

}  // namespace dpd

namespace dpd {

cudaError_t launch_init_box(const Packed &P, int slot0, int n, float Lx, float Ly, float Lz,
                            float vscale, uint64_t seed, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_init_box<<<blocks_for(n, 256), 256, 0, s>>>(P, slot0, n, Lx, Ly, Lz, vscale, (uint32_t)seed,
                                                 (uint32_t)(seed >> 32));
  k_zero_momentum<<<1, 1024, 0, s>>>(P, slot0, n);
  return cudaGetLastError();
}

cudaError_t launch_repack(const float4 *opos, const float4 *ovel, float4 *npos, float4 *nvel,
                          const int *newbase, const int *src0, int nbox, int ntot,
                          cudaStream_t s) {
  if (ntot <= 0) return cudaSuccess;
  k_repack<<<blocks_for(ntot, 256), 256, 0, s>>>(opos, ovel, npos, nvel, newbase, src0, nbox,
                                                  ntot);
  return cudaGetLastError();
}

cudaError_t launch_sample(const Packed &P, const StatsWork *work, int nwork, const int *wbeg,
                          const long long *from, int every, int nbins, double *part, double *acc,
                          cudaStream_t s) {
  if (nwork <= 0 || every <= 0) return cudaSuccess;
  k_sample<<<nwork, 256, 2 * nbins * sizeof(double), s>>>(P, work, from, every, nbins, part);
  k_sample_acc<<<blocks_for(P.nbox, 128), 128, 0, s>>>(work, wbeg, P.nbox, nbins, part, acc);
  return cudaGetLastError();
}

}  // namespace dpd
