// CUDA kernels of the DPD fluid step for sm_103a.
//
// One step, every stage a kernel over the packed particle slots:
//   1. integrate_bin  kick (completing the previous step), kick, drift, wrap
//                     (Sec. 3.1 item 5, Eq. 1); cell of the new position and
//                     its arrival rank by an atomic count (Sec. 3.2);
//   2. scan           exclusive scan of the cell counts into cell starts
//                     (three passes: tile sums, scan of the tile sums, apply);
//   3. bin_keys       record each slot's old index at its arrival position;
//   4. bin_scatter    rank by old index inside the cell (a stable counting
//                     sort) and move position and velocity to the new slot;
//   5. force          pair forces of Eqs. 2-5 over the 27 neighbouring cells
//                     (full stencil) or 13 cells + own cell with Newton's third
//                     law (half stencil, Sec. 3.2), plus the body force.
// All arithmetic is FP32; statistics reduce in FP64.
#include <cuda_runtime.h>

#include <cstdint>

#include "dpd_device.cuh"
#include "kernels.h"

namespace dpd {

constexpr int kBinThreads = 256;
constexpr int kForceThreads = 128;  // must equal kTileThreads (shared list layout)
constexpr int kListCap = 24;   // pair-list entries per thread (shared memory)
constexpr int kFlushAt = 12;   // a warp drains its lists after a row once any lane exceeds this
constexpr float kSqrt3Scale = (float)(1.7320508075688772 / 16777216.0);  // sqrt(3) 2^-24

template <bool SINGLE>
__device__ __forceinline__ BoxDev box_of(const Packed &P, int b) {
  if constexpr (SINGLE) {
    return P.single;
  } else {
    return P.boxes[b];
  }
}

// ------------------------------------------------------------------ load
__global__ void k_load(Packed P, int slot0, int n, const float *__restrict__ pos3,
                       const float *__restrict__ vel3, float Lx, float Ly, float Lz) {
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
  P.pos[slot0 + i] = make_float4(x[0], x[1], x[2], __int_as_float(i));
  P.vel[slot0 + i] = make_float4(vel3[3 * i], vel3[3 * i + 1], vel3[3 * i + 2], 0.0f);
}

// ------------------------------------------------------- integrate + count
// Full periodic fold for a coordinate that left [0, L) by more than one edge.
__device__ __forceinline__ float refold(float x, float L) {
  if (x >= 0.0f && x < L) return x;
  x = x - L * floorf(x / L);
  return (x >= 0.0f && x < L) ? x : 0.0f;
}

template <bool SINGLE>
__global__ void __launch_bounds__(kBinThreads) k_integrate_bin(Packed P, bool move) {
  const int p = blockIdx.x * kBinThreads + threadIdx.x;
  if (p >= P.ntot) return;
  const int b = SINGLE ? 0 : find_box(P.pbase, P.nbox, p);
  const BoxDev B = box_of<SINGLE>(P, b);
  float4 x = P.pos[p];
  float4 v = P.vel[p];
  if (move && P.st[b].remaining > 0) {
    const float4 f = P.frc[p];
    const float h = B.hdt_m;
    if (P.st[b].pending) {  // second half kick of the previous step
      v.x = fmaf(h, f.x, v.x);
      v.y = fmaf(h, f.y, v.y);
      v.z = fmaf(h, f.z, v.z);
    }
    v.x = fmaf(h, f.x, v.x);  // first half kick of this step
    v.y = fmaf(h, f.y, v.y);
    v.z = fmaf(h, f.z, v.z);
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
  P.cellOf[p] = c;
  P.slotIn[p] = atomicAdd(P.count + c, 1);
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
  P.keyTmp[P.start[P.cellOf[p]] + P.slotIn[p]] = p;
}

__global__ void __launch_bounds__(kBinThreads) k_bin_scatter(Packed P, bool zero_frc) {
  const int p = blockIdx.x * kBinThreads + threadIdx.x;
  if (p >= P.ntot) return;
  const int c = P.cellOf[p];
  const int s0 = P.start[c], s1 = P.start[c + 1];
  int rank = 0;
  for (int t = s0; t < s1; ++t) rank += (P.keyTmp[t] < p) ? 1 : 0;
  const int dst = s0 + rank;
  P.pos[dst] = P.pos2[p];
  P.vel[dst] = P.vel2[p];
  if (zero_frc) P.frc[dst] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ------------------------------------------------------------------ force
// Pair lists: each thread appends the neighbours found inside rc to its own
// column of a shared-memory list (entry k of thread t at lst[k * kForceThreads + t]),
// then drains the list computing the pair forces.  An entry is 4 bytes: the
// neighbour slot j (26 bits) and the periodic-image code of the pair:
//   bit 26/28/30  the neighbour image is r_j - L on x/y/z (j near the top face)
//   bit 27/29/31  i is taken at r_i - L on x/y/z (i near the top face)
// Both subtractions are exact in FP32 (the shifted coordinate lies in
// [2L/3, L)), so no rounding error of size ulp(L) enters r_ij.
constexpr uint32_t kSlotMask = (1u << 26) - 1u;
constexpr uint32_t kCodeJX = 1u << 26, kCodeIX = 1u << 27, kCodeJY = 1u << 28,
                   kCodeIY = 1u << 29, kCodeJZ = 1u << 30, kCodeIZ = 1u << 31;

// Candidate pass over slots [j0, j1): appends every j with 0 < r_ij^2 < rc^2.
// The append is branch-free (the slot is written every iteration and kept only
// on a hit), so the lanes of a warp stay converged.  Returns the slot at which
// the list became full, or -1 when the range was scanned completely.
template <bool JSHIFT>
__device__ __forceinline__ int scan_range(const float4 *__restrict__ pos, int j0, int j1,
                                          float ax, float ay, float az, float jsx, float jsy,
                                          float jsz, float rc2, uint32_t code,
                                          uint32_t *__restrict__ lst, int &cnt) {
  for (int j = j0; j < j1; ++j) {
    const float4 pj = __ldg(pos + j);
    float dx, dy, dz;
    if constexpr (JSHIFT) {
      dx = ax - (pj.x - jsx);
      dy = ay - (pj.y - jsy);
      dz = az - (pj.z - jsz);
    } else {
      dx = ax - pj.x;
      dy = ay - pj.y;
      dz = az - pj.z;
    }
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const bool hit = (r2 < rc2) & (r2 > 0.0f);
    lst[cnt * kForceThreads] = (uint32_t)j | code;
    cnt += hit ? 1 : 0;
    if (cnt == kListCap) return j;
  }
  return -1;
}

// Force on one target particle in slot p from the 27-cell (full) or 13-cell
// + own-cell (half) neighbourhood, reading neighbours from global memory.
// Every lane of the warp must call this (dead lanes with alive = false) since
// list drains are decided warp-wide.
template <bool HALF>
__device__ __forceinline__ void force_direct(const Packed &P, const BoxDev &B, const BoxState &S,
                                             int p, bool alive, uint32_t *__restrict__ lst) {
  float4 pi = make_float4(0.f, 0.f, 0.f, 0.f), vi = pi;
  if (alive) {
    pi = P.pos[p];
    vi = P.vel[p];
  }
  int cx, cy, cz;
  unpack_cell(__float_as_int(vi.w), cx, cy, cz);
  const uint32_t idi = __float_as_uint(pi.w);
  const uint32_t slo = (uint32_t)S.step, shi = (uint32_t)(S.step >> 32);
  const float Lx = B.L[0], Ly = B.L[1], Lz = B.L[2];
  const int nx = B.n[0], ny = B.n[1], nz = B.n[2];

  float fx = 0.f, fy = 0.f, fz = 0.f, vir = 0.f;
  int cnt = 0;

  auto drain = [&]() {
    for (int k = 0; k < cnt; ++k) {
      const uint32_t e = lst[k * kForceThreads];
      const int j = (int)(e & kSlotMask);
      const float4 pj = __ldg(P.pos + j);
      const float4 vj = __ldg(P.vel + j);
      float dx, dy, dz;
      if (e & ~kSlotMask) {  // pair across a box face (rare)
        dx = ((e & kCodeIX) ? pi.x - Lx : pi.x) - ((e & kCodeJX) ? pj.x - Lx : pj.x);
        dy = ((e & kCodeIY) ? pi.y - Ly : pi.y) - ((e & kCodeJY) ? pj.y - Ly : pj.y);
        dz = ((e & kCodeIZ) ? pi.z - Lz : pi.z) - ((e & kCodeJZ) ? pj.z - Lz : pj.z);
      } else {
        dx = pi.x - pj.x;
        dy = pi.y - pj.y;
        dz = pi.z - pj.z;
      }
      const uint32_t idj = __float_as_uint(pj.w);
      const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      const float rinv = rsqrtf(r2);
      const float r = r2 * rinv;
      const float w = fmaxf(fmaf(-r, B.inv_rc, 1.0f), 0.0f);
      const float wR = (B.kexp == 1.0f) ? w : powf(w, B.kexp);
      const float ev = fmaf(dx, vi.x - vj.x, fmaf(dy, vi.y - vj.y, dz * (vi.z - vj.z))) * rinv;
      const uint32_t u = pair_word(idi, idj, slo, shi, B.seed_lo, B.seed_hi);
      const float fc = B.a * w;
      const float s = fmaf(B.sig * wR, noise_int(u), fmaf(-B.gamma * wR * wR, ev, fc)) * rinv;
      const float gx = s * dx, gy = s * dy, gz = s * dz;
      fx += gx;
      fy += gy;
      fz += gz;
      const float vterm = fc * r;
      vir += vterm;
      if constexpr (HALF) {
        atomicAdd(P.frc + j, make_float4(-gx, -gy, -gz, vterm));
      }
    }
    cnt = 0;
  };

  // One contiguous slot range with a fixed image code; drains when the list fills.
  auto range = [&](int j0, int j1, float ax, float ay, float az, float jsx, float jsy, float jsz,
                   uint32_t code) {
    while (j0 < j1) {
      const int stop = (code & (kCodeJX | kCodeJY | kCodeJZ))
                           ? scan_range<true>(P.pos, j0, j1, ax, ay, az, jsx, jsy, jsz, B.rc2,
                                              code, lst, cnt)
                           : scan_range<false>(P.pos, j0, j1, ax, ay, az, 0.f, 0.f, 0.f, B.rc2,
                                               code, lst, cnt);
      if (stop < 0) break;
      drain();
      j0 = stop + 1;
    }
  };

  // Cells cx-1..cx+1 (or cx..cx+1 from `xlo`) of one row; one range unless
  // the row crosses an x face.
  auto row = [&](int rowbase, float ay, float az, float jsy, float jsz, uint32_t code) {
    if (cx >= 1 && cx <= nx - 2) {
      range(__ldg(P.start + rowbase + cx - 1), __ldg(P.start + rowbase + cx + 2), pi.x, ay, az,
            0.f, jsy, jsz, code);
    } else {
      for (int dxc = -1; dxc <= 1; ++dxc) {
        int x = cx + dxc;
        float ax = pi.x, jsx = 0.f;
        uint32_t c = code;
        if (x < 0) {
          x += nx;
          jsx = Lx;
          c |= kCodeJX;
        } else if (x >= nx) {
          x -= nx;
          ax = pi.x - Lx;
          c |= kCodeIX;
        }
        range(__ldg(P.start + rowbase + x), __ldg(P.start + rowbase + x + 1), ax, ay, az, jsx,
              jsy, jsz, c);
      }
    }
  };

  auto rowfor = [&](int dy, int dz) {
    int z = cz + dz, y = cy + dy;
    float az = pi.z, jsz = 0.f, ay = pi.y, jsy = 0.f;
    uint32_t code = 0;
    if (z < 0) {
      z += nz;
      jsz = Lz;
      code |= kCodeJZ;
    } else if (z >= nz) {
      z -= nz;
      az = pi.z - Lz;
      code |= kCodeIZ;
    }
    if (y < 0) {
      y += ny;
      jsy = Ly;
      code |= kCodeJY;
    } else if (y >= ny) {
      y -= ny;
      ay = pi.y - Ly;
      code |= kCodeIY;
    }
    if (alive) row(B.cellBase + (z * ny + y) * nx, ay, az, jsy, jsz, code);
    if (__any_sync(0xffffffffu, cnt > kFlushAt)) drain();
  };

  if constexpr (!HALF) {
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy) rowfor(dy, dz);
  } else {
    // Half stencil: own cell (slots after p) and cell cx+1 of the own row, the
    // row dy=+1 of the own plane, and the three rows of the plane dz=+1.
    if (alive) {
      const int rowbase = B.cellBase + (cz * ny + cy) * nx;
      if (cx + 1 <= nx - 1) {
        range(p + 1, __ldg(P.start + rowbase + cx + 2), pi.x, pi.y, pi.z, 0.f, 0.f, 0.f, 0u);
      } else {
        range(p + 1, __ldg(P.start + rowbase + cx + 1), pi.x, pi.y, pi.z, 0.f, 0.f, 0.f, 0u);
        range(__ldg(P.start + rowbase), __ldg(P.start + rowbase + 1), pi.x - Lx, pi.y, pi.z, 0.f,
              0.f, 0.f, kCodeIX);
      }
    }
    if (__any_sync(0xffffffffu, cnt > kFlushAt)) drain();
    rowfor(1, 0);
    rowfor(-1, 1);
    rowfor(0, 1);
    rowfor(1, 1);
  }
  drain();

  if (!alive) return;
  if (B.fb_mode != 0) {  // body force (Sec. 4.2 periodic Poiseuille, or constant)
    float add = B.fb;
    if (B.fb_mode == 2) {
      const float xg = (B.fb_grad == 0) ? pi.x : (B.fb_grad == 1) ? pi.y : pi.z;
      add = (xg <= B.fb_half) ? -B.fb : B.fb;
    }
    if (B.fb_flow == 0)
      fx += add;
    else if (B.fb_flow == 1)
      fy += add;
    else
      fz += add;
  }
  if constexpr (HALF) {
    atomicAdd(P.frc + p, make_float4(fx, fy, fz, vir));
  } else {
    P.frc[p] = make_float4(fx, fy, fz, vir);
  }
}

template <bool SINGLE, bool HALF>
__global__ void __launch_bounds__(kForceThreads) k_force(Packed P) {
  __shared__ uint32_t smem_list[kListCap * kForceThreads];
  const int p = blockIdx.x * kForceThreads + threadIdx.x;
  bool alive = p < P.ntot;
  const int b = (!SINGLE && alive) ? find_box(P.pbase, P.nbox, p) : 0;
  const BoxDev B = box_of<SINGLE>(P, b);
  const BoxState S = P.st[b];
  alive = alive && S.adv;
  force_direct<HALF>(P, B, S, p, alive, smem_list + threadIdx.x);
}

// ------------------------------------------------------- staged force tiles
// A thread block owns a run of `nc` consecutive cells (cx0 .. cx0+nc-1) of
// one x-row of one box.  It copies the 9 neighbouring row segments -- cells
// cx0-1 .. cx0+nc of rows (cy+dy, cz+dz) -- into shared memory, positions
// and velocities, then every thread takes a target particle of its own row
// and scans its 27 cells from shared memory.
//
// Periodic images: a neighbour image r_j - L (j in the top cells, row or
// cell wrapped below) is stored pre-shifted, which is exact in FP32 because
// that coordinate lies in [2L/3, L).  An image r_j + L is never formed:
// the target uses r_i - L instead (exact for the same reason): per row for
// y and z, per thread for the wrapped cell 0 at the x end of the row.
struct TileRow {
  int rb;                  // packed index of the row's first cell
  int gBeg, lenBeg;        // wrapped cell nx-1 (x image - L), only when cx0 == 0
  int gMain, lenMain;      // cells max(cx0-1,0) .. min(cx0+nc, nx-1)
  int gEnd, lenEnd;        // wrapped cell 0, only when cx0 + nc == nx
  int off;                 // first shared-memory slot of the row
  float jsy, jsz;          // pre-shift of stored y / z (0 or L)
  uint32_t ish;            // i-shift code bits for y / z (kCodeIY / kCodeIZ)
  int pad;
};

// Scan staged candidates [j0, j1) against one target; entries are the staged
// index (16 bits) plus i-shift code bits.  Returns the index at which the
// list filled, or -1.
__device__ __forceinline__ int scan_staged(const float4 *__restrict__ sPos, int j0, int j1,
                                           float ax, float ay, float az, float rc2, uint32_t code,
                                           uint32_t *__restrict__ lst, int stride, int &cnt,
                                           int cap) {
  for (int j = j0; j < j1; ++j) {
    const float4 pj = sPos[j];
    const float dx = ax - pj.x, dy = ay - pj.y, dz = az - pj.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const bool hit = (r2 < rc2) & (r2 > 0.0f);
    lst[cnt * stride] = (uint32_t)j | code;
    cnt += hit ? 1 : 0;
    if (cnt == cap) return j;
  }
  return -1;
}

template <bool SINGLE>
__global__ void __launch_bounds__(kTileThreads) k_force_tiles(Packed P, TileGrid G) {
  extern __shared__ float4 tile_smem[];
  __shared__ TileRow rows[9];
  __shared__ int sB[9][kTileMaxCells + 3];
  __shared__ int sTotal;

  const int tid = threadIdx.x;
  int b, cy, cz, cx0, nc;
  BoxDev B;
  if constexpr (SINGLE) {
    B = P.single;
    b = 0;
    const int t = blockIdx.x;
    const int rowi = t / G.tpr;
    cx0 = (t - rowi * G.tpr) * G.tc;
    nc = min(G.tc, B.n[0] - cx0);
    cy = rowi % B.n[1];
    cz = rowi / B.n[1];
  } else {
    const int4 d = G.list[blockIdx.x];
    b = d.x;
    cy = d.y;
    cz = d.z;
    cx0 = d.w & 0xFFFF;
    nc = d.w >> 16;
    B = P.boxes[b];
  }
  const BoxState S = P.st[b];
  if (!S.adv) return;  // uniform over the block
  const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
  const float Lx = B.L[0], Ly = B.L[1], Lz = B.L[2];
  const int m0 = max(cx0 - 1, 0), m1 = min(cx0 + nc, nx - 1);

  if (tid < 9) {
    const int dz = tid / 3 - 1, dy = tid % 3 - 1;
    int zz = cz + dz, yy = cy + dy;
    TileRow R;
    R.jsy = 0.f;
    R.jsz = 0.f;
    R.ish = 0u;
    if (zz < 0) {
      zz += nz;
      R.jsz = Lz;
    } else if (zz >= nz) {
      zz -= nz;
      R.ish |= kCodeIZ;
    }
    if (yy < 0) {
      yy += ny;
      R.jsy = Ly;
    } else if (yy >= ny) {
      yy -= ny;
      R.ish |= kCodeIY;
    }
    R.rb = B.cellBase + (zz * ny + yy) * nx;
    R.gMain = __ldg(P.start + R.rb + m0);
    R.lenMain = __ldg(P.start + R.rb + m1 + 1) - R.gMain;
    R.gBeg = 0;
    R.lenBeg = 0;
    if (cx0 == 0) {
      R.gBeg = __ldg(P.start + R.rb + nx - 1);
      R.lenBeg = __ldg(P.start + R.rb + nx) - R.gBeg;
    }
    R.gEnd = 0;
    R.lenEnd = 0;
    if (cx0 + nc == nx) {
      R.gEnd = __ldg(P.start + R.rb);
      R.lenEnd = __ldg(P.start + R.rb + 1) - R.gEnd;
    }
    R.off = 0;
    R.pad = 0;
    rows[tid] = R;
  }
  __syncthreads();
  if (tid == 0) {
    int off = 0;
    for (int r = 0; r < 9; ++r) {
      rows[r].off = off;
      off += rows[r].lenBeg + rows[r].lenMain + rows[r].lenEnd;
    }
    sTotal = off;
  }
  __syncthreads();
  const int total = sTotal;
  const bool staged = total <= G.stage_cap;
  float4 *sPos = tile_smem;
  float4 *sVel = tile_smem + G.stage_cap;
  uint32_t *lst = reinterpret_cast<uint32_t *>(tile_smem + 2 * G.stage_cap);

  // targets: the tile's own cells in the centre row (rows[4] is dy = dz = 0)
  const int t0 = __ldg(P.start + rows[4].rb + cx0);
  const int t1 = __ldg(P.start + rows[4].rb + cx0 + nc);

  if (!staged) {
    // too many particles to stage: read neighbours from global memory
    for (int base = t0; base < t1; base += kTileThreads) {
      const int p = base + tid;
      force_direct<false>(P, B, S, p, p < t1, lst + tid);
    }
    return;
  }

  // cell boundaries inside the staged rows: sB[r][k] = first staged slot of
  // virtual cell cx0 - 1 + k, k = 0 .. nc + 2
  for (int idx = tid; idx < 9 * (nc + 3); idx += kTileThreads) {
    const int r = idx / (nc + 3), k = idx - r * (nc + 3);
    const TileRow &R = rows[r];
    const int x = cx0 - 1 + k;
    int v;
    if (x < m0)
      v = R.off;
    else if (x <= m1 + 1)
      v = R.off + R.lenBeg + (__ldg(P.start + R.rb + x) - R.gMain);
    else
      v = R.off + R.lenBeg + R.lenMain + R.lenEnd;
    sB[r][k] = v;
  }
  // copy the neighbourhood (coalesced float4 loads)
  for (int r = 0; r < 9; ++r) {
    const TileRow &R = rows[r];
    const int len = R.lenBeg + R.lenMain + R.lenEnd;
    for (int i = tid; i < len; i += kTileThreads) {
      int g;
      float xs = 0.f;
      if (i < R.lenBeg) {
        g = R.gBeg + i;
        xs = Lx;
      } else if (i < R.lenBeg + R.lenMain) {
        g = R.gMain + (i - R.lenBeg);
      } else {
        g = R.gEnd + (i - R.lenBeg - R.lenMain);
      }
      float4 q = __ldg(P.pos + g);
      q.x -= xs;
      q.y -= R.jsy;
      q.z -= R.jsz;
      sPos[R.off + i] = q;
      sVel[R.off + i] = __ldg(P.vel + g);
    }
  }
  __syncthreads();

  const float rc2 = B.rc2;
  const uint32_t slo = (uint32_t)S.step, shi = (uint32_t)(S.step >> 32);
  const bool xend = (cx0 + nc == nx);
  for (int base = t0; base < t1; base += kTileThreads) {
    const int p = base + tid;
    const bool alive = p < t1;
    float4 pi = make_float4(0.f, 0.f, 0.f, 0.f), vi = pi;
    if (alive) {
      pi = __ldg(P.pos + p);
      vi = __ldg(P.vel + p);
    }
    int cx, cyy, czz;
    unpack_cell(__float_as_int(vi.w), cx, cyy, czz);
    const int kt = cx - cx0 + 1;  // virtual cell of the target, 1..nc
    const uint32_t idi = __float_as_uint(pi.w);
    float fx = 0.f, fy = 0.f, fz = 0.f, vir = 0.f;
    int cnt = 0;
    uint32_t *my = lst + tid;

    auto drain = [&]() {
      for (int k = 0; k < cnt; ++k) {
        const uint32_t e = my[k * kTileThreads];
        const int j = (int)(e & 0xFFFFu);
        const float4 pj = sPos[j];
        const float4 vj = sVel[j];
        const float ax = (e & kCodeIX) ? pi.x - Lx : pi.x;
        const float ay = (e & kCodeIY) ? pi.y - Ly : pi.y;
        const float az = (e & kCodeIZ) ? pi.z - Lz : pi.z;
        const float dx = ax - pj.x, dy = ay - pj.y, dz = az - pj.z;
        const uint32_t idj = __float_as_uint(pj.w);
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float rinv = rsqrtf(r2);
        const float r = r2 * rinv;
        const float w = fmaxf(fmaf(-r, B.inv_rc, 1.0f), 0.0f);
        const float wR = (B.kexp == 1.0f) ? w : powf(w, B.kexp);
        const float ev =
            fmaf(dx, vi.x - vj.x, fmaf(dy, vi.y - vj.y, dz * (vi.z - vj.z))) * rinv;
        const uint32_t u = pair_word(idi, idj, slo, shi, B.seed_lo, B.seed_hi);
        const float fc = B.a * w;
        const float sc = fmaf(B.sig * wR, noise_int(u), fmaf(-B.gamma * wR * wR, ev, fc)) * rinv;
        fx = fmaf(sc, dx, fx);
        fy = fmaf(sc, dy, fy);
        fz = fmaf(sc, dz, fz);
        vir = fmaf(fc, r, vir);
      }
      cnt = 0;
    };

    for (int r = 0; r < 9; ++r) {
      if (alive) {
        const TileRow &R = rows[r];
        const float ay = (R.ish & kCodeIY) ? pi.y - Ly : pi.y;
        const float az = (R.ish & kCodeIZ) ? pi.z - Lz : pi.z;
        int j0 = sB[r][kt - 1];
        const int j1 = sB[r][kt + 2];
        // the wrapped cell 0 past the x end is seen from r_i - L
        const int jx = (xend && kt == nc) ? sB[r][nc + 1] : j1;
        while (j0 < jx) {
          const int stop = scan_staged(sPos, j0, jx, pi.x, ay, az, rc2, R.ish, my, kTileThreads,
                                       cnt, kListCap);
          if (stop < 0) break;
          drain();
          j0 = stop + 1;
        }
        j0 = max(j0, jx);
        while (j0 < j1) {
          const int stop = scan_staged(sPos, j0, j1, pi.x - Lx, ay, az, rc2, R.ish | kCodeIX, my,
                                       kTileThreads, cnt, kListCap);
          if (stop < 0) break;
          drain();
          j0 = stop + 1;
        }
      }
      if (__any_sync(0xffffffffu, cnt > kFlushAt)) drain();
    }
    drain();
    if (alive) {
      if (B.fb_mode != 0) {
        float add = B.fb;
        if (B.fb_mode == 2) {
          const float xg = (B.fb_grad == 0) ? pi.x : (B.fb_grad == 1) ? pi.y : pi.z;
          add = (xg <= B.fb_half) ? -B.fb : B.fb;
        }
        if (B.fb_flow == 0)
          fx += add;
        else if (B.fb_flow == 1)
          fy += add;
        else
          fz += add;
      }
      P.frc[p] = make_float4(fx, fy, fz, vir);
    }
  }
}

// ------------------------------------------------------------------ stats
constexpr int kStatsThreads = 256;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kStatsThreads) k_stats(Packed P, const StatsWork *__restrict__ work,
                                                         double *__restrict__ out) {
  const StatsWork w = work[blockIdx.x];
  const BoxDev B = P.boxes[w.box];
  const BoxState S = P.st[w.box];
  const float h = S.pending ? B.hdt_m : 0.0f;
  double acc[kStatsFields] = {0, 0, 0, 0, 0, 0};
  for (int p = w.begin + threadIdx.x; p < w.end; p += kStatsThreads) {
    float4 v = P.vel[p];
    const float4 f = P.frc[p];
    v.x = fmaf(h, f.x, v.x);
    v.y = fmaf(h, f.y, v.y);
    v.z = fmaf(h, f.z, v.z);
    acc[0] += (double)v.x;
    acc[1] += (double)v.y;
    acc[2] += (double)v.z;
    acc[3] += (double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z;
    acc[4] += (double)f.w;
    acc[5] += 1.0;
  }
  __shared__ double red[kStatsFields][kStatsThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kStatsFields; ++k) {
    const double s = warp_sum_d(acc[k]);
    if (lane == 0) red[k][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x < kStatsFields) {
    double s = 0.0;
    for (int q = 0; q < kStatsThreads / 32; ++q) s += red[threadIdx.x][q];
    out[(size_t)blockIdx.x * kStatsFields + threadIdx.x] = s;
  }
}

// ----------------------------------------------------------------- gather
__global__ void k_gather(Packed P, int box, int slot0, int n, float *__restrict__ pos3,
                         float *__restrict__ vel3, float *__restrict__ frc3) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int p = slot0 + k;
  const float4 x = P.pos[p];
  const int id = __float_as_int(x.w);
  if (id < 0 || id >= n) {
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
                            uint32_t *__restrict__ out, float *__restrict__ xi) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint32_t u = pair_word(lo[k], hi[k], slo, shi, klo, khi);
  out[k] = u;
  if (xi) xi[k] = __fmul_rn(noise_int(u), kSqrt3Scale);
}

// ================================================================ launchers
static inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

cudaError_t launch_load(const Packed &P, int slot0, int n, const float *pos3, const float *vel3,
                        float Lx, float Ly, float Lz, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_load<<<blocks_for(n, 256), 256, 0, s>>>(P, slot0, n, pos3, vel3, Lx, Ly, Lz);
  return cudaGetLastError();
}

size_t tile_smem_bytes(int stage_cap) {
  return (size_t)stage_cap * 2 * sizeof(float4) + (size_t)kListCap * kTileThreads * sizeof(uint32_t);
}

cudaError_t prepare_device() {
  // staged tiles may use more than the default 48 KB of dynamic shared memory
  const int maxb = 200 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_force_tiles<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, maxb);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_force_tiles<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              maxb);
}

static cudaError_t launch_force(const Packed &P, const StepConfig &cfg, cudaStream_t s) {
  const bool single = (P.nbox == 1);
  if (cfg.stencil == 1) {
    if (single)
      k_force<true, true><<<blocks_for(P.ntot, kForceThreads), kForceThreads, 0, s>>>(P);
    else
      k_force<false, true><<<blocks_for(P.ntot, kForceThreads), kForceThreads, 0, s>>>(P);
  } else if (cfg.tiles && cfg.grid.ntiles > 0) {
    const size_t smem = tile_smem_bytes(cfg.grid.stage_cap);
    if (single)
      k_force_tiles<true><<<cfg.grid.ntiles, kTileThreads, smem, s>>>(P, cfg.grid);
    else
      k_force_tiles<false><<<cfg.grid.ntiles, kTileThreads, smem, s>>>(P, cfg.grid);
  } else {
    if (single)
      k_force<true, false><<<blocks_for(P.ntot, kForceThreads), kForceThreads, 0, s>>>(P);
    else
      k_force<false, false><<<blocks_for(P.ntot, kForceThreads), kForceThreads, 0, s>>>(P);
  }
  return cudaGetLastError();
}

cudaError_t launch_step(const Packed &P, bool move, bool advance, const StepConfig &cfg,
                        cudaStream_t s) {
  if (P.ntot <= 0) return cudaSuccess;
  const bool single = (P.nbox == 1);
  const int gb = blocks_for(P.ntot, kBinThreads);
  if (single)
    k_integrate_bin<true><<<gb, kBinThreads, 0, s>>>(P, move);
  else
    k_integrate_bin<false><<<gb, kBinThreads, 0, s>>>(P, move);
  const int nt = scan_tiles(P.ncell);
  k_scan_reduce<<<nt, kScanThreads, 0, s>>>(P.count, P.bsum);
  k_scan_bsum<<<1, 1024, 0, s>>>(P.bsum, nt);
  k_scan_apply<<<nt, kScanThreads, 0, s>>>(P, advance);
  k_bin_keys<<<gb, kBinThreads, 0, s>>>(P);
  k_bin_scatter<<<gb, kBinThreads, 0, s>>>(P, cfg.stencil == 1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_force(P, cfg, s);
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
  k_bin_keys<<<gb, kBinThreads, 0, s>>>(P);
  if ((e = cudaEventRecord(ev[3], s)) != cudaSuccess) return e;
  k_bin_scatter<<<gb, kBinThreads, 0, s>>>(P, cfg.stencil == 1);
  if ((e = cudaEventRecord(ev[4], s)) != cudaSuccess) return e;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_force(P, cfg, s)) != cudaSuccess) return e;
  return cudaEventRecord(ev[5], s);
}

cudaError_t launch_stats(const Packed &P, const StatsWork *work, int nwork, double *out,
                         cudaStream_t s) {
  if (nwork <= 0) return cudaSuccess;
  k_stats<<<nwork, kStatsThreads, 0, s>>>(P, work, out);
  return cudaGetLastError();
}

cudaError_t launch_gather(const Packed &P, int box, int slot0, int n, float *pos3, float *vel3,
                          float *frc3, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_gather<<<blocks_for(n, 256), 256, 0, s>>>(P, box, slot0, n, pos3, vel3, frc3);
  return cudaGetLastError();
}

cudaError_t launch_debug_rng(const uint32_t *lo, const uint32_t *hi, long long n, uint64_t step,
                             uint64_t seed, uint32_t *out, float *xi, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_debug_rng<<<blocks_for(n, 256), 256, 0, s>>>(lo, hi, n, (uint32_t)step,
                                                 (uint32_t)(step >> 32), (uint32_t)seed,
                                                 (uint32_t)(seed >> 32), out, xi);
  return cudaGetLastError();
}

}  // namespace dpd
