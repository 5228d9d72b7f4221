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
constexpr int kForceThreads = 128;
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
// Candidate pass: test every particle j of a contiguous slot range against i
// and append those inside rc to i's list as (r_ij, j).  jsh[] are the image
// shifts subtracted from r_j (non-zero only for ranges across a box face).
template <bool JSHIFT>
__device__ __forceinline__ void scan_range(const float4 *__restrict__ pos, int j0, int j1, int p,
                                           float aix, float aiy, float aiz, float jsx, float jsy,
                                           float jsz, float rc2, float4 *__restrict__ lst,
                                           int &cnt, bool &full) {
  for (int j = j0; j < j1; ++j) {
    const float4 pj = __ldg(pos + j);
    float dx, dy, dz;
    if constexpr (JSHIFT) {
      dx = aix - (pj.x - jsx);
      dy = aiy - (pj.y - jsy);
      dz = aiz - (pj.z - jsz);
    } else {
      dx = aix - pj.x;
      dy = aiy - pj.y;
      dz = aiz - pj.z;
    }
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (r2 < rc2 && r2 > 0.0f && j != p) {
      lst[cnt * kForceThreads] = make_float4(dx, dy, dz, __int_as_float(j));
      ++cnt;
      if (cnt == kListCap) {
        full = true;
        return;
      }
    }
  }
}

template <bool SINGLE, bool HALF>
__global__ void __launch_bounds__(kForceThreads) k_force(Packed P) {
  extern __shared__ float4 smem_list[];
  float4 *lst = smem_list + threadIdx.x;  // entry k of this thread at lst[k * kForceThreads]
  const int p = blockIdx.x * kForceThreads + threadIdx.x;
  bool alive = p < P.ntot;
  const int b = (!SINGLE && alive) ? find_box(P.pbase, P.nbox, p) : 0;
  const BoxDev B = box_of<SINGLE>(P, b);
  const BoxState S = P.st[b];
  alive = alive && S.adv;

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

  // Pair forces for every listed neighbour (Eqs. 3-5); empties the list.
  auto drain = [&]() {
    for (int k = 0; k < cnt; ++k) {
      const float4 e = lst[k * kForceThreads];
      const int j = __float_as_int(e.w);
      const float4 vj = __ldg(P.vel + j);
      const uint32_t idj = __float_as_uint(__ldg(&P.pos[j].w));
      const float r2 = fmaf(e.x, e.x, fmaf(e.y, e.y, e.z * e.z));
      const float rinv = rsqrtf(r2);
      const float r = r2 * rinv;
      const float w = fmaxf(fmaf(-r, B.inv_rc, 1.0f), 0.0f);
      const float wR = (B.kexp == 1.0f) ? w : powf(w, B.kexp);
      const float ev =
          fmaf(e.x, vi.x - vj.x, fmaf(e.y, vi.y - vj.y, e.z * (vi.z - vj.z))) * rinv;
      const uint32_t u = pair_word(idi, idj, slo, shi, B.seed_lo, B.seed_hi);
      const float fc = B.a * w;
      const float s = fmaf(B.sig * wR, noise_int(u), fmaf(-B.gamma * wR * wR, ev, fc)) * rinv;
      const float gx = s * e.x, gy = s * e.y, gz = s * e.z;
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

  // One contiguous slot range with a fixed image shift.
  auto range = [&](int j0, int j1, float aix, float aiy, float aiz, float jsx, float jsy,
                   float jsz) {
    while (j0 < j1) {
      bool full = false;
      const int before = cnt;
      if (jsx != 0.f || jsy != 0.f || jsz != 0.f)
        scan_range<true>(P.pos, j0, j1, p, aix, aiy, aiz, jsx, jsy, jsz, B.rc2, lst, cnt, full);
      else
        scan_range<false>(P.pos, j0, j1, p, aix, aiy, aiz, 0.f, 0.f, 0.f, B.rc2, lst, cnt, full);
      if (!full) break;
      // list full: find where the scan stopped, drain, continue after it
      const int jlast = __float_as_int(lst[(kListCap - 1) * kForceThreads].w);
      (void)before;
      drain();
      j0 = jlast + 1;
    }
  };

  // Three cells cx-1..cx+1 of one row; a single range unless the row crosses an x face.
  auto row = [&](int rowbase, int xlo, float aiy, float aiz, float jsy, float jsz) {
    if (cx + xlo >= 0 && cx + 1 <= nx - 1) {
      range(__ldg(P.start + rowbase + cx + xlo), __ldg(P.start + rowbase + cx + 2), pi.x, aiy, aiz,
            0.f, jsy, jsz);
    } else {
      for (int dx = xlo; dx <= 1; ++dx) {
        int x = cx + dx;
        float aix = pi.x, jsx = 0.f;
        if (x < 0) {
          x += nx;
          jsx = Lx;  // neighbour image at r_j - L
        } else if (x >= nx) {
          x -= nx;
          aix = pi.x - Lx;  // i seen from the far side: r_i - L
        }
        range(__ldg(P.start + rowbase + x), __ldg(P.start + rowbase + x + 1), aix, aiy, aiz, jsx,
              jsy, jsz);
      }
    }
  };

  if constexpr (!HALF) {
    for (int dz = -1; dz <= 1; ++dz) {
      int z = cz + dz;
      float aiz = pi.z, jsz = 0.f;
      if (z < 0) {
        z += nz;
        jsz = Lz;
      } else if (z >= nz) {
        z -= nz;
        aiz = pi.z - Lz;
      }
      for (int dy = -1; dy <= 1; ++dy) {
        int y = cy + dy;
        float aiy = pi.y, jsy = 0.f;
        if (y < 0) {
          y += ny;
          jsy = Ly;
        } else if (y >= ny) {
          y -= ny;
          aiy = pi.y - Ly;
        }
        if (alive) row(B.cellBase + (z * ny + y) * nx, -1, aiy, aiz, jsy, jsz);
        if (__any_sync(0xffffffffu, cnt > kFlushAt)) drain();
      }
    }
  } else {
    // Half stencil: own cell (slots after p) and cell cx+1 of the own row, the
    // row dy=+1 of the own plane, and the three rows of the plane dz=+1.
    if (alive) {
      const int rowbase = B.cellBase + (cz * ny + cy) * nx;
      if (cx + 1 <= nx - 1) {
        range(p + 1, __ldg(P.start + rowbase + cx + 2), pi.x, pi.y, pi.z, 0.f, 0.f, 0.f);
      } else {
        range(p + 1, __ldg(P.start + rowbase + cx + 1), pi.x, pi.y, pi.z, 0.f, 0.f, 0.f);
        range(__ldg(P.start + rowbase), __ldg(P.start + rowbase + 1), pi.x - Lx, pi.y, pi.z, 0.f,
              0.f, 0.f);
      }
    }
    if (__any_sync(0xffffffffu, cnt > kFlushAt)) drain();
    for (int r = 0; r < 4; ++r) {
      const int dz = (r == 0) ? 0 : 1;
      const int dy = (r == 0) ? 1 : r - 2;
      int z = cz + dz;
      float aiz = pi.z, jsz = 0.f;
      if (z >= nz) {
        z -= nz;
        aiz = pi.z - Lz;
      }
      int y = cy + dy;
      float aiy = pi.y, jsy = 0.f;
      if (y < 0) {
        y += ny;
        jsy = Ly;
      } else if (y >= ny) {
        y -= ny;
        aiy = pi.y - Ly;
      }
      if (alive) row(B.cellBase + (z * ny + y) * nx, -1, aiy, aiz, jsy, jsz);
      if (__any_sync(0xffffffffu, cnt > kFlushAt)) drain();
    }
  }
  drain();

  if (!alive) return;
  // body force (Sec. 4.2 periodic Poiseuille, or constant)
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
  if constexpr (HALF) {
    atomicAdd(P.frc + p, make_float4(fx, fy, fz, vir));
  } else {
    P.frc[p] = make_float4(fx, fy, fz, vir);
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

static size_t force_smem() { return sizeof(float4) * kListCap * kForceThreads; }

template <bool SINGLE, bool HALF>
static cudaError_t launch_force(const Packed &P, cudaStream_t s) {
  const size_t smem = force_smem();
  k_force<SINGLE, HALF><<<blocks_for(P.ntot, kForceThreads), kForceThreads, smem, s>>>(P);
  return cudaGetLastError();
}

cudaError_t prepare_device() {
  const int smem = (int)force_smem();
  cudaError_t e;
  e = cudaFuncSetAttribute(k_force<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_force<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_force<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_force<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem);
}

cudaError_t launch_step(const Packed &P, bool move, bool advance, int stencil, cudaStream_t s) {
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
  const bool half = (stencil == 1);
  k_bin_scatter<<<gb, kBinThreads, 0, s>>>(P, half);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (single)
    return half ? launch_force<true, true>(P, s) : launch_force<true, false>(P, s);
  return half ? launch_force<false, true>(P, s) : launch_force<false, false>(P, s);
}

cudaError_t launch_step_timed(const Packed &P, int stencil, cudaStream_t s, cudaEvent_t *ev) {
  if (P.ntot <= 0) return cudaSuccess;
  const bool single = (P.nbox == 1);
  const int gb = blocks_for(P.ntot, kBinThreads);
  const bool half = (stencil == 1);
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
  k_bin_scatter<<<gb, kBinThreads, 0, s>>>(P, half);
  if ((e = cudaEventRecord(ev[4], s)) != cudaSuccess) return e;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (single)
    e = half ? launch_force<true, true>(P, s) : launch_force<true, false>(P, s);
  else
    e = half ? launch_force<false, true>(P, s) : launch_force<false, false>(P, s);
  if (e != cudaSuccess) return e;
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
