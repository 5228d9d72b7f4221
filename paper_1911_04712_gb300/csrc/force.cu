// Force kernels of the DPD step: pair forces (Sec. 2.1, Eqs. 2-5) over the
// cell list (Sec. 3.2).  One thread per target particle collects its
// neighbours inside rc into a shared-memory pair list and then evaluates
// them; the variants differ in block size, list capacity and how a warp
// drains its lists (per lane, balanced in list order, or spread over the
// lanes with atomic sums), chosen per density band from tuning tables.
// General variants also serve Gaussian noise and several species.  The full
// stencil can fuse the next step's integrate into its epilogue.  Plus the
// optional shared-memory staged tiles.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <vector>

#include "dpd_device.cuh"
#include "force_direct.cuh"
#include "kernels.h"

namespace dpd {

constexpr int kTileListCap = 24;

static inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

// One thread per target slot in [slot0, slot1).
template <bool SINGLE, bool HALF, int NT, int CAP, bool BAL, bool GAUSS, bool SPREAD>
__global__ void __launch_bounds__(NT) k_force(Packed P, int slot0, int slot1, bool fuse) {
  constexpr int kListWords = BAL ? 1 : CAP * NT;
  __shared__ uint32_t smem_list[kListWords];
  __shared__ WarpScratch<BAL ? CAP : 4> smem_warp[BAL ? NT / 32 : 1];
  __shared__ float4 smem_own[SPREAD ? 2 * NT : 1];
  const int p = slot0 + blockIdx.x * NT + threadIdx.x;
  const bool real = p < slot1;
  bool alive = real;
  int b = 0;
  if constexpr (!SINGLE) b = find_box_warp(P.pbase, P.nbox, min(p, P.ntot - 1));
  const BoxState S = P.st[b];
  alive = alive && S.adv;
  // Lanes of this warp in more than one box.  Every lane counts, dead ones
  // too: past the end of a band they belong to the next band's box, and the
  // balanced and spread drains hand them other lanes' entries.  Such warps
  // are left to k_force_warps (the host lists them per band).
  if constexpr (!SINGLE && (BAL || SPREAD)) {
    const int b0 = __shfl_sync(0xffffffffu, b, 0);
    if (!__all_sync(0xffffffffu, b == b0)) return;
  }
  constexpr bool mixed = false;
  auto run = [&](const BoxDev &B) {
    if constexpr (BAL) {
      WarpScratch<CAP> *W = &smem_warp[threadIdx.x >> 5];
      force_direct<HALF, NT, CAP, true, GAUSS>(P, B, S, p, alive,
                                               W->list + (threadIdx.x & 31) * (CAP + 1), W,
                                               nullptr, mixed, fuse, real);
    } else if constexpr (SPREAD) {
      force_direct<HALF, NT, CAP, false, GAUSS, true>(P, B, S, p, alive, smem_list + threadIdx.x,
                                                      nullptr, smem_own + (threadIdx.x >> 5) * 64,
                                                      mixed, fuse, real);
    } else {
      force_direct<HALF, NT, CAP, false, GAUSS>(P, B, S, p, alive, smem_list + threadIdx.x,
                                                nullptr, nullptr, false, fuse, real);
    }
  };
  if constexpr (SINGLE) {
    run(P.single);
  } else {
    run(P.boxes[b]);  // read where used from the box table, not copied into registers
  }
}

// The warps of a packed set whose slots span two boxes, one block of 32
// threads each (first slots in warp_start), with the per-lane drain: each
// lane evaluates only its own pairs, with its own box's parameters.
template <bool HALF, int CAP, bool GAUSS>
__global__ void __launch_bounds__(32)
    k_force_warps(Packed P, const int *__restrict__ warp_start, int slot1, bool fuse) {
  __shared__ uint32_t smem_list[CAP * 32];
  const int p = warp_start[blockIdx.x] + (int)threadIdx.x;
  const bool real = p < slot1;
  const int b = find_box(P.pbase, P.nbox, min(p, P.ntot - 1));
  const BoxState S = P.st[b];
  const bool alive = real && S.adv;
  force_direct<HALF, 32, CAP, false, GAUSS>(P, P.boxes[b], S, p, alive, smem_list + threadIdx.x,
                                            nullptr, nullptr, false, fuse, real);
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
    nc = min(G.tc, B.n[0] / kSlicesX - cx0);
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
  // the tile works in whole cells: cell x of a row is slices kSlicesX x .. kSlicesX x + kSlicesX - 1
  const int nx = B.n[0] / kSlicesX, ny = B.n[1], nz = B.n[2];
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
    R.rb = B.cellBase + (zz * ny + yy) * B.n[0];
    if (!DPD_IN_BOUNDS(R.rb >= 0 && R.rb + B.n[0] <= P.ncell, P.err)) R.rb = 0;
    R.gMain = __ldg(P.start + R.rb + kSlicesX * m0);
    R.lenMain = __ldg(P.start + R.rb + kSlicesX * (m1 + 1)) - R.gMain;
    R.gBeg = 0;
    R.lenBeg = 0;
    if (cx0 == 0) {
      R.gBeg = __ldg(P.start + R.rb + kSlicesX * (nx - 1));
      R.lenBeg = __ldg(P.start + R.rb + kSlicesX * nx) - R.gBeg;
    }
    R.gEnd = 0;
    R.lenEnd = 0;
    if (cx0 + nc == nx) {
      R.gEnd = __ldg(P.start + R.rb);
      R.lenEnd = __ldg(P.start + R.rb + kSlicesX) - R.gEnd;
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
  const int t0 = __ldg(P.start + rows[4].rb + kSlicesX * cx0);
  const int t1 = __ldg(P.start + rows[4].rb + kSlicesX * (cx0 + nc));
  if (!DPD_IN_BOUNDS(t0 >= 0 && t0 <= t1 && t1 <= P.ntot, P.err)) return;

  if (!staged) {
    // too many particles to stage: read neighbours from global memory
    for (int base = t0; base < t1; base += kTileThreads) {
      const int p = base + tid;
      force_direct<false, kTileThreads, kTileListCap>(P, B, S, p, p < t1, lst + tid);
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
      v = R.off + R.lenBeg + (__ldg(P.start + R.rb + kSlicesX * x) - R.gMain);
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
      if (!DPD_IN_BOUNDS(g >= 0 && g < P.ntot, P.err)) g = 0;
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
    int sx, cyy, czz;
    unpack_cell(__float_as_int(vi.w), sx, cyy, czz);
    int kt = sx / kSlicesX - cx0 + 1;  // virtual cell of the target, 1..nc
    if (alive && !DPD_IN_BOUNDS(kt >= 1 && kt <= nc, P.err)) kt = 1;
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
        float fr;
        if (B.noise == 0) {
          const uint32_t u = pair_word(idi, idj, slo, shi, B.seed_lo, B.seed_hi);
          fr = B.sig * wR * noise_int(u);
        } else {
          const uint2 u = pair_words(idi, idj, slo, shi, B.seed_lo, B.seed_hi);
          fr = B.sig_g * wR * gauss_xi(u.x, u.y);
        }
        const float fc = B.a * w;
        const float sc = (fr + fmaf(-B.gamma * wR * wR, ev, fc)) * rinv;
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
                                       cnt, kTileListCap);
          if (stop < 0) break;
          drain();
          j0 = stop + 1;
        }
        j0 = max(j0, jx);
        while (j0 < j1) {
          const int stop = scan_staged(sPos, j0, j1, pi.x - Lx, ay, az, rc2, R.ish | kCodeIX, my,
                                       kTileThreads, cnt, kTileListCap);
          if (stop < 0) break;
          drain();
          j0 = stop + 1;
        }
      }
      if (__any_sync(0xffffffffu, cnt > kTileListCap / 2)) drain();
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

// ================================================================ variants
// Direct-kernel variants: (threads per block, pair-list entries per thread).
struct VariantInfo {
  int threads, cap;
};
// Variants 7..9 use the balanced drain, 10..12 the spread drain (half
// stencil; with the full stencil they run the per-lane drain); 13 is the
// brick kernel staged through shared memory (half stencil; with the full
// stencil it runs variant 0).
static const VariantInfo kVariants[kNumForceVariants] = {
    {128, 24}, {128, 16}, {128, 32}, {256, 24}, {64, 24}, {64, 32}, {256, 32},
    {64, 24}, {128, 24}, {256, 24}, {64, 32}, {128, 32}, {128, 24},
    {kBrickThreads, kBrickListCap}};

int force_variant_info(int v, int *threads, int *cap) {
  if (v < 0 || v >= kNumForceVariants) return -1;
  *threads = kVariants[v].threads;
  *cap = kVariants[v].cap;
  return 0;
}

template <bool SINGLE, bool HALF, int NT, int CAP, bool BAL = false, bool GAUSS = false,
          bool SPREAD = false>
static void launch_k(const Packed &P, int s0, int s1, bool fuse, cudaStream_t s) {
  if (s1 > s0)
    k_force<SINGLE, HALF, NT, CAP, BAL, GAUSS, SPREAD && HALF>
        <<<blocks_for(s1 - s0, NT), NT, 0, s>>>(P, s0, s1, fuse);
}

template <bool SINGLE, bool HALF>
static void launch_variant(int v, bool gauss, const Packed &P, int s0, int s1, bool fuse,
                           cudaStream_t s) {
  if (gauss) {  // general kernels: bands holding Gaussian-noise or several-species boxes
    if constexpr (HALF)
      launch_k<SINGLE, HALF, 128, 24, false, true, true>(P, s0, s1, fuse, s);  // spread drain
    else
      launch_k<SINGLE, HALF, 128, 24, false, true>(P, s0, s1, fuse, s);
    return;
  }
  switch (v) {
    case 1: launch_k<SINGLE, HALF, 128, 16>(P, s0, s1, fuse, s); break;
    case 2: launch_k<SINGLE, HALF, 128, 32>(P, s0, s1, fuse, s); break;
    case 3: launch_k<SINGLE, HALF, 256, 24>(P, s0, s1, fuse, s); break;
    case 4: launch_k<SINGLE, HALF, 64, 24>(P, s0, s1, fuse, s); break;
    case 5: launch_k<SINGLE, HALF, 64, 32>(P, s0, s1, fuse, s); break;
    case 6: launch_k<SINGLE, HALF, 256, 32>(P, s0, s1, fuse, s); break;
    case 7: launch_k<SINGLE, HALF, 64, 24, true>(P, s0, s1, fuse, s); break;
    case 8: launch_k<SINGLE, HALF, 128, 24, true>(P, s0, s1, fuse, s); break;
    case 9: launch_k<SINGLE, HALF, 256, 24, true>(P, s0, s1, fuse, s); break;
    case 10: launch_k<SINGLE, HALF, 64, 32, false, false, true>(P, s0, s1, fuse, s); break;
    case 11: launch_k<SINGLE, HALF, 128, 32, false, false, true>(P, s0, s1, fuse, s); break;
    case 12: launch_k<SINGLE, HALF, 128, 24, false, false, true>(P, s0, s1, fuse, s); break;
    default: launch_k<SINGLE, HALF, 128, 24>(P, s0, s1, fuse, s); break;
  }
}

size_t tile_smem_bytes(int stage_cap) {
  return (size_t)stage_cap * 2 * sizeof(float4) +
         (size_t)kTileListCap * kTileThreads * sizeof(uint32_t);
}

cudaError_t prepare_device() {
  // staged tiles may use more than the default 48 KB of dynamic shared memory
  const int maxb = 200 * 1024;
  cudaError_t e = prepare_brick();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_force_tiles<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, maxb);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_force_tiles<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              maxb);
}

cudaError_t launch_force(const Packed &P, const StepConfig &cfg, cudaStream_t s, bool fuse) {
  const bool single = (P.nbox == 1);
  const bool half = (cfg.stencil == 1);
  if (fuse && half) return cudaErrorInvalidValue;  // the half stencil's forces end in atomics
  if (!half && cfg.tiles && cfg.grid.ntiles > 0) {
    if (fuse) return cudaErrorInvalidValue;  // the staged tiles store forces only
    const size_t smem = tile_smem_bytes(cfg.grid.stage_cap);
    if (single)
      k_force_tiles<true><<<cfg.grid.ntiles, kTileThreads, smem, s>>>(P, cfg.grid);
    else
      k_force_tiles<false><<<cfg.grid.ntiles, kTileThreads, smem, s>>>(P, cfg.grid);
    return cudaGetLastError();
  }
  ForceBand whole{0, P.ntot, 0, 0};
  const ForceBand *bands = cfg.nbands > 0 ? cfg.band : &whole;
  const int nb = cfg.nbands > 0 ? cfg.nbands : 1;
  for (int k = 0; k < nb; ++k) {
    const ForceBand &b = bands[k];
    if (half && !b.gauss && b.variant == kBrickVariant && cfg.nbands > 0 && cfg.bricks.items) {
      const cudaError_t e = launch_force_brick(P, cfg.bricks, b.item0, b.item1, s);
      if (e != cudaSuccess) return e;
      continue;
    }
    if (!single && cfg.grouped && cfg.hboxes && cfg.nbands > 0 &&
        grouped_variant(b.variant, b.gauss != 0, half)) {
      // box-grouped launches: no warp spans two boxes
      const cudaError_t e = launch_force_group(P, cfg.hboxes, b.box0, b.box1, b.variant, s);
      if (e != cudaSuccess) return e;
      continue;
    }
    if (single) {
      if (half)
        launch_variant<true, true>(b.variant, b.gauss, P, b.slot0, b.slot1, false, s);
      else
        launch_variant<true, false>(b.variant, b.gauss, P, b.slot0, b.slot1, fuse, s);
    } else {
      if (half)
        launch_variant<false, true>(b.variant, b.gauss, P, b.slot0, b.slot1, false, s);
      else
        launch_variant<false, false>(b.variant, b.gauss, P, b.slot0, b.slot1, fuse, s);
      // the band's two-box warps, skipped by the warp-cooperative kernels
      if (cfg.nbands > 0 && b.mw_count > 0 && cfg.mixed_warps &&
          cooperative_variant(b.variant, b.gauss != 0, half)) {
        const int *ws = cfg.mixed_warps + b.mw_off;
        if (half) {
          if (b.gauss)
            k_force_warps<true, 24, true><<<b.mw_count, 32, 0, s>>>(P, ws, b.slot1, false);
          else
            k_force_warps<true, 24, false><<<b.mw_count, 32, 0, s>>>(P, ws, b.slot1, false);
        } else {
          k_force_warps<false, 24, false><<<b.mw_count, 32, 0, s>>>(P, ws, b.slot1, fuse);
        }
      }
    }
  }
  return cudaGetLastError();
}

// ============================================================ tuning table
// Process-wide maps from density band to direct-kernel variant: table
// stencil + 2 * packed, i.e. 0/1 for a single box (full/half stencil) and
// 2/3 for packed sets of several boxes (whose kernels look up each lane's
// box and differ in register use).  A packed table that was never set
// falls back to the single-box table of its stencil.  Bands are given by
// increasing upper bounds of rho (particles per rc^3); densities above the
// last bound use the last band.
namespace {
struct Tuning {
  std::vector<double> upper;
  std::vector<int> variant;
};
std::mutex g_tune_mu;
Tuning g_tune[4] = {{{1e30}, {0}}, {{1e30}, {0}}, {}, {}};

const Tuning &effective(int table) {  // g_tune_mu held
  return g_tune[table].upper.empty() ? g_tune[table & 1] : g_tune[table];
}
}  // namespace

int tuning_set(int table, int n, const double *upper, const int *variant) {
  if (table < 0 || table > 3 || n < 1 || n > kMaxBands) return -1;
  for (int k = 0; k < n; ++k) {
    if (variant[k] < 0 || variant[k] >= kNumForceVariants) return -1;
    if (k > 0 && !(upper[k] > upper[k - 1])) return -1;
  }
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune[table].upper.assign(upper, upper + n);
  g_tune[table].variant.assign(variant, variant + n);
  return 0;
}

int tuning_get(int table, int max, double *upper, int *variant) {
  if (table < 0 || table > 3) return -1;
  std::lock_guard<std::mutex> g(g_tune_mu);
  const Tuning &t = effective(table);
  const int n = (int)t.upper.size();
  for (int k = 0; k < n && k < max; ++k) {
    if (upper) upper[k] = t.upper[k];
    if (variant) variant[k] = t.variant[k];
  }
  return n;
}

int tuned_band(int table, double rho) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  const Tuning &t = effective(table & 3);
  for (size_t k = 0; k < t.upper.size(); ++k)
    if (rho <= t.upper[k]) return (int)k;
  return (int)t.upper.size() - 1;
}

int tuned_variant(int table, double rho) {
  const int band = tuned_band(table, rho);
  std::lock_guard<std::mutex> g(g_tune_mu);
  return effective(table & 3).variant[band];
}

}  // namespace dpd
