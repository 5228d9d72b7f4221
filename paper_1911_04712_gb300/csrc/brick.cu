// Brick force kernel of the DPD step (half stencil): pair forces of Eqs. 2-5
// over the cell list of Sec. 3.2, with Newton's third law, staged through
// shared memory.
//
// A thread block owns a brick of target cells: by x bz rows (y, z) of one
// box and a range of x slices.  It walks the range in chunks of w slices.
// For a chunk it copies, from the cell-ordered global arrays, every
// particle the chunk's targets can pair with under the half stencil into
// shared memory: rows y0-1 .. y0+by of the planes z0 .. z0+bz, slices
// s-2 .. s+w+1 (the two slices on each side hold every neighbour within rc
// of a target, since a slice is at least rc/2 wide), positions, velocities
// and a zeroed force accumulator per staged particle.  The width w is the
// largest (up to kBrickWMax) whose staged particles fit the capacity; where
// even one slice does not fit, the brick is split into single rows.
//
// Each warp then takes 32 targets at a time.  Every lane scans its target's
// five stencil rows -- the own row forward from the target, the row dy = +1
// of its plane and the three rows dy = -1, 0, +1 of the plane above, each
// over the slices sl-2 .. sl+2 -- and appends the staged index of every
// candidate with 0 < r^2 < rc^2 to its own list.  A drain spreads the warp's
// list entries evenly over the lanes (each lane a run of consecutive
// entries, so a run mostly stays with one owner): the pair force of Eqs. 3-5
// is added to the owner's register sum, which goes to its accumulator when
// the owner changes, and -F_ij goes to j's accumulator by a shared-memory
// atomic.  Finally every staged accumulator is added to the global force
// array (zeroed by the reorder) with one vector atomic per particle.
//
// Periodic images: a row or slices wrapped below the box (logical index -1,
// -2) are stored shifted by -L, which is exact in FP32 (the coordinate lies
// in [L/2, L)).  An image above the box (logical index n, n+1) is stored
// unshifted and flagged in the staged velocity's w word; a target pairing
// with it is taken at r_i - L on that axis (exact for the same reason).
#include <cuda_runtime.h>

#include <cstdint>

#include "dpd_device.cuh"
#include "kernels.h"

namespace dpd {

namespace {

constexpr int kBT = kBrickThreads;
constexpr int kBW = kBT / 32;                 // warps per block
constexpr int kCols = kBrickWMax + 5;         // slice starts per staged row (w + 4 slices)
constexpr int kLCap = kBrickListCap;          // list entries per lane
constexpr int kU = 4;                         // candidates per scan iteration
constexpr uint32_t kHiX = 1u, kHiY = 2u, kHiZ = 4u;  // image-above flags

// One staged row of a chunk.
struct SRow {
  int g;          // start[] index of the row's slice 0: cellBase + (z ny + y) nx
  float sy, sz;   // pre-shift subtracted from stored y / z
  uint32_t hi;    // kHiY / kHiZ when the row is an image above the box
  int off;        // first staged index of the row
  int gseg[3];    // first global slot of the low-wrap, main and high-wrap slices
};

struct BrickShared {
  SRow rows[kBrickMaxRows];
  int tpre[kBrickMaxBY * kBrickMaxBZ + 1];  // target-row prefix of target counts
  int off[kBW][33];                         // drain: list offsets of each warp's lanes
  int own[kBT];                             // each thread's current target (staged index)
  int tot[32];                              // staged particles of a chunk of width w + 1
  int w, ntarget, next, tl, th;
};

__device__ __forceinline__ bool in_rc(float r2, uint32_t rc2m1) {
  return (__float_as_uint(r2) - 1u) < rc2m1;  // 0 < r2 < rc2 on the bit patterns
}

template <bool SINGLE>
struct Brick {
  const Packed &P;
  const BoxDev &B;
  BrickShared &S;
  float4 *sPos, *sVel;             // staged positions (id in w) and velocities (image flags in w)
  float *sX, *sY, *sZ;             // the positions again as separate arrays, for the scan
  float *sFx, *sFy, *sFz, *sFw;    // force accumulators (w: r . F^C)
  int *sCnt;        // [row][kCols]: row-relative start of each staged slice
  uint16_t *sList;  // [entry][thread]
  int caps;         // staged capacity
  uint32_t slo, shi;

  // Pair force of Eq. 2's summand for target (pi, vi) and staged neighbour j:
  // F_ij and r . F^C (Eqs. 3-5, sigma^2 = 2 gamma kT, w_D = w_R^2).
  __device__ __forceinline__ float4 pair(const float4 &pi, const float4 &vi, const float4 &pj,
                                         const float4 &vj, bool any_hi) const {
    float ax = pi.x, ay = pi.y, az = pi.z;
    if (any_hi) {
      const uint32_t fl = __float_as_uint(vj.w);
      if (fl) {
        if (fl & kHiX) ax -= B.L[0];
        if (fl & kHiY) ay -= B.L[1];
        if (fl & kHiZ) az -= B.L[2];
      }
    }
    const float dx = ax - pj.x, dy = ay - pj.y, dz = az - pj.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    const float w = fmaxf(fmaf(-r, B.inv_rc, 1.0f), 0.0f);
    const float wR = (B.kexp == 1.0f) ? w : powf(w, B.kexp);
    const float ev = fmaf(dx, vi.x - vj.x, fmaf(dy, vi.y - vj.y, dz * (vi.z - vj.z))) * rinv;
    const uint32_t u = pair_word(__float_as_uint(pi.w), __float_as_uint(pj.w), slo, shi,
                                 B.seed_lo, B.seed_hi);
    const float fr = B.sig * wR * noise_int(u);
    const float fc = B.a * w;
    const float s = (fr + fmaf(-B.gamma * wR * wR, ev, fc)) * rinv;
    return make_float4(__fmul_rn(s, dx), __fmul_rn(s, dy), __fmul_rn(s, dz), __fmul_rn(fc, r));
  }

  // Process target rows (y0 .. y0+by-1, z0 .. z0+bz-1), slices [sA, sB).
  // Returns sB when done, or the first slice whose single-slice chunk does
  // not fit the staging capacity.
  __device__ int range(int y0, int by, int z0, int bz, int sA, int sB) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
    const int nrows = (by + 2) * (bz + 1);
    const int ntr = by * bz;
    for (int s = sA; s < sB;) {
      const int wcap = min(kBrickWMax, sB - s);
      const int nt = wcap + 4;  // staged slices at the widest chunk
      // 1. a warp per staged row: row geometry, particles per staged slice
      //    (a warp scan gives the row-relative slice starts), the row's
      //    staged count for every chunk width (summed over rows by shared
      //    atomics), and its first global slots
      for (int R = warp; R < nrows; R += kBW) {
        const int ly = R % (by + 2), lz = R / (by + 2);
        int y = y0 - 1 + ly, z = z0 + lz;
        float sy = 0.f;
        uint32_t hi = 0u;
        if (y < 0) {
          y += ny;
          sy = B.L[1];
        } else if (y >= ny) {
          y -= ny;
          hi |= kHiY;
        }
        if (z >= nz) {
          z -= nz;
          hi |= kHiZ;
        }
        const int g = B.cellBase + (z * ny + y) * nx;
        int run = 0;
        for (int t0 = 0; t0 < nt; t0 += 32) {
          const int t = t0 + lane;
          int c = 0;
          if (t < nt) {
            int xg = s - 2 + t;
            xg += (xg < 0) ? nx : ((xg >= nx) ? -nx : 0);
            if (DPD_IN_BOUNDS(g + xg >= 0 && g + xg < P.ncell, P.err))
              c = __ldg(P.start + g + xg + 1) - __ldg(P.start + g + xg);
          }
          int incl = c;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
          }
          if (t < nt) sCnt[R * kCols + t + 1] = run + incl;
          run += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) {
          sCnt[R * kCols] = 0;
          SRow &Rw = S.rows[R];
          Rw.g = g;
          Rw.sy = sy;
          Rw.sz = 0.f;
          Rw.hi = hi;
          // first global slots: low-wrap slices (logical s-2 .. -1 at nx+s-2 ..),
          // main slices from max(s-2, 0), high-wrap slices from 0
          Rw.gseg[0] = __ldg(P.start + g + min(max(nx + s - 2, 0), nx));
          Rw.gseg[1] = __ldg(P.start + g + max(s - 2, 0));
          Rw.gseg[2] = __ldg(P.start + g);
        }
        __syncwarp();
        if (lane < wcap) atomicAdd(&S.tot[lane], sCnt[R * kCols + lane + 5]);
      }
      if (tid == 0) {
        S.tl = max(2 - s, 0);                // staged slices below the box: t < tl
        S.th = min(nx - (s - 2), nt);        // staged slices above the box: t >= th
      }
      __syncthreads();
      // 2. the widest chunk that fits (staged counts grow with w), row
      //    offsets and the target rows' prefix, by warp scans
      if (warp == 0) {
        const unsigned ok = __ballot_sync(0xffffffffu, lane < wcap && S.tot[lane] <= caps);
        const int w = __popc(ok);
        int v = (w > 0 && lane < nrows) ? sCnt[lane * kCols + w + 4] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int u = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += u;
        }
        if (lane < nrows) S.rows[lane].off = incl - v;
        int tc = 0;
        if (w > 0 && lane < ntr) {
          const int R = (lane / by) * (by + 2) + 1 + lane % by;
          tc = sCnt[R * kCols + w + 2] - sCnt[R * kCols + 2];
        }
        int tin = tc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int u = __shfl_up_sync(0xffffffffu, tin, o);
          if (lane >= o) tin += u;
        }
        if (lane <= ntr) S.tpre[lane] = tin - tc;  // tpre[ntr] = the total
        const int ttot = __shfl_sync(0xffffffffu, tin, 31);
        if (lane == 0) {
          S.w = w;
          S.ntarget = ttot;
          S.next = 0;
          S.th = min(S.th, w + 4);
        }
      }
      __syncthreads();
      const int w = S.w;
      if (w == 0) {  // block-uniform: not even one slice fits
        if (tid < 32) S.tot[tid] = 0;
        __syncthreads();
        return s;
      }
      const int tl = S.tl, th = S.th;
      const bool any_hi = (th < w + 4) || (y0 - 1 + by + 1 >= ny) || (z0 + bz >= nz);
      // 6. stage the chunk: a warp per row
      for (int R = warp; R < nrows; R += kBW) {
        const SRow &Rw = S.rows[R];
        const int l1 = sCnt[R * kCols + tl], l2 = sCnt[R * kCols + th], n = sCnt[R * kCols + w + 4];
        for (int k = lane; k < n; k += 32) {
          int gk;
          uint32_t fl = Rw.hi;
          float sx = 0.f;
          if (k < l1) {
            gk = Rw.gseg[0] + k;
            sx = B.L[0];
          } else if (k < l2) {
            gk = Rw.gseg[1] + (k - l1);
          } else {
            gk = Rw.gseg[2] + (k - l2);
            fl |= kHiX;
          }
          const int d = Rw.off + k;
          if (!DPD_IN_BOUNDS(gk >= 0 && gk < P.ntot && d < caps, P.err)) continue;
          float4 p = P.pos[gk];
          float4 v = P.vel[gk];
          p.x -= sx;
          p.y -= Rw.sy;
          p.z -= Rw.sz;
          v.w = __uint_as_float(fl);
          sPos[d] = p;
          sVel[d] = v;
          sX[d] = p.x;
          sY[d] = p.y;
          sZ[d] = p.z;
          sFx[d] = 0.f;
          sFy[d] = 0.f;
          sFz[d] = 0.f;
          sFw[d] = 0.f;
        }
      }
      __syncthreads();
      // 7. targets, 32 per warp at a time
      const int T = S.ntarget;
      const uint32_t rc2m1 = __float_as_uint(B.rc2) - 1u;
      for (;;) {
        int grp = 0;
        if (lane == 0) grp = atomicAdd(&S.next, 1);
        grp = __shfl_sync(0xffffffffu, grp, 0);
        if (grp * 32 >= T) break;
        const int t = grp * 32 + lane;
        const bool alive = t < T;
        int q = 0, R0 = 0, ly = 1, lz = 0, sl = 2;
        float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
        if (alive) {
          int k = 0;
          while (k + 1 < ntr && S.tpre[k + 1] <= t) ++k;
          ly = 1 + k % by;
          lz = k / by;
          R0 = lz * (by + 2) + ly;
          q = S.rows[R0].off + sCnt[R0 * kCols + 2] + (t - S.tpre[k]);
          pi = sPos[q];
          sl = cell_axis(pi.x, B.invh[0], nx) - (s - 2);
          sl = min(max(sl, 2), w + 1);
        }
        S.own[tid] = q;
        int cnt = 0;
        uint16_t *my = sList + tid;

        // Drain: the warp's entries spread evenly over the lanes, each lane a
        // run of consecutive entries (owner-sorted); F_ij to the owner's
        // register sum, -F_ij to j by a shared-memory atomic.
        auto drain = [&]() {
          int incl = cnt;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
          }
          const int total = __shfl_sync(0xffffffffu, incl, 31);
          if (total == 0) return;
          int *off = S.off[warp];
          off[lane] = incl - cnt;
          if (lane == 31) off[32] = total;
          __syncwarp();
          const int K = (total + 31) >> 5;
          int g = lane * K;
          const int gend = min(g + K, total);
          int o = 0;
#pragma unroll
          for (int st = 16; st >= 1; st >>= 1)
            if (off[o + st] <= g) o += st;
          int obeg = off[o], onext = off[o + 1];
          int qi = S.own[warp * 32 + o];
          float4 ppi = sPos[qi], pvi = sVel[qi];
          float fx = 0.f, fy = 0.f, fz = 0.f, fw = 0.f;
          for (int k = 0; k < K; ++k) {
            if (g < gend) {
              if (g >= onext) {
                atomicAdd(sFx + qi, fx);
                atomicAdd(sFy + qi, fy);
                atomicAdd(sFz + qi, fz);
                atomicAdd(sFw + qi, fw);
                fx = fy = fz = fw = 0.f;
                do {
                  ++o;
                  obeg = onext;
                  onext = off[o + 1];
                } while (g >= onext);
                qi = S.own[warp * 32 + o];
                ppi = sPos[qi];
                pvi = sVel[qi];
              }
              const int jj = (int)sList[(g - obeg) * kBT + warp * 32 + o];
              const float4 pj = sPos[jj], vj = sVel[jj];
              const float4 f = pair(ppi, pvi, pj, vj, any_hi);
              fx += f.x;
              fy += f.y;
              fz += f.z;
              fw += f.w + f.w;  // both members' share of r . F^C on the owner
              atomicAdd(sFx + jj, -f.x);
              atomicAdd(sFy + jj, -f.y);
              atomicAdd(sFz + jj, -f.z);
              ++g;
            }
          }
          if (lane * K < total) {
            atomicAdd(sFx + qi, fx);
            atomicAdd(sFy + qi, fy);
            atomicAdd(sFz + qi, fz);
            atomicAdd(sFw + qi, fw);
          }
          __syncwarp();
          cnt = 0;
        };

        // Candidates [j, j1) against (ax, ay, az); stops early when the
        // list is nearly full.
        auto scan = [&](int &j, int j1, float ax, float ay, float az) {
          while (j < j1) {
            float4 c[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
              const int k = min(j + u, j1 - 1);
              c[u] = make_float4(sX[k], sY[k], sZ[k], 0.f);
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
              const float dx = ax - c[u].x, dy = ay - c[u].y, dz = az - c[u].z;
              const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
              my[cnt * kBT] = (uint16_t)(j + u);
              cnt += (j + u < j1 && in_rc(r2, rc2m1)) ? 1 : 0;
            }
            j += kU;
            if (cnt > kLCap - kU) return;
          }
        };

        // Rows of the half stencil in a warp-uniform loop: own row (forward
        // from the target), dy = +1 of its plane, dy = -1, 0, +1 of the plane
        // above; one drain point (lists nearly full, or after the last row).
        int r = -1, ca = 0, cb = 0, jm = 0, jb = 0;
        float ay = 0.f, az = 0.f;
        bool row_done = true;
        for (;;) {
          if (row_done) {
            if (++r == 5) break;
            const int dly = (r == 0) ? 0 : (r == 1 ? 1 : r - 3);
            const int dlz = (r < 2) ? 0 : 1;
            const int R = (lz + dlz) * (by + 2) + (ly + dly);
            const SRow &Rw = S.rows[R];
            const int base = Rw.off;
            ca = (r == 0) ? q + 1 : base + sCnt[R * kCols + sl - 2];
            jb = base + sCnt[R * kCols + sl + 3];
            jm = (th < sl + 3) ? base + sCnt[R * kCols + max(th, sl - 2)] : jb;
            cb = jm;
            ay = (Rw.hi & kHiY) ? pi.y - B.L[1] : pi.y;
            az = (Rw.hi & kHiZ) ? pi.z - B.L[2] : pi.z;
          }
          if (alive) {
            if (ca < jm) scan(ca, jm, pi.x, ay, az);
            if (ca >= jm && cnt <= kLCap - kU && cb < jb) scan(cb, jb, pi.x - B.L[0], ay, az);
          }
          row_done = !__any_sync(0xffffffffu, alive && (ca < jm || cb < jb));
          if (__any_sync(0xffffffffu, cnt > kLCap - kU) || (row_done && r == 4)) drain();
        }
        if (alive && B.fb_mode != 0) {  // body force (Sec. 4.2 periodic Poiseuille, or constant)
          float add = B.fb;
          if (B.fb_mode == 2) {
            const float xg = (B.fb_grad == 0) ? pi.x : (B.fb_grad == 1) ? pi.y : pi.z;
            add = (xg <= B.fb_half) ? -B.fb : B.fb;
          }
          float *fp = ((B.fb_flow == 0) ? sFx : (B.fb_flow == 1) ? sFy : sFz) + q;
          atomicAdd(fp, add);
        }
      }
      __syncthreads();
      // 8. add the staged accumulators to the global forces
      if (tid < 32) S.tot[tid] = 0;
      for (int R = warp; R < nrows; R += kBW) {
        const SRow &Rw = S.rows[R];
        const int l1 = sCnt[R * kCols + tl], l2 = sCnt[R * kCols + th], n = sCnt[R * kCols + w + 4];
        for (int k = lane; k < n; k += 32) {
          const int gk = (k < l1) ? Rw.gseg[0] + k
                                  : ((k < l2) ? Rw.gseg[1] + (k - l1) : Rw.gseg[2] + (k - l2));
          const int d = Rw.off + k;
          const float4 f = make_float4(sFx[d], sFy[d], sFz[d], sFw[d]);
          if ((f.x != 0.f || f.y != 0.f || f.z != 0.f || f.w != 0.f) &&
              DPD_IN_BOUNDS(gk >= 0 && gk < P.ntot, P.err))
            atomicAdd(P.frc + gk, f);
        }
      }
      __syncthreads();
      s += w;
    }
    return sB;
  }
};

// One block per work item {box, y0 | by << 16, z0 | bz << 16, s0 | s1 << 16}.
template <bool SINGLE>
__global__ void __launch_bounds__(kBT, 3) k_force_brick(Packed P, const int4 *__restrict__ items,
                                                     int caps) {
  extern __shared__ float4 brick_smem[];
  __shared__ BrickShared S;
  const int4 it = items[blockIdx.x];
  const int b = it.x;
  if (threadIdx.x < 32) S.tot[threadIdx.x] = 0;
  __syncthreads();
  const BoxState st = P.st[b];
  if (!st.adv) return;  // block-uniform
  const BoxDev &B = SINGLE ? P.single : P.boxes[b];
  Brick<SINGLE> K{P, B, S};
  K.sPos = brick_smem;
  K.sVel = K.sPos + caps;
  K.sX = reinterpret_cast<float *>(K.sVel + caps);
  K.sY = K.sX + caps;
  K.sZ = K.sY + caps;
  K.sFx = K.sZ + caps;
  K.sFy = K.sFx + caps;
  K.sFz = K.sFy + caps;
  K.sFw = K.sFz + caps;
  K.sCnt = reinterpret_cast<int *>(K.sFw + caps);
  K.sList = reinterpret_cast<uint16_t *>(K.sCnt + kBrickMaxRows * kCols);
  K.caps = caps;
  K.slo = (uint32_t)st.step;
  K.shi = (uint32_t)(st.step >> 32);
  const int y0 = it.y & 0xFFFF, by = it.y >> 16, z0 = it.z & 0xFFFF, bz = it.z >> 16;
  const int s0 = it.w & 0xFFFF, s1 = it.w >> 16;
  const int sf = K.range(y0, by, z0, bz, s0, s1);
  if (sf < s1) {
    // even one slice of the whole brick does not fit: single rows from there
    for (int k = 0; k < by * bz; ++k) {
      const int s2 = K.range(y0 + k % by, 1, z0 + k / by, 1, sf, s1);
      if (s2 < s1 && threadIdx.x == 0) atomicOr(P.err, kErrCapacity);
    }
  }
}

}  // namespace

size_t brick_smem_bytes(int caps) {
  return (size_t)caps * (2 * sizeof(float4) + 7 * sizeof(float)) +
         (size_t)kBrickMaxRows * kCols * sizeof(int) +
         (size_t)kLCap * kBT * sizeof(uint16_t);
}

cudaError_t prepare_brick() {
  const int maxb = (int)brick_smem_bytes(kBrickMaxCaps);
  cudaError_t e =
      cudaFuncSetAttribute(k_force_brick<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_force_brick<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              maxb);
}

cudaError_t launch_force_brick(const Packed &P, const BrickGrid &G, int i0, int i1,
                               cudaStream_t s) {
  if (i1 <= i0) return cudaSuccess;
  const size_t smem = brick_smem_bytes(G.caps);
  if (P.nbox == 1)
    k_force_brick<true><<<i1 - i0, kBT, smem, s>>>(P, G.items + i0, G.caps);
  else
    k_force_brick<false><<<i1 - i0, kBT, smem, s>>>(P, G.items + i0, G.caps);
  return cudaGetLastError();
}

}  // namespace dpd
