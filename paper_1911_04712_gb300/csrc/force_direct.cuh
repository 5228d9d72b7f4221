// The direct force routine shared by the force kernels (force.cu) and the
// box-grouped packed launches (group.cu): pair forces (Sec. 2.1, Eqs. 2-5)
// on one target particle over the cell list (Sec. 3.2), through a
// per-thread pair list in shared memory.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "dpd_device.cuh"
#include "kernels.h"

namespace dpd {

// Candidates loaded per iteration of the candidate pass.
constexpr int kScanUnroll = 4;

// ------------------------------------------------------------------ force
// Pair lists: each thread appends the neighbours found inside rc to its own
// column of a shared-memory list (entry k of thread t at lst[k * NT + t], NT threads),
// then drains the list computing the pair forces.  An entry is 4 bytes: the
// neighbour slot j (26 bits) and the periodic-image code of the pair:
//   bit 26/28/30  the neighbour image is r_j - L on x/y/z (j near the top face)
//   bit 27/29/31  i is taken at r_i - L on x/y/z (i near the top face)
// Both subtractions are exact in FP32 (the shifted coordinate lies in
// [2L/3, L)), so no rounding error of size ulp(L) enters r_ij.
constexpr uint32_t kSlotMask = (1u << 26) - 1u;
constexpr uint32_t kCodeJX = 1u << 26, kCodeIX = 1u << 27, kCodeJY = 1u << 28,
                   kCodeIY = 1u << 29, kCodeJZ = 1u << 30, kCodeIZ = 1u << 31;

// 0 < r2 < rc2 as one unsigned compare of the bit patterns (both are
// non-negative floats, whose bit patterns order like their values).
__device__ __forceinline__ bool in_range(float r2, uint32_t rc2_bits_minus_1) {
  return (__float_as_uint(r2) - 1u) < rc2_bits_minus_1;
}

// Candidate pass over slots [j0, j1): appends every j with 0 < r_ij^2 < rc^2.
// The append is branch-free (the slot is written every candidate and kept
// only on a hit), so the lanes of a warp stay converged; U candidates are
// loaded per iteration (the last iteration masked).  Needs at least U free
// list entries on entry.  Returns the next slot to scan (possibly >= j1) when
// the list has fewer than U free entries, or -1 when the range was scanned
// completely.
template <bool JSHIFT, int LS, int CAP, int U>
__device__ __forceinline__ int scan_range(const float4 *__restrict__ pos, int j0, int j1,
                                          float ax, float ay, float az, float jsx, float jsy,
                                          float jsz, uint32_t rc2m1, uint32_t code,
                                          uint32_t *__restrict__ lst, int &cnt) {
  for (int j = j0; j < j1; j += U) {
    float4 q[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      q[u] = (u == 0 || j + u < j1) ? __ldg(pos + j + u) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      float dx, dy, dz;
      if constexpr (JSHIFT) {
        dx = ax - (q[u].x - jsx);
        dy = ay - (q[u].y - jsy);
        dz = az - (q[u].z - jsz);
      } else {
        dx = ax - q[u].x;
        dy = ay - q[u].y;
        dz = az - q[u].z;
      }
      const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      lst[cnt * LS] = (uint32_t)(j + u) | code;
      cnt += ((u == 0 || j + u < j1) && in_range(r2, rc2m1)) ? 1 : 0;
    }
    if (cnt > CAP - U) return j + U;
  }
  return -1;
}

// Per-warp scratch of the balanced drain.  List of lane l: list[l * (CAP+1) + k].
template <int CAP>
struct WarpScratch {
  uint32_t list[32 * (CAP + 1)];
  float4 own_pos[32];   // each lane's target position (w: id bits)
  float4 own_vel[32];
  float4 res[32];       // pair results of the chunk being processed
  int start[32];        // lane whose list starts at this chunk position, or -1
};

// Force on one target particle in slot p from the 27-cell (full) or 13-cell
// + own-cell (half) neighbourhood, each row scanned over the x slices within
// rc of the particle, reading neighbours from global memory.  Every lane of
// the warp must call this (dead lanes with alive = false): the rows are
// walked in a warp-uniform loop and the lists are drained at a single
// warp-uniform point, when a list is nearly full or after a row once any
// lane holds more than FLUSH entries.  BX is the type holding the box
// constants: BoxDev, or the compact BoxHot of a grouped launch (uniform
// noise, one species, half stencil).
template <bool HALF, int NT, int CAP, bool BAL = false, bool GAUSS = false, bool SPREAD = false,
          typename BX = BoxDev>
__device__ __forceinline__ void force_direct(const Packed &P, const BX &B, const BoxState &S,
                                             int p, bool alive, uint32_t *__restrict__ lst,
                                             WarpScratch<CAP> *W = nullptr,
                                             float4 *__restrict__ own = nullptr,
                                             bool mixed = false, bool fuse = false,
                                             bool real = false) {
  static_assert(!SPREAD || (HALF && !BAL), "the spread drain serves the half stencil");
  static_assert(CAP >= 4, "list too short");
  // lists are drained after a row once a lane holds more than FLUSH
  // entries: a quarter of the list for the spread drain (draining a row's
  // entries together keeps the neighbours each round gathers in few cache
  // lines), half for the per-lane drains (whose lanes idle on short lists)
  constexpr int FLUSH = SPREAD ? CAP / 4 : CAP / 2;
  constexpr int U = kScanUnroll;
  constexpr int LS = BAL ? 1 : NT;  // list stride: own row of the warp scratch, or a column
  float4 pi = make_float4(0.f, 0.f, 0.f, 0.f), vi = pi;
  if (alive && !DPD_IN_BOUNDS(p >= 0 && p < P.ntot, P.err)) alive = false;
  if (alive) {
    pi = P.pos[p];
    vi = P.vel[p];
  }
  int cx, cy, cz;
  unpack_cell(__float_as_int(vi.w), cx, cy, cz);
  const uint32_t idi = __float_as_uint(pi.w);
  const uint32_t slo = (uint32_t)S.step, shi = (uint32_t)(S.step >> 32);
  const float Lx = B.L[0], Ly = B.L[1], Lz = B.L[2];
  const int nx = B.n[0], ny = B.n[1], nz = B.n[2];  // nx: x slices
  // x window of every row: the slices xlo .. xhi hold every neighbour with
  // |x_j - x_i| < rc (the margin makes it conservative)
  const int xlo = __float2int_rd((pi.x - B.xwin) * B.invh[0]);
  const int xhi = __float2int_rd((pi.x + B.xwin) * B.invh[0]);
  const uint32_t rc2m1 = __float_as_uint(B.rc2) - 1u;
  const bool k_is_one = (B.kexp == 1.0f);
  if constexpr (SPREAD) {
    own[threadIdx.x & 31] = pi;  // w: id bits
    own[32 + (threadIdx.x & 31)] = vi;
  }

  float fx = 0.f, fy = 0.f, fz = 0.f, vir = 0.f;
  int cnt = 0;

  // Pair force of one list entry for a target at (qi, ui): F_ij (3) and r . F^C.
  auto pair_at = [&](uint32_t e, const float4 &pj, const float4 &vj, const float4 &qi,
                     const float4 &ui) -> float4 {
    const int j = (int)(e & kSlotMask);
    float dx, dy, dz;
    if (e & ~kSlotMask) {  // pair across a box face (rare)
      dx = ((e & kCodeIX) ? qi.x - Lx : qi.x) - ((e & kCodeJX) ? pj.x - Lx : pj.x);
      dy = ((e & kCodeIY) ? qi.y - Ly : qi.y) - ((e & kCodeJY) ? pj.y - Ly : pj.y);
      dz = ((e & kCodeIZ) ? qi.z - Lz : qi.z) - ((e & kCodeJZ) ? pj.z - Lz : pj.z);
    } else {
      dx = qi.x - pj.x;
      dy = qi.y - pj.y;
      dz = qi.z - pj.z;
    }
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    // interaction parameters; the general kernels also serve boxes of
    // several species, whose pair of species picks them (and a cut-off
    // rc_st <= rc that the pair must be inside)
    float pa = B.a, pgam = B.gamma, psig = B.sig, psig_g = 0.f, pinv_rc = B.inv_rc;
    uint32_t idi_ = __float_as_uint(qi.w), idj_ = __float_as_uint(pj.w);
    if constexpr (GAUSS) {
      psig_g = B.sig_g;
      if (B.nspec > 1) {
        const int k = (int)((idi_ >> kSpeciesShift) * kMaxSpecies + (idj_ >> kSpeciesShift));
        if (!(r2 < B.sp_rc2[k])) return make_float4(0.f, 0.f, 0.f, 0.f);
        pa = B.sp_a[k];
        pgam = B.sp_gamma[k];
        psig = B.sp_sig[k];
        psig_g = B.sp_sig_g[k];
        pinv_rc = B.sp_inv_rc[k];
      }
      idi_ &= kIdMask;  // the pair noise takes the ids alone
      idj_ &= kIdMask;
    }
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    const float w = fmaxf(fmaf(-r, pinv_rc, 1.0f), 0.0f);
    const float wR = k_is_one ? w : powf(w, B.kexp);
    const float ev = fmaf(dx, ui.x - vj.x, fmaf(dy, ui.y - vj.y, dz * (ui.z - vj.z))) * rinv;
    float fr;  // random term sigma w_R xi / sqrt(dt)
    if constexpr (GAUSS) {  // general kernels: Gaussian noise or several species
      const uint2 u = pair_words(idi_, idj_, slo, shi, B.seed_lo, B.seed_hi);
      if (B.noise == 0)
        fr = psig * wR * noise_int(u.x);
      else
        fr = psig_g * wR * gauss_xi(u.x, u.y);
    } else {
      const uint32_t u = pair_word(idi_, idj_, slo, shi, B.seed_lo, B.seed_hi);
      fr = psig * wR * noise_int(u);
    }
    const float fc = pa * w;
    const float s = (fr + fmaf(-pgam * wR * wR, ev, fc)) * rinv;
    // rounded products (no fusion into the caller's sums), so that every
    // drain order-preserving variant adds exactly the same terms
    const float4 g = make_float4(__fmul_rn(s, dx), __fmul_rn(s, dy), __fmul_rn(s, dz),
                                 __fmul_rn(fc, r));
    if constexpr (HALF) atomicAdd(P.frc + j, make_float4(-g.x, -g.y, -g.z, g.w));
    return g;
  };
  auto pair = [&](uint32_t e, const float4 &qi, const float4 &ui) -> float4 {
    const int j = (int)(e & kSlotMask);
    if (!DPD_IN_BOUNDS(j < P.ntot, P.err)) return make_float4(0.f, 0.f, 0.f, 0.f);
    return pair_at(e, __ldg(P.pos + j), __ldg(P.vel + j), qi, ui);
  };

  // Balanced drain.  Every lane first evaluates its own entries below M,
  // the warp's mean list length (rounded down), in list order.  The entries
  // beyond M of the longer lists are then processed 32 at a time, one per
  // lane whatever lane owns them, through the warp scratch, and each owner
  // adds those results after its own, again in list order.  So every
  // particle's sum has the order of the per-lane drain (the same bits),
  // while the lanes idle only on the short lists' shortfall below M.
  auto drain_balanced = [&]() {
    const int lane = threadIdx.x & 31;
    int all = cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) all += __shfl_xor_sync(0xffffffffu, all, o);
    if (all == 0) return;
    const int M = all >> 5;
    if (!DPD_IN_BOUNDS(cnt <= CAP, P.err)) cnt = 0;
    const int ov = max(cnt - M, 0);  // this lane's entries M .. cnt - 1
    int incl = ov;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int off = incl - ov;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    W->own_pos[lane] = make_float4(pi.x, pi.y, pi.z, __uint_as_float(idi));
    W->own_vel[lane] = vi;
    // steps 0 .. M-1: own entries; then one step per chunk of 32 shared entries
    const int nsteps = M + (total + 31) / 32;
    int carry = 0;
    for (int t = 0; t < nsteps; ++t) {
      const bool own_step = t < M;  // warp-uniform
      uint32_t e = 0;
      int who = lane;
      bool valid;
      if (own_step) {
        valid = t < cnt;
        if (valid) e = lst[t * LS];
      } else {
        const int base = (t - M) * 32;
        W->start[lane] = -1;
        __syncwarp();
        if (ov > 0 && off >= base && off < base + 32) W->start[off - base] = lane;
        __syncwarp();
        const unsigned starts = __ballot_sync(0xffffffffu, W->start[lane] >= 0);
        const unsigned upto = starts & (0xffffffffu >> (31 - lane));
        who = upto ? W->start[31 - __clz(upto)] : carry;
        carry = __shfl_sync(0xffffffffu, who, 31);
        const int offo = __shfl_sync(0xffffffffu, off, who);
        const int g = base + lane;
        valid = g < total && DPD_IN_BOUNDS(M + (g - offo) < CAP, P.err);
        if (valid) e = W->list[who * (CAP + 1) + M + (g - offo)];
      }
      float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
      if (valid) r = pair(e, W->own_pos[who], W->own_vel[who]);
      if (own_step) {
        fx += r.x;
        fy += r.y;
        fz += r.z;
        vir += r.w;
      } else {
        const int base = (t - M) * 32;
        W->res[lane] = r;
        __syncwarp();
        const int lo = max(off - base, 0), hi = min(off + ov - base, 32);
        for (int q = lo; q < hi; ++q) {
          const float4 u = W->res[q];
          fx += u.x;
          fy += u.y;
          fz += u.z;
          vir += u.w;
        }
        __syncwarp();
      }
    }
    cnt = 0;
  };

  // Spread drain (half stencil): the warp's list entries are processed 32
  // at a time, one per lane whatever lane owns them; the owner of entry g is
  // found by a binary search over the lanes' list offsets, and both F_ij on
  // i and -F_ij on j go to memory as atomic adds (the half stencil's sums
  // have no fixed order anyway).  Lane o's target and velocity are in
  // own[o] and own[32 + o].
  auto drain_spread = [&]() {
    const int lane = threadIdx.x & 31;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int off = incl - cnt;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    __syncwarp();  // every lane's list is complete
    const uint32_t *wl = lst - lane;  // column of the warp's lane 0
    const int pw = p - lane;          // slot of the warp's lane 0
    for (int base = 0; base < total; base += 32) {
      const int g = base + lane;
      int o = 0;  // last lane whose list starts at or before g
#pragma unroll
      for (int s = 16; s >= 1; s >>= 1) {
        const int t = __shfl_sync(0xffffffffu, off, o + s);
        if (t <= g) o += s;
      }
      const int offo = __shfl_sync(0xffffffffu, off, o);
      if (g < total && DPD_IN_BOUNDS(g - offo >= 0 && g - offo < CAP, P.err)) {
        const uint32_t e = wl[(g - offo) * LS + o];
        const int j = (int)(e & kSlotMask);
        if (DPD_IN_BOUNDS(j < P.ntot && pw + o >= 0 && pw + o < P.ntot, P.err)) {
          const float4 r = pair_at(e, __ldg(P.pos + j), __ldg(P.vel + j), own[o], own[32 + o]);
          atomicAdd(P.frc + pw + o, r);
        }
      }
    }
    __syncwarp();  // lists may be refilled
    cnt = 0;
  };

  // The balanced and spread drains evaluate entries of other lanes with this
  // lane's box parameters and step, so a warp whose lanes (live or not) span
  // two boxes (`mixed`, warp-uniform) drains per lane.
  auto drain = [&]() {
    if constexpr (BAL) {
      if (!mixed) {
        drain_balanced();
        return;
      }
    }
    if constexpr (SPREAD) {
      if (!mixed) {
        drain_spread();
        return;
      }
    }
    if (!DPD_IN_BOUNDS(cnt <= CAP, P.err)) cnt = 0;
    for (int k = 0; k < cnt; ++k) {
      const float4 g = pair(lst[k * LS], pi, vi);
      fx += g.x;
      fy += g.y;
      fz += g.z;
      vir += g.w;
    }
    cnt = 0;
  };

  // Rows of the stencil.  Full: (dy, dz) in {-1,0,1}^2.  Half: the own row
  // (forward from the slot after p), row dy=+1 of the own plane, and the
  // three rows of the plane dz=+1.
  constexpr int NROWS = HALF ? 5 : 9;
#pragma unroll 1
  for (int r = 0; r < NROWS; ++r) {
    int dy, dz;
    if constexpr (HALF) {
      dz = (r < 2) ? 0 : 1;
      dy = (r == 0) ? 0 : (r == 1 ? 1 : r - 3);
    } else {
      dz = r / 3 - 1;
      dy = r - 3 * (r / 3) - 1;
    }
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
    const int rowbase = B.cellBase + (z * ny + y) * nx;
    const bool row_ok = DPD_IN_BOUNDS(rowbase >= 0 && rowbase + nx <= P.ncell, P.err);
    // Slices xlo .. xhi of the row: one range of slots, or two across an x
    // face, where the far part is the image r_j - L (xlo < 0) or is seen
    // from r_i - L (xhi >= nx).  Half stencil, own row: forward from the
    // slot after p (pairs within one slice belong to the lower slot).
    const bool own = HALF && r == 0;
    const int lo = own ? cx : xlo, hi = xhi;
    const int nseg =
        (alive && row_ok && DPD_IN_BOUNDS(lo >= -nx && lo <= hi && hi < 2 * nx, P.err))
            ? ((lo < 0 || hi >= nx) ? 2 : 1)
            : 0;
    auto segment = [&](int sg, int &j0, int &j1, float &ax, float &jsx, uint32_t &c) {
      ax = pi.x;
      jsx = 0.f;
      c = code;
      if (lo < 0) {  // slices lo + nx .. nx - 1 as r_j - L, then 0 .. hi
        if (sg == 0) {
          j0 = __ldg(P.start + rowbase + lo + nx);
          j1 = __ldg(P.start + rowbase + nx);
          jsx = Lx;
          c |= kCodeJX;
        } else {
          j0 = __ldg(P.start + rowbase);
          j1 = __ldg(P.start + rowbase + hi + 1);
        }
      } else if (hi >= nx) {  // lo .. nx - 1, then 0 .. hi - nx seen from r_i - L
        if (sg == 0) {
          j0 = own ? p + 1 : __ldg(P.start + rowbase + lo);
          j1 = __ldg(P.start + rowbase + nx);
        } else {
          j0 = __ldg(P.start + rowbase);
          j1 = __ldg(P.start + rowbase + hi - nx + 1);
          ax = pi.x - Lx;
          c |= kCodeIX;
        }
      } else {
        j0 = own ? p + 1 : __ldg(P.start + rowbase + lo);
        j1 = __ldg(P.start + rowbase + hi + 1);
      }
      if (!DPD_IN_BOUNDS(j0 >= 0 && j0 <= j1 && j1 <= P.ntot, P.err)) j0 = j1 = 0;
    };
    int sg = 0, j = 0, j1 = 0;
    float ax = 0.f, jsx = 0.f;
    uint32_t c = 0;
    if (nseg > 0) segment(0, j, j1, ax, jsx, c);
    for (;;) {
      bool more = false;
      if (sg < nseg) {
        if (!DPD_IN_BOUNDS(cnt <= CAP - U, P.err)) cnt = 0;
        const int stop = (c & (kCodeJX | kCodeJY | kCodeJZ))
                             ? scan_range<true, LS, CAP, U>(P.pos, j, j1, ax, ay, az, jsx, jsy, jsz,
                                                         rc2m1, c, lst, cnt)
                             : scan_range<false, LS, CAP, U>(P.pos, j, j1, ax, ay, az, 0.f, 0.f, 0.f,
                                                          rc2m1, c, lst, cnt);
        if (stop >= 0 && stop < j1) {
          j = stop;  // list nearly full: continue this segment after a drain
          more = true;
        } else if (++sg < nseg) {
          segment(sg, j, j1, ax, jsx, c);
          more = true;
        }
      }
      const bool any_more = __any_sync(0xffffffffu, more);
      if (__any_sync(0xffffffffu, cnt > CAP - U) ||
          (!any_more && __any_sync(0xffffffffu, cnt > FLUSH)))
        drain();
      if (!any_more) break;
    }
  }
  drain();

  if (!alive) {
    // fused step, box not advanced: the next step only bins this slot
    if constexpr (!HALF) {
      if (fuse && real)  // stopped box: keeps its slots
        integrate_one(P, B, p, P.pos[p], P.vel[p], 0.f, 0.f, 0.f, false, false, true);
    }
    return;
  }
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
  } else if (fuse) {
    // the full stencil's force on p is complete here: the next step's row a1
    // for p, instead of storing the force for a separate integrate pass.  A
    // box that stops after this step keeps its force for later read-outs.
    const bool moves = S.remaining > 0;
    integrate_one(P, B, p, pi, vi, fx, fy, fz, moves, true, !moves);
    if (!moves) P.frc[p] = make_float4(fx, fy, fz, vir);
  } else {
    P.frc[p] = make_float4(fx, fy, fz, vir);
  }
}

}  // namespace dpd
