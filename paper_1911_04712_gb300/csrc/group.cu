// Box-grouped force launches for packed sets with the half stencil (pair
// forces, Sec. 2.1 Eqs. 2-5, over the cell list of Sec. 3.2).  Each block
// takes consecutive slots of one box only, so no warp spans two boxes and
// every warp-cooperative drain applies.  The constants of up to
// kGroupBoxes boxes travel in the kernel parameters: a block finds its box
// by a search over the parameter table that depends on the block index
// alone, so the box's constants are block-uniform values, as the single-box
// kernels' are, instead of per-thread registers loaded from the box table.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "dpd_device.cuh"
#include "force_direct.cuh"
#include "kernels.h"

namespace dpd {

BoxHot box_hot(const BoxDev &B) {
  BoxHot h{};
  for (int k = 0; k < 3; ++k) {
    h.L[k] = B.L[k];
    h.invh[k] = B.invh[k];
    h.n[k] = B.n[k];
  }
  h.xwin = B.xwin;
  h.cellBase = B.cellBase;
  h.pbase = B.pbase;
  h.np = B.np;
  h.a = B.a;
  h.gamma = B.gamma;
  h.sig = B.sig;
  h.rc2 = B.rc2;
  h.inv_rc = B.inv_rc;
  h.kexp = B.kexp;
  h.fb = B.fb;
  h.fb_half = B.fb_half;
  h.fb_mode = B.fb_mode;
  h.fb_flow = B.fb_flow;
  h.fb_grad = B.fb_grad;
  h.seed_lo = B.seed_lo;
  h.seed_hi = B.seed_hi;
  return h;
}

namespace {

// The kernels are the spread-drain variants: the per-lane and balanced
// drains, compiled this way, need twice the registers of their packed
// kernels and stay with those.  The compiler's 60 registers (eight blocks
// of 128 threads per SM) ran 5 % faster than a bound of 56 (nine blocks),
// under which the block-uniform constants are re-read more often.
template <int NT, int CAP>
__global__ void __launch_bounds__(NT)
    k_force_group(Packed P, const __grid_constant__ BoxGroup G) {
  __shared__ uint32_t smem_list[CAP * NT];
  __shared__ float4 smem_own[2 * NT];
  // the block's box: the last k with blk[k] <= blockIdx.x (block-uniform)
  const int bx = (int)blockIdx.x;
  int lo = 0, hi = G.nbox - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (G.blk[mid] <= bx)
      lo = mid;
    else
      hi = mid - 1;
  }
  const BoxHot &B = G.hot[lo];
  const int p = B.pbase + (bx - G.blk[lo]) * NT + (int)threadIdx.x;
  const bool real = p < B.pbase + B.np;  // lanes past the box's end are dead
  const BoxState S = P.st[G.box[lo]];
  const bool alive = real && S.adv;
  force_direct<true, NT, CAP, false, false, true>(P, B, S, p, alive, smem_list + threadIdx.x,
                                                  nullptr, smem_own + (threadIdx.x >> 5) * 64,
                                                  false, false, real);
}

template <int NT, int CAP>
cudaError_t launch_g(const Packed &P, const BoxGroup &G, cudaStream_t s) {
  if (G.nbox > 0 && G.blk[G.nbox] > 0) k_force_group<NT, CAP><<<G.blk[G.nbox], NT, 0, s>>>(P, G);
  return cudaGetLastError();
}

cudaError_t launch_group_variant(int v, const Packed &P, const BoxGroup &G, cudaStream_t s) {
  switch (v) {  // the spread variants of force.cu: threads x list capacity
    case 10: return launch_g<64, 32>(P, G, s);
    case 11: return launch_g<128, 32>(P, G, s);
    default: return launch_g<128, 24>(P, G, s);
  }
}

}  // namespace

cudaError_t launch_force_group(const Packed &P, const BoxDev *hboxes, int box0, int box1,
                               int variant, cudaStream_t s) {
  int nt = 0, cap = 0;
  if (!hboxes || box0 < 0 || box1 > P.nbox || !grouped_variant(variant, false, true) ||
      force_variant_info(variant, &nt, &cap) != 0)
    return cudaErrorInvalidValue;
  // one parameter table per launch: about 27 KB, kept off the caller's stack
  static thread_local BoxGroup G;
  for (int b = box0; b < box1;) {
    G.nbox = 0;
    long long blocks = 0;
    for (; b < box1 && G.nbox < kGroupBoxes; ++b) {
      const BoxDev &B = hboxes[b];
      const long long nblk = ((long long)B.np + nt - 1) / nt;
      if (nblk == 0) continue;  // an empty box has no targets
      G.blk[G.nbox] = (int)blocks;
      G.box[G.nbox] = b;
      G.hot[G.nbox] = box_hot(B);
      ++G.nbox;
      blocks += nblk;
    }
    G.blk[G.nbox] = (int)blocks;  // at most 2^26 slots: fits an int
    const cudaError_t e = launch_group_variant(variant, P, G, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace dpd
