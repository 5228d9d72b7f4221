// Engine implementation: device buffers, the per-step launch sequence, CUDA
// graph capture of step chunks, and the FP64 statistics reduction.
#include "engine.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "dpd.h"

namespace dpd {

static thread_local std::string t_err;

int set_error(int code, const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_err = buf;
  return code;
}
void clear_error() { t_err.clear(); }
const char *last_error_text() { return t_err.c_str(); }

int check_params(const BoxParams &bp, int n[3]) {
  if (!(bp.rc > 0.0) || !std::isfinite(bp.rc)) return set_error(DPD_ERR_ARG, "rc must be > 0");
  double cells = 1.0;
  for (int k = 0; k < 3; ++k) {
    if (!std::isfinite(bp.L[k]) || !(bp.L[k] >= 3.0 * bp.rc))
      return set_error(DPD_ERR_ARG, "box edge %d = %g must be >= 3 rc = %g", k, bp.L[k],
                       3.0 * bp.rc);
    const double nd = std::floor(bp.L[k] / bp.rc);
    if (nd > kMaxCellsPerAxis)
      return set_error(DPD_ERR_ARG, "box edge %d spans %g cells; at most %d per axis", k, nd,
                       kMaxCellsPerAxis);
    n[k] = (int)nd * (k == 0 ? kSlicesX : 1);
    cells *= (double)n[k];
  }
  if (cells > (double)kMaxCellEntries)
    return set_error(DPD_ERR_ARG, "too many cells (%g x-slices; at most %lld)", cells,
                     kMaxCellEntries);
  auto nonneg = [](double v) { return std::isfinite(v) && v >= 0.0; };
  if (!nonneg(bp.a)) return set_error(DPD_ERR_ARG, "a must be >= 0");
  if (!nonneg(bp.gamma)) return set_error(DPD_ERR_ARG, "gamma must be >= 0");
  if (!nonneg(bp.kT)) return set_error(DPD_ERR_ARG, "kT must be >= 0");
  if (!(bp.dt > 0.0) || !std::isfinite(bp.dt)) return set_error(DPD_ERR_ARG, "dt must be > 0");
  if (!(bp.mass > 0.0) || !std::isfinite(bp.mass))
    return set_error(DPD_ERR_ARG, "mass must be > 0");
  if (!(bp.kexp > 0.0 && bp.kexp <= 1.0))
    return set_error(DPD_ERR_ARG, "weight exponent k must be in (0, 1]");
  if (bp.fb_mode < 0 || bp.fb_mode > 2 || !std::isfinite(bp.fb))
    return set_error(DPD_ERR_ARG, "bad body force");
  if (bp.fb_flow < 0 || bp.fb_flow > 2 || bp.fb_grad < 0 || bp.fb_grad > 2)
    return set_error(DPD_ERR_ARG, "body-force axes must be 0, 1 or 2");
  if (bp.noise != 0 && bp.noise != 1) return set_error(DPD_ERR_ARG, "noise must be 0 or 1");
  if (bp.nspec < 1 || bp.nspec > kMaxSpecies)
    return set_error(DPD_ERR_ARG, "species count must be 1..%d", kMaxSpecies);
  for (int s = 0; s < bp.nspec && bp.nspec > 1; ++s)
    for (int t = 0; t < bp.nspec; ++t) {
      const int k = 4 * s + t, kt = 4 * t + s;
      if (bp.sa[k] != bp.sa[kt] || bp.sg[k] != bp.sg[kt] || bp.src[k] != bp.src[kt])
        return set_error(DPD_ERR_ARG, "species tables must be symmetric (%d, %d)", s, t);
      if (!nonneg(bp.sa[k]) || !nonneg(bp.sg[k]))
        return set_error(DPD_ERR_ARG, "species (%d, %d): a and gamma must be >= 0", s, t);
      if (!(bp.src[k] > 0.0 && bp.src[k] <= bp.rc))
        return set_error(DPD_ERR_ARG, "species (%d, %d): cut-off must be in (0, rc = %g]", s, t,
                         bp.rc);
    }
  return DPD_OK;
}

BoxDev make_box_dev(const BoxParams &bp, int cellBase, int pbase, int np) {
  BoxDev d{};
  int n[3];
  double lmax = 0.0;
  for (int k = 0; k < 3; ++k) {
    n[k] = (int)std::floor(bp.L[k] / bp.rc) * (k == 0 ? kSlicesX : 1);
    d.L[k] = (float)bp.L[k];
    d.n[k] = n[k];
    d.invh[k] = (float)((double)n[k] / bp.L[k]);
    lmax = std::max(lmax, bp.L[k]);
  }
  d.xwin = (float)(bp.rc + 16.0 * std::ldexp(std::max(lmax, bp.rc), -23));
  d.cellBase = cellBase;
  d.pbase = pbase;
  d.np = np;
  d.a = (float)bp.a;
  d.gamma = (float)bp.gamma;
  const double sigma = std::sqrt(2.0 * bp.gamma * bp.kT);  // fluctuation-dissipation
  d.sig = (float)(sigma * std::sqrt(3.0) / 16777216.0 / std::sqrt(bp.dt));
  d.sig_g = (float)(sigma / std::sqrt(bp.dt));
  d.noise = bp.noise;
  d.rc2 = (float)(bp.rc * bp.rc);
  d.inv_rc = (float)(1.0 / bp.rc);
  d.kexp = (float)bp.kexp;
  d.hdt_m = (float)(0.5 * bp.dt / bp.mass);
  d.dt = (float)bp.dt;
  d.fb = (float)bp.fb;
  d.fb_mode = bp.fb_mode;
  d.fb_flow = bp.fb_flow;
  d.fb_grad = bp.fb_grad;
  d.fb_half = (float)(0.5 * bp.L[bp.fb_grad]);
  d.seed_lo = (uint32_t)(bp.seed & 0xffffffffu);
  d.seed_hi = (uint32_t)(bp.seed >> 32);
  d.nspec = bp.nspec;
  for (int k = 0; k < kMaxSpecies * kMaxSpecies; ++k) {
    const bool multi = bp.nspec > 1;
    const double a = multi ? bp.sa[k] : bp.a, g = multi ? bp.sg[k] : bp.gamma;
    const double rc = multi ? bp.src[k] : bp.rc;
    const double sg = std::sqrt(2.0 * g * bp.kT);  // fluctuation-dissipation, per pair of species
    d.sp_a[k] = (float)a;
    d.sp_gamma[k] = (float)g;
    d.sp_sig[k] = (float)(sg * std::sqrt(3.0) / 16777216.0 / std::sqrt(bp.dt));
    d.sp_sig_g[k] = (float)(sg / std::sqrt(bp.dt));
    d.sp_rc2[k] = (float)(rc * rc);
    d.sp_inv_rc[k] = rc > 0.0 ? (float)(1.0 / rc) : 0.0f;
  }
  return d;
}

// ------------------------------------------------------------------ engine
Engine::Engine() {}

Engine::~Engine() {
  if (device_ >= 0) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != device_) cudaSetDevice(device_);
    // No stream synchronisation here: the caller's stream may already be
    // gone; cudaFree waits for the device, and an in-flight graph is freed
    // when it completes.
    drop_graph();
    free_all();
    if (d_.err) cudaFree(d_.err);
    if (h_err_) cudaFreeHost(h_err_);
    if (d_tiles_) cudaFree(d_tiles_);
    if (d_mixed_) cudaFree(d_mixed_);
    if (d_bricks_) cudaFree(d_bricks_);
    for (void *q : {(void *)d_wbeg_, (void *)d_from_, (void *)d_acc_, (void *)d_spart_})
      if (q) cudaFree(q);
    if (h_sum_) cudaFreeHost(h_sum_);
    if (cap_) cudaStreamDestroy(cap_);
    if (cur >= 0 && cur != device_) cudaSetDevice(cur);
  }
}

int Engine::init() {
  int dev = -1;
  DPD_CUDA_TRY(cudaGetDevice(&dev));
  int count = 0;
  DPD_CUDA_TRY(cudaGetDeviceCount(&count));
  if (count <= 0) return set_error(DPD_ERR_CUDA, "no CUDA device");
  device_ = dev;
  static std::mutex mu;
  static bool prepared[256] = {false};
  {
    std::lock_guard<std::mutex> g(mu);
    if (dev < 256 && !prepared[dev]) {
      DPD_CUDA_TRY(prepare_device());
      prepared[dev] = true;
    }
  }
  DPD_CUDA_TRY(cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking));
  DPD_CUDA_TRY(cudaMalloc(&d_.err, sizeof(unsigned)));
  DPD_CUDA_TRY(cudaMemset(d_.err, 0, sizeof(unsigned)));
  DPD_CUDA_TRY(cudaMallocHost(&h_err_, sizeof(unsigned)));
  *h_err_ = 0u;
  return DPD_OK;
}

int Engine::set_stream(cudaStream_t s) {
  stream_ = s;
  return DPD_OK;
}

int Engine::set_stencil(int stencil) {
  if (stencil != 0 && stencil != 1) return set_error(DPD_ERR_ARG, "stencil must be 0 or 1");
  if (stencil != cfg_.stencil) {
    cfg_.stencil = stencil;
    drop_graph();
    if (!boxes_.empty()) return build_bands();
  }
  return DPD_OK;
}

int Engine::set_variant(int variant) {
  if (variant < -1 || variant >= kNumForceVariants)
    return set_error(DPD_ERR_ARG, "force variant must be -1..%d", kNumForceVariants - 1);
  variant_override_ = variant;
  drop_graph();
  return boxes_.empty() ? DPD_OK : build_bands();
}

int Engine::set_fuse(bool on) {
  fuse_ = on;
  drop_graph();
  return DPD_OK;
}

// The force kernel can do the next step's kick/drift/bin only when it owns
// each particle's whole force (full stencil, direct kernels) and nothing
// reads the state between the two steps (no sampling).
bool Engine::fused_steps() const {
  return fuse_ && cfg_.stencil == 0 && !cfg_.tiles && sample_every_ <= 0;
}

int Engine::refresh_bands() {
  drop_graph();
  return boxes_.empty() ? DPD_OK : build_bands();
}

// Group consecutive boxes that use the same direct-kernel variant into
// bands (contiguous slot ranges), one force launch each.
int Engine::build_bands() {
  const int nb = nbox();
  std::vector<ForceBand> runs;
  for (int b = 0; b < nb; ++b) {
    const BoxDev &B = boxes_[b];
    const double rho = (double)B.np / ((double)B.L[0] * B.L[1] * B.L[2]);
    const int table = cfg_.stencil + (nb > 1 ? 2 : 0);  // packed sets have their own table
    int v = variant_override_ >= 0 ? variant_override_ : tuned_variant(table, rho);
    // the brick kernel stages one cell row's stencil (6 rows x 5 slices) at
    // the least: a box whose mean density fills half the staging capacity
    // that way runs the default direct kernel instead
    if (v == kBrickVariant && 30.0 * B.np / ((double)B.n[0] * B.n[1] * B.n[2]) >
                                  0.5 * kBrickCaps)
      v = 0;
    const int g = B.noise != 0 || B.nspec > 1;  // general kernel
    if (!runs.empty() && runs.back().variant == v && runs.back().gauss == g) {
      runs.back().slot1 = pbase_[b + 1];
      runs.back().item1 = brick_beg_[b + 1];
      runs.back().box1 = b + 1;
    } else {
      ForceBand fb{pbase_[b], pbase_[b + 1], v, g};
      fb.item0 = brick_beg_[b];
      fb.item1 = brick_beg_[b + 1];
      fb.box0 = b;
      fb.box1 = b + 1;
      runs.push_back(fb);
    }
  }
  if ((int)runs.size() > kMaxBands) {
    // too fragmented (boxes not ordered by band): one launch with the
    // variant that covers the most particles
    std::vector<long long> cover(kNumForceVariants, 0);
    int anyg = 0;
    for (const auto &r : runs) {
      cover[r.variant] += r.slot1 - r.slot0;
      anyg |= r.gauss;
    }
    const int best = (int)(std::max_element(cover.begin(), cover.end()) - cover.begin());
    runs.assign(1, ForceBand{0, ntot_, best, anyg});
    runs[0].item0 = 0;
    runs[0].item1 = (int)bricks_h_.size();
    runs[0].box0 = 0;
    runs[0].box1 = nb;
  }
  // Packed sets: the warps of each band whose slots span two boxes (the
  // device tests the same: the box of the first and of the last slot, the
  // slots clamped to the packed set).  Warp-cooperative kernels skip them.
  std::vector<int> mixed;
  auto box_of_slot = [&](int p) {
    return (int)(std::upper_bound(pbase_.begin(), pbase_.end(), p) - pbase_.begin()) - 1;
  };
  for (auto &r : runs) {
    r.mw_off = (int)mixed.size();
    if (nb > 1)
      for (int p0 = r.slot0; p0 < r.slot1; p0 += 32)
        if (box_of_slot(p0) != box_of_slot(std::min(p0 + 31, ntot_ - 1))) mixed.push_back(p0);
    r.mw_count = (int)mixed.size() - r.mw_off;
  }
  if (mixed.size() > cap_mixed_) {
    if (d_mixed_) cudaFree(d_mixed_);
    d_mixed_ = nullptr;
    cap_mixed_ = 0;
    DPD_CUDA_TRY(cudaMalloc(&d_mixed_, mixed.size() * 2 * sizeof(int)));
    cap_mixed_ = mixed.size() * 2;
  }
  if (!mixed.empty())
    DPD_CUDA_TRY(cudaMemcpyAsync(d_mixed_, mixed.data(), mixed.size() * sizeof(int),
                                 cudaMemcpyHostToDevice, stream_));
  cfg_.mixed_warps = d_mixed_;
  cfg_.hboxes = boxes_.data();
  cfg_.nbands = (int)runs.size();
  for (int k = 0; k < cfg_.nbands; ++k) cfg_.band[k] = runs[k];
  return DPD_OK;
}

int Engine::set_tiling(int use_tiles, int tc, int stage_cap) {
  if (tc < 0 || tc > kTileMaxCells) return set_error(DPD_ERR_ARG, "cells per tile must be 0..%d", kTileMaxCells);
  if (stage_cap != 0 && (stage_cap < 64 || stage_cap > 4096))
    return set_error(DPD_ERR_ARG, "staging capacity must be 0 or 64..4096 particles");
  cfg_.tiles = use_tiles != 0;
  tile_tc_override_ = tc;
  stage_cap_override_ = stage_cap;
  drop_graph();
  if (!boxes_.empty()) return build_tiles();
  return DPD_OK;
}

// Cells per tile and staging capacity by density: about 9 (tc + 2) rho
// particles are staged; tc is chosen so that this stays near 900 (about
// 100 targets per block of 128 threads).
static int tile_cells_for(double rho, int nx) {
  int tc = (int)std::lround(102.0 / std::max(rho, 0.5)) - 2;
  tc = std::max(2, std::min(tc, kTileMaxCells));
  return std::min(tc, nx);
}

int Engine::build_tiles() {
  const int nb = nbox();
  int stage_need = 0;
  tiles_h_.clear();
  int tc_single = 0;
  for (int b = 0; b < nb; ++b) {
    const BoxDev &B = boxes_[b];
    const int ncx = B.n[0] / kSlicesX;  // tiles are runs of whole cells
    const double V = (double)B.L[0] * B.L[1] * B.L[2];
    const double rho = (double)B.np / V;
    int tc = tile_tc_override_ > 0 ? std::min(tile_tc_override_, ncx) : tile_cells_for(rho, ncx);
    const double h3 = V / ((double)ncx * B.n[1] * B.n[2]);
    const int need = (int)std::ceil(9.0 * (tc + 2) * rho * h3 * 1.35) + 64;
    stage_need = std::max(stage_need, need);
    if (b == 0) tc_single = tc;
    if (nb > 1) {
      const int tpr = (ncx + tc - 1) / tc;
      for (int cz = 0; cz < B.n[2]; ++cz)
        for (int cy = 0; cy < B.n[1]; ++cy)
          for (int t = 0; t < tpr; ++t) {
            const int cx0 = t * tc;
            const int nc = std::min(tc, ncx - cx0);
            tiles_h_.push_back(make_int4(b, cy, cz, cx0 | (nc << 16)));
          }
    }
  }
  int cap = stage_cap_override_ > 0 ? stage_cap_override_ : ((stage_need + 63) / 64) * 64;
  cap = std::min(cap, 4096);
  cfg_.grid.stage_cap = cap;
  if (nb == 1) {
    const BoxDev &B = boxes_[0];
    cfg_.grid.list = nullptr;
    cfg_.grid.tc = tc_single;
    cfg_.grid.tpr = (B.n[0] / kSlicesX + tc_single - 1) / tc_single;
    cfg_.grid.ntiles = cfg_.grid.tpr * B.n[1] * B.n[2];
  } else {
    if (tiles_h_.size() > cap_tiles_) {
      if (d_tiles_) cudaFree(d_tiles_);
      d_tiles_ = nullptr;
      DPD_CUDA_TRY(cudaMalloc(&d_tiles_, tiles_h_.size() * sizeof(int4)));
      cap_tiles_ = tiles_h_.size();
    }
    DPD_CUDA_TRY(cudaMemcpyAsync(d_tiles_, tiles_h_.data(), tiles_h_.size() * sizeof(int4),
                                 cudaMemcpyHostToDevice, stream_));
    cfg_.grid.list = d_tiles_;
    cfg_.grid.tc = 0;
    cfg_.grid.tpr = 0;
    cfg_.grid.ntiles = (int)tiles_h_.size();
  }
  return DPD_OK;
}

// Brick shape of a box: the target rows (by x bz) that stage the fewest
// particles per target while a chunk of several slices still fits the
// staging capacity at the box's mean density (the kernel narrows a chunk
// where the density is higher, and splits a brick into rows where even one
// slice does not fit).
static void brick_shape(const BoxDev &B, int caps, int *by_out, int *bz_out, int *w_out) {
  const double V = (double)B.L[0] * B.L[1] * B.L[2];
  const double ps = (double)B.np / V * V / ((double)B.n[0] * B.n[1] * B.n[2]);  // per slice
  double best = 1e300;
  int by = 1, bz = 1, wb = 1;
  for (int y = 1; y <= std::min(kBrickMaxBY, B.n[1]); ++y)
    for (int z = 1; z <= std::min(kBrickMaxBZ, B.n[2]); ++z) {
      const int nrows = (y + 2) * (z + 1);
      int w = (int)std::floor(0.75 * caps / (nrows * std::max(ps, 1e-3))) - 4;
      w = std::min(std::min(w, kBrickWMax), B.n[0]);
      if (w < 2) continue;
      const double ov = (double)nrows * (w + 4) / ((double)y * z * w);
      if (ov < best - 1e-9) {
        best = ov;
        by = y;
        bz = z;
        wb = w;
      }
    }
  *by_out = by;
  *bz_out = bz;
  *w_out = wb;
}

int Engine::build_bricks() {
  const int nb = nbox();
  const int caps = kBrickCaps;
  bricks_h_.clear();
  brick_beg_.assign(nb + 1, 0);
  for (int b = 0; b < nb; ++b) {
    brick_beg_[b] = (int)bricks_h_.size();
    const BoxDev &B = boxes_[b];
    if (B.np <= 0) continue;
    int by, bz, w;
    brick_shape(B, caps, &by, &bz, &w);
    const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
    const int nby = (ny + by - 1) / by, nbz = (nz + bz - 1) / bz;
    // x pieces of about 2048 targets, at least two chunks wide
    const double ps = (double)B.np / ((double)nx * ny * nz);
    int xs = (int)std::lround(2048.0 / std::max(by * bz * ps, 1e-3));
    xs = std::max(std::min(xs, nx), std::min(2 * w, nx));
    const int npx = (nx + xs - 1) / xs;
    for (int kz = 0, z0 = 0; kz < nbz; ++kz) {
      const int bzk = nz / nbz + (kz < nz % nbz ? 1 : 0);
      for (int ky = 0, y0 = 0; ky < nby; ++ky) {
        const int byk = ny / nby + (ky < ny % nby ? 1 : 0);
        for (int kx = 0, s0 = 0; kx < npx; ++kx) {
          const int len = nx / npx + (kx < nx % npx ? 1 : 0);
          bricks_h_.push_back(make_int4(b, y0 | (byk << 16), z0 | (bzk << 16), s0 | ((s0 + len) << 16)));
          s0 += len;
        }
        y0 += byk;
      }
      z0 += bzk;
    }
  }
  brick_beg_[nb] = (int)bricks_h_.size();
  if (bricks_h_.size() > cap_bricks_) {
    if (d_bricks_) cudaFree(d_bricks_);
    d_bricks_ = nullptr;
    cap_bricks_ = 0;
    DPD_CUDA_TRY(cudaMalloc(&d_bricks_, bricks_h_.size() * sizeof(int4)));
    cap_bricks_ = bricks_h_.size();
  }
  if (!bricks_h_.empty())
    DPD_CUDA_TRY(cudaMemcpyAsync(d_bricks_, bricks_h_.data(), bricks_h_.size() * sizeof(int4),
                                 cudaMemcpyHostToDevice, stream_));
  cfg_.bricks.items = d_bricks_;
  cfg_.bricks.nitems = (int)bricks_h_.size();
  cfg_.bricks.caps = caps;
  return DPD_OK;
}

void Engine::drop_graph() {
  for (cudaGraphExec_t *g : {&graph_, &graph1_})
    if (*g) {
      cudaGraphExecDestroy(*g);
      *g = nullptr;
    }
}

int Engine::free_all() {
  void *ptrs[] = {d_.pos,   d_.vel,    d_.frc,   d_.pos2,  d_.vel2,  d_.cellOf, d_.slotIn,
                  d_.keyTmp, d_.count, d_.start, d_.bsum,  d_.boxes, d_.pbase,  d_.st,
                  d_.work,  d_.part};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  unsigned *err = d_.err;  // the error word lives as long as the engine
  d_ = DeviceArrays{};
  d_.err = err;
  return DPD_OK;
}

size_t Engine::device_bytes() const {
  return d_.capP * (5 * sizeof(float4) + 3 * sizeof(int)) +
         d_.capC * 2 * sizeof(int) + (d_.capC / kScanTile + 1) * sizeof(int) +
         d_.capB * (sizeof(BoxDev) + sizeof(int) + sizeof(BoxState)) +
         d_.capW * (sizeof(StatsWork) + kStatsFields * sizeof(double));
}

template <typename T>
static cudaError_t grow(T *&ptr, size_t n) {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  return cudaMalloc(&ptr, std::max<size_t>(n, 1) * sizeof(T));
}

int Engine::reserve(size_t np, size_t nc, size_t nb) {
  if (np > d_.capP) {
    drop_graph();
    const size_t cap = std::max(np, d_.capP + d_.capP / 4);
    DPD_CUDA_TRY(grow(d_.pos, cap));
    DPD_CUDA_TRY(grow(d_.vel, cap));
    DPD_CUDA_TRY(grow(d_.frc, cap));
    DPD_CUDA_TRY(grow(d_.pos2, cap));
    DPD_CUDA_TRY(grow(d_.vel2, cap));
    DPD_CUDA_TRY(grow(d_.cellOf, cap));
    DPD_CUDA_TRY(grow(d_.slotIn, cap));
    DPD_CUDA_TRY(grow(d_.keyTmp, cap));
    DPD_CUDA_TRY(cudaMemset(d_.frc, 0, cap * sizeof(float4)));
    d_.capP = cap;
  }
  const size_t tiles = (size_t)scan_tiles((int)nc);
  const size_t ncap = tiles * kScanTile;
  if (ncap > d_.capC) {
    drop_graph();
    if (tiles > (size_t)kScanMaxTiles)
      return set_error(DPD_ERR_ARG, "too many cells for one scan (%zu)", nc);
    DPD_CUDA_TRY(grow(d_.count, ncap));
    DPD_CUDA_TRY(grow(d_.start, ncap));
    DPD_CUDA_TRY(grow(d_.bsum, tiles));
    DPD_CUDA_TRY(cudaMemset(d_.count, 0, ncap * sizeof(int)));
    d_.capC = ncap;
  }
  if (nb > d_.capB) {
    drop_graph();
    const size_t cap = std::max(nb, d_.capB * 2);
    DPD_CUDA_TRY(grow(d_.boxes, cap));
    DPD_CUDA_TRY(grow(d_.pbase, cap + 1));
    DPD_CUDA_TRY(grow(d_.st, cap));
    d_.capB = cap;
  }
  return DPD_OK;
}

Packed Engine::packed() const {
  Packed P{};
  P.pos = d_.pos;
  P.vel = d_.vel;
  P.frc = d_.frc;
  P.pos2 = d_.pos2;
  P.vel2 = d_.vel2;
  P.cellOf = d_.cellOf;
  P.slotIn = d_.slotIn;
  P.keyTmp = d_.keyTmp;
  P.count = d_.count;
  P.start = d_.start;
  P.bsum = d_.bsum;
  P.boxes = d_.boxes;
  P.pbase = d_.pbase;
  P.st = d_.st;
  P.err = d_.err;
  P.ntot = ntot_;
  P.ncell = ncell_;
  P.nbox = (int)boxes_.size();
  if (!boxes_.empty()) P.single = boxes_[0];
  return P;
}

int Engine::layout(const std::vector<BoxParams> &params, const std::vector<int64_t> &np) {
  if (params.size() != np.size() || params.empty())
    return set_error(DPD_ERR_ARG, "layout needs one particle count per box");
  std::vector<BoxDev> boxes(params.size());
  std::vector<int> pbase(params.size() + 1);
  int64_t ptot = 0, ctot = 0;
  for (size_t b = 0; b < params.size(); ++b) {
    int n[3];
    int rc = check_params(params[b], n);
    if (rc) return rc;
    if (np[b] < 0) return set_error(DPD_ERR_ARG, "negative particle count");
    pbase[b] = (int)ptot;
    boxes[b] = make_box_dev(params[b], (int)ctot, (int)ptot, (int)np[b]);
    ptot += np[b];
    ctot += (int64_t)n[0] * n[1] * n[2];
    if (ptot > kMaxSlots || ctot > kMaxCellEntries)
      return set_error(DPD_ERR_ARG, "packed set too large (%lld particles, %lld cells)",
                       (long long)ptot, (long long)ctot);
  }
  pbase[params.size()] = (int)ptot;
  int rc = reserve((size_t)ptot, (size_t)ctot, params.size());
  if (rc) return rc;
  params_ = params;
  boxes_ = boxes;
  pbase_ = pbase;
  ntot_ = (int)ptot;
  ncell_ = (int)ctot;
  st_host_.assign(params.size(), BoxState{0ull, 0ll, 0, 0});
  from_h_.assign(params.size(), 0ll);
  work_dirty_ = true;
  drop_graph();
  DPD_CUDA_TRY(cudaMemcpyAsync(d_.boxes, boxes_.data(), boxes_.size() * sizeof(BoxDev),
                               cudaMemcpyHostToDevice, stream_));
  DPD_CUDA_TRY(cudaMemcpyAsync(d_.pbase, pbase_.data(), pbase_.size() * sizeof(int),
                               cudaMemcpyHostToDevice, stream_));
  int rc2 = build_tiles();
  if (!rc2) rc2 = build_bricks();
  if (!rc2) rc2 = build_bands();
  if (!rc2) rc2 = build_work();
  if (!rc2 && sample_every_ > 0) rc2 = ensure_sampling_buffers();
  return rc2;
}

bool Engine::restart_same_layout(const std::vector<int64_t> &np) {
  if (boxes_.empty() || np.size() != boxes_.size() || sample_every_ > 0) return false;
  for (size_t b = 0; b < np.size(); ++b)
    if (np[b] != (int64_t)(pbase_[b + 1] - pbase_[b])) return false;
  st_host_.assign(np.size(), BoxState{0ull, 0ll, 0, 0});
  from_h_.assign(np.size(), 0ll);
  return true;
}

int Engine::update_params(const std::vector<BoxParams> &params) {
  if (params.size() != boxes_.size()) return set_error(DPD_ERR_ARG, "box count changed");
  for (size_t b = 0; b < params.size(); ++b) {
    int n[3];
    int rc = check_params(params[b], n);
    if (rc) return rc;
    const BoxDev nb = make_box_dev(params[b], boxes_[b].cellBase, boxes_[b].pbase, boxes_[b].np);
    if (nb.n[0] != boxes_[b].n[0] || nb.n[1] != boxes_[b].n[1] || nb.n[2] != boxes_[b].n[2])
      return set_error(DPD_ERR_ARG, "box edges or rc changed the cell grid; reload the state");
    boxes_[b] = nb;
  }
  params_ = params;
  drop_graph();
  DPD_CUDA_TRY(cudaMemcpyAsync(d_.boxes, boxes_.data(), boxes_.size() * sizeof(BoxDev),
                               cudaMemcpyHostToDevice, stream_));
  return DPD_OK;
}

int Engine::load_box(int box, const float *pos, const float *vel, bool device_ptr,
                     const int32_t *species) {
  NvtxRange range("dpd load state");
  if (box < 0 || box >= nbox()) return set_error(DPD_ERR_ARG, "box index out of range");
  const int n = pbase_[box + 1] - pbase_[box];
  if (n == 0) return DPD_OK;
  if (!pos || !vel) return set_error(DPD_ERR_ARG, "null position or velocity array");
  const float *p3 = pos, *v3 = vel;
  if (!device_ptr) {
    float *sp = reinterpret_cast<float *>(d_.pos2), *sv = reinterpret_cast<float *>(d_.vel2);
    DPD_CUDA_TRY(cudaMemcpyAsync(sp, pos, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice,
                                 stream_));
    DPD_CUDA_TRY(cudaMemcpyAsync(sv, vel, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice,
                                 stream_));
    p3 = sp;
    v3 = sv;
    if (species) {  // host species: through the key scratch, free between steps
      DPD_CUDA_TRY(cudaMemcpyAsync(d_.keyTmp, species, (size_t)n * sizeof(int32_t),
                                   cudaMemcpyHostToDevice, stream_));
      species = d_.keyTmp;
    }
  }
  const BoxDev &B = boxes_[box];
  DPD_CUDA_TRY(launch_load(packed(), pbase_[box], n, p3, v3, B.L[0], B.L[1], B.L[2], stream_,
                           species, params_[box].nspec));
  return DPD_OK;
}

void Engine::set_box_state(int box, uint64_t step0, int64_t remaining) {
  st_host_[box] = BoxState{step0, remaining, 0, 1};
}

int Engine::set_remaining(int box, int64_t remaining) {
  if (box < 0 || box >= nbox()) return set_error(DPD_ERR_ARG, "box index out of range");
  st_host_[box].remaining = remaining;
  DPD_CUDA_TRY(cudaMemcpyAsync(&d_.st[box].remaining, &st_host_[box].remaining,
                               sizeof(long long), cudaMemcpyHostToDevice, stream_));
  return DPD_OK;
}

int Engine::rebuild() {
  for (auto &s : st_host_) s.adv = 1;
  DPD_CUDA_TRY(cudaMemcpyAsync(d_.st, st_host_.data(), st_host_.size() * sizeof(BoxState),
                               cudaMemcpyHostToDevice, stream_));
  if (sample_every_ > 0) {
    int rc = ensure_sampling_buffers();
    if (rc) return rc;
    DPD_CUDA_TRY(cudaMemcpyAsync(d_from_, from_h_.data(), from_h_.size() * sizeof(long long),
                                 cudaMemcpyHostToDevice, stream_));
  }
  DPD_CUDA_TRY(launch_step(packed(), false, false, cfg_, stream_));
  return DPD_OK;
}

int Engine::capture_graph(int nsteps, cudaGraphExec_t *out) {
  if (*out) {
    cudaGraphExecDestroy(*out);
    *out = nullptr;
  }
  const Packed P = packed();
  cudaGraph_t g = nullptr;
  DPD_CUDA_TRY(cudaStreamBeginCapture(cap_, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  const bool fz = fused_steps();  // steps inside the chunk fused, the last one plain
  for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
    e = launch_step(P, true, true, cfg_, cap_, fz && k > 0, fz && k + 1 < nsteps);
    if (e == cudaSuccess && sample_every_ > 0)
      e = launch_sample(P, d_.work, (int)work_.size(), d_wbeg_, d_from_, sample_every_, nbins_,
                        d_spart_, d_acc_, cap_);
  }
  cudaError_t e2 = cudaStreamEndCapture(cap_, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return set_error(DPD_ERR_CUDA, "graph capture failed: %s",
                     cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *out = nullptr;
    return set_error(DPD_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
  }
  return DPD_OK;
}

int Engine::step(int64_t nsteps) {
  NvtxRange range("dpd step");
  if (nsteps < 0) return set_error(DPD_ERR_ARG, "nsteps must be >= 0");
  if (ntot_ == 0 || nsteps == 0) {
    for (auto &s : st_host_) {
      const int64_t k = std::min<int64_t>(s.remaining, nsteps);
      s.step += (unsigned long long)k;
      s.remaining -= k;
      if (k > 0) s.pending = 1;
    }
    if (ntot_ == 0 && nsteps > 0) {
      DPD_CUDA_TRY(cudaMemcpyAsync(d_.st, st_host_.data(), st_host_.size() * sizeof(BoxState),
                                   cudaMemcpyHostToDevice, stream_));
    }
    return DPD_OK;
  }
  int64_t left = nsteps;
  if (graph_chunk > 1 && left >= graph_chunk) {
    if (!graph_) {
      int rc = capture_graph(graph_chunk, &graph_);
      if (rc) return rc;
    }
    while (left >= graph_chunk) {
      DPD_CUDA_TRY(cudaGraphLaunch(graph_, stream_));
      left -= graph_chunk;
    }
  }
  if (left == 1 && graph_chunk > 1) {  // one step: a cached one-step graph, one launch
    if (!graph1_) {
      int rc = capture_graph(1, &graph1_);
      if (rc) return rc;
    }
    DPD_CUDA_TRY(cudaGraphLaunch(graph1_, stream_));
    left = 0;
  }
  const Packed P = packed();
  const bool fz = fused_steps();  // the last step of the call stays plain: read-outs follow
  for (int64_t k = 0; k < left; ++k) {
    DPD_CUDA_TRY(launch_step(P, true, true, cfg_, stream_, fz && k > 0, fz && k + 1 < left));
    int rc = launch_extra(P, stream_);
    if (rc) return rc;
  }
  for (auto &s : st_host_) {
    const int64_t k = std::min<int64_t>(s.remaining, nsteps);
    s.step += (unsigned long long)k;
    s.remaining -= k;
    if (k > 0) s.pending = 1;
  }
  return DPD_OK;
}

int Engine::profile(int64_t nsteps, double *stage_ms) {
  for (int k = 0; k < kNumStages; ++k) stage_ms[k] = 0.0;
  if (nsteps <= 0 || ntot_ == 0) return step(nsteps);
  cudaEvent_t ev[kNumStages + 1] = {};
  for (auto &e : ev) DPD_CUDA_TRY(cudaEventCreate(&e));
  const Packed P = packed();
  int rc = DPD_OK;
  for (int64_t s = 0; s < nsteps && rc == DPD_OK; ++s) {
    cudaError_t e = launch_step_timed(P, cfg_, stream_, ev);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[kNumStages]);
    if (e != cudaSuccess) {
      rc = set_error(DPD_ERR_CUDA, "profiled step: %s", cudaGetErrorString(e));
      break;
    }
    for (int k = 0; k < kNumStages; ++k) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
      stage_ms[k] += ms / (double)nsteps;
    }
  }
  for (auto &e : ev) cudaEventDestroy(e);
  if (rc) return rc;
  for (auto &st : st_host_) {
    const int64_t k = std::min<int64_t>(st.remaining, nsteps);
    st.step += (unsigned long long)k;
    st.remaining -= k;
    if (k > 0) st.pending = 1;
  }
  return DPD_OK;
}

int Engine::sync() {
  DPD_CUDA_TRY(cudaStreamSynchronize(stream_));
  return DPD_OK;
}

int Engine::check_error() {
  int rc = fetch_error();
  if (rc) return rc;
  DPD_CUDA_TRY(cudaStreamSynchronize(stream_));
  return take_error();
}

int Engine::fetch_error() {
  DPD_CUDA_TRY(cudaMemcpyAsync(h_err_, d_.err, sizeof(unsigned), cudaMemcpyDeviceToHost, stream_));
  return DPD_OK;
}

int Engine::take_error() {
  const unsigned h = *h_err_;
  *h_err_ = 0u;
  if (h) {
    DPD_CUDA_TRY(cudaMemsetAsync(d_.err, 0, sizeof(unsigned), stream_));
    if (h & kErrBounds)
      return set_error(DPD_ERR_INTERNAL, "a kernel's index check failed (checked build)");
    if (h & kErrSpecies)
      return set_error(DPD_ERR_ARG, "a particle species is outside 0..nspec-1");
    if (h & kErrCapacity)
      return set_error(DPD_ERR_NUMERIC,
                       "local density beyond the brick force kernel's staging capacity "
                       "(select another force variant)");
    return set_error(DPD_ERR_NUMERIC, "device flagged %s%s",
                     (h & kErrNonFinite) ? "non-finite positions/velocities " : "",
                     (h & kErrRunaway) ? "a particle moving more than one box edge per step" : "");
  }
  return DPD_OK;
}

int Engine::gather(int box, float *pos, float *vel, float *frc, bool device_ptr) {
  NvtxRange range("dpd read state");
  if (box < 0 || box >= nbox()) return set_error(DPD_ERR_ARG, "box index out of range");
  const int n = pbase_[box + 1] - pbase_[box];
  const Packed P = packed();
  if (n == 0 || device_ptr) {
    if (n > 0) DPD_CUDA_TRY(launch_gather(P, box, pbase_[box], n, pos, vel, frc, stream_));
    int rc = fetch_error();
    if (rc) return rc;
    DPD_CUDA_TRY(cudaStreamSynchronize(stream_));
    return DPD_OK;
  }
  float *sp = reinterpret_cast<float *>(d_.pos2), *sv = reinterpret_cast<float *>(d_.vel2);
  const size_t bytes = (size_t)n * 3 * sizeof(float);
  if (pos || vel) {
    DPD_CUDA_TRY(launch_gather(P, box, pbase_[box], n, pos ? sp : nullptr, vel ? sv : nullptr,
                               nullptr, stream_));
    if (pos) DPD_CUDA_TRY(cudaMemcpyAsync(pos, sp, bytes, cudaMemcpyDeviceToHost, stream_));
    if (vel) DPD_CUDA_TRY(cudaMemcpyAsync(vel, sv, bytes, cudaMemcpyDeviceToHost, stream_));
  }
  if (frc) {
    DPD_CUDA_TRY(launch_gather(P, box, pbase_[box], n, nullptr, nullptr, sp, stream_));
    DPD_CUDA_TRY(cudaMemcpyAsync(frc, sp, bytes, cudaMemcpyDeviceToHost, stream_));
  }
  int rc = fetch_error();
  if (rc) return rc;
  DPD_CUDA_TRY(cudaStreamSynchronize(stream_));
  return DPD_OK;
}

int Engine::build_work() {
  const int nb = nbox();
  constexpr int kChunk = 4096;  // particles per statistics block
  work_.clear();
  wbeg_.assign(nb + 1, 0);
  for (int b = 0; b < nb; ++b) {
    wbeg_[b] = (int)work_.size();
    const int s0 = pbase_[b], s1 = pbase_[b + 1];
    if (s1 == s0) {
      work_.push_back(StatsWork{b, s0, s0, 0});
      continue;
    }
    for (int q = s0; q < s1; q += kChunk) work_.push_back(StatsWork{b, q, std::min(q + kChunk, s1), 0});
  }
  wbeg_[nb] = (int)work_.size();
  if (work_.size() + nb > d_.capW) {  // partials of the work items, then per-box totals
    if (d_.work) cudaFree(d_.work);
    if (d_.part) cudaFree(d_.part);
    d_.work = nullptr;
    d_.part = nullptr;
    const size_t cap = (work_.size() + nb) * 2;
    DPD_CUDA_TRY(cudaMalloc(&d_.work, cap * sizeof(StatsWork)));
    DPD_CUDA_TRY(cudaMalloc(&d_.part, cap * kStatsFields * sizeof(double)));
    d_.capW = cap;
  }
  if (wbeg_.size() > cap_wbeg_) {
    if (d_wbeg_) cudaFree(d_wbeg_);
    d_wbeg_ = nullptr;
    DPD_CUDA_TRY(cudaMalloc(&d_wbeg_, wbeg_.size() * 2 * sizeof(int)));
    cap_wbeg_ = wbeg_.size() * 2;
  }
  DPD_CUDA_TRY(cudaMemcpyAsync(d_.work, work_.data(), work_.size() * sizeof(StatsWork),
                               cudaMemcpyHostToDevice, stream_));
  DPD_CUDA_TRY(cudaMemcpyAsync(d_wbeg_, wbeg_.data(), wbeg_.size() * sizeof(int),
                               cudaMemcpyHostToDevice, stream_));
  work_dirty_ = false;
  return DPD_OK;
}

int Engine::copy_box_raw(int box, float4 *pos, float4 *vel, float4 *frc, bool to_host) {
  if (box < 0 || box >= nbox()) return set_error(DPD_ERR_ARG, "box index out of range");
  const size_t n = (size_t)(pbase_[box + 1] - pbase_[box]), o = (size_t)pbase_[box];
  const cudaMemcpyKind k = to_host ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice;
  float4 *dev[3] = {d_.pos + o, d_.vel + o, d_.frc + o};
  float4 *host[3] = {pos, vel, frc};
  for (int a = 0; a < 3; ++a) {
    if (!host[a] || n == 0) continue;
    if (to_host)
      DPD_CUDA_TRY(cudaMemcpyAsync(host[a], dev[a], n * sizeof(float4), k, stream_));
    else
      DPD_CUDA_TRY(cudaMemcpyAsync(dev[a], host[a], n * sizeof(float4), k, stream_));
  }
  DPD_CUDA_TRY(cudaStreamSynchronize(stream_));
  return DPD_OK;
}

int Engine::box_sums(std::vector<double> &sums) {
  NvtxRange range("dpd statistics");
  const int nb = nbox();
  if (work_dirty_) {
    int rc = build_work();
    if (rc) return rc;
  }
  // partial sums per work item, then per-box totals on the device (work
  // order), behind the partials in the same buffer; one small copy to pinned memory
  const size_t nsum = (size_t)nb * kStatsFields;
  if (nsum > cap_hsum_) {
    if (h_sum_) cudaFreeHost(h_sum_);
    h_sum_ = nullptr;
    DPD_CUDA_TRY(cudaMallocHost(&h_sum_, nsum * 2 * sizeof(double)));
    cap_hsum_ = nsum * 2;
  }
  double *box_out = d_.part + work_.size() * kStatsFields;  // capacity: work items + boxes
  DPD_CUDA_TRY(launch_stats(packed(), d_.work, (int)work_.size(), d_.part, stream_, d_wbeg_, nb,
                            box_out));
  DPD_CUDA_TRY(cudaMemcpyAsync(h_sum_, box_out, nsum * sizeof(double), cudaMemcpyDeviceToHost,
                               stream_));
  int rc = fetch_error();
  if (rc) return rc;
  DPD_CUDA_TRY(cudaStreamSynchronize(stream_));
  sums.assign(h_sum_, h_sum_ + nsum);
  return DPD_OK;
}

// ------------------------------------------------------------ served form
int Engine::enable_sampling(int every, int nbins) {
  if (every < 0 || nbins < 0 || nbins > 64)
    return set_error(DPD_ERR_ARG, "sampling: every >= 0, 0 <= nbins <= 64");
  sample_every_ = every;
  nbins_ = nbins;
  drop_graph();
  if (!boxes_.empty() && every > 0) return ensure_sampling_buffers();
  return DPD_OK;
}

int Engine::ensure_sampling_buffers() {
  const size_t nb = boxes_.size(), f = (size_t)sample_fields();
  if (nb > cap_from_) {
    if (d_from_) cudaFree(d_from_);
    d_from_ = nullptr;
    DPD_CUDA_TRY(cudaMalloc(&d_from_, nb * 2 * sizeof(long long)));
    cap_from_ = nb * 2;
    drop_graph();
  }
  if (nb * f > cap_acc_) {
    std::vector<double> keep;
    if (d_acc_) cudaFree(d_acc_);
    d_acc_ = nullptr;
    DPD_CUDA_TRY(cudaMalloc(&d_acc_, nb * f * 2 * sizeof(double)));
    DPD_CUDA_TRY(cudaMemsetAsync(d_acc_, 0, nb * f * 2 * sizeof(double), stream_));
    cap_acc_ = nb * f * 2;
    drop_graph();
  }
  if (work_.size() * f > cap_spart_) {
    if (d_spart_) cudaFree(d_spart_);
    d_spart_ = nullptr;
    DPD_CUDA_TRY(cudaMalloc(&d_spart_, work_.size() * f * 2 * sizeof(double)));
    cap_spart_ = work_.size() * f * 2;
    drop_graph();
  }
  return DPD_OK;
}

int Engine::launch_extra(const Packed &P, cudaStream_t s) {
  if (sample_every_ <= 0) return DPD_OK;
  DPD_CUDA_TRY(launch_sample(P, d_.work, (int)work_.size(), d_wbeg_, d_from_, sample_every_,
                             nbins_, d_spart_, d_acc_, s));
  return DPD_OK;
}

int Engine::zero_acc(int box) {
  if (box < 0 || box >= nbox() || !d_acc_) return set_error(DPD_ERR_ARG, "no accumulator");
  const size_t f = (size_t)sample_fields();
  DPD_CUDA_TRY(cudaMemsetAsync(d_acc_ + (size_t)box * f, 0, f * sizeof(double), stream_));
  return DPD_OK;
}

int Engine::read_acc(int box, double *out) {
  if (box < 0 || box >= nbox() || !d_acc_) return set_error(DPD_ERR_ARG, "no accumulator");
  const size_t f = (size_t)sample_fields();
  DPD_CUDA_TRY(cudaMemcpyAsync(out, d_acc_ + (size_t)box * f, f * sizeof(double),
                               cudaMemcpyDeviceToHost, stream_));
  DPD_CUDA_TRY(cudaStreamSynchronize(stream_));
  return DPD_OK;
}

int Engine::init_box(int box, uint64_t seed) {
  if (box < 0 || box >= nbox()) return set_error(DPD_ERR_ARG, "box index out of range");
  const BoxParams &bp = params_[box];
  const float vscale = (float)std::sqrt(bp.kT / bp.mass);
  DPD_CUDA_TRY(launch_init_box(packed(), pbase_[box], pbase_[box + 1] - pbase_[box],
                               (float)bp.L[0], (float)bp.L[1], (float)bp.L[2], vscale, seed,
                               stream_));
  return DPD_OK;
}

int Engine::repack(const std::vector<BoxParams> &params, const std::vector<int64_t> &np,
                   const std::vector<int> &src) {
  NvtxRange range("dpd repack");
  if (params.size() != np.size() || src.size() != np.size() || params.empty())
    return set_error(DPD_ERR_ARG, "repack: inconsistent sizes");
  const std::vector<int> old_pbase = pbase_;
  const std::vector<BoxState> old_st = st_host_;
  const std::vector<long long> old_from = from_h_;
  const int old_ntot = ntot_;
  const size_t f = (size_t)sample_fields();
  std::vector<double> old_acc;
  if (sample_every_ > 0 && d_acc_ && !boxes_.empty()) {
    old_acc.resize(boxes_.size() * f);
    DPD_CUDA_TRY(cudaMemcpyAsync(old_acc.data(), d_acc_, old_acc.size() * sizeof(double),
                                 cudaMemcpyDeviceToHost, stream_));
    DPD_CUDA_TRY(cudaStreamSynchronize(stream_));
  }
  std::vector<int> newbase(np.size() + 1, 0), src0(np.size(), -1);
  for (size_t k = 0; k < np.size(); ++k) {
    newbase[k + 1] = newbase[k] + (int)np[k];
    if (src[k] >= 0) {
      if (src[k] >= (int)old_st.size() || old_pbase[src[k] + 1] - old_pbase[src[k]] != np[k])
        return set_error(DPD_ERR_ARG, "repack: box %zu does not match its source", k);
      src0[k] = old_pbase[src[k]];
    }
  }
  const int new_ntot = newbase.back();
  int *d_nb = nullptr, *d_src = nullptr;
  DPD_CUDA_TRY(cudaMalloc(&d_nb, newbase.size() * sizeof(int)));
  DPD_CUDA_TRY(cudaMalloc(&d_src, src0.size() * sizeof(int)));
  DPD_CUDA_TRY(cudaMemcpyAsync(d_nb, newbase.data(), newbase.size() * sizeof(int),
                               cudaMemcpyHostToDevice, stream_));
  DPD_CUDA_TRY(cudaMemcpyAsync(d_src, src0.data(), src0.size() * sizeof(int),
                               cudaMemcpyHostToDevice, stream_));
  cudaError_t e = cudaSuccess;
  if ((size_t)new_ntot > d_.capP) {
    // grow: gather straight from the old arrays into new ones
    const size_t cap = std::max((size_t)new_ntot, d_.capP + d_.capP / 4);
    float4 *np_ = nullptr, *nv_ = nullptr;
    e = cudaMalloc(&np_, cap * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&nv_, cap * sizeof(float4));
    if (e == cudaSuccess)
      e = launch_repack(d_.pos, d_.vel, np_, nv_, d_nb, d_src, (int)np.size(), new_ntot, stream_);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream_);
    if (e != cudaSuccess) {
      if (np_) cudaFree(np_);
      if (nv_) cudaFree(nv_);
      cudaFree(d_nb);
      cudaFree(d_src);
      return set_error(e == cudaErrorMemoryAllocation ? DPD_ERR_NOMEM : DPD_ERR_CUDA,
                       "repack: %s", cudaGetErrorString(e));
    }
    float4 *keep_pos = np_, *keep_vel = nv_;
    drop_graph();
    void *olds[] = {d_.pos, d_.vel, d_.frc, d_.pos2, d_.vel2, d_.cellOf, d_.slotIn, d_.keyTmp};
    for (void *q : olds)
      if (q) cudaFree(q);
    d_.pos = d_.vel = d_.frc = d_.pos2 = d_.vel2 = nullptr;
    d_.cellOf = d_.slotIn = d_.keyTmp = nullptr;
    d_.capP = 0;
    int rc = reserve((size_t)new_ntot, 0, 0);   // allocates the rest at a new capacity
    if (rc) {
      cudaFree(keep_pos);
      cudaFree(keep_vel);
      cudaFree(d_nb);
      cudaFree(d_src);
      return rc;
    }
    cudaFree(d_.pos);
    cudaFree(d_.vel);
    d_.pos = keep_pos;
    d_.vel = keep_vel;
  } else {
    e = cudaMemcpyAsync(d_.pos2, d_.pos, (size_t)old_ntot * sizeof(float4),
                        cudaMemcpyDeviceToDevice, stream_);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_.vel2, d_.vel, (size_t)old_ntot * sizeof(float4),
                          cudaMemcpyDeviceToDevice, stream_);
    if (e == cudaSuccess)
      e = launch_repack(d_.pos2, d_.vel2, d_.pos, d_.vel, d_nb, d_src, (int)np.size(), new_ntot,
                        stream_);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream_);
    if (e != cudaSuccess) {
      cudaFree(d_nb);
      cudaFree(d_src);
      return set_error(DPD_ERR_CUDA, "repack: %s", cudaGetErrorString(e));
    }
  }
  cudaFree(d_nb);
  cudaFree(d_src);
  int rc = layout(params, np);
  if (rc) return rc;
  for (size_t k = 0; k < np.size(); ++k) {
    if (src[k] >= 0) {
      st_host_[k] = old_st[src[k]];
      from_h_[k] = old_from[src[k]];
    }
  }
  if (sample_every_ > 0) {
    std::vector<double> acc(np.size() * f, 0.0);
    for (size_t k = 0; k < np.size(); ++k)
      if (src[k] >= 0 && !old_acc.empty())
        std::copy(old_acc.begin() + (size_t)src[k] * f, old_acc.begin() + (size_t)(src[k] + 1) * f,
                  acc.begin() + k * f);
    DPD_CUDA_TRY(cudaMemcpyAsync(d_acc_, acc.data(), acc.size() * sizeof(double),
                                 cudaMemcpyHostToDevice, stream_));
    DPD_CUDA_TRY(cudaStreamSynchronize(stream_));
  }
  return DPD_OK;
}

}  // namespace dpd
