// C ABI of the single-box context (dpd_*) and the debug entry points.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>

#include "dpd.h"
#include "engine.h"

namespace dpd {
const char *last_error_text();
}

using dpd::BoxParams;
using dpd::Engine;

struct dpd_ctx {
  Engine eng;
  BoxParams bp{};
  int64_t n = 0;
  bool loaded = false;
  int tiles = 0, tile_cells = 0, stage_cap = 0;
};

extern "C" {

static_assert(DPD_MAX_SPECIES == dpd::kMaxSpecies, "species limit of the header and the kernels");

const char *dpd_last_error(void) { return dpd::last_error_text(); }

#define DPD_STR2(x) #x
#define DPD_STR(x) DPD_STR2(x)
const char *dpd_version(void) {
#if defined(DPD_CHECKED) && DPD_CHECKED
  return "gb300-dpd 0.1 (sm_103a, Philox-4x32-" DPD_STR(DPD_PHILOX_ROUNDS) ", checked)";
#else
  return "gb300-dpd 0.1 (sm_103a, Philox-4x32-" DPD_STR(DPD_PHILOX_ROUNDS) ")";
#endif
}

int dpd_philox_rounds(void) { return DPD_PHILOX_ROUNDS; }

int dpd_create(dpd_ctx **out, const double box[3], double a, double gamma, double kT, double rc,
               double dt, uint64_t seed) {
  dpd::clear_error();
  if (!out || !box) return dpd::set_error(DPD_ERR_ARG, "null argument");
  *out = nullptr;
  BoxParams bp{};
  for (int k = 0; k < 3; ++k) bp.L[k] = box[k];
  bp.a = a;
  bp.gamma = gamma;
  bp.kT = kT;
  bp.rc = rc;
  bp.dt = dt;
  bp.mass = 1.0;
  bp.kexp = 1.0;
  bp.fb = 0.0;
  bp.fb_mode = 0;
  bp.fb_flow = 2;
  bp.fb_grad = 0;
  bp.seed = seed;
  int ncell[3];
  int rc_ = dpd::check_params(bp, ncell);
  if (rc_) return rc_;
  dpd_ctx *c = new (std::nothrow) dpd_ctx();
  if (!c) return dpd::set_error(DPD_ERR_NOMEM, "host allocation failed");
  c->bp = bp;
  rc_ = c->eng.init();
  if (rc_) {
    delete c;
    return rc_;
  }
  *out = c;
  return DPD_OK;
}

int dpd_destroy(dpd_ctx *ctx) {
  delete ctx;
  return DPD_OK;
}

int dpd_set_param(dpd_ctx *ctx, int key, double value) {
  dpd::clear_error();
  if (!ctx) return dpd::set_error(DPD_ERR_ARG, "null context");
  BoxParams bp = ctx->bp;
  auto axis = [&](int &dst) -> int {
    if (!(value == 0.0 || value == 1.0 || value == 2.0))
      return dpd::set_error(DPD_ERR_ARG, "axis must be 0, 1 or 2");
    dst = (int)value;
    return DPD_OK;
  };
  int rc = DPD_OK;
  switch (key) {
    case DPD_PARAM_KEXP: bp.kexp = value; break;
    case DPD_PARAM_MASS: bp.mass = value; break;
    case DPD_PARAM_BODYFORCE:
      bp.fb = value;
      bp.fb_mode = (value != 0.0) ? 1 : 0;
      break;
    case DPD_PARAM_POISEUILLE_F:
      bp.fb = value;
      bp.fb_mode = (value != 0.0) ? 2 : 0;
      break;
    case DPD_PARAM_FLOW_AXIS: rc = axis(bp.fb_flow); break;
    case DPD_PARAM_GRAD_AXIS: rc = axis(bp.fb_grad); break;
    case DPD_PARAM_STENCIL:
      if (!(value == DPD_STENCIL_FULL || value == DPD_STENCIL_HALF))
        return dpd::set_error(DPD_ERR_ARG, "stencil must be DPD_STENCIL_FULL or DPD_STENCIL_HALF");
      return ctx->eng.set_stencil((int)value);
    case DPD_PARAM_FORCE_TILES:
    case DPD_PARAM_TILE_CELLS:
    case DPD_PARAM_STAGE_CAP: {
      if (!(value >= 0.0 && value <= 1e6) || value != (double)(int)value)
        return dpd::set_error(DPD_ERR_ARG, "tiling parameters are non-negative integers");
      int t = ctx->tiles, c = ctx->tile_cells, cap = ctx->stage_cap;
      if (key == DPD_PARAM_FORCE_TILES) t = (value != 0.0);
      if (t && ctx->bp.nspec > 1)
        return dpd::set_error(DPD_ERR_ARG, "the staged force tiles serve one species only");
      if (key == DPD_PARAM_TILE_CELLS) c = (int)value;
      if (key == DPD_PARAM_STAGE_CAP) cap = (int)value;
      rc = ctx->eng.set_tiling(t, c, cap);
      if (rc) return rc;
      ctx->tiles = t;
      ctx->tile_cells = c;
      ctx->stage_cap = cap;
      return DPD_OK;
    }
    case DPD_PARAM_NOISE:
      if (!(value == DPD_NOISE_UNIFORM || value == DPD_NOISE_GAUSSIAN))
        return dpd::set_error(DPD_ERR_ARG, "noise must be DPD_NOISE_UNIFORM or DPD_NOISE_GAUSSIAN");
      bp.noise = (int)value;
      break;
    case DPD_PARAM_FORCE_VARIANT:
      if (!(value >= -1.0 && value < DPD_NUM_FORCE_VARIANTS) || value != std::floor(value))
        return dpd::set_error(DPD_ERR_ARG, "force variant must be -1..%d",
                              DPD_NUM_FORCE_VARIANTS - 1);
      return ctx->eng.set_variant((int)value);
    case DPD_PARAM_FUSE:
      if (!(value == 0.0 || value == 1.0)) return dpd::set_error(DPD_ERR_ARG, "fuse must be 0 or 1");
      return ctx->eng.set_fuse(value != 0.0);
    default: return dpd::set_error(DPD_ERR_ARG, "unknown parameter key %d", key);
  }
  if (rc) return rc;
  int ncell[3];
  rc = dpd::check_params(bp, ncell);
  if (rc) return rc;
  ctx->bp = bp;
  if (ctx->loaded) return ctx->eng.update_params({bp});
  return DPD_OK;
}

int dpd_get_param(const dpd_ctx *ctx, int key, double *value) {
  dpd::clear_error();
  if (!ctx || !value) return dpd::set_error(DPD_ERR_ARG, "null argument");
  const BoxParams &bp = ctx->bp;
  const dpd::StepConfig &cfg = ctx->eng.step_config();
  switch (key) {
    case DPD_PARAM_KEXP: *value = bp.kexp; break;
    case DPD_PARAM_MASS: *value = bp.mass; break;
    case DPD_PARAM_BODYFORCE: *value = bp.fb_mode == 1 ? bp.fb : 0.0; break;
    case DPD_PARAM_POISEUILLE_F: *value = bp.fb_mode == 2 ? bp.fb : 0.0; break;
    case DPD_PARAM_FLOW_AXIS: *value = bp.fb_flow; break;
    case DPD_PARAM_GRAD_AXIS: *value = bp.fb_grad; break;
    case DPD_PARAM_STENCIL: *value = cfg.stencil; break;
    case DPD_PARAM_FORCE_TILES: *value = cfg.tiles ? 1.0 : 0.0; break;
    case DPD_PARAM_TILE_CELLS: *value = ctx->loaded ? cfg.grid.tc : ctx->tile_cells; break;
    case DPD_PARAM_STAGE_CAP: *value = ctx->loaded ? cfg.grid.stage_cap : ctx->stage_cap; break;
    case DPD_PARAM_NOISE: *value = bp.noise; break;
    case DPD_PARAM_FORCE_VARIANT:
      *value = (ctx->loaded && cfg.nbands > 0) ? cfg.band[0].variant : ctx->eng.variant_override();
      break;
    case DPD_PARAM_FUSE: *value = ctx->eng.fuse() ? 1.0 : 0.0; break;
    default: return dpd::set_error(DPD_ERR_ARG, "unknown parameter key %d", key);
  }
  return DPD_OK;
}

int dpd_set_stream(dpd_ctx *ctx, void *stream) {
  dpd::clear_error();
  if (!ctx) return dpd::set_error(DPD_ERR_ARG, "null context");
  return ctx->eng.set_stream((cudaStream_t)stream);
}

int dpd_set_state_species(dpd_ctx *ctx, int64_t n, const float *pos, const float *vel,
                          const int32_t *species, int where) {
  dpd::clear_error();
  if (!ctx) return dpd::set_error(DPD_ERR_ARG, "null context");
  if (n < 0 || n > dpd::kMaxSlots) return dpd::set_error(DPD_ERR_ARG, "bad particle count");
  if (where != DPD_WHERE_HOST && where != DPD_WHERE_DEVICE)
    return dpd::set_error(DPD_ERR_ARG, "where must be DPD_WHERE_HOST or DPD_WHERE_DEVICE");
  if (n > 0 && (!pos || !vel)) return dpd::set_error(DPD_ERR_ARG, "null position or velocity");
  if (species && where == DPD_WHERE_HOST)
    for (int64_t i = 0; i < n; ++i)
      if (species[i] < 0 || species[i] >= ctx->bp.nspec)
        return dpd::set_error(DPD_ERR_ARG, "particle %lld: species %d outside 0..%d",
                              (long long)i, species[i], ctx->bp.nspec - 1);
  // a loaded context of the same size keeps its layout (its parameters
  // reach the engine as they change)
  const bool same = ctx->loaded && ctx->eng.restart_same_layout({n});
  ctx->loaded = false;
  int rc = same ? DPD_OK : ctx->eng.layout({ctx->bp}, {n});
  if (rc) return rc;
  rc = ctx->eng.load_box(0, pos, vel, where == DPD_WHERE_DEVICE, species);
  if (rc) return rc;
  ctx->eng.set_box_state(0, 0, INT64_MAX / 4);
  rc = ctx->eng.rebuild();
  if (rc) return rc;
  if (species && where == DPD_WHERE_DEVICE && (rc = ctx->eng.check_error())) return rc;
  ctx->n = n;
  ctx->loaded = true;
  return DPD_OK;
}

int dpd_set_state(dpd_ctx *ctx, int64_t n, const float *pos, const float *vel, int where) {
  return dpd_set_state_species(ctx, n, pos, vel, nullptr, where);
}

int dpd_set_species(dpd_ctx *ctx, int nspecies, const double *a, const double *gamma,
                    const double *rc) {
  dpd::clear_error();
  if (!ctx) return dpd::set_error(DPD_ERR_ARG, "null context");
  if (nspecies < 1 || nspecies > dpd::kMaxSpecies)
    return dpd::set_error(DPD_ERR_ARG, "species count must be 1..%d", dpd::kMaxSpecies);
  if (nspecies > 1 && (!a || !gamma || !rc)) return dpd::set_error(DPD_ERR_ARG, "null table");
  if (ctx->loaded && nspecies != ctx->bp.nspec)
    return dpd::set_error(DPD_ERR_STATE,
                          "the species count changes only before dpd_set_state_species");
  if (nspecies > 1 && ctx->tiles)
    return dpd::set_error(DPD_ERR_ARG, "the staged force tiles serve one species only");
  BoxParams bp = ctx->bp;
  bp.nspec = nspecies;
  for (int k = 0; k < 16; ++k) bp.sa[k] = bp.sg[k] = bp.src[k] = 0.0;
  for (int s = 0; s < nspecies && nspecies > 1; ++s)
    for (int t = 0; t < nspecies; ++t) {
      bp.sa[4 * s + t] = a[nspecies * s + t];
      bp.sg[4 * s + t] = gamma[nspecies * s + t];
      bp.src[4 * s + t] = rc[nspecies * s + t];
    }
  int ncell[3];
  int r = dpd::check_params(bp, ncell);
  if (r) return r;
  ctx->bp = bp;
  if (ctx->loaded) return ctx->eng.update_params({bp});
  return DPD_OK;
}

int dpd_get_species(const dpd_ctx *ctx, int *nspecies, double *a, double *gamma, double *rc) {
  dpd::clear_error();
  if (!ctx || !nspecies) return dpd::set_error(DPD_ERR_ARG, "null argument");
  const BoxParams &bp = ctx->bp;
  *nspecies = bp.nspec;
  for (int s = 0; s < bp.nspec && bp.nspec > 1; ++s)
    for (int t = 0; t < bp.nspec; ++t) {
      if (a) a[bp.nspec * s + t] = bp.sa[4 * s + t];
      if (gamma) gamma[bp.nspec * s + t] = bp.sg[4 * s + t];
      if (rc) rc[bp.nspec * s + t] = bp.src[4 * s + t];
    }
  return DPD_OK;
}

int dpd_step(dpd_ctx *ctx, int64_t nsteps) {
  dpd::clear_error();
  if (!ctx) return dpd::set_error(DPD_ERR_ARG, "null context");
  if (!ctx->loaded) return dpd::set_error(DPD_ERR_STATE, "dpd_step before dpd_set_state");
  return ctx->eng.step(nsteps);
}

int dpd_get_state(dpd_ctx *ctx, float *pos, float *vel, int where) {
  dpd::clear_error();
  if (!ctx) return dpd::set_error(DPD_ERR_ARG, "null context");
  if (!ctx->loaded) return dpd::set_error(DPD_ERR_STATE, "no state loaded");
  if (where != DPD_WHERE_HOST && where != DPD_WHERE_DEVICE)
    return dpd::set_error(DPD_ERR_ARG, "bad where");
  int rc = ctx->eng.gather(0, pos, vel, nullptr, where == DPD_WHERE_DEVICE);
  if (rc) return rc;
  return ctx->eng.take_error();
}

int dpd_get_forces(dpd_ctx *ctx, float *force, int where) {
  dpd::clear_error();
  if (!ctx) return dpd::set_error(DPD_ERR_ARG, "null context");
  if (!ctx->loaded) return dpd::set_error(DPD_ERR_STATE, "no state loaded");
  if (where != DPD_WHERE_HOST && where != DPD_WHERE_DEVICE)
    return dpd::set_error(DPD_ERR_ARG, "bad where");
  int rc = ctx->eng.gather(0, nullptr, nullptr, force, where == DPD_WHERE_DEVICE);
  if (rc) return rc;
  return ctx->eng.take_error();
}

int dpd_get_stats(dpd_ctx *ctx, dpd_stats *out) {
  dpd::clear_error();
  if (!ctx || !out) return dpd::set_error(DPD_ERR_ARG, "null argument");
  if (!ctx->loaded) return dpd::set_error(DPD_ERR_STATE, "no state loaded");
  std::vector<double> s;
  int rc = ctx->eng.box_sums(s);
  if (rc) return rc;
  const BoxParams &bp = ctx->bp;
  const double m = bp.mass, V = bp.L[0] * bp.L[1] * bp.L[2];
  const int64_t n = ctx->n;
  for (int k = 0; k < 3; ++k) out->momentum[k] = m * s[k];
  out->kinetic = 0.5 * m * s[3];
  out->kT = (n > 1) ? 2.0 * out->kinetic / (3.0 * (double)(n - 1)) : 0.0;
  out->virial = 0.5 * s[4];  // each pair was counted by both members
  out->pressure = (double)n * out->kT / V + out->virial / (3.0 * V);
  out->step = (int64_t)ctx->eng.box_state(0).step;
  out->n = n;
  return ctx->eng.take_error();  // fetched with the sums
}

namespace {
struct CheckpointHeader {
  char magic[8];       // "DPDCKPT2"
  int64_t n;
  double box[3], a, gamma, kT, rc, dt;
  uint64_t seed;
  unsigned long long step;
  long long remaining;
  int pending, stencil;
  int nspec, pad_;
  double sa[16], sg[16], src[16];
};
}  // namespace

int64_t dpd_checkpoint_size(const dpd_ctx *ctx) {
  if (!ctx) return 0;
  return (int64_t)sizeof(CheckpointHeader) + ctx->n * 3 * (int64_t)sizeof(float4);
}

int dpd_checkpoint_save(dpd_ctx *ctx, void *buf, int64_t bytes) {
  dpd::clear_error();
  if (!ctx || !buf) return dpd::set_error(DPD_ERR_ARG, "null argument");
  if (!ctx->loaded) return dpd::set_error(DPD_ERR_STATE, "no state loaded");
  if (bytes < dpd_checkpoint_size(ctx))
    return dpd::set_error(DPD_ERR_ARG, "buffer of %lld bytes, need %lld", (long long)bytes,
                          (long long)dpd_checkpoint_size(ctx));
  CheckpointHeader h{};
  std::memcpy(h.magic, "DPDCKPT2", 8);
  h.n = ctx->n;
  for (int k = 0; k < 3; ++k) h.box[k] = ctx->bp.L[k];
  h.a = ctx->bp.a;
  h.gamma = ctx->bp.gamma;
  h.kT = ctx->bp.kT;
  h.rc = ctx->bp.rc;
  h.dt = ctx->bp.dt;
  h.seed = ctx->bp.seed;
  const dpd::BoxState &st = ctx->eng.box_state(0);
  h.step = st.step;
  h.remaining = st.remaining;
  h.pending = st.pending;
  h.stencil = ctx->eng.step_config().stencil;
  h.nspec = ctx->bp.nspec;
  std::memcpy(h.sa, ctx->bp.sa, sizeof h.sa);
  std::memcpy(h.sg, ctx->bp.sg, sizeof h.sg);
  std::memcpy(h.src, ctx->bp.src, sizeof h.src);
  std::memcpy(buf, &h, sizeof h);
  float4 *arr = reinterpret_cast<float4 *>(static_cast<char *>(buf) + sizeof h);
  return ctx->eng.copy_box_raw(0, arr, arr + ctx->n, arr + 2 * ctx->n, true);
}

int dpd_checkpoint_load(dpd_ctx *ctx, const void *buf, int64_t bytes) {
  dpd::clear_error();
  if (!ctx || !buf) return dpd::set_error(DPD_ERR_ARG, "null argument");
  if (bytes < (int64_t)sizeof(CheckpointHeader))
    return dpd::set_error(DPD_ERR_ARG, "buffer too small for a checkpoint");
  CheckpointHeader h;
  std::memcpy(&h, buf, sizeof h);
  if (std::memcmp(h.magic, "DPDCKPT2", 8) != 0)
    return dpd::set_error(DPD_ERR_STATE, "not a checkpoint");
  const dpd::BoxParams &bp = ctx->bp;
  if (h.box[0] != bp.L[0] || h.box[1] != bp.L[1] || h.box[2] != bp.L[2] || h.a != bp.a ||
      h.gamma != bp.gamma || h.kT != bp.kT || h.rc != bp.rc || h.dt != bp.dt || h.seed != bp.seed ||
      h.nspec != bp.nspec || std::memcmp(h.sa, bp.sa, sizeof h.sa) != 0 ||
      std::memcmp(h.sg, bp.sg, sizeof h.sg) != 0 || std::memcmp(h.src, bp.src, sizeof h.src) != 0)
    return dpd::set_error(DPD_ERR_STATE, "checkpoint was made with other box parameters");
  if (h.n < 0 || bytes < (int64_t)sizeof h + h.n * 3 * (int64_t)sizeof(float4))
    return dpd::set_error(DPD_ERR_ARG, "checkpoint buffer truncated");
  ctx->loaded = false;
  int rc = ctx->eng.layout({ctx->bp}, {h.n});
  if (rc) return rc;
  const float4 *arr = reinterpret_cast<const float4 *>(static_cast<const char *>(buf) + sizeof h);
  rc = ctx->eng.copy_box_raw(0, const_cast<float4 *>(arr), const_cast<float4 *>(arr + h.n),
                             const_cast<float4 *>(arr + 2 * h.n), false);
  if (rc) return rc;
  dpd::BoxState st{h.step, h.remaining, h.pending, 1};
  ctx->eng.set_box_state_raw(0, st);
  rc = ctx->eng.set_stencil(h.stencil);
  if (rc) return rc;
  rc = ctx->eng.rebuild();  // cell list from the saved order; force recomputed at the saved step
  if (rc) return rc;
  ctx->n = h.n;
  ctx->loaded = true;
  return DPD_OK;
}

int dpd_profile_steps(dpd_ctx *ctx, int64_t nsteps, double *stage_ms) {
  dpd::clear_error();
  if (!ctx || !stage_ms) return dpd::set_error(DPD_ERR_ARG, "null argument");
  if (!ctx->loaded) return dpd::set_error(DPD_ERR_STATE, "no state loaded");
  if (nsteps < 0) return dpd::set_error(DPD_ERR_ARG, "nsteps must be >= 0");
  return ctx->eng.profile(nsteps, stage_ms);
}

int64_t dpd_num_particles(const dpd_ctx *ctx) { return ctx ? ctx->n : 0; }

int dpd_debug_rng(const uint32_t *lo, const uint32_t *hi, int64_t n, uint64_t step, uint64_t seed,
                  int noise, uint32_t *out0, uint32_t *out1, float *xi, void *stream) {
  dpd::clear_error();
  if (n < 0) return dpd::set_error(DPD_ERR_ARG, "negative count");
  if (noise != DPD_NOISE_UNIFORM && noise != DPD_NOISE_GAUSSIAN)
    return dpd::set_error(DPD_ERR_ARG, "bad noise mode");
  if (n == 0) return DPD_OK;
  if (!lo || !hi || !out0) return dpd::set_error(DPD_ERR_ARG, "null device pointer");
  cudaStream_t s = (cudaStream_t)stream;
  DPD_CUDA_TRY(dpd::launch_debug_rng(lo, hi, n, step, seed, noise, out0, out1, xi, s));
  DPD_CUDA_TRY(cudaStreamSynchronize(s));
  return DPD_OK;
}

}  // extern "C"
