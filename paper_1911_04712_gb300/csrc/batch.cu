// C ABI of the multi-box batch (dpd_batch_*) and of the kernel tuning table.
//
// The batch packer orders the boxes by density band (so that every band is a
// contiguous slot range with one force-kernel variant), lays them out in one
// Engine, and maps the caller's box indices to packed positions.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>
#include <numeric>
#include <vector>

#include "dpd.h"
#include "engine.h"

using dpd::BoxParams;
using dpd::Engine;

struct dpd_batch {
  Engine eng;
  std::vector<BoxParams> params;  // caller order
  std::vector<int64_t> n;
  std::vector<int64_t> steps;
  std::vector<int> slot;          // packed position of caller box b
  std::vector<char> loaded;
  int nloaded = 0;
  bool dirty = true;
  int tiles = 0, tile_cells = 0, stage_cap = 0;
};

static int batch_ready(dpd_batch *b) {
  if (b->nloaded < (int)b->params.size())
    return dpd::set_error(DPD_ERR_STATE, "%d of %d boxes have no state yet",
                          (int)b->params.size() - b->nloaded, (int)b->params.size());
  if (b->dirty) {
    int rc = b->eng.rebuild();
    if (rc) return rc;
    b->dirty = false;
  }
  return DPD_OK;
}

static int box_index(const dpd_batch *b, int box) {
  if (box < 0 || box >= (int)b->params.size())
    return dpd::set_error(DPD_ERR_ARG, "box %d out of range (batch has %d)", box,
                          (int)b->params.size());
  return DPD_OK;
}

extern "C" {

int dpd_force_variant_info(int v, int *threads, int *list_capacity) {
  dpd::clear_error();
  if (!threads || !list_capacity) return dpd::set_error(DPD_ERR_ARG, "null argument");
  if (dpd::force_variant_info(v, threads, list_capacity))
    return dpd::set_error(DPD_ERR_ARG, "variant %d out of range", v);
  return DPD_OK;
}

int dpd_tuning_set(int table, int nbands, const double *rho_upper, const int *variant) {
  dpd::clear_error();
  if (!rho_upper || !variant) return dpd::set_error(DPD_ERR_ARG, "null argument");
  if (dpd::tuning_set(table, nbands, rho_upper, variant))
    return dpd::set_error(DPD_ERR_ARG,
                          "bad tuning table (table 0..3, 1..%d bands, increasing bounds, "
                          "variants 0..%d)",
                          DPD_MAX_DENSITY_BANDS, DPD_NUM_FORCE_VARIANTS - 1);
  return DPD_OK;
}

int dpd_tuning_get(int table, int max, double *rho_upper, int *variant, int *nbands) {
  dpd::clear_error();
  if (!nbands) return dpd::set_error(DPD_ERR_ARG, "null argument");
  const int n = dpd::tuning_get(table, max, rho_upper, variant);
  if (n < 0) return dpd::set_error(DPD_ERR_ARG, "table must be 0..3");
  *nbands = n;
  return DPD_OK;
}

int dpd_batch_create(dpd_batch **out, int nbox, const dpd_box_desc *descs) {
  dpd::clear_error();
  if (!out) return dpd::set_error(DPD_ERR_ARG, "null argument");
  *out = nullptr;
  if (nbox <= 0 || !descs) return dpd::set_error(DPD_ERR_ARG, "a batch needs at least one box");
  std::vector<BoxParams> params(nbox);
  std::vector<int64_t> n(nbox), steps(nbox);
  std::vector<int> band(nbox);
  for (int i = 0; i < nbox; ++i) {
    const dpd_box_desc &d = descs[i];
    BoxParams bp{};
    for (int k = 0; k < 3; ++k) bp.L[k] = d.box[k];
    bp.a = d.a;
    bp.gamma = d.gamma;
    bp.kT = d.kT;
    bp.rc = d.rc;
    bp.dt = d.dt;
    bp.mass = d.mass == 0.0 ? 1.0 : d.mass;
    bp.kexp = d.kexp == 0.0 ? 1.0 : d.kexp;
    bp.fb = d.body_force;
    bp.fb_mode = d.body_force == 0.0 ? 0 : d.body_mode;
    bp.fb_flow = d.flow_axis;
    bp.fb_grad = d.grad_axis;
    bp.seed = d.seed;
    bp.noise = d.noise;
    bp.nspec = d.nspecies <= 1 ? 1 : d.nspecies;
    if (bp.nspec > 1)
      for (int k = 0; k < DPD_MAX_SPECIES * DPD_MAX_SPECIES; ++k) {
        bp.sa[k] = d.species_a[k];
        bp.sg[k] = d.species_gamma[k];
        bp.src[k] = d.species_rc[k];
      }
    int nc[3];
    int rc = dpd::check_params(bp, nc);
    if (rc) return dpd::set_error(rc, "box %d: %s", i, dpd_last_error());
    if (d.n < 0) return dpd::set_error(DPD_ERR_ARG, "box %d: negative particle count", i);
    params[i] = bp;
    n[i] = d.n;
    steps[i] = d.steps > 0 ? d.steps : INT64_MAX / 4;
    const double rho = (double)d.n / (d.box[0] * d.box[1] * d.box[2]);
    band[i] = dpd::tuned_band(DPD_TUNING_PACKED, rho);  // density band of the packed tables
  }
  // pack by density band, keeping the caller's order inside a band
  std::vector<int> order(nbox);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return band[x] < band[y]; });
  dpd_batch *b = new (std::nothrow) dpd_batch();
  if (!b) return dpd::set_error(DPD_ERR_NOMEM, "host allocation failed");
  b->params = params;
  b->n = n;
  b->steps = steps;
  b->slot.assign(nbox, 0);
  b->loaded.assign(nbox, 0);
  std::vector<BoxParams> packed_params(nbox);
  std::vector<int64_t> packed_n(nbox);
  for (int k = 0; k < nbox; ++k) {
    b->slot[order[k]] = k;
    packed_params[k] = params[order[k]];
    packed_n[k] = n[order[k]];
  }
  int rc = b->eng.init();
  if (!rc) rc = b->eng.layout(packed_params, packed_n);
  if (rc) {
    delete b;
    return rc;
  }
  b->eng.graph_chunk = 32;
  *out = b;
  return DPD_OK;
}

int dpd_batch_destroy(dpd_batch *b) {
  delete b;
  return DPD_OK;
}

int dpd_batch_num_boxes(const dpd_batch *b) { return b ? (int)b->params.size() : 0; }

int dpd_batch_set_stream(dpd_batch *b, void *stream) {
  dpd::clear_error();
  if (!b) return dpd::set_error(DPD_ERR_ARG, "null batch");
  return b->eng.set_stream((cudaStream_t)stream);
}

int dpd_batch_set_option(dpd_batch *b, int key, double value) {
  dpd::clear_error();
  if (!b) return dpd::set_error(DPD_ERR_ARG, "null batch");
  auto as_int = [&](int lo, int hi, int *v) -> int {
    if (!(value >= lo && value <= hi) || value != std::floor(value))
      return dpd::set_error(DPD_ERR_ARG, "option %d must be an integer in %d..%d", key, lo, hi);
    *v = (int)value;
    return DPD_OK;
  };
  int v = 0, rc = DPD_OK;
  switch (key) {
    case DPD_PARAM_STENCIL:
      if ((rc = as_int(0, 1, &v))) return rc;
      return b->eng.set_stencil(v);
    case DPD_PARAM_FORCE_VARIANT:
      if ((rc = as_int(-1, DPD_NUM_FORCE_VARIANTS - 1, &v))) return rc;
      return b->eng.set_variant(v);
    case DPD_PARAM_FUSE:
      if ((rc = as_int(0, 1, &v))) return rc;
      return b->eng.set_fuse(v != 0);
    case DPD_PARAM_FORCE_TILES:
    case DPD_PARAM_TILE_CELLS:
    case DPD_PARAM_STAGE_CAP: {
      if ((rc = as_int(0, 1 << 20, &v))) return rc;
      int t = b->tiles, c = b->tile_cells, cap = b->stage_cap;
      if (key == DPD_PARAM_FORCE_TILES) t = v != 0;
      for (const BoxParams &bp : b->params)
        if (t && bp.nspec > 1)
          return dpd::set_error(DPD_ERR_ARG, "the staged force tiles serve one species only");
      if (key == DPD_PARAM_TILE_CELLS) c = v;
      if (key == DPD_PARAM_STAGE_CAP) cap = v;
      if ((rc = b->eng.set_tiling(t, c, cap))) return rc;
      b->tiles = t;
      b->tile_cells = c;
      b->stage_cap = cap;
      return DPD_OK;
    }
    case DPD_BATCH_GRAPH_CHUNK:
      if ((rc = as_int(1, 1 << 20, &v))) return rc;
      b->eng.graph_chunk = v;
      return b->eng.refresh_bands();
    default: return dpd::set_error(DPD_ERR_ARG, "unknown batch option %d", key);
  }
}

int dpd_batch_set_state_species(dpd_batch *b, int box, const float *pos, const float *vel,
                                const int32_t *species, int where) {
  dpd::clear_error();
  if (!b) return dpd::set_error(DPD_ERR_ARG, "null batch");
  int rc = box_index(b, box);
  if (rc) return rc;
  if (where != DPD_WHERE_HOST && where != DPD_WHERE_DEVICE)
    return dpd::set_error(DPD_ERR_ARG, "bad where");
  const int nspec = b->params[box].nspec;
  if (species && where == DPD_WHERE_HOST)
    for (int64_t i = 0; i < b->n[box]; ++i)
      if (species[i] < 0 || species[i] >= nspec)
        return dpd::set_error(DPD_ERR_ARG, "box %d, particle %lld: species %d outside 0..%d", box,
                              (long long)i, species[i], nspec - 1);
  const int k = b->slot[box];
  rc = b->eng.load_box(k, pos, vel, where == DPD_WHERE_DEVICE, species);
  if (rc) return rc;
  if (species && where == DPD_WHERE_DEVICE && (rc = b->eng.check_error())) return rc;
  b->eng.set_box_state(k, 0, b->steps[box]);
  if (!b->loaded[box]) {
    b->loaded[box] = 1;
    b->nloaded++;
  }
  b->dirty = true;
  return DPD_OK;
}

int dpd_batch_set_state(dpd_batch *b, int box, const float *pos, const float *vel, int where) {
  return dpd_batch_set_state_species(b, box, pos, vel, nullptr, where);
}

int dpd_batch_step(dpd_batch *b, int64_t nsteps) {
  dpd::clear_error();
  if (!b) return dpd::set_error(DPD_ERR_ARG, "null batch");
  if (nsteps < 0) return dpd::set_error(DPD_ERR_ARG, "nsteps must be >= 0");
  int rc = batch_ready(b);
  if (rc) return rc;
  return b->eng.step(nsteps);
}

int dpd_batch_profile_steps(dpd_batch *b, int64_t nsteps, double *stage_ms) {
  dpd::clear_error();
  if (!b || !stage_ms) return dpd::set_error(DPD_ERR_ARG, "null argument");
  if (nsteps < 0) return dpd::set_error(DPD_ERR_ARG, "nsteps must be >= 0");
  int rc = batch_ready(b);
  if (rc) return rc;
  return b->eng.profile(nsteps, stage_ms);
}

int dpd_batch_get_state(dpd_batch *b, int box, float *pos, float *vel, int where) {
  dpd::clear_error();
  if (!b) return dpd::set_error(DPD_ERR_ARG, "null batch");
  int rc = box_index(b, box);
  if (rc) return rc;
  if (where != DPD_WHERE_HOST && where != DPD_WHERE_DEVICE)
    return dpd::set_error(DPD_ERR_ARG, "bad where");
  if ((rc = batch_ready(b))) return rc;
  rc = b->eng.gather(b->slot[box], pos, vel, nullptr, where == DPD_WHERE_DEVICE);
  if (rc) return rc;
  return b->eng.take_error();
}

int dpd_batch_get_forces(dpd_batch *b, int box, float *force, int where) {
  dpd::clear_error();
  if (!b) return dpd::set_error(DPD_ERR_ARG, "null batch");
  int rc = box_index(b, box);
  if (rc) return rc;
  if (where != DPD_WHERE_HOST && where != DPD_WHERE_DEVICE)
    return dpd::set_error(DPD_ERR_ARG, "bad where");
  if ((rc = batch_ready(b))) return rc;
  rc = b->eng.gather(b->slot[box], nullptr, nullptr, force, where == DPD_WHERE_DEVICE);
  if (rc) return rc;
  return b->eng.take_error();
}

int dpd_batch_get_stats(dpd_batch *b, dpd_stats *out) {
  dpd::clear_error();
  if (!b || !out) return dpd::set_error(DPD_ERR_ARG, "null argument");
  int rc = batch_ready(b);
  if (rc) return rc;
  std::vector<double> s;
  if ((rc = b->eng.box_sums(s))) return rc;
  for (int box = 0; box < (int)b->params.size(); ++box) {
    const int k = b->slot[box];
    const double *q = &s[(size_t)k * dpd::kStatsFields];
    const BoxParams &bp = b->params[box];
    const double m = bp.mass, V = bp.L[0] * bp.L[1] * bp.L[2];
    const int64_t n = b->n[box];
    dpd_stats &o = out[box];
    for (int c = 0; c < 3; ++c) o.momentum[c] = m * q[c];
    o.kinetic = 0.5 * m * q[3];
    o.kT = (n > 1) ? 2.0 * o.kinetic / (3.0 * (double)(n - 1)) : 0.0;
    o.virial = 0.5 * q[4];
    o.pressure = (double)n * o.kT / V + o.virial / (3.0 * V);
    o.step = (int64_t)b->eng.box_state(k).step;
    o.n = n;
  }
  return b->eng.take_error();  // fetched with the sums
}

}  // extern "C"
