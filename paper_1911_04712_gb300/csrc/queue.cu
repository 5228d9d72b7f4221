// C ABI of the served form (dpd_queue_*): continuous batching of
// independent DPD runs on one GPU.
//
// A worker thread owns an Engine whose packed set is the resident requests.
// It runs the resident boxes in chunks of steps; between chunks it retires
// the boxes that reached their step count (reading their accumulated
// statistics into results) and admits waiting requests while the HBM ledger
// and the resident-box limit allow, then repacks the survivors and the new
// boxes into one layout.  A new box's initial state is the caller's (copied
// at submission by dpd_queue_submit_state) or drawn on the device from its
// seed.  Every box is stepped and sampled at its own step indices,
// so a request's result does not depend on what else was resident.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dpd.h"
#include "engine.h"

using dpd::BoxParams;
using dpd::Engine;

namespace {

using Clock = std::chrono::steady_clock;

// A caller's initial state (n x 3 positions then n x 3 velocities, host).
using InitState = std::shared_ptr<const std::vector<float>>;

struct Pending {
  uint64_t ticket;
  BoxParams bp;
  int64_t n, steps;
  size_t bytes;
  double t_submit;
  InitState init;          // null: drawn on the device from the seed
  bool keep_final = false;  // keep the final state for dpd_queue_final_state
};

struct Resident {
  uint64_t ticket;
  BoxParams bp;
  int64_t n, steps;
  size_t bytes;
  double t_submit, t_admit;
  InitState init;
  bool keep_final = false;
};

// Cell-list entries (x slices of the cells) of a request's box.
int64_t request_cells(const BoxParams &bp) {
  int64_t c = dpd::kSlicesX;
  for (int k = 0; k < 3; ++k) c *= (int64_t)std::floor(bp.L[k] / bp.rc);
  return c;
}

size_t request_bytes(const BoxParams &bp, int64_t n) {
  // particle arrays (5 float4 + 3 int32) and cell arrays (2 int32), plus slack
  return (size_t)n * (5 * 16 + 3 * 4) + (size_t)request_cells(bp) * 2 * 4 + 4096;
}

}  // namespace

struct dpd_queue {
  Engine eng;
  int device = 0;
  cudaStream_t stream = nullptr;
  dpd_queue_opts opts{};
  size_t budget = 0, in_use = 0;
  std::mutex mu;
  std::condition_variable cv, cv_done;
  std::deque<Pending> pending;
  std::vector<Resident> resident;  // engine box order
  std::unordered_map<uint64_t, dpd_result> done;
  std::unordered_map<uint64_t, std::vector<float>> finals;  // kept final states (id order)
  std::unordered_map<uint64_t, int> state;  // 0 pending, 1 resident, 2 done
  uint64_t next_ticket = 1;
  bool stop = false;
  int error = DPD_OK;
  std::string error_text;
  std::thread worker;
  Clock::time_point t0 = Clock::now();
  double busy_s = 0.0;
  long double particle_steps = 0.0;
  int64_t admitted = 0, completed = 0;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

static void finish_locked(dpd_queue *q, const Resident &r, const double *acc, int status) {
  if (q->state[r.ticket] == 2) return;  // finished once only
  dpd_result res{};
  res.status = status;
  res.n = r.n;
  res.steps = r.steps;
  res.t_submit = r.t_submit;
  res.t_admit = r.t_admit;
  res.t_done = q->now();
  const int nb = q->opts.nbins;
  res.nbins = nb;
  if (acc && status == DPD_OK) {
    const double S = acc[0];
    const double V = r.bp.L[0] * r.bp.L[1] * r.bp.L[2];
    res.samples = (int64_t)S;
    if (S > 0 && r.n > 1) {
      res.kT_mean = r.bp.mass * acc[1] / (3.0 * (double)(r.n - 1) * S);
      const double vir = 0.5 * acc[2] / S;
      res.pressure_mean = (double)r.n * res.kT_mean / V + vir / (3.0 * V);
    }
    for (int b = 0; b < nb && b < 64; ++b)
      res.profile[b] = acc[3 + nb + b] > 0 ? acc[3 + b] / acc[3 + nb + b] : 0.0;
  }
  q->done[r.ticket] = res;
  q->state[r.ticket] = 2;
  q->in_use -= r.bytes;  // the ledger is released when a request finishes
  q->completed++;
}

// Block until the queue's stream has finished, up to `limit_s` seconds.
static int wait_stream(dpd_queue *q, double limit_s) {
  cudaEvent_t ev;
  DPD_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  DPD_CUDA_TRY(cudaEventRecord(ev, q->stream));
  const auto t0 = Clock::now();
  for (;;) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) {
      cudaEventDestroy(ev);
      return dpd::set_error(DPD_ERR_CUDA, "queue stream: %s", cudaGetErrorString(e));
    }
    if (std::chrono::duration<double>(Clock::now() - t0).count() > limit_s) {
      cudaEventDestroy(ev);
      return dpd::set_error(DPD_ERR_TIMEOUT, "queue chunk did not finish in %.0f s", limit_s);
    }
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
  cudaEventDestroy(ev);
  return DPD_OK;
}

static void fail_all_locked(dpd_queue *q, int code) {
  q->error = code;
  q->error_text = dpd_last_error();
  for (const auto &r : q->resident) finish_locked(q, r, nullptr, code);
  q->resident.clear();
  while (!q->pending.empty()) {
    const Pending p = q->pending.front();
    q->pending.pop_front();
    Resident r{p.ticket, p.bp, p.n, p.steps, p.bytes, p.t_submit, q->now()};
    q->in_use += p.bytes;
    finish_locked(q, r, nullptr, code);
  }
  q->cv_done.notify_all();
}

static bool identity(const std::vector<int> &src) {
  for (size_t k = 0; k < src.size(); ++k)
    if (src[k] != (int)k) return false;
  return true;
}

static void worker_main(dpd_queue *q) {
  cudaSetDevice(q->device);
  const int fields = 3 + 2 * q->opts.nbins;
  for (;;) {
    std::vector<int> src;
    std::vector<Resident> next;
    std::vector<char> fresh;
    std::vector<char> done_before;  // finished or cancelled before this chunk
    {
      std::unique_lock<std::mutex> lk(q->mu);
      q->cv.wait_for(lk, std::chrono::milliseconds(20),
                     [&] { return q->stop || !q->pending.empty() || !q->resident.empty(); });
      if (q->stop) return;
      if (q->error) {
        fail_all_locked(q, q->error);
        continue;
      }
      // boundary.  Finished (or cancelled) runs stay in the packed set,
      // frozen, until a re-layout pays: when nothing runs any more, when
      // they hold an eighth of the set's particles, or when waiting runs
      // could be admitted (at once, or by dropping finished runs that hold
      // a thirty-second of the set or free a slot under the box limit).  A re-layout drops them and admits
      // waiting runs; otherwise the set and its captured graphs are kept.
      int64_t all_n = 0, dead_n = 0, slots_all = 0, cells_all = 0;
      size_t dead_b = 0;
      for (const auto &r : q->resident) {
        all_n += r.n;
        slots_all += r.n;
        cells_all += request_cells(r.bp);
        if (q->state[r.ticket] == 2) {
          dead_n += r.n;
          ++dead_b;
        }
      }
      bool relayout = dead_b == q->resident.size() || dead_n * 8 >= all_n;
      if (!relayout && !q->pending.empty()) {
        auto it = q->pending.begin();
        if (q->opts.policy == 1)
          it = std::min_element(q->pending.begin(), q->pending.end(),
                                [](const Pending &a, const Pending &b) {
                                  return (double)a.n * a.steps < (double)b.n * b.steps;
                                });
        const bool fits = q->in_use + it->bytes <= q->budget &&
                          (int64_t)q->resident.size() < q->opts.max_boxes &&
                          slots_all + it->n <= dpd::kMaxSlots &&
                          cells_all + request_cells(it->bp) <= dpd::kMaxCellEntries;
        // a full box limit is freed by dropping any finished run
        relayout = fits || (dead_b > 0 && (dead_n * 32 >= all_n ||
                                           (int64_t)q->resident.size() >= q->opts.max_boxes));
      }
      if (!relayout) {
        for (size_t k = 0; k < q->resident.size(); ++k) {
          next.push_back(q->resident[k]);
          src.push_back((int)k);
          fresh.push_back(0);
          done_before.push_back(q->state[q->resident[k].ticket] == 2 ? 1 : 0);
        }
      } else {
        for (size_t k = 0; k < q->resident.size(); ++k) {
          if (q->state[q->resident[k].ticket] == 2) continue;
          next.push_back(q->resident[k]);
          src.push_back((int)k);
          fresh.push_back(0);
          done_before.push_back(0);
        }
      }
      // admit waiting requests while the ledger, the box limit and the packed
      // set's slot and cell capacity allow
      int64_t slots = 0, cells = 0;
      for (const auto &r : next) {
        slots += r.n;
        cells += request_cells(r.bp);
      }
      while (relayout && !q->pending.empty() && (int64_t)next.size() < q->opts.max_boxes) {
        auto it = q->pending.begin();
        if (q->opts.policy == 1)
          it = std::min_element(q->pending.begin(), q->pending.end(),
                                [](const Pending &a, const Pending &b) {
                                  return (double)a.n * a.steps < (double)b.n * b.steps;
                                });
        if (q->in_use + it->bytes > q->budget) break;
        if (slots + it->n > dpd::kMaxSlots || cells + request_cells(it->bp) > dpd::kMaxCellEntries)
          break;
        slots += it->n;
        cells += request_cells(it->bp);
        next.push_back(Resident{it->ticket, it->bp, it->n, it->steps, it->bytes, it->t_submit,
                                q->now(), it->init, it->keep_final});
        q->in_use += it->bytes;
        q->state[it->ticket] = 1;
        q->admitted++;
        q->pending.erase(it);
        src.push_back(-1);
        fresh.push_back(1);
        done_before.push_back(0);
      }
      bool live = false;
      for (size_t k = 0; k < next.size(); ++k) live = live || !done_before[k];
      q->resident = next;
      if (next.empty() || !live) continue;
    }
    int rc = DPD_OK;
    if (q->eng.nbox() != (int)next.size() || !identity(src)) {
      std::vector<BoxParams> params;
      std::vector<int64_t> np;
      for (const auto &r : next) {
        params.push_back(r.bp);
        np.push_back(r.n);
      }
      rc = q->eng.repack(params, np, src);
      for (size_t k = 0; rc == DPD_OK && k < next.size(); ++k) {
        if (!fresh[k]) continue;
        if (next[k].init) {
          const float *x = next[k].init->data();
          rc = q->eng.load_box((int)k, x, x + 3 * next[k].n, false);
        } else {
          rc = q->eng.init_box((int)k, next[k].bp.seed);
        }
        if (rc == DPD_OK) {
          q->eng.set_box_state((int)k, 0, next[k].steps);
          q->eng.set_sample_from((int)k, next[k].steps / 2);
          rc = q->eng.zero_acc((int)k);
        }
      }
      if (rc == DPD_OK) rc = q->eng.rebuild();
    }
    // cancelled runs still in the set stop moving
    for (int k = 0; rc == DPD_OK && k < q->eng.nbox(); ++k)
      if (done_before[k] && q->eng.box_state(k).remaining > 0) rc = q->eng.set_remaining(k, 0);
    // one chunk, ending no later than the earliest finish of a running box
    int64_t chunk = q->opts.chunk_steps;
    long double ps = 0.0;
    for (int k = 0; k < q->eng.nbox(); ++k)
      if (q->eng.box_state(k).remaining > 0)
        chunk = std::min<int64_t>(chunk, q->eng.box_state(k).remaining);
    for (int k = 0; k < q->eng.nbox(); ++k)
      ps += (long double)q->eng.box_n(k) *
            (long double)std::min<int64_t>(chunk, q->eng.box_state(k).remaining);
    const auto tc = Clock::now();
    if (rc == DPD_OK) rc = q->eng.step(chunk);
    if (rc == DPD_OK) rc = wait_stream(q, q->opts.chunk_timeout_s);
    if (rc == DPD_OK) rc = q->eng.check_error();
    const double dt = std::chrono::duration<double>(Clock::now() - tc).count();
    // read out the boxes that reached their step count
    std::vector<std::pair<int, std::vector<double>>> outs;
    std::vector<std::pair<uint64_t, std::vector<float>>> fin;
    for (int k = 0; rc == DPD_OK && k < q->eng.nbox(); ++k) {
      if (!done_before[k] && q->eng.box_state(k).remaining <= 0) {
        std::vector<double> acc(fields);
        rc = q->eng.read_acc(k, acc.data());
        outs.emplace_back(k, std::move(acc));
        if (rc == DPD_OK && q->resident[k].keep_final) {
          const int64_t n = q->resident[k].n;
          std::vector<float> xv((size_t)(6 * n));
          rc = q->eng.gather(k, xv.data(), xv.data() + 3 * n, nullptr, false);
          if (rc == DPD_OK) rc = q->eng.take_error();
          fin.emplace_back(q->resident[k].ticket, std::move(xv));
        }
      }
    }
    std::lock_guard<std::mutex> lk(q->mu);
    if (rc != DPD_OK) {
      fail_all_locked(q, rc);
      continue;
    }
    q->busy_s += dt;
    q->particle_steps += ps;
    for (auto &f : fin) q->finals[f.first] = std::move(f.second);
    for (auto &o : outs) finish_locked(q, q->resident[o.first], o.second.data(), DPD_OK);
    if (!outs.empty()) q->cv_done.notify_all();
  }
}

extern "C" {

int dpd_queue_create(dpd_queue **out, size_t hbm_budget_bytes, const dpd_queue_opts *opts) {
  dpd::clear_error();
  if (!out) return dpd::set_error(DPD_ERR_ARG, "null argument");
  *out = nullptr;
  if (hbm_budget_bytes == 0) return dpd::set_error(DPD_ERR_ARG, "HBM budget must be > 0");
  dpd_queue_opts o{};
  if (opts) o = *opts;
  if (o.max_boxes <= 0) o.max_boxes = 4096;
  if (o.chunk_steps <= 0) o.chunk_steps = 100;
  if (o.sample_every <= 0) o.sample_every = 20;
  if (o.nbins < 0 || o.nbins > 64) return dpd::set_error(DPD_ERR_ARG, "nbins must be 0..64");
  if (o.nbins == 0) o.nbins = 16;
  if (o.policy != 0 && o.policy != 1) return dpd::set_error(DPD_ERR_ARG, "policy must be 0 or 1");
  if (o.stencil != 0 && o.stencil != 1) return dpd::set_error(DPD_ERR_ARG, "bad stencil");
  if (!(o.chunk_timeout_s > 0)) o.chunk_timeout_s = 600.0;
  dpd_queue *q = new (std::nothrow) dpd_queue();
  if (!q) return dpd::set_error(DPD_ERR_NOMEM, "host allocation failed");
  q->opts = o;
  q->budget = hbm_budget_bytes;
  int rc = q->eng.init();
  if (!rc) {
    cudaGetDevice(&q->device);
    cudaError_t e = cudaStreamCreateWithFlags(&q->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) rc = dpd::set_error(DPD_ERR_CUDA, "%s", cudaGetErrorString(e));
  }
  if (!rc) rc = q->eng.set_stream(q->stream);
  if (!rc) rc = q->eng.set_stencil(o.stencil);
  if (!rc) rc = q->eng.enable_sampling((int)o.sample_every, o.nbins);
  if (rc) {
    if (q->stream) cudaStreamDestroy(q->stream);
    delete q;
    return rc;
  }
  q->worker = std::thread(worker_main, q);
  *out = q;
  return DPD_OK;
}

int dpd_queue_destroy(dpd_queue *q) {
  if (!q) return DPD_OK;
  {
    std::lock_guard<std::mutex> lk(q->mu);
    q->stop = true;
  }
  q->cv.notify_all();
  if (q->worker.joinable()) q->worker.join();
  cudaStream_t s = q->stream;
  delete q;
  if (s) cudaStreamDestroy(s);
  return DPD_OK;
}

}  // extern "C"

static int submit(dpd_queue *q, const dpd_request *req, const float *pos, const float *vel,
                  bool keep_final, uint64_t *ticket) {
  dpd::clear_error();
  if (!q || !req || !ticket) return dpd::set_error(DPD_ERR_ARG, "null argument");
  BoxParams bp{};
  for (int k = 0; k < 3; ++k) bp.L[k] = req->box[k];
  bp.a = req->a;
  bp.gamma = req->gamma;
  bp.kT = req->kT;
  bp.rc = req->rc;
  bp.dt = req->dt;
  bp.mass = 1.0;
  bp.kexp = 1.0;
  bp.fb = req->body_force;
  bp.fb_mode = req->body_force == 0.0 ? 0 : req->body_mode;
  bp.fb_flow = req->flow_axis;
  bp.fb_grad = req->grad_axis;
  bp.seed = req->seed;
  bp.noise = req->noise;
  int nc[3];
  int rc = dpd::check_params(bp, nc);
  if (rc) return rc;
  if (req->steps <= 0) return dpd::set_error(DPD_ERR_ARG, "steps must be > 0");
  int64_t n = req->n;
  if (n <= 0) {
    if (!(req->rho > 0)) return dpd::set_error(DPD_ERR_ARG, "give n > 0 or rho > 0");
    n = (int64_t)std::llround(req->rho * bp.L[0] * bp.L[1] * bp.L[2]);
  }
  if (n < 2 || n > dpd::kMaxSlots)
    return dpd::set_error(DPD_ERR_ARG, "particle count out of range");
  InitState init;
  if (pos || vel) {
    if (!pos || !vel) return dpd::set_error(DPD_ERR_ARG, "give both positions and velocities");
    if (req->n <= 0) return dpd::set_error(DPD_ERR_ARG, "a caller's state needs n > 0");
    auto v = std::make_shared<std::vector<float>>((size_t)(6 * n));
    std::memcpy(v->data(), pos, (size_t)n * 3 * sizeof(float));
    std::memcpy(v->data() + 3 * n, vel, (size_t)n * 3 * sizeof(float));
    init = v;
  }
  const size_t bytes = request_bytes(bp, n);
  std::lock_guard<std::mutex> lk(q->mu);
  if (q->error) return dpd::set_error(q->error, "queue failed earlier: %s", q->error_text.c_str());
  if (bytes > q->budget)
    return dpd::set_error(DPD_ERR_NOMEM, "request needs %zu bytes, budget is %zu", bytes,
                          q->budget);
  const uint64_t t = q->next_ticket++;
  q->pending.push_back(Pending{t, bp, n, req->steps, bytes, q->now(), init, keep_final});
  q->state[t] = 0;
  *ticket = t;
  q->cv.notify_all();
  return DPD_OK;
}

extern "C" {

int dpd_queue_submit(dpd_queue *q, const dpd_request *req, uint64_t *ticket) {
  return submit(q, req, nullptr, nullptr, false, ticket);
}

int dpd_queue_submit_state(dpd_queue *q, const dpd_request *req, const float *pos,
                           const float *vel, int keep_final, uint64_t *ticket) {
  if (!pos || !vel) {
    dpd::clear_error();
    return dpd::set_error(DPD_ERR_ARG, "null position or velocity array");
  }
  return submit(q, req, pos, vel, keep_final != 0, ticket);
}

int dpd_queue_final_state(dpd_queue *q, uint64_t ticket, float *pos, float *vel) {
  dpd::clear_error();
  if (!q || !pos || !vel) return dpd::set_error(DPD_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lk(q->mu);
  auto it = q->state.find(ticket);
  if (it == q->state.end()) return dpd::set_error(DPD_ERR_ARG, "unknown ticket");
  if (it->second != 2) return dpd::set_error(DPD_ERR_BUSY, "request %llu not finished",
                                             (unsigned long long)ticket);
  auto f = q->finals.find(ticket);
  if (f == q->finals.end())
    return dpd::set_error(DPD_ERR_STATE, "request %llu kept no final state",
                          (unsigned long long)ticket);
  const size_t half = f->second.size() / 2;
  std::memcpy(pos, f->second.data(), half * sizeof(float));
  std::memcpy(vel, f->second.data() + half, half * sizeof(float));
  return DPD_OK;
}

int dpd_queue_poll(dpd_queue *q, uint64_t ticket, int *done) {
  dpd::clear_error();
  if (!q || !done) return dpd::set_error(DPD_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lk(q->mu);
  auto it = q->state.find(ticket);
  if (it == q->state.end()) return dpd::set_error(DPD_ERR_ARG, "unknown ticket %llu",
                                                  (unsigned long long)ticket);
  *done = it->second == 2;
  return DPD_OK;
}

int dpd_queue_result(dpd_queue *q, uint64_t ticket, dpd_result *out) {
  dpd::clear_error();
  if (!q || !out) return dpd::set_error(DPD_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lk(q->mu);
  auto it = q->state.find(ticket);
  if (it == q->state.end()) return dpd::set_error(DPD_ERR_ARG, "unknown ticket");
  if (it->second != 2) return dpd::set_error(DPD_ERR_BUSY, "request %llu not finished",
                                             (unsigned long long)ticket);
  *out = q->done[ticket];
  return DPD_OK;
}

int dpd_queue_cancel(dpd_queue *q, uint64_t ticket) {
  dpd::clear_error();
  if (!q) return dpd::set_error(DPD_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lk(q->mu);
  auto it = q->state.find(ticket);
  if (it == q->state.end()) return dpd::set_error(DPD_ERR_ARG, "unknown ticket");
  if (it->second == 2) return DPD_OK;
  for (auto p = q->pending.begin(); p != q->pending.end(); ++p) {
    if (p->ticket == ticket) {
      Resident r{p->ticket, p->bp, p->n, p->steps, p->bytes, p->t_submit, q->now()};
      q->in_use += p->bytes;
      q->pending.erase(p);
      finish_locked(q, r, nullptr, DPD_ERR_STATE);
      q->cv_done.notify_all();
      return DPD_OK;
    }
  }
  for (const auto &r : q->resident)
    if (r.ticket == ticket) finish_locked(q, r, nullptr, DPD_ERR_STATE);  // dropped at the next boundary
  q->cv_done.notify_all();
  return DPD_OK;
}

int dpd_queue_wait_all(dpd_queue *q, double timeout_s) {
  dpd::clear_error();
  if (!q) return dpd::set_error(DPD_ERR_ARG, "null argument");
  std::unique_lock<std::mutex> lk(q->mu);
  auto idle = [&] {
    if (!q->pending.empty()) return false;
    for (const auto &r : q->resident)
      if (q->state[r.ticket] != 2) return false;
    return true;
  };
  const bool ok = q->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), idle);
  if (!ok) return dpd::set_error(DPD_ERR_TIMEOUT, "requests still running after %.1f s", timeout_s);
  if (q->error) return dpd::set_error(q->error, "%s", q->error_text.c_str());
  return DPD_OK;
}

int dpd_queue_get_stats(dpd_queue *q, dpd_queue_stats *out) {
  dpd::clear_error();
  if (!q || !out) return dpd::set_error(DPD_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lk(q->mu);
  out->pending = (int64_t)q->pending.size();
  int64_t res = 0;
  for (const auto &r : q->resident)
    if (q->state[r.ticket] != 2) res++;
  out->resident = res;
  out->admitted = q->admitted;
  out->completed = q->completed;
  out->bytes_in_use = q->in_use;
  out->particle_steps = (double)q->particle_steps;
  out->busy_seconds = q->busy_s;
  out->clock_seconds = q->now();
  return DPD_OK;
}

}  // extern "C"
