// Request loop with continuous batching: FSLBM runs of different domain
// sizes are admitted as device memory and slots free up, stay resident on
// the device, and advance together in the shared launches of a batch
// (fslbm_batch_*); finished runs are read back, retired and their memory
// returned for the next admissions.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "fslbm_ctx.h"

using namespace fslbm;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
  int64_t id = 0;
  fslbm_domain dom{};
  fslbm_bc_variant variant = FSLBM_OM;
  fslbm_params prm{};
  std::vector<double> fill, vel, den;
  std::vector<uint8_t> flags;
  int steps = 0;
  size_t bytes = 0;
  double t_submit = 0.0;
};

struct Active {
  Req r;
  fslbm_ctx* ctx = nullptr;
  int done = 0;
  double t_admit = 0.0;
};

struct Done {
  fslbm_result res{};
  std::vector<double> fill;
  std::vector<uint8_t> flags;
};

}  // namespace

struct fslbm_server {
  fslbm_server_config cfg{};
  cudaStream_t stream = nullptr;
  std::deque<Req> queue;
  std::vector<Active> active;
  fslbm_batch* batch = nullptr;
  bool dirty = false;
  std::map<int64_t, Done> done;
  int64_t next_id = 1;
  size_t used = 0;
  size_t budget = 0;
  fslbm_server_stats st{};
  std::string err;
};

namespace {

fslbm_status sfail(fslbm_server* s, fslbm_status e, const std::string& msg) {
  if (s) s->err = msg;
  return e;
}

void drop_batch(fslbm_server* s) {
  if (s->batch) {
    fslbm_batch_destroy(s->batch);
    s->batch = nullptr;
  }
}

// Retire finished runs: read back fill levels, flags and observables.
fslbm_status retire(fslbm_server* s) {
  const double t = now_s();
  for (size_t k = 0; k < s->active.size();) {
    Active& a = s->active[k];
    if (a.done < a.r.steps) {
      ++k;
      continue;
    }
    Done d;
    const size_t N = (size_t)a.r.dom.nx * a.r.dom.ny * a.r.dom.nz;
    d.fill.resize(N);
    d.flags.resize(N);
    fslbm_status e = fslbm_read_fields(a.ctx, nullptr, d.fill.data(), d.flags.data(), nullptr);
    fslbm_obs obs{};
    const fslbm_status eo = fslbm_observables(a.ctx, &obs);
    if (e == FSLBM_OK) e = eo;
    d.res.id = a.r.id;
    d.res.status = (int)e;
    d.res.steps = a.done;
    d.res.obs = obs;
    d.res.cells = (int64_t)N;
    d.res.t_queue = a.t_admit - a.r.t_submit;
    d.res.t_result = t - a.r.t_submit;
    s->st.completed += 1;
    s->st.cell_updates += (double)N * a.done;
    s->done[a.r.id] = std::move(d);
    fslbm_destroy(a.ctx);
    s->used -= a.r.bytes;
    s->active.erase(s->active.begin() + (long)k);
    s->dirty = true;
  }
  return FSLBM_OK;
}

// Admit queued requests in arrival order while slots and memory allow.
fslbm_status admit(fslbm_server* s) {
  while (!s->queue.empty() && (int)s->active.size() < s->cfg.max_active) {
    Req& r = s->queue.front();
    if (s->used + r.bytes > s->budget && !s->active.empty()) break;  // wait for memory
    fslbm_ctx* c = nullptr;
    r.prm.stream = (void*)s->stream;
    fslbm_status e = fslbm_create(&r.dom, s->cfg.lattice, s->cfg.collision, r.variant, &r.prm, &c);
    if (e == FSLBM_ENOMEM && !s->active.empty()) break;  // retry after a retirement
    if (e == FSLBM_OK)
      e = fslbm_init(c, r.fill.data(), r.flags.data(), r.vel.empty() ? nullptr : r.vel.data(),
                     r.den.empty() ? nullptr : r.den.data());
    if (e != FSLBM_OK) {
      // the request cannot run: report it as finished with its status
      Done d;
      d.res.id = r.id;
      d.res.status = (int)e;
      d.res.t_result = now_s() - r.t_submit;
      s->done[r.id] = std::move(d);
      if (c) fslbm_destroy(c);
      s->queue.pop_front();
      continue;
    }
    Active a;
    a.r = std::move(r);
    a.ctx = c;
    a.t_admit = now_s();
    s->used += a.r.bytes;
    s->active.push_back(std::move(a));
    s->queue.pop_front();
    s->dirty = true;
    s->st.admitted += 1;
    if (s->active.size() > (size_t)s->st.max_active_seen) s->st.max_active_seen = (int)s->active.size();
  }
  return FSLBM_OK;
}

}  // namespace

extern "C" {

fslbm_status fslbm_server_create(const fslbm_server_config* cfg, fslbm_server** out) {
  if (!cfg || !out || cfg->max_active < 1 || cfg->chunk_steps < 1) return FSLBM_EINVAL;
  if (cfg->lattice != FSLBM_D3Q19 && cfg->lattice != FSLBM_D3Q27) return FSLBM_EINVAL;
  if (cfg->collision != FSLBM_SRT && cfg->collision != FSLBM_TRT) return FSLBM_EINVAL;
  if (cfg->precision < FSLBM_FP64 || cfg->precision > FSLBM_FP16SMC) return FSLBM_EINVAL;
  fslbm_server* s = new (std::nothrow) fslbm_server();
  if (!s) return FSLBM_ENOMEM;
  s->cfg = *cfg;
  s->stream = (cudaStream_t)cfg->stream;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    delete s;
    return FSLBM_ECUDA;
  }
  s->budget = cfg->memory_budget > 0 ? (size_t)cfg->memory_budget : (size_t)(0.9 * (double)fr);
  *out = s;
  return FSLBM_OK;
}

fslbm_status fslbm_server_submit(fslbm_server* s, const fslbm_request* rq, int64_t* id) {
  if (!s || !rq || !rq->fill || !rq->flags || rq->steps < 0) return FSLBM_EINVAL;
  if (rq->params.precision != s->cfg.precision)
    return sfail(s, FSLBM_EINVAL, "request precision differs from the server's");
  if (rq->params.bubble_model && rq->params.bubble_relabel_every > 0)
    return sfail(s, FSLBM_EINVAL, "bubble relabelling runs in single-domain contexts only");
  Req r;
  r.dom = rq->domain;
  r.variant = rq->bc_variant;
  r.prm = rq->params;
  r.steps = rq->steps;
  fslbm_status e = fslbm_memory_estimate(&r.dom, s->cfg.lattice, s->cfg.precision,
                                         rq->velocity != nullptr, &r.bytes);
  if (e != FSLBM_OK) return sfail(s, e, "bad domain");
  if (r.bytes > s->budget) return sfail(s, FSLBM_ENOMEM, "request larger than the memory budget");
  const size_t N = (size_t)r.dom.nx * r.dom.ny * r.dom.nz;
  r.fill.assign(rq->fill, rq->fill + N);
  r.flags.assign(rq->flags, rq->flags + N);
  if (rq->velocity) r.vel.assign(rq->velocity, rq->velocity + 3 * N);
  if (rq->density) r.den.assign(rq->density, rq->density + N);
  r.id = s->next_id++;
  r.t_submit = now_s();
  s->queue.push_back(std::move(r));
  s->st.submitted += 1;
  if (id) *id = s->queue.back().id;
  return FSLBM_OK;
}

fslbm_status fslbm_server_poll(fslbm_server* s, int* n_active) {
  if (!s) return FSLBM_EINVAL;
  fslbm_status e = admit(s);
  if (e != FSLBM_OK) return e;
  if (!s->active.empty()) {
    if (s->dirty || !s->batch) {
      drop_batch(s);
      std::vector<fslbm_ctx*> m;
      for (const Active& a : s->active) m.push_back(a.ctx);
      e = fslbm_batch_create(m.data(), (int)m.size(), (void*)s->stream, &s->batch);
      if (e != FSLBM_OK) return sfail(s, e, "batch creation failed");
      s->dirty = false;
      s->st.batch_rebuilds += 1;
    }
    int k = s->cfg.chunk_steps;
    for (const Active& a : s->active) k = std::min(k, a.r.steps - a.done);
    if (k > 0) {
      e = fslbm_batch_step(s->batch, k);
      if (e != FSLBM_OK) return sfail(s, e, fslbm_batch_last_error(s->batch));
      e = fslbm_batch_sync(s->batch, nullptr);
      if (e != FSLBM_OK && e != FSLBM_EUNSTABLE) return sfail(s, e, fslbm_batch_last_error(s->batch));
      for (Active& a : s->active) a.done += k;
      s->st.batch_steps += k;
    }
    e = retire(s);
    if (e != FSLBM_OK) return e;
  }
  if (n_active) *n_active = (int)s->active.size();
  return FSLBM_OK;
}

fslbm_status fslbm_server_result(fslbm_server* s, int64_t id, fslbm_result* res, double* fill,
                                 uint8_t* flags) {
  if (!s || !res) return FSLBM_EINVAL;
  auto it = s->done.find(id);
  if (it == s->done.end()) return FSLBM_ESTATE;  // not finished (or unknown)
  *res = it->second.res;
  if (fill && !it->second.fill.empty())
    std::memcpy(fill, it->second.fill.data(), it->second.fill.size() * sizeof(double));
  if (flags && !it->second.flags.empty())
    std::memcpy(flags, it->second.flags.data(), it->second.flags.size());
  s->done.erase(it);
  return FSLBM_OK;
}

fslbm_status fslbm_server_stats_get(const fslbm_server* s, fslbm_server_stats* out) {
  if (!s || !out) return FSLBM_EINVAL;
  *out = s->st;
  out->queued = (int)s->queue.size();
  out->active = (int)s->active.size();
  out->memory_used = (int64_t)s->used;
  out->memory_budget = (int64_t)s->budget;
  return FSLBM_OK;
}

void fslbm_server_destroy(fslbm_server* s) {
  if (!s) return;
  drop_batch(s);
  for (Active& a : s->active) fslbm_destroy(a.ctx);
  delete s;
}

const char* fslbm_server_last_error(const fslbm_server* s) { return s ? s->err.c_str() : "null server"; }

}  // extern "C"
