// C ABI of batches: many domains of different sizes advance together, one
// launch per phase of the step over a block table of the member domains.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fslbm_band_list.cuh"
#include "fslbm_ctx.h"

using namespace fslbm;

struct fslbm_batch {
  std::vector<fslbm_ctx*> m;
  Ops ops;
  int collision = 1;               // collision variant of the members (coll_of)
  cudaStream_t stream = nullptr;   // caller's stream (may be NULL)
  cudaStream_t cap = nullptr;      // capture stream
  Fork fork{nullptr, nullptr, nullptr};
  cudaEvent_t done = nullptr;
  std::vector<cudaEvent_t> mev;    // one per member: its stream's latest work
  DomRec* d_recs = nullptr;
  int* d_off = nullptr;
  int* d_chunk = nullptr;          // prefix of the members' interface-list chunks (n + 1)
  int* d_cnt = nullptr;            // their list counters of kb_compact_band (n)
  int nchunks = 0;
  BatchPlan plan{};
  std::vector<DomRec> h_recs;
  cudaGraphExec_t graph = nullptr;
  int sms = 152;
  fslbm_tuning tune{};
  long long launches = 0;          // kernels launched by batch steps
  std::string err;
};

namespace {


fslbm_status bfail(fslbm_batch* b, fslbm_status s, const std::string& msg) {
  if (b) b->err = msg;
  return s;
}

fslbm_status bcuda(fslbm_batch* b, cudaError_t e, const char* where) {
  return bfail(b, e == cudaErrorMemoryAllocation ? FSLBM_ENOMEM : FSLBM_ECUDA,
               std::string(where) + ": " + cudaGetErrorString(e));
}

int max_bulk_blocks(const fslbm_batch* b) {
  if (b->m[0]->prm.precision == FSLBM_FP64) return 2;
  return (b->collision & 2) ? 3 : kBulkMinBlocks32;  // the Smagorinsky sweep is compiled for 3
}

cudaError_t capture(fslbm_batch* b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  b->ops.batch_step(b->d_recs, b->plan, b->sms * b->tune.band_blocks_per_sm,
                    b->sms * b->tune.bulk_blocks_per_sm, b->collision, b->cap, &b->fork);
  // every member's next interface list rewritten in cell order
  const int n = (int)b->m.size();
  cudaMemsetAsync(b->d_cnt, 0, (size_t)n * sizeof(int), b->cap);
  kb_compact_band<<<b->nchunks < 8 * b->sms ? b->nchunks : 8 * b->sms, kBlock, 0, b->cap>>>(
      b->d_recs, b->d_chunk, n, b->d_cnt);
  e = cudaStreamEndCapture(b->cap, &g);
  if (e != cudaSuccess) return e;
  e = prioritise_nodes(g, b->ops.batch_bulk_fn[b->collision], nullptr);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  return e;
}

// Upload the block table (each member's pointers, parameters and current
// parity) behind the members' pending work.
cudaError_t upload(fslbm_batch* b) {
  cudaError_t e = cudaSuccess;
  for (size_t k = 0; k < b->m.size() && e == cudaSuccess; ++k) {
    fslbm_ctx* c = b->m[k];
    b->h_recs[k].d = c->d;
    b->h_recs[k].p = c->kp;
    b->h_recs[k].parity = c->parity;
    e = cudaEventRecord(b->mev[k], c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->mev[k], 0);
  }
  // pageable source: the call returns once the host buffer has been staged
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_recs, b->h_recs.data(), b->h_recs.size() * sizeof(DomRec),
                        cudaMemcpyHostToDevice, b->stream);
  return e;
}

// Launch n steps and order the members' later work after them.
cudaError_t launch(fslbm_batch* b, int n) {
  cudaError_t e = upload(b);
  for (int s = 0; s < n && e == cudaSuccess; ++s) e = cudaGraphLaunch(b->graph, b->stream);
  if (e == cudaSuccess) e = cudaEventRecord(b->done, b->stream);
  for (size_t k = 0; k < b->m.size() && e == cudaSuccess; ++k)
    e = cudaStreamWaitEvent(b->m[k]->stream, b->done, 0);
  if (e == cudaSuccess) {
    for (fslbm_ctx* c : b->m) {
      c->parity ^= (n & 1);
      c->step += n;
    }
    b->launches += (long long)n * b->ops.batch_step_launches;
  }
  return e;
}

}  // namespace

extern "C" {

fslbm_status fslbm_batch_create(fslbm_ctx* const* members, int n, void* stream, fslbm_batch** out) {
  if (!members || n <= 0 || !out) return FSLBM_EINVAL;
  for (int k = 0; k < n; ++k) {
    if (!members[k] || !members[k]->initialized) return FSLBM_ESTATE;
    for (int j = 0; j < k; ++j)
      if (members[j] == members[k]) return FSLBM_EINVAL;
    const fslbm_ctx* a = members[0];
    const fslbm_ctx* c = members[k];
    if (c->q != a->q || c->prm.precision != a->prm.precision || coll_of(c->kp) != coll_of(a->kp))
      return FSLBM_EINVAL;
    // bubble relabelling runs between single-domain steps only
    if (c->kp.bubble_model && c->prm.bubble_relabel_every > 0) return FSLBM_EINVAL;
  }
  fslbm_batch* b = new (std::nothrow) fslbm_batch();
  if (!b) return FSLBM_ENOMEM;
  b->m.assign(members, members + n);
  b->ops = members[0]->ops;
  b->collision = coll_of(members[0]->kp);
  for (int k = 0; k < n; ++k) {
    const KParams& kp = members[k]->kp;
    if (kp.slip[0] | kp.slip[1] | kp.slip[2]) b->collision |= 4;  // free-slip faces
  }
  b->stream = (cudaStream_t)stream;
  b->h_recs.resize((size_t)n);
  int dev = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) b->sms = 152;
  b->tune.bulk_blocks_per_sm = max_bulk_blocks(b);
  b->tune.band_blocks_per_sm = 2;
  b->tune.ms_per_step = 0.0;
  cudaError_t e = cudaMalloc(&b->d_recs, (size_t)n * sizeof(DomRec));
  // four prefix arrays of n + 1 entries, then the bulk sweep's hand-out
  // counter and the fused sweep's tile counter
  if (e == cudaSuccess) e = cudaMalloc(&b->d_off, (4 * (size_t)(n + 1) + 2) * sizeof(int));
  if (e == cudaSuccess) {
    // interface-list chunks of each member: fixed by its cell count
    std::vector<int> off((size_t)n + 1, 0);
    for (int k = 0; k < n; ++k) off[k + 1] = off[k] + (members[k]->kp.N + kCompactChunk - 1) / kCompactChunk;
    b->nchunks = off[n];
    e = cudaMalloc(&b->d_chunk, ((size_t)n + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_cnt, (size_t)n * sizeof(int));
    if (e == cudaSuccess)
      e = cudaMemcpy(b->d_chunk, off.data(), ((size_t)n + 1) * sizeof(int), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->fork.side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork.fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork.join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  b->mev.assign((size_t)n, nullptr);
  for (int k = 0; k < n && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(&b->mev[k], cudaEventDisableTiming);
  if (e == cudaSuccess) {
    b->plan.n = n;
    b->plan.tiles = b->d_off;
    b->plan.bulk = b->d_off + (n + 1);
    b->plan.band = b->d_off + 2 * (n + 1);
    b->plan.all = b->d_off + 3 * (n + 1);
    e = capture(b);
  }
  if (e != cudaSuccess) {
    const fslbm_status s = e == cudaErrorMemoryAllocation ? FSLBM_ENOMEM : FSLBM_ECUDA;
    cudaGetLastError();
    fslbm_batch_destroy(b);
    return s;
  }
  *out = b;
  return FSLBM_OK;
}

fslbm_status fslbm_batch_step(fslbm_batch* b, int n) {
  if (!b) return FSLBM_EINVAL;
  if (n < 0) return bfail(b, FSLBM_EINVAL, "negative step count");
  if (n == 0) return FSLBM_OK;
  const cudaError_t e = launch(b, n);
  if (e != cudaSuccess) return bcuda(b, e, "fslbm_batch_step");
  return FSLBM_OK;
}

fslbm_status fslbm_batch_sync(fslbm_batch* b, fslbm_status* member_status) {
  if (!b) return FSLBM_EINVAL;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "fslbm_batch_sync");
  fslbm_status worst = FSLBM_OK;
  for (size_t k = 0; k < b->m.size(); ++k) {
    int herr[4] = {0, 0, 0, 0};
    e = cudaMemcpy(herr, b->m[k]->d.err, sizeof(herr), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, e, "fslbm_batch_sync");
    const fslbm_status s = herr[0] ? FSLBM_EUNSTABLE : FSLBM_OK;
    if (member_status) member_status[k] = s;
    if (s != FSLBM_OK) worst = s;
  }
  return worst == FSLBM_OK ? FSLBM_OK : bfail(b, worst, "a member became unstable");
}

fslbm_status fslbm_batch_set_tuning(fslbm_batch* b, const fslbm_tuning* t) {
  if (!b || !t) return FSLBM_EINVAL;
  if (t->bulk_blocks_per_sm < 1 || t->bulk_blocks_per_sm > max_bulk_blocks(b) ||
      t->band_blocks_per_sm < 1 || t->band_blocks_per_sm > 16)
    return bfail(b, FSLBM_EINVAL, "tuning out of range");
  const fslbm_tuning old = b->tune;
  b->tune.bulk_blocks_per_sm = t->bulk_blocks_per_sm;
  b->tune.band_blocks_per_sm = t->band_blocks_per_sm;
  const cudaError_t e = capture(b);
  if (e != cudaSuccess) {
    b->tune = old;
    cudaGetLastError();
    capture(b);
    return bcuda(b, e, "fslbm_batch_set_tuning");
  }
  return FSLBM_OK;
}

fslbm_status fslbm_batch_autotune(fslbm_batch* b, int steps, fslbm_tuning* chosen) {
  if (!b || steps < 1) return FSLBM_EINVAL;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaError_t e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  fslbm_tuning best = b->tune;
  best.ms_per_step = -1.0;
  const int band_opts[4] = {1, 2, 4, 8};
  for (int bulk = 1; bulk <= max_bulk_blocks(b) && e == cudaSuccess; ++bulk) {
    for (int oi = 0; oi < 4 && e == cudaSuccess; ++oi) {
      b->tune.bulk_blocks_per_sm = bulk;
      b->tune.band_blocks_per_sm = band_opts[oi];
      e = capture(b);
      if (e == cudaSuccess) e = launch(b, 1);  // warm-up of this candidate
      if (e == cudaSuccess) e = cudaEventRecord(t0, b->stream);
      if (e == cudaSuccess) e = launch(b, steps);
      if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
      const double per = (double)ms / steps;
      if (e == cudaSuccess && (best.ms_per_step < 0.0 || per < best.ms_per_step)) {
        best = b->tune;
        best.ms_per_step = per;
      }
    }
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (e != cudaSuccess) return bcuda(b, e, "fslbm_batch_autotune");
  b->tune = best;
  e = capture(b);
  if (e != cudaSuccess) return bcuda(b, e, "fslbm_batch_autotune");
  if (chosen) *chosen = best;
  return FSLBM_OK;
}

fslbm_status fslbm_batch_get_tuning(const fslbm_batch* b, fslbm_tuning* t) {
  if (!b || !t) return FSLBM_EINVAL;
  *t = b->tune;
  return FSLBM_OK;
}

fslbm_status fslbm_batch_launches(const fslbm_batch* b, int64_t* n) {
  if (!b || !n) return FSLBM_EINVAL;
  *n = b->launches;
  return FSLBM_OK;
}

void fslbm_batch_destroy(fslbm_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->d_recs) cudaFree(b->d_recs);
  if (b->d_off) cudaFree(b->d_off);
  if (b->d_chunk) cudaFree(b->d_chunk);
  if (b->d_cnt) cudaFree(b->d_cnt);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->fork.side) cudaStreamDestroy(b->fork.side);
  if (b->fork.fork) cudaEventDestroy(b->fork.fork);
  if (b->fork.join) cudaEventDestroy(b->fork.join);
  if (b->done) cudaEventDestroy(b->done);
  for (cudaEvent_t ev : b->mev)
    if (ev) cudaEventDestroy(ev);
  delete b;
}

const char* fslbm_batch_last_error(const fslbm_batch* b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"
