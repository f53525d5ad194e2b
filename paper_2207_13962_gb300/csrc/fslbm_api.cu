// C ABI of the FSLBM library (include/fslbm.h): context management, initial
// state, CUDA-graph step driver, observables, field readback, checkpoints.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/fslbm.h"
#include "fslbm_ctx.h"
#include "fslbm_kernels.cuh"

using namespace fslbm;



namespace fslbm {

fslbm_status fail(fslbm_ctx* c, fslbm_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

fslbm_status cuda_fail(fslbm_ctx* c, cudaError_t e, const char* where) {
  return fail(c, e == cudaErrorMemoryAllocation ? FSLBM_ENOMEM : FSLBM_ECUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

// The interface-band kernels form a chain of short, latency-bound launches
// that runs beside the bulk sweep on a forked stream.  Their graph nodes get
// the device's highest priority, so that the block scheduler places their
// blocks first whenever an SM has room.  Nodes of skip0 / skip1 (the bulk
// sweep) keep the default priority.
cudaError_t prioritise_nodes(cudaGraph_t g, const void* skip0, const void* skip1) {
#if FSLBM_BAND_PRIO
  int least = 0, greatest = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
  if (e != cudaSuccess) return e;
  size_t n = 0;
  e = cudaGraphGetNodes(g, nullptr, &n);
  if (e != cudaSuccess || n == 0) return e;
  std::vector<cudaGraphNode_t> nodes(n);
  e = cudaGraphGetNodes(g, nodes.data(), &n);
  for (size_t i = 0; e == cudaSuccess && i < n; ++i) {
    cudaGraphNodeType t;
    e = cudaGraphNodeGetType(nodes[i], &t);
    if (e != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams kp;
    e = cudaGraphKernelNodeGetParams(nodes[i], &kp);
    if (e != cudaSuccess) break;
    if (kp.func == skip0 || kp.func == skip1) continue;
    cudaLaunchAttributeValue v;
    std::memset(&v, 0, sizeof(v));
    v.priority = greatest;
    e = cudaGraphKernelNodeSetAttribute(nodes[i], cudaLaunchAttributePriority, &v);
  }
  return e;
#else
  (void)g;
  (void)skip0;
  (void)skip1;
  return cudaSuccess;
#endif
}

}  // namespace fslbm

namespace {

const char* kVersion = "fslbm-gb300 1.0";


template <class T>
cudaError_t dalloc(fslbm_ctx* c, T** p, size_t bytes) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, bytes < 16 ? 16 : bytes);
  if (e == cudaSuccess) {
    c->allocs.push_back(v);
    *p = (T*)v;
  }
  return e;
}

void dfree(fslbm_ctx* c, void* p) {
  if (!p) return;
  for (size_t i = 0; i < c->allocs.size(); ++i)
    if (c->allocs[i] == p) {
      cudaFree(p);
      c->allocs.erase(c->allocs.begin() + (long)i);
      return;
    }
}

void destroy_graphs(fslbm_ctx* c) {
  for (int i = 0; i < 2; ++i)
    if (c->graph[i]) {
      cudaGraphExecDestroy(c->graph[i]);
      c->graph[i] = nullptr;
    }
}

cudaError_t build_graphs(fslbm_ctx* c) {
  destroy_graphs(c);
  for (int par = 0; par < 2; ++par) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    c->ops.step(c->d, c->kp, par, c->band_grid, c->bulk_grid, c->cap_stream, nullptr, &c->fork);
    e = cudaStreamEndCapture(c->cap_stream, &g);
    if (e != cudaSuccess) return e;
    e = prioritise_nodes(g, c->ops.bulk_fn[coll_of(c->kp) | slip_bit(c->kp)], nullptr);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph[par], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int launches_per_step(const fslbm_ctx* c) {
  return c->ops.step_launches + ((c->kp.bubble_model && c->d.nb > 0) ? 1 : 0);
}


bool valid_enum(int v, int lo, int hi) { return v >= lo && v <= hi; }

}  // namespace

extern "C" {

const char* fslbm_version(void) { return kVersion; }

void fslbm_params_default(fslbm_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->omega = 1.0;
  p->trt_magic = 3.0 / 16.0;
  p->eps_phi = 1e-2;
  p->p_v0 = 1.0 / 3.0;
  p->precision = FSLBM_FP32;
  p->om3_fallback = FSLBM_NBKC;
  p->bubble_model = 0;
  p->stream = nullptr;
  p->smagorinsky_cs = 0.0;
}

const char* fslbm_last_error(const fslbm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

fslbm_status fslbm_create(const fslbm_domain* domain, fslbm_lattice lattice,
                          fslbm_collision collision, fslbm_bc_variant bc_variant,
                          const fslbm_params* params, fslbm_ctx** out) {
  if (!domain || !params || !out) return FSLBM_EINVAL;
  if (domain->nx < 1 || domain->ny < 1 || domain->nz < 1) return FSLBM_EINVAL;
  const long long N = (long long)domain->nx * domain->ny * domain->nz;
  if (N > 400LL * 1000 * 1000) return FSLBM_EINVAL;
  if (lattice != FSLBM_D3Q19 && lattice != FSLBM_D3Q27) return FSLBM_EINVAL;
  if (!valid_enum(collision, 0, 1) || !valid_enum(bc_variant, 1, 4)) return FSLBM_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (!valid_enum(domain->periodic[a], FSLBM_NO_SLIP, FSLBM_FREE_SLIP)) return FSLBM_EINVAL;
  if (!(params->smagorinsky_cs >= 0.0)) return FSLBM_EINVAL;
  if (params->bubble_relabel_every < 0) return FSLBM_EINVAL;
  if (!valid_enum(params->precision, 0, 5)) return FSLBM_EINVAL;
  if (params->om3_fallback != FSLBM_NBRC && params->om3_fallback != FSLBM_NBKC) return FSLBM_EINVAL;
  if (!(params->omega > 0.0 && params->omega < 2.0)) return FSLBM_EINVAL;
  if (collision == FSLBM_TRT && !(params->trt_magic > 0.0)) return FSLBM_EINVAL;
  if (!(params->eps_phi >= 0.0) || !(params->p_v0 > 0.0)) return FSLBM_EINVAL;

  fslbm_ctx* c = new (std::nothrow) fslbm_ctx();
  if (!c) return FSLBM_ENOMEM;
  c->dom = *domain;
  c->q = (int)lattice;
  c->collision = (int)collision;
  c->variant = (int)bc_variant;
  c->prm = *params;
  c->stream = (cudaStream_t)params->stream;
  switch (params->precision) {
    case FSLBM_FP64: c->ops = ops_f64(c->q); break;
    case FSLBM_FP32: c->ops = ops_f32(c->q); break;
    case FSLBM_FP16S: c->ops = ops_f16s(c->q); break;
    case FSLBM_BF16S: c->ops = ops_bf16s(c->q); break;
    case FSLBM_FP32MC: c->ops = ops_f32mc(c->q); break;
    default: c->ops = ops_f16smc(c->q); break;
  }
  KParams& k = c->kp;
  k.nx = domain->nx;
  k.ny = domain->ny;
  k.nz = domain->nz;
  for (int a = 0; a < 3; ++a) {
    k.per[a] = domain->periodic[a] == FSLBM_PERIODIC ? 1 : 0;
    k.slip[a] = domain->periodic[a] == FSLBM_FREE_SLIP ? 1 : 0;
  }
  k.N = (int)N;
  k.Np = (N + 63) / 64 * 64;
  k.omega = params->omega;
  if (collision == FSLBM_TRT) {
    k.om_m = 1.0 / (0.5 + params->trt_magic / (1.0 / params->omega - 0.5));
  } else {
    k.om_m = params->omega;
  }
  k.pref_p = 1.0 - 0.5 * k.omega;
  k.pref_m = 1.0 - 0.5 * k.om_m;
  k.magic = params->trt_magic;
  k.cs = params->smagorinsky_cs;
  for (int a = 0; a < 3; ++a) k.g[a] = params->g[a];
  k.sigma = params->sigma;
  k.eps = params->eps_phi;
  k.pv0 = params->p_v0;
  {
    const int identity[3] = {0, 1, 2};
    set_layout(k, identity);
  }
  k.variant = (int)bc_variant;
  k.om3_fb = params->om3_fallback;
  k.bubble_model = params->bubble_model ? 1 : 0;
  k.collision = (int)collision;
  set_float_params(k);

  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 152;
  c->band_grid = sms * 2;
  // the persistent bulk sweep leaves FSLBM_BULK_RESERVE block slots per SM to
  // the interface-band kernels that run beside it
  // (and never more blocks than can be resident at once: the sweep's work
  // is split statically over its blocks)
  int bulk_per_sm = c->ops.bulk_blocks_per_sm - FSLBM_BULK_RESERVE;
  {
    int fit = 0;
    const void* fn = c->ops.bulk_fn[coll_of(k) | slip_bit(k)];
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, fn, kBulkBlock, c->ops.bulk_smem) == cudaSuccess &&
        fit > 0 && fit < bulk_per_sm)
      bulk_per_sm = fit;
  }
  c->bulk_grid = sms * bulk_per_sm;

  DPtrs& d = c->d;
  std::memset(&d, 0, sizeof(d));
  const size_t n4 = (size_t)((N + 3) / 4 * 4);
  cudaError_t e = cudaSuccess;
  const size_t pdf_bytes = pdf_buffer_bytes(c->ops, c->q, k.Np);
  const size_t rs = c->ops.real_size;
#define ALLOC(ptr, bytes)                                 \
  if (e == cudaSuccess) e = dalloc(c, &(ptr), (bytes));
  ALLOC(d.pdf[0], pdf_bytes);
  ALLOC(d.pdf[1], pdf_bytes);
  // flags padded to whole 32-byte segments (the TMA bulk sweep copies them)
  const size_t n32 = (size_t)((N + 31) / 32 * 32);
  ALLOC(d.flags, n32);
  ALLOC(d.wallmask, N * sizeof(uint32_t));
  ALLOC(d.phi, N * sizeof(double));
  ALLOC(d.mass, N * sizeof(double));
  ALLOC(d.bid, N * sizeof(int));
  ALLOC(d.cls, n4);
  ALLOC(d.mark, n4);
  ALLOC(d.conv, n4);
  ALLOC(d.cfin, n4);
  ALLOC(d.claim, n4);
  ALLOC(d.rcv, n4);
  ALLOC(d.share, N * sizeof(double));
  ALLOC(d.band[0], N * sizeof(int));
  ALLOC(d.band[1], N * sizeof(int));
  ALLOC(d.counts, 8 * sizeof(int));
  const long long ntiles = (long long)((domain->nx + 7) / 8) * ((domain->ny + 7) / 8) * ((domain->nz + 7) / 8);
  ALLOC(d.tiles[0], ntiles * sizeof(int));
  ALLOC(d.tiles[1], ntiles * sizeof(int));
  ALLOC(d.tile_mark, ntiles * sizeof(int));
  const long long nseg = (N + kSegCells - 1) / kSegCells;
  ALLOC(d.segs, nseg * sizeof(int));
  ALLOC(d.seg_mark, nseg * sizeof(int));
  ALLOC(d.newlist, N * sizeof(int));
  ALLOC(d.nhat, 3 * N * rs);
  ALLOC(d.rhog, N * rs);
  ALLOC(d.mom_rho, N * sizeof(double));
  ALLOC(d.mom_u, 3 * N * rs);
  ALLOC(d.m_next, N * sizeof(double));
  ALLOC(d.phi_next, N * sizeof(double));
  ALLOC(d.rho_band, N * sizeof(double));
  ALLOC(d.err, 4 * sizeof(int));
  d.red_blocks = sms * 2;
  ALLOC(d.red, (size_t)d.red_blocks * kObsFields * sizeof(double));
  ALLOC(c->d_obs, kObsFields * sizeof(double));
#undef ALLOC
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->fork.side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->fork.fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->fork.join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.claim, 0, n4, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.rcv, 0, n4, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.tile_mark, 0, ntiles * sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.err, 0, 4 * sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    fslbm_status s = e == cudaErrorMemoryAllocation ? FSLBM_ENOMEM : FSLBM_ECUDA;
    cudaGetLastError();
    fslbm_destroy(c);
    return s;
  }
  *out = c;
  return FSLBM_OK;
}

fslbm_status fslbm_memory_estimate(const fslbm_domain* domain, fslbm_lattice lattice, int precision,
                                   int with_velocity, size_t* bytes) {
  if (!domain || !bytes || domain->nx < 1 || domain->ny < 1 || domain->nz < 1) return FSLBM_EINVAL;
  if (lattice != FSLBM_D3Q19 && lattice != FSLBM_D3Q27) return FSLBM_EINVAL;
  if (precision < FSLBM_FP64 || precision > FSLBM_FP16SMC) return FSLBM_EINVAL;
  const double Nd = (double)domain->nx * domain->ny * domain->nz;
  if (Nd > 2147483647.0) return FSLBM_EINVAL;
  const size_t N = (size_t)Nd;
  const size_t Np = (N + 63) / 64 * 64;
  const size_t elem = precision == FSLBM_FP64 ? 8
                      : (precision == FSLBM_FP32 || precision == FSLBM_FP32MC) ? 4
                                                                               : 2;
  const size_t rest = (precision == FSLBM_FP32MC || precision == FSLBM_FP16SMC) ? 4 : 0;
  const size_t rs = precision == FSLBM_FP64 ? 8 : 4;
  const size_t n4 = (N + 3) / 4 * 4;
  const size_t ntiles =
      (size_t)((domain->nx + 7) / 8) * ((domain->ny + 7) / 8) * ((domain->nz + 7) / 8);
  const size_t nseg = (N + kSegCells - 1) / kSegCells;
  size_t b = 2 * ((size_t)lattice * Np * elem + Np * rest);  // PDFs, two buffers
  b += 6 * n4 + (N + 31) / 32 * 32;                      // cls, mark, conv, cfin, claim, rcv; flags
  b += N * (4 + 8 + 8 + 4 + 8 + 4 + 4 + 4);              // wallmask phi mass bid share band[2] newlist
  b += N * (7 * rs + 4 * 8);                             // nhat rhog mom m_next phi_next rho_band
  b += 3 * ntiles * 4 + 2 * nseg * 4 + 4096;             // tiles, segments, counters, partials
  b += 2 * (N * (1 + 8 + 8) + (with_velocity ? 24 * N : 0));  // fslbm_init staging in the
                                                           // caller's and the storage order
  *bytes = b;
  return FSLBM_OK;
}

void fslbm_destroy(fslbm_ctx* c) {
  if (!c) return;
  if (c->stream || c->cap_stream) cudaStreamSynchronize(c->stream);
  destroy_graphs(c);
  if (c->ev_made)
    for (int i = 0; i < StageEvents::kMarks; ++i) cudaEventDestroy(c->ev.ev[i]);
  for (void* p : c->allocs) cudaFree(p);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->fork.side) cudaStreamDestroy(c->fork.side);
  if (c->fork.fork) cudaEventDestroy(c->fork.fork);
  if (c->fork.join) cudaEventDestroy(c->fork.join);
  delete c;
}

namespace {

// Storage order for a domain's initial flags (caller order, on the device):
// the contiguous axis with the fewest liquid-holding 32-cell groups, i.e.
// the fullest warps of the bulk sweep, the other two axes in the caller's
// order.  x stays contiguous unless another axis needs at most 95 % of its
// groups.
cudaError_t choose_layout(fslbm_ctx* c, const uint8_t* raw_ext, int ax[3]) {
  ax[0] = 0;
  ax[1] = 1;
  ax[2] = 2;
  unsigned long long* cnt = nullptr;
  cudaError_t e = dalloc(c, &cnt, 3 * sizeof(unsigned long long));
  unsigned long long h[3] = {0, 0, 0};
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, 3 * sizeof(unsigned long long), c->stream);
  const int grid = (c->kp.N + kBlock - 1) / kBlock;
  for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
    KParams k = c->kp;
    const int order[3] = {a, a == 0 ? 1 : 0, a == 2 ? 1 : 2};
    set_layout(k, order);
    k_layout_census<<<grid, kBlock, 0, c->stream>>>(raw_ext, k, cnt + a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  dfree(c, cnt);
  if (e != cudaSuccess) return e;
  int best = 0;
  for (int a = 1; a < 3; ++a)
    if ((double)h[a] <= 0.95 * (double)h[0] && h[a] < h[best]) best = a;
  ax[0] = best;
  ax[1] = best == 0 ? 1 : 0;
  ax[2] = best == 2 ? 1 : 2;
  return cudaSuccess;
}

}  // namespace

fslbm_status fslbm_set_axis_order(fslbm_ctx* c, const int* order) {
  if (!c) return FSLBM_EINVAL;
  if (!order) {
    c->req_axis[0] = c->req_axis[1] = c->req_axis[2] = -1;
    return FSLBM_OK;
  }
  const bool ok = order[0] >= 0 && order[0] < 3 && order[1] >= 0 && order[1] < 3 && order[2] >= 0 &&
                  order[2] < 3 && order[0] != order[1] && order[0] != order[2] && order[1] != order[2];
  if (!ok) return fail(c, FSLBM_EINVAL, "axis order must be a permutation of 0, 1, 2");
  for (int a = 0; a < 3; ++a) c->req_axis[a] = order[a];
  return FSLBM_OK;
}

fslbm_status fslbm_get_axis_order(const fslbm_ctx* c, int* order) {
  if (!c || !order) return FSLBM_EINVAL;
  for (int a = 0; a < 3; ++a) order[a] = c->kp.ax[a];
  return FSLBM_OK;
}

fslbm_status fslbm_init(fslbm_ctx* c, const double* fill, const uint8_t* flags,
                        const double* velocity, const double* density) {
  if (!c) return FSLBM_EINVAL;
  if (!fill || !flags) return fail(c, FSLBM_EINVAL, "fill and flags are required");
  const size_t N = (size_t)c->kp.N;
  // flag values and the closed interface layer are checked on the device
  // (k_init_check) once the flags are uploaded
  cudaStream_t st = c->stream;
  uint8_t *raw = nullptr, *raw_ext = nullptr;
  double *dfill = nullptr, *dvel = nullptr, *dden = nullptr;
  double *fill_ext = nullptr, *vel_ext = nullptr, *den_ext = nullptr;
  int* bad = nullptr;
  cudaError_t e = dalloc(c, &raw_ext, N);
  if (e == cudaSuccess) e = dalloc(c, &fill_ext, N * sizeof(double));
  if (e == cudaSuccess && velocity) e = dalloc(c, &vel_ext, 3 * N * sizeof(double));
  if (e == cudaSuccess && density) e = dalloc(c, &den_ext, N * sizeof(double));
  if (e == cudaSuccess) e = dalloc(c, &bad, sizeof(int));
  auto cleanup = [&]() {
    if (raw != raw_ext) dfree(c, raw);
    if (dfill != fill_ext) dfree(c, dfill);
    if (dvel != vel_ext) dfree(c, dvel);
    if (dden != den_ext) dfree(c, dden);
    dfree(c, raw_ext);
    dfree(c, fill_ext);
    dfree(c, vel_ext);
    dfree(c, den_ext);
    dfree(c, bad);
  };
  if (e == cudaSuccess) e = cudaMemcpyAsync(raw_ext, flags, N, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(fill_ext, fill, N * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && velocity)
    e = cudaMemcpyAsync(vel_ext, velocity, 3 * N * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && density)
    e = cudaMemcpyAsync(den_ext, density, N * sizeof(double), cudaMemcpyHostToDevice, st);
  // storage order: the requested one, else the one whose bulk warps are
  // fullest for these flags; the previous one is restored if init fails
  const KParams kp_prev = c->kp;
  int ax[3] = {c->req_axis[0], c->req_axis[1], c->req_axis[2]};
  if (e == cudaSuccess && ax[0] < 0) e = choose_layout(c, raw_ext, ax);
  if (e == cudaSuccess) set_layout(c->kp, ax);
  raw = raw_ext;
  dfill = fill_ext;
  dvel = vel_ext;
  dden = den_ext;
  if (e == cudaSuccess && !is_identity_layout(c->kp)) {
    // staging copies in the storage order
    const int grid = (c->kp.N + kBlock - 1) / kBlock;
    raw = nullptr;
    dfill = dvel = dden = nullptr;
    e = dalloc(c, &raw, N);
    if (e == cudaSuccess) e = dalloc(c, &dfill, N * sizeof(double));
    if (e == cudaSuccess && velocity) e = dalloc(c, &dvel, 3 * N * sizeof(double));
    if (e == cudaSuccess && density) e = dalloc(c, &dden, N * sizeof(double));
    if (e == cudaSuccess) {
      k_to_storage<uint8_t><<<grid, kBlock, 0, st>>>(raw_ext, raw, c->kp, 1);
      k_to_storage<double><<<grid, kBlock, 0, st>>>(fill_ext, dfill, c->kp, 1);
      if (velocity) k_to_storage<double><<<grid, kBlock, 0, st>>>(vel_ext, dvel, c->kp, 3);
      if (density) k_to_storage<double><<<grid, kBlock, 0, st>>>(den_ext, dden, c->kp, 1);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), st);
  int hbad = 0;
  if (e == cudaSuccess) {
    c->ops.init_check(c->kp, raw, bad, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cleanup();
    c->kp = kp_prev;
    return cuda_fail(c, e, "fslbm_init upload");
  }
  if (hbad) {
    cleanup();
    c->kp = kp_prev;
    return fail(c, FSLBM_EINVAL,
                (hbad & 1) ? "flag value > 3"
                           : "a liquid cell touches a gas cell (interface layer not closed)");
  }
  // bubbles: connected gas regions labelled on the device, fixed-point
  // initial volumes
  DPtrs& d = c->d;
  dfree(c, d.V0);
  dfree(c, d.pV);
  dfree(c, d.gas_cnt);
  dfree(c, d.iface_fix);
  dfree(c, d.Vcur);
  d.V0 = d.pV = d.Vcur = nullptr;
  d.gas_cnt = d.iface_fix = nullptr;
  int nb = 0;
  const int gcells = (c->kp.N + kBlock - 1) / kBlock;
  if (c->kp.bubble_model) {
    const int nchunks = (c->kp.N + kCcChunk - 1) / kCcChunk;
    int* lab = d.band[1];      // free until the first step
    int* root_id = d.newlist;  // free until the first step
    int *cnt = nullptr, *off = nullptr;
    if (e == cudaSuccess) e = dalloc(c, &cnt, (size_t)nchunks * sizeof(int));
    if (e == cudaSuccess) e = dalloc(c, &off, (size_t)(nchunks + 1) * sizeof(int));
    if (e == cudaSuccess) {
      k_cc_init<<<gcells, kBlock, 0, st>>>(raw, c->kp.N, lab);
      c->ops.cc_union(raw, c->kp, lab, st);
      k_cc_compress<<<gcells, kBlock, 0, st>>>(c->kp.N, lab);
      k_cc_count<<<nchunks, kBlock, 0, st>>>(c->kp, lab, cnt);
      k_cc_scan<<<1, 1024, 0, st>>>(nchunks, cnt, off);
      k_cc_number<<<nchunks, 32, 0, st>>>(c->kp, lab, off, root_id);
      c->ops.cc_assign(raw, c->kp, lab, root_id, d.bid, st);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nb, off + nchunks, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(c, cnt);
    dfree(c, off);
  } else if (e == cudaSuccess) {
    e = cudaMemsetAsync(d.bid, 0xff, N * sizeof(int), st);
  }
  d.nb = nb;
  const size_t nbb = (size_t)(nb > 0 ? nb : 1);
  c->nb_cap = (int)nbb;
  if (e == cudaSuccess) e = dalloc(c, &d.V0, nbb * sizeof(double));
  if (e == cudaSuccess) e = dalloc(c, &d.pV, nbb * sizeof(double));
  if (e == cudaSuccess) e = dalloc(c, &d.gas_cnt, nbb * sizeof(long long));
  if (e == cudaSuccess) e = dalloc(c, &d.iface_fix, nbb * sizeof(long long));
  if (e == cudaSuccess) e = dalloc(c, &d.Vcur, nbb * sizeof(double));
  if (e == cudaSuccess && nb > 0) {
    e = cudaMemsetAsync(d.gas_cnt, 0, nbb * sizeof(long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.iface_fix, 0, nbb * sizeof(long long), st);
    if (e == cudaSuccess) {
      k_cc_volumes<<<gcells, kBlock, 0, st>>>(raw, dfill, c->kp.N, d.bid, d.gas_cnt, d.iface_fix);
      k_cc_v0<<<(nb + 255) / 256, 256, 0, st>>>(nb, d.gas_cnt, d.iface_fix, d.V0, d.Vcur, d.pV,
                                                 c->kp.pv0);
      e = cudaGetLastError();
    }
  }
  // clear both PDF buffers: gas and obstacle slots hold no PDFs of their
  // own (obstacle slots receive reflected copies from their neighbours)
  const size_t pdf_bytes = pdf_buffer_bytes(c->ops, c->q, c->kp.Np);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.pdf[0], 0, pdf_bytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.pdf[1], 0, pdf_bytes, st);
  if (e == cudaSuccess) {
    c->ops.init_cells(d, c->kp, raw, dfill, dvel, dden, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(d.counts, 0, 8 * sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.err, 0, 4 * sizeof(int), st);
  // a context initialised again still holds the tile marks of its last step
  if (e == cudaSuccess) {
    const size_t nt = (size_t)((c->dom.nx + 7) / 8) * ((c->dom.ny + 7) / 8) * ((c->dom.nz + 7) / 8);
    e = cudaMemsetAsync(d.tile_mark, 0, nt * sizeof(int), st);
  }
  if (e == cudaSuccess) {
    k_compact_full<<<(c->kp.N + kBlock - 1) / kBlock, kBlock, 0, st>>>(d.flags, c->kp.N, d.band[0],
                                                                      &d.counts[0]);
    k_tiles_of_band<<<c->band_grid, kBlock, 0, st>>>(d, c->kp, 0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(d.seg_mark, 0, (size_t)((N + kSegCells - 1) / kSegCells) * sizeof(int), st);
  if (e == cudaSuccess) {
    k_segs_init<<<(c->kp.N + kBlock - 1) / kBlock, kBlock, 0, st>>>(d, c->kp);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(c, e, "fslbm_init");
  c->parity = 0;
  c->step = 0;
  c->initialized = true;
  e = build_graphs(c);
  if (e != cudaSuccess) {
    c->initialized = false;
    return cuda_fail(c, e, "graph capture");
  }
  return FSLBM_OK;
}

// Bubble coalescence and segmentation between steps (fslbm_params::
// bubble_relabel_every): the bubbles are labelled again from the current
// flags with the kernels of init; the overlap of old and new bubbles (in
// 2^-32 fixed point, exact integer sums) comes to the host, which divides
// each old bubble's gas reference V0 over the new ones in proportion to the
// volume of its cells that each holds (in the oracle's order of operations:
// ascending old id), adds the volume of cells that carried no id (gas at
// p^V(0)), and uploads the new V0; the new bubbles' volumes and pressures
// follow.  The step's scratch lists serve as work space (free between
// steps).  The graphs are captured again when the bubble count changes.
namespace {
fslbm_status relabel_bubbles(fslbm_ctx* c) {
  DPtrs& d = c->d;
  const KParams& k = c->kp;
  cudaStream_t st = c->stream;
  const int N = k.N;
  const int gcells = (N + kBlock - 1) / kBlock;
  const int nchunks = (N + kCcChunk - 1) / kCcChunk;
  int* lab = d.band[c->parity ^ 1];
  int* root_id = d.newlist;
  int* old_bid = (int*)d.m_next;
  uint8_t* raw = (uint8_t*)d.phi_next;
  const int nb_old = d.nb;
  int *cnt = nullptr, *off = nullptr;
  cudaError_t e = cudaMemcpyAsync(old_bid, d.bid, (size_t)N * sizeof(int), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = dalloc(c, &cnt, (size_t)nchunks * sizeof(int));
  if (e == cudaSuccess) e = dalloc(c, &off, (size_t)(nchunks + 1) * sizeof(int));
  int nb_new = 0;
  if (e == cudaSuccess) {
    k_types<<<gcells, kBlock, 0, st>>>(d.flags, N, raw);
    k_cc_init<<<gcells, kBlock, 0, st>>>(raw, N, lab);
    c->ops.cc_union(raw, k, lab, st);
    k_cc_compress<<<gcells, kBlock, 0, st>>>(N, lab);
    k_cc_count<<<nchunks, kBlock, 0, st>>>(k, lab, cnt);
    k_cc_scan<<<1, 1024, 0, st>>>(nchunks, cnt, off);
    k_cc_number<<<nchunks, 32, 0, st>>>(k, lab, off, root_id);
    c->ops.cc_assign(raw, k, lab, root_id, d.bid, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nb_new, off + nchunks, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dfree(c, cnt);
  dfree(c, off);
  if (e != cudaSuccess) return cuda_fail(c, e, "bubble relabelling");
  const size_t W = (size_t)nb_new + 1;
  if ((size_t)(nb_old > 0 ? nb_old : 1) * W > ((size_t)1 << 26))
    return fail(c, FSLBM_ENOMEM, "bubble relabelling: too many bubbles for the overlap table");
  long long *M = nullptr, *fr = nullptr;
  const size_t nM = (size_t)(nb_old > 0 ? nb_old : 1) * W, nfr = (size_t)(nb_new > 0 ? nb_new : 1);
  e = dalloc(c, &M, nM * sizeof(long long));
  if (e == cudaSuccess) e = dalloc(c, &fr, nfr * sizeof(long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(M, 0, nM * sizeof(long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(fr, 0, nfr * sizeof(long long), st);
  if (e == cudaSuccess) {
    k_bubble_overlap<<<gcells, kBlock, 0, st>>>(raw, d.phi, old_bid, d.bid, N, (int)W, M, fr);
    e = cudaGetLastError();
  }
  std::vector<long long> hM(nM), hfr(nfr);
  std::vector<double> V0_old((size_t)(nb_old > 0 ? nb_old : 1), 0.0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hM.data(), M, nM * sizeof(long long), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hfr.data(), fr, nfr * sizeof(long long), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && nb_old > 0)
    e = cudaMemcpyAsync(V0_old.data(), d.V0, (size_t)nb_old * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dfree(c, M);
  dfree(c, fr);
  if (e != cudaSuccess) return cuda_fail(c, e, "bubble relabelling");
  std::vector<long long> row((size_t)(nb_old > 0 ? nb_old : 1), 0);
  // the volume each old bubble hands on to new bubbles (column 0 excluded)
  for (int A = 0; A < nb_old; ++A)
    for (size_t j = 1; j < W; ++j) row[A] += hM[(size_t)A * W + j];
  std::vector<double> V0_new(nfr, 0.0);
  for (int C = 0; C < nb_new; ++C) {
    double sum = 0.0;
    for (int A = 0; A < nb_old; ++A) {
      const long long m = hM[(size_t)A * W + (size_t)(C + 1)];
      if (m == 0 || row[A] == 0) continue;
      const double share = (double)m / (double)row[A];
      const double part = V0_old[A] * share;
      sum = sum + part;
    }
    const double free_part = (double)hfr[C] / 4294967296.0;
    V0_new[C] = sum + free_part;
  }
  // per-bubble arrays for the new count (grown when it exceeds the capacity)
  const bool grown = nb_new > c->nb_cap;
  if (grown) {
    dfree(c, d.V0);
    dfree(c, d.pV);
    dfree(c, d.gas_cnt);
    dfree(c, d.iface_fix);
    dfree(c, d.Vcur);
    d.V0 = d.pV = d.Vcur = nullptr;
    d.gas_cnt = d.iface_fix = nullptr;
    const size_t cap = (size_t)nb_new * 2;
    e = dalloc(c, &d.V0, cap * sizeof(double));
    if (e == cudaSuccess) e = dalloc(c, &d.pV, cap * sizeof(double));
    if (e == cudaSuccess) e = dalloc(c, &d.gas_cnt, cap * sizeof(long long));
    if (e == cudaSuccess) e = dalloc(c, &d.iface_fix, cap * sizeof(long long));
    if (e == cudaSuccess) e = dalloc(c, &d.Vcur, cap * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(c, e, "bubble relabelling");
    c->nb_cap = (int)cap;
  }
  if (nb_new > 0) {
    e = cudaMemcpyAsync(d.V0, V0_new.data(), (size_t)nb_new * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.gas_cnt, 0, (size_t)nb_new * sizeof(long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.iface_fix, 0, (size_t)nb_new * sizeof(long long), st);
    if (e == cudaSuccess) {
      k_cc_volumes<<<gcells, kBlock, 0, st>>>(raw, d.phi, N, d.bid, d.gas_cnt, d.iface_fix);
      k_relabel_pressure<<<(nb_new + 255) / 256, 256, 0, st>>>(nb_new, d.gas_cnt, d.iface_fix, d.V0, d.Vcur,
                                                                d.pV, k.pv0);
      e = cudaGetLastError();
    }
    // the host vectors must outlive the copy
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "bubble relabelling");
  }
  d.nb = nb_new;
  c->relabels += 1;
  if (nb_new != nb_old || grown) {
    e = build_graphs(c);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph capture after bubble relabelling");
  }
  return FSLBM_OK;
}
}  // namespace

fslbm_status fslbm_step(fslbm_ctx* c, int n) {
  if (!c) return FSLBM_EINVAL;
  if (!c->initialized) return fail(c, FSLBM_ESTATE, "step before init");
  if (n < 0) return fail(c, FSLBM_EINVAL, "negative step count");
  for (int s = 0; s < n; ++s) {
    cudaError_t e;
    if (c->timing) {
      c->ops.step(c->d, c->kp, c->parity, c->band_grid, c->bulk_grid, c->stream, &c->ev, nullptr);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventSynchronize(c->ev.ev[StageEvents::kMarks - 1]);
      if (e == cudaSuccess) {
        for (int k = 0; k < StageEvents::kStages; ++k) {
          float ms = 0.f;
          cudaEventElapsedTime(&ms, c->ev.ev[k], c->ev.ev[k + 1]);
          c->stage_ms[k] += ms;
        }
      }
    } else {
      e = cudaGraphLaunch(c->graph[c->parity], c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "fslbm_step");
    c->launches += launches_per_step(c);
    c->parity ^= 1;
    c->step += 1;
    const int K = c->prm.bubble_relabel_every;
    if (K > 0 && c->kp.bubble_model && c->step % K == 0) {
      const fslbm_status rs = relabel_bubbles(c);
      if (rs != FSLBM_OK) return rs;
    }
  }
  return FSLBM_OK;
}

fslbm_status fslbm_sync(fslbm_ctx* c) {
  if (!c) return FSLBM_EINVAL;
  int herr[4] = {0, 0, 0, 0};
  cudaError_t e = cudaMemcpyAsync(herr, c->d.err, sizeof(herr), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "fslbm_sync");
  if (herr[0]) return fail(c, FSLBM_EUNSTABLE, "instability: |u|^2 >= c_s^2, rho <= 0 or NaN");
  if (herr[1]) return fail(c, FSLBM_ETIMEOUT, "a bounded wait for bulk-sweep copies gave up");
  return FSLBM_OK;
}

fslbm_status fslbm_observables(fslbm_ctx* c, fslbm_obs* out) {
  if (!c || !out) return FSLBM_EINVAL;
  if (!c->initialized) return fail(c, FSLBM_ESTATE, "observables before init");
  double h[kObsFields];
  c->ops.observables(c->d, c->kp, c->parity, c->d_obs, c->stream);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h, c->d_obs, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "fslbm_observables");
  std::memset(out, 0, sizeof(*out));
  out->step = c->step;
  out->total_mass = h[0];
  out->max_u = h[1];
  out->liquid_volume = h[2];
  out->nan_seen = h[3] != 0.0;
  out->n_gas = (int64_t)llround(h[4]);
  out->n_interface = (int64_t)llround(h[5]);
  out->n_liquid = (int64_t)llround(h[6]);
  out->n_obstacle = (int64_t)llround(h[7]);
  out->n_bubbles = c->d.nb;
  fslbm_status s = fslbm_sync(c);
  if (s != FSLBM_OK) return s;
  if (out->nan_seen || !(out->max_u < std::sqrt(1.0 / 3.0)))
    return fail(c, FSLBM_EUNSTABLE, "instability: max |u| >= c_s or NaN");
  return FSLBM_OK;
}

fslbm_status fslbm_read_fields(fslbm_ctx* c, double* pdf, double* fill, uint8_t* flags,
                               double* mass) {
  if (!c) return FSLBM_EINVAL;
  if (!c->initialized) return fail(c, FSLBM_ESTATE, "read before init");
  const size_t N = (size_t)c->kp.N;
  cudaStream_t st = c->stream;
  cudaError_t e = cudaSuccess;
  if (pdf) {
    double* tmp = nullptr;
    e = dalloc(c, &tmp, (size_t)c->q * N * sizeof(double));
    if (e == cudaSuccess) {
      c->ops.pdf_out(c->d, c->kp, c->parity, tmp, st);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(pdf, tmp, (size_t)c->q * N * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(c, tmp);
  }
  if (is_identity_layout(c->kp)) {
    if (e == cudaSuccess && fill)
      e = cudaMemcpyAsync(fill, c->d.phi, N * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && mass)
      e = cudaMemcpyAsync(mass, c->d.mass, N * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && flags) e = cudaMemcpyAsync(flags, c->d.flags, N, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  } else if (e == cudaSuccess && (fill || mass || flags)) {
    // the fields in the caller's cell order, through one staging array
    double* tmp = nullptr;
    e = dalloc(c, &tmp, N * sizeof(double));
    const int grid = (c->kp.N + kBlock - 1) / kBlock;
    auto out = [&](const double* src, double* host) {
      if (e != cudaSuccess || !host) return;
      k_to_caller<double><<<grid, kBlock, 0, st>>>(src, tmp, c->kp);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaMemcpyAsync(host, tmp, N * sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    };
    out(c->d.phi, fill);
    out(c->d.mass, mass);
    if (e == cudaSuccess && flags) {
      k_to_caller<uint8_t><<<grid, kBlock, 0, st>>>(c->d.flags, (uint8_t*)tmp, c->kp);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaMemcpyAsync(flags, tmp, N, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    dfree(c, tmp);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "fslbm_read_fields");
  if (flags)
    for (size_t i = 0; i < N; ++i) flags[i] &= F_TYPE;
  return FSLBM_OK;
}

fslbm_status fslbm_bubbles(fslbm_ctx* c, double* volume, double* pressure, int cap, int* n_out) {
  if (!c) return FSLBM_EINVAL;
  if (!c->initialized) return fail(c, FSLBM_ESTATE, "bubbles before init");
  const int nb = c->d.nb;
  if (n_out) *n_out = nb;
  const int m = nb < cap ? nb : cap;
  if (m <= 0) return FSLBM_OK;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess && pressure)
    e = cudaMemcpy(pressure, c->d.pV, m * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && volume)
    e = cudaMemcpy(volume, c->d.Vcur, m * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "fslbm_bubbles");
  return FSLBM_OK;
}

fslbm_status fslbm_set_timing(fslbm_ctx* c, int enable) {
  if (!c) return FSLBM_EINVAL;
  if (enable && !c->ev_made) {
    for (int i = 0; i < StageEvents::kMarks; ++i) {
      cudaError_t e = cudaEventCreate(&c->ev.ev[i]);
      if (e != cudaSuccess) return cuda_fail(c, e, "event create");
    }
    c->ev_made = true;
  }
  c->timing = enable != 0;
  for (int k = 0; k < StageEvents::kStages; ++k) c->stage_ms[k] = 0.0;
  c->launches = 0;
  return FSLBM_OK;
}

fslbm_status fslbm_stage_times(fslbm_ctx* c, double* ms, int cap, int* n_launches) {
  if (!c) return FSLBM_EINVAL;
  for (int k = 0; k < StageEvents::kStages && k < cap; ++k) ms[k] = c->stage_ms[k];
  if (n_launches) *n_launches = (int)c->launches;
  return FSLBM_OK;
}

fslbm_status fslbm_interface_count(fslbm_ctx* c, int64_t* n) {
  if (!c || !n) return FSLBM_EINVAL;
  if (!c->initialized) return fail(c, FSLBM_ESTATE, "before init");
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, &c->d.counts[c->parity], sizeof(int), cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "interface count");
  *n = h;
  return FSLBM_OK;
}

fslbm_status fslbm_work_counts(fslbm_ctx* c, int64_t* interface_cells, int64_t* liquid_segments,
                               int64_t* geometry_tiles) {
  if (!c) return FSLBM_EINVAL;
  if (!c->initialized) return fail(c, FSLBM_ESTATE, "before init");
  int h[8];
  cudaError_t e = cudaMemcpyAsync(h, c->d.counts, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "work counts");
  if (interface_cells) *interface_cells = h[c->parity];
  if (liquid_segments) *liquid_segments = h[5];
  if (geometry_tiles) *geometry_tiles = h[3 + c->parity];
  return FSLBM_OK;
}

// ------------------------------------------------------------ checkpoints
namespace {
// The arrays are saved in the context's storage order, which the header
// records; a checkpoint loads only into a context with the same order.
struct CkptHeader {
  char magic[8];
  int nx, ny, nz, q, precision, nb;
  int ax[3], reserved;
  int64_t step;
  int64_t pdf_bytes;
};
}  // namespace

fslbm_status fslbm_save(fslbm_ctx* c, void* buf, size_t* size) {
  if (!c || !size) return FSLBM_EINVAL;
  if (!c->initialized) return fail(c, FSLBM_ESTATE, "save before init");
  const size_t N = (size_t)c->kp.N;
  const size_t nb = (size_t)c->d.nb;
  const size_t pdf_bytes = pdf_buffer_bytes(c->ops, c->q, c->kp.Np);
  const size_t need = sizeof(CkptHeader) + pdf_bytes + N + 2 * N * sizeof(double) +
                      N * sizeof(int) + nb * (3 * sizeof(double) + sizeof(long long));
  if (!buf) {
    *size = need;
    return FSLBM_OK;
  }
  if (*size < need) return fail(c, FSLBM_EINVAL, "checkpoint buffer too small");
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "FSLBMCK2", 8);
  h.nx = c->kp.nx;
  h.ny = c->kp.ny;
  h.nz = c->kp.nz;
  h.q = c->q;
  h.precision = c->prm.precision;
  h.nb = (int)nb;
  for (int a = 0; a < 3; ++a) h.ax[a] = c->kp.ax[a];
  h.step = c->step;
  h.pdf_bytes = (int64_t)pdf_bytes;
  char* p = (char*)buf;
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  auto d2h = [&](const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpy(p, src, bytes, cudaMemcpyDeviceToHost);
    p += bytes;
  };
  d2h(c->d.pdf[c->parity], pdf_bytes);
  d2h(c->d.flags, N);
  d2h(c->d.phi, N * sizeof(double));
  d2h(c->d.mass, N * sizeof(double));
  d2h(c->d.bid, N * sizeof(int));
  d2h(c->d.V0, nb * sizeof(double));
  d2h(c->d.pV, nb * sizeof(double));
  d2h(c->d.Vcur, nb * sizeof(double));
  d2h(c->d.gas_cnt, nb * sizeof(long long));
  if (e != cudaSuccess) return cuda_fail(c, e, "fslbm_save");
  *size = need;
  return FSLBM_OK;
}

fslbm_status fslbm_load(fslbm_ctx* c, const void* buf, size_t size) {
  if (!c || !buf) return FSLBM_EINVAL;
  if (!c->initialized) return fail(c, FSLBM_ESTATE, "load needs an initialised context");
  if (size < sizeof(CkptHeader)) return fail(c, FSLBM_EINVAL, "checkpoint too small");
  CkptHeader h;
  std::memcpy(&h, buf, sizeof(h));
  const size_t N = (size_t)c->kp.N;
  const size_t pdf_bytes = pdf_buffer_bytes(c->ops, c->q, c->kp.Np);
  if (std::memcmp(h.magic, "FSLBMCK2", 8) != 0 || h.nx != c->kp.nx || h.ny != c->kp.ny ||
      h.nz != c->kp.nz || h.q != c->q || h.precision != c->prm.precision ||
      (h.nb != c->d.nb && !c->kp.bubble_model) || h.nb < 0 ||
      h.pdf_bytes != (int64_t)pdf_bytes || h.ax[0] != c->kp.ax[0] || h.ax[1] != c->kp.ax[1] ||
      h.ax[2] != c->kp.ax[2])
    return fail(c, FSLBM_EINVAL, "checkpoint does not match this context");
  const size_t nb = (size_t)h.nb;
  const size_t need = sizeof(CkptHeader) + pdf_bytes + N + 2 * N * sizeof(double) +
                      N * sizeof(int) + nb * (3 * sizeof(double) + sizeof(long long));
  if (size < need) return fail(c, FSLBM_EINVAL, "checkpoint truncated");
  const char* p = (const char*)buf + sizeof(h);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  // a run whose bubbles were relabelled may hold another bubble count
  const bool nb_changed = (int)nb != c->d.nb;
  const bool grown = e == cudaSuccess && (int)nb > c->nb_cap;
  if (grown) {
    dfree(c, c->d.V0);
    dfree(c, c->d.pV);
    dfree(c, c->d.gas_cnt);
    dfree(c, c->d.iface_fix);
    dfree(c, c->d.Vcur);
    c->d.V0 = c->d.pV = c->d.Vcur = nullptr;
    c->d.gas_cnt = c->d.iface_fix = nullptr;
    e = dalloc(c, &c->d.V0, nb * sizeof(double));
    if (e == cudaSuccess) e = dalloc(c, &c->d.pV, nb * sizeof(double));
    if (e == cudaSuccess) e = dalloc(c, &c->d.gas_cnt, nb * sizeof(long long));
    if (e == cudaSuccess) e = dalloc(c, &c->d.iface_fix, nb * sizeof(long long));
    if (e == cudaSuccess) e = dalloc(c, &c->d.Vcur, nb * sizeof(double));
    if (e == cudaSuccess) c->nb_cap = (int)nb;
  }
  c->d.nb = (int)nb;
  auto h2d = [&](void* dst, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpy(dst, p, bytes, cudaMemcpyHostToDevice);
    p += bytes;
  };
  h2d(c->d.pdf[0], pdf_bytes);
  h2d(c->d.flags, N);
  h2d(c->d.phi, N * sizeof(double));
  h2d(c->d.mass, N * sizeof(double));
  h2d(c->d.bid, N * sizeof(int));
  h2d(c->d.V0, nb * sizeof(double));
  h2d(c->d.pV, nb * sizeof(double));
  h2d(c->d.Vcur, nb * sizeof(double));
  h2d(c->d.gas_cnt, nb * sizeof(long long));
  if (e == cudaSuccess && nb) e = cudaMemset(c->d.iface_fix, 0, nb * sizeof(long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d.counts, 0, 8 * sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d.err, 0, 4 * sizeof(int), c->stream);
  if (e == cudaSuccess) {
    const size_t nt = (size_t)((c->kp.nx + 7) / 8) * ((c->kp.ny + 7) / 8) * ((c->kp.nz + 7) / 8);
    e = cudaMemsetAsync(c->d.tile_mark, 0, nt * sizeof(int), c->stream);
  }
  if (e == cudaSuccess) {
    k_compact_full<<<(c->kp.N + kBlock - 1) / kBlock, kBlock, 0, c->stream>>>(c->d.flags, c->kp.N,
                                                                             c->d.band[0], &c->d.counts[0]);
    k_tiles_of_band<<<c->band_grid, kBlock, 0, c->stream>>>(c->d, c->kp, 0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d.seg_mark, 0, (size_t)((N + kSegCells - 1) / kSegCells) * sizeof(int), c->stream);
  if (e == cudaSuccess) {
    k_segs_init<<<(c->kp.N + kBlock - 1) / kBlock, kBlock, 0, c->stream>>>(c->d, c->kp);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "fslbm_load");
  c->parity = 0;
  c->step = h.step;
  if (nb_changed || grown) {
    e = build_graphs(c);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph capture after fslbm_load");
  }
  return FSLBM_OK;
}

}  // extern "C"
