// fslbm_observables_noalloc: the whole-domain observables reduction for
// callers that cannot allocate device memory.
//
// Some callers are not allowed to call cudaMalloc: a host framework that owns
// all device memory through its own pooling allocator (a raw allocation would
// bypass its accounting and can fail under its budget), or a latency-critical
// loop in which an allocation may synchronize the device.  This entry point
// takes the state arrays and the output from the caller and keeps its block
// partials in a fixed file-scope device array instead of context memory.
#include <cuda_runtime.h>

#include <climits>
#include <cstring>
#include <mutex>

#include "../../include/fslbm.h"
#include "fslbm_kernels.cuh"

using namespace fslbm;

namespace {

// Fixed partial-sum blocks; the reduction grid never exceeds this, whatever
// the domain size (the kernels stride over the cells).
constexpr int kNoAllocBlocks = 1024;
constexpr int kMaxDevices = 64;

// Shared by every call on a device until the process exits; its contents are
// those of the last call.  Each call overwrites every partial it reads, so
// nothing has to be cleared between calls.
static __device__ __align__(256) double g_obs_scratch[kNoAllocBlocks * kObsFields + kObsFields];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {nullptr};
int g_blocks[kMaxDevices] = {0};

// Device address of g_obs_scratch on the current device (set up once per
// device; the host-side symbol itself is not a device address).
cudaError_t scratch_for(int dev, double** ptr, int* blocks) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_obs_scratch);
    if (e != cudaSuccess) return e;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int b = 2 * sms;
    g_blocks[dev] = b < kNoAllocBlocks ? b : kNoAllocBlocks;
    g_scratch_addr[dev] = (double*)p;
  }
  *ptr = g_scratch_addr[dev];
  *blocks = g_blocks[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" fslbm_status fslbm_observables_noalloc(const fslbm_domain* domain, int q, const double* g,
                                                  const double* pdf, const uint8_t* flags,
                                                  const double* fill, const double* mass,
                                                  fslbm_obs* out, void* stream) {
  if (!domain || !g || !pdf || !flags || !fill || !mass || !out) return FSLBM_EINVAL;
  if (q != 19 && q != 27) return FSLBM_EINVAL;
  if (domain->nx < 1 || domain->ny < 1 || domain->nz < 1) return FSLBM_EINVAL;
  const long long N = (long long)domain->nx * domain->ny * domain->nz;
  if (N > (long long)INT_MAX) return FSLBM_EINVAL;  // cell indices are 32-bit
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FSLBM_ECUDA;
  double* scratch = nullptr;
  int blocks = 0;
  if (scratch_for(dev, &scratch, &blocks) != cudaSuccess) return FSLBM_ECUDA;

  KParams p;
  std::memset(&p, 0, sizeof(p));
  p.nx = domain->nx;
  p.ny = domain->ny;
  p.nz = domain->nz;
  p.N = (int)N;
  p.Np = N;
  {
    const int identity[3] = {0, 1, 2};  // the caller's arrays: x contiguous
    set_layout(p, identity);
  }
  for (int a = 0; a < 3; ++a) p.g[a] = g[a];
  set_float_params(p);
  DPtrs d;
  std::memset(&d, 0, sizeof(d));
  d.pdf[0] = (void*)pdf;
  d.flags = (uint8_t*)flags;
  d.phi = (double*)fill;
  d.mass = (double*)mass;
  d.red = scratch;
  d.red_blocks = blocks;
  double* result = scratch + (size_t)kNoAllocBlocks * kObsFields;
  cudaStream_t st = (cudaStream_t)stream;
  if (q == 19)
    k_obs_partial<19, StoreF64><<<blocks, kBlock, 0, st>>>(d, p, 0, scratch);
  else
    k_obs_partial<27, StoreF64><<<blocks, kBlock, 0, st>>>(d, p, 0, scratch);
  k_obs_final<<<1, 32, 0, st>>>(scratch, blocks, result);
  double h[kObsFields];
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, result, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return FSLBM_ECUDA;
  std::memset(out, 0, sizeof(*out));
  out->total_mass = h[0];
  out->max_u = h[1];
  out->liquid_volume = h[2];
  out->nan_seen = h[3] != 0.0;
  out->n_gas = (int64_t)llround(h[4]);
  out->n_interface = (int64_t)llround(h[5]);
  out->n_liquid = (int64_t)llround(h[6]);
  out->n_obstacle = (int64_t)llround(h[7]);
  return FSLBM_OK;
}
