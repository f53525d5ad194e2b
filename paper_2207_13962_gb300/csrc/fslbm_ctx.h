// Host-side state of one domain (the fslbm_ctx of the C ABI) and helpers
// shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/fslbm.h"
#include "fslbm_internal.h"

// Graph nodes of the interface-band kernels get the highest priority (1) or
// the default one (0); the persistent bulk sweep leaves FSLBM_BULK_RESERVE
// block slots per SM to them.
#ifndef FSLBM_BAND_PRIO
#define FSLBM_BAND_PRIO 1
#endif
#ifndef FSLBM_BULK_RESERVE
#define FSLBM_BULK_RESERVE 0
#endif

struct fslbm_ctx {
  fslbm_domain dom;
  int q = 19, collision = 1, variant = 3;
  fslbm_params prm;
  fslbm::KParams kp;
  int req_axis[3] = {-1, -1, -1};  // requested storage order, -1: chosen at init
  fslbm::DPtrs d;
  fslbm::Ops ops;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  fslbm::Fork fork{nullptr, nullptr, nullptr};
  int bulk_grid = 608;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int parity = 0;
  int64_t step = 0;
  bool initialized = false;
  int band_grid = 608;
  bool timing = false;
  fslbm::StageEvents ev;
  bool ev_made = false;
  double stage_ms[fslbm::StageEvents::kStages] = {};
  long long launches = 0;
  int nb_cap = 1;           // entries of the per-bubble arrays
  long long relabels = 0;   // bubble relabellings done
  double* d_obs = nullptr;
  std::vector<void*> allocs;
  std::string err;
};

namespace fslbm {
fslbm_status fail(fslbm_ctx* c, fslbm_status s, const std::string& msg);
fslbm_status cuda_fail(fslbm_ctx* c, cudaError_t e, const char* where);
cudaError_t prioritise_nodes(cudaGraph_t g, const void* skip0, const void* skip1);
}  // namespace fslbm
