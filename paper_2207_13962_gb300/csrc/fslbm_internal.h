// Internal interface between the C-ABI layer and the per-precision engines.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "fslbm_common.cuh"

namespace fslbm {

// CUDA events between the kernels of a step (geometry, bulk, interface,
// resolve, count, apply, finalize, bubbles) for opt-in per-stage timing.
struct StageEvents {
  static constexpr int kMarks = 9;
  static constexpr int kStages = kMarks - 1;
  cudaEvent_t ev[kMarks];
  void mark(int i, cudaStream_t st) { cudaEventRecord(ev[i], st); }
};

// Side stream and events that let the bulk sweep run concurrently with the
// interface-band kernels of the same step.
struct Fork {
  cudaStream_t side;
  cudaEvent_t fork, join;
};

struct Ops {
  void (*init_cells)(const DPtrs&, const KParams&, const uint8_t* raw, const double* fill,
                     const double* vel, const double* den, cudaStream_t);
  void (*init_check)(const KParams&, const uint8_t* raw, int* bad, cudaStream_t);
  // bubble labelling at init: unions of neighbouring gas cells, ids of cells
  void (*cc_union)(const uint8_t* raw, const KParams&, int* lab, cudaStream_t);
  void (*cc_assign)(const uint8_t* raw, const KParams&, const int* lab, const int* root_id,
                    int* bid, cudaStream_t);
  void (*step)(const DPtrs&, const KParams&, int parity, int band_grid, int bulk_grid,
               cudaStream_t, StageEvents*, const Fork*);
  void (*observables)(const DPtrs&, const KParams&, int parity, double* out, cudaStream_t);
  void (*pdf_out)(const DPtrs&, const KParams&, int parity, double* out, cudaStream_t);
  size_t elem_size;
  size_t real_size;
  size_t rest_size;        // bytes per cell of the int32 rest slice (0: none)
  const void* bulk_fn[8];  // the bulk sweep kernels of each variant (bit 0 TRT,
                           // bit 1 Smagorinsky, bit 2 free-slip faces): graph nodes of
                           // every other kernel get the higher priority
  int bulk_blocks_per_sm;  // resident blocks per SM of the persistent bulk sweep
  size_t bulk_smem;        // its dynamic shared memory per block
  int step_launches;       // kernels one step launches (without the bubble kernel)
  // one step of every domain of a block table (see DomRec, BatchPlan)
  void (*batch_step)(DomRec* recs, const BatchPlan& plan, int band_grid, int bulk_grid,
                     int collision, cudaStream_t, const Fork*);
  const void* batch_bulk_fn[8];
  int batch_step_launches;  // kernels one batched step launches
};

// Collision variant of a parameter block: bit 0 TRT (else SRT), bit 1 the
// Smagorinsky model.
inline int coll_of(const KParams& p) { return (p.collision ? 1 : 0) | (p.cs > 0.0 ? 2 : 0); }
// Bit 2 of a kernel variant: the domain has free-slip faces.
inline int slip_bit(const KParams& p) { return (p.slip[0] | p.slip[1] | p.slip[2]) ? 4 : 0; }

// One engine per lattice and storage format, each compiled from
// fslbm_engine_inst.cu into an object of its own.
Ops ops_f64_q19();
Ops ops_f64_q27();
Ops ops_f32_q19();
Ops ops_f32_q27();
Ops ops_f16s_q19();
Ops ops_f16s_q27();
Ops ops_bf16s_q19();
Ops ops_bf16s_q27();
Ops ops_f32mc_q19();
Ops ops_f32mc_q27();
Ops ops_f16smc_q19();
Ops ops_f16smc_q27();
inline Ops ops_f64(int q) { return q == 27 ? ops_f64_q27() : ops_f64_q19(); }
inline Ops ops_f32(int q) { return q == 27 ? ops_f32_q27() : ops_f32_q19(); }
inline Ops ops_f16s(int q) { return q == 27 ? ops_f16s_q27() : ops_f16s_q19(); }
inline Ops ops_bf16s(int q) { return q == 27 ? ops_bf16s_q27() : ops_bf16s_q19(); }
inline Ops ops_f32mc(int q) { return q == 27 ? ops_f32mc_q27() : ops_f32mc_q19(); }
inline Ops ops_f16smc(int q) { return q == 27 ? ops_f16smc_q27() : ops_f16smc_q19(); }

// Bytes of one PDF buffer: q slices of Np stored values, plus the int32 rest
// slice of the mass-conserving formats.
inline size_t pdf_buffer_bytes(const Ops& o, int q, long long Np) {
  return (size_t)q * (size_t)Np * o.elem_size + (size_t)Np * o.rest_size;
}

}  // namespace fslbm
