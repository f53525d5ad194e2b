// FP32 engine: FP32 PDFs and arithmetic; fill level and mass stay FP64.
#include "fslbm_engine.cuh"

namespace fslbm {
Ops ops_f32(int q) { return q == 27 ? Engine<27, StoreF32>::ops() : Engine<19, StoreF32>::ops(); }
}  // namespace fslbm
