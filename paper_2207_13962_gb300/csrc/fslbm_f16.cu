// Reduced-precision engines: PDFs stored as FP16 or BF16 deviations f - w_i,
// FP32 arithmetic; fill level, mass and bubble sums stay FP64.
#include "fslbm_engine.cuh"

namespace fslbm {
Ops ops_f16s(int q) { return q == 27 ? Engine<27, StoreF16S>::ops() : Engine<19, StoreF16S>::ops(); }
Ops ops_bf16s(int q) {
  return q == 27 ? Engine<27, StoreBF16S>::ops() : Engine<19, StoreBF16S>::ops();
}
}  // namespace fslbm
