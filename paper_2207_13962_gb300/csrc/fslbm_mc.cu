// Mass-conserving engines: moving PDFs stored as FP32 or FP16 deviations on
// a fixed grid, the rest PDF in an FP64 slice that takes up every rounding
// of the collision, FP32 arithmetic; fill level, mass and bubble sums FP64.
#include "fslbm_engine.cuh"

namespace fslbm {
Ops ops_f32mc(int q) { return q == 27 ? Engine<27, StoreF32MC>::ops() : Engine<19, StoreF32MC>::ops(); }
Ops ops_f16smc(int q) {
  return q == 27 ? Engine<27, StoreF16SMC>::ops() : Engine<19, StoreF16SMC>::ops();
}
}  // namespace fslbm
