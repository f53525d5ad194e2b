// FP64 engine.  This translation unit is compiled with --fmad=false so that
// each expression rounds as written, matching the CPU oracle bit for bit.
#include "fslbm_engine.cuh"

namespace fslbm {
Ops ops_f64(int q) { return q == 27 ? Engine<27, StoreF64>::ops() : Engine<19, StoreF64>::ops(); }
}  // namespace fslbm
