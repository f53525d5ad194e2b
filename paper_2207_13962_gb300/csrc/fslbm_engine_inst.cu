// One engine (a lattice and a PDF storage format) per object file: the build
// compiles this source once per pair with FSLBM_INST_NAME, FSLBM_INST_Q and
// FSLBM_INST_STORE defined (the FP64 engine without multiply-add contraction),
// so the engines compile in parallel.
#include "fslbm_engine.cuh"

#if !defined(FSLBM_INST_NAME) || !defined(FSLBM_INST_Q) || !defined(FSLBM_INST_STORE)
#error "FSLBM_INST_NAME, FSLBM_INST_Q and FSLBM_INST_STORE must be defined"
#endif

namespace fslbm {
Ops FSLBM_INST_NAME() { return Engine<FSLBM_INST_Q, FSLBM_INST_STORE>::ops(); }
}  // namespace fslbm
