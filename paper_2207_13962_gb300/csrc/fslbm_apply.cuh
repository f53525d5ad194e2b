// The apply stage of the FSLBM step (arXiv 2207.13962, Sec. 2.2: PDFs of new
// interface cells, excess-mass redistribution) as two kernels that the FP32
// and 16-bit engines run side by side in the step's graph.
#pragma once

#include "fslbm_kernels.cuh"

namespace fslbm {

// k_apply does both parts in one launch: the new interface cells first (few
// cells, long dependent chains: neighbour types, then the values they
// select, then the moments or PDFs those select), then the excess gather of
// the band (many cells, short chains).  The parts touch disjoint cells and
// read only what earlier kernels of the step wrote (shares, moment cache,
// post-collision PDFs, final marks), so they are independent, and the
// step's time for the stage is the longer of the two chains instead of
// their sum.  apply_cell is the same per-cell code in both forms.
template <int Q, class S>
__global__ void __launch_bounds__(128) k_apply_new(DPtrs d, KParams p, int parity) {
  const int nnew = d.counts[2];
  const int total = gridDim.x * blockDim.x;
  // dealt round-robin over the blocks, so that the chains spread over all SMs
  for (int j = threadIdx.x * gridDim.x + blockIdx.x; j < nnew; j += total) apply_cell<Q, S>(d, p, parity, j);
}

template <int Q, class S>
__global__ void __launch_bounds__(128) k_apply_band(DPtrs d, KParams p, int parity) {
  const int nnew = d.counts[2];
  const int nband = d.counts[parity];
  const int total = gridDim.x * blockDim.x;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nband; k += total)
    apply_cell<Q, S>(d, p, parity, nnew + k);
}

}  // namespace fslbm
