// The interface list of the next step in cell order (arXiv 2207.13962,
// Sec. 2.2: the interface layer, whose cells the band kernels update).
// Kept in its own header: it is not part of the bulk sweep's sources.
#pragma once

#include "fslbm_cell.cuh"

namespace fslbm {

// Every interface cell of the final flags, in increasing cell index within
// each 4096-cell chunk.  A warp scans 512 consecutive cells (16 a lane, one
// 16-byte load); the block adds its eight warps' counts in shared memory
// and reserves its entries with one atomic per chunk, so a step issues a
// few thousand atomics on the list counter instead of one per warp (same-
// address atomics serialise in L2).  The order of the list changes no
// result (the band kernels read time-t neighbours and gather), but
// neighbouring entries then hold neighbouring cells, so the loads of a warp
// in the band kernels share sectors.  Appending the surviving cells warp by
// warp (the batched finalize does, before kb_compact_band rewrites its
// lists) interleaves runs from unrelated places a little more every step:
// on the 160x160x1024 Taylor bubble the interface kernel took 47.8 us just
// after init and 81 us fifty steps later, 47 us with the list in cell order.
constexpr int kCompactCells = 16;                       // cells a lane scans
constexpr int kCompactChunk = (kBlock / 32) * 32 * kCompactCells;  // cells a block scans at once

// One block's chunk [chunk, chunk + kCompactChunk) of a domain of N cells:
// its interface cells, appended in increasing index to list at the
// positions one atomic on *counter reserves (every thread of the block
// calls it; the chunk start is a multiple of 16, and flags 16-byte aligned).
__device__ __forceinline__ void compact_chunk(const uint8_t* __restrict__ flags, long long N,
                                              long long chunk, int* __restrict__ list, int* counter) {
  __shared__ int s_warp[kBlock / 32];
  __shared__ int s_base;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const long long c0 = chunk + (long long)wib * 32 * kCompactCells + (long long)kCompactCells * lane;
  unsigned m = 0u;  // interface cells among the lane's 16
  if (c0 + kCompactCells <= N) {
    const uint4 v = *reinterpret_cast<const uint4*>(flags + c0);
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < kCompactCells; ++j)
      if (((w[j >> 2] >> (8 * (j & 3))) & F_TYPE) == T_IFACE) m |= 1u << j;
  } else {
    for (int j = 0; j < kCompactCells && c0 + j < N; ++j)
      if ((flags[c0 + j] & F_TYPE) == T_IFACE) m |= 1u << j;
  }
  const int cnt = __popc(m);
  int incl = cnt;  // inclusive prefix sum over the lanes
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_warp[wib] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int w = 0; w < kBlock / 32; ++w) {
      const int t = s_warp[w];
      s_warp[w] = run;  // exclusive prefix over the warps
      run += t;
    }
    s_base = run > 0 ? atomicAdd(counter, run) : 0;
  }
  __syncthreads();
  int pos = s_base + s_warp[wib] + incl - cnt;
  while (m) {
    const int j = __ffs(m) - 1;
    m &= m - 1u;
    list[pos++] = (int)(c0 + j);
  }
  __syncthreads();  // s_warp and s_base are rewritten by the next chunk
}

// Single domain, after k_finalize (which leaves the next list empty).
static __global__ void __launch_bounds__(kBlock) k_compact_band(DPtrs d, KParams p, int parity) {
  const long long N = p.N;
  for (long long chunk = (long long)blockIdx.x * kCompactChunk; chunk < N;
       chunk += (long long)gridDim.x * kCompactChunk)
    compact_chunk(d.flags, N, chunk, d.band[parity ^ 1], &d.counts[parity ^ 1]);
}

// All domains of a batch, at the end of a batched step (after the buffer
// swap, so a domain's next list is band[parity]).  The batched finalize has
// already appended the same cells in warp order and set the list's count;
// this rewrites the entries in cell order, counting with cnt[k] (n entries,
// zero before the launch).  chunk_off[k]: prefix of the domains' chunk
// counts (n + 1 entries).
static __global__ void __launch_bounds__(kBlock) kb_compact_band(const DomRec* __restrict__ recs,
                                                                 const int* __restrict__ chunk_off, int n,
                                                                 int* cnt) {
  const int total = chunk_off[n];
  for (int g = blockIdx.x; g < total; g += gridDim.x) {
    int lo = 0, hi = n - 1;  // the domain k with chunk_off[k] <= g < chunk_off[k + 1]
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (chunk_off[mid] <= g) lo = mid;
      else hi = mid - 1;
    }
    const DomRec& r = recs[lo];
    compact_chunk(r.d.flags, r.p.N, (long long)(g - chunk_off[lo]) * kCompactChunk, r.d.band[r.parity],
                  &cnt[lo]);
  }
}

}  // namespace fslbm
