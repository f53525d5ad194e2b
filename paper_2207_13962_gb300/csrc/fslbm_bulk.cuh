// Bulk sweep of the FSLBM step (arXiv 2207.13962, Sec. 2.1): the pull
// stream-collide of liquid cells over the liquid segment list.  Kept in its
// own header so that the recorded DRAM traffic of this kernel is tied to the
// sources it is built from (this file, the cell layer and the common types).
#pragma once

#include "fslbm_cell.cuh"

namespace fslbm {
// ------------------------------------------------------------ bulk sweep
// Pull stream-collide of liquid cells (Eqs. nm-lbm-streaming, -collision)
// with bounce-back at obstacles.  Interface and gas cells are skipped.
//
// Bounce-back through the obstacle's slot: a fluid cell x whose pull source
// x - c_i is an obstacle cell writes, besides its own PDFs, f*_ibar(x) into
// slot i of that obstacle cell.  That slot is pulled by x alone, so the write
// is race-free, and next step x pulls its bounced-back PDF from the constant
// offset like any interior cell: the bulk sweep reads at constant offsets
// except next to a non-periodic domain face (own-slot bounce-back) or across
// a periodic face (wrapped index), which take the general path.  Every
// kernel that produces post-collision PDFs of a fluid cell (bulk, interface,
// new interface cells, init) writes these reflected copies.
constexpr int kBulkBlock = 256;

// One liquid cell, loads straight from global memory (storage formats of
// 2 bytes, and batches).
template <int Q, class S, int COLL>
__device__ __forceinline__ void bulk_cell(const DPtrs& d, const KParams& p, int parity, int c,
                                          uint8_t fl, bool general) {
  using R = typename S::Real;
  using T = typename S::T;
  const T* __restrict__ A = (const T*)d.pdf[parity];
  T* __restrict__ B = (T*)d.pdf[parity ^ 1];
  const long long Np = p.Np;
  R f[Q];
  // the mass-conserving formats hold the rest PDF in an FP64 slice
  constexpr int i0 = S::kExactRest ? 1 : 0;
  if (!general) {
    const T* Ac = A + c;
#pragma unroll
    for (int i = i0; i < Q; ++i) f[i] = load_w<S, Q>(Ac[p.dofs[i]], i);
  } else {
    int x, y, z;
    decode(p, c, x, y, z);
#pragma unroll
    for (int i = i0; i < Q; ++i)
      f[i] = load_w<S, Q>(A[pull_index_general<Q, coll_slip(COLL)>(p, d.flags, c, x, y, z, i)], i);
  }
  long long s_in = 0;
  if constexpr (S::kExactRest) {
    // the received stored values in grid steps, summed exactly
    const int r0 = rest_slice<Q, S>(A, Np)[c];
    f[0] = from_steps<S>(r0);
    s_in = r0;
#pragma unroll
    for (int i = 1; i < Q; ++i) s_in += grid_steps32<S>(f[i]);
  }
  bool bad = false;
  collide_any<Q, S, COLL>(f, p, bad);
  store_cell<Q, S, true>(B, Np, c, f, s_in, bad);
  if (fl & F_NEAR_WALL) write_reflected<Q, S>(d, p, B, c, d.wallmask[c], general, f);
  if (bad) d.err[0] = 1;
}

// One warp's share of the direct bulk sweep: groups [w G, w G + G) of the
// liquid group list, G = 32 / kSegCells (every lane of the warp calls it).
// Gas lanes that share a 32-byte sector of a PDF slice with a liquid lane
// store zero PDFs (gas values are never read): the sector is then written
// whole, which spares HBM a read-modify-write of it.  Interface lanes (the
// interface kernel writes them concurrently) and obstacle lanes (reflected
// copies) store nothing.
#ifndef FSLBM_BULK_FILL
#define FSLBM_BULK_FILL 1
#endif
template <int Q, class S, int COLL>
__device__ __forceinline__ void bulk_unit(const DPtrs& d, const KParams& p, int parity, int w,
                                          int nseg) {
  using T = typename S::T;
  using R = typename S::Real;
  constexpr int kGroups = 32 / kSegCells;
  constexpr int kFill = (32 / (int)sizeof(T)) < kSegCells ? (32 / (int)sizeof(T)) : kSegCells;
  const int lane = threadIdx.x & 31;
  const int e = w * kGroups + lane / kSegCells;
  const int c = e < nseg ? d.segs[e] * kSegCells + (lane % kSegCells) : p.N;
  const uint8_t fl = c < p.N ? d.flags[c] : (uint8_t)T_IFACE;
  const int t = fl & F_TYPE;
  const bool liq = t == T_LIQ;
  // the whole warp takes the general path when one of its cells needs it
  const bool general = __any_sync(0xffffffffu, liq && (fl & (F_FACE | F_WRAP)));
  const unsigned lm = __ballot_sync(0xffffffffu, liq);
  if (liq) {
    bulk_cell<Q, S, COLL>(d, p, parity, c, fl, general);
  } else if (FSLBM_BULK_FILL) {
    const unsigned grp = (lm >> (lane & ~(kFill - 1))) & ((1u << kFill) - 1u);
    if (grp && t == T_GAS) {
      T* __restrict__ B = (T*)d.pdf[parity ^ 1];
#pragma unroll
      for (int i = S::kExactRest ? 1 : 0; i < Q; ++i) B[(long long)i * p.Np + c] = S::store(R(0.0), W<Q, R>(i));
    }
    if constexpr (S::kExactRest) {
      // the int32 rest slice: 8 cells per 32-byte sector
      if (((lm >> (lane & ~7)) & 0xffu) && t == T_GAS) rest_slice<Q, S>(d.pdf[parity ^ 1], p.Np)[c] = 0;
    }
  }
}

// Warp-sized units of the list are handed out kBulkChunk consecutive ones at
// a time from a per-step counter (counts[6]: zero at init, cleared again by
// the finalize kernel of every step), so a warp sweeps neighbouring
// segments one after another while the 32-byte sectors they share are still
// in L2, and the grid works on one front of the list.  0 = a fixed stride
// over the list.
#ifndef FSLBM_BULK_DYN
#define FSLBM_BULK_DYN 4
#endif
constexpr int kBulkChunk = FSLBM_BULK_DYN;

// Resident blocks per SM a bulk sweep is compiled for: the FP32 engines
// kBulkMinBlocks32 (64 registers), 3 with the Smagorinsky model (its
// momentum flux needs more), the FP64 engine 2.
template <class S, int COLL>
constexpr int bulk_min_blocks() {
  return sizeof(typename S::Real) == 4 ? (coll_les(COLL) ? 3 : kBulkMinBlocks32) : 2;
}

// The sweep over the liquid segments by the warps of a persistent grid.
template <int Q, class S, int COLL>
__device__ __forceinline__ void bulk_sweep(const DPtrs& d, const KParams& p, int parity) {
  constexpr int kGroups = 32 / kSegCells;
  const int nseg = d.counts[5];
  if constexpr (kBulkChunk > 0) {
    const int nw = (nseg + kGroups - 1) / kGroups;
    for (;;) {
      int base = 0;
      if ((threadIdx.x & 31) == 0) base = atomicAdd(&d.counts[6], kBulkChunk);
      base = __shfl_sync(0xffffffffu, base, 0);
      if (base >= nw) break;
      const int end = base + kBulkChunk < nw ? base + kBulkChunk : nw;
      for (int w = base; w < end; ++w) bulk_unit<Q, S, COLL>(d, p, parity, w, nseg);
    }
  } else {
    const int warps = (gridDim.x * kBulkBlock) >> 5;
    for (int w = (blockIdx.x * kBulkBlock + threadIdx.x) >> 5; w * kGroups < nseg; w += warps)
      bulk_unit<Q, S, COLL>(d, p, parity, w, nseg);
  }
}

template <int Q, class S, int COLL>
__global__ void __launch_bounds__(kBulkBlock, (bulk_min_blocks<S, COLL>()))
    k_bulk(DPtrs d, KParams p, int parity) {
  bulk_sweep<Q, S, COLL>(d, p, parity);
}

}  // namespace fslbm
