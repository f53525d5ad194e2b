// TMA-staged variant of the bulk sweep (arXiv 2207.13962, Sec. 2.1), built
// when FSLBM_BULK_TMA is 1 (off by default: on GB300 it is slower than the
// direct sweep, see the comment below).  Same cells, same arithmetic and
// the same stores as k_bulk, for the plain storage formats and collisions
// without the Smagorinsky model.
//
// Not to be enabled as it stands: when a bounded wait on a stage's copies
// gives up, the warp drains the copies it issued with waits that are bounded
// too; if those give up as well, the block can exit while bulk copies into
// its shared memory are still in flight, and they would land in the shared
// memory of a block that starts later on the SM.  The timeout path must
// first wait for every copy already issued before the variant is used.
#pragma once

#include "fslbm_bulk.cuh"

namespace fslbm {

#ifndef FSLBM_BULK_TMA
#define FSLBM_BULK_TMA 0
#endif

// Collision, store and reflected copies of one liquid cell whose pulled
// PDFs (working representation) are in f (the second half of bulk_cell).
template <int Q, class S, int COLL>
__device__ __forceinline__ void bulk_finish(const DPtrs& d, const KParams& p, int parity, int c,
                                            uint8_t fl, typename S::Real* f) {
  using T = typename S::T;
  T* __restrict__ B = (T*)d.pdf[parity ^ 1];
  bool bad = false;
  collide_any<Q, S, COLL>(f, p, bad);
  T* Bc = B + c;
#pragma unroll
  for (int i = 0; i < Q; ++i) Bc[(long long)i * p.Np] = store_w<S, Q>(f[i], i);
  if (fl & F_NEAR_WALL) write_reflected<Q, S>(d, p, B, c, d.wallmask[c], false, f);
  if (bad) d.err[0] = 1;
}

// ------------------------------------------------ TMA-staged bulk sweep
// FP32 and 16-bit engines.  Each warp streams its 32-cell segments through
// a two-stage ring in shared memory: while it collides segment k, the bulk
// copy engine (cp.async.bulk, completion counted on an mbarrier) brings in
// segment k + 1's 19 (27) pull windows and 32 flag bytes.  A window is the
// 32 cells of slice i a segment pulls from, widened to 16-byte boundaries.
// The bytes in flight per SM are then set by the ring, not by the registers
// of the loads, which is what limits the direct sweep where a third of the
// lanes of a segment hold no liquid.  Measured on GB300 it is slower all
// the same (Taylor bubble 0.86 ms against 0.55 ms, 256^3 box 0.98 against
// 0.47 ms): one bulk copy per 144-byte window costs the copy engine about
// 30 SM cycles, and 20 of them per 32 cells outpace what it issues.  Warps next to a domain face (general
// path) load directly; their window copies are still waited for.  Every
// wait is bounded: on expiry the warp records it in err[1], drains its
// copies (bounded again) and stops.
constexpr int kTmaStages = 2;
template <class T>
__host__ __device__ constexpr int tma_align() { return 16 / (int)sizeof(T); }  // elements per 16 B
template <class T>
__host__ __device__ constexpr int tma_win() { return 32 + tma_align<T>(); }    // window elements
template <int Q, class T>
__host__ __device__ constexpr int tma_stage_bytes() { return Q * tma_win<T>() * (int)sizeof(T) + 32; }
template <int Q, class T>
__host__ __device__ constexpr size_t tma_smem() {
  return (size_t)(kBulkBlock / 32) * kTmaStages * (tma_stage_bytes<Q, T>() + 8);
}
#ifndef FSLBM_TMA_SPIN
#define FSLBM_TMA_SPIN (1 << 22)
#endif

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// true once the phase with the given parity has completed; false when the
// bounded number of polls ran out
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < FSLBM_TMA_SPIN; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Element index where segment seg's window of slice i starts (16-byte
// aligned, clamped into the buffer of q * Np elements) and the offset of
// the segment's first pull source in it.
template <class T>
__device__ __forceinline__ long long tma_win_start(const KParams& p, int q, int i, int seg, int& shift) {
  constexpr int AL = tma_align<T>();
  const long long src = p.dofs[i] + (long long)seg * 32;
  long long a = src >= 0 ? (src / AL) * AL : 0;
  const long long last = (long long)q * p.Np - tma_win<T>();
  if (a > last) a = last;
  shift = (int)(src - a);
  return a;
}

// Lane 0: arm the stage's barrier with its byte count and start its copies.
template <int Q, class T>
__device__ __forceinline__ void tma_issue(const DPtrs& d, const KParams& p, const T* A, int seg,
                                          unsigned char* stage, uint32_t bar) {
  constexpr int WB = tma_win<T>() * (int)sizeof(T);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
               "r"((uint32_t)tma_stage_bytes<Q, T>())
               : "memory");
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    int sh;
    const long long a = tma_win_start<T>(p, Q, i, seg, sh);
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(stage + i * WB)),
        "l"(A + a), "r"((uint32_t)WB), "r"(bar)
        : "memory");
  }
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], 32, [%2];" ::"r"(
          smem_addr(stage + Q * WB)),
      "l"(d.flags + (long long)seg * 32), "r"(bar)
      : "memory");
}

template <int Q, class S, int COLL>
__global__ void __launch_bounds__(kBulkBlock, kBulkMinBlocks32) k_bulk_tma(DPtrs d, KParams p, int parity) {
  using T = typename S::T;
  using R = typename S::Real;
  constexpr int WB = tma_win<T>() * (int)sizeof(T);
  constexpr int SB = tma_stage_bytes<Q, T>();
  extern __shared__ __align__(128) unsigned char t_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  unsigned char* ring = t_smem + (size_t)wib * kTmaStages * SB;
  uint64_t* bars = (uint64_t*)(t_smem + (size_t)(kBulkBlock / 32) * kTmaStages * SB) + wib * kTmaStages;
  const uint32_t bar0 = smem_addr(&bars[0]), bar1 = smem_addr(&bars[1]);
  const T* A = (const T*)d.pdf[parity];
  T* __restrict__ B = (T*)d.pdf[parity ^ 1];
  const int nseg = d.counts[5];
  const int warps = gridDim.x * (kBulkBlock / 32);
  const int w0 = blockIdx.x * (kBulkBlock / 32) + wib;
  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  int seg0 = w0 < nseg ? d.segs[w0] : -1;
  int seg1 = w0 + warps < nseg ? d.segs[w0 + warps] : -1;
  if (lane == 0 && seg0 >= 0) tma_issue<Q, T>(d, p, A, seg0, ring, bar0);
  int k = 0;
  for (int w = w0; w < nseg; w += warps, ++k) {
    const int st = k & 1;
    const int seg2 = w + 2 * warps < nseg ? d.segs[w + 2 * warps] : -1;
    // the other stage last held segment k - 1, whose values every lane has
    // consumed (they fed the stores of the previous iteration)
    __syncwarp();
    if (lane == 0 && seg1 >= 0) tma_issue<Q, T>(d, p, A, seg1, ring + (st ^ 1) * SB, st ? bar0 : bar1);
    if (!mbar_wait(st ? bar1 : bar0, (uint32_t)((k >> 1) & 1))) {
      if (lane == 0) d.err[1] = 1;
      // drain this stage's copies and the ones issued above (bounded), then stop
      mbar_wait(st ? bar1 : bar0, (uint32_t)((k >> 1) & 1));
      if (seg1 >= 0) mbar_wait(st ? bar0 : bar1, (uint32_t)(((k + 1) >> 1) & 1));
      return;
    }
    const unsigned char* sg = ring + st * SB;
    const int c = seg0 * 32 + lane;
    const uint8_t fl = c < p.N ? sg[Q * WB + lane] : (uint8_t)T_IFACE;
    const int t = fl & F_TYPE;
    const bool liq = t == T_LIQ;
    const bool general = __any_sync(0xffffffffu, liq && (fl & (F_FACE | F_WRAP)));
    const unsigned lm = __ballot_sync(0xffffffffu, liq);
    if (liq) {
      if (!general) {
        R f[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          int sh;
          (void)tma_win_start<T>(p, Q, i, seg0, sh);
          f[i] = load_w<S, Q>(((const T*)(sg + i * WB))[sh + lane], i);
        }
        bulk_finish<Q, S, COLL>(d, p, parity, c, fl, f);
      } else {
        bulk_cell<Q, S, COLL>(d, p, parity, c, fl, true);
      }
    } else if (FSLBM_BULK_FILL) {
      constexpr int kFill = 32 / (int)sizeof(T);
      const unsigned grp = (lm >> (lane & ~(kFill - 1))) & ((1u << kFill) - 1u);
      if (grp && t == T_GAS) {
#pragma unroll
        for (int i = 0; i < Q; ++i) B[(long long)i * p.Np + c] = S::store(R(0.0), W<Q, R>(i));
      }
    }
    seg0 = seg1;
    seg1 = seg2;
  }
}

}  // namespace fslbm
