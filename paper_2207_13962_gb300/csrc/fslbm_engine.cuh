// Host-side launch sequence of one FSLBM step for a given lattice and PDF
// storage format.  Included by the per-precision translation units, each of
// which exports one table of entry points (Ops) to the C-ABI layer.
#pragma once

#include "fslbm_internal.h"
#include <type_traits>

#include "fslbm_kernels.cuh"
#include "fslbm_band_list.cuh"
#include "fslbm_apply.cuh"

namespace fslbm {

// Calls f with the collision variant as a compile-time constant
// (bit 0: TRT, bit 1: Smagorinsky model, bit 2: free-slip faces).
template <class F>
inline void with_coll(int coll, F&& f) {
  switch (coll) {
    case 0: f(std::integral_constant<int, 0>{}); break;
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 5: f(std::integral_constant<int, 5>{}); break;
    case 6: f(std::integral_constant<int, 6>{}); break;
    default: f(std::integral_constant<int, 7>{}); break;
  }
}

// The kernels' variant: the collision variant and, in bit 2, whether the
// domain has free-slip faces (the free-slip logic is compiled only then).
inline int iface_coll(const KParams& p) { return coll_of(p) | slip_bit(p); }

template <int Q, class S>
struct Engine {
  // the FP32 and 16-bit engines stream the bulk sweep through TMA copies
  static constexpr bool kTmaBulk = S::kDev && !S::kExactRest && FSLBM_BULK_TMA != 0;
  // persistent bulk blocks per SM the sweep is compiled for
  static constexpr int bulk_blocks_per_sm() {
    return sizeof(typename S::Real) == 4 ? kBulkMinBlocks32 : 2;
  }
  static int grid_cells(const KParams& p) { return (p.N + kBlock - 1) / kBlock; }
  // blocks of k_compact_band: one chunk of kCompactChunk cells each, at most
  // 4 per band block (8 per SM; the grid loops over the remaining chunks)
  static int compact_grid(const KParams& p, int band_grid) {
    const long long chunks = ((long long)p.N + kCompactChunk - 1) / kCompactChunk;
    const long long cap = 4LL * band_grid;
    return (int)(chunks < cap ? chunks : cap);
  }
  // the FP32 and 16-bit engines fold the geometry pass into the bulk sweep
  static constexpr bool kFusedGeo = sizeof(typename S::Real) == 4 && !kTmaBulk;
  // shared-memory carveout (percent of the 228 KB) that holds a tile buffer
  // for every persistent block of the fused sweep; the rest stays L1
  static constexpr int fused_carveout() {
    return (kBulkMinBlocks32 * ((int)geometry_smem<typename S::Real>() + 1024) * 100 + 228 * 1024 - 1) /
           (228 * 1024);
  }

  static void init_cells(const DPtrs& d, const KParams& p, const uint8_t* raw, const double* fill,
                         const double* vel, const double* den, cudaStream_t st) {
    k_init_cells<Q, S><<<grid_cells(p), kBlock, 0, st>>>(raw, fill, vel, den, d, p, 0);
  }
  static void init_check(const KParams& p, const uint8_t* raw, int* bad, cudaStream_t st) {
    k_init_check<Q><<<grid_cells(p), kBlock, 0, st>>>(raw, p, bad);
  }
  static void cc_union(const uint8_t* raw, const KParams& p, int* lab, cudaStream_t st) {
    k_cc_union<Q><<<grid_cells(p), kBlock, 0, st>>>(raw, p, lab);
  }
  static void cc_assign(const uint8_t* raw, const KParams& p, const int* lab, const int* root_id,
                        int* bid, cudaStream_t st) {
    k_cc_assign<Q><<<grid_cells(p), kBlock, 0, st>>>(raw, p, lab, root_id, bid);
  }

  // One step reading pdf[parity], band[parity]; writing the other buffers.
  // With a Fork (and no stage events) the bulk sweep runs on the side stream
  // while geometry, interface update and the first conversion passes run on
  // the main stream; the streams join before k_apply, the first kernel that
  // reads post-collision PDFs of liquid cells.
  static void step(const DPtrs& d, const KParams& p, int parity, int band_grid, int bulk_grid,
                   cudaStream_t st, StageEvents* ev, const Fork* fk) {
    const int coll = iface_coll(p);
    if constexpr (kFusedGeo) {
      // geometry and bulk in one persistent launch, then the band chain
      constexpr size_t sm = geometry_smem<typename S::Real>();
      if (ev) {
        ev->mark(0, st);
        ev->mark(1, st);
      }
      with_coll(coll, [&](auto C) { k_bulk_geo<Q, S, decltype(C)::value><<<bulk_grid, kBulkBlock, sm, st>>>(d, p, parity); });
      if (ev) ev->mark(2, st);
      with_coll(coll, [&](auto C) {
        k_interface<Q, S, decltype(C)::value><<<band_grid * 2, 128, 0, st>>>(d, p, parity);
      });
      if (ev) ev->mark(3, st);
      // three resident blocks per SM (75 registers): about one band cell a thread
      k_resolve<Q><<<band_grid * 3 / 2, kBlock, 0, st>>>(d, p, parity);
      if (ev) ev->mark(4, st);
      k_count<Q><<<band_grid, kBlock, 0, st>>>(d, p, parity);
      if (ev) ev->mark(5, st);
      // the two independent parts of the apply stage, side by side in the
      // graph (one after the other while stages are timed)
      const bool side = fk && !ev;
      if (side) {
        cudaEventRecord(fk->fork, st);
        cudaStreamWaitEvent(fk->side, fk->fork, 0);
      }
      k_apply_new<Q, S><<<band_grid, 128, 0, side ? fk->side : st>>>(d, p, parity);
      if (side) cudaEventRecord(fk->join, fk->side);
      k_apply_band<Q, S><<<band_grid * 2, 128, 0, st>>>(d, p, parity);
      if (side) cudaStreamWaitEvent(st, fk->join, 0);
      if (ev) ev->mark(6, st);
      k_finalize<<<band_grid, kBlock, 0, st>>>(d, p, parity);
      // the bubble pressures (from finalize's sums) and the list rebuild (from
      // its flags) are independent: side by side in the graph as well
      const bool bub = p.bubble_model && d.nb > 0;
      const bool bub_side = side && bub;
      if (bub_side) {
        cudaEventRecord(fk->fork, st);
        cudaStreamWaitEvent(fk->side, fk->fork, 0);
        k_bubble<<<1, 256, 0, fk->side>>>(d, p);
        cudaEventRecord(fk->join, fk->side);
      }
      k_compact_band<<<compact_grid(p, band_grid), kBlock, 0, st>>>(d, p, parity);
      if (ev) ev->mark(7, st);
      if (bub && !bub_side) k_bubble<<<1, 256, 0, st>>>(d, p);
      if (bub_side) cudaStreamWaitEvent(st, fk->join, 0);
      if (ev) ev->mark(8, st);
      return;
    }
    auto bulk = [&](cudaStream_t s2) {
      with_coll(coll, [&](auto C) {
        constexpr int CO = decltype(C)::value;
        if constexpr (kTmaBulk && !coll_les(CO)) {
          constexpr size_t sm = tma_smem<Q, typename S::T>();
          k_bulk_tma<Q, S, CO><<<bulk_grid, kBulkBlock, sm, s2>>>(d, p, parity);
        } else {
          k_bulk<Q, S, CO><<<bulk_grid, kBulkBlock, 0, s2>>>(d, p, parity);
        }
      });
    };
    const bool forked = fk && !ev;
    auto fork_bulk = [&]() {
      cudaEventRecord(fk->fork, st);
      cudaStreamWaitEvent(fk->side, fk->fork, 0);
      bulk(fk->side);
      cudaEventRecord(fk->join, fk->side);
    };
    if (ev) ev->mark(0, st);
    if (forked) fork_bulk();
    k_geometry<Q, S><<<band_grid * kGeoGridMult, kGeoBlock, geometry_smem<typename S::Real>(), st>>>(d, p, parity);
    if (ev) ev->mark(1, st);
    if (!forked) bulk(st);
    if (ev) ev->mark(2, st);
    with_coll(coll, [&](auto C) {
      k_interface<Q, S, decltype(C)::value><<<band_grid * 2, 128, 0, st>>>(d, p, parity);
    });
    if (ev) ev->mark(3, st);
    k_resolve<Q><<<band_grid, kBlock, 0, st>>>(d, p, parity);
    if (ev) ev->mark(4, st);
    k_count<Q><<<band_grid, kBlock, 0, st>>>(d, p, parity);
    if (ev) ev->mark(5, st);
    if (forked) cudaStreamWaitEvent(st, fk->join, 0);
    k_apply<Q, S><<<band_grid * 2, 128, 0, st>>>(d, p, parity);
    if (ev) ev->mark(6, st);
    k_finalize<<<band_grid, kBlock, 0, st>>>(d, p, parity);
    k_compact_band<<<compact_grid(p, band_grid), kBlock, 0, st>>>(d, p, parity);
    if (ev) ev->mark(7, st);
    if (p.bubble_model && d.nb > 0) k_bubble<<<1, 256, 0, st>>>(d, p);
    if (ev) ev->mark(8, st);
  }

  // One step of all domains of a block table.  Same stages and stream fork
  // as step(); the plan kernels lay out each phase's work on the device, and
  // the last kernel swaps every domain's buffers.  collision: the variant
  // shared by the members (coll_of), with bit 2 set when one of them has
  // free-slip faces.
  static void batch_step(DomRec* recs, const BatchPlan& pl, int band_grid, int bulk_grid,
                         int collision, cudaStream_t st, const Fork* fk) {
    kb_plan_front<<<1, 1024, 0, st>>>(recs, pl);
    if constexpr (kFusedGeo) {
      constexpr size_t sm = geometry_smem<typename S::Real>();
      with_coll(collision, [&](auto C) {
        kb_bulk_geo<Q, S, decltype(C)::value><<<bulk_grid, kBulkBlock, sm, st>>>(recs, pl);
      });
      with_coll(collision, [&](auto C) {
        kb_interface<Q, S, decltype(C)::value><<<band_grid * 2, 128, 0, st>>>(recs, pl);
      });
      kb_resolve<Q><<<band_grid, kBlock, 0, st>>>(recs, pl);
      kb_count<Q><<<band_grid, kBlock, 0, st>>>(recs, pl);
      kb_plan_back<<<1, 1024, 0, st>>>(recs, pl);
      kb_apply<Q, S><<<band_grid * 2, 128, 0, st>>>(recs, pl);
      kb_finalize<<<band_grid, kBlock, 0, st>>>(recs, pl);
      kb_bubble_end<<<pl.n, 256, 0, st>>>(recs);
      (void)fk;
      return;
    }
    cudaEventRecord(fk->fork, st);
    cudaStreamWaitEvent(fk->side, fk->fork, 0);
    with_coll(collision, [&](auto C) {
      kb_bulk<Q, S, decltype(C)::value><<<bulk_grid, kBulkBlock, 0, fk->side>>>(recs, pl);
    });
    cudaEventRecord(fk->join, fk->side);
    kb_geometry<Q, S><<<band_grid * kGeoGridMult, kGeoBlock, geometry_smem<typename S::Real>(), st>>>(recs, pl);
    with_coll(collision, [&](auto C) {
      kb_interface<Q, S, decltype(C)::value><<<band_grid * 2, 128, 0, st>>>(recs, pl);
    });
    kb_resolve<Q><<<band_grid, kBlock, 0, st>>>(recs, pl);
    kb_count<Q><<<band_grid, kBlock, 0, st>>>(recs, pl);
    kb_plan_back<<<1, 1024, 0, st>>>(recs, pl);
    cudaStreamWaitEvent(st, fk->join, 0);
    kb_apply<Q, S><<<band_grid * 2, 128, 0, st>>>(recs, pl);
    kb_finalize<<<band_grid, kBlock, 0, st>>>(recs, pl);
    kb_bubble_end<<<pl.n, 256, 0, st>>>(recs);
  }

  static void observables(const DPtrs& d, const KParams& p, int parity, double* out,
                          cudaStream_t st) {
    k_obs_partial<Q, S><<<d.red_blocks, kBlock, 0, st>>>(d, p, parity, d.red);
    k_obs_final<<<1, 32, 0, st>>>(d.red, d.red_blocks, out);
  }

  static void pdf_out(const DPtrs& d, const KParams& p, int parity, double* out, cudaStream_t st) {
    k_pdf_out<Q, S><<<grid_cells(p), kBlock, 0, st>>>(d, p, parity, out);
  }

  static Ops ops() {
    cudaFuncSetAttribute(k_geometry<Q, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)geometry_smem<typename S::Real>());
    cudaFuncSetAttribute(kb_geometry<Q, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)geometry_smem<typename S::Real>());
    if constexpr (kTmaBulk) {
      cudaFuncSetAttribute(k_bulk_tma<Q, S, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tma_smem<Q, typename S::T>());
      cudaFuncSetAttribute(k_bulk_tma<Q, S, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tma_smem<Q, typename S::T>());
      // all persistent blocks resident at once: the most shared memory
      cudaFuncSetAttribute(k_bulk_tma<Q, S, 0>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      cudaFuncSetAttribute(k_bulk_tma<Q, S, 1>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    Ops o;
    o.init_cells = &init_cells;
    o.init_check = &init_check;
    o.cc_union = &cc_union;
    o.cc_assign = &cc_assign;
    o.step = &step;
    o.observables = &observables;
    o.pdf_out = &pdf_out;
    o.elem_size = sizeof(typename S::T);
    o.real_size = sizeof(typename S::Real);
    o.rest_size = S::kExactRest ? sizeof(int) : 0;
    if constexpr (kFusedGeo) {
      const void* fns[8] = {(const void*)&k_bulk_geo<Q, S, 0>, (const void*)&k_bulk_geo<Q, S, 1>,
                            (const void*)&k_bulk_geo<Q, S, 2>, (const void*)&k_bulk_geo<Q, S, 3>,
                            (const void*)&k_bulk_geo<Q, S, 4>, (const void*)&k_bulk_geo<Q, S, 5>,
                            (const void*)&k_bulk_geo<Q, S, 6>, (const void*)&k_bulk_geo<Q, S, 7>};
      for (int c = 0; c < 8; ++c) {
        o.bulk_fn[c] = fns[c];
        cudaFuncSetAttribute(fns[c], cudaFuncAttributePreferredSharedMemoryCarveout, fused_carveout());
      }
    } else {
      if constexpr (kTmaBulk) {
        o.bulk_fn[0] = (const void*)&k_bulk_tma<Q, S, 0>;
        o.bulk_fn[1] = (const void*)&k_bulk_tma<Q, S, 1>;
      } else {
        o.bulk_fn[0] = (const void*)&k_bulk<Q, S, 0>;
        o.bulk_fn[1] = (const void*)&k_bulk<Q, S, 1>;
      }
      o.bulk_fn[2] = (const void*)&k_bulk<Q, S, 2>;
      o.bulk_fn[3] = (const void*)&k_bulk<Q, S, 3>;
      o.bulk_fn[4] = (const void*)&k_bulk<Q, S, 4>;
      o.bulk_fn[5] = (const void*)&k_bulk<Q, S, 5>;
      o.bulk_fn[6] = (const void*)&k_bulk<Q, S, 6>;
      o.bulk_fn[7] = (const void*)&k_bulk<Q, S, 7>;
    }
    o.bulk_blocks_per_sm = bulk_blocks_per_sm();
    o.step_launches = 8;  // fused: the apply stage is two kernels
    o.bulk_smem = kTmaBulk ? tma_smem<Q, typename S::T>() : kFusedGeo ? geometry_smem<typename S::Real>() : 0;
    o.batch_step = &batch_step;
    // two plan kernels, geometry, bulk sweep, interface update, resolve,
    // count, apply, finalize, bubbles + buffer swap (one less when the
    // geometry is folded into the sweep)
    o.batch_step_launches = kFusedGeo ? 10 : 11;  // with kb_compact_band, launched by the batch
    if constexpr (kFusedGeo) {
      const void* fns[8] = {(const void*)&kb_bulk_geo<Q, S, 0>, (const void*)&kb_bulk_geo<Q, S, 1>,
                            (const void*)&kb_bulk_geo<Q, S, 2>, (const void*)&kb_bulk_geo<Q, S, 3>,
                            (const void*)&kb_bulk_geo<Q, S, 4>, (const void*)&kb_bulk_geo<Q, S, 5>,
                            (const void*)&kb_bulk_geo<Q, S, 6>, (const void*)&kb_bulk_geo<Q, S, 7>};
      for (int c = 0; c < 8; ++c) {
        o.batch_bulk_fn[c] = fns[c];
        cudaFuncSetAttribute(fns[c], cudaFuncAttributePreferredSharedMemoryCarveout, fused_carveout());
      }
    } else {
      o.batch_bulk_fn[0] = (const void*)&kb_bulk<Q, S, 0>;
      o.batch_bulk_fn[1] = (const void*)&kb_bulk<Q, S, 1>;
      o.batch_bulk_fn[2] = (const void*)&kb_bulk<Q, S, 2>;
      o.batch_bulk_fn[3] = (const void*)&kb_bulk<Q, S, 3>;
      o.batch_bulk_fn[4] = (const void*)&kb_bulk<Q, S, 4>;
      o.batch_bulk_fn[5] = (const void*)&kb_bulk<Q, S, 5>;
      o.batch_bulk_fn[6] = (const void*)&kb_bulk<Q, S, 6>;
      o.batch_bulk_fn[7] = (const void*)&kb_bulk<Q, S, 7>;
    }
    return o;
  }
};

}  // namespace fslbm
