// FSLBM step kernels (arXiv 2207.13962, Sec. 2-3), templated on the lattice
// (Q = 19 / 27) and the PDF storage format S (FP64, FP32, FP16/BF16 shifted).
//
// One step, in stream order:
//   k_geometry   band   K8 smoothing, Parker-Youngs normal, FDM curvature,
//                       gas density rho^G, Thuerey class
//   k_bulk       grid   pull stream + bounce-back + collide of liquid cells
//   k_interface  band   pull, free-surface BC of the chosen variant, mass
//                       exchange, fill update, collide, conversion marks
//   k_resolve    band   conflict rule, claims of gas/liquid neighbours
//   k_count      band   excess-mass receivers, deferral, shares
//   k_apply      band+new  excess gather, new interface cells' PDFs
//   k_finalize   band+new  final flags, next interface list, bubble sums
//   k_bubble     1 block   bubble volume pressure
// The interface work runs only on the compacted list of interface cells
// ("band") and on the cells that conversion turns into interface cells.
// Conversion and excess redistribution are gather-only: each cell computes
// its own new values from its neighbours, so the flag field is deterministic.
//
// In the FP64 instantiation the kernels are compiled without FMA contraction
// and every expression keeps the association and summation order of the
// plain CPU oracle, so results agree to the last bit.
#pragma once

#include "fslbm_bulk_tma.cuh"
#include <type_traits>

namespace fslbm {

// ------------------------------------------------------------------ init
// Validates raw flags: values <= 3 and no liquid cell next to a gas cell.
template <int Q>
__global__ void k_init_check(const uint8_t* __restrict__ raw, KParams p, int* bad) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.N) return;
  uint8_t t = raw[c];
  if (t > 3) {
    atomicOr(bad, 1);
    return;
  }
  if (t != T_LIQ) return;
  int x, y, z;
  decode(p, c, x, y, z);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    int n = nbr(p, x, y, z, CX(i), CY(i), CZ(i));
    if (n >= 0 && raw[n] == T_GAS) atomicOr(bad, 2);
  }
}

// Initial fields: phi, m = phi rho (Eq. nm-fslbm-mass), f = f^eq(rho, u).
template <int Q, class S>
__global__ void k_init_cells(const uint8_t* __restrict__ raw, const double* __restrict__ fill,
                             const double* __restrict__ vel, const double* __restrict__ den,
                             DPtrs d, KParams p, int parity) {
  using R = typename S::Real;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.N) return;
  const uint8_t t = raw[c];
  int x, y, z;
  decode(p, c, x, y, z);
  uint8_t fl = t;
  uint32_t wm = 0u;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    int n = nbr(p, x, y, z, CX(i), CY(i), CZ(i));
    if (n < 0) fl |= F_FACE;
    else if (raw[n] == T_OBST) fl |= F_NEAR_WALL;
    const int X = x + CX(i), Y = y + CY(i), Z = z + CZ(i);
    if (n >= 0 && (X < 0 || X >= p.nx || Y < 0 || Y >= p.ny || Z < 0 || Z >= p.nz)) fl |= F_WRAP;
    const int s = nbr(p, x, y, z, -CX(i), -CY(i), -CZ(i));
    if (s >= 0 && raw[s] == T_OBST) wm |= 1u << i;
  }
  d.flags[c] = fl;
  d.wallmask[c] = wm;
  const double r = den ? den[c] : 1.0;
  d.phi[c] = (t == T_LIQ) ? 1.0 : (t == T_IFACE) ? fill[c] : 0.0;
  d.mass[c] = (t == T_LIQ) ? r : (t == T_IFACE) ? fill[c] * r : 0.0;
  d.cls[c] = 0;
  d.mark[c] = 0;
  d.conv[c] = 0;
  d.cfin[c] = 0;
  d.claim[c] = 0;
  d.share[c] = 0.0;
  typename S::T* P = (typename S::T*)d.pdf[parity];
  typename S::T* P2 = (typename S::T*)d.pdf[parity ^ 1];
  const bool fluid = (t == T_LIQ || t == T_IFACE);
  if (!fluid) return;  // gas and obstacle slots stay as cleared (obstacle
                       // slots receive their neighbours' reflected copies)
  R fe[Q];
  if constexpr (S::kDev) {
    // deviation f^eq - w in FP32 from drho = rho - 1 taken in FP64 (every
    // term is then of the size of a deviation)
    const R ux = vel ? R(vel[c]) : R(0.0);
    const R uy = vel ? R(vel[(long long)p.N + c]) : R(0.0);
    const R uz = vel ? R(vel[2LL * p.N + c]) : R(0.0);
#pragma unroll
    for (int i = 0; i < Q; ++i) fe[i] = feq_dev<Q, R>(i, R(r - 1.0), R(r), ux, uy, uz);
  } else {
    const R ux = vel ? R(vel[c]) : R(0.0);
    const R uy = vel ? R(vel[(long long)p.N + c]) : R(0.0);
    const R uz = vel ? R(vel[2LL * p.N + c]) : R(0.0);
#pragma unroll
    for (int i = 0; i < Q; ++i) fe[i] = feq_i<Q, R>(i, R(r), ux, uy, uz);
  }
  // the mass-conserving formats store the density deviation r - 1 (to
  // their grid): the rest PDF takes up the rounding of the others
  bool over = false;
  const long long s_in = S::kExactRest ? __double2ll_rn((r - 1.0) * (double)(1LL << grid_shift<S>())) : 0;
  store_cell<Q, S>(P, p.Np, c, fe, s_in, over);
  store_cell<Q, S>(P2, p.Np, c, fe, s_in, over);
  if (wm) {
    write_reflected<Q, S>(d, p, P, c, wm, (fl & F_WRAP) != 0, fe);
    write_reflected<Q, S>(d, p, P2, c, wm, (fl & F_WRAP) != 0, fe);
  }
}

// Ordered-by-warp compaction of all interface cells into a list.
static __global__ void k_compact_full(const uint8_t* __restrict__ flags, int N, int* list,
                               int* count) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  bool pred = (c < N) && ((flags[c] & F_TYPE) == T_IFACE);
  int pos = warp_append(count, pred);
  if (pred) list[pos] = c;
}

// -------------------------------------------------------- bubble labels
// Connected gas regions (lattice neighbourhood, periodic wrap) at init, on
// the device.  Union-find with lock-free hooking: every gas cell starts as
// its own root; a union hooks the root with the larger caller index
// x + nx (y + ny z) under the other with compare-and-swap (a root is
// re-parented only while it is still a root), so every root ends as the
// cell of its component with the lowest caller index, whatever the storage
// order.  Bubbles are then numbered in the order of their roots' caller
// indices, i.e. of their lowest cell index.
__device__ __forceinline__ int cc_find(const int* lab, int x) {
  int p = lab[x];
  while (p != x) {
    x = p;
    p = lab[x];
  }
  return x;
}

static __global__ void k_cc_init(const uint8_t* __restrict__ raw, int N, int* lab) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < N) lab[c] = raw[c] == T_GAS ? c : -1;
}

template <int Q>
__global__ void k_cc_union(const uint8_t* __restrict__ raw, KParams p, int* lab) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.N || raw[c] != T_GAS) return;
  int x, y, z;
  decode(p, c, x, y, z);
  for (int i = 1; i < Q; ++i) {
    const int n = nbr(p, x, y, z, CX(i), CY(i), CZ(i));
    if (n < 0 || n >= c || raw[n] != T_GAS) continue;  // each pair once (storage order)
    int a = cc_find(lab, c), b = cc_find(lab, n);
    while (a != b) {
      if (ext_index(p, a) > ext_index(p, b)) {
        const int t = a;
        a = b;
        b = t;
      }
      const int old = atomicCAS(&lab[b], b, a);  // hook root b under a
      if (old == b) break;
      b = cc_find(lab, old);
      a = cc_find(lab, a);
    }
  }
}

static __global__ void k_cc_compress(int N, int* lab) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < N && lab[c] >= 0) lab[c] = cc_find(lab, c);
}

// Storage index of the cell with caller index e.
__device__ __forceinline__ int storage_of_ext(const KParams& p, int e) {
  const int x = e % p.nx, t = e / p.nx;
  return cidx(p, x, t % p.ny, t / p.ny);
}

// Roots per block of kCcChunk cells, counted in the caller's cell order
// (pass 1 of the numbering).
constexpr int kCcChunk = 1024;
static __global__ void k_cc_count(KParams p, const int* __restrict__ lab, int* block_roots) {
  __shared__ int cnt;
  const int N = p.N;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int mine = 0;
  for (int k = threadIdx.x; k < kCcChunk; k += blockDim.x) {
    const long long e = (long long)blockIdx.x * kCcChunk + k;
    if (e < N) {
      const int c = storage_of_ext(p, (int)e);
      if (lab[c] == c) ++mine;
    }
  }
  atomicAdd(&cnt, mine);
  __syncthreads();
  if (threadIdx.x == 0) block_roots[blockIdx.x] = cnt;
}

// Exclusive scan of the per-block root counts (one block); total in off[n].
static __global__ void k_cc_scan(int nblocks, const int* __restrict__ block_roots, int* off) {
  block_prefix(nblocks, off, [&](int k) { return block_roots[k]; });
}

// Bubble id of every root in the caller's index order (pass 2): warps walk
// their block's chunk in order, so ranks within the chunk follow the index.
static __global__ void k_cc_number(KParams p, const int* __restrict__ lab, const int* __restrict__ off,
                                   int* root_id) {
  __shared__ int base;
  const int N = p.N;
  if (threadIdx.x == 0) base = off[blockIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  // one warp numbers the chunk sequentially in 32-cell steps
  if (threadIdx.x < 32) {
    int b = base;
    for (int k = 0; k < kCcChunk; k += 32) {
      const long long e = (long long)blockIdx.x * kCcChunk + k + lane;
      const int c = e < N ? storage_of_ext(p, (int)e) : -1;
      const bool root = c >= 0 && lab[c] == c;
      const unsigned m = __ballot_sync(0xffffffffu, root);
      if (root) root_id[c] = b + __popc(m & ((1u << lane) - 1u));
      b += __popc(m);
    }
  }
}

// Bubble id of gas cells (their root's number) and of interface cells (the
// lowest id among their gas neighbours); -1 elsewhere.
template <int Q>
__global__ void k_cc_assign(const uint8_t* __restrict__ raw, KParams p, const int* __restrict__ lab,
                            const int* __restrict__ root_id, int* bid) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.N) return;
  const uint8_t t = raw[c];
  if (t == T_GAS) {
    bid[c] = root_id[lab[c]];
    return;
  }
  int best = -1;
  if (t == T_IFACE) {
    int x, y, z;
    decode(p, c, x, y, z);
    for (int i = 1; i < Q; ++i) {
      const int n = nbr(p, x, y, z, CX(i), CY(i), CZ(i));
      if (n < 0 || raw[n] != T_GAS) continue;
      const int b = root_id[lab[n]];
      if (best < 0 || b < best) best = b;
    }
  }
  bid[c] = best;
}

// Initial bubble volumes in 2^-32 fixed point: gas cells count 1, interface
// cells 1 - phi (the same terms as the step's volume sums).
static __global__ void k_cc_volumes(const uint8_t* __restrict__ raw, const double* __restrict__ fill,
                                    int N, const int* __restrict__ bid, long long* gas_cnt,
                                    long long* iface_fix) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int b = -1;
  long long g = 0, v = 0;
  if (c < N) {
    b = bid[c];
    if (b >= 0 && raw[c] == T_GAS) g = 1;
    if (b >= 0 && raw[c] == T_IFACE) v = __double2ll_rn((1.0 - fill[c]) * 4294967296.0);
  }
  unsigned remaining = __ballot_sync(0xffffffffu, b >= 0);
  while (remaining) {
    const int leader = __ffs(remaining) - 1;
    const int bb = __shfl_sync(0xffffffffu, b, leader);
    const bool mine = b == bb;
    long long sg = mine ? g : 0, sv = mine ? v : 0;
    for (int o = 16; o > 0; o >>= 1) {
      sg += __shfl_xor_sync(0xffffffffu, sg, o);
      sv += __shfl_xor_sync(0xffffffffu, sv, o);
    }
    if (lane == leader) {
      if (sg) atomicAdd((unsigned long long*)&gas_cnt[bb], (unsigned long long)sg);
      if (sv) atomicAdd((unsigned long long*)&iface_fix[bb], (unsigned long long)sv);
    }
    remaining &= ~__ballot_sync(0xffffffffu, mine);
  }
}

static __global__ void k_cc_v0(int nb, const long long* gas_cnt, long long* iface_fix, double* V0,
                               double* Vcur, double* pV, double pv0) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const long long acc = gas_cnt[b] * 4294967296LL + iface_fix[b];
  const double V = __ll2double_rn(acc) / 4294967296.0;
  V0[b] = V;
  Vcur[b] = V;
  pV[b] = pv0;
  iface_fix[b] = 0;
}

// ------------------------------------------------- bubble relabelling
// Coalescence and segmentation of bubbles between steps: the bubbles are
// labelled again from the current flags (the kernels above), and the gas of
// each old bubble goes to the new ones in proportion to the fixed-point
// volume of its cells that each holds (the host combines the overlaps).

// Cell types of the flags (the labelling kernels take bare types).
static __global__ void k_types(const uint8_t* __restrict__ flags, int N, uint8_t* raw) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < N) raw[c] = flags[c] & F_TYPE;
}

// Overlap of old and new bubbles in 2^-32 fixed point: M[A * W + C + 1]
// for a cell of old id A and new id C (column 0: no new bubble), fr[C] for
// the cells of new bubble C that carried no id.  Integer sums, one atomic
// per (old, new) pair present in a warp.
static __global__ void k_bubble_overlap(const uint8_t* __restrict__ raw, const double* __restrict__ phi,
                                        const int* __restrict__ old_bid, const int* __restrict__ bid, int N,
                                        int W, long long* M, long long* fr) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  long long key = -1, v = 0;
  if (c < N) {
    const uint8_t t = raw[c];
    if (t == T_GAS) v = 4294967296LL;
    else if (t == T_IFACE) v = __double2ll_rn((1.0 - phi[c]) * 4294967296.0);
    if (t == T_GAS || t == T_IFACE) {
      const int A = old_bid[c], C = bid[c];
      if (A >= 0) key = (long long)A * W + (C + 1);
      else if (C >= 0) key = -2 - (long long)C;  // fr[C]
    }
  }
  unsigned remaining = __ballot_sync(0xffffffffu, key != -1);
  while (remaining) {
    const int leader = __ffs(remaining) - 1;
    const long long kk = __shfl_sync(0xffffffffu, key, leader);
    const bool mine = key == kk;
    long long sv = mine ? v : 0;
    for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
    if (lane == leader && sv) {
      long long* dst = kk >= 0 ? &M[kk] : &fr[-2 - kk];
      atomicAdd((unsigned long long*)dst, (unsigned long long)sv);
    }
    remaining &= ~__ballot_sync(0xffffffffu, mine);
  }
}

// Volumes and pressures of the new bubbles (p^V = p^V(0) V0 / V, as in the
// step's bubble update), with their gas reference V0 already set.
static __global__ void k_relabel_pressure(int nb, const long long* gas_cnt, long long* iface_fix,
                                          const double* V0, double* Vcur, double* pV, double pv0) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const long long acc = gas_cnt[b] * 4294967296LL + iface_fix[b];
  const double V = __ll2double_rn(acc) / 4294967296.0;
  pV[b] = (V > 0.0) ? (pv0 * V0[b]) / V : pv0;
  Vcur[b] = V;
  iface_fix[b] = 0;
}

// ------------------------------------------------------------- geometry
// K8 weights (1 - r^2/4)^4 on the 3x3x3 block: r^2 = 0, 1, 2, 3.
template <class R>
__device__ __forceinline__ R k8w(int n2) {
  return n2 == 0 ? R(1.0) : n2 == 1 ? R(0.31640625) : n2 == 2 ? R(0.0625) : R(0.00390625);
}

// Geometry on 8^3 tiles that hold interface cells (tile list built by
// k_finalize).  The tile's fill levels with a halo of 3 sit in shared memory;
// phi~ (K8 smoothing, radius 2) is formed on the 12^3 sub-box, n^ (Parker-
// Youngs, Eq. nm-fslbm-normal) on the 10^3 sub-box and kappa = -div(n^) on
// the interface cells of the tile.  Obstacle and out-of-domain stencil
// points take the stencil centre's value.  In the FP64 engine each value
// uses the same arithmetic and summation order as a per-cell evaluation.
constexpr int GT = 8;                    // tile edge
constexpr int GE = GT + 6;               // box edge with halo 3
constexpr int GB = GE * GE * GE;         // 2744 box positions
constexpr int GS = GT + 4;               // phi~ sub-box edge (12)
constexpr int GN = GT + 2;               // n^ sub-box edge (10)
constexpr int kGeoBlock = 192;  // the z-column phases use 144 and 100 threads
#ifndef FSLBM_GEO_LOAD_BATCH
#define FSLBM_GEO_LOAD_BATCH 6
#endif
constexpr int kGeoLoadBatch = FSLBM_GEO_LOAD_BATCH;  // box positions a thread loads at once
// geometry blocks per interface-band block: each tile's block runs four
// dependent shared-memory phases, so many resident tiles hide the latency
#ifndef FSLBM_GEO_MULT
#define FSLBM_GEO_MULT 3
#endif
constexpr int kGeoGridMult = FSLBM_GEO_MULT;
#ifndef FSLBM_GEO_MINB
#define FSLBM_GEO_MINB 3
#endif
constexpr int kGeoMinBlocks = FSLBM_GEO_MINB;  // resident geometry blocks per SM compiled for

// Fill level stored for obstacle and out-of-domain box positions: stencils
// substitute their centre's value there (no fill level comes near it).
template <class R>
__device__ __forceinline__ R kObstacle() { return R(-1.0e30); }
template <class R>
__device__ __forceinline__ bool is_obstacle(R v) { return v < R(-1.0e29); }

// Shared memory of one tile: the fill-level box, whose space the normals
// take over once the smoothing has read it, the smoothed sub-box and the
// types.
constexpr int kGeoBoxSlots = GB > 3 * GN * GN * GN ? GB : 3 * GN * GN * GN;
template <class R>
constexpr size_t geometry_smem() {
  return sizeof(R) * (kGeoBoxSlots + GS * GS * GS) + GB;
}

// One 8^3 tile of the geometry pass (all NT threads of the block call it).
template <int Q, class S, int NT = kGeoBlock>
__device__ __forceinline__ void geometry_tile(const DPtrs& d, const KParams& p, int tile,
                                              unsigned char* g_smem) {
  using R = typename S::Real;
  constexpr int kPer = (GB + NT - 1) / NT;  // box positions per thread
  R* sphi = (R*)g_smem;
  R* snh = sphi;  // written after the smoothing's last read of sphi
  R* sps = sphi + kGeoBoxSlots;
  uint8_t* styp = (uint8_t*)(sps + GS * GS * GS);
  const int ntx = (p.nx + GT - 1) / GT, nty = (p.ny + GT - 1) / GT;
  R* nhat = (R*)d.nhat;
  R* rhog = (R*)d.rhog;
  const R wsum = R(3.6796875);

    const int tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
    const int ox = tx * GT - 3, oy = ty * GT - 3, oz = tz * GT - 3;
    // all of a thread's global reads of the box are issued before the first
    // shared-memory store (NT threads, kPer positions each)
    __syncthreads();
    // Thread t loads box position t + r NT counted in the cells'
    // storage order (its first coordinate runs along the contiguous axis),
    // so that the loads of a warp coalesce whatever the storage order; the
    // shared-memory box itself is indexed in the caller's axes.
    auto box_pos = [&](int b, int& i, int& j, int& k) {
      const int k0 = b % GE, k1 = (b / GE) % GE, k2 = b / (GE * GE);
      i = sel3(p.inv[0], k0, k1, k2);
      j = sel3(p.inv[1], k0, k1, k2);
      k = sel3(p.inv[2], k0, k1, k2);
    };
    // in kLoadRounds rounds of at most kBatch positions, so that the loads in
    // flight fit the registers of a 64-register thread
    constexpr int kBatch = kGeoLoadBatch < kPer ? kGeoLoadBatch : kPer;
    bool solid_here = false;  // an obstacle or a position outside the domain
#pragma unroll
    for (int r0 = 0; r0 < kPer; r0 += kBatch) {
      uint8_t tv[kBatch];
      R pv[kBatch];
#pragma unroll
      for (int q = 0; q < kBatch; ++q) {
        const int b = threadIdx.x + (r0 + q) * NT;
        tv[q] = 4;  // outside the domain: solid
        pv[q] = R(0.0);
        if (r0 + q < kPer && b < GB) {
          int i, j, k;
          box_pos(b, i, j, k);
          const int X = wrapc(ox + i, p.nx, p.per[0]);
          const int Y = wrapc(oy + j, p.ny, p.per[1]);
          const int Z = wrapc(oz + k, p.nz, p.per[2]);
          if (X >= 0 && Y >= 0 && Z >= 0) {
            const int c = cidx(p, X, Y, Z);
            tv[q] = d.flags[c] & F_TYPE;
            if constexpr (sizeof(R) == 4) pv[q] = d2f(d.phi[c]);
            else pv[q] = d.phi[c];
          }
        }
      }
#pragma unroll
      for (int q = 0; q < kBatch; ++q) {
        const int b = threadIdx.x + (r0 + q) * NT;
        if (r0 + q < kPer && b < GB) {
          int i, j, k;
          box_pos(b, i, j, k);
          const int bs = i + GE * (j + GE * k);
          styp[bs] = tv[q];
          sphi[bs] = tv[q] >= T_OBST ? kObstacle<R>() : pv[q];
          solid_here |= tv[q] >= T_OBST;
        }
      }
    }
    // without an obstacle in the box the stencils below need no
    // substitution (most tiles)
    const bool solid = __syncthreads_or(solid_here) != 0;
    // The FP32 engines evaluate the same stencils grouped by z-plane.  The K8
    // weights depend on r^2 only, so a plane contributes its centre, the sum
    // of its 4 in-plane face neighbours and of its 4 in-plane corners; the
    // Parker-Youngs weights (2-|d|)(2-|d'|) factor into [1 2 1] x [1 2 1] x
    // [-1 0 1].  An obstacle point takes the value of the stencil's centre,
    // which is the same for every plane of the window, so a plane keeps the
    // sum over its other points and, beside it, the (weighted) count of its
    // obstacle points, which multiplies the centre value at the end.  Each
    // plane's sums are formed once and slide along z (other rounding than a
    // per-cell evaluation, a fraction of its operations and registers).
    auto planes32 = [&](auto SOLID) {
      constexpr bool kSolid = decltype(SOLID)::value;
      auto nz = [&](R v) { return (kSolid && is_obstacle(v)) ? R(0.0) : v; };
      auto ob = [&](R v) { return (kSolid && is_obstacle(v)) ? R(1.0) : R(0.0); };
      if (threadIdx.x < GS * GS) {
        const int i = threadIdx.x % GS + 1, j = threadIdx.x / GS + 1;
        // centre, face sum, corner sum and their obstacle counts
        auto plane = [&](int kk, R& c0, R& f4, R& c4, R& nf, R& nc) {
          const R* q = sphi + i + GE * (j + GE * kk);
          c0 = q[0];
          const R a = q[-1], b = q[1], c = q[-GE], e = q[GE];
          const R u = q[-GE - 1], v = q[-GE + 1], w = q[GE - 1], x = q[GE + 1];
          f4 = (nz(a) + nz(b)) + (nz(c) + nz(e));
          c4 = (nz(u) + nz(v)) + (nz(w) + nz(x));
          if constexpr (kSolid) {
            nf = (ob(a) + ob(b)) + (ob(c) + ob(e));
            nc = (ob(u) + ob(v)) + (ob(w) + ob(x));
          }
        };
        R cm, fm, km, nfm = R(0.0), ncm = R(0.0);
        R c0, f0, k0, nf0 = R(0.0), nc0 = R(0.0);
        R cp, fp, kp, nfp = R(0.0), ncp = R(0.0);
        plane(0, cm, fm, km, nfm, ncm);
        plane(1, c0, f0, k0, nf0, nc0);
        const R inv = R(1.0) / wsum;
#pragma unroll
        for (int k = 1; k <= GS; ++k) {
          plane(k + 1, cp, fp, kp, nfp, ncp);
          R out;
          if (kSolid && is_obstacle(c0)) {
            out = kObstacle<R>();
          } else {
            const R pc = c0;
            const R zm = (kSolid && is_obstacle(cm)) ? pc : cm, zp = (kSolid && is_obstacle(cp)) ? pc : cp;
            R s1 = (f0 + zm) + zp, s2 = (k0 + fm) + fp, s3 = km + kp;
            if constexpr (kSolid) {
              s1 = s1 + nf0 * pc;
              s2 = s2 + (nc0 + nfm + nfp) * pc;
              s3 = s3 + (ncm + ncp) * pc;
            }
            out = (pc + k8w<R>(1) * s1 + k8w<R>(2) * s2 + k8w<R>(3) * s3) * inv;
          }
          sps[(i - 1) + GS * ((j - 1) + GS * (k - 1))] = out;
          cm = c0; fm = f0; km = k0; nfm = nf0; ncm = nc0;
          c0 = cp; f0 = fp; k0 = kp; nf0 = nfp; nc0 = ncp;
        }
      }
      __syncthreads();
      if (threadIdx.x < GN * GN) {
        const int i = threadIdx.x % GN + 2, j = threadIdx.x / GN + 2;
        // per plane: gx = S_y D_x psi, gy = S_x D_y psi, s = S_x S_y psi over
        // the points that are not obstacles, and the same weights summed
        // over the obstacle points (gxo, gyo, so)
        auto plane = [&](int kk, R& ctr, R& gx, R& gy, R& sm, R& gxo, R& gyo, R& so) {
          const R* q = sps + (i - 1) + GS * ((j - 1) + GS * (kk - 1));
          const R a00 = q[-GS - 1], a01 = q[-GS], a02 = q[-GS + 1];
          const R a10 = q[-1], a11 = q[0], a12 = q[1];
          const R a20 = q[GS - 1], a21 = q[GS], a22 = q[GS + 1];
          ctr = a11;
          gx = (nz(a02) - nz(a00)) + R(2.0) * (nz(a12) - nz(a10)) + (nz(a22) - nz(a20));
          gy = (nz(a20) - nz(a00)) + R(2.0) * (nz(a21) - nz(a01)) + (nz(a22) - nz(a02));
          sm = (nz(a00) + R(2.0) * nz(a01) + nz(a02)) + R(2.0) * (nz(a10) + R(2.0) * nz(a11) + nz(a12)) +
               (nz(a20) + R(2.0) * nz(a21) + nz(a22));
          if constexpr (kSolid) {
            gxo = (ob(a02) - ob(a00)) + R(2.0) * (ob(a12) - ob(a10)) + (ob(a22) - ob(a20));
            gyo = (ob(a20) - ob(a00)) + R(2.0) * (ob(a21) - ob(a01)) + (ob(a22) - ob(a02));
            so = (ob(a00) + R(2.0) * ob(a01) + ob(a02)) + R(2.0) * (ob(a10) + R(2.0) * ob(a11) + ob(a12)) +
                 (ob(a20) + R(2.0) * ob(a21) + ob(a22));
          }
        };
        R t, xm, ym, sm, xom = R(0.0), yom = R(0.0), som = R(0.0);
        R c0, x0, y0, s0, xo0 = R(0.0), yo0 = R(0.0), so0 = R(0.0);
        R cp, xp, yp, sp, xop = R(0.0), yop = R(0.0), sop = R(0.0);
        plane(1, t, xm, ym, sm, xom, yom, som);
        plane(2, c0, x0, y0, s0, xo0, yo0, so0);
#pragma unroll
        for (int k = 2; k < 2 + GN; ++k) {
          plane(k + 1, cp, xp, yp, sp, xop, yop, sop);
          R n0 = R(0.0), n1 = R(0.0), n2 = R(0.0);
          if (!(kSolid && is_obstacle(c0))) {
            n0 = xm + R(2.0) * x0 + xp;
            n1 = ym + R(2.0) * y0 + yp;
            n2 = sp - sm;
            if constexpr (kSolid) {
              n0 = n0 + (xom + R(2.0) * xo0 + xop) * c0;
              n1 = n1 + (yom + R(2.0) * yo0 + yop) * c0;
              n2 = n2 + (sop - som) * c0;
            }
          }
          const R l2 = n0 * n0 + n1 * n1 + n2 * n2;
          const R il = l2 > R(0.0) ? rsqrtf(l2) : R(0.0);
          const int s3 = (i - 2) + GN * ((j - 2) + GN * (k - 2));
          snh[s3] = n0 * il;
          snh[GN * GN * GN + s3] = n1 * il;
          snh[2 * GN * GN * GN + s3] = n2 * il;
          xm = x0; ym = y0; sm = s0; xom = xo0; yom = yo0; som = so0;
          c0 = cp; x0 = xp; y0 = yp; s0 = sp; xo0 = xop; yo0 = yop; so0 = sop;
        }
      }
    };
    auto stencils = [&](auto SOLID) {
      constexpr bool kSolid = decltype(SOLID)::value;
      // smoothed fill level on the 12^3 sub-box: one thread per z-column,
      // the 3x3x3 window slides along z in registers
      if (threadIdx.x < GS * GS) {
        const int i = threadIdx.x % GS + 1, j = threadIdx.x / GS + 1;
        R w[3][9];  // planes k-1, k, k+1 of the window, (dy, dx) row-major
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int e = 0; e < 9; ++e)
            w[q + 1][e] = sphi[(i + e % 3 - 1) + GE * ((j + e / 3 - 1) + GE * q)];
#pragma unroll
        for (int k = 1; k <= GS; ++k) {
#pragma unroll
          for (int e = 0; e < 9; ++e) {
            w[0][e] = w[1][e];
            w[1][e] = w[2][e];
            w[2][e] = sphi[(i + e % 3 - 1) + GE * ((j + e / 3 - 1) + GE * (k + 1))];
          }
          const R pc = w[1][4];
          R out = kObstacle<R>();
          if (!kSolid || !is_obstacle(pc)) {
            R acc = R(0.0);
#pragma unroll
            for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
              for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                  const R raw = w[dz + 1][(dy + 1) * 3 + dx + 1];
                  const R v = (kSolid && is_obstacle(raw)) ? pc : raw;
                  acc = acc + k8w<R>(dx * dx + dy * dy + dz * dz) * v;
                }
            out = acc / wsum;
          }
          sps[(i - 1) + GS * ((j - 1) + GS * (k - 1))] = out;
        }
      }
      __syncthreads();
      // Parker-Youngs normal on the 10^3 sub-box, z-columns as above
      if (threadIdx.x < GN * GN) {
        const int i = threadIdx.x % GN + 2, j = threadIdx.x / GN + 2;
        auto psi = [&](int ii, int jj, int kk) { return sps[(ii - 1) + GS * ((jj - 1) + GS * (kk - 1))]; };
        R w[3][9];
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int e = 0; e < 9; ++e) w[q + 1][e] = psi(i + e % 3 - 1, j + e / 3 - 1, 1 + q);
#pragma unroll
        for (int k = 2; k < 2 + GN; ++k) {
#pragma unroll
          for (int e = 0; e < 9; ++e) {
            w[0][e] = w[1][e];
            w[1][e] = w[2][e];
            w[2][e] = psi(i + e % 3 - 1, j + e / 3 - 1, k + 1);
          }
          auto at = [&](int dx, int dy, int dz) { return w[dz + 1][(dy + 1) * 3 + dx + 1]; };
          const R pc = at(0, 0, 0);
          R out[3] = {R(0.0), R(0.0), R(0.0)};
          if (!kSolid || !is_obstacle(pc)) {
            R nn[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              R acc = R(0.0);
#pragma unroll
              for (int pp = -1; pp <= 1; ++pp)
#pragma unroll
                for (int r = -1; r <= 1; ++r) {
                  const int ax = (a == 0) ? 1 : r, ay = (a == 0) ? r : (a == 1) ? 1 : pp,
                            az = (a == 2) ? 1 : pp;
                  const int bx = (a == 0) ? -1 : ax, by = (a == 1) ? -1 : ay, bz = (a == 2) ? -1 : az;
                  const R rp = at(ax, ay, az), rm = at(bx, by, bz);
                  const R vp = (kSolid && is_obstacle(rp)) ? pc : rp;
                  const R vm = (kSolid && is_obstacle(rm)) ? pc : rm;
                  const R wt = (pp == 0 && r == 0) ? R(4.0) : (pp == 0 || r == 0) ? R(2.0) : R(1.0);
                  acc = acc + wt * (vp - vm);
                }
              nn[a] = acc;
            }
            const R len = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
#pragma unroll
            for (int a = 0; a < 3; ++a) out[a] = (len > R(0.0)) ? nn[a] / len : R(0.0);
          }
          const int s3 = (i - 2) + GN * ((j - 2) + GN * (k - 2));
          snh[s3] = out[0];
          snh[GN * GN * GN + s3] = out[1];
          snh[2 * GN * GN * GN + s3] = out[2];
        }
      }
    };
    if constexpr (sizeof(R) == 4) {
      if (solid) planes32(std::true_type{});
      else planes32(std::false_type{});
    } else {
      if (solid) stencils(std::true_type{});
      else stencils(std::false_type{});
    }
    __syncthreads();
    // curvature, gas density and Thuerey class of the tile's interface cells
    for (int s = threadIdx.x; s < GT * GT * GT; s += blockDim.x) {
      const int i = s % GT + 3, j = (s / GT) % GT + 3, k = s / (GT * GT) + 3;
      const int X = ox + i, Y = oy + j, Z = oz + k;
      if (X >= p.nx || Y >= p.ny || Z >= p.nz) continue;
      const int b = i + GE * (j + GE * k);
      if (styp[b] != T_IFACE) continue;
      const int c = cidx(p, X, Y, Z);
      auto nh = [&](int a, int ii, int jj, int kk) {
        return snh[a * GN * GN * GN + (ii - 2) + GN * ((jj - 2) + GN * (kk - 2))];
      };
      R acc = R(0.0);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int ex = (a == 0), ey = (a == 1), ez = (a == 2);
        const R vc = nh(a, i, j, k);
        const R vp = (styp[b + ex + GE * (ey + GE * ez)] >= T_OBST) ? vc : nh(a, i + ex, j + ey, k + ez);
        const R vm = (styp[b - ex - GE * (ey + GE * ez)] >= T_OBST) ? vc : nh(a, i - ex, j - ey, k - ez);
        acc = acc + (vp - vm);
      }
      const R kappa = R(-0.5) * acc;
      const int bb = d.bid[c];
      if constexpr (S::kDev) {
        // rho^G - 1 = 3 (p^V - 1/3) + 3 sigma kappa, formed in FP64
        const double pv = (p.bubble_model && bb >= 0) ? d.pV[bb] : p.pv0;
        rhog[c] = R(3.0 * (pv - 1.0 / 3.0) + 3.0 * p.sigma * (double)kappa);
      } else {
        const R pv = (p.bubble_model && bb >= 0) ? R(d.pV[bb]) : R(p.pv0);
        rhog[c] = R(3.0) * (pv + R(p.sigma) * kappa);
      }
      nhat[3LL * c + 0] = nh(0, i, j, k);
      nhat[3LL * c + 1] = nh(1, i, j, k);
      nhat[3LL * c + 2] = nh(2, i, j, k);
      bool hl = false, hg = false;
#pragma unroll
      for (int q = 1; q < Q; ++q) {
        const int t = styp[b + CX(q) + GE * (CY(q) + GE * CZ(q))];
        hl |= (t == T_LIQ);
        hg |= (t == T_GAS);
      }
      d.cls[c] = (!hl && hg) ? CL_NF : (hl && !hg) ? CL_NE : CL_STD;
    }
    if (threadIdx.x == 0) d.tile_mark[tile] = 0;
  }

// Resets the work-list counters that this step fills (next band list, new
// cells, next tile list).
__device__ __forceinline__ void reset_step_counts(const DPtrs& d, int parity) {
  d.counts[parity ^ 1] = 0;
  d.counts[2] = 0;
  d.counts[3 + (parity ^ 1)] = 0;
}

template <int Q, class S>
__global__ void __launch_bounds__(kGeoBlock, kGeoMinBlocks) k_geometry(DPtrs d, KParams p, int parity) {
  extern __shared__ __align__(16) unsigned char g_smem[];
  if (blockIdx.x == 0 && threadIdx.x == 0) reset_step_counts(d, parity);
  const int ntiles = d.counts[3 + parity];
  for (int tt = blockIdx.x; tt < ntiles; tt += gridDim.x)
    geometry_tile<Q, S>(d, p, d.tiles[parity][tt], g_smem);
}

// The bulk sweep with the geometry pass folded in (FP32 and 16-bit
// engines).  Every kGeoFuseEvery-th block of the persistent grid first
// takes geometry tiles, one at a time from a per-step counter (counts[7]:
// zero at init, cleared again by the finalize kernel of every step), until
// none is left, and then joins the other blocks on the bulk units.  The
// tiles so run at the sweep's occupancy (four blocks of 256 threads per SM
// instead of three of 192) with no launch boundary before the sweep.  On the
// 160x160x1024 Taylor bubble: separate kernels 77.5 + 295 us, every block
// first on tiles (1) 345 us, every second block (2) 364 us, every fourth
// 361 us: the sweep needs all its blocks to keep HBM busy, so blocks held
// by tiles slow it by about what running the tiles beside it saves.
#ifndef FSLBM_GEO_FUSE_EVERY
#define FSLBM_GEO_FUSE_EVERY 1
#endif
constexpr int kGeoFuseEvery = FSLBM_GEO_FUSE_EVERY;

template <int Q, class S, int COLL>
__global__ void __launch_bounds__(kBulkBlock, (bulk_min_blocks<S, COLL>()))
    k_bulk_geo(DPtrs d, KParams p, int parity) {
  extern __shared__ __align__(16) unsigned char g_smem[];
  __shared__ int s_tile;
  if (blockIdx.x == 0 && threadIdx.x == 0) reset_step_counts(d, parity);
  if (blockIdx.x % kGeoFuseEvery == 0) {
    const int ntiles = d.counts[3 + parity];
    for (;;) {
      __syncthreads();  // every thread has read the previous s_tile
      if (threadIdx.x == 0) s_tile = atomicAdd(&d.counts[7], 1);
      __syncthreads();
      const int tt = s_tile;
      if (tt >= ntiles) break;
      geometry_tile<Q, S, kBulkBlock>(d, p, d.tiles[parity][tt], g_smem);
    }
  }
  bulk_sweep<Q, S, COLL>(d, p, parity);
}

// ------------------------------------------------------- interface update
// Directions whose neighbour data the mass exchange reads ahead at once, and
// resident blocks of 128 threads per SM the FP32/FP16 interface kernels are
// compiled for (the kernel is latency-bound: three blocks cap it at 168
// registers a thread, which every variant fits without spilling; four
// blocks at 128 registers measured 10 % slower on the Taylor bubble (118 vs
// 107 us); the FP64 engine keeps two).  FSLBM_IFACE_MINB, when defined,
// sets the bound for the FP32 and 16-bit engines.
#ifndef FSLBM_IFACE_CHUNK
#define FSLBM_IFACE_CHUNK 6
#endif

constexpr int kIfaceChunk = FSLBM_IFACE_CHUNK;
// Half-width of the band of n^.c_i values that count as a tie n.c_i = 0
// (Appendix A assumes that only c_0 ties; at mirror planes of the interface
// a component of n^ is zero in exact arithmetic and rounding-sized in any
// precision, so the sign alone would decide by rounding).  Exact in FP32
// and FP64 alike.
constexpr double kTie = 0x1p-20;
template <class S, int COLL>
constexpr int iface_min_blocks() {
#ifdef FSLBM_IFACE_MINB
  return sizeof(typename S::Real) == 4 ? FSLBM_IFACE_MINB : 2;
#else
  return sizeof(typename S::Real) == 4 ? 3 : 2;
#endif
}
// Pull with the free-surface BC (Eq. nm-fslbm-boundary-condition) on the
// variant's set R (Sec. 3), mass exchange (Eq. nm-fslbm-mass-flux) with
// Thuerey's adjustment, fill update phi = m / rho, collision, marks.
template <int Q, class S, int COLL>
__device__ __forceinline__ void interface_cell(const DPtrs& d, const KParams& p, int parity, int k,
                                               bool& bad) {
  using R = typename S::Real;
  using T = typename S::T;
  const int* __restrict__ band = d.band[parity];
  const T* __restrict__ A = (const T*)d.pdf[parity];
  T* __restrict__ B = (T*)d.pdf[parity ^ 1];
  const long long Np = p.Np;
  const uint8_t* __restrict__ flags = d.flags;
  const R* nhat = (const R*)d.nhat;
  const R* rhog = (const R*)d.rhog;

    const int c = band[k];
    int x, y, z;
    decode(p, c, x, y, z);
    // neighbours x + c_i and their types (independent loads issued together);
    // the pull source of direction i is the neighbour in direction ibar.  A
    // cell beside a free-slip face links to the mirror image of a neighbour
    // across it, whose PDF arrives with the wall-normal component reversed.
    const bool slipface = coll_slip(COLL) && (flags[c] & F_FACE) && (p.slip[0] | p.slip[1] | p.slip[2]);
    int nid[Q];
    int nt[Q];
    nid[0] = c;
    nt[0] = T_IFACE;
    if (!slipface) {
#pragma unroll
      for (int i = 1; i < Q; ++i) nid[i] = nbr(p, x, y, z, CX(i), CY(i), CZ(i));
    } else {
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        int j;
        bool mir;
        nid[i] = pull_source<Q>(p, x, y, z, OPP(i), j, mir);
      }
    }
#pragma unroll
    for (int i = 1; i < Q; ++i) nt[i] = ntype(flags, nid[i]);
    R fx[Q], f[Q];
    unsigned miss = 0u;
#pragma unroll
    for (int i = 0; i < Q; ++i) fx[i] = load_own<Q, S>(A, Np, c, i);
    f[0] = fx[0];  // the rest PDF stays in the cell
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int st = nt[OPP(i)];
      const int src = nid[OPP(i)];
      if (st == T_GAS) miss |= 1u << i;
      const bool fluid = (st == T_LIQ || st == T_IFACE);
      int j = i;  // the PDF that arrives in direction i
      if (slipface) {
        bool mir;
        (void)pull_source<Q>(p, x, y, z, i, j, mir);
      }
      const T v = A[(long long)(fluid ? j : OPP(i)) * Np + (fluid ? src : c)];
      f[i] = load_w<S, Q>(v, i);
      if (st == T_GAS) f[i] = R(0.0);
    }
    // mass exchange with the streamed (not yet reconstructed) PDFs:
    // a = f*_ibar(x + c_i) equals the pulled f_ibar(x).  With deviations
    // (w_i = w_ibar cancels) a liquid link's difference enters exactly, as a
    // float pair, so a liquid neighbour's PDF sum changes by exactly -dm_i;
    // an interface link's term is the float product of the same operands
    // that the neighbour negates, so the two terms cancel exactly.
    const double phic = d.phi[c];
    const int clc = d.cls[c];
    double dm = 0.0;
    FAcc acc;
    const float phicf = d2f(phic);
    // class and fill level of the interface neighbours, read a chunk of
    // directions at a time ahead of the (ordered) accumulation
    constexpr int kChunk = kIfaceChunk;
#pragma unroll
    for (int i0 = 1; i0 < Q; i0 += kChunk) {
      int cl9[kChunk];
      double ph9[kChunk];
#pragma unroll
      for (int a = 0; a < kChunk; ++a) {
        const int i = i0 + a;
        if (i < Q && nt[i] == T_IFACE) {
          cl9[a] = d.cls[nid[i]];
          ph9[a] = d.phi[nid[i]];
        }
      }
#pragma unroll
      for (int a = 0; a < kChunk; ++a) {
        const int i = i0 + a;
        if (i >= Q) continue;
        const int ntp = nt[i];
        if (ntp == T_GAS || ntp == T_OBST) continue;
        const R fa = f[OPP(i)];
        const R fb = fx[i];
        if constexpr (S::kDev) {
          const float w = W<Q, float>(i);
          if (ntp == T_LIQ) {
            acc.add_diff(fa, fb);
          } else {
            const int cln = cl9[a];
            float v;
            if (clc == cln) v = __fsub_rn(fa, fb);
            else if (clc == CL_STD) v = (cln == CL_NF) ? __fadd_rn(fa, w) : -__fadd_rn(fb, w);
            else if (clc == CL_NF) v = -__fadd_rn(fb, w);
            else v = __fadd_rn(fa, w);
            acc.add(__fmul_rn(__fmul_rn(0.5f, __fadd_rn(phicf, d2f(ph9[a]))), v));
          }
        } else {
          if (ntp == T_LIQ) {
            dm = dm + (double)(fa - fb);
          } else {
            const int cln = cl9[a];
            R v;
            if (clc == cln) v = fa - fb;
            else if (clc == CL_STD) v = (cln == CL_NF) ? fa : -fb;
            else if (clc == CL_NF) v = -fb;
            else v = fa;
            dm = dm + 0.5 * (phic + ph9[a]) * (double)v;
          }
        }
      }
    }
    if constexpr (S::kDev) dm = acc.value();
    const double mn = d.mass[c] + dm;
    // BC velocity from the cell's own post-collision PDFs
    R rc, jx, jy, jz;
    sums<Q, R>(fx, rc, jx, jy, jz);
    if constexpr (S::kDev) rc = R(1.0) + rc;
    const R ux = jx / rc - R(0.5) * gpar<R>(p, 0);
    const R uy = jy / rc - R(0.5) * gpar<R>(p, 1);
    const R uz = jz / rc - R(0.5) * gpar<R>(p, 2);
    // set R of the variant (Sec. 3) and reconstruction; |n^.c_i| <= kTie
    // counts as a tie (n.c_i = 0): NBRC reconstructs ties, NBKC does not
    const R n0 = nhat[3LL * c], n1 = nhat[3LL * c + 1], n2 = nhat[3LL * c + 2];
    int v = p.variant;
    if (v == 4) v = (__popc(miss) >= 3) ? 3 : p.om3_fb;
    const R rg = rhog[c];  // rho^G (FP64 engine) or rho^G - 1
    const R tie = R(kTie);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      bool rec = (miss >> i) & 1u;
      const R dot = R(CX(i)) * n0 + R(CY(i)) * n1 + R(CZ(i)) * n2;
      if (v == 1 && dot >= -tie) rec = true;
      if (v == 2 && dot > tie) rec = true;
      if (rec) {
        const int j = OPP(i);
        if constexpr (S::kDev) {
          const R rgf = R(1.0) + rg;
          f[i] = (feq_dev<Q, R>(i, rg, rgf, ux, uy, uz) + feq_dev<Q, R>(j, rg, rgf, ux, uy, uz)) - fx[j];
        } else {
          f[i] = (feq_i<Q, R>(i, rg, ux, uy, uz) + feq_i<Q, R>(j, rg, ux, uy, uz)) - fx[j];
        }
      }
    }
    long long s_in = 0;  // the mass-conserving formats: the received values in grid steps
    if constexpr (S::kExactRest) {
#pragma unroll
      for (int i = 0; i < Q; ++i) s_in += grid_steps<S>(f[i]);
    }
    double rho = collide_any<Q, S, COLL>(f, p, bad);
    // moments of the stored post-collision PDFs, in post_moments' arithmetic
    // (new interface cells average them over their neighbours)
    R mu[3];
    if constexpr (S::kDev) {
      // the density as the stored PDFs hold it (FP64 sum of the stored
      // values): the mass a conversion to liquid hands over to them
      double sd = 0.0;
      R fs[Q];
      if constexpr (S::kExactRest) {
        store_cell<Q, S>(B, Np, c, f, s_in, bad);
        const int r0 = rest_slice<Q, S>(B, Np)[c];
        long long n = r0;
        fs[0] = from_steps<S>(r0);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          const T v = S::stored(f[i]);
          fs[i] = S::loadd(v);
          n += S::steps(v);
        }
        sd = (double)n * (1.0 / (double)(1LL << S::kShift));
      } else {
        FAcc sa;  // the float sum carried as a pair: FP64 accuracy, FP32 operations
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const T v = S::stored(f[i]);
          B[(long long)i * Np + c] = v;
          fs[i] = S::loadd(v);
          sa.add(fs[i]);
        }
        sd = sa.value();
      }
      rho = 1.0 + sd;
      R r0, jx0, jy0, jz0;
      sums<Q, R>(fs, r0, jx0, jy0, jz0);
      const R rr = R(rho);
      mu[0] = jx0 / rr - R(0.5) * gpar<R>(p, 0);
      mu[1] = jy0 / rr - R(0.5) * gpar<R>(p, 1);
      mu[2] = jz0 / rr - R(0.5) * gpar<R>(p, 2);
      d.mom_rho[c] = rho;
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) B[(long long)i * Np + c] = store_w<S, Q>(f[i], i);
      R r0, jx0, jy0, jz0;
      sums<Q, R>(f, r0, jx0, jy0, jz0);
      mu[0] = jx0 / r0 - R(0.5) * gpar<R>(p, 0);
      mu[1] = jy0 / r0 - R(0.5) * gpar<R>(p, 1);
      mu[2] = jz0 / r0 - R(0.5) * gpar<R>(p, 2);
      d.mom_rho[c] = (double)r0;
    }
    {
      R* mu_out = (R*)d.mom_u;
      mu_out[3LL * c + 0] = mu[0];
      mu_out[3LL * c + 1] = mu[1];
      mu_out[3LL * c + 2] = mu[2];
    }
    {
      const uint8_t fl = flags[c];
      if (fl & F_NEAR_WALL) write_reflected<Q, S>(d, p, B, c, d.wallmask[c], (fl & F_WRAP) != 0, f);
    }
    double phin;
    if constexpr (S::kDev) {
      // mn / rho from the float reciprocal and one Newton step in FP64
      // (relative error about 2^-46; an FP64 division takes tens of FP64
      // operations)
      const double r0 = (double)__frcp_rn(d2f(rho));
      const double q0 = mn * r0;
      phin = fma(fma(-q0, rho, mn), r0, q0);
    } else {
      phin = mn / rho;
    }
    d.m_next[k] = mn;
    d.phi_next[k] = phin;
    d.rho_band[k] = rho;
    d.mark[c] = (phin > 1.0 + p.eps) ? CV_TOL : (phin < -p.eps) ? CV_TOG : CV_NONE;
  }

template <int Q, class S, int COLL>
__global__ void __launch_bounds__(128, (iface_min_blocks<S, COLL>())) k_interface(DPtrs d, KParams p, int parity) {
  const int n = d.counts[parity];
  bool bad = false;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    interface_cell<Q, S, COLL>(d, p, parity, k, bad);
  if (bad) d.err[0] = 1;
}

// -------------------------------------------------------------- conversion
// These passes are chains of dependent neighbour reads over a few hundred
// converting cells, so their duration is the number of round trips to
// memory along the longest chain.  Each pass reads the neighbours' values
// one level at a time for all directions together (types, then the values
// the types select, then the values those select) and writes only after
// the last read; the arithmetic and its order are those of a per-direction
// loop.

// Neighbour indices of (x, y, z) and their types (T_OBST outside the domain).
template <int Q>
__device__ __forceinline__ void neighbour_types(const DPtrs& d, const KParams& p, int x, int y,
                                                int z, int* nid, uint8_t* nt) {
#pragma unroll
  for (int i = 1; i < Q; ++i) nid[i] = nbr(p, x, y, z, CX(i), CY(i), CZ(i));
#pragma unroll
  for (int i = 1; i < Q; ++i) nt[i] = nid[i] >= 0 ? (uint8_t)(d.flags[nid[i]] & F_TYPE) : (uint8_t)T_OBST;
}

// Commit m, phi; conflict rule (a cell marked for gas stays interface next
// to a cell marked for liquid); claim gas neighbours of cells turning liquid
// and liquid neighbours of cells turning gas as new interface cells.
template <int Q>
__device__ __forceinline__ void resolve_cell(const DPtrs& d, const KParams& p, int parity, int k) {
  const int c = d.band[parity][k];
  uint8_t cv = d.mark[c];
  d.mass[c] = d.m_next[k];
  d.phi[c] = d.phi_next[k];
  if (cv == CV_NONE) {
    d.conv[c] = CV_NONE;
    return;
  }
  int x, y, z;
  decode(p, c, x, y, z);
  int nid[Q];
  uint8_t nt[Q];
  neighbour_types<Q>(d, p, x, y, z, nid, nt);
  if (cv == CV_TOG) {
    uint8_t mk[Q];
#pragma unroll
    for (int i = 1; i < Q; ++i) mk[i] = nt[i] == T_IFACE ? d.mark[nid[i]] : (uint8_t)CV_NONE;
#pragma unroll
    for (int i = 1; i < Q; ++i)
      if (mk[i] == CV_TOL) cv = CV_NONE;
  }
  d.conv[c] = cv;
  if (cv == CV_NONE) return;
  const int want = (cv == CV_TOL) ? T_GAS : T_LIQ;
  // claim first (the atomics are independent of one another), then reserve
  // all of this cell's new entries with one atomic (the list's order enters
  // no result)
  unsigned fresh = 0u;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    if (nt[i] != want) continue;
    const int nb = nid[i];
    unsigned* word = (unsigned*)(d.claim + (nb & ~3));
    const unsigned bit = 1u << (8 * (nb & 3));
    const unsigned old = atomicOr(word, bit);
    if (!(old & bit)) fresh |= 1u << i;
  }
  if (!fresh) return;
  int pos = atomicAdd(&d.counts[2], __popc(fresh));
#pragma unroll
  for (int i = 1; i < Q; ++i)
    if ((fresh >> i) & 1u) d.newlist[pos++] = nid[i];
}

template <int Q>
__global__ void __launch_bounds__(kBlock) k_resolve(DPtrs d, KParams p, int parity) {
  const int n = d.counts[parity];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    resolve_cell<Q>(d, p, parity, k);
}

// Excess-mass receivers (Eq. nm-fslbm-excess-mass): interface cells after
// conversion in the lattice neighbourhood (interface cells that do not
// convert, and the gas or liquid cells that conversion claims); none -> the
// conversion is deferred.
template <int Q>
__device__ __forceinline__ void count_cell(const DPtrs& d, const KParams& p, int parity, int k) {
  const int c = d.band[parity][k];
  const uint8_t cv = d.conv[c];
  if (cv == CV_NONE) {
    d.cfin[c] = CV_NONE;
    return;
  }
  const double m = d.mass[c];
  const double rb = d.rho_band[k];
  int x, y, z;
  decode(p, c, x, y, z);
  int nid[Q];
  uint8_t nt[Q];
  neighbour_types<Q>(d, p, x, y, z, nid, nt);
  uint8_t nv[Q];  // conv of interface neighbours, claim of gas and liquid ones
#pragma unroll
  for (int i = 1; i < Q; ++i)
    nv[i] = nt[i] == T_IFACE ? d.conv[nid[i]] : nt[i] != T_OBST ? d.claim[nid[i]] : (uint8_t)0;
  int nrecv = 0;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const bool post = nt[i] == T_IFACE ? nv[i] == CV_NONE : nt[i] != T_OBST && nv[i] != 0;
    nrecv += post ? 1 : 0;
  }
  if (nrecv == 0) {
    d.cfin[c] = CV_DEFER;
    return;
  }
  const double mex = (cv == CV_TOL) ? (m - rb) : m;
  d.share[c] = mex / (double)nrecv;
  d.cfin[c] = cv;
  // flag the interface neighbours, which gather this cell's share: the
  // others skip the gather (it would add nothing)
#pragma unroll
  for (int i = 1; i < Q; ++i)
    if (nt[i] == T_IFACE) d.rcv[nid[i]] = 1;
}

template <int Q>
__global__ void __launch_bounds__(kBlock) k_count(DPtrs d, KParams p, int parity) {
  const int n = d.counts[parity];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    count_cell<Q>(d, p, parity, k);
}

__device__ __forceinline__ bool is_converted(uint8_t f) { return f == CV_TOL || f == CV_TOG; }

// 2-bit fields per direction (types T_*, conversion states CV_*)
__device__ __forceinline__ int field2(uint64_t m, int i) { return (int)((m >> (2 * i)) & 3u); }

// Sum of the excess shares of converted neighbours, in direction order.
// cfm: 2-bit cfin of the interface neighbours (CV_NONE elsewhere).
template <int Q>
__device__ __forceinline__ double gather_shares(const DPtrs& d, const int* nid, uint64_t cfm) {
  double sh[Q];
#pragma unroll
  for (int i = 1; i < Q; ++i) sh[i] = is_converted((uint8_t)field2(cfm, i)) ? d.share[nid[i]] : 0.0;
  double s = 0.0;
#pragma unroll
  for (int i = 1; i < Q; ++i)
    if (is_converted((uint8_t)field2(cfm, i))) s = s + sh[i];
  return s;
}

// Excess gather for all interface cells after conversion; PDFs of new
// interface cells from gas: f* = f^eq(mean rho, mean u) over liquid and old
// interface neighbours; new interface cells from liquid: m = rho, phi = 1.
template <int Q, class S>
__device__ __forceinline__ void apply_cell(const DPtrs& d, const KParams& p, int parity, int k) {
  using R = typename S::Real;
  using T = typename S::T;
  // the new cells come first: their dependent chains are the longest, so
  // they start with the launch
  const int nnew = d.counts[2];
  T* __restrict__ B = (T*)d.pdf[parity ^ 1];
  const long long Np = p.Np;

  const bool is_band = k >= nnew;
  if (is_band) k -= nnew;
  const int c = is_band ? d.band[parity][k] : d.newlist[k];
  int x, y, z;
  int nid[Q];
  if (is_band) {
    const bool gather = d.rcv[c] != 0;
    const uint8_t f = d.cfin[c];
    if (gather) d.rcv[c] = 0;
    if (f == CV_TOL) {
      d.phi[c] = 1.0;
      d.mass[c] = d.rho_band[k];
      return;
    }
    if (f == CV_TOG) {
      d.phi[c] = 0.0;
      d.mass[c] = 0.0;
      return;
    }
    // a deferred cell stays interface and keeps its mass: it was not counted
    // among its converting neighbours' receivers
    if (f == CV_DEFER) return;
    const double m0 = d.mass[c];
    // an interface cell that no converted cell flagged receives nothing:
    // m + 0 and (m + 0) / rho are the m and phi that k_resolve stored
    // (m_next and phi_next = m_next / rho), unless m is -0
    if (!gather && !(m0 == 0.0 && signbit(m0))) return;
    const double rb = d.rho_band[k];
    double s = 0.0;
    if (gather) {
      decode(p, c, x, y, z);
#pragma unroll
      for (int i = 1; i < Q; ++i) nid[i] = nbr(p, x, y, z, CX(i), CY(i), CZ(i));
      unsigned ifm = 0u;  // interface neighbours
#pragma unroll
      for (int i = 1; i < Q; ++i)
        if (nid[i] >= 0 && (d.flags[nid[i]] & F_TYPE) == T_IFACE) ifm |= 1u << i;
      uint64_t cfm = 0;
#pragma unroll
      for (int i = 1; i < Q; ++i)
        if ((ifm >> i) & 1u) cfm |= (uint64_t)(d.cfin[nid[i]] & 3u) << (2 * i);
      s = gather_shares<Q>(d, nid, cfm);
    }
    const double m = m0 + s;
    d.mass[c] = m;
    d.phi[c] = m / rb;
    return;
  }

  // a new interface cell (gas or liquid before this step)
  const uint8_t fl = d.flags[c];
  const int t = fl & F_TYPE;
  decode(p, c, x, y, z);
#pragma unroll
  for (int i = 1; i < Q; ++i) nid[i] = nbr(p, x, y, z, CX(i), CY(i), CZ(i));
  uint64_t ntm = 0;
#pragma unroll
  for (int i = 1; i < Q; ++i)
    ntm |= (uint64_t)(nid[i] >= 0 ? (d.flags[nid[i]] & F_TYPE) : T_OBST) << (2 * i);
  uint64_t cfm = 0;   // cfin of interface neighbours
  uint32_t clm = 0u;  // claimed gas or liquid neighbours
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int nt = field2(ntm, i);
    if (nt == T_IFACE) cfm |= (uint64_t)(d.cfin[nid[i]] & 3u) << (2 * i);
    if ((nt == T_GAS || nt == T_LIQ) && d.claim[nid[i]] != 0) clm |= 1u << i;
  }
  const double s = gather_shares<Q>(d, nid, cfm);
  if (t == T_GAS) {
    // neighbours that stay or turn liquid, or stay interface
    unsigned use = 0u;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int nt = field2(ntm, i);
      if (nt == T_IFACE && field2(cfm, i) != CV_TOG) use |= 1u << i;
      if (nt == T_LIQ && !((clm >> i) & 1u)) use |= 1u << i;
    }
    double sr = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    int cnt = 0;
    unsigned liq_use = 0u;
#pragma unroll
    for (int i = 1; i < Q; ++i)
      if (((use >> i) & 1u) && field2(ntm, i) == T_LIQ) liq_use |= 1u << i;
    if (liq_use) {
      // liquid neighbours (none next to a gas cell while the interface layer
      // is closed) form their moments from the stored PDFs: direction order
      for (int i = 1; i < Q; ++i) {
        if (!((use >> i) & 1u)) continue;
        double rn;
        R un[3];
        if (field2(ntm, i) == T_IFACE) {
          const R* mu = (const R*)d.mom_u;
          rn = d.mom_rho[nid[i]];
          un[0] = mu[3LL * nid[i] + 0];
          un[1] = mu[3LL * nid[i] + 1];
          un[2] = mu[3LL * nid[i] + 2];
        } else {
          post_moments<Q, S>(B, Np, nid[i], p, rn, un);
        }
        sr = sr + rn;
        sx = sx + (double)un[0];
        sy = sy + (double)un[1];
        sz = sz + (double)un[2];
        ++cnt;
      }
    }
    // moments cached by the interface kernel, read a few directions at a time
    constexpr int kChunk = 5;
#pragma unroll
    for (int i0 = 1; liq_use == 0u && i0 < Q; i0 += kChunk) {
      double rn[kChunk];
      R un[kChunk][3];
#pragma unroll
      for (int a = 0; a < kChunk; ++a) {
        const int i = i0 + a;
        if (i < Q && ((use >> i) & 1u) && field2(ntm, i) == T_IFACE) {
          const R* mu = (const R*)d.mom_u;
          rn[a] = d.mom_rho[nid[i]];
          un[a][0] = mu[3LL * nid[i] + 0];
          un[a][1] = mu[3LL * nid[i] + 1];
          un[a][2] = mu[3LL * nid[i] + 2];
        }
      }
#pragma unroll
      for (int a = 0; a < kChunk; ++a) {
        const int i = i0 + a;
        if (i >= Q || !((use >> i) & 1u)) continue;
        sr = sr + rn[a];
        sx = sx + (double)un[a][0];
        sy = sy + (double)un[a][1];
        sz = sz + (double)un[a][2];
        ++cnt;
      }
    }
    double rb = 1.0, ub0 = 0.0, ub1 = 0.0, ub2 = 0.0;
    if (cnt > 0) {
      rb = sr / (double)cnt;
      ub0 = sx / (double)cnt;
      ub1 = sy / (double)cnt;
      ub2 = sz / (double)cnt;
    }
    const uint32_t wm = (fl & F_NEAR_WALL) ? d.wallmask[c] : 0u;
    R fn[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if constexpr (S::kDev)
        fn[i] = feq_dev<Q, R>(i, R(rb - 1.0), R(rb), R(ub0), R(ub1), R(ub2));
      else
        fn[i] = feq_i<Q, R>(i, R(rb), R(ub0), R(ub1), R(ub2));
    }
    bool over = false;
    const long long s_new = S::kExactRest ? __double2ll_rn((rb - 1.0) * (double)(1LL << grid_shift<S>())) : 0;
    store_cell<Q, S>(B, Np, c, fn, s_new, over);
    if (over) d.err[0] = 1;
    if (fl & F_NEAR_WALL) write_reflected<Q, S>(d, p, B, c, wm, (fl & F_WRAP) != 0, fn);
    const double m = 0.0 + s;
    d.mass[c] = m;
    d.phi[c] = m / rb;
  } else {  // from liquid
    int bb[Q];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int nt = field2(ntm, i);
      const bool gas_after = (nt == T_GAS && !((clm >> i) & 1u)) || (nt == T_IFACE && field2(cfm, i) == CV_TOG);
      bb[i] = gas_after ? d.bid[nid[i]] : -1;
    }
    double rn;
    R un[3];
    post_moments<Q, S>(B, Np, c, p, rn, un);
    int best = -1;
#pragma unroll
    for (int i = 1; i < Q; ++i)
      if (bb[i] >= 0 && (best < 0 || bb[i] < best)) best = bb[i];
    const double m = rn + s;
    d.mass[c] = m;
    d.phi[c] = m / rn;
    d.bid[c] = best;
  }
}

template <int Q, class S>
__global__ void __launch_bounds__(128) k_apply(DPtrs d, KParams p, int parity) {
  // the new interface cells (long dependent chains) are dealt round-robin
  // over the blocks, cell j to thread j / G of block j mod G, so that they
  // spread over all SMs instead of filling the first blocks; the band cells
  // follow in order
  const int nnew = d.counts[2];
  const int total = gridDim.x * blockDim.x;
  for (int j = threadIdx.x * gridDim.x + blockIdx.x; j < nnew; j += total) apply_cell<Q, S>(d, p, parity, j);
  const int nband = d.counts[parity];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nband; k += total)
    apply_cell<Q, S>(d, p, parity, nnew + k);
}

// Fixed-point bubble-volume term round((1 - phi) 2^32).
__device__ __forceinline__ long long vol_fix(double one_minus_phi) {
  return __double2ll_rn(one_minus_phi * 4294967296.0);
}

// Adds the geometry tile of cell c (c < 0: none) to a tile list once; every
// lane of the warp must call it.
__device__ __forceinline__ void mark_tile(const DPtrs& d, const KParams& p, int c, int* list,
                                          int* count) {
  int tile = -1;
  if (c >= 0) {
    int x, y, z;
    decode(p, c, x, y, z);
    const int ntx = (p.nx + 7) / 8, nty = (p.ny + 7) / 8;
    tile = (x >> 3) + ntx * ((y >> 3) + nty * (z >> 3));
  }
  const unsigned peers = __match_any_sync(0xffffffffu, tile);
  const bool lead = tile >= 0 && (int)(threadIdx.x & 31u) == __ffs(peers) - 1;
  const bool fresh = lead && atomicExch(&d.tile_mark[tile], 1) == 0;
  const int pos = warp_append(count, fresh);
  if (fresh) list[pos] = tile;
}

// Adds the kSegCells-cell group of cell c (c < 0: none) to the liquid group
// list once; every lane of the warp must call it.
__device__ __forceinline__ void mark_seg(const DPtrs& d, int c) {
  const int seg = c >= 0 ? (c / kSegCells) : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, seg);
  const bool lead = seg >= 0 && (int)(threadIdx.x & 31u) == __ffs(peers) - 1;
  const bool fresh = lead && atomicExch(&d.seg_mark[seg], 1) == 0;
  const int pos = warp_append(&d.counts[5], fresh);
  if (fresh) d.segs[pos] = seg;
}

// Initial liquid group list (blocks of 256 cover whole groups).
static __global__ void k_segs_init(DPtrs d, KParams p) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool liq = c < p.N && (d.flags[c] & F_TYPE) == T_LIQ;
  const unsigned b = __ballot_sync(0xffffffffu, liq);
  const unsigned gmask = kSegCells == 32 ? 0xffffffffu : ((1u << kSegCells) - 1u);
  const bool fresh = (lane % kSegCells) == 0 && ((b >> lane) & gmask) != 0;
  if (fresh) d.seg_mark[c / kSegCells] = 1;
  const int pos = warp_append(&d.counts[5], fresh);
  if (fresh) d.segs[pos] = c / kSegCells;
}

// Tile list of an interface list (initial state and checkpoint load).
static __global__ void k_tiles_of_band(DPtrs d, KParams p, int parity) {
  const int n = d.counts[parity];
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int base = wid * 32; base < n; base += warps * 32) {
    const int k = base + (threadIdx.x & 31);
    mark_tile(d, p, k < n ? d.band[parity][k] : -1, d.tiles[parity], &d.counts[3 + parity]);
  }
}

// Final flags, next interface list, bubble gas counts and interface sums.
// Entries [base, base + 32) of the band + new-cell list (every lane of the
// warp calls it).  kAppend: append the cells that stay or become interface
// to the next interface list (the batched step); a single domain rebuilds
// that list in cell order with k_compact_band instead.
template <bool kAppend = true>
__device__ __forceinline__ void finalize_warp(const DPtrs& d, const KParams& p, int parity,
                                              int base) {
  const int* __restrict__ band = d.band[parity];
  int* __restrict__ next = d.band[parity ^ 1];
  const int nb_ = d.counts[parity];
  const int total = nb_ + d.counts[2];
  const int lane = threadIdx.x & 31;

    const int k = base + lane;
    bool keep = false, to_liq = false;
    int c = -1, bub = -1, dgas = 0;
    long long vfix = 0;
    if (k < total) {
      const bool is_band = k < nb_;
      c = is_band ? band[k] : d.newlist[k - nb_];
      const uint8_t fl = d.flags[c];
      const int b = d.bid[c];
      if (is_band) {
        const uint8_t f = d.cfin[c];
        if (f == CV_TOL) {
          d.flags[c] = (fl & ~F_TYPE) | T_LIQ;
          d.bid[c] = -1;
          to_liq = true;
        } else if (f == CV_TOG) {
          d.flags[c] = (fl & ~F_TYPE) | T_GAS;
          dgas = 1;
        } else {
          keep = true;
        }
      } else {
        if ((fl & F_TYPE) == T_GAS) dgas = -1;
        d.flags[c] = (fl & ~F_TYPE) | T_IFACE;
        d.claim[c] = 0;
        keep = true;
      }
      if (p.bubble_model && b >= 0) {
        bub = b;
        if (keep) vfix = vol_fix(1.0 - d.phi[c]);
      }
    }
    if (p.bubble_model) {
      // integer sums per bubble id present in the warp, one atomic each
      // (integer addition: the result does not depend on the order)
      unsigned remaining = 0xffffffffu;
      while (remaining) {
        const int leader = __ffs(remaining) - 1;
        const int bb = __shfl_sync(0xffffffffu, bub, leader);
        const bool mine = (bub == bb);
        long long sv = mine ? vfix : 0, sg = mine ? (long long)dgas : 0;
        for (int o = 16; o > 0; o >>= 1) {
          sv += __shfl_xor_sync(0xffffffffu, sv, o);
          sg += __shfl_xor_sync(0xffffffffu, sg, o);
        }
        if (lane == leader && bb >= 0) {
          if (sv) atomicAdd((unsigned long long*)&d.iface_fix[bb], (unsigned long long)sv);
          if (sg) atomicAdd((unsigned long long*)&d.gas_cnt[bb], (unsigned long long)sg);
        }
        remaining &= ~__ballot_sync(0xffffffffu, mine);
      }
    }
    if constexpr (kAppend) {
      const int pos = warp_append(&d.counts[parity ^ 1], keep);
      if (keep) next[pos] = c;
    } else {
      (void)next;
    }
    mark_tile(d, p, keep ? c : -1, d.tiles[parity ^ 1], &d.counts[3 + (parity ^ 1)]);
    mark_seg(d, to_liq ? c : -1);
  }

static __global__ void __launch_bounds__(kBlock) k_finalize(DPtrs d, KParams p, int parity) {
  const int total = d.counts[parity] + d.counts[2];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    d.counts[6] = 0;  // the next step's bulk hand-out
    d.counts[7] = 0;  // and geometry-tile hand-out
  }
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int base = wid * 32; base < total; base += warps * 32) finalize_warp<false>(d, p, parity, base);
}

// p^V_b = p^V_b(0) V_b(0) / V_b (Eq. nm-fslbm-pressure-volume).
__device__ __forceinline__ void bubble_update(const DPtrs& d, const KParams& p) {
  for (int b = threadIdx.x; b < d.nb; b += blockDim.x) {
    const long long acc = d.gas_cnt[b] * 4294967296LL + d.iface_fix[b];
    const double V = __ll2double_rn(acc) / 4294967296.0;
    d.pV[b] = (V > 0.0) ? (p.pv0 * d.V0[b]) / V : p.pv0;
    d.Vcur[b] = V;
    d.iface_fix[b] = 0;
  }
}

static __global__ void k_bubble(DPtrs d, KParams p) { bubble_update(d, p); }

// ------------------------------------------------------------ observables
// Per-block partials: [0] mass, [1] max|u|, [2] liquid volume, [3] nan,
// [4..7] counts of gas, interface, liquid, obstacle.
constexpr int kObsFields = 8;

template <int Q, class S>
__global__ void __launch_bounds__(kBlock) k_obs_partial(DPtrs d, KParams p, int parity,
                                                        double* part) {
  using R = typename S::Real;
  const typename S::T* P = (const typename S::T*)d.pdf[parity];
  // the mass is summed per thread with Neumaier's compensation, then
  // pairwise across threads and blocks
  double mass = 0.0, mcomp = 0.0, umax = 0.0, vol = 0.0, nan = 0.0, cnt[4] = {0, 0, 0, 0};
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < p.N; c += gridDim.x * blockDim.x) {
    const int t = d.flags[c] & F_TYPE;
    cnt[t] += 1.0;
    if (t == T_LIQ || t == T_IFACE) {
      double r;
      R u[3];
      post_moments<Q, S>(P, p.Np, c, p, r, u);
      const double uu = sqrt((double)u[0] * u[0] + (double)u[1] * u[1] + (double)u[2] * u[2]);
      if (!(uu == uu) || !(r > 0.0)) nan = 1.0;
      if (uu > umax) umax = uu;
      {
        const double x = (t == T_LIQ) ? r : d.mass[c];
        const double s = mass + x;
        mcomp += (fabs(mass) >= fabs(x)) ? ((mass - s) + x) : ((x - s) + mass);
        mass = s;
      }
      vol += d.phi[c];
      if (!(d.mass[c] == d.mass[c])) nan = 1.0;
    }
  }
  __shared__ double sh[kObsFields][kBlock / 32];
  double v[kObsFields] = {mass + mcomp, umax, vol, nan, cnt[0], cnt[1], cnt[2], cnt[3]};
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int f = 0; f < kObsFields; ++f) {
    double a = v[f];
    for (int o = 16; o > 0; o >>= 1) {
      const double b = __shfl_down_sync(0xffffffffu, a, o);
      a = (f == 1 || f == 3) ? fmax(a, b) : a + b;
    }
    if (lane == 0) sh[f][w] = a;
  }
  __syncthreads();
  if (threadIdx.x < kObsFields) {
    const int f = threadIdx.x;
    double a = sh[f][0];
    for (int i = 1; i < kBlock / 32; ++i) a = (f == 1 || f == 3) ? fmax(a, sh[f][i]) : a + sh[f][i];
    part[blockIdx.x * kObsFields + f] = a;
  }
}

static __global__ void k_obs_final(const double* part, int nblocks, double* out) {
  const int f = threadIdx.x;
  if (f >= kObsFields) return;
  double a = part[f];
  for (int b = 1; b < nblocks; ++b) {
    const double v = part[b * kObsFields + f];
    a = (f == 1 || f == 3) ? fmax(a, v) : a + v;
  }
  out[f] = a;
}

// PDFs of the current buffer as FP64 (zero on gas and obstacle cells), in
// the caller's cell order: thread e writes the cell with caller index e.
template <int Q, class S>
__global__ void k_pdf_out(DPtrs d, KParams p, int parity, double* out) {
  using R = typename S::Real;
  const typename S::T* P = (const typename S::T*)d.pdf[parity];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p.N) return;
  const int c = storage_of_ext(p, e);
  const int t = d.flags[c] & F_TYPE;
  const bool fluid = (t == T_LIQ || t == T_IFACE);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    double v;
    if constexpr (S::kExactRest) {
      if (i == 0) {
        out[(long long)i * p.N + e] =
            fluid ? (double)rest_slice<Q, S>(P, p.Np)[c] * (1.0 / (double)(1LL << S::kShift)) + W<Q, double>(0)
                  : 0.0;
        continue;
      }
    }
    if constexpr (S::kDev)
      v = (double)S::loadd(P[(long long)i * p.Np + c]) + W<Q, double>(i);
    else
      v = (double)S::load(P[(long long)i * p.Np + c], W<Q, R>(i));
    out[(long long)i * p.N + e] = fluid ? v : 0.0;
  }
}

// ------------------------------------------------------------ storage order
// Liquid-holding kSegCells-cell groups of the storage order p over flags
// given in the caller's order (one warp = one 32-cell group): the work list
// length of the bulk sweep if the cells were stored that way.
static __global__ void k_layout_census(const uint8_t* __restrict__ raw_ext, KParams p,
                                       unsigned long long* groups) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const bool liq = c < p.N && raw_ext[ext_index(p, c)] == T_LIQ;
  const unsigned b = __ballot_sync(0xffffffffu, liq);
  if ((threadIdx.x & 31) == 0 && b) {
    int n = 0;
    for (int g = 0; g < 32; g += kSegCells) n += ((b >> g) & (kSegCells == 32 ? 0xffffffffu : ((1u << kSegCells) - 1u))) != 0u;
    atomicAdd(groups, (unsigned long long)n);
  }
}

// Arrays between the caller's cell order and the storage order: ncomp
// consecutive arrays of N entries each.
template <class T>
__global__ void k_to_storage(const T* __restrict__ ext, T* __restrict__ st, KParams p, int ncomp) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.N) return;
  const int e = ext_index(p, c);
  for (int k = 0; k < ncomp; ++k) st[(long long)k * p.N + c] = ext[(long long)k * p.N + e];
}
template <class T>
__global__ void k_to_caller(const T* __restrict__ st, T* __restrict__ ext, KParams p) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p.N) return;
  ext[e] = st[storage_of_ext(p, e)];
}

// ---------------------------------------------------------------- batches
// Many domains of different sizes advance in one launch per phase.  The
// block table is an array of DomRec; the plan kernels turn each domain's
// device-side list counts into prefix offsets, and every batched kernel maps
// its global work index to (domain, local index) by binary search over the
// offsets.  Domain ranges of the cell lists are padded to multiples of 32,
// so a warp never straddles two domains and the warp-collective code of the
// single-domain bodies runs unchanged.

// Largest domain k < n with off[k] <= g (off non-decreasing, off[0] = 0).
__device__ __forceinline__ int find_domain(const int* __restrict__ off, int n, int g) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int round32(int v) { return (v + 31) & ~31; }

// Plan of the first phase (before geometry): resets the counters this step
// fills and lays out tiles, bulk warp units and band cells.
static __global__ void kb_plan_front(DomRec* recs, BatchPlan pl) {
  constexpr int kGroups = 32 / kSegCells;
  if (threadIdx.x == 0) {
    *(pl.all + pl.n + 1) = 0;  // the bulk sweep's hand-out counter
    *(pl.all + pl.n + 2) = 0;  // and the fused sweep's tile counter
  }
  for (int k = threadIdx.x; k < pl.n; k += blockDim.x) reset_step_counts(recs[k].d, recs[k].parity);
  __syncthreads();
  block_prefix(pl.n, pl.tiles, [&](int k) { return recs[k].d.counts[3 + recs[k].parity]; });
  block_prefix(pl.n, pl.bulk, [&](int k) { return (recs[k].d.counts[5] + kGroups - 1) / kGroups; });
  block_prefix(pl.n, pl.band, [&](int k) { return round32(recs[k].d.counts[recs[k].parity]); });
}

// Plan of the second phase (after the new-cell list is complete).
static __global__ void kb_plan_back(DomRec* recs, BatchPlan pl) {
  block_prefix(pl.n, pl.all, [&](int k) {
    return round32(recs[k].d.counts[recs[k].parity] + recs[k].d.counts[2]);
  });
}

template <int Q, class S>
__global__ void __launch_bounds__(kGeoBlock, kGeoMinBlocks) kb_geometry(const DomRec* __restrict__ recs, BatchPlan pl) {
  extern __shared__ __align__(16) unsigned char g_smem[];
  const int total = pl.tiles[pl.n];
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    const int k = find_domain(pl.tiles, pl.n, t);
    const DomRec& r = recs[k];
    geometry_tile<Q, S>(r.d, r.p, r.d.tiles[r.parity][t - pl.tiles[k]], g_smem);
  }
}

// The batch's bulk hand-out counter: the int after the four prefix arrays
// of the plan (n + 1 entries each), cleared by kb_plan_front every step.
__device__ __forceinline__ int* batch_bulk_ctr(const BatchPlan& pl) { return pl.all + pl.n + 1; }

// Units of all domains handed out as in k_bulk, kBulkChunk at a time.
template <int Q, class S, int COLL>
__device__ __forceinline__ void batch_bulk_sweep(const DomRec* __restrict__ recs, const BatchPlan& pl) {
  const int total = pl.bulk[pl.n];
  auto unit = [&](int w) {
    const int k = find_domain(pl.bulk, pl.n, w);
    const DomRec& r = recs[k];
    bulk_unit<Q, S, COLL>(r.d, r.p, r.parity, w - pl.bulk[k], r.d.counts[5]);
  };
  if constexpr (kBulkChunk > 0) {
    for (;;) {
      int base = 0;
      if ((threadIdx.x & 31) == 0) base = atomicAdd(batch_bulk_ctr(pl), kBulkChunk);
      base = __shfl_sync(0xffffffffu, base, 0);
      if (base >= total) break;
      const int end = base + kBulkChunk < total ? base + kBulkChunk : total;
      for (int w = base; w < end; ++w) unit(w);
    }
  } else {
    const int warps = (gridDim.x * kBulkBlock) >> 5;
    for (int w = (blockIdx.x * kBulkBlock + threadIdx.x) >> 5; w < total; w += warps) unit(w);
  }
}

template <int Q, class S, int COLL>
__global__ void __launch_bounds__(kBulkBlock, (bulk_min_blocks<S, COLL>()))
    kb_bulk(const DomRec* __restrict__ recs, BatchPlan pl) {
  batch_bulk_sweep<Q, S, COLL>(recs, pl);
}

// The batch's bulk sweep with the geometry tiles of all domains folded in,
// as k_bulk_geo: the blocks first take tiles from the plan's tile counter
// (the int after the bulk hand-out counter), then bulk units.
template <int Q, class S, int COLL>
__global__ void __launch_bounds__(kBulkBlock, (bulk_min_blocks<S, COLL>()))
    kb_bulk_geo(const DomRec* __restrict__ recs, BatchPlan pl) {
  extern __shared__ __align__(16) unsigned char g_smem[];
  __shared__ int s_tile;
  if (blockIdx.x % kGeoFuseEvery == 0) {
    const int total = pl.tiles[pl.n];
    for (;;) {
      __syncthreads();  // every thread has read the previous s_tile
      if (threadIdx.x == 0) s_tile = atomicAdd(batch_bulk_ctr(pl) + 1, 1);
      __syncthreads();
      const int t = s_tile;
      if (t >= total) break;
      const int k = find_domain(pl.tiles, pl.n, t);
      const DomRec& r = recs[k];
      geometry_tile<Q, S, kBulkBlock>(r.d, r.p, r.d.tiles[r.parity][t - pl.tiles[k]], g_smem);
    }
  }
  batch_bulk_sweep<Q, S, COLL>(recs, pl);
}

template <int Q, class S, int COLL>
__global__ void __launch_bounds__(128, (iface_min_blocks<S, COLL>())) kb_interface(const DomRec* __restrict__ recs, BatchPlan pl) {
  const int total = pl.band[pl.n];
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    const int k = find_domain(pl.band, pl.n, g);
    const DomRec& r = recs[k];
    const int i = g - pl.band[k];
    if (i >= r.d.counts[r.parity]) continue;
    bool bad = false;
    interface_cell<Q, S, COLL>(r.d, r.p, r.parity, i, bad);
    if (bad) r.d.err[0] = 1;
  }
}

template <int Q>
__global__ void __launch_bounds__(kBlock) kb_resolve(const DomRec* __restrict__ recs, BatchPlan pl) {
  const int total = pl.band[pl.n];
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    const int k = find_domain(pl.band, pl.n, g);
    const DomRec& r = recs[k];
    const int i = g - pl.band[k];
    if (i < r.d.counts[r.parity]) resolve_cell<Q>(r.d, r.p, r.parity, i);
  }
}

template <int Q>
__global__ void __launch_bounds__(kBlock) kb_count(const DomRec* __restrict__ recs, BatchPlan pl) {
  const int total = pl.band[pl.n];
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    const int k = find_domain(pl.band, pl.n, g);
    const DomRec& r = recs[k];
    const int i = g - pl.band[k];
    if (i < r.d.counts[r.parity]) count_cell<Q>(r.d, r.p, r.parity, i);
  }
}

template <int Q, class S>
__global__ void __launch_bounds__(128) kb_apply(const DomRec* __restrict__ recs, BatchPlan pl) {
  const int total = pl.all[pl.n];
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    const int k = find_domain(pl.all, pl.n, g);
    const DomRec& r = recs[k];
    const int i = g - pl.all[k];
    if (i < r.d.counts[r.parity] + r.d.counts[2]) apply_cell<Q, S>(r.d, r.p, r.parity, i);
  }
}

static __global__ void __launch_bounds__(kBlock) kb_finalize(const DomRec* __restrict__ recs, BatchPlan pl) {
  const int total = pl.all[pl.n];
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int base = wid * 32; base < total; base += warps * 32) {
    const int k = find_domain(pl.all, pl.n, base);
    const DomRec& r = recs[k];
    finalize_warp(r.d, r.p, r.parity, base - pl.all[k]);
  }
}

// Bubble pressures of every domain (one block each), then the step is done
// and the domain's buffers swap.
static __global__ void kb_bubble_end(DomRec* recs) {
  DomRec& r = recs[blockIdx.x];
  if (r.p.bubble_model && r.d.nb > 0) bubble_update(r.d, r.p);
  __syncthreads();
  if (threadIdx.x == 0) r.parity ^= 1;
}

}  // namespace fslbm
