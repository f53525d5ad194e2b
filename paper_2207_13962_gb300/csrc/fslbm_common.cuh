// Device-side building blocks of the FSLBM step: lattice tables, cell-flag
// bits, PDF storage formats and the parameter block passed to every kernel.
//
// Lattices D3Q19 / D3Q27 of Sec. 2.1 (weights from the standard sets); the
// direction order is the one documented in include/fslbm.h.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fslbm {

// ----------------------------------------------------------------- flags
// bits 0-1: cell type; static bits (computed once at init): bit 2 "a lattice
// neighbour is an obstacle cell", bit 3 "a lattice neighbour lies across a
// periodic face", bit 4 "a lattice neighbour lies outside a non-periodic
// face".
enum : uint8_t { T_GAS = 0, T_IFACE = 1, T_LIQ = 2, T_OBST = 3 };
enum : uint8_t { F_TYPE = 3, F_NEAR_WALL = 4, F_WRAP = 8, F_FACE = 16 };
// Thuerey classes of interface cells.
enum : uint8_t { CL_STD = 0, CL_NF = 1, CL_NE = 2 };
// Conversion marks.
enum : uint8_t { CV_NONE = 0, CV_TOL = 1, CV_TOG = 2, CV_DEFER = 3 };

// ------------------------------------------------------------- lattice
// Direction i encoded as (cx+1) + 3 (cy+1) + 9 (cz+1).
__host__ __device__ constexpr int dcode(int i) {
  return i == 0    ? 13
         : i == 1  ? 14
         : i == 2  ? 12
         : i == 3  ? 16
         : i == 4  ? 10
         : i == 5  ? 22
         : i == 6  ? 4
         : i == 7  ? 17
         : i == 8  ? 9
         : i == 9  ? 11
         : i == 10 ? 15
         : i == 11 ? 23
         : i == 12 ? 3
         : i == 13 ? 5
         : i == 14 ? 21
         : i == 15 ? 25
         : i == 16 ? 1
         : i == 17 ? 7
         : i == 18 ? 19
         : i == 19 ? 26
         : i == 20 ? 0
         : i == 21 ? 8
         : i == 22 ? 18
         : i == 23 ? 20
         : i == 24 ? 6
         : i == 25 ? 24
                   : 2;
}
__host__ __device__ constexpr int CX(int i) { return dcode(i) % 3 - 1; }
__host__ __device__ constexpr int CY(int i) { return (dcode(i) / 3) % 3 - 1; }
__host__ __device__ constexpr int CZ(int i) { return dcode(i) / 9 - 1; }
__host__ __device__ constexpr int OPP(int i) {
  return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
}
__host__ __device__ constexpr int N2(int i) {
  return CX(i) * CX(i) + CY(i) * CY(i) + CZ(i) * CZ(i);
}

template <int Q, class R>
__host__ __device__ constexpr R W(int i) {
  return Q == 19 ? (N2(i) == 0   ? R(1.0 / 3.0)
                    : N2(i) == 1 ? R(1.0 / 18.0)
                                 : R(1.0 / 36.0))
                 : (N2(i) == 0   ? R(8.0 / 27.0)
                    : N2(i) == 1 ? R(2.0 / 27.0)
                    : N2(i) == 2 ? R(1.0 / 54.0)
                                 : R(1.0 / 216.0));
}

// -------------------------------------------------------------- storage
// T: stored type; Real: arithmetic type.
//
// FP64 stores f and computes in FP64 with the plain CPU oracle's expressions
// (bitwise parity).  The other formats store the deviation d = f - w_i from
// the rest state and compute in FP32 on deviations: with |d| ~ 1e-3 instead
// of |f| ~ 0.1, the rounding of every stored value and of every collision is
// ~100x smaller in absolute terms, which is what keeps the liquid mass (a sum
// of stored PDFs) from drifting.  FP16 stores d * 2^15 (|d| <= 1 stays below
// the FP16 maximum 65504, and deviations down to ~4e-9 stay normal numbers);
// BF16 has FP32's exponent range and stores d unscaled.
//   loadd / stored: stored value <-> deviation (FP32 formats only)
//   load / store:   stored value <-> absolute PDF f
struct StoreF64 {
  using T = double;
  using Real = double;
  static constexpr int code = 0;
  static constexpr bool kDev = false;
  static constexpr bool kExactRest = false;
  __device__ static __forceinline__ Real load(T v, Real) { return v; }
  __device__ static __forceinline__ T store(Real f, Real) { return f; }
};
struct StoreF32 {
  using T = float;
  using Real = float;
  static constexpr int code = 1;
  static constexpr bool kDev = true;
  static constexpr bool kExactRest = false;
  __device__ static __forceinline__ float loadd(T v) { return v; }
  __device__ static __forceinline__ T stored(float d) { return d; }
  __device__ static __forceinline__ Real load(T v, Real w) { return loadd(v) + w; }
  __device__ static __forceinline__ T store(Real f, Real w) { return stored(f - w); }
};
struct StoreF16S {
  using T = __half;
  using Real = float;
  static constexpr int code = 2;
  static constexpr bool kDev = true;
  static constexpr bool kExactRest = false;
  __device__ static __forceinline__ float loadd(T v) { return __half2float(v) * 0x1p-15f; }
  __device__ static __forceinline__ T stored(float d) { return __float2half_rn(d * 0x1p15f); }
  __device__ static __forceinline__ Real load(T v, Real w) { return loadd(v) + w; }
  __device__ static __forceinline__ T store(Real f, Real w) { return stored(f - w); }
};
struct StoreBF16S {
  using T = __nv_bfloat16;
  using Real = float;
  static constexpr int code = 3;
  static constexpr bool kDev = true;
  static constexpr bool kExactRest = false;
  __device__ static __forceinline__ float loadd(T v) { return __bfloat162float(v); }
  __device__ static __forceinline__ T stored(float d) { return __float2bfloat16_rn(d); }
  __device__ static __forceinline__ Real load(T v, Real w) { return loadd(v) + w; }
  __device__ static __forceinline__ T store(Real f, Real w) { return stored(f - w); }
};

// Mass-conserving variants of the FP32 and FP16 deviation formats.  The
// q - 1 moving deviations are stored as in the base format, but only values
// on the grid of multiples of 2^-kShift: FP32 values are rounded to it, and
// FP16 values (d 2^15) keep their own rounding where its step is coarser
// than the grid and are rounded to the grid below.  Every stored value is
// then an integer number of grid steps, and the rest deviation d_0 is stored
// as that integer (int32) in a slice of its own after the q slices of the
// buffer.  A collision stores d_0 = (sum of the stored values it received)
// - (sum of the q - 1 moving values it stores), computed in integers: a
// liquid cell's stored sum (its density) is exactly the one it received,
// streaming and bounce-back move stored values unchanged, and the liquid's
// total mass does not drift.  The sums run in integer arithmetic (no FP64,
// whose rate is low on this GPU).  The grid bounds the deviations to
// |d| < 2^(31 - kShift) (2^-3 for FP32MC, 2 for FP16SMC); a value beyond is
// reported as an instability.
struct StoreF32MC {
  using T = float;
  using Real = float;
  static constexpr int code = 4;
  static constexpr bool kDev = true;
  static constexpr bool kExactRest = true;
  static constexpr int kShift = 34;
  __device__ static __forceinline__ float loadd(T v) { return v; }
  __device__ static __forceinline__ T stored(float d) { return rintf(d * 0x1p34f) * 0x1p-34f; }
  // the stored value in grid steps (exact: |v| 2^34 < 2^31 on the grid)
  __device__ static __forceinline__ int steps(T v) { return __float2int_rn(v * 0x1p34f); }
  __device__ static __forceinline__ Real load(T v, Real w) { return loadd(v) + w; }
  __device__ static __forceinline__ T store(Real f, Real w) { return stored(f - w); }
};
struct StoreF16SMC {
  using T = __half;
  using Real = float;
  static constexpr int code = 5;
  static constexpr bool kDev = true;
  static constexpr bool kExactRest = true;
  static constexpr int kShift = 30;
  __device__ static __forceinline__ float loadd(T v) { return __half2float(v) * 0x1p-15f; }
  __device__ static __forceinline__ T stored(float d) {
    const float x = d * 0x1p15f;  // the value held in FP16
    // below 2^-4 the FP16 step is finer than the grid step 2^-15 of x
    return fabsf(x) < 0.0625f ? __float2half_rn(rintf(x * 0x1p15f) * 0x1p-15f) : __float2half_rn(x);
  }
  __device__ static __forceinline__ int steps(T v) { return __float2int_rn(__half2float(v) * 0x1p15f); }
  __device__ static __forceinline__ Real load(T v, Real w) { return loadd(v) + w; }
  __device__ static __forceinline__ T store(Real f, Real w) { return stored(f - w); }
};

// ------------------------------------------------- division by invariants
// Unsigned division of n < 2^31 by a run-time constant d through one
// multiply-high (Granlund & Montgomery, "Division by invariant integers using
// multiplication", 1994): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (mulhi(n, m) + n) >> l.
struct FastDiv {
  unsigned d, m, l;
  __device__ __forceinline__ unsigned div(unsigned n) const { return (__umulhi(n, m) + n) >> l; }
};
inline FastDiv make_fastdiv(unsigned d) {
  FastDiv f;
  f.d = d;
  f.l = 0;
  while ((1ull << f.l) < d) ++f.l;
  f.m = (unsigned)((((1ull << f.l) - d) << 32) / d + 1ull);
  return f;
}

// Resident blocks of 256 threads per SM that the bulk sweep is compiled for
// (FP32 arithmetic; the FP64 engine uses 2); its persistent grid is this
// many blocks per SM.
#ifndef FSLBM_BULK_MINB
#define FSLBM_BULK_MINB 4
#endif
constexpr int kBulkMinBlocks32 = FSLBM_BULK_MINB;

// Granularity of the bulk sweep's work list: groups of kSegCells consecutive
// cells that hold liquid; a warp takes 32 / kSegCells groups.  32 keeps each
// warp-wide load one contiguous 128-byte row of a PDF slice: smaller groups
// raise lane occupancy on ragged liquid regions but split every load into
// separate sectors, which measured slower on GB300 (0.82 vs 0.59 ms per sweep
// of the 160 x 160 x 1024 Taylor bubble for 8-cell groups).
#ifndef FSLBM_SEG_CELLS
#define FSLBM_SEG_CELLS 32
#endif
constexpr int kSegCells = FSLBM_SEG_CELLS;
static_assert(kSegCells == 8 || kSegCells == 16 || kSegCells == 32, "segment size");

// Direction whose components are those of direction i with the ones along
// the axes in mask (bit 0 x, 1 y, 2 z) reversed: the specular image of i at
// walls normal to those axes.
struct ReflectTable {
  signed char j[27][8];
};
__host__ __device__ constexpr int dir_of_code(int code) {
  int r = -1;
  for (int i = 0; i < 27; ++i)
    if (dcode(i) == code) r = i;
  return r;
}
__host__ __device__ constexpr ReflectTable make_reflect_table() {
  ReflectTable t{};
  for (int i = 0; i < 27; ++i)
    for (int m = 0; m < 8; ++m) {
      const int cx = (m & 1) ? -CX(i) : CX(i);
      const int cy = (m & 2) ? -CY(i) : CY(i);
      const int cz = (m & 4) ? -CZ(i) : CZ(i);
      t.j[i][m] = (signed char)dir_of_code((cx + 1) + 3 * (cy + 1) + 9 * (cz + 1));
    }
  return t;
}
__constant__ constexpr ReflectTable kReflect = make_reflect_table();

// ----------------------------------------------------------- parameters
// Storage order of the cells.  The caller's coordinates (x, y, z) and cell
// index x + nx (y + ny z) are fixed; inside the library any axis may be the
// contiguous one.  ax[k] is the caller's axis at storage position k (k = 0
// contiguous), so a cell's storage index is c = a0 + m0 (a1 + m1 a2), a_k
// its coordinate along axis ax[k] and m_k that axis' size; sx, sy, sz are
// the strides of x, y, z in c and inv[a] the storage position of axis a.
// Direction labels, their vectors and all arithmetic stay in the caller's
// axes: only index computations see the storage order.
struct KParams {
  FastDiv div0, div1;  // division by m0 and m1 (decoding a storage index)
  int ax[3], inv[3];
  int m0, m1;
  int sx, sy, sz;
  int off[27];         // storage-index offset of direction i: c_i . (sx, sy, sz)
  long long dofs[27];  // i * Np - off[i]: pull source of interior cells
  int nx, ny, nz;
  int per[3];   // periodic axes
  int slip[3];  // axes with free-slip walls (specular reflection) outside
  int N;        // cells
  long long Np; // padded cells per PDF direction slice
  double omega, om_m, pref_p, pref_m;  // SRT: pref_p = 1 - omega/2
  double magic;  // TRT magic parameter (omega- of the LES-adjusted omega+)
  double cs;     // Smagorinsky constant, 0: no LES
  double g[3];
  // FP32 copies of the parameters the FP32 engines use in every cell (a
  // double-to-float conversion on the device runs on the FP64 pipe)
  float fg[3], fomega, fom_m, fpref_p, fpref_m, fmagic, fcs;
  double sigma, eps, pv0;
  int variant, om3_fb, bubble_model, collision;
};

// Fills the storage-order fields of k (nx, ny, nz and Np already set) for
// the axis order ax (a permutation of 0, 1, 2; ax[0] contiguous).
inline void set_layout(KParams& k, const int ax[3]) {
  const int n[3] = {k.nx, k.ny, k.nz};
  int s[3];
  for (int pos = 0; pos < 3; ++pos) {
    k.ax[pos] = ax[pos];
    k.inv[ax[pos]] = pos;
  }
  k.m0 = n[ax[0]];
  k.m1 = n[ax[1]];
  s[ax[0]] = 1;
  s[ax[1]] = k.m0;
  s[ax[2]] = k.m0 * k.m1;
  k.sx = s[0];
  k.sy = s[1];
  k.sz = s[2];
  k.div0 = make_fastdiv((unsigned)k.m0);
  k.div1 = make_fastdiv((unsigned)k.m1);
  for (int i = 0; i < 27; ++i) {
    k.off[i] = CX(i) * k.sx + CY(i) * k.sy + CZ(i) * k.sz;
    k.dofs[i] = (long long)i * k.Np - k.off[i];
  }
}

inline bool is_identity_layout(const KParams& k) { return k.ax[0] == 0 && k.ax[1] == 1 && k.ax[2] == 2; }

// Fills the FP32 copies of k's FP64 parameters (rounded to nearest, as a
// device conversion would).
inline void set_float_params(KParams& k) {
  for (int a = 0; a < 3; ++a) k.fg[a] = (float)k.g[a];
  k.fomega = (float)k.omega;
  k.fom_m = (float)k.om_m;
  k.fpref_p = (float)k.pref_p;
  k.fpref_m = (float)k.pref_m;
  k.fmagic = (float)k.magic;
  k.fcs = (float)k.cs;
}

// Gravity component a in the arithmetic type R.
template <class R>
__device__ __forceinline__ R gpar(const KParams& p, int a) {
  if constexpr (sizeof(R) == 4) return p.fg[a];
  else return p.g[a];
}

// FP64 arithmetic and conversions run on this GPU's small FP64 unit (two
// lanes a clock per SM), so the FP32 engines keep it out of per-neighbour
// work with the two helpers below.

// x rounded to the nearest float (ties to even) with integer operations.
// Magnitudes below 2^-126 give a signed zero (the fill levels and masses it
// converts never come near); infinities and NaN take the conversion
// instruction.
__device__ __forceinline__ float d2f(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ex = (hi >> 20) & 0x7ffu;
  const unsigned sign = hi & 0x80000000u;
  if (ex == 0x7ffu) return __double2float_rn(x);
  const int fe = (int)ex - 1023 + 127;
  if (fe <= 0) return __uint_as_float(sign);
  if (fe >= 255) return __uint_as_float(sign | 0x7f800000u);
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);  // top 23 mantissa bits
  const unsigned rem = lo & 0x1fffffffu;                    // the 29 dropped bits
  unsigned r = sign | ((unsigned)fe << 23) | m;
  // round to nearest, ties to even; a carry out of the mantissa raises the
  // exponent (to infinity past the largest float)
  if (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) r += 1u;
  return __uint_as_float(r);
}

// A sum of floats held as an unevaluated pair hi + lo: each addition's
// rounding error (Knuth's TwoSum, exact in round-to-nearest) goes to lo, so
// the pair carries about 48 significant bits.
struct FAcc {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float s = __fadd_rn(hi, v);
    const float bv = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(v, bv));
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  // adds a - b exactly (its rounding error goes to lo as well)
  __device__ __forceinline__ void add_diff(float a, float b) {
    const float s = __fsub_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float e = __fsub_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fadd_rn(b, bv));
    add(s);
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Device pointers of one domain.
struct DPtrs {
  void* pdf[2];
  uint8_t* flags;
  uint32_t* wallmask;  // bit i: the pull source of direction i is an obstacle
                       // cell (static); sources outside the domain are not
                       // included
  double* phi;
  double* mass;
  int* bid;
  uint8_t* cls;
  uint8_t* mark;
  uint8_t* conv;
  uint8_t* cfin;
  uint8_t* claim;
  uint8_t* rcv;    // 1: an interface cell next to a cell that converts this
                   // step (set by the count kernel, cleared by apply)
  double* share;
  int* band[2];
  int* counts;   // [0],[1]: band list counts; [2]: new-cell list count;
                 // [3],[4]: geometry tile list counts; [5]: segment count;
                 // [6], [7]: the step's bulk-unit and tile hand-out
  int* tiles[2]; // geometry tiles (8^3) holding interface cells
  int* tile_mark;
  int* segs;     // 32-cell segments (linear index / 32) holding liquid;
  int* seg_mark; // grows when cells turn liquid, count in counts[5]
  int* newlist;
  void* nhat;    // Real[3 * cap]
  void* rhog;    // Real[cap]
  double* mom_rho;  // rho and u of the interface cells' post-collision PDFs,
  void* mom_u;      // (Real[3 * N]) written by the interface kernel in the
                    // same arithmetic as post_moments, read for new cells
  double* m_next;
  double* phi_next;
  double* rho_band;
  double* V0;
  double* pV;
  double* Vcur;
  long long* gas_cnt;
  long long* iface_fix;
  int nb;
  int* err;      // [0] instability seen
  double* red;   // observable partials
  int red_blocks;
};

// One domain of a batch (a block-table entry): device pointers, parameters
// and the parity of the PDF buffer that holds its current state.
struct DomRec {
  DPtrs d;
  KParams p;
  int parity;
};

// Prefix offsets (n + 1 entries each, device memory) of the domains' work in
// the units of each batched kernel, recomputed on the device every step:
//   tiles: geometry tiles; bulk: warp units of the bulk sweep;
//   band: interface cells rounded up to a multiple of 32 (warp-aligned);
//   all: interface + new interface cells rounded up to a multiple of 32.
struct BatchPlan {
  int n;
  int* tiles;
  int* bulk;
  int* band;
  int* all;
};

}  // namespace fslbm
