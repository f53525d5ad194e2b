// Lattice-cell layer of the FSLBM kernels (arXiv 2207.13962, Sec. 2):
// index helpers, equilibrium, Guo forcing, SRT/TRT collision in the stored
// representation, storage conversions, moments of stored PDFs and the
// bounce-back through obstacle slots.  Shared by the bulk sweep and the
// interface kernels.
#pragma once

#include "fslbm_common.cuh"

namespace fslbm {
constexpr int kBlock = 256;

// ------------------------------------------------------------ index helpers
__device__ __forceinline__ int wrapc(int X, int n, int per) {
  if (X >= 0 && X < n) return X;
  if (!per) return -1;
  X %= n;
  if (X < 0) X += n;
  return X;
}
__device__ __forceinline__ int sel3(int k, int a0, int a1, int a2) {
  return k == 0 ? a0 : (k == 1 ? a1 : a2);
}
// caller coordinates (x, y, z) of the cell with storage index c
__device__ __forceinline__ void decode(const KParams& p, int c, int& x, int& y, int& z) {
  const int t = (int)p.div0.div((unsigned)c);
  const int a0 = c - t * p.m0;
  const int a2 = (int)p.div1.div((unsigned)t);
  const int a1 = t - a2 * p.m1;
  x = sel3(p.inv[0], a0, a1, a2);
  y = sel3(p.inv[1], a0, a1, a2);
  z = sel3(p.inv[2], a0, a1, a2);
}
// storage index of the cell at caller coordinates (X, Y, Z) inside the domain
__device__ __forceinline__ int cidx(const KParams& p, int X, int Y, int Z) {
  return X * p.sx + Y * p.sy + Z * p.sz;
}
// the caller's index x + nx (y + ny z) of the cell with storage index c
__device__ __forceinline__ int ext_index(const KParams& p, int c) {
  int x, y, z;
  decode(p, c, x, y, z);
  return x + p.nx * (y + p.ny * z);
}
// neighbour of (x,y,z) at offset (dx,dy,dz); -1 outside a non-periodic face
__device__ __forceinline__ int nbr(const KParams& p, int x, int y, int z, int dx, int dy,
                                   int dz) {
  int X = wrapc(x + dx, p.nx, p.per[0]);
  int Y = wrapc(y + dy, p.ny, p.per[1]);
  int Z = wrapc(z + dz, p.nz, p.per[2]);
  if (X < 0 || Y < 0 || Z < 0) return -1;
  return cidx(p, X, Y, Z);
}
__device__ __forceinline__ int ntype(const uint8_t* flags, int n) {
  return n < 0 ? T_OBST : (flags[n] & F_TYPE);
}

// warp-aggregated append; every lane of the warp must call it
__device__ __forceinline__ int warp_append(int* counter, bool pred) {
  const unsigned lane = threadIdx.x & 31u;
  unsigned b = __ballot_sync(0xffffffffu, pred);
  int base = 0;
  if (lane == 0 && b) base = atomicAdd(counter, __popc(b));
  base = __shfl_sync(0xffffffffu, base, 0);
  return pred ? base + __popc(b & ((1u << lane) - 1u)) : -1;
}

// Block-wide exclusive prefix sum (one block) of values f(k), k < n, into
// off[0..n]; f must not read off.
template <class F>
__device__ __forceinline__ void block_prefix(int n, int* off, F f) {
  __shared__ int carry;
  __shared__ int wsum[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int base = 0; base < n; base += blockDim.x) {
    const int k = base + threadIdx.x;
    const int v = k < n ? f(k) : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int t = lane < nw ? wsum[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      wsum[lane] = t;
    }
    __syncthreads();
    const int incl = x + (wid > 0 ? wsum[wid - 1] : 0) + carry;
    if (k < n) off[k + 1] = incl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) off[0] = 0;
}

// ---------------------------------------------------------- cell algebra
// Eq. nm-lbm-equilibrium with c_s^2 = 1/3.
template <int Q, class R>
__device__ __forceinline__ R feq_i(int i, R rho, R ux, R uy, R uz) {
  R cu = R(CX(i)) * ux + R(CY(i)) * uy + R(CZ(i)) * uz;
  R usq = ux * ux + uy * uy + uz * uz;
  R t = R(1.0) + R(3.0) * cu;
  t = t + R(4.5) * cu * cu;
  t = t - R(1.5) * usq;
  return W<Q, R>(i) * rho * t;
}
// Guo source without its (1 - omega/2) factor (Eq. nm-lbm-force-guo).
template <int Q, class R>
__device__ __forceinline__ R guo_i(int i, R ux, R uy, R uz, R Fx, R Fy, R Fz) {
  R cx = R(CX(i)), cy = R(CY(i)), cz = R(CZ(i));
  R cu = cx * ux + cy * uy + cz * uz;
  R cF = cx * Fx + cy * Fy + cz * Fz;
  R uF = ux * Fx + uy * Fy + uz * Fz;
  R t = R(3.0) * (cF - uF) + R(9.0) * cu * cF;
  return W<Q, R>(i) * t;
}
// rho = sum f (Eq. nm-lbm-density); j sums in direction order.
template <int Q, class R>
__device__ __forceinline__ void sums(const R* f, R& r, R& jx, R& jy, R& jz) {
  r = R(0.0);
#pragma unroll
  for (int i = 0; i < Q; ++i) r = r + f[i];
  jx = R(0.0);
#pragma unroll
  for (int i = 0; i < Q; ++i)
    if (CX(i) != 0) jx = jx + R(CX(i)) * f[i];
  jy = R(0.0);
#pragma unroll
  for (int i = 0; i < Q; ++i)
    if (CY(i) != 0) jy = jy + R(CY(i)) * f[i];
  jz = R(0.0);
#pragma unroll
  for (int i = 0; i < Q; ++i)
    if (CZ(i) != 0) jz = jz + R(CZ(i)) * f[i];
}

// Collision of one cell (Eqs. nm-lbm-collision, nm-lbm-velocity with
// F = rho g, SRT relaxing towards f^eq, or TRT).  f is overwritten with f*.
// Returns rho; sets unstable when |u|^2 >= c_s^2, rho <= 0 or NaN.
template <int Q, class R, int COLL>
__device__ __forceinline__ R collide(R* f, const KParams& p, bool& unstable) {
  R rho, jx, jy, jz;
  sums<Q, R>(f, rho, jx, jy, jz);
  const R gx = R(p.g[0]), gy = R(p.g[1]), gz = R(p.g[2]);
  R ux = jx / rho + R(0.5) * gx;
  R uy = jy / rho + R(0.5) * gy;
  R uz = jz / rho + R(0.5) * gz;
  R Fx = rho * gx, Fy = rho * gy, Fz = rho * gz;
  R usq = ux * ux + uy * uy + uz * uz;
  if (!(usq < R(1.0 / 3.0)) || !(rho > R(0.0))) unstable = true;
  if (COLL == 0) {
    const R om = R(p.omega), pref = R(p.pref_p);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      R fe = feq_i<Q, R>(i, rho, ux, uy, uz);
      R s = guo_i<Q, R>(i, ux, uy, uz, Fx, Fy, Fz);
      f[i] = f[i] - om * (f[i] - fe) + pref * s;
    }
  } else {
    // TRT on the pairs (i, ibar): the symmetric parts are shared, the
    // antisymmetric parts change sign (same roundings as a per-i loop).
    const R omp = R(p.omega), omm = R(p.om_m), prp = R(p.pref_p), prm = R(p.pref_m);
    {
      const R fe = feq_i<Q, R>(0, rho, ux, uy, uz);
      const R sr = guo_i<Q, R>(0, ux, uy, uz, Fx, Fy, Fz);
      const R fp = R(0.5) * (f[0] + f[0]), fm = R(0.5) * (f[0] - f[0]);
      const R ep = R(0.5) * (fe + fe), em = R(0.5) * (fe - fe);
      const R sp = R(0.5) * (sr + sr), sm = R(0.5) * (sr - sr);
      f[0] = f[0] - omp * (fp - ep) - omm * (fm - em) + prp * sp + prm * sm;
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
      const int j = i + 1;
      const R fei = feq_i<Q, R>(i, rho, ux, uy, uz), fej = feq_i<Q, R>(j, rho, ux, uy, uz);
      const R si = guo_i<Q, R>(i, ux, uy, uz, Fx, Fy, Fz), sj = guo_i<Q, R>(j, ux, uy, uz, Fx, Fy, Fz);
      const R fp = R(0.5) * (f[i] + f[j]);
      const R ep = R(0.5) * (fei + fej);
      const R sp = R(0.5) * (si + sj);
      const R fmi = R(0.5) * (f[i] - f[j]), fmj = R(0.5) * (f[j] - f[i]);
      const R emi = R(0.5) * (fei - fej), emj = R(0.5) * (fej - fei);
      const R smi = R(0.5) * (si - sj), smj = R(0.5) * (sj - si);
      const R oi = f[i] - omp * (fp - ep) - omm * (fmi - emi) + prp * sp + prm * smi;
      const R oj = f[j] - omp * (fp - ep) - omm * (fmj - emj) + prp * sp + prm * smj;
      f[i] = oi;
      f[j] = oj;
    }
  }
  return rho;
}

// Equilibrium deviation f^eq_i - w_i = w_i (drho + rho (3 c.u + 4.5 (c.u)^2
// - 1.5 u.u)) with drho = rho - 1 (Eq. nm-lbm-equilibrium).
template <int Q, class R>
__device__ __forceinline__ R feq_dev(int i, R drho, R rho, R ux, R uy, R uz) {
  const R cu = R(CX(i)) * ux + R(CY(i)) * uy + R(CZ(i)) * uz;
  const R usq = ux * ux + uy * uy + uz * uz;
  return W<Q, R>(i) * (drho + rho * (R(3.0) * cu + R(4.5) * cu * cu - R(1.5) * usq));
}

// Collision of the FP32 engines on deviations d_i = f_i - w_i (the same
// TRT/SRT with Guo forcing as collide()).  Evaluated per direction pair
// (i, ibar) from the symmetric and antisymmetric parts of f^eq - w
// (w (drho + rho (4.5 (c.u)^2 - 1.5 u.u)) and 3 w rho c.u) and of the
// source; SRT is the case omega- = omega+.  Every intermediate is of the
// size of a deviation, so its rounding is too.  Returns drho.
template <int Q, int COLL>
__device__ __forceinline__ float collide_dev(float* d, const KParams& p, bool& unstable) {
  float dr = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    dr += d[i];
    if (CX(i) != 0) jx += float(CX(i)) * d[i];
    if (CY(i) != 0) jy += float(CY(i)) * d[i];
    if (CZ(i) != 0) jz += float(CZ(i)) * d[i];
  }
  const float rho = 1.0f + dr;
  const float gx = float(p.g[0]), gy = float(p.g[1]), gz = float(p.g[2]);
  const float inv = __frcp_rn(rho);
  const float ux = jx * inv + 0.5f * gx, uy = jy * inv + 0.5f * gy, uz = jz * inv + 0.5f * gz;
  const float Fx = rho * gx, Fy = rho * gy, Fz = rho * gz;
  const float usq = ux * ux + uy * uy + uz * uz;
  if (!(usq < 1.0f / 3.0f) || !(rho > 0.f)) unstable = true;
  const float omp = float(p.omega), prp = float(p.pref_p);
  const float omm = COLL == 0 ? omp : float(p.om_m), prm = COLL == 0 ? prp : float(p.pref_m);
  const float base = dr - 1.5f * rho * usq;
  const float uF3 = 3.0f * (ux * Fx + uy * Fy + uz * Fz);
  {
    const float w = W<Q, float>(0);
    d[0] = d[0] - omp * (d[0] - w * base) - prp * w * uF3;
  }
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const int j = i + 1;
    const float w = W<Q, float>(i);
    const float cu = float(CX(i)) * ux + float(CY(i)) * uy + float(CZ(i)) * uz;
    const float cF = float(CX(i)) * Fx + float(CY(i)) * Fy + float(CZ(i)) * Fz;
    const float es = w * (base + 4.5f * rho * cu * cu);
    const float ea = 3.0f * w * rho * cu;
    const float ss = w * (9.0f * cu * cF - uF3);
    const float sa = 3.0f * w * cF;
    const float fp = 0.5f * (d[i] + d[j]);
    const float fm = 0.5f * (d[i] - d[j]);
    const float A = omp * (fp - es) - prp * ss;
    const float B = omm * (fm - ea) - prm * sa;
    const float di = d[i] - A - B;
    const float dj = d[j] - A + B;
    d[i] = di;
    d[j] = dj;
  }
  return dr;
}

// Collision in the engine's working representation (absolute f in FP64,
// deviations otherwise); returns rho.
template <int Q, class S, int COLL>
__device__ __forceinline__ double collide_any(typename S::Real* f, const KParams& p,
                                              bool& unstable) {
  if constexpr (!S::kDev)
    return collide<Q, double, COLL>(f, p, unstable);
  else
    return 1.0 + (double)collide_dev<Q, COLL>(f, p, unstable);
}

// PDF i of cell c in the working representation.
template <class S, int Q>
__device__ __forceinline__ typename S::Real load_w(typename S::T v, int i) {
  if constexpr (S::kDev)
    return S::loadd(v);
  else
    return S::load(v, W<Q, typename S::Real>(i));
}
template <class S, int Q>
__device__ __forceinline__ typename S::T store_w(typename S::Real v, int i) {
  if constexpr (S::kDev)
    return S::stored(v);
  else
    return S::store(v, W<Q, typename S::Real>(i));
}

// ------------------------------------------- mass-conserving formats
// The FP64 rest slice that follows the q slices of a PDF buffer.
template <int Q, class S>
__device__ __forceinline__ double* rest_slice(const void* P, long long Np) {
  return (double*)((typename S::T*)P + (long long)Q * Np);
}
template <class S>
__device__ __forceinline__ double snap_rest(double d0) {
  return snap_grid(d0, S::kGrid, 1.0 / S::kGrid);
}

// Stores the post-collision PDFs f (working representation) of storage
// cell c into buffer B.  For the mass-conserving formats s_in is the FP64
// sum of the values the collision received: the rest deviation becomes
// s_in minus the sum of the stored moving values (exact when the inputs
// were stored values, as for liquid cells; rounded to the grid otherwise).
template <int Q, class S>
__device__ __forceinline__ void store_cell(typename S::T* B, long long Np, long long c,
                                           const typename S::Real* f, double s_in) {
  if constexpr (S::kExactRest) {
    double s_out = 0.0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const typename S::T v = S::stored(f[i]);
      B[(long long)i * Np + c] = v;
      s_out += (double)S::loadd(v);
    }
    rest_slice<Q, S>(B, Np)[c] = snap_rest<S>(s_in - s_out);
  } else {
    (void)s_in;
#pragma unroll
    for (int i = 0; i < Q; ++i) B[(long long)i * Np + c] = store_w<S, Q>(f[i], i);
  }
}

// PDF i of storage cell c of buffer P in the working representation (the
// rest PDF of the mass-conserving formats from its FP64 slice).
template <int Q, class S>
__device__ __forceinline__ typename S::Real load_own(const typename S::T* P, long long Np, long long c,
                                                     int i) {
  if constexpr (S::kExactRest) {
    if (i == 0) return (typename S::Real)rest_slice<Q, S>(P, Np)[c];
  }
  return load_w<S, Q>(P[(long long)i * Np + c], i);
}

// rho and u of a cell from its post-collision PDFs: rho u = sum c f* - F/2.
// With deviations, rho = 1 + sum d is summed in FP64 from the stored values,
// so that it equals the cell's mass as the PDFs hold it.
template <int Q, class S>
__device__ __forceinline__ void post_moments(const typename S::T* P, long long Np, int c,
                                             const KParams& p, double& rho,
                                             typename S::Real u[3]) {
  using R = typename S::Real;
  R f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] = load_own<Q, S>(P, Np, c, i);
  R r, jx, jy, jz;
  sums<Q, R>(f, r, jx, jy, jz);
  R rr = r;
  if constexpr (S::kDev) {
    double sd = 0.0;
#pragma unroll
    for (int i = 0; i < Q; ++i)
      sd += (S::kExactRest && i == 0) ? rest_slice<Q, S>(P, Np)[c] : (double)f[i];
    rho = 1.0 + sd;
    rr = R(rho);
  } else {
    rho = r;
  }
  u[0] = jx / rr - R(0.5) * R(p.g[0]);
  u[1] = jy / rr - R(0.5) * R(p.g[1]);
  u[2] = jz / rr - R(0.5) * R(p.g[2]);
}

// ------------------------------------------------- bounce-back via obstacle slots
// Slice-i index of the pull source of direction i of cell c at (x, y, z):
// the neighbour x - c_i, wrapped across periodic faces, or the cell's own
// slot ibar (bounce-back) when the source lies outside a non-periodic face.
template <int Q>
__device__ __forceinline__ long long pull_index_general(const KParams& p, int c, int x, int y,
                                                        int z, int i) {
  int X = x - CX(i), Y = y - CY(i), Z = z - CZ(i);
  bool out = false;
  if (X < 0 || X >= p.nx) {
    if (p.per[0]) X = X < 0 ? X + p.nx : X - p.nx;
    else out = true;
  }
  if (Y < 0 || Y >= p.ny) {
    if (p.per[1]) Y = Y < 0 ? Y + p.ny : Y - p.ny;
    else out = true;
  }
  if (Z < 0 || Z >= p.nz) {
    if (p.per[2]) Z = Z < 0 ? Z + p.nz : Z - p.nz;
    else out = true;
  }
  return out ? (long long)OPP(i) * p.Np + c : (long long)i * p.Np + cidx(p, X, Y, Z);
}

// Reflected copies of a fluid cell's post-collision PDFs (working
// representation f) into the slots of its obstacle pull sources.
template <int Q, class S>
__device__ __forceinline__ void write_reflected(const DPtrs& d, const KParams& p, typename S::T* B,
                                                int c, uint32_t wm, bool general,
                                                const typename S::Real* f) {
  int x = 0, y = 0, z = 0;
  if (general) decode(p, c, x, y, z);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    if (!((wm >> i) & 1u)) continue;
    const long long idx = general ? pull_index_general<Q>(p, c, x, y, z, i) : p.dofs[i] + c;
    B[idx] = store_w<S, Q>(f[OPP(i)], i);
  }
}

}  // namespace fslbm
