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

// Collision variants: bit 0 TRT (else SRT), bit 1 the Smagorinsky model;
// the interface kernels also carry bit 2: the domain has free-slip faces.
__host__ __device__ constexpr bool coll_trt(int coll) { return (coll & 1) != 0; }
__host__ __device__ constexpr bool coll_les(int coll) { return (coll & 2) != 0; }
__host__ __device__ constexpr bool coll_slip(int coll) { return (coll & 4) != 0; }

// Relaxation time of the Smagorinsky model (Sec. 2.1, Eqs.
// nm-lbm-turbulence-viscosity to nm-lbm-turublence-relaxation-time):
// tau = (tau0 + sqrt(tau0^2 + 2 sqrt(2) (C_S dx)^2 Qbar / (rho c_s^4))) / 2
// with Qbar = sqrt(2 sum_ab Q_ab Q_ab) of the momentum flux
// Q_ab = sum_i c_ia c_ib (f_i - f^eq_i) of the PDFs entering the collision
// (dx = 1, c_s^4 = 1/9); the six independent Q_ab are given.
template <class R>
__device__ __forceinline__ R les_tau(R qxx, R qyy, R qzz, R qxy, R qxz, R qyz, R rho, R omega, R cs) {
  const R q2 = qxx * qxx + qyy * qyy + qzz * qzz + R(2.0) * (qxy * qxy + qxz * qxz + qyz * qyz);
  const R qbar = sqrt(R(2.0) * q2);
  const R tau0 = R(1.0) / omega;
  return R(0.5) * (tau0 + sqrt(tau0 * tau0 + R(2.0) * sqrt(R(2.0)) * (cs * cs) * qbar / (rho * (R(1.0) / R(9.0)))));
}

// Collision of one cell (Eqs. nm-lbm-collision, nm-lbm-velocity with
// F = rho g, SRT relaxing towards f^eq, or TRT; with the Smagorinsky model
// when coll_les(COLL)).  f is overwritten with f*.  Returns rho; sets
// unstable when |u|^2 >= c_s^2, rho <= 0 or NaN.
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
  R omega = R(p.omega);
  if constexpr (coll_les(COLL)) {
    // momentum flux of the non-equilibrium part, summed in direction order
    R qxx = R(0.0), qyy = R(0.0), qzz = R(0.0), qxy = R(0.0), qxz = R(0.0), qyz = R(0.0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const R cx = R(CX(i)), cy = R(CY(i)), cz = R(CZ(i));
      const R dn = f[i] - feq_i<Q, R>(i, rho, ux, uy, uz);
      qxx = qxx + cx * cx * dn;
      qyy = qyy + cy * cy * dn;
      qzz = qzz + cz * cz * dn;
      qxy = qxy + cx * cy * dn;
      qxz = qxz + cx * cz * dn;
      qyz = qyz + cy * cz * dn;
    }
    omega = R(1.0) / les_tau<R>(qxx, qyy, qzz, qxy, qxz, qyz, rho, omega, R(p.cs));
  }
  if constexpr (!coll_trt(COLL)) {
    const R om = omega, pref = coll_les(COLL) ? R(1.0) - R(0.5) * omega : R(p.pref_p);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      R fe = feq_i<Q, R>(i, rho, ux, uy, uz);
      R s = guo_i<Q, R>(i, ux, uy, uz, Fx, Fy, Fz);
      f[i] = f[i] - om * (f[i] - fe) + pref * s;
    }
  } else {
    // TRT on the pairs (i, ibar): the symmetric parts are shared, the
    // antisymmetric parts change sign (same roundings as a per-i loop).
    // With the model, omega- follows from the adjusted omega+ through the
    // magic parameter.
    R omp = R(p.omega), omm = R(p.om_m), prp = R(p.pref_p), prm = R(p.pref_m);
    if constexpr (coll_les(COLL)) {
      omp = omega;
      omm = R(1.0) / (R(0.5) + R(p.magic) / (R(1.0) / omp - R(0.5)));
      prp = R(1.0) - R(0.5) * omp;
      prm = R(1.0) - R(0.5) * omm;
    }
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
  // The engines are compiled without multiply-add contraction (so that a
  // cell's arithmetic does not depend on the kernel it is inlined into); the
  // multiply-adds of this hot loop are written out as fused operations.
  const float rho = 1.0f + dr;
  const float gx = p.fg[0], gy = p.fg[1], gz = p.fg[2];
  const float inv = __frcp_rn(rho);
  const float ux = __fmaf_rn(jx, inv, 0.5f * gx), uy = __fmaf_rn(jy, inv, 0.5f * gy),
              uz = __fmaf_rn(jz, inv, 0.5f * gz);
  const float Fx = rho * gx, Fy = rho * gy, Fz = rho * gz;
  const float usq = __fmaf_rn(ux, ux, __fmaf_rn(uy, uy, uz * uz));
  if (!(usq < 1.0f / 3.0f) || !(rho > 0.f)) unstable = true;
  float omp = p.fomega, prp = p.fpref_p;
  float omm = coll_trt(COLL) ? p.fom_m : omp, prm = coll_trt(COLL) ? p.fpref_m : prp;
  const float base = __fmaf_rn(-1.5f * rho, usq, dr);
  const float r45 = 4.5f * rho;
  if constexpr (coll_les(COLL)) {
    // momentum flux of the non-equilibrium part: the pair (i, ibar) shares
    // c_a c_b, and d_i - e_i + d_ibar - e_ibar = d_i + d_ibar - 2 es (the
    // antisymmetric parts cancel)
    float qxx = 0.f, qyy = 0.f, qzz = 0.f, qxy = 0.f, qxz = 0.f, qyz = 0.f;
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
      const float cx = float(CX(i)), cy = float(CY(i)), cz = float(CZ(i));
      const float cu = cx * ux + cy * uy + cz * uz;
      const float es = W<Q, float>(i) * __fmaf_rn(r45 * cu, cu, base);
      const float dn = __fmaf_rn(-2.0f, es, d[i] + d[i + 1]);
      qxx += cx * cx * dn;
      qyy += cy * cy * dn;
      qzz += cz * cz * dn;
      qxy += cx * cy * dn;
      qxz += cx * cz * dn;
      qyz += cy * cz * dn;
    }
    omp = 1.0f / les_tau<float>(qxx, qyy, qzz, qxy, qxz, qyz, rho, omp, p.fcs);
    prp = 1.0f - 0.5f * omp;
    if constexpr (coll_trt(COLL)) {
      omm = 1.0f / (0.5f + p.fmagic / (1.0f / omp - 0.5f));
      prm = 1.0f - 0.5f * omm;
    } else {
      omm = omp;
      prm = prp;
    }
  }
  const float uF3 = 3.0f * __fmaf_rn(ux, Fx, __fmaf_rn(uy, Fy, uz * Fz));
  {
    const float w = W<Q, float>(0);
    const float t0 = __fmaf_rn(-w, base, d[0]);  // d_0 - w base
    d[0] = __fmaf_rn(-omp, t0, __fmaf_rn(-prp * w, uF3, d[0]));
  }
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const int j = i + 1;
    const float w = W<Q, float>(i);
    const float cu = float(CX(i)) * ux + float(CY(i)) * uy + float(CZ(i)) * uz;
    const float cF = float(CX(i)) * Fx + float(CY(i)) * Fy + float(CZ(i)) * Fz;
    const float es = w * __fmaf_rn(r45 * cu, cu, base);
    const float ea = (3.0f * w) * rho * cu;
    const float ss = w * __fmaf_rn(9.0f * cu, cF, -uF3);
    const float sa = (3.0f * w) * cF;
    const float fp = 0.5f * (d[i] + d[j]);
    const float fm = 0.5f * (d[i] - d[j]);
    const float A = __fmaf_rn(omp, fp - es, -prp * ss);
    const float B = __fmaf_rn(omm, fm - ea, -prm * sa);
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
// Grid exponent of a format (0 for the formats without exact rest).
template <class S>
__host__ __device__ constexpr int grid_shift() {
  if constexpr (S::kExactRest) return S::kShift;
  else return 0;
}

// The int32 rest slice (grid steps) that follows the q slices of a PDF buffer.
template <int Q, class S>
__device__ __forceinline__ int* rest_slice(const void* P, long long Np) {
  return (int*)((typename S::T*)P + (long long)Q * Np);
}
// A working value (deviation) in grid steps, rounded to the nearest.
template <class S>
__device__ __forceinline__ long long grid_steps(float d) {
  return __float2ll_rn(d * (float)(1LL << S::kShift));
}
// The same for a working value that is a stored value (exact, 32-bit).
template <class S>
__device__ __forceinline__ int grid_steps32(float d) {
  return __float2int_rn(d * (float)(1LL << S::kShift));
}
template <class S>
__device__ __forceinline__ float from_steps(long long n) {
  return (float)n * (1.0f / (float)(1LL << S::kShift));
}

// Stores the post-collision PDFs f (working representation) of storage
// cell c into buffer B.  For the mass-conserving formats s_in is the sum of
// the values the collision received, in grid steps: the rest deviation
// becomes s_in minus the stored moving values (so the stored sum is s_in);
// a rest outside the int32 range sets bad.
// A store that marks its line evict-first in the caches (the bulk sweep's
// output is read again only next step, after the band kernels): 1 under
// FSLBM_BULK_STCS, else a plain store.
#ifndef FSLBM_BULK_STCS
#define FSLBM_BULK_STCS 0
#endif
template <bool kStream, class T>
__device__ __forceinline__ void st_pdf(T* p, T v) {
  if constexpr (kStream && FSLBM_BULK_STCS != 0) {
    if constexpr (sizeof(T) == 4) __stcs(reinterpret_cast<unsigned int*>(p), *reinterpret_cast<unsigned int*>(&v));
    else if constexpr (sizeof(T) == 2) __stcs(reinterpret_cast<unsigned short*>(p), *reinterpret_cast<unsigned short*>(&v));
    else __stcs(reinterpret_cast<unsigned long long*>(p), *reinterpret_cast<unsigned long long*>(&v));
  } else {
    *p = v;
  }
}

template <int Q, class S, bool kStream = false>
__device__ __forceinline__ void store_cell(typename S::T* B, long long Np, long long c,
                                           const typename S::Real* f, long long s_in, bool& bad) {
  if constexpr (S::kExactRest) {
    constexpr float kRange = 2147483648.0f / (float)(1LL << S::kShift);  // |d| bound of the grid
    long long s_out = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      if (!(fabsf(f[i]) < kRange)) bad = true;
      const typename S::T v = S::stored(f[i]);
      st_pdf<kStream>(&B[(long long)i * Np + c], v);
      s_out += S::steps(v);
    }
    long long r = s_in - s_out;
    if (r > 2147483647LL || r < -2147483647LL) {
      bad = true;
      r = r > 0 ? 2147483647LL : -2147483647LL;
    }
    st_pdf<kStream>(&rest_slice<Q, S>(B, Np)[c], (int)r);
  } else {
    (void)s_in;
    (void)bad;
#pragma unroll
    for (int i = 0; i < Q; ++i) st_pdf<kStream>(&B[(long long)i * Np + c], store_w<S, Q>(f[i], i));
  }
}

// PDF i of storage cell c of buffer P in the working representation (the
// rest PDF of the mass-conserving formats from its grid steps).
template <int Q, class S>
__device__ __forceinline__ typename S::Real load_own(const typename S::T* P, long long Np, long long c,
                                                     int i) {
  if constexpr (S::kExactRest) {
    if (i == 0) return from_steps<S>(rest_slice<Q, S>(P, Np)[c]);
  }
  return load_w<S, Q>(P[(long long)i * Np + c], i);
}

// Sum of the stored PDFs (deviations) of storage cell c: FP64 for the
// deviation formats, exact from the grid steps for the mass-conserving ones.
template <int Q, class S>
__device__ __forceinline__ double stored_sum(const typename S::T* P, long long Np, long long c,
                                             const typename S::Real* f) {
  if constexpr (S::kExactRest) {
    long long n = rest_slice<Q, S>(P, Np)[c];
#pragma unroll
    for (int i = 1; i < Q; ++i) n += S::steps(P[(long long)i * Np + c]);
    return (double)n * (1.0 / (double)(1LL << S::kShift));
  } else {
    double sd = 0.0;
#pragma unroll
    for (int i = 0; i < Q; ++i) sd += (double)f[i];
    return sd;
  }
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
    const double sd = stored_sum<Q, S>(P, Np, c, f);
    rho = 1.0 + sd;
    rr = R(rho);
  } else {
    rho = r;
  }
  u[0] = jx / rr - R(0.5) * gpar<R>(p, 0);
  u[1] = jy / rr - R(0.5) * gpar<R>(p, 1);
  u[2] = jz / rr - R(0.5) * gpar<R>(p, 2);
}

// ------------------------------------------------- bounce-back via obstacle slots
// Pull source of direction i of the cell at (x, y, z) (Eq. nm-lbm-streaming):
// the cell x - c_i, wrapped across periodic faces, whose PDF i arrives
// (j = i).  Across a free-slip face the source is the mirror image: the
// coordinate along that axis stays the cell's own and the arriving PDF is
// the one with that component of c_i reversed (the specular reflection of
// Sec. 2.1).  Returns the source's storage index, or -1 across a no-slip
// face (bounce-back).  mirrored: the source was reflected at a wall.
template <int Q>
__device__ __forceinline__ int pull_source(const KParams& p, int x, int y, int z, int i, int& j,
                                           bool& mirrored) {
  int X = x - CX(i), Y = y - CY(i), Z = z - CZ(i);
  int m = 0;
  bool out = false;
  if (X < 0 || X >= p.nx) {
    if (p.per[0]) X = X < 0 ? X + p.nx : X - p.nx;
    else if (p.slip[0]) X = x, m |= 1;
    else out = true;
  }
  if (Y < 0 || Y >= p.ny) {
    if (p.per[1]) Y = Y < 0 ? Y + p.ny : Y - p.ny;
    else if (p.slip[1]) Y = y, m |= 2;
    else out = true;
  }
  if (Z < 0 || Z >= p.nz) {
    if (p.per[2]) Z = Z < 0 ? Z + p.nz : Z - p.nz;
    else if (p.slip[2]) Z = z, m |= 4;
    else out = true;
  }
  j = m ? (int)kReflect.j[i][m] : i;
  mirrored = m != 0;
  return out ? -1 : cidx(p, X, Y, Z);
}

// Index (slice and cell) of the value a liquid cell c at (x, y, z) pulls in
// direction i: its source's PDF (wrapped across periodic faces; with SLIP,
// reflected at free-slip faces), or its own PDF ibar (bounce-back) when the
// source lies across a no-slip face or the mirror image across a free-slip
// face is an obstacle cell.  Without SLIP the free-slip logic is not
// compiled (domains without free-slip faces).
template <int Q, bool SLIP>
__device__ __forceinline__ long long pull_index_general(const KParams& p, const uint8_t* flags, int c,
                                                        int x, int y, int z, int i) {
  if constexpr (SLIP) {
    int j;
    bool mir;
    const int s = pull_source<Q>(p, x, y, z, i, j, mir);
    if (s < 0 || (mir && (flags[s] & F_TYPE) == T_OBST)) return (long long)OPP(i) * p.Np + c;
    return (long long)j * p.Np + s;
  } else {
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
}

// Slot of the obstacle pull source x - c_i (inside the domain or across a
// periodic face) that a fluid cell's reflected copy goes to.
template <int Q>
__device__ __forceinline__ long long obstacle_slot(const KParams& p, int x, int y, int z, int i) {
  const int X = wrapc(x - CX(i), p.nx, p.per[0]);
  const int Y = wrapc(y - CY(i), p.ny, p.per[1]);
  const int Z = wrapc(z - CZ(i), p.nz, p.per[2]);
  return (long long)i * p.Np + cidx(p, X, Y, Z);
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
    const long long idx = general ? obstacle_slot<Q>(p, x, y, z, i) : p.dofs[i] + c;
    B[idx] = store_w<S, Q>(f[OPP(i)], i);
  }
}

}  // namespace fslbm
