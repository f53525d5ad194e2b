// Seed-fill front detection (Sec. 4.3, cylindrical dam break: the liquid
// front's radius is taken over the interface cells that a seed fill started
// at a domain boundary reaches, so that only the outermost interface cells
// count).  The fill runs in one z-layer through the cells that are gas or
// obstacle, over in-plane face neighbours (across periodic faces too),
// seeded with every such cell on the layer's edge; a front cell is an
// interface cell of the layer with a reached gas cell among its in-plane
// face neighbours.  On the device the fill is a connected-component
// labelling of the layer's gas-or-obstacle cells (union-find, the same
// lock-free hooking as the bubble labels) followed by marking the
// components that hold an edge cell.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "fslbm_cell.cuh"
#include "fslbm_ctx.h"

using namespace fslbm;

namespace {

constexpr int kFrontBlock = 256;

__device__ __forceinline__ bool outside_cell(uint8_t t) { return t == T_GAS || t == T_OBST; }

// Layer index m = x + nx y of the in-plane neighbour k (+x, -x, +y, -y) of
// (x, y), or -1 across a non-periodic edge.
__device__ __forceinline__ int layer_nbr(const KParams& p, int x, int y, int k) {
  const int X = wrapc(x + (k == 0) - (k == 1), p.nx, p.per[0]);
  const int Y = wrapc(y + (k == 2) - (k == 3), p.ny, p.per[1]);
  return (X < 0 || Y < 0) ? -1 : X + p.nx * Y;
}

__device__ __forceinline__ int front_find(const int* lab, int x) {
  int q = lab[x];
  while (q != x) {
    x = q;
    q = lab[x];
  }
  return x;
}

__global__ void k_front_init(KParams p, const uint8_t* __restrict__ flags, int layer, int* lab,
                             uint8_t* seeded, uint8_t* type) {
  const int M = p.nx * p.ny;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const uint8_t t = flags[cidx(p, m % p.nx, m / p.nx, layer)] & F_TYPE;
  type[m] = t;
  lab[m] = outside_cell(t) ? m : -1;
  seeded[m] = 0;
}

// Each pair of face neighbours once (+x and +y); the root with the larger
// index is hooked under the other with compare-and-swap.
__global__ void k_front_union(KParams p, const uint8_t* __restrict__ type, int* lab) {
  const int M = p.nx * p.ny;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M || !outside_cell(type[m])) return;
  const int x = m % p.nx, y = m / p.nx;
  for (int k = 0; k < 4; k += 2) {
    const int n = layer_nbr(p, x, y, k);
    if (n < 0 || n == m || !outside_cell(type[n])) continue;
    int a = front_find(lab, m), b = front_find(lab, n);
    while (a != b) {
      if (a > b) {
        const int t = a;
        a = b;
        b = t;
      }
      const int old = atomicCAS(&lab[b], b, a);
      if (old == b) break;
      b = front_find(lab, old);
      a = front_find(lab, a);
    }
  }
}

__global__ void k_front_seed(KParams p, const uint8_t* __restrict__ type, int* lab, uint8_t* seeded) {
  const int M = p.nx * p.ny;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M || !outside_cell(type[m])) return;
  const int r = front_find(lab, m);
  lab[m] = r;
  const int x = m % p.nx, y = m / p.nx;
  if (x == 0 || x == p.nx - 1 || y == 0 || y == p.ny - 1) seeded[r] = 1;
}

// acc: [0] count, [1] minimum radius bits, [2] maximum radius bits (radii
// are non-negative, so their bit patterns order like the values), [3] sum
// of the radii (FP64).
__global__ void k_front_mark(KParams p, const uint8_t* __restrict__ type, const int* __restrict__ lab,
                             const uint8_t* __restrict__ seeded, double xc, double yc, uint8_t* front,
                             unsigned long long* acc) {
  const int M = p.nx * p.ny;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  bool hit = false;
  const int x = m % p.nx, y = m / p.nx;
  if (type[m] == T_IFACE) {
    for (int k = 0; k < 4; ++k) {
      const int n = layer_nbr(p, x, y, k);
      if (n >= 0 && type[n] == T_GAS && seeded[lab[n]]) hit = true;
    }
  }
  front[m] = hit ? 1 : 0;
  if (!hit) return;
  const double dx = __dsub_rn((double)x + 0.5, xc), dy = __dsub_rn((double)y + 0.5, yc);
  const double r = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
  const unsigned long long bits = (unsigned long long)__double_as_longlong(r);
  atomicAdd(&acc[0], 1ull);
  atomicMin(&acc[1], bits);
  atomicMax(&acc[2], bits);
  atomicAdd((double*)&acc[3], r);
}

}  // namespace

extern "C" fslbm_status fslbm_front(fslbm_ctx* c, int layer, double xc, double yc, fslbm_front_stats* out,
                                    uint8_t* front_mask) {
  if (!c || !out) return FSLBM_EINVAL;
  if (!c->initialized) return fail(c, FSLBM_ESTATE, "front before init");
  if (layer < 0 || layer >= c->kp.nz || !std::isfinite(xc) || !std::isfinite(yc))
    return fail(c, FSLBM_EINVAL, "front: layer outside the domain or centre not finite");
  const KParams& p = c->kp;
  const size_t M = (size_t)p.nx * (size_t)p.ny;
  cudaStream_t st = c->stream;
  void* buf = nullptr;
  const size_t bytes = 4 * sizeof(unsigned long long) + M * sizeof(int) + 3 * M;
  cudaError_t e = cudaMallocAsync(&buf, bytes, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "fslbm_front");
  unsigned long long* acc = (unsigned long long*)buf;
  int* lab = (int*)(acc + 4);
  uint8_t* seeded = (uint8_t*)(lab + M);
  uint8_t* type = seeded + M;
  uint8_t* front = type + M;
  const unsigned long long init[4] = {0ull, 0x7ff0000000000000ull, 0ull, 0ull};
  e = cudaMemcpyAsync(acc, init, sizeof(init), cudaMemcpyHostToDevice, st);
  const int grid = (int)((M + kFrontBlock - 1) / kFrontBlock);
  if (e == cudaSuccess) {
    k_front_init<<<grid, kFrontBlock, 0, st>>>(p, c->d.flags, layer, lab, seeded, type);
    k_front_union<<<grid, kFrontBlock, 0, st>>>(p, type, lab);
    k_front_seed<<<grid, kFrontBlock, 0, st>>>(p, type, lab, seeded);
    k_front_mark<<<grid, kFrontBlock, 0, st>>>(p, type, lab, seeded, xc, yc, front, acc);
    e = cudaGetLastError();
  }
  unsigned long long h[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && front_mask) e = cudaMemcpyAsync(front_mask, front, M, cudaMemcpyDeviceToHost, st);
  const cudaError_t ef = cudaFreeAsync(buf, st);
  if (e == cudaSuccess) e = ef;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(c, e, "fslbm_front");
  std::memset(out, 0, sizeof(*out));
  out->count = (int64_t)h[0];
  if (h[0] > 0) {
    double v;
    std::memcpy(&v, &h[1], sizeof(v));
    out->r_min = v;
    std::memcpy(&v, &h[2], sizeof(v));
    out->r_max = v;
    std::memcpy(&v, &h[3], sizeof(v));
    out->r_mean = v / (double)h[0];
  }
  return FSLBM_OK;
}
