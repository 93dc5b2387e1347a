// Structure factor of caller-given modes whose only scratch is a static
// device array (the allocation-free entry point rbsog_structure_factor_static):
//   k_sf_static      per (tile, k): FP64 partial sum_j q_j e^{i k.r_j} over the
//                    tile's atoms, phase from the exact integer m.u (Sec. 2.2,
//                    rho(k) of Eq. (Long)); one thread per k.
//   k_sf_static_sum  one warp per k: fixed-order sum of the tile partials.
// Every partial the second kernel reads is written by the first in the same
// call, so nothing in the scratch has to start at zero.
#include <mutex>

#include "rbsog_internal.cuh"

namespace rb {

static_assert(SF_STATIC_PMAX == RBSOG_SF_STATIC_PMAX, "static scratch size and the ABI limit differ");

static __device__ __align__(256) double2 g_sf_part[SF_STATIC_PMAX * SF_STATIC_TILES];

__global__ void __launch_bounds__(256) k_sf_static(View p, int P, const int *__restrict__ m, int ntile,
                                                   int tile_atoms, double2 *__restrict__ part) {
  __shared__ uint4 sa[256];
  __shared__ double sq[256];
  const int tid = threadIdx.x;
  const int tile = blockIdx.x;
  const int k = blockIdx.y * 256 + tid;
  uint32_t mx = 0u, my = 0u, mz = 0u;
  if (k < P) {
    mx = (uint32_t)m[3 * k];
    my = (uint32_t)m[3 * k + 1];
    mz = (uint32_t)m[3 * k + 2];
  }
  const int64_t n = p.n;
  const int64_t a0 = (int64_t)tile * tile_atoms;
  const int64_t a1 = min(a0 + (int64_t)tile_atoms, n);
  double re = 0.0, im = 0.0;
  for (int64_t base = a0; base < a1; base += 256) {
    const int cnt = (int)min((int64_t)256, a1 - base);
    __syncthreads();
    if (tid < cnt) {
      const int64_t a = base + tid;
      sa[tid] = make_uint4(fixed_point(p.x[a], p.invL[0]), fixed_point(p.x[n + a], p.invL[1]),
                           fixed_point(p.x[2 * n + a], p.invL[2]), 0u);
      sq[tid] = p.qs[p.spc[a]];
    }
    __syncthreads();
    for (int j = 0; j < cnt; j++) {
      const uint4 u = sa[j];
      const uint32_t th = mx * u.x + my * u.y + mz * u.z;  // mod 2^32 = one turn
      double s, c;
      sincospi((double)(int)th * 4.656612873077393e-10, &s, &c);  // * 2^-31
      re += sq[j] * c;
      im += sq[j] * s;
    }
  }
  if (k < P) part[(int64_t)k * ntile + tile] = make_double2(re, im);
}

__global__ void __launch_bounds__(256) k_sf_static_sum(int P, int ntile, const double2 *__restrict__ part,
                                                       double *__restrict__ rho) {
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (k >= P) return;
  double re = 0.0, im = 0.0;
  for (int t = lane; t < ntile; t += 32) {
    const double2 d = part[(int64_t)k * ntile + t];
    re += d.x;
    im += d.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, o);
    im += __shfl_down_sync(0xffffffffu, im, o);
  }
  if (lane == 0) {
    rho[2 * k] = re;
    rho[2 * k + 1] = im;
  }
}

// Device address of g_sf_part, looked up once per device (the device must be
// current) and cached; the lookup may load this module, so the first call on
// a device must not be inside stream capture.  A cudaDeviceReset invalidates
// the cached address together with every context of the device.
cudaError_t sf_static_scratch(int dev, void **out) {
  static std::mutex mu;
  static void *addr[SF_STATIC_MAX_DEVICES] = {};
  if (dev < 0 || dev >= SF_STATIC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void *a = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&a, g_sf_part);
    if (e != cudaSuccess) return e;
    addr[dev] = a;
  }
  *out = addr[dev];
  return cudaSuccess;
}

void launch_sf_static(const View &v, int P, const int *m, double *rho, void *scratch, cudaStream_t st) {
  int ntile = (int)std::min<int64_t>(SF_STATIC_TILES, (v.n + 255) / 256);
  ntile = std::max(ntile, 1);
  const int tile_atoms = (int)((v.n + ntile - 1) / ntile);
  ntile = (int)((v.n + tile_atoms - 1) / tile_atoms);
  double2 *part = (double2 *)scratch;
  k_sf_static<<<dim3(ntile, (P + 255) / 256), 256, 0, st>>>(v, P, m, ntile, tile_atoms, part);
  k_sf_static_sum<<<(P + 7) / 8, 256, 0, st>>>(P, ntile, part, rho);
}

}  // namespace rb
