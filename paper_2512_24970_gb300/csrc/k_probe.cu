// Throughput probes behind the rooflines of the measurement (rbsog_probe_peak):
// every thread runs PROBE_CHAINS independent multiply-add chains for `iters`
// iterations, so the pipe under test is the only limit; the chains' values
// are summed into `out` so that nothing is eliminated.  One launch of
// PROBE_BLOCKS_PER_SM blocks per SM is timed with CUDA events after one
// warm-up launch.
#include <cuda_runtime.h>

#include "rbsog_internal.cuh"

namespace rb {

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_BLOCK = 512;
constexpr int PROBE_BLOCKS_PER_SM = 4;

__global__ void __launch_bounds__(PROBE_BLOCK) k_probe_f32(float *out, int iters, float a, float b) {
  float x[PROBE_CHAINS];
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; j++) x[j] = (float)(threadIdx.x + j);
  for (int it = 0; it < iters; it++)
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; j++) x[j] = __fmaf_rn(x[j], a, b);
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; j++) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_BLOCK) k_probe_f32x2(float *out, int iters, float a, float b) {
  unsigned long long x[PROBE_CHAINS];
  const unsigned long long a2 = pk2(a, a), b2 = pk2(b, b);
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; j++) x[j] = pk2((float)(threadIdx.x + j), (float)(threadIdx.x - j));
  for (int it = 0; it < iters; it++)
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; j++) x[j] = fma2(x[j], a2, b2);
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; j++) {
    float u, v;
    up2(x[j], u, v);
    s += u + v;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_BLOCK) k_probe_f64(float *out, int iters, double a, double b) {
  double x[PROBE_CHAINS];
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; j++) x[j] = (double)(threadIdx.x + j);
  for (int it = 0; it < iters; it++)
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; j++) x[j] = __fma_rn(x[j], a, b);
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; j++) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

__global__ void __launch_bounds__(PROBE_BLOCK) k_probe_imad(float *out, int iters, uint32_t a, uint32_t b) {
  uint32_t x[PROBE_CHAINS];
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; j++) x[j] = threadIdx.x * 2654435761u + j;
  for (int it = 0; it < iters; it++)
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; j++) x[j] = x[j] * a + b;
  uint32_t s = 0u;
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; j++) s ^= x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

// lane operations (one multiply-add each, two per FP32x2 lane pair) per second
cudaError_t probe_peak(int dev, int kind, double *ops) {
  cudaError_t e = cudaSetDevice(dev);
  int nsm = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int nblk = PROBE_BLOCKS_PER_SM * nsm;
  const int iters = kind == RBSOG_PROBE_FP64 ? 2048 : 16384;
  float *out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&out, sizeof(float) * (size_t)nblk * PROBE_BLOCK);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.0f;
  for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {   // warm-up, then timed
    cudaEventRecord(e0, st);
    switch (kind) {
      case RBSOG_PROBE_FP32: k_probe_f32<<<nblk, PROBE_BLOCK, 0, st>>>(out, iters, 0.999f, 1e-3f); break;
      case RBSOG_PROBE_FP32X2: k_probe_f32x2<<<nblk, PROBE_BLOCK, 0, st>>>(out, iters, 0.999f, 1e-3f); break;
      case RBSOG_PROBE_FP64: k_probe_f64<<<nblk, PROBE_BLOCK, 0, st>>>(out, iters, 0.999, 1e-3); break;
      default: k_probe_imad<<<nblk, PROBE_BLOCK, 0, st>>>(out, iters, 2654435761u, 12345u); break;
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e == cudaSuccess) {
    const double lanes = (double)nblk * PROBE_BLOCK * (kind == RBSOG_PROBE_FP32X2 ? 2.0 : 1.0);
    *ops = lanes * PROBE_CHAINS * (double)iters / (1e-3 * (double)ms);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (out) cudaFree(out);
  return e;
}

}  // namespace rb

extern "C" int rbsog_probe_peak(int cuda_device, int kind, double *ops_per_s) {
  if (!ops_per_s || kind < RBSOG_PROBE_FP32 || kind > RBSOG_PROBE_IMAD) return RBSOG_E_INVAL;
  return rb::probe_peak(cuda_device, kind, ops_per_s) == cudaSuccess ? RBSOG_OK : RBSOG_E_CUDA;
}
