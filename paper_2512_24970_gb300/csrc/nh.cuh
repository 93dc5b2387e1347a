// Device side of the Nose-Hoover chain thermostat (see k_nh.cu): the chain's
// half step, the opening half step every k_prepare block runs, and the
// fixed-order block sum of m v^2.  Included by the translation units whose
// kernels use them.
#pragma once

#include "rbsog_internal.cuh"

namespace rb {

__device__ __forceinline__ double nh_G(const View &p, const double *v, int j, double k2) {
  if (j == 0) return (k2 - p.nh_g * p.nh_kT) / p.nh_Q[0];
  return (p.nh_Q[j - 1] * v[j - 1] * v[j - 1] - p.nh_kT) / p.nh_Q[j];
}

__device__ __forceinline__ void nh_kick(const View &p, double *v, int j, double k2, double d) {
  if (j + 1 < p.nh_M) {
    const double x = exp(-0.25 * d * v[j + 1]);
    v[j] = (v[j] * x + 0.5 * d * nh_G(p, v, j, k2)) * x;
  } else {
    v[j] += 0.5 * d * nh_G(p, v, j, k2);
  }
}

// One half step (length dt/2) of the chain (eta, v) for twice the kinetic
// energy k2 [eV]; returns the velocity scale and leaves k2 * s^2 in k2.
__device__ __forceinline__ double nh_half_step(const View &p, double *eta, double *v, double &k2) {
  const double d = 0.5 * p.dt;
  for (int j = p.nh_M - 1; j >= 0; j--) nh_kick(p, v, j, k2, d);
  const double s = exp(-d * v[0]);
  k2 *= s * s;
  for (int j = 0; j < p.nh_M; j++) eta[j] += d * v[j];
  for (int j = 0; j < p.nh_M; j++) nh_kick(p, v, j, k2, d);
  return s;
}

// Fixed-order block sum of one value per thread (blockDim.x a multiple of 32,
// at most 1024); the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double x) {
  __shared__ double ws[32];
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = x;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += ws[w];
  return t;
}

__device__ __forceinline__ double mv2(const View &p, int64_t i) {
  if (i >= p.n) return 0.0;
  const int64_t n = p.n;
  const double vx = p.v[i], vy = p.v[n + i], vz = p.v[2 * n + i];
  return p.massv[p.spc[i]] * (vx * vx + vy * vy + vz * vz);
}

// sum of the ke_part partials in fixed order, in eV (twice the kinetic
// energy); valid in thread 0
__device__ __forceinline__ double ke2_total(const View &p) {
  double x = 0.0;
  for (int b = threadIdx.x; b < p.nh_nblk; b += blockDim.x) x += p.ke_part[b];
  return block_sum(x) / FCONV;
}

// The opening half step from the A copy and 2K of the current velocities
// (the partials of m v^2 the previous step's closing scale, or the priming,
// left); block 0 stores the result as B.
__device__ __forceinline__ double nh_open(const View &p) {
  __shared__ double s_open;
  double k2 = ke2_total(p);
  if (threadIdx.x == 0) {
    double eta[RBSOG_MAX_NH_CHAIN], v[RBSOG_MAX_NH_CHAIN];
    for (int j = 0; j < p.nh_M; j++) {
      eta[j] = p.nh[NH_A_ETA + j];
      v[j] = p.nh[NH_A_V + j];
    }
    const double s = nh_half_step(p, eta, v, k2);
    if (blockIdx.x == 0) {
      for (int j = 0; j < p.nh_M; j++) {
        p.nh[NH_B_ETA + j] = eta[j];
        p.nh[NH_B_V + j] = v[j];
      }
    }
    s_open = s;
  }
  __syncthreads();
  return s_open;
}

}  // namespace rb
