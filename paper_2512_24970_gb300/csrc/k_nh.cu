// Nose-Hoover chain thermostat of the NVT runs (Sec. 3; chain and splitting
// after Martyna, Tuckerman and Klein, Mol. Phys. 87 (1996) 1117): a half step
// of the chain before the first half kick and after the second.
//   chain     masses Q_0 = g kT tau^2, Q_j = kT tau^2, g = 3N - 3; forces
//             G_0 = (2K - g kT)/Q_0, G_j = (Q_{j-1} v_{j-1}^2 - kT)/Q_j.  A half
//             step of length d = dt/2: v_j from the chain's end down to v_0,
//             each damped by e^{-d v_{j+1}/4} before and after its kick d G_j/2;
//             the velocity scale s = e^{-d v_0}; eta_j += d v_j; then v_0 up to
//             the chain's end again with 2K scaled by s^2.
//   state     nh[NH_A...]: the chain between steps (after the closing half
//             step); nh[NH_B...]: after the opening half step, written by block
//             0 of k_prepare.  Every k_prepare block runs the opening half step
//             itself from the A copy and the m v^2 partials (same inputs, same
//             result), so it needs no kernel of its own.
//   k_ke_part sum_i m_i v_i^2 per block (for velocities set from outside;
//             k_finish and k_nh_scale write the same partials within a step);
//   k_nh_close one block: the partials in fixed order, the closing half step
//             (B -> A) and its velocity scale; k_nh_scale applies that scale.
//   k_kin_part / k_kin_sum  the kinetic tensor K_ab = sum_i m_i v_ia v_ib of
//             the current velocities (block sums, then one block in block
//             order), the velocity half of the stress S = K + W whose xy
//             component is the Green-Kubo shear stress of Sec. 3.
#include "nh.cuh"

namespace rb {

__global__ void __launch_bounds__(PREP_BLOCK) k_ke_part(View p) {
  const double t = block_sum(mv2(p, (int64_t)blockIdx.x * blockDim.x + threadIdx.x));
  if (threadIdx.x == 0) p.ke_part[blockIdx.x] = t;
}

// The closing half step of a step (B -> A) from the m v^2 partials k_finish
// left; its velocity scale goes to NH_S_CLOSE.
__global__ void __launch_bounds__(256) k_nh_close(View p) {
  double k2 = ke2_total(p);
  if (threadIdx.x != 0) return;
  double eta[RBSOG_MAX_NH_CHAIN], v[RBSOG_MAX_NH_CHAIN];
  for (int j = 0; j < p.nh_M; j++) {
    eta[j] = p.nh[NH_B_ETA + j];
    v[j] = p.nh[NH_B_V + j];
  }
  const double s = nh_half_step(p, eta, v, k2);
  for (int j = 0; j < p.nh_M; j++) {
    p.nh[NH_A_ETA + j] = eta[j];
    p.nh[NH_A_V + j] = v[j];
  }
  p.nh[NH_S_CLOSE] = s;
}

// Scale the velocities by the closing factor and leave the partials of m v^2
// of the scaled velocities for the next step's opening half step (the same
// partials k_ke_part writes for velocities set from outside).
__global__ void __launch_bounds__(PREP_BLOCK) k_nh_scale(View p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < p.n) {
    const double s = p.nh[NH_S_CLOSE];
    for (int a = 0; a < 3; a++) p.v[a * p.n + i] *= s;
  }
  const double t = block_sum(mv2(p, i));
  if (threadIdx.x == 0) p.ke_part[blockIdx.x] = t;
}

// (xx, yy, zz, xy, xz, yz), the order of the virial
__global__ void __launch_bounds__(PREP_BLOCK) k_kin_part(View p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double t[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (i < p.n) {
    const int64_t n = p.n;
    const double m = p.massv[p.spc[i]];
    const double vx = p.v[i], vy = p.v[n + i], vz = p.v[2 * n + i];
    t[0] = m * vx * vx; t[1] = m * vy * vy; t[2] = m * vz * vz;
    t[3] = m * vx * vy; t[4] = m * vx * vz; t[5] = m * vy * vz;
  }
  for (int c = 0; c < 6; c++) {
    const double b = block_sum(t[c]);
    if (threadIdx.x == 0) p.kin_part[6 * (int64_t)blockIdx.x + c] = b;
    __syncthreads();                              // block_sum's scratch is reused
  }
}

__global__ void __launch_bounds__(256) k_kin_sum(View p) {
  for (int c = 0; c < 6; c++) {
    double x = 0.0;
    for (int b = threadIdx.x; b < p.nh_nblk; b += blockDim.x) x += p.kin_part[6 * (int64_t)b + c];
    const double t = block_sum(x);
    if (threadIdx.x == 0) p.kin[c] = t / FCONV;   // amu A^2/ps^2 -> eV
    __syncthreads();
  }
}

void launch_kinetic_tensor(const View &v, cudaStream_t st) {
  k_kin_part<<<(unsigned)v.nh_nblk, PREP_BLOCK, 0, st>>>(v);
  k_kin_sum<<<1, 256, 0, st>>>(v);
}

void launch_nh_close(const View &v, cudaStream_t st) {
  k_nh_close<<<1, 256, 0, st>>>(v);
  k_nh_scale<<<(unsigned)v.nh_nblk, PREP_BLOCK, 0, st>>>(v);
}

void launch_nh_prime(const View &v, cudaStream_t st) {
  k_ke_part<<<(unsigned)v.nh_nblk, PREP_BLOCK, 0, st>>>(v);
}

}  // namespace rb
