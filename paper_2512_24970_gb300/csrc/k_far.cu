// Stage (d) far field and stage (e) second half (Sec. 2.2, Eq. (long-rangeforce)):
//   k_rho_*   structure-factor partials rho(k_p) = sum_j q_j e^{i k_p . r_j} over
//             an atom tile, phase k . r = 2 pi (m . u mod 2^32) / 2^32 reduced
//             exactly in uint32; FP32 polynomial sincos with FP32 accumulation
//             over at most 256 atoms, then FP64 (mixed), or FP64 sincospi (FP64).
//   k_reduce  fixed-order FP64 sum over tiles (one block per k), the per-k
//             force records: c_p Im rho_p, c_p Re rho_p (FP64), or arg rho_p as
//             an exact 32-bit turn and c_p |rho_p| k_p (mixed).
//   k_corr    F^corr and U_N (and in energy evaluations the pair virial) from
//             the near-field warp partials, fixed order.
//   k_farforce_* F_F,i = -(k_e q_i / V) sum_p c_p k_p Im(e^{-i k_p.r_i} rho_p).
//   k_finish  F_i = F_N,i - F^corr + F_F,i and the closing half kick of the MD step.
#include <algorithm>

#include "nh.cuh"

namespace rb {

constexpr double TWO_PI = 6.283185307179586;

// Mixed phase e^{i 2 pi th / 2^32}: FP32 polynomial with exact half-turn
// reduction (sincos_turn).
__device__ __forceinline__ void sincos_phase_f(uint32_t th, float &s, float &c) { sincos_turn(th, s, c); }
__device__ __forceinline__ void sincos_phase_d(uint32_t th, double &s, double &c) {
  sincospi((double)(int)th * 4.656612873077393e-10, &s, &c);  // * 2^-31
}

// FP64 structure factor: one block per (tile, 512 modes), two modes per
// thread, FP64 sincospi of the exact phase and FP64 sums.
__global__ void __launch_bounds__(RHO_BLOCK) k_rho_fp64(View p) {
  __shared__ uint4 sa[256];
  __shared__ double sq[256];
  const int tid = threadIdx.x;
  const int tile = blockIdx.x;
  const int64_t a0 = (int64_t)tile * p.tile_atoms;
  const int64_t a1 = min(a0 + (int64_t)p.tile_atoms, p.n);
  uint32_t mx[RHO_KPT], my[RHO_KPT], mz[RHO_KPT];
  int kk[RHO_KPT];
#pragma unroll
  for (int t = 0; t < RHO_KPT; t++) {
    kk[t] = blockIdx.y * (RHO_BLOCK * RHO_KPT) + t * RHO_BLOCK + tid;
    const int4 m = kk[t] < p.P ? p.km[kk[t]] : make_int4(0, 0, 0, 0);
    mx[t] = (uint32_t)m.x; my[t] = (uint32_t)m.y; mz[t] = (uint32_t)m.z;
  }
  double re[RHO_KPT], im[RHO_KPT];
#pragma unroll
  for (int t = 0; t < RHO_KPT; t++) re[t] = im[t] = 0.0;
  for (int64_t base = a0; base < a1; base += 256) {
    const int cnt = (int)min((int64_t)256, a1 - base);
    __syncthreads();
    if (tid < cnt) {
      const uint4 u = p.ua[base + tid];
      sa[tid] = u;
      sq[tid] = p.qs[u.w];
    }
    __syncthreads();
    for (int a = 0; a < cnt; a++) {
      const uint4 u = sa[a];
      const double q = sq[a];
#pragma unroll
      for (int t = 0; t < RHO_KPT; t++) {
        const uint32_t th = mx[t] * u.x + my[t] * u.y + mz[t] * u.z;
        double s, c;
        sincos_phase_d(th, s, c);
        re[t] += q * c;
        im[t] += q * s;
      }
    }
  }
#pragma unroll
  for (int t = 0; t < RHO_KPT; t++) {
    if (kk[t] < p.P) {
      double *d = p.rho_part + 2 * ((int64_t)kk[t] * p.ntile + tile);
      d[0] = re[t];
      d[1] = im[t];
    }
  }
}

// Mixed structure factor.  A block holds G groups of GT = 256 / NP threads;
// thread t of every group takes the NP pairs of modes 2 NP t ... 2 NP t +
// 2 NP - 1 of the block's 512 (one packed FP32x2 lane per mode), group g the
// g-th share of the tile's atoms.  Per (atom, mode): the exact phase
// th = m.u mod 2^32 with the half-turn offset 2^30 folded into its
// multiply-add chain, phi and the half-turn bit from it (half_turn_2r), the
// minimax sine (packed) and cosine (per lane, so that the FMA pipe's two
// halves share the work with the integer multiply-adds, which run on one of
// them), the half-turn sign on the charge, and FP32 sums over at most
// RHO_FLUSH atoms, added in FP64.  The groups' FP64 sums are added in group
// order in shared memory: one partial per (mode, tile).  MINB is the
// occupancy the register allocation is bounded for.  PK = false evaluates the
// same operations per lane in scalar FP32 instructions (bit for bit the same
// results; it leaves the FMA pipe's two halves to be filled independently).
constexpr int RHO_MCHUNK = 256;                  // atoms staged in shared memory per group and round
// FP32 partial sums run over at most RHO_FLUSH atoms before they are added
// exactly (TwoSum into an FP32 pair): on lattice-like configurations the sums
// over one sublattice are coherent (of order the number of atoms) while rho
// is small, so the FP32 rounding of a partial sum grows with its length; 64
// atoms keep it near 64 * 2^-24 of the largest partial.  (FP64 adds of the
// partials cost the FP64 pipe, which is narrow on this part.)
constexpr int RHO_FLUSH = 64;
constexpr int RHO_WARP_TILES = 160;  // tiles up to which the tile sums take a warp per mode
constexpr int RHO_KTILE = RHO_BLOCK * RHO_KPT;    // modes per block row (512)
template <int NP, int G, int MINB, int PK>
__device__ __forceinline__ void rho_mixed_body(const View &p, int bid) {
  constexpr int GT = RHO_BLOCK / NP;
  __shared__ uint4 sa[G][RHO_MCHUNK];
  __shared__ double2 sg[G > 1 ? G - 1 : 1][RHO_KTILE];
  static_assert(RHO_KPT == 2 && GT * NP * 2 == RHO_KTILE, "packed pairs of modes per thread");
  const int tid = threadIdx.x, grp = tid / GT, gt = tid % GT;
  const int tile = bid % p.ntile;                // blocks: tiles fastest, then columns of modes
  const int kb = (bid / p.ntile) * RHO_KTILE + 2 * NP * gt;
  const int64_t a0 = (int64_t)tile * p.tile_atoms;
  const int64_t a1 = min(a0 + (int64_t)p.tile_atoms, p.n);
  const int sub = (p.tile_atoms + G - 1) / G;
  const int64_t g0 = min(a0 + (int64_t)grp * sub, a1), g1 = min(g0 + sub, a1);
  int4 m[2 * NP];
#pragma unroll
  for (int t = 0; t < 2 * NP; t++) m[t] = kb + t < p.P ? p.km[kb + t] : make_int4(0, 0, 0, 0);
  // the flushed partials' sums as unevaluated FP32 pairs hi + lo per mode
  // (Knuth's TwoSum: hi + lo is the exact sum of the flushed partials up to
  // the rounding of lo), two modes per packed register
  unsigned long long shr[NP], slr[NP], shi[NP], sli[NP];
#pragma unroll
  for (int q = 0; q < NP; q++) shr[q] = slr[q] = shi[q] = sli[q] = 0ull;
  const int nch = (sub + RHO_MCHUNK - 1) / RHO_MCHUNK;   // the same for every group
  for (int c = 0; c < nch; c++) {
    const int64_t base = g0 + (int64_t)c * RHO_MCHUNK;
    const int cnt = (int)max((int64_t)0, min((int64_t)RHO_MCHUNK, g1 - base));
    __syncthreads();
    for (int e = gt; e < cnt; e += GT) {
      uint4 u = p.ua[base + e];
      u.w = __float_as_uint((float)p.qs[u.w]);
      sa[grp][e] = u;
    }
    __syncthreads();
    for (int a0 = 0; a0 < cnt; a0 += RHO_FLUSH) {
    unsigned long long fr[NP], fi[NP];
#pragma unroll
    for (int q = 0; q < NP; q++) fr[q] = fi[q] = 0ull;
    const int a1 = min(cnt, a0 + RHO_FLUSH);
#pragma unroll 4
    for (int a = a0; a < a1; a++) {
      const uint4 u = sa[grp][a];
      const float q = __uint_as_float(u.w);
#pragma unroll
      for (int j = 0; j < NP; j++) {
        const int4 mA = m[2 * j], mB = m[2 * j + 1];
        const uint32_t t0 = (uint32_t)mA.x * u.x + ((uint32_t)mA.y * u.y + ((uint32_t)mA.z * u.z + 0x40000000u));
        const uint32_t t1 = (uint32_t)mB.x * u.x + ((uint32_t)mB.y * u.y + ((uint32_t)mB.z * u.z + 0x40000000u));
        if (PK) {
          const unsigned long long phi = half_turn_phi2(t0, t1);
          const unsigned long long z = mul2(phi, phi);
          const unsigned long long sn = sin_poly2(phi, z);
          unsigned long long cs;
          if (PK == 2) {
            cs = cos_poly2(z);
          } else {
            float z0, z1;
            up2(z, z0, z1);
            cs = pk2(cos_poly(z0), cos_poly(z1));
          }
          const unsigned long long q2 = pk2(flip_by(q, t0), flip_by(q, t1));
          fr[j] = fma2(q2, cs, fr[j]);
          fi[j] = fma2(q2, sn, fi[j]);
        } else {
          const float p0 = half_turn_2r(t0) * SC_PI32, p1 = half_turn_2r(t1) * SC_PI32;
          const float z0 = p0 * p0, z1 = p1 * p1;
          const float q0 = flip_by(q, t0), q1 = flip_by(q, t1);
          float r0, r1, i0, i1;
          up2(fr[j], r0, r1);
          up2(fi[j], i0, i1);
          r0 = __fmaf_rn(q0, cos_poly(z0), r0);
          r1 = __fmaf_rn(q1, cos_poly(z1), r1);
          i0 = __fmaf_rn(q0, sin_poly(p0, z0), i0);
          i1 = __fmaf_rn(q1, sin_poly(p1, z1), i1);
          fr[j] = pk2(r0, r1);
          fi[j] = pk2(i0, i1);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < NP; j++) {
      two_sum2(shr[j], slr[j], fr[j]);
      two_sum2(shi[j], sli[j], fi[j]);
    }
    }
  }
  double re[2 * NP], im[2 * NP];
#pragma unroll
  for (int j = 0; j < NP; j++) {
    float h0, h1, l0, l1;
    up2(shr[j], h0, h1);
    up2(slr[j], l0, l1);
    re[2 * j] = (double)h0 + (double)l0;
    re[2 * j + 1] = (double)h1 + (double)l1;
    up2(shi[j], h0, h1);
    up2(sli[j], l0, l1);
    im[2 * j] = (double)h0 + (double)l0;
    im[2 * j + 1] = (double)h1 + (double)l1;
  }
  if (G > 1) {
    if (grp > 0)
#pragma unroll
      for (int t = 0; t < 2 * NP; t++) sg[grp - 1][2 * NP * gt + t] = make_double2(re[t], im[t]);
    __syncthreads();
    if (grp != 0) return;
#pragma unroll
    for (int g = 0; g < G - 1; g++)
#pragma unroll
      for (int t = 0; t < 2 * NP; t++) {
        const double2 e = sg[g][2 * NP * gt + t];
        re[t] += e.x;
        im[t] += e.y;
      }
  }
#pragma unroll
  for (int t = 0; t < 2 * NP; t++)
    if (kb + t < p.P) {
      double *d = p.rho_part + 2 * ((int64_t)(kb + t) * p.ntile + tile);
      d[0] = re[t];
      d[1] = im[t];
    }
}
template <int NP, int G, int MINB, int PK>
__global__ void __launch_bounds__(G * (RHO_BLOCK / NP), MINB) k_rho_mixed(View p) {
  rho_mixed_body<NP, G, MINB, PK>(p, blockIdx.x);
}
template <int NP, int G, int MINB, int PK>
__global__ void __launch_bounds__(G * (RHO_BLOCK / NP), MINB) kp_rho_mixed(Pack pk) {
  RB_PACK_PROLOGUE(pk);
  (void)nb;
  rho_mixed_body<NP, G, MINB, PK>(sv, bid);
}

// the structure factor's launch shapes (rbsog_schedule::rho_variant):
// (pairs per thread, groups per block, blocks per SM of the register bound,
// packed); variants 4..7 are 0..3 in scalar FP32, 8 and 9 are 0 and 1 with
// the cosine packed as well
constexpr int RHO_VARIANTS = 10;
constexpr int RHO_VARIANT_NP[RHO_VARIANTS] = {1, 1, 2, 2, 1, 1, 2, 2, 1, 1};
constexpr int RHO_VARIANT_G[RHO_VARIANTS] = {2, 1, 2, 4, 2, 1, 2, 4, 2, 1};

// F^corr = (1/N) sum of the near-field warp partials, and U_N.  Block b sums
// the fixed slice b of the partials (thread-strided, then a fixed tree); the
// last block to finish adds the CORR_BLOCKS block sums in index order, so the
// result does not depend on which block finishes when.
constexpr int CORR_BLOCKS = 64;
// NV partials per warp (= p.npart): sum F_N (3), U_N and, in energy
// evaluations, the pair virial (6)
template <int NV>
__device__ __forceinline__ void corr_body(const View &p, int blk) {
  __shared__ double red[NV][256];
  __shared__ bool last;
  constexpr int nv = NV;
  const int t = threadIdx.x;
  const int np = p.nblk_near * NEAR_WARPS;
  const int per = (np + CORR_BLOCKS - 1) / CORR_BLOCKS;
  const int b0 = blk * per, b1 = min(b0 + per, np);
  double f[NV] = {};
  for (int b = b0 + t; b < b1; b += 256)
#pragma unroll
    for (int a = 0; a < NV; a++) f[a] += p.near_part[(int64_t)NV * b + a];
#pragma unroll
  for (int a = 0; a < NV; a++) red[a][t] = f[a];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (t < o)
#pragma unroll
      for (int a = 0; a < NV; a++) red[a][t] += red[a][t + o];
    __syncthreads();
  }
  if (t < nv) p.corr_part[NEAR_NPART * blk + t] = red[t][0];
  __threadfence();
  __syncthreads();
  if (t == 0) last = (atomicAdd(p.corr_ticket, 1u) == CORR_BLOCKS - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the CORR_BLOCKS block sums of each value, one per thread, then a fixed tree
  static_assert(CORR_BLOCKS <= 256, "one block sum per thread");
  for (int a = 0; a < nv; a++) red[a][t] = t < CORR_BLOCKS ? __ldcg(p.corr_part + NEAR_NPART * t + a) : 0.0;
  __syncthreads();
  for (int o = CORR_BLOCKS / 2; o > 0; o >>= 1) {
    if (t < o)
      for (int a = 0; a < nv; a++) red[a][t] += red[a][t + o];
    __syncthreads();
  }
  if (t < nv) {
    const double v = red[t][0];
    if (t < 3) p.red[t] = v / (double)p.n;
    else if (t == 3) p.red[3] = v;
    else p.red[5 + (t - 4)] = v;                  // W_N
  }
  if (t == 0) *p.corr_ticket = 0u;                // ready for the next evaluation
}
template <int NV>
__global__ void __launch_bounds__(256) k_corr(View p) { corr_body<NV>(p, blockIdx.x); }

// The per-k outputs of the tile sums (sr0, si0) = rho(k_p): rho, the force
// record (FP64: c Im rho, c Re rho; mixed: the KPair half of mode k), c |rho|^2
// and, in energy evaluations, the per-k virial term.
template <typename R>
__device__ __forceinline__ void reduce_tail(const View &p, int k, double sr0, double si0) {
  p.rho[2 * k] = sr0;
  p.rho[2 * k + 1] = si0;
  const int4 m = p.km[k];
  const double c = p.kc[k];
  const double kx = (double)m.x * p.kunit[0];     // k = 2 pi m / L
  const double ky = (double)m.y * p.kunit[1];
  const double kz_ = (double)m.z * p.kunit[2];
  if (sizeof(R) == 4) {
    // the mixed force record: Psi = arg(rho) in 2^-32 turn (plus the
    // half-turn offset 2^30), K = c |rho| k (Eq. (long-rangeforce) with
    // Im(e^{-i k.r} rho) = |rho| sin(arg rho - k.r))
    const double turn = atan2(si0, sr0) * (1.0 / TWO_PI);      // (-1/2, 1/2]
    const uint32_t psi = (uint32_t)(unsigned long long)(long long)llrint(turn * 4294967296.0);
    const double R = c * hypot(sr0, si0);
    KPair &kp = p.kpair[k >> 1];
    const int h = k & 1;
    int *ra = h ? &kp.b.x : &kp.a.x;
    ra[0] = -m.x; ra[1] = -m.y; ra[2] = -m.z;
    ra[3] = (int)(psi + 0x40000000u);
    float *kxy = &kp.kxy.x, *kz = &kp.kz.x;
    kxy[h] = (float)(R * kx);
    kxy[2 + h] = (float)(R * ky);
    kz[h] = (float)(R * kz_);
    if (!h && k == p.P - 1) {                      // odd P: the pair's second mode is zero
      kp.b = make_int4(0, 0, 0, 0);
      kxy[1] = kxy[3] = kz[1] = 0.0f;
    }
  } else {
    double *o = p.kfd + 5 * (int64_t)k;
    o[0] = kx; o[1] = ky; o[2] = kz_; o[3] = c * si0; o[4] = c * sr0;
  }
  p.uf[k] = c * (sr0 * sr0 + si0 * si0);
  if (p.want_vir) {
    // (Fhat'/Fhat)(k^2) of the SOG transform, a_m = (b^m s)^2 = 1 / (2 h_m):
    // Fhat ~ sum_m w_m a_m^{3/2} e^{-a_m k^2/2}, Fhat' ~ -sum_m w_m a_m^{3/2} (a_m/2) e^{-a_m k^2/2}
    const double k2 = kx * kx + ky * ky + kz_ * kz_;
    double num = 0.0, den = 0.0;
    for (int g = 0; g < p.G; g++) {
      const double a = 0.5 / p.sog_h[g];
      const double t = p.sog_w[g] * a * sqrt(a) * exp(-0.5 * a * k2);
      den += t;
      num += 0.5 * a * t;
    }
    p.vf[k] = -c * (num / den) * (sr0 * sr0 + si0 * si0);
  }
}

// One block per k: fixed-order sum over tiles (thread-strided partial sums,
// a shuffle tree per warp, the eight warp sums in order), then reduce_tail.
template <typename R>
__device__ __forceinline__ void reduce_body(const View &p, int k) {
  __shared__ double2 wsum[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (k < p.P) {
    const double2 *d = reinterpret_cast<const double2 *>(p.rho_part) + (int64_t)k * p.ntile;
    double r = 0.0, i = 0.0;
    for (int t = threadIdx.x; t < p.ntile; t += 256) {
      const double2 v = d[t];
      r += v.x;
      i += v.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      r += __shfl_down_sync(0xffffffffu, r, o);
      i += __shfl_down_sync(0xffffffffu, i, o);
    }
    if (lane == 0) wsum[w] = make_double2(r, i);
    __syncthreads();
    if (threadIdx.x == 0) {
      double sr0 = 0.0, si0 = 0.0;
      for (int u = 0; u < 8; u++) {
        sr0 += wsum[u].x;
        si0 += wsum[u].y;
      }
      reduce_tail<R>(p, k, sr0, si0);
    }
  }
}

// One warp per k (8 modes per block of 256): lane-strided partial sums (eight
// loads in flight per lane), a shuffle tree, then reduce_tail by lane 0.  For
// few tiles per mode, where a block per mode would mostly wait on its tail.
template <typename R>
__device__ __forceinline__ void reduce_warp_body(const View &p, int bid) {
  const int lane = threadIdx.x & 31;
  const int k = bid * 8 + (threadIdx.x >> 5);
  if (k >= p.P) return;
  const double2 *d = reinterpret_cast<const double2 *>(p.rho_part) + (int64_t)k * p.ntile;
  double r = 0.0, i = 0.0;
#pragma unroll 8
  for (int t = lane; t < p.ntile; t += 32) {
    const double2 v = d[t];
    r += v.x;
    i += v.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    r += __shfl_down_sync(0xffffffffu, r, o);
    i += __shfl_down_sync(0xffffffffu, i, o);
  }
  if (lane == 0) reduce_tail<R>(p, k, r, i);
}

template <typename R>
__global__ void __launch_bounds__(256) k_reduce(View p) { reduce_body<R>(p, blockIdx.x); }
template <typename R>
__global__ void __launch_bounds__(256) k_reduce_warp(View p) { reduce_warp_body<R>(p, blockIdx.x); }
__global__ void __launch_bounds__(256) kp_reduce(Pack pk) {
  RB_PACK_PROLOGUE_REF(pk);
  (void)nb;
  reduce_warp_body<float>(sv, bid);
}

// Energies: U_F* = k_e/(2V) sum_p c_p |rho_p|^2 (fixed order); U_self is host-side.
// The far-field virial, minus the strain derivative of U_F* (k . r does not
// change, k_a -> k_a - eps_ab k_b, V -> V (1 + tr eps)):
//   W_F,ab = delta_ab U_F* + (k_e/V) sum_p c_p (Fhat'/Fhat)(k_p^2) k_pa k_pb |rho_p|^2.
__global__ void k_energy(View p) {
  if (threadIdx.x != 0) return;
  double u = 0.0;
  double w[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int k = 0; k < p.P; k++) {
    u += p.uf[k];
    if (p.want_vir) {
      const int4 m = p.km[k];
      const double ka[3] = {TWO_PI * (double)m.x / p.L[0], TWO_PI * (double)m.y / p.L[1],
                            TWO_PI * (double)m.z / p.L[2]};
      const double v = p.vf[k];
      w[0] += v * ka[0] * ka[0]; w[1] += v * ka[1] * ka[1]; w[2] += v * ka[2] * ka[2];
      w[3] += v * ka[0] * ka[1]; w[4] += v * ka[0] * ka[2]; w[5] += v * ka[1] * ka[2];
    }
  }
  const double U = KE / (2.0 * p.V) * u;
  p.red[4] = U;
  if (p.want_vir)
    for (int c = 0; c < 6; c++) p.red[11 + c] = KE / p.V * w[c] + (c < 3 ? U : 0.0);
}

// FP64 far force: one thread per atom, the k-batch staged in shared memory,
// F_F,i = -(k_e q_i / V) sum_p k_p (c Im rho_p cos th - c Re rho_p sin th).
__global__ void __launch_bounds__(FORCE_BLOCK) k_farforce_fp64(View p) {
  __shared__ int4 sm[FORCE_KCHUNK];
  __shared__ double skd[FORCE_KCHUNK * 5];
  const int tid = threadIdx.x;
  const int64_t i = (int64_t)blockIdx.x * FORCE_BLOCK + tid;
  const bool act = i < p.n;
  const uint4 u = act ? p.ua[i] : make_uint4(0, 0, 0, 0);
  double ax = 0.0, ay = 0.0, az = 0.0;
  for (int k0 = 0; k0 < p.P; k0 += FORCE_KCHUNK) {
    const int cnt = min(FORCE_KCHUNK, p.P - k0);
    __syncthreads();
    for (int k = tid; k < cnt; k += FORCE_BLOCK) {
      sm[k] = p.km[k0 + k];
      for (int a = 0; a < 5; a++) skd[5 * k + a] = p.kfd[5 * (int64_t)(k0 + k) + a];
    }
    __syncthreads();
    for (int k = 0; k < cnt; k++) {
      const int4 m = sm[k];
      const uint32_t th = (uint32_t)m.x * u.x + (uint32_t)m.y * u.y + (uint32_t)m.z * u.z;
      double s, c;
      sincos_phase_d(th, s, c);
      const double *kd = skd + 5 * k;
      const double sv = c * kd[3] - s * kd[4];
      ax += sv * kd[0];
      ay += sv * kd[1];
      az += sv * kd[2];
    }
  }
  if (!act) return;
  const int64_t n = p.n;
  const double pre = p.qfar[(int)u.w];          // -k_e q_i / V
  p.FFd[i] = pre * ax; p.FFd[n + i] = pre * ay; p.FFd[2 * n + i] = pre * az;
}

// Mixed far force, Eq. (long-rangeforce) with Im(e^{-i k.r} rho) =
// |rho| sin(arg rho - k.r):
//   F_F,i = -(k_e q_i / V) sum_p K_p sin(2 pi (Psi_p - m_p.u_i) / 2^32),
// K_p = c_p |rho_p| k_p and Psi_p = arg rho_p in 2^-32 turn from k_reduce
// (KPair records), so each (atom, mode) takes one exact integer phase (three
// multiply-adds from Psi_p + 2^30), one sine polynomial (two modes per packed
// FP32x2 instruction) and three FMA.  A block's FORCE_BLOCK / 32 warps are
// (far_S k segments) x (atom warps); a thread takes A atoms (lane + 32 a of
// its atom warp's range) and every far_S-th pair of modes; the segments' FP32
// sums are added in segment order in shared memory, per chunk of FAR_PCHUNK
// pairs, and the chunks in FP64.  PK = 0: the phase factors in scalar FP32
// (bit for bit the same as PK = 1); PK = 2: also the accumulation in packed
// lanes (one lane per mode of the pair, the lanes added at the end: another
// order of the same FP32 terms).
template <int A, int PK>
__device__ __forceinline__ void farforce_mixed_body(const View &p, int bid) {
  __shared__ KPair sk[FAR_PCHUNK];
  __shared__ float sred[FORCE_BLOCK / 32 * A * 32 * 3];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int S = p.far_S, AW = (FORCE_BLOCK / 32) / S;
  const int sg = w / AW, aw = w % AW;
  const int64_t base = (int64_t)bid * (AW * 32 * A) + (int64_t)aw * (32 * A) + lane;
  const int64_t n = p.n;
  uint32_t ux[A], uy[A], uz[A];
#pragma unroll
  for (int a = 0; a < A; a++) {
    const int64_t i = base + 32 * a;
    const uint4 u = i < n ? p.ua[i] : make_uint4(0, 0, 0, 0);
    ux[a] = u.x; uy[a] = u.y; uz[a] = u.z;
  }
  double ax[A], ay[A], az[A];
#pragma unroll
  for (int a = 0; a < A; a++) ax[a] = ay[a] = az[a] = 0.0;
  const int npair = (p.P + 1) >> 1;
  for (int c0 = 0; c0 < npair; c0 += FAR_PCHUNK) {
    const int cnt = min(FAR_PCHUNK, npair - c0);
    __syncthreads();
    {
      const int4 *src = reinterpret_cast<const int4 *>(p.kpair + c0);
      int4 *dst = reinterpret_cast<int4 *>(sk);
      for (int e = tid; e < 4 * cnt; e += FORCE_BLOCK) dst[e] = src[e];
    }
    __syncthreads();
    float fx[A], fy[A], fz[A];
    unsigned long long gx[A], gy[A], gz[A];
#pragma unroll
    for (int a = 0; a < A; a++) {
      fx[a] = fy[a] = fz[a] = 0.0f;
      gx[a] = gy[a] = gz[a] = 0ull;
    }
#pragma unroll 2
    for (int j = sg; j < cnt; j += S) {
      const int4 ra = sk[j].a, rb = sk[j].b;
      const float4 kxy = sk[j].kxy;
      const float2 kz = sk[j].kz;
#pragma unroll
      for (int a = 0; a < A; a++) {
        const uint32_t t0 = (uint32_t)ra.x * ux[a] + ((uint32_t)ra.y * uy[a] + ((uint32_t)ra.z * uz[a] + (uint32_t)ra.w));
        const uint32_t t1 = (uint32_t)rb.x * ux[a] + ((uint32_t)rb.y * uy[a] + ((uint32_t)rb.z * uz[a] + (uint32_t)rb.w));
        float s0, s1;
        if (PK) {
          const unsigned long long phi = half_turn_phi2(t0, t1);
          up2(sin_poly2(phi, mul2(phi, phi)), s0, s1);
        } else {
          const float p0 = half_turn_2r(t0) * SC_PI32, p1 = half_turn_2r(t1) * SC_PI32;
          s0 = sin_poly(p0, p0 * p0);
          s1 = sin_poly(p1, p1 * p1);
        }
        s0 = flip_by(s0, t0);
        s1 = flip_by(s1, t1);
        if (PK == 2) {                             // the two modes in two lanes, summed at the end
          const unsigned long long s2 = pk2(s0, s1);
          gx[a] = fma2(s2, pk2(kxy.x, kxy.y), gx[a]);
          gy[a] = fma2(s2, pk2(kxy.z, kxy.w), gy[a]);
          gz[a] = fma2(s2, pk2(kz.x, kz.y), gz[a]);
        } else {
          fx[a] = __fmaf_rn(s1, kxy.y, __fmaf_rn(s0, kxy.x, fx[a]));
          fy[a] = __fmaf_rn(s1, kxy.w, __fmaf_rn(s0, kxy.z, fy[a]));
          fz[a] = __fmaf_rn(s1, kz.y, __fmaf_rn(s0, kz.x, fz[a]));
        }
      }
    }
    if (PK == 2)
#pragma unroll
      for (int a = 0; a < A; a++) {
        float u0, u1;
        up2(gx[a], u0, u1); fx[a] = u0 + u1;
        up2(gy[a], u0, u1); fy[a] = u0 + u1;
        up2(gz[a], u0, u1); fz[a] = u0 + u1;
      }
    if (S > 1) {                                  // the segments' sums, in segment order
      float *r = sred + ((aw * A) * 32 + lane) * 3;
      if (sg > 0)
#pragma unroll
        for (int a = 0; a < A; a++) {
          float *q = r + (((sg - 1) * AW * A + a) * 32) * 3;
          q[0] = fx[a]; q[1] = fy[a]; q[2] = fz[a];
        }
      __syncthreads();
      if (sg == 0)
        for (int t = 0; t < S - 1; t++)
#pragma unroll
          for (int a = 0; a < A; a++) {
            const float *q = r + ((t * AW * A + a) * 32) * 3;
            fx[a] += q[0]; fy[a] += q[1]; fz[a] += q[2];
          }
    }
#pragma unroll
    for (int a = 0; a < A; a++) {
      ax[a] += (double)fx[a]; ay[a] += (double)fy[a]; az[a] += (double)fz[a];
    }
  }
  if (sg != 0) return;
#pragma unroll
  for (int a = 0; a < A; a++) {
    const int64_t i = base + 32 * a;
    if (i >= n) continue;
    const double pre = p.qfar[p.ua[i].w];        // -k_e q_i / V
    p.FFf[i] = (float)(pre * ax[a]); p.FFf[n + i] = (float)(pre * ay[a]); p.FFf[2 * n + i] = (float)(pre * az[a]);
  }
}
template <int A, int PK>
__global__ void __launch_bounds__(FORCE_BLOCK) k_farforce_mixed(View p) {
  farforce_mixed_body<A, PK>(p, blockIdx.x);
}
template <int A, int PK>
__global__ void __launch_bounds__(FORCE_BLOCK) kp_farforce_mixed(Pack pk) {
  RB_PACK_PROLOGUE(pk);
  (void)nb;
  farforce_mixed_body<A, PK>(sv, bid);
}

// F_i = F_N,i - F^corr + F_F,i, and the closing half kick of the MD step
// (Nose-Hoover: with the block's sum of m v^2 for the chain's closing half step).
// Three threads per atom, one per component (component-major blocks of
// PREP_BLOCK atoms, as k_prepare): the FP64 kick runs on three times the warps;
// the atom's first thread forms m v^2 from the three updated components.
template <typename R, int MODE>
__device__ __forceinline__ void finish_body(const View &p, int bid) {
  constexpr bool MIX = sizeof(R) == 4;
  __shared__ double sv3[3][PREP_BLOCK];
  __shared__ double fcorr[3];
  const int c = threadIdx.x / PREP_BLOCK, li = threadIdx.x % PREP_BLOCK;
  const int64_t i = (int64_t)bid * PREP_BLOCK + li;
  const int64_t n = p.n;
  const bool first = bid == 0 && threadIdx.x == 0;
  // F^corr = (1/N) sum F_N: from the fixed-point totals in force-only
  // evaluations (block 0 also files it where k_corr would), else from k_corr
  if (threadIdx.x < 3) {
    const int t = threadIdx.x;
    double fc;
    if (p.npart == 4) {
      unsigned long long sum = 0ull;             // integer: any order gives the same total
      for (int k = 0; k < CORR_COPIES; k++) sum += p.corr_acc[16 * k + t];
      fc = (double)(long long)sum * (1.0 / CORR_FIX) / (double)n;
      if (bid == 0) p.red[t] = fc;
    } else {
      fc = p.red[t];
    }
    fcorr[t] = fc;
  }
  __syncthreads();
  // the step counter advances here, after both branches joined: every kernel
  // of the step that reads it (k-batch, noise, shell batch) has finished
  if (MODE != 0 && first) *p.step += 1;
  if (first && p.auto_lists) *p.lflag = 0;     // the build flag of the next step starts down
  const bool act = i < n;
  if (act) {
    const double fn = MIX ? (double)p.FNf[c * n + i] : p.FNd[c * n + i];
    const double ff = MIX ? (double)p.FFf[c * n + i] : p.FFd[c * n + i];
    const double F = fn - fcorr[c] + ff;
    if (MIX) p.Ff[c * n + i] = (float)F;
    else p.Fd[c * n + i] = F;
    if (MODE != 0) {
      const double kick = p.kick[p.spc[i]];
      const double Fa = MIX ? (double)(float)F : F;
      p.v[c * n + i] += kick * Fa;
      sv3[c][li] = p.v[c * n + i];
    }
  }
  if (MODE != 0 && p.integ == RBSOG_NOSE_HOOVER) {
    __syncthreads();
    double m2 = 0.0;
    if (c == 0 && act) {
      const double vx = sv3[0][li], vy = sv3[1][li], vz = sv3[2][li];
      m2 = p.massv[p.spc[i]] * (vx * vx + vy * vy + vz * vz);
    }
    const double t = block_sum(m2);
    if (threadIdx.x == 0) p.ke_part[bid] = t;
  }
}
template <typename R, int MODE>
__global__ void __launch_bounds__(3 * PREP_BLOCK) k_finish(View p) { finish_body<R, MODE>(p, blockIdx.x); }
__global__ void __launch_bounds__(3 * PREP_BLOCK) kp_finish(Pack pk) {
  RB_PACK_PROLOGUE(pk);
  (void)nb;
  finish_body<float, 1>(sv, bid);
}

__global__ void k_sincos(int64_t n, const uint32_t *th, float *s, float *c) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float a, b;
  sincos_phase_f(th[i], a, b);
  s[i] = a;
  c[i] = b;
}
void launch_sincos(int64_t n, const uint32_t *th, float *s, float *c, cudaStream_t st) {
  k_sincos<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, th, s, c);
}

void launch_rho(const View &v, cudaStream_t st) {
  const dim3 g(v.ntile * ((v.P + RHO_KTILE - 1) / RHO_KTILE));
  if (v.prec == RBSOG_MIXED) {
    const int var = v.rho_var;
    const int threads = RHO_VARIANT_G[var] * (RHO_BLOCK / RHO_VARIANT_NP[var]);
    switch (var) {
      case 1: k_rho_mixed<1, 1, 2, 1><<<g, threads, 0, st>>>(v); break;
      case 2: k_rho_mixed<2, 2, 2, 1><<<g, threads, 0, st>>>(v); break;
      case 3: k_rho_mixed<2, 4, 1, 1><<<g, threads, 0, st>>>(v); break;
      case 4: k_rho_mixed<1, 2, 2, 0><<<g, threads, 0, st>>>(v); break;
      case 5: k_rho_mixed<1, 1, 2, 0><<<g, threads, 0, st>>>(v); break;
      case 6: k_rho_mixed<2, 2, 2, 0><<<g, threads, 0, st>>>(v); break;
      case 7: k_rho_mixed<2, 4, 1, 0><<<g, threads, 0, st>>>(v); break;
      case 8: k_rho_mixed<1, 2, 2, 2><<<g, threads, 0, st>>>(v); break;
      case 9: k_rho_mixed<1, 1, 2, 2><<<g, threads, 0, st>>>(v); break;
      default: k_rho_mixed<1, 2, 2, 1><<<g, threads, 0, st>>>(v); break;
    }
  } else {
    k_rho_fp64<<<dim3(v.ntile, (v.P + RHO_KTILE - 1) / RHO_KTILE), RHO_BLOCK, 0, st>>>(v);
  }
}

void launch_rhosum(const View &v, cudaStream_t st, bool energy) {
  if (v.rho_reduce == 2 || (v.rho_reduce == 0 && v.ntile <= RHO_WARP_TILES)) {   // a warp per k
    const int g = (std::max(1, v.P) + 7) / 8;
    if (v.prec == RBSOG_MIXED) k_reduce_warp<float><<<g, 256, 0, st>>>(v);
    else k_reduce_warp<double><<<g, 256, 0, st>>>(v);
  } else {                                      // a block per k
    const int g = std::max(1, v.P);
    if (v.prec == RBSOG_MIXED) k_reduce<float><<<g, 256, 0, st>>>(v);
    else k_reduce<double><<<g, 256, 0, st>>>(v);
  }
  if (energy) k_energy<<<1, 32, 0, st>>>(v);
}

// Energy evaluations only: force-only evaluations take F^corr from the
// fixed-point totals in k_finish.
void launch_corr(const View &v, cudaStream_t st, int step_off) {
  (void)step_off;
  if (v.npart == NEAR_NPART) k_corr<NEAR_NPART><<<CORR_BLOCKS, 256, 0, st>>>(v);
}

int far_atoms_per_block(const View &v) {
  return (FORCE_BLOCK / 32 / v.far_S) * 32 * v.far_A;
}

void launch_farforce(const View &v, cudaStream_t st) {
  if (v.prec == RBSOG_MIXED) {
    const int g = (int)((v.n + far_atoms_per_block(v) - 1) / far_atoms_per_block(v));
#define RB_FAR(AA)                                                                   \
  do {                                                                               \
    if (v.far_packed == 2) k_farforce_mixed<AA, 2><<<g, FORCE_BLOCK, 0, st>>>(v);      \
    else if (v.far_packed == 1) k_farforce_mixed<AA, 1><<<g, FORCE_BLOCK, 0, st>>>(v); \
    else k_farforce_mixed<AA, 0><<<g, FORCE_BLOCK, 0, st>>>(v);                        \
  } while (0)
    if (v.far_A == 1) RB_FAR(1);
    else if (v.far_A == 2) RB_FAR(2);
    else RB_FAR(4);
#undef RB_FAR
  } else {
    const int g = (int)((v.n + FORCE_BLOCK - 1) / FORCE_BLOCK);
    k_farforce_fp64<<<g, FORCE_BLOCK, 0, st>>>(v);
  }
}

void launch_finish(const View &v, cudaStream_t st, int mode) {
  const int g = (int)((v.n + PREP_BLOCK - 1) / PREP_BLOCK);   // the ke_part blocks of k_nh_scale
  if (v.prec == RBSOG_MIXED) {
    if (mode == 0) k_finish<float, 0><<<g, 3 * PREP_BLOCK, 0, st>>>(v);
    else k_finish<float, 1><<<g, 3 * PREP_BLOCK, 0, st>>>(v);
  } else {
    if (mode == 0) k_finish<double, 0><<<g, 3 * PREP_BLOCK, 0, st>>>(v);
    else k_finish<double, 1><<<g, 3 * PREP_BLOCK, 0, st>>>(v);
  }
}

int pack_blocks(const View &v, int kind) {
  switch (kind) {
    case PK_KSAMPLE: return v.fixed_k ? 0 : v.nblk_kq;
    case PK_PREP: return (int)((v.n + PREP_BLOCK - 1) / PREP_BLOCK);
    case PK_ONE: return 1;
    case PK_ROWS: return (int)(((int64_t)v.nc[1] * v.nc[2] * 32 + 255) / 256);
    case PK_ATOM256: return (int)((v.n + 255) / 256);
    case PK_NEAR: return v.nblk_near;
    case PK_NEAR_W0: return v.wrap ? 0 : v.nblk_near;
    case PK_NEAR_W1: return v.wrap ? v.nblk_near : 0;
    case PK_RHO: return v.ntile * ((v.P + RHO_KTILE - 1) / RHO_KTILE);
    case PK_REDUCE: return (std::max(1, v.P) + 7) / 8;
    case PK_FAR: return (int)((v.n + far_atoms_per_block(v) - 1) / far_atoms_per_block(v));
    default: return 0;
  }
}

// Packed launches of an ensemble (mixed precision, the schedule of the plan).
void pack_rho(const PackPlan &q, cudaStream_t st) {
  const int g = q.total[PK_RHO], threads = RHO_VARIANT_G[q.rho_var] * (RHO_BLOCK / RHO_VARIANT_NP[q.rho_var]);
  const Pack k = q.pack(PK_RHO);
  switch (q.rho_var) {
    case 1: kp_rho_mixed<1, 1, 2, 1><<<g, threads, 0, st>>>(k); break;
    case 2: kp_rho_mixed<2, 2, 2, 1><<<g, threads, 0, st>>>(k); break;
    case 3: kp_rho_mixed<2, 4, 1, 1><<<g, threads, 0, st>>>(k); break;
    case 4: kp_rho_mixed<1, 2, 2, 0><<<g, threads, 0, st>>>(k); break;
    case 5: kp_rho_mixed<1, 1, 2, 0><<<g, threads, 0, st>>>(k); break;
    case 6: kp_rho_mixed<2, 2, 2, 0><<<g, threads, 0, st>>>(k); break;
    case 7: kp_rho_mixed<2, 4, 1, 0><<<g, threads, 0, st>>>(k); break;
    case 8: kp_rho_mixed<1, 2, 2, 2><<<g, threads, 0, st>>>(k); break;
    case 9: kp_rho_mixed<1, 1, 2, 2><<<g, threads, 0, st>>>(k); break;
    default: kp_rho_mixed<1, 2, 2, 1><<<g, threads, 0, st>>>(k); break;
  }
}
void pack_rhosum(const PackPlan &q, cudaStream_t st) {
  kp_reduce<<<q.total[PK_REDUCE], 256, 0, st>>>(q.pack(PK_REDUCE));
}
void pack_farforce(const PackPlan &q, cudaStream_t st) {
  const int g = q.total[PK_FAR];
  const Pack k = q.pack(PK_FAR);
#define RB_FARP(AA)                                                                   \
  do {                                                                                \
    if (q.far_packed == 2) kp_farforce_mixed<AA, 2><<<g, FORCE_BLOCK, 0, st>>>(k);      \
    else if (q.far_packed == 1) kp_farforce_mixed<AA, 1><<<g, FORCE_BLOCK, 0, st>>>(k); \
    else kp_farforce_mixed<AA, 0><<<g, FORCE_BLOCK, 0, st>>>(k);                        \
  } while (0)
  if (q.far_A == 1) RB_FARP(1);
  else if (q.far_A == 2) RB_FARP(2);
  else RB_FARP(4);
#undef RB_FARP
}
void pack_finish(const PackPlan &q, cudaStream_t st) {
  kp_finish<<<q.total[PK_PREP], 3 * PREP_BLOCK, 0, st>>>(q.pack(PK_PREP));
}

}  // namespace rb
