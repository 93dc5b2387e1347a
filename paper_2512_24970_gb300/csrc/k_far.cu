// Stage (d) far field and stage (e) second half (Sec. 2.2, Eq. (long-rangeforce)):
//   k_rho     structure-factor partials rho(k_p) = sum_j q_j e^{i k_p . r_j} over
//             an atom tile, phase k . r = 2 pi (m . u mod 2^32) / 2^32 reduced
//             exactly in uint32; FP32 polynomial sincos with FP32 accumulation
//             over at most 256 atoms, then FP64 (mixed), or FP64 sincospi (FP64).
//   k_reduce  fixed-order FP64 sum over tiles (one block per k), the per-k
//             force coefficients c_p Im rho_p, c_p Re rho_p.
//   k_corr    F^corr and U_N (and in energy evaluations the pair virial) from
//             the near-field warp partials, fixed order.
//   k_farforce F_F,i = -(k_e q_i / V) sum_p c_p k_p Im(e^{-i k_p.r_i} rho_p).
//   k_finish  F_i = F_N,i - F^corr + F_F,i and the closing half kick of the MD step.
#include "nh.cuh"

namespace rb {

constexpr double TWO_PI = 6.283185307179586;

// Mixed phase e^{i 2 pi th / 2^32}: FP32 polynomial with exact half-turn
// reduction (sincos_turn).
__device__ __forceinline__ void sincos_phase_f(uint32_t th, float &s, float &c) { sincos_turn(th, s, c); }
__device__ __forceinline__ void sincos_phase_d(uint32_t th, double &s, double &c) {
  sincospi((double)(int)th * 4.656612873077393e-10, &s, &c);  // * 2^-31
}

template <typename R>
__global__ void __launch_bounds__(RHO_BLOCK) k_rho(View p) {
  constexpr bool MIX = sizeof(R) == 4;
  __shared__ uint4 sa[256];
  __shared__ R sq[256];
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
      sq[tid] = (R)p.qs[u.w];
    }
    __syncthreads();
    if (MIX) {
      // the thread's two k in packed pairs
      static_assert(RHO_KPT == 2, "packed structure factor takes two k per thread");
      unsigned long long fr = 0ull, fi = 0ull;
#pragma unroll 4
      for (int a = 0; a < cnt; a++) {
        const uint4 u = sa[a];
        const float q = (float)sq[a];
        const uint32_t th0 = mx[0] * u.x + my[0] * u.y + mz[0] * u.z;
        const uint32_t th1 = mx[1] * u.x + my[1] * u.y + mz[1] * u.z;
        unsigned long long s2, c2;
        sincos_turn2(th0, th1, s2, c2);
        const unsigned long long q2 = pk2(q, q);
        fr = fma2(q2, c2, fr);
        fi = fma2(q2, s2, fi);
      }
      float r0, r1, i0, i1;
      up2(fr, r0, r1);
      up2(fi, i0, i1);
      re[0] += (double)r0; re[1] += (double)r1;
      im[0] += (double)i0; im[1] += (double)i1;
    } else {
      for (int a = 0; a < cnt; a++) {
        const uint4 u = sa[a];
        const double q = (double)sq[a];
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

// F^corr = (1/N) sum of the near-field warp partials, and U_N.  Block b sums
// the fixed slice b of the partials (thread-strided, then a fixed tree); the
// last block to finish adds the CORR_BLOCKS block sums in index order, so the
// result does not depend on which block finishes when.
constexpr int CORR_BLOCKS = 64;
// NV partials per warp (= p.npart): sum F_N (3), U_N and, in energy
// evaluations, the pair virial (6)
template <int NV>
__global__ void __launch_bounds__(256) k_corr(View p) {
  __shared__ double red[NV][256];
  __shared__ bool last;
  constexpr int nv = NV;
  const int t = threadIdx.x, blk = blockIdx.x;
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

// One block per k: fixed-order sum over tiles (thread-strided partial sums,
// a shuffle tree per warp, the eight warp sums in order), per-k force
// coefficients (and, in energy evaluations, the per-k virial term).
template <typename R>
__global__ void __launch_bounds__(256) k_reduce(View p) {
  __shared__ double2 wsum[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int k = blockIdx.x;
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
      p.rho[2 * k] = sr0;
      p.rho[2 * k + 1] = si0;
      const int4 m = p.km[k];
      const double c = p.kc[k];
      const double kx = TWO_PI * (double)m.x / p.L[0];
      const double ky = TWO_PI * (double)m.y / p.L[1];
      const double kz = TWO_PI * (double)m.z / p.L[2];
      const double A = c * si0, B = c * sr0;
      if (sizeof(R) == 4) {
        p.kff[k] = make_float4((float)kx, (float)ky, (float)kz, (float)A);
        p.kfB[k] = (float)B;
      } else {
        double *o = p.kfd + 5 * (int64_t)k;
        o[0] = kx; o[1] = ky; o[2] = kz; o[3] = A; o[4] = B;
      }
      p.uf[k] = c * (sr0 * sr0 + si0 * si0);
      if (p.want_vir) {
        // (Fhat'/Fhat)(k^2) of the SOG transform, a_m = (b^m s)^2 = 1 / (2 h_m):
        // Fhat ~ sum_m w_m a_m^{3/2} e^{-a_m k^2/2}, Fhat' ~ -sum_m w_m a_m^{3/2} (a_m/2) e^{-a_m k^2/2}
        const double k2 = kx * kx + ky * ky + kz * kz;
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
  }
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

template <typename R>
__global__ void __launch_bounds__(FORCE_BLOCK) k_farforce(View p) {
  constexpr bool MIX = sizeof(R) == 4;
  // per k: (m_x, m_y, m_z, bits of -c Re rho); mixed: per pair of k the packed
  // (k_x, k_x'; k_y, k_y') and (k_z, k_z'; c Im rho, c' Im rho')
  __shared__ int4 sm[FORCE_KCHUNK];
  __shared__ float4 ska[MIX ? FORCE_KCHUNK / 2 : 1];
  __shared__ float4 skb[MIX ? FORCE_KCHUNK / 2 : 1];
  __shared__ double skd[MIX ? 1 : FORCE_KCHUNK * 5];
  __shared__ float sred[MIX ? FORCE_TPA - 1 : 1][MIX ? FORCE_BLOCK / FORCE_TPA : 1][3];
  const int tid = threadIdx.x;
  // MIX: FORCE_TPA warps per 32 atoms; warp segment g takes the k pairs
  // g, g + FORCE_TPA, ... (warp-uniform shared-memory reads)
  constexpr int TPA_ = MIX ? FORCE_TPA : 1;
  constexpr int APB_ = FORCE_BLOCK / TPA_;    // atoms per block
  const int w = tid >> 5, lane = tid & 31;
  const int g = MIX ? w / (APB_ / 32) : 0;
  const int al = MIX ? (w % (APB_ / 32)) * 32 + lane : tid;   // atom of the block
  const int64_t i = (int64_t)blockIdx.x * APB_ + al;
  const bool act = i < p.n;
  const uint4 u = act ? p.ua[i] : make_uint4(0, 0, 0, 0);
  double ax = 0.0, ay = 0.0, az = 0.0;
  for (int k0 = 0; k0 < p.P; k0 += FORCE_KCHUNK) {
    const int cnt = min(FORCE_KCHUNK, p.P - k0);
    const int cnt2 = (cnt + 1) & ~1;          // an odd chunk ends with a zero pair member
    __syncthreads();
    for (int k = tid; k < cnt2; k += FORCE_BLOCK) {
      if (MIX) {
        int4 m = make_int4(0, 0, 0, 0);
        float4 kf = make_float4(0.f, 0.f, 0.f, 0.f);
        float B = 0.0f;
        if (k < cnt) {
          m = p.km[k0 + k];
          kf = p.kff[k0 + k];
          B = p.kfB[k0 + k];
        }
        sm[k] = make_int4(m.x, m.y, m.z, __float_as_int(-B));
        float *a4 = reinterpret_cast<float *>(&ska[k >> 1]);
        float *b4 = reinterpret_cast<float *>(&skb[k >> 1]);
        a4[k & 1] = kf.x;
        a4[2 + (k & 1)] = kf.y;
        b4[k & 1] = kf.z;
        b4[2 + (k & 1)] = kf.w;
      } else if (k < cnt) {
        sm[k] = p.km[k0 + k];
        for (int a = 0; a < 5; a++) skd[5 * k + a] = p.kfd[5 * (int64_t)(k0 + k) + a];
      }
    }
    __syncthreads();
    if (MIX) {
      unsigned long long fx = 0ull, fy = 0ull, fz = 0ull;
#pragma unroll 2
      for (int k = 2 * g; k < cnt2; k += 2 * TPA_) {
        const int4 m0 = sm[k], m1 = sm[k + 1];
        const uint32_t th0 = (uint32_t)m0.x * u.x + (uint32_t)m0.y * u.y + (uint32_t)m0.z * u.z;
        const uint32_t th1 = (uint32_t)m1.x * u.x + (uint32_t)m1.y * u.y + (uint32_t)m1.z * u.z;
        unsigned long long s2, c2;
        sincos_turn2(th0, th1, s2, c2);
        const float4 ka = ska[k >> 1], kb = skb[k >> 1];
        // Im(e^{-i theta} rho) c = c Im rho cos - c Re rho sin, two k at once
        const unsigned long long sv =
            fma2(c2, pk2(kb.z, kb.w), mul2(s2, pk2(__int_as_float(m0.w), __int_as_float(m1.w))));
        fx = fma2(sv, pk2(ka.x, ka.y), fx);
        fy = fma2(sv, pk2(ka.z, ka.w), fy);
        fz = fma2(sv, pk2(kb.x, kb.y), fz);
      }
      float x0, x1, y0, y1, z0, z1;
      up2(fx, x0, x1);
      up2(fy, y0, y1);
      up2(fz, z0, z1);
      float sx = x0 + x1, sy = y0 + y1, sz = z0 + z1;
      if (MIX && TPA_ > 1) {                   // the segments' sums, in segment order
        if (g > 0) {
          sred[g - 1][al][0] = sx;
          sred[g - 1][al][1] = sy;
          sred[g - 1][al][2] = sz;
        }
        __syncthreads();
        if (g == 0)
          for (int t = 0; t < TPA_ - 1; t++) {
            sx += sred[t][al][0];
            sy += sred[t][al][1];
            sz += sred[t][al][2];
          }
      }
      ax += (double)sx; ay += (double)sy; az += (double)sz;
    } else {
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
  }
  if (!act || g != 0) return;
  const int64_t n = p.n;
  const double pre = p.qfar[(int)u.w];          // -k_e q_i / V
  if (MIX) {
    p.FFf[i] = (float)(pre * ax); p.FFf[n + i] = (float)(pre * ay); p.FFf[2 * n + i] = (float)(pre * az);
  } else {
    p.FFd[i] = pre * ax; p.FFd[n + i] = pre * ay; p.FFd[2 * n + i] = pre * az;
  }
}

// F_i = F_N,i - F^corr + F_F,i, and the closing half kick of the MD step
// (Nose-Hoover: with the block's sum of m v^2 for the chain's closing half step).
// Three threads per atom, one per component (component-major blocks of
// PREP_BLOCK atoms, as k_prepare): the FP64 kick runs on three times the warps;
// the atom's first thread forms m v^2 from the three updated components.
template <typename R, int MODE>
__global__ void __launch_bounds__(3 * PREP_BLOCK) k_finish(View p) {
  constexpr bool MIX = sizeof(R) == 4;
  __shared__ double sv3[3][PREP_BLOCK];
  const int c = threadIdx.x / PREP_BLOCK, li = threadIdx.x % PREP_BLOCK;
  const int64_t i = (int64_t)blockIdx.x * PREP_BLOCK + li;
  const int64_t n = p.n;
  const bool first = blockIdx.x == 0 && threadIdx.x == 0;
  // the step counter advances here, after both branches joined: every kernel
  // of the step that reads it (k-batch, noise, shell batch) has finished
  if (MODE != 0 && first) *p.step += 1;
  if (first && p.auto_lists) *p.lflag = 0;     // the build flag of the next step starts down
  const bool act = i < n;
  if (act) {
    const double fn = MIX ? (double)p.FNf[c * n + i] : p.FNd[c * n + i];
    const double ff = MIX ? (double)p.FFf[c * n + i] : p.FFd[c * n + i];
    const double F = fn - p.red[c] + ff;
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
    if (threadIdx.x == 0) p.ke_part[blockIdx.x] = t;
  }
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
  const dim3 g(v.ntile, (v.P + RHO_BLOCK * RHO_KPT - 1) / (RHO_BLOCK * RHO_KPT));
  if (v.prec == RBSOG_MIXED) k_rho<float><<<g, RHO_BLOCK, 0, st>>>(v);
  else k_rho<double><<<g, RHO_BLOCK, 0, st>>>(v);
}

void launch_rhosum(const View &v, cudaStream_t st, bool energy) {
  const int g = max(1, v.P);                    // one block per k
  if (v.prec == RBSOG_MIXED) k_reduce<float><<<g, 256, 0, st>>>(v);
  else k_reduce<double><<<g, 256, 0, st>>>(v);
  if (energy) k_energy<<<1, 32, 0, st>>>(v);
}

void launch_corr(const View &v, cudaStream_t st, int step_off) {
  (void)step_off;
  if (v.npart == NEAR_NPART) k_corr<NEAR_NPART><<<CORR_BLOCKS, 256, 0, st>>>(v);
  else k_corr<4><<<CORR_BLOCKS, 256, 0, st>>>(v);
}

void launch_farforce(const View &v, cudaStream_t st) {
  const int apb = v.prec == RBSOG_MIXED ? FORCE_BLOCK / FORCE_TPA : FORCE_BLOCK;   // atoms per block
  const int g = (int)((v.n + apb - 1) / apb);
  if (v.prec == RBSOG_MIXED) k_farforce<float><<<g, FORCE_BLOCK, 0, st>>>(v);
  else k_farforce<double><<<g, FORCE_BLOCK, 0, st>>>(v);
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

}  // namespace rb
