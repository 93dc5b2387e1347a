// Internal definitions of the GB300 RBSOG + RBL library: the device view of a
// context (all device pointers and per-system scalars passed by value to every
// kernel), device helpers (Philox4x32-10, fixed-point phases, the FP32 list
// predicate), pair-parameter records and the kernel launchers of each
// translation unit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rbsog.h"

namespace rb {

constexpr double KE = 14.3996454784;     // eV * Angstrom / e^2
constexpr double FCONV = 9648.53321;     // (eV/A)/amu -> A/ps^2
constexpr double KBOLTZ = 8.617333262e-5;  // eV/K

constexpr int NT_TAB = 512;        // intervals of the FP32 SOG tables on [0, r_shell^2]
constexpr int PREP_BLOCK = 128;    // threads per block of k_prepare and k_finish (atoms spread over the SMs)
constexpr int NEAR_BLOCK = 128;    // threads per block of the near-field kernel
constexpr int NEAR_CHUNK = 8;      // atoms per warp of the near-field kernel (4 threads each)
constexpr int NEAR_WARPS = 4;      // warps per near-field block
// Force-only evaluations sum F_N over all atoms (for F^corr) as 64-bit
// integers in units of 2^-40: integer addition does not depend on the order
// in which the warps add, so one atomic add per warp keeps the result
// reproducible bit for bit without a reduction pass.  Each warp's FP64
// partial is rounded once (2^-41 at most); the total must stay below 2^23
// in magnitude (it is a sum of random-batch noise, of order sqrt(N) |F|).
constexpr double CORR_FIX = 1099511627776.0;          // 2^40
// Warp w adds to copy w % CORR_COPIES (its own cache line), so that no
// single address takes every warp's atomic; k_finish adds the copies.
constexpr int CORR_COPIES = 32;
constexpr int NEAR_NPART = 10;     // per-warp partials: sum F_N (3), U_N, pair virial (6)
constexpr int RHO_BLOCK = 256;     // threads per block of the FP64 structure-factor kernel
constexpr int RHO_KPT = 2;         // k-vectors per thread in the structure-factor kernels
constexpr int FORCE_BLOCK = 256;   // threads per block of the far-field force kernels
constexpr int FORCE_KCHUNK = 512;  // k-vectors staged in shared memory per chunk (FP64)
constexpr int FAR_PCHUNK = 256;    // mixed: k pairs staged in shared memory per chunk
constexpr int STENCIL = 5;         // cells per axis in the neighbour stencil (cell >= r_shell/2)

// sorted atoms carry (caller id | species << 28) in one word
constexpr int SU_SP_SHIFT = 28;
constexpr uint32_t SU_ID_MASK = (1u << SU_SP_SHIFT) - 1u;
constexpr uint32_t SU_PAD = 0xFFFFFFFFu;   // padding slot
constexpr float FAR_AWAY = 1e30f;          // coordinate of a padding slot: fails every predicate
constexpr int CELL_ALIGN = 4;              // cell ranges are rounded up to this many slots

// device error bits (latched with atomicOr)
constexpr int ERR_CORE_CAP = 1;
constexpr int ERR_CELL_SHELL_CAP = 2;
constexpr int ERR_PR_CAP = 4;
constexpr int ERR_SKIN = 8;       // kept lists: an atom moved by more than skin/2
constexpr int ERR_KEPT_CAP = 16;  // kept lists: |A| > RBSOG_MAX_CORE or |B| > RBSOG_MAX_KEPT

// Nose-Hoover chain state in View::nh: the chain between steps (A: eta, v
// after the closing half step), the closing half step's velocity scale, and
// the chain after the opening half step (B, written by k_prepare).
constexpr int NH_A_ETA = 0, NH_A_V = 8, NH_S_CLOSE = 17, NH_B_ETA = 24, NH_B_V = 32;
constexpr int NH_STATE = 40;
static_assert(RBSOG_MAX_NH_CHAIN <= 8, "chain state layout");

// Pair record, mixed precision: force phi(r) r_ij with
//   phi = kqq (1/r^3 - G(r^2)) + Ar/r * 2^((sig - r) lr) - (C6 + D8/r^2)/r^8
// and pair energy kqq (1/r - F(r^2)) + A 2^((sig - r) lr) - (C + D/r^2)/r^6.
struct PairF {
  float kqq, Ar, lr, sig;
  float C6, D8, A, C;
  float D, pad0, pad1, pad2;
};
static_assert(sizeof(PairF) == 48, "pair record read as three 16-byte words");
// Mixed far-force record of the modes 2j and 2j + 1, one 64-byte line:
//   a, b = (-m_x, -m_y, -m_z, Psi + 2^30) of each mode, Psi = arg(rho_p) in
//   units of 2^-32 turn (so Psi - m.u is the exact integer phase of
//   sin(arg rho_p - k_p.r));
//   kxy = (K_x, K'_x, K_y, K'_y), kz = (K_z, K'_z), K = c_p |rho_p| k_p.
// A missing second mode (odd P) is all zero.
struct KPair {
  int4 a, b;
  float4 kxy;
  float2 kz, pad;
};
static_assert(sizeof(KPair) == 64, "k-pair record is one 64-byte line");
// Pair record, FP64: the Eq. (BMH) parameters and k_e q_i q_j.
struct PairD {
  double kqq, A, sig, rho, C, D;
};

// Everything a kernel needs, by value.
struct alignas(16) View {
  int64_t n;
  int ns, M, prec, whole_shell;
  int P_R, P_F, P;        // P = modes in use (P_F, or the fixed list length)
  int fixed_k;
  int integ;
  uint64_t seed;
  double L[3], invL[3], V;
  float hp[3];            // fl32(L * 2^-23): predicate scale (23-bit coordinates)
  float hf[3];            // fl32(L * 2^-32): mixed force scale of the low bits
  double hd[3];           // L * 2^-32
  double kunit[3];        // 2 pi / L
  float rc2f, rs2f;
  // species-dependent core radii: core iff r^2 < rc2p[s_i * ns + s_j] (<= rc2f)
  int core_pair;
  float rc2p[RBSOG_MAX_SPECIES * RBSOG_MAX_SPECIES];
  // kept (skin) lists: kept = list_every >= 1; build = this evaluation builds
  // them (the step graph has a build and a keep variant)
  int kept, build;
  int auto_lists;         // kept lists rebuilt when an atom moved by skin/2 (flag set on the device)
  int *lflag;             // [1] auto_lists: this step rebuilds (set by k_prepare or the host)
  unsigned long long *nbuild;  // [1] list builds so far
  float rl2f;             // fl32((r_shell + skin)^2), outer radius of a build
  int a_inside;           // kept lists: (r_core + skin)^2 < 0.98 r_shell^2, so every member of A
                          // stays inside r_shell while no atom moves by skin/2
  double half_skin2;      // (skin / 2)^2, shaded down: the displacement limit
  int *lA, *lB;           // [nslot][RBSOG_MAX_CORE], [nslot][RBSOG_MAX_KEPT] member slots
  int2 *nAB;              // [nslot] (|A|, |B|) of each slot
  int *bsel;              // [nslot][P_R] this step's shell batch: the drawn members' slots, in draw order
  unsigned short *lB16;   // [nslot][RBSOG_MAX_KEPT] B again, as 16-bit slot offsets (see kept_b16_encode)
  int *b16_over;          // [1] set by a build when some offset of B does not fit 16 bits (then lB is read)
  int kept_wide;          // read the 32-bit rows lB whatever the build found (parity hook)
  double *xb;             // [3][n] positions at the last build
  int nc[3], ncell, small;
  int wrap;               // near field reduces differences to the minimum image (short box)
  float tscale;           // NT_TAB / r_shell^2
  double S;
  double dt, c1;
  double qs[RBSOG_MAX_SPECIES];
  double kick[RBSOG_MAX_SPECIES];    // 0.5 dt FCONV / m
  double qfar[RBSOG_MAX_SPECIES];    // -k_e q / V (far-force prefactor)
  double sig_ou[RBSOG_MAX_SPECIES];  // sqrt((1 - c1^2) kT FCONV / m)
  double massv[RBSOG_MAX_SPECIES];   // masses [amu]
  // Nose-Hoover chain (integrator RBSOG_NOSE_HOOVER)
  int nh_M, nh_nblk;      // chain length; blocks of the m v^2 partials (k_finish layout)
  double nh_kT, nh_g;     // kT [eV]; degrees of freedom 3N - 3
  double nh_Q[RBSOG_MAX_NH_CHAIN];  // chain masses [eV ps^2]
  double *nh;             // [NH_STATE] chain state
  double *ke_part;        // [nh_nblk] sum m v^2 per k_finish block
  double *kin_part;       // [nh_nblk][6] block sums of m v_a v_b (kinetic tensor)
  double *kin;            // [6] kinetic tensor K_ab = sum_i m_i v_ia v_ib [eV]
  int G;                  // M + 1
  int ntile, tile_atoms, nblk_atoms, nblk_kq, nblk_near;
  // per-atom state, caller order ([3][n] SoA)
  double *x, *v;
  float *Ff, *FNf, *FFf;
  double *Fd, *FNd, *FFd;
  const int *spc;         // [n] species
  uint4 *ua;              // [n] (u_x, u_y, u_z, species)
  int *cellid;            // [n]
  // binning
  int *cell_count, *cell_start, *cell_cursor;
  int *row_count;         // [ny*nz] atoms per row of cells (follows cell_count)
  int *row_start;         // [ny*nz] first slot of each row
  int *perm_tmp, *perm, *slot_of;
  uint32_t *key_tmp;      // [nslot] u_x of perm_tmp (binning scratch)
  int *row_chunk;         // [ny*nz + 1] first near-field chunk of each row of cells
  int2 *chunk_info;       // [chunks] (row of cells, first slot) of each near-field chunk
  // sorted, padded slots: every cell's range is rounded up to a multiple of 4;
  // pads sit at FAR_AWAY (sx, sy, sz) with su.w = SU_PAD
  float *sx, *sy, *sz;    // [nslot] 23-bit coordinates v = u >> 9 as exact floats
  uint4 *su;              // [nslot] (u_x, u_y, u_z, caller id | species << SU_SP_SHIFT)
  int nslot;              // n + 3 * ncell
  double *near_part;      // [nblk_near * NEAR_WARPS][npart]: sum F_N (x,y,z), pair energy, pair virial (6)
  unsigned long long *corr_acc;  // [CORR_COPIES][16] force-only evaluations: sum F_N (x, y, z) in units
                                 // of 2^-40 (two's complement), one 128-byte line per copy
  int npart;              // partials per warp: 4, or NEAR_NPART in energy evaluations
  int want_vir;           // energy evaluation: also the far-field virial terms
  double *vf;             // [Pmax] c_p (Fhat'/Fhat)(k_p^2) |rho_p|^2 (energy evaluations)
  double *corr_part;      // [64][4] block sums of near_part
  unsigned *corr_ticket;  // blocks of the F^corr reduction done (reset by the last)
  // far field
  int4 *km;               // [Pmax] lattice vectors m
  double *kc;             // [Pmax] weights c_p
  double *rho_part;       // [P][ntile][2]
  double *rho;            // [P][2]
  double *uf;             // [P] c_p |rho_p|^2
  KPair *kpair;           // [Pmax / 2 + 1] mixed far-force records, one per pair of modes
  int far_A, far_S;       // mixed far force: atoms per thread, k segments per block
  int rho_var;            // mixed structure factor: launch shape (rbsog_schedule::rho_variant)
  int far_packed;         // mixed far force: 0 scalar FP32, 1 packed phase factors, 2 packed accumulation too
  int near_bps;           // kept near field: resident blocks per SM (0: one block per 4 runs of slots)
  int near_wide;          // kept near field: a thread's first members of A and of the batch gathered at once
  int rho_reduce;         // tile sums: 0 auto, 1 a block per mode, 2 a warp per mode
  int nsm;                // SMs of the device
  double *kfd;            // [Pmax][5] FP64 (k_x, k_y, k_z, c Im rho, c Re rho)
  double *red;            // [24]: F^corr (3), U_N, U_F*, W_N (6) at 5, W_F* (6) at 11
  int *err;
  long long *step;
  // tables
  const PairF *pf;        // [ns*ns]
  const PairD *pd;        // [ns*ns]
  const double *sog_wa;   // [M+1] w_m / a_m
  const double *sog_w;    // [M+1] w_m
  const double *sog_h;    // [M+1] 1 / (2 a_m)
  const float4 *gtab;     // [NT_TAB] cubic of G(x) = sum w_m/a_m e^{-x/(2 a_m)}
  const float4 *ftab;     // [NT_TAB] cubic of F(x) = sum w_m e^{-x/(2 a_m)}
  const unsigned long long *cmix;  // [3G]
  const unsigned long long *cdf;   // flat 1-D CDFs
  const int *cdf_off0, *cdf_off2, *cdf_nmax;  // [3G]
};

static_assert(sizeof(View) % 16 == 0, "a view is copied in 16-byte words");

// A packed launch of an ensemble: the blocks of every replica in one grid.
// Block b belongs to replica r with b0[r] <= b < b0[r + 1]; views[r] is the
// replica's view (device memory).  Each kernel's body takes (view, block
// index, number of blocks) so that a single launch (blockIdx.x, gridDim.x)
// and a packed one run the same code.
struct Pack {
  const View *views;
  const int *b0;      // [R + 1]
  int R;
};
__device__ __forceinline__ int pack_replica(const Pack &k) {
  const int b = (int)blockIdx.x;
  int lo = 0, hi = k.R - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(k.b0 + mid) <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}
// the replica's view into the block's shared copy (every thread calls it)
__device__ __forceinline__ void pack_view(View &dst, const View *src) {
  const int4 *s = reinterpret_cast<const int4 *>(src);
  int4 *d = reinterpret_cast<int4 *>(&dst);
  for (int e = threadIdx.x; e < (int)(sizeof(View) / 16); e += blockDim.x) d[e] = __ldg(s + e);
  __syncthreads();
}
// Body of a packed kernel: `r` the replica, `sv` its view, (bid, nb) the
// block's index and the replica's block count.  RB_PACK_PROLOGUE copies the
// view into shared memory (kernels whose blocks read it many times);
// RB_PACK_PROLOGUE_REF reads it in place (short blocks: the copy would cost
// more than the reads).
#define RB_PACK_PROLOGUE(pk)                                  \
  __shared__ View sv;                                         \
  const int r_ = pack_replica(pk);                            \
  pack_view(sv, (pk).views + r_);                             \
  const int bid = (int)blockIdx.x - __ldg((pk).b0 + r_);      \
  const int nb = __ldg((pk).b0 + r_ + 1) - __ldg((pk).b0 + r_)
#define RB_PACK_PROLOGUE_REF(pk)                              \
  const int r_ = pack_replica(pk);                            \
  const View &sv = (pk).views[r_];                            \
  const int bid = (int)blockIdx.x - __ldg((pk).b0 + r_);      \
  const int nb = __ldg((pk).b0 + r_ + 1) - __ldg((pk).b0 + r_)

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32 multiplies
// (0xD2511F53, 0xCD9E8D57) with the key bumped by the Weyl constants.
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Draw of the method: counter (index, step_lo, step_hi, stream << 24 | block),
// key = seed.  Streams: 0 shell batch, 1 k-batch, 2 Langevin noise.
__device__ __forceinline__ uint4 draw(uint64_t seed, long long step, uint32_t index,
                                      uint32_t stream, uint32_t block) {
  const unsigned long long st = (unsigned long long)step;
  return philox(make_uint4(index, (uint32_t)st, (uint32_t)(st >> 32), (stream << 24) | block),
                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// Exact int -> float for |x| < 2^22 with one integer add and one float add.
__device__ __forceinline__ float i2f_small(int x) {
  return __int_as_float(x + 0x4B400000) - 12582912.0f;
}

// (sin, cos) of the angle 2 pi th / 2^32 in FP32 for an exact integer phase th.
// The half turn h is taken off in integer arithmetic: m = the top bit of
// th + 2^30, r = th ^ m = th - h 2^31 (two's complement) in [-2^30, 2^30), so
// phi = 2 pi r / 2^32 lies in [-pi/2, pi/2); r is rounded to FP32 (at most
// 2^6 of 2^32 in a turn off, ~1e-7 rad) and scaled.  sin and cos of phi are
// minimax polynomials of degree 9 and 10 on [-pi/2, pi/2] (absolute error
// 4.9e-9 and 4.3e-10 with the binary32 coefficients, below FP32 rounding;
// derived by csrc/sincos_coeffs.py), and sin(phi + h pi) = (-1)^h sin(phi),
// cos likewise: one sign flip by m.  No MUFU: its approximation error is
// smooth in the angle and adds coherently over atoms sharing a phase.
constexpr float SC_S3 = -1.666665673e-01f, SC_S5 = 8.333008736e-03f, SC_S7 = -1.980603120e-04f,
                SC_S9 = 2.598852234e-06f;
constexpr float SC_C2 = -5.000000000e-01f, SC_C4 = 4.166665673e-02f, SC_C6 = -1.388858538e-03f,
                SC_C8 = 2.477017915e-05f, SC_C10 = -2.620901967e-07f;
constexpr float SC_TURN32 = (float)(6.283185307179586 / 4294967296.0);  // 2 pi / 2^32
__device__ __forceinline__ void sincos_turn(uint32_t th, float &s, float &c) {
  const uint32_t m = (th + 0x40000000u) & 0x80000000u;
  const float phi = __int2float_rn((int)(th ^ m)) * SC_TURN32;
  const float z = phi * phi;
  const float ps = __fmaf_rn(__fmaf_rn(__fmaf_rn(SC_S9, z, SC_S7), z, SC_S5), z, SC_S3);
  const float sn = __fmaf_rn(ps * z, phi, phi);
  const float pc =
      __fmaf_rn(__fmaf_rn(__fmaf_rn(__fmaf_rn(SC_C10, z, SC_C8), z, SC_C6), z, SC_C4), z, SC_C2);
  const float cs = __fmaf_rn(pc, z, 1.0f);
  s = __int_as_float(__float_as_int(sn) ^ (int)m);
  c = __int_as_float(__float_as_int(cs) ^ (int)m);
}

// 32-bit fixed-point fractional coordinate floor(frac(x / L) 2^32).
__device__ __forceinline__ uint32_t fixed_point(double x, double invL) {
  const double t = __dmul_rn(x, invL);
  const double y = floor(__dmul_rn(t, 4294967296.0));
  return (uint32_t)(unsigned long long)(long long)y;
}

// cell index of a fixed-point coordinate on an axis with nc cells
__device__ __forceinline__ int cell_of(uint32_t u, int nc) {
  return (int)(((unsigned long long)u * (unsigned long long)nc) >> 32);
}

// FP32 list predicate: r^2 from exact 23-bit differences (as floats) d_a.
__device__ __forceinline__ float pred_r2(float dx, float dy, float dz, const float hp[3]) {
  const float ax = __fmul_rn(dx, hp[0]);
  const float ay = __fmul_rn(dy, hp[1]);
  const float az = __fmul_rn(dz, hp[2]);
  float r2 = __fmul_rn(ax, ax);
  r2 = __fmaf_rn(ay, ay, r2);
  r2 = __fmaf_rn(az, az, r2);
  return r2;
}

// 16-bit form of a kept-list member: the slot offset j - i reduced modulo the
// slot count M into [-M/2, M/2).  Slots run cell by cell with z slowest, so
// the members of a list (within r_shell + skin, across periodic faces too)
// lie within a few layers of cells of the atom's own slot in this cyclic
// order.  Returns false when the offset needs more than 16 bits.
__device__ __forceinline__ bool kept_b16_encode(int j, int i, int M, unsigned short &e) {
  int d = j - i;
  if (2 * d >= M) d -= M;
  else if (2 * d < -M) d += M;
  e = (unsigned short)d;
  return d >= -32768 && d <= 32767;
}
__device__ __forceinline__ int kept_b16_decode(unsigned short e, int i, int M) {
  int j = i + (int)(short)e;
  if (j < 0) j += M;
  else if (j >= M) j -= M;
  return j;
}

// Packed FP32x2 arithmetic (two IEEE binary32 operations per instruction,
// round to nearest, no contraction): same results as the scalar forms.
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void up2(unsigned long long r, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// (hi, lo) += x lane by lane, hi + lo kept as an unevaluated sum: Knuth's
// TwoSum gives the rounding error of hi + x exactly, which goes into lo.
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  return fma2(b, pk2(-1.0f, -1.0f), a);         // a - b, one rounding
}
__device__ __forceinline__ void two_sum2(unsigned long long &hi, unsigned long long &lo, unsigned long long x) {
  const unsigned long long s = add2(hi, x);
  const unsigned long long bp = sub2(s, hi);
  const unsigned long long e = add2(sub2(hi, sub2(s, bp)), sub2(x, bp));
  hi = s;
  lo = add2(lo, e);
}

// sincos_turn of two phases at once: the FP32 steps in packed pairs, the
// half-turn bookkeeping per lane; lane by lane the same results.
__device__ __forceinline__ void sincos_turn2(uint32_t th0, uint32_t th1, unsigned long long &s2,
                                             unsigned long long &c2) {
  const uint32_t m0 = (th0 + 0x40000000u) & 0x80000000u, m1 = (th1 + 0x40000000u) & 0x80000000u;
  const unsigned long long phi = mul2(pk2(__int2float_rn((int)(th0 ^ m0)), __int2float_rn((int)(th1 ^ m1))),
                                      pk2(SC_TURN32, SC_TURN32));
  const unsigned long long z = mul2(phi, phi);
  const unsigned long long ps =
      fma2(fma2(fma2(pk2(SC_S9, SC_S9), z, pk2(SC_S7, SC_S7)), z, pk2(SC_S5, SC_S5)), z, pk2(SC_S3, SC_S3));
  const unsigned long long sn = fma2(mul2(ps, z), phi, phi);
  const unsigned long long pc =
      fma2(fma2(fma2(fma2(pk2(SC_C10, SC_C10), z, pk2(SC_C8, SC_C8)), z, pk2(SC_C6, SC_C6)), z,
                pk2(SC_C4, SC_C4)),
           z, pk2(SC_C2, SC_C2));
  const unsigned long long cs = fma2(pc, z, pk2(1.0f, 1.0f));
  const unsigned long long mm = ((unsigned long long)m1 << 32) | m0;   // the sign of each lane
  s2 = sn ^ mm;
  c2 = cs ^ mm;
}

// The same half-turn reduction from t = th + 2^30, the offset folded into the
// phase's multiply-add chain: h is bit 31 of t, and (int)((t << 1) + 2^31) is
// 2 r exactly (r = th ^ m of sincos_turn), so phi = (float)(2 r) * fl(pi / 2^32)
// is bit for bit sincos_turn's phi (2 r converts to twice r's float, and
// fl(pi / 2^32) is half of fl(2 pi / 2^32)).  One shift-add and one conversion
// per phase; the sign (-1)^h is applied by the caller to whatever it
// multiplies (the charge in rho, the sine in the far force).
constexpr float SC_PI32 = (float)(3.141592653589793 / 4294967296.0);  // pi / 2^32
__device__ __forceinline__ float half_turn_2r(uint32_t t) {
  return __int2float_rn((int)((t << 1) + 0x80000000u));
}
// packed phi of two phases
__device__ __forceinline__ unsigned long long half_turn_phi2(uint32_t t0, uint32_t t1) {
  return mul2(pk2(half_turn_2r(t0), half_turn_2r(t1)), pk2(SC_PI32, SC_PI32));
}
// sin(phi) of sincos_turn's minimax polynomial, two lanes, z = phi^2
__device__ __forceinline__ unsigned long long sin_poly2(unsigned long long phi, unsigned long long z) {
  const unsigned long long ps =
      fma2(fma2(fma2(pk2(SC_S9, SC_S9), z, pk2(SC_S7, SC_S7)), z, pk2(SC_S5, SC_S5)), z, pk2(SC_S3, SC_S3));
  return fma2(mul2(ps, z), phi, phi);
}
// sin(phi) of sincos_turn's minimax polynomial, one lane (the lane-by-lane
// twin of sin_poly2)
__device__ __forceinline__ float sin_poly(float phi, float z) {
  const float ps = __fmaf_rn(__fmaf_rn(__fmaf_rn(SC_S9, z, SC_S7), z, SC_S5), z, SC_S3);
  return __fmaf_rn(ps * z, phi, phi);
}
// cos(phi) of sincos_turn's minimax polynomial, two lanes, z = phi^2
__device__ __forceinline__ unsigned long long cos_poly2(unsigned long long z) {
  const unsigned long long pc =
      fma2(fma2(fma2(fma2(pk2(SC_C10, SC_C10), z, pk2(SC_C8, SC_C8)), z, pk2(SC_C6, SC_C6)), z,
                pk2(SC_C4, SC_C4)),
           z, pk2(SC_C2, SC_C2));
  return fma2(pc, z, pk2(1.0f, 1.0f));
}
// cos(phi) of sincos_turn's minimax polynomial, one lane
__device__ __forceinline__ float cos_poly(float z) {
  const float pc =
      __fmaf_rn(__fmaf_rn(__fmaf_rn(__fmaf_rn(SC_C10, z, SC_C8), z, SC_C6), z, SC_C4), z, SC_C2);
  return __fmaf_rn(pc, z, 1.0f);
}
// x with its sign flipped where bit 31 of t is set
__device__ __forceinline__ float flip_by(float x, uint32_t t) {
  return __uint_as_float(__float_as_uint(x) ^ (t & 0x80000000u));
}

// Packed constants of the list predicate seen from one atom image:
// (-ix, -ix), (-iy, -iy), (-iz, -iz), (hx, hx), (hy, hy), (hz, hz).
struct PredX4 {
  unsigned long long nx, ny, nz, hx, hy, hz;
};
__device__ __forceinline__ PredX4 pred_x4_setup(float ix, float iy, float iz, const float hp[3]) {
  PredX4 c;
  c.nx = pk2(-ix, -ix); c.ny = pk2(-iy, -iy); c.nz = pk2(-iz, -iz);
  c.hx = pk2(hp[0], hp[0]); c.hy = pk2(hp[1], hp[1]); c.hz = pk2(hp[2], hp[2]);
  return c;
}
// The list predicate of pred_r2 for the four padded slots j0..j0+3 (j0 a
// multiple of CELL_ALIGN), two candidates per instruction: r^2 of
// ((v_j - v_i + shift) * h) with the shift folded into (ix, iy, iz).  The
// 16-byte loads deliver the coordinate pairs already packed.
__device__ __forceinline__ void pred_r2_x4(const float *sx, const float *sy, const float *sz, int j0,
                                           const PredX4 &c, float r2[4]) {
  const ulonglong2 X = __ldg(reinterpret_cast<const ulonglong2 *>(sx + j0));
  const ulonglong2 Y = __ldg(reinterpret_cast<const ulonglong2 *>(sy + j0));
  const ulonglong2 Z = __ldg(reinterpret_cast<const ulonglong2 *>(sz + j0));
  const unsigned long long ax0 = mul2(add2(X.x, c.nx), c.hx), ax1 = mul2(add2(X.y, c.nx), c.hx);
  const unsigned long long ay0 = mul2(add2(Y.x, c.ny), c.hy), ay1 = mul2(add2(Y.y, c.ny), c.hy);
  const unsigned long long az0 = mul2(add2(Z.x, c.nz), c.hz), az1 = mul2(add2(Z.y, c.nz), c.hz);
  unsigned long long q0 = mul2(ax0, ax0), q1 = mul2(ax1, ax1);
  q0 = fma2(ay0, ay0, q0);
  q1 = fma2(ay1, ay1, q1);
  q0 = fma2(az0, az0, q0);
  q1 = fma2(az1, az1, q1);
  up2(q0, r2[0], r2[1]);
  up2(q1, r2[2], r2[3]);
}
__device__ __forceinline__ void pred_r2_x4(const float *sx, const float *sy, const float *sz, int j0,
                                           float ix, float iy, float iz, const float hp[3],
                                           float r2[4]) {
  pred_r2_x4(sx, sy, sz, j0, pred_x4_setup(ix, iy, iz, hp), r2);
}

// 23-bit minimum-image difference v_j - v_i (sign-extended), exact.
__device__ __forceinline__ int wrap23(uint32_t uj, uint32_t ui) {
  return ((int)(((uj >> 9) - (ui >> 9)) << 9)) >> 9;
}

// 64-bit CDF pick: #{i < len-1 : C[i] <= U} by binary search.
__device__ __forceinline__ int cdf_pick(const unsigned long long *C, int len, unsigned long long U) {
  int lo = 0, hi = len - 1;  // answer in [0, len-1]
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (C[mid] <= U) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// The same count #{i < len-1 : C[i] <= U} by one warp: each round samples the
// remaining range at 32 evenly spaced entries and keeps the bracket (two
// dependent loads for tables of up to 1024 entries).  All lanes return it.
__device__ __forceinline__ int cdf_pick_warp(const unsigned long long *C, int len, unsigned long long U,
                                             int lane) {
  int base = 0, cnt = len - 1, ans = 0;
  while (cnt > 0) {
    const int s = (cnt + 31) >> 5;
    const bool le = (lane * s < cnt) && (C[base + lane * s] <= U);
    const int k = __popc(__ballot_sync(0xffffffffu, le));
    if (k == 0) break;
    ans += (k - 1) * s + 1;
    if (s == 1) break;
    base += (k - 1) * s + 1;
    cnt = min(s - 1, cnt - ((k - 1) * s + 1));
  }
  return ans;
}

// ---------------------------------------------------------------------------
// Launchers (one translation unit each).
// MODE: 0 = evaluate only, 1 = velocity Verlet step, 2 = BAOAB step.
void launch_prepare(const View &v, cudaStream_t st, int mode, int step_off);
void launch_ksample(const View &v, cudaStream_t st, int step_off);
void launch_bin(const View &v, cudaStream_t st);
void launch_near(const View &v, cudaStream_t st, int step_off, bool energy);
void launch_build_lists(const View &v, cudaStream_t st);
void launch_sample_batch(const View &v, cudaStream_t st, int step_off);
void launch_near_kept(const View &v, cudaStream_t st, int step_off, bool energy);
void launch_kept_batch_used(const View &v, cudaStream_t st, const long long *sel, int nsel, int *batch);
void launch_kept_lists(const View &v, cudaStream_t st, int step_off, const long long *sel, int nsel,
                       int cap_a, int cap_b, int *A, int *nA, int *B, int *nB, int *batch, int *nbatch,
                       double *weight);
void launch_rho(const View &v, cudaStream_t st);
void launch_rhosum(const View &v, cudaStream_t st, bool energy);
void launch_corr(const View &v, cudaStream_t st, int step_off);
void launch_farforce(const View &v, cudaStream_t st);
void launch_finish(const View &v, cudaStream_t st, int mode);
void launch_nh_close(const View &v, cudaStream_t st);
void launch_nh_prime(const View &v, cudaStream_t st);
void launch_kinetic_tensor(const View &v, cudaStream_t st);
void launch_lists(const View &v, cudaStream_t st, int step_off, const long long *sel, int nsel,
                  int cap_core, int cap_shell, int *core, int *ncore, int *shell, int *nshell,
                  int *batch, int *nbatch, double *weight);
void launch_sincos(int64_t n, const uint32_t *th, float *s, float *c, cudaStream_t st);

// Packed launches of an ensemble: one grid per stage over every replica.
// Kinds of block tables (blocks per replica of each launch shape).
enum PackKind {
  PK_KSAMPLE,   // k-batch: one warp per sample
  PK_PREP,      // integrator kernels: PREP_BLOCK atoms per block
  PK_ONE,       // one block per replica (row scan)
  PK_ROWS,      // a warp per row of cells (cell prefix)
  PK_ATOM256,   // one thread per atom, blocks of 256 (scatter, rank)
  PK_NEAR,      // near-field warps over runs of slots (kept lists)
  PK_NEAR_W0,   // the list walk of replicas without minimum-image wrapping (others: no blocks)
  PK_NEAR_W1,   // ... with it
  PK_RHO,       // structure-factor tiles x columns of modes
  PK_REDUCE,    // one block per mode
  PK_FAR,       // far-force blocks
  PK_KINDS
};
struct PackPlan {
  const View *views = nullptr;     // [R] device copies of the replicas' step views
  int R = 0;
  const int *b0[PK_KINDS] = {};    // [R + 1] device prefix tables
  int total[PK_KINDS] = {};
  int rho_var = 0, far_A = 2, far_packed = 1;   // the replicas' common far-field schedule
  int near_wide = 0;
  Pack pack(int k) const { return Pack{views, b0[k], R}; }
};
// blocks of replica view v in launch shape `kind` (host)
int pack_blocks(const View &v, int kind);
void pack_ksample(const PackPlan &q, cudaStream_t st, int step_off);
void pack_prepare(const PackPlan &q, cudaStream_t st, int mode, int step_off);
void pack_bin(const PackPlan &q, cudaStream_t st);
void pack_near(const PackPlan &q, cudaStream_t st, int step_off);
void pack_build_lists(const PackPlan &q, cudaStream_t st);
void pack_sample_batch(const PackPlan &q, cudaStream_t st, int step_off);
void pack_near_kept(const PackPlan &q, cudaStream_t st, int step_off);
void pack_rho(const PackPlan &q, cudaStream_t st);
void pack_rhosum(const PackPlan &q, cudaStream_t st);
void pack_farforce(const PackPlan &q, cudaStream_t st);
void pack_finish(const PackPlan &q, cudaStream_t st);
int far_atoms_per_block(const View &v);

// Allocation-free structure factor (k_static.cu): static scratch of
// SF_STATIC_PMAX modes x SF_STATIC_TILES tile partials of 16 B (2 MiB).
constexpr int SF_STATIC_PMAX = 1024;
constexpr int SF_STATIC_TILES = 128;
constexpr int SF_STATIC_MAX_DEVICES = 64;
cudaError_t sf_static_scratch(int dev, void **out);
void launch_sf_static(const View &v, int P, const int *m, double *rho, void *scratch, cudaStream_t st);
void launch_aos_to_soa(const double *aos, double *soa, int64_t n, cudaStream_t st);
void launch_aos_to_soa_step(const double *aos, double *soa, int64_t n, long long *step, long long s,
                            cudaStream_t st);
void launch_soa_to_aos_d(const double *soa, double *aos, int64_t n, cudaStream_t st);
void launch_soa_to_aos_f(const float *soa, double *aos, int64_t n, cudaStream_t st);

}  // namespace rb
