// Stages (a2), (b), (c): one fused kernel per step builds the random batch list
// and evaluates the near field (Sec. 2.2): list predicate over the cell
// stencil, Floyd's P_R-of-N_shell shell batch without replacement (Philox
// stream 0), core + weighted batch pair forces.  The pair force is
// Eq. (Fshort) (SOG residual + BMH, k_e on Coulomb): FP32 with the SOG sum
// tabulated (mixed) or analytic FP64 over m = 0..M.  The block's FP64 partial
// sums of F_N feed the momentum correction F^corr.  With kept (skin) lists
// the walk's BUILD variant writes the lists and k_near_kept evaluates them.
#include <algorithm>

#include "rbsog_internal.cuh"

namespace rb {

// ---------------------------------------------------------------------------
// Stencil of one axis: position k = 0..4 in ascending cell order.  For n >= 5
// the offsets o = -2..2 are rotated so the wrapped cells sort by index; the
// shift (in 23-bit units) maps the neighbour image next to atom i.
struct Axis {
  int ci, n, rot;
};
__device__ __forceinline__ Axis make_axis(int ci, int n) {
  Axis a;
  a.ci = ci;
  a.n = n;
  a.rot = (ci < 2) ? (2 - ci) : ((ci + 2 >= n) ? (n - ci + 2) : 0);
  return a;
}
__device__ __forceinline__ int axis_count(const Axis &a, bool small) {
  return (small && a.n < STENCIL) ? a.n : STENCIL;
}
// cell index and shift of stencil position k
__device__ __forceinline__ int axis_cell(const Axis &a, int k, bool small, float &shift) {
  if (small && a.n < STENCIL) {  // all cells of a short axis, ascending; shift per pair
    shift = 0.0f;
    return k;
  }
  int o = k + a.rot;
  o = (o >= STENCIL ? o - STENCIL : o) - 2;
  const int c = a.ci + o;
  if (c < 0) { shift = -8388608.0f; return c + a.n; }
  if (c >= a.n) { shift = 8388608.0f; return c - a.n; }
  shift = 0.0f;
  return c;
}

// Predicate r^2 of the candidate at slot j seen from atom i.
template <bool SMALL>
__device__ __forceinline__ float cand_r2(const View &p, int j, float ix, float iy, float iz,
                                         uint4 ui) {
  if (SMALL) {
    const uint4 uj = p.su[j];
    if (uj.w == SU_PAD) return FAR_AWAY;
    return pred_r2((float)wrap23(uj.x, ui.x), (float)wrap23(uj.y, ui.y), (float)wrap23(uj.z, ui.z), p.hp);
  } else {
    return pred_r2(p.sx[j] - ix, p.sy[j] - iy, p.sz[j] - iz, p.hp);
  }
}

// ---------------------------------------------------------------------------
// Pair terms.
struct PairOut {
  float fx, fy, fz, e;
};

// With ENERGY also the pair energy and the pair virial r_ij (x) f_ij
// (xx, yy, zz, xy, xz, yz) into wv.
template <bool ENERGY>
__device__ __forceinline__ void pair_mixed(const View &p, const PairF &q, const float4 *gt,
                                           uint4 ui, uint4 uj, float &fx, float &fy, float &fz,
                                           float &e, float *wv) {
  float d[3];
  const uint32_t a3[3] = {ui.x - uj.x, ui.y - uj.y, ui.z - uj.z};
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const int dl = (int)a3[a];
    d[a] = __fmaf_rn(i2f_small(dl >> 9), p.hp[a], __fmul_rn(i2f_small(dl & 511), p.hf[a]));
  }
  const float x = __fmaf_rn(d[2], d[2], __fmaf_rn(d[1], d[1], d[0] * d[0]));
  // 1/r from the hardware reciprocal square root refined by one Newton step
  // (relative error ~1 ulp), r = x / r
  float rinv = rsqrtf(x);
  rinv = rinv * __fmaf_rn(-0.5f * x * rinv, rinv, 1.5f);
  const float r = x * rinv;
  const float rinv2 = rinv * rinv;
  const float t = x * p.tscale;
  const int it = min((int)t, NT_TAB - 1);
  const float f = t - (float)it;
  const float4 c = __ldg(gt + it);
  const float G = __fmaf_rn(__fmaf_rn(__fmaf_rn(c.w, f, c.z), f, c.y), f, c.x);
  const float ex = exp2f((q.sig - r) * q.lr);
  const float r4 = rinv2 * rinv2;
  const float r8 = r4 * r4;
  const float phi = q.kqq * (rinv2 * rinv - G) + q.Ar * rinv * ex - (q.C6 + q.D8 * rinv2) * r8;
  fx += phi * d[0];
  fy += phi * d[1];
  fz += phi * d[2];
  if (ENERGY) {
    const float4 cf = p.ftab[it];
    const float Fv = __fmaf_rn(__fmaf_rn(__fmaf_rn(cf.w, f, cf.z), f, cf.y), f, cf.x);
    e += q.kqq * (rinv - Fv) + q.A * ex - (q.C + q.D * rinv2) * r4 * rinv2;
    const float f0 = phi * d[0], f1 = phi * d[1], f2 = phi * d[2];
    wv[0] += d[0] * f0; wv[1] += d[1] * f1; wv[2] += d[2] * f2;
    wv[3] += d[0] * f1; wv[4] += d[0] * f2; wv[5] += d[1] * f2;
  }
}

template <bool ENERGY>
__device__ __forceinline__ void pair_fp64(const View &p, const PairD &q, const double *wa,
                                          const double *w, const double *h2, uint4 ui, uint4 uj,
                                          double &fx, double &fy, double &fz, double &e, double *wv) {
  const double dx = (double)(int)(ui.x - uj.x) * p.hd[0];
  const double dy = (double)(int)(ui.y - uj.y) * p.hd[1];
  const double dz = (double)(int)(ui.z - uj.z) * p.hd[2];
  const double x = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  const double r = sqrt(x);
  double g = 0.0, fsum = 0.0;
  for (int m = 0; m < p.G; m++) {
    const double ex = exp(-x * h2[m]);
    g += wa[m] * ex;
    if (ENERGY) fsum += w[m] * ex;
  }
  const double rep = q.A * exp((q.sig - r) / q.rho);
  const double r6 = x * x * x, r8 = r6 * x;
  const double phi = q.kqq * (1.0 / (x * r) - g) + rep / (q.rho * r) - 6.0 * q.C / r8 - 8.0 * q.D / (r8 * x);
  fx += phi * dx;
  fy += phi * dy;
  fz += phi * dz;
  if (ENERGY) {
    e += q.kqq * (1.0 / r - fsum) + rep - q.C / r6 - q.D / r8;
    const double f0 = phi * dx, f1 = phi * dy, f2 = phi * dz;
    wv[0] += dx * f0; wv[1] += dy * f1; wv[2] += dz * f2;
    wv[3] += dx * f1; wv[4] += dx * f2; wv[5] += dy * f2;
  }
}

// ---------------------------------------------------------------------------
// Floyd's algorithm: P_R distinct positions of [0, nshell), ascending.
__device__ __forceinline__ void floyd(const View &p, long long s, uint32_t id, int nshell,
                                      int *t) {
  const int PR = p.P_R;
  uint4 w = make_uint4(0, 0, 0, 0);
  for (int r = 0; r < PR; r++) {
    if ((r & 1) == 0) w = draw(p.seed, s, id, 0u, (uint32_t)(r >> 1));
    const unsigned long long U = (r & 1) ? (((unsigned long long)w.w << 32) | w.z)
                                         : (((unsigned long long)w.y << 32) | w.x);
    const uint32_t J = (uint32_t)(nshell - PR + r);
    const uint32_t tt = (uint32_t)__umul64hi(U, (unsigned long long)J + 1ull);
    bool present = false;
    for (int k = 0; k < r; k++) present |= (t[k] == (int)tt);
    t[r] = present ? (int)J : (int)tt;
  }
  for (int a = 1; a < PR; a++) {
    const int v = t[a];
    int b = a - 1;
    while (b >= 0 && t[b] > v) {
      t[b + 1] = t[b];
      b--;
    }
    t[b + 1] = v;
  }
}

template <typename R>
struct Acc {
  R x = 0, y = 0, z = 0, e = 0;
  R w[6] = {0, 0, 0, 0, 0, 0};   // pair virial (energy evaluations only)
};

// Pair force of atom i with the sorted candidate uj (species in its top bits).
template <typename R, bool ENERGY>
__device__ __forceinline__ void add_pair(const View &p, const PairF *spf, const PairD *spd,
                                         const float4 *sg, const double *swa, const double *sw,
                                         const double *sh2, int spi, uint4 ui, uint4 uj, Acc<R> &a) {
  const int spj = (int)(uj.w >> SU_SP_SHIFT);
  if constexpr (sizeof(R) == 4) {
    float a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    // the pair record through the read-only cache (three 16-byte loads)
    const float4 *src = reinterpret_cast<const float4 *>(spf + spi * p.ns + spj);
    const float4 r0 = __ldg(src), r1 = __ldg(src + 1), r2 = __ldg(src + 2);
    PairF q;
    q.kqq = r0.x; q.Ar = r0.y; q.lr = r0.z; q.sig = r0.w;
    q.C6 = r1.x; q.D8 = r1.y; q.A = r1.z; q.C = r1.w;
    q.D = r2.x;
    pair_mixed<ENERGY>(p, q, sg, ui, uj, a0, a1, a2, a3, a.w);
    a.x += a0; a.y += a1; a.z += a2; a.e += a3;
  } else {
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    pair_fp64<ENERGY>(p, spd[spi * p.ns + spj], swa, sw, sh2, ui, uj, a0, a1, a2, a3, a.w);
    a.x += a0; a.y += a1; a.z += a2; a.e += a3;
  }
}

// One warp per chunk of up to NEAR_CHUNK = 8 consecutive sorted slots of one
// row of cells (fixed cell y and z); TPA = 4 threads per atom.  The atoms of
// a chunk share the stencil rows (y, z) of their row of cells.  Along x, a
// stencil row's candidates are the union of the chunk's five-cell
// x-stencils: one or two runs of sorted slots in ascending cell index, i.e.
// in the canonical order (cell index, caller index).  On short boxes
// (WRAP) a row whose union would meet itself is taken whole, and every
// difference is reduced to the minimum image.
//  pass 1  thread g of every atom tests the candidates of stencil rows g,
//          g + 4, ... with the FP32 list predicate, four slots per step;
//          all eight atoms walk the same slots at the same time (broadcast
//          loads).  Each row gives bit masks over its candidates: the shell
//          mask stays in shared memory, core members go to a short list.
//  pass 2  per-row shell counts -> prefix (canonical index of each row's
//          first shell member).  Floyd's P_R-of-N_shell draw: the group's
//          threads compute the Philox words and candidate positions in
//          parallel, its first thread resolves them in order.
//  pass 3  sample t: its row by binary search of the prefix, its slot as the
//          (t - prefix)-th set bit of the row's shell mask; weight N_shell/P_R.
//  pass 4  the group's core lists, dealt round-robin over its threads.
constexpr int TPA = 4;
constexpr int APW = NEAR_CHUNK;              // atoms per warp
constexpr int APB = NEAR_WARPS * NEAR_CHUNK; // atoms per block
constexpr int NROW = STENCIL * STENCIL;      // stencil rows (y, z)
// candidate groups one atom's chunk may test: culled rows (the common case),
// or the whole rows of a short box (WRAP: 25 rows of at most
// RBSOG_MAX_ROW_SLOTS / 4 groups)
constexpr int GBYTES_CULLED = 352;
constexpr int GBYTES_BUILD = 512;            // kept-list builds: outer radius r_shell + skin
constexpr int GBYTES_WRAP = STENCIL * STENCIL * RBSOG_MAX_ROW_SLOTS / CELL_ALIGN;
constexpr int SHELL_BITS = RBSOG_MAX_SHELL;  // shell members one bitmask can index
constexpr int WMAX = 8;                      // union x-cells of a chunk
static_assert(TPA * NEAR_CHUNK == 32 && NEAR_WARPS * 32 == NEAR_BLOCK, "near-field block layout");
static_assert(RBSOG_MAX_ROW_SLOTS % 32 == 0 && RBSOG_MAX_ROW_SLOTS <= 128, "row position needs 7 bits");

// position of the k-th (from 0) set bit of m; k < popc(m)
__device__ __forceinline__ int select_bit(uint32_t m, int k) {
  int pos = 0, c = __popc(m & 0xFFFFu);
  if (k >= c) { k -= c; m >>= 16; pos += 16; }
  c = __popc(m & 0xFFu);
  if (k >= c) { k -= c; m >>= 8; pos += 8; }
  c = __popc(m & 0xFu);
  if (k >= c) { k -= c; m >>= 4; pos += 4; }
  c = __popc(m & 0x3u);
  if (k >= c) { k -= c; m >>= 2; pos += 2; }
  return pos + ((k >= (int)(m & 1u)) ? 1 : 0);
}

// d (23-bit units, exact integer) reduced to the minimum image; values far
// outside the box (padding slots) stay far
__device__ __forceinline__ float min_image23(float d) {
  const float k = fminf(fmaxf(rintf(d * 1.1920928955078125e-07f), -1.0f), 1.0f);
  return __fmaf_rn(k, -8388608.0f, d);
}

// predicate r^2 of slots j0..j0+3 with every difference reduced to the minimum image
__device__ __forceinline__ void pred_r2_x4_wrap(const View &p, int j0, float ix, float iy, float iz,
                                                float r2[4]) {
  const float4 X = __ldg(reinterpret_cast<const float4 *>(p.sx + j0));
  const float4 Y = __ldg(reinterpret_cast<const float4 *>(p.sy + j0));
  const float4 Z = __ldg(reinterpret_cast<const float4 *>(p.sz + j0));
  r2[0] = pred_r2(min_image23(X.x - ix), min_image23(Y.x - iy), min_image23(Z.x - iz), p.hp);
  r2[1] = pred_r2(min_image23(X.y - ix), min_image23(Y.y - iy), min_image23(Z.y - iz), p.hp);
  r2[2] = pred_r2(min_image23(X.z - ix), min_image23(Y.z - iy), min_image23(Z.z - iz), p.hp);
  r2[3] = pred_r2(min_image23(X.w - ix), min_image23(Y.w - iy), min_image23(Z.w - iz), p.hp);
}

// slot of candidate position pos of a row (a0, na, b0, nb)
__device__ __forceinline__ int row_slot(const int4 &sg, int pos) {
  return pos < sg.y ? sg.x + pos : sg.z + (pos - sg.y);
}

// First slot of row-of-cells rb whose sorted x coordinate is >= v (upper:
// > v); the search is confined to the cells around v's cell.
__device__ __forceinline__ int sx_bound(const View &p, int rb, float v, bool upper) {
  const int nc0 = p.nc[0];
  const int c = min(max((int)(v * ((float)nc0 * 1.1920928955078125e-07f)), 0), nc0 - 1);
  int lo = p.cell_start[rb + max(c - 1, 0)], hi = p.cell_start[rb + min(c + 2, nc0)];
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const float x = __ldg(p.sx + mid);
    if (upper ? (x <= v) : (x < v)) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// pred_r2_x4 with the results left packed: q0 = (r2[0], r2[1]), q1 = (r2[2], r2[3])
__device__ __forceinline__ void pred_r2_x4_packed(const float *sx, const float *sy, const float *sz, int j0,
                                                  const PredX4 &c, unsigned long long &q0,
                                                  unsigned long long &q1) {
  const ulonglong2 X = __ldg(reinterpret_cast<const ulonglong2 *>(sx + j0));
  const ulonglong2 Y = __ldg(reinterpret_cast<const ulonglong2 *>(sy + j0));
  const ulonglong2 Z = __ldg(reinterpret_cast<const ulonglong2 *>(sz + j0));
  const unsigned long long ax0 = mul2(add2(X.x, c.nx), c.hx), ax1 = mul2(add2(X.y, c.nx), c.hx);
  const unsigned long long ay0 = mul2(add2(Y.x, c.ny), c.hy), ay1 = mul2(add2(Y.y, c.ny), c.hy);
  const unsigned long long az0 = mul2(add2(Z.x, c.nz), c.hz), az1 = mul2(add2(Z.y, c.nz), c.hz);
  q0 = fma2(az0, az0, fma2(ay0, ay0, mul2(ax0, ax0)));
  q1 = fma2(az1, az1, fma2(ay1, ay1, mul2(ax1, ax1)));
}

// One partial per warp of sum F_N and of the pair energy (FP32 sums of the
// warp's eight atoms in mixed precision, FP64 otherwise).  Force-only
// evaluations (NP = 4) add the F_N sum to the fixed-point totals instead
// (CORR_FIX); energy evaluations write every partial for k_corr.
template <bool MIX, int NP>
__device__ __forceinline__ void warp_partials(const View &p, double part[NEAR_NPART], int wchunk, int lane) {
  if constexpr (NP == 4) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      if (MIX) {
        float f = (float)part[c];
        for (int o = 16; o > 0; o >>= 1) f += __shfl_down_sync(0xffffffffu, f, o);
        part[c] = (double)f;
      } else {
        for (int o = 16; o > 0; o >>= 1) part[c] += __shfl_down_sync(0xffffffffu, part[c], o);
      }
    }
    if (lane == 0) {
      unsigned long long *acc = p.corr_acc + 16 * (wchunk % CORR_COPIES);
#pragma unroll
      for (int c = 0; c < 3; c++) atomicAdd(acc + c, (unsigned long long)__double2ll_rn(part[c] * CORR_FIX));
    }
    return;
  }
#pragma unroll
  for (int c = 0; c < NP; c++) {
    if (MIX) {
      float f = (float)part[c];
      for (int o = 16; o > 0; o >>= 1) f += __shfl_down_sync(0xffffffffu, f, o);
      part[c] = (double)f;
    } else {
      for (int o = 16; o > 0; o >>= 1) part[c] += __shfl_down_sync(0xffffffffu, part[c], o);
    }
  }
  if (lane == 0) {
    double *d = p.near_part + NP * (int64_t)wchunk;
#pragma unroll
    for (int c = 0; c < NP; c++) d[c] = part[c];
  }
}

// Sum an atom's exact part fc and batch part fs over its TPA threads; its
// first thread writes F_N = fc + wgt fs (caller order) and its warp-partial
// terms.
template <typename R, bool ENERGY>
__device__ __forceinline__ void combine_atom(const View &p, Acc<R> &fc, Acc<R> &fs, R wgt, bool active,
                                             int g, uint4 ui, double part[NEAR_NPART]) {
#pragma unroll
  for (int o = 1; o < TPA; o <<= 1) {
    fc.x += __shfl_xor_sync(0xffffffffu, fc.x, o, TPA);
    fc.y += __shfl_xor_sync(0xffffffffu, fc.y, o, TPA);
    fc.z += __shfl_xor_sync(0xffffffffu, fc.z, o, TPA);
    fs.x += __shfl_xor_sync(0xffffffffu, fs.x, o, TPA);
    fs.y += __shfl_xor_sync(0xffffffffu, fs.y, o, TPA);
    fs.z += __shfl_xor_sync(0xffffffffu, fs.z, o, TPA);
    if (ENERGY) {
      fc.e += __shfl_xor_sync(0xffffffffu, fc.e, o, TPA);
      fs.e += __shfl_xor_sync(0xffffffffu, fs.e, o, TPA);
#pragma unroll
      for (int c = 0; c < 6; c++) {
        fc.w[c] += __shfl_xor_sync(0xffffffffu, fc.w[c], o, TPA);
        fs.w[c] += __shfl_xor_sync(0xffffffffu, fs.w[c], o, TPA);
      }
    }
  }
  if (active && g == 0) {
    const R Fx = fc.x + wgt * fs.x, Fy = fc.y + wgt * fs.y, Fz = fc.z + wgt * fs.z;
    const int64_t id = ui.w & SU_ID_MASK, n = p.n;
    if (sizeof(R) == 4) {
      p.FNf[id] = (float)Fx; p.FNf[n + id] = (float)Fy; p.FNf[2 * n + id] = (float)Fz;
    } else {
      p.FNd[id] = (double)Fx; p.FNd[n + id] = (double)Fy; p.FNd[2 * n + id] = (double)Fz;
    }
    part[0] = (double)Fx; part[1] = (double)Fy; part[2] = (double)Fz;
    part[3] = (double)((R)0.5 * (fc.e + wgt * fs.e));
    if (ENERGY)
#pragma unroll
      for (int c = 0; c < 6; c++) part[4 + c] = (double)((R)0.5 * (fc.w[c] + wgt * fs.w[c]));
  }
}

// BUILD: the same walk with the outer radius r_list = r_shell + skin builds
// the kept lists instead (A = core members, B = the rest inside r_list, both
// in canonical order, i.e. ascending slot) and evaluates nothing.
template <typename R, bool WRAP, bool ENERGY, bool BUILD>
__device__ __forceinline__ void near_body(const View &p, int step_off, int bid, int nbk) {
  constexpr bool MIX = sizeof(R) == 4;
  // per-atom rows padded by one word so that the eight atoms of a warp hit distinct banks
  constexpr int GBYTES = WRAP ? GBYTES_WRAP : (BUILD ? GBYTES_BUILD : GBYTES_CULLED);
  __shared__ __align__(16) unsigned char gres[APB][GBYTES + 4]; // per group of 4 candidates: r < r_shell (bits 0-3), r < r_core (4-7)
  __shared__ unsigned char scnt[APB][NROW];      // shell members of each stencil row
  __shared__ unsigned char ccnt[BUILD ? APB : 1][BUILD ? NROW : 1];  // core members (BUILD)
  __shared__ unsigned short spre[APB][NROW + 1]; // exclusive prefix of the counts
  __shared__ unsigned short stsel[APB][RBSOG_MAX_PR + 2];
  __shared__ uint32_t bmask[APB][SHELL_BITS / 32 + 1];
  __shared__ unsigned short score[APB][RBSOG_MAX_CORE + 2];  // core list (row << 7 | position)
  __shared__ int4 rseg[NEAR_WARPS][NROW];        // candidate runs (a0, na, b0, nb)
  __shared__ float4 rsh[NEAR_WARPS][NROW];       // image shifts (x of run a, x of run b, y, z)
  __shared__ int rgo[NEAR_WARPS][NROW + 1];      // first group of each row (flattened)
  __shared__ int rbo[NEAR_WARPS][NROW];          // first byte of each row in gres
  const PairF *spf = p.pf;                       // pair records, read through the read-only cache
  const PairD *spd = p.pd;
  const int tid = threadIdx.x;
  const float4 *sg4 = p.gtab;
  const double *swa = p.sog_wa, *sw = p.sog_w, *sh2 = p.sog_h;
  const long long s = *p.step + step_off;
  // the binning's histograms are consumed: clear them for the next evaluation
  for (int64_t c = (int64_t)bid * NEAR_BLOCK + tid; c < (int64_t)p.ncell + p.nc[1] * p.nc[2];
       c += (int64_t)nbk * NEAR_BLOCK)
    p.cell_count[c] = 0;
  if (BUILD) {
    // automatic kept lists: only a step whose k_prepare raised the flag builds
    if (p.auto_lists && *(volatile const int *)p.lflag == 0) return;
    if (bid == 0 && tid == 0) atomicAdd(p.nbuild, 1ull);
  }
  const int warp = tid >> 5, lane = tid & 31;
  const int a = warp * APW + lane / TPA;      // atom row of the shared arrays
  const int g = lane % TPA;
  const int nrow = p.nc[1] * p.nc[2];
  const int chunk = bid * NEAR_WARPS + warp;
  double part[NEAR_NPART] = {};
  if (chunk < p.row_chunk[nrow]) {
    // ---- the chunk ------------------------------------------------------------
    const int2 cinfo = p.chunk_info[chunk];   // (row of cells, first slot)
    const int row = cinfo.x, base = cinfo.y;
    const int nc0 = p.nc[0];
    const int rend = p.cell_start[(row + 1) * nc0];
    const int cend = min(base + APW, rend);
    const int slot = base + lane / TPA;
    const uint4 u0 = p.su[min(slot, cend - 1)];
    const bool active = slot < cend && u0.w != SU_PAD;
    const int mslot = active ? slot : base;     // the first slot of a chunk is an atom
    const uint4 ui = active ? u0 : p.su[base];
    const float3 me = make_float3(p.sx[mslot], p.sy[mslot], p.sz[mslot]);
    const int spi = (int)(ui.w >> SU_SP_SHIFT);
    const Axis ay = make_axis(row % p.nc[1], p.nc[1]), az = make_axis(row / p.nc[1], p.nc[2]);
    const int nky = axis_count(ay, WRAP), nkz = axis_count(az, WRAP);
    const int nr = nky * nkz;
    const int cxi = cell_of(ui.x, nc0);
    const int cx_lo = __reduce_min_sync(0xffffffffu, cxi), cx_hi = __reduce_max_sync(0xffffffffu, cxi);
    const int W = cx_hi - cx_lo + STENCIL;     // union x-cells of the chunk
    const bool full = WRAP && W > nc0;         // the whole row (minimum image per pair)
    bool over = !full && W > WMAX;
    // ---- candidate runs and image shifts of the stencil rows ------------------
    // Rows of cells are sorted by x.  Without WRAP, lane r culls stencil row r
    // to the union, over the chunk's atoms, of the x-intervals that can hold a
    // neighbour (|dx| <= sqrt(r_s^2 - gap_y^2 - gap_z^2) with the gaps to the
    // row's y and z slabs, all widened), inside the union of their five-cell
    // x-stencils; the interval becomes one or two runs of slots by binary
    // search.  Runs are widened to whole groups of CELL_ALIGN slots: a slot
    // outside every atom's interval fails the predicate, and a slot in both
    // runs of a row passes for at most one of its two images (L >= 2 r_shell).
    float qx[APW], qy[APW], qz[APW];
#pragma unroll
    for (int q = 0; q < APW; q++) {
      qx[q] = __shfl_sync(0xffffffffu, me.x, TPA * q);
      qy[q] = __shfl_sync(0xffffffffu, me.y, TPA * q);
      qz[q] = __shfl_sync(0xffffffffu, me.z, TPA * q);
    }
    const uint32_t qact = __ballot_sync(0xffffffffu, active);   // bit TPA*q: atom q
    if (lane < nr) {
      const int kz = lane / nky, ky = lane - kz * nky;
      float shy, shz;
      const int cy = axis_cell(ay, ky, WRAP, shy);
      const int cz = axis_cell(az, kz, WRAP, shz);
      const int rb = nc0 * (cy + p.nc[1] * cz);
      const int rs0 = p.cell_start[rb], rs1 = p.cell_start[rb + nc0];   // the row (padded end)
      int a0 = 0, a1 = 0, b0 = 0, b1 = 0;
      float sa = 0.0f, sb = 0.0f;
      const int xs = cx_lo - 2, xe = cx_hi + 2;
      if (over) {                              // rejected chunk: empty rows
      } else if (WRAP) {
        if (full) {
          a0 = rs0; a1 = rs1;
        } else if (xs < 0) {                   // cells 0..xe, then nc0+xs..nc0-1
          a0 = rs0; a1 = p.cell_start[rb + xe + 1];
          b0 = p.cell_start[rb + nc0 + xs]; b1 = rs1;
        } else if (xe >= nc0) {                // cells 0..xe-nc0, then xs..nc0-1
          a0 = rs0; a1 = p.cell_start[rb + xe - nc0 + 1];
          b0 = p.cell_start[rb + xs]; b1 = rs1;
        } else {
          a0 = p.cell_start[rb + xs]; a1 = p.cell_start[rb + xe + 1];
        }
      } else {
        const float cwx = 8388608.0f / (float)nc0;
        const float cwy = 8388608.0f / (float)p.nc[1], cwz = 8388608.0f / (float)p.nc[2];
        const float ylo = __fmaf_rn((float)cy, cwy, shy) - 4.0f, yhi = __fmaf_rn((float)(cy + 1), cwy, shy) + 4.0f;
        const float zlo = __fmaf_rn((float)cz, cwz, shz) - 4.0f, zhi = __fmaf_rn((float)(cz + 1), cwz, shz) + 4.0f;
        const float cull2 = (BUILD ? p.rl2f : p.rs2f) * 1.0005f;
        const float unit = 1.0001f / p.hp[0];   // 23-bit units per Angstrom along x, widened
        float xlo = 3.0e7f, xhi = -3.0e7f;
#pragma unroll
        for (int q = 0; q < APW; q++) {
          if (!((qact >> (TPA * q)) & 1u)) continue;
          const float gy = fmaxf(0.0f, fmaxf(ylo - qy[q], qy[q] - yhi)) * p.hp[1];
          const float gz = fmaxf(0.0f, fmaxf(zlo - qz[q], qz[q] - zhi)) * p.hp[2];
          const float R2 = cull2 - gy * gy - gz * gz;
          if (R2 > 0.0f) {
            const float Rc = __fmaf_rn(sqrtf(R2), unit, 8.0f);
            xlo = fminf(xlo, qx[q] - Rc);
            xhi = fmaxf(xhi, qx[q] + Rc);
          }
        }
        xlo = fmaxf(xlo, (float)xs * cwx - 8.0f);
        xhi = fminf(xhi, (float)(xe + 1) * cwx + 8.0f);
        if (xlo <= xhi) {
          if (xlo < 0.0f) {                    // [0, xhi], then [xlo + 2^23, 2^23) at image -L
            a0 = rs0; a1 = sx_bound(p, rb, xhi, true);
            b0 = sx_bound(p, rb, xlo + 8388608.0f, false); b1 = rs1; sb = -8388608.0f;
          } else if (xhi >= 8388608.0f) {      // [0, xhi - 2^23] at image +L, then [xlo, 2^23)
            a0 = rs0; a1 = sx_bound(p, rb, xhi - 8388608.0f, true); sa = 8388608.0f;
            b0 = sx_bound(p, rb, xlo, false); b1 = rs1;
          } else {
            a0 = sx_bound(p, rb, xlo, false); a1 = sx_bound(p, rb, xhi, true);
          }
        }
      }
      a0 &= ~(CELL_ALIGN - 1);
      a1 = max(a0, min((a1 + CELL_ALIGN - 1) & ~(CELL_ALIGN - 1), rs1));
      b0 &= ~(CELL_ALIGN - 1);
      b1 = max(b0, min((b1 + CELL_ALIGN - 1) & ~(CELL_ALIGN - 1), rs1));
      if (WRAP && b1 > b0 && a1 >= b0) {      // touching runs of one image order merge
        a1 = b1;
        b0 = b1 = 0;
      }
      rseg[warp][lane] = make_int4(a0, a1 - a0, b0, b1 - b0);
      rsh[warp][lane] = make_float4(sa, sb, shy, shz);
    }
    // ---- flattened groups of four candidates: row r holds groups
    // [rgo[r], rgo[r+1]) and bytes [rbo[r], rbo[r] + groups) of gres ----------
    {
      const int len = lane < nr ? rseg[warp][lane].y + rseg[warp][lane].w : 0;
      if (len > RBSOG_MAX_ROW_SLOTS) over = true;
      const int ng = len / CELL_ALIGN, nbyte = (ng + 3) & ~3;
      int ig = ng, ib = nbyte;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y1 = __shfl_up_sync(0xffffffffu, ig, o), y2 = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) { ig += y1; ib += y2; }
      }
      if (lane < nr) {
        rgo[warp][lane] = ig - ng;
        rbo[warp][lane] = ib - nbyte;
      }
      if (lane == 31) rgo[warp][nr] = ig;
      if (__shfl_sync(0xffffffffu, ib, 31) > GBYTES) over = true;
    }
    over = __any_sync(0xffffffffu, over);
    __syncwarp();
    // ---- pass 1: the chunk's groups dealt round-robin over an atom's four
    // threads (all eight atoms test the same group at the same time) ---------
    const float outer2 = BUILD ? p.rl2f : p.rs2f;
    const unsigned long long RS2 = pk2(-outer2, -outer2), RC2 = pk2(-p.rc2f, -p.rc2f);
    if (!over) {
      const int G = rgo[warp][nr];
      int r = -1, rg0 = 0, rg1 = 0, bo = 0;
      int4 sg = make_int4(0, 0, 0, 0);
      PredX4 pc = pred_x4_setup(me.x, me.y, me.z, p.hp);
      unsigned long long nxa = 0ull, nxb = 0ull;
      for (int gi = g; gi < G; gi += TPA) {
        if (gi >= rg1) {                          // next row holding group gi
          do { r++; rg1 = rgo[warp][r + 1]; } while (gi >= rg1);
          rg0 = rgo[warp][r];
          bo = rbo[warp][r];
          sg = rseg[warp][r];
          const float4 sh = rsh[warp][r];
          pc = pred_x4_setup(me.x - sh.x, me.y - sh.z, me.z - sh.w, p.hp);
          nxa = pc.nx;
          nxb = pk2(sh.y - me.x, sh.y - me.x);
        }
        const int pos = CELL_ALIGN * (gi - rg0);
        const bool inb = pos >= sg.y;
        const int j0 = inb ? sg.z + (pos - sg.y) : sg.x + pos;
        unsigned long long q0, q1;
        if (WRAP) {
          float r2v[4];
          pred_r2_x4_wrap(p, j0, me.x, me.y, me.z, r2v);
          q0 = pk2(r2v[0], r2v[1]);
          q1 = pk2(r2v[2], r2v[3]);
        } else {
          pc.nx = inb ? nxb : nxa;
          pred_r2_x4_packed(p.sx, p.sy, p.sz, j0, pc, q0, q1);
        }
        // sign of r^2 - threshold: set iff r^2 < threshold (r^2 = +inf at pads)
        float s0, s1, s2, s3, c0, c1, c2, c3;
        up2(add2(q0, RS2), s0, s1);
        up2(add2(q1, RS2), s2, s3);
        up2(add2(q0, RC2), c0, c1);
        up2(add2(q1, RC2), c2, c3);
        uint32_t bits = __float_as_uint(c3) >> 31;
        bits = __funnelshift_l(__float_as_uint(c2), bits, 1);
        bits = __funnelshift_l(__float_as_uint(c1), bits, 1);
        bits = __funnelshift_l(__float_as_uint(c0), bits, 1);
        bits = __funnelshift_l(__float_as_uint(s3), bits, 1);
        bits = __funnelshift_l(__float_as_uint(s2), bits, 1);
        bits = __funnelshift_l(__float_as_uint(s1), bits, 1);
        bits = __funnelshift_l(__float_as_uint(s0), bits, 1);
        const unsigned d = (unsigned)(slot - j0);
        if (d < 4u) bits &= ~(0x11u << d);        // not the atom itself
        gres[a][bo + (pos >> 2)] = (unsigned char)bits;
      }
    }
    __syncwarp();
    // ---- species-dependent core radii: a core member (tested against the
    // largest radius) whose pair radius is smaller moves to the shell; its
    // predicate value is recomputed exactly (the minimum-image difference of
    // 23-bit coordinates is an exact integer, as in the tests above) --------
    if (p.core_pair) {                          // warp-uniform: every lane meets the barrier below
      for (int r = g; active && !over && r < nr; r += TPA) {
        const int ng = rgo[warp][r + 1] - rgo[warp][r];
        const int4 sg = rseg[warp][r];
        unsigned char *gb = &gres[a][rbo[warp][r]];
        for (int gi = 0; gi < ng; gi++) {
          uint32_t x = gb[gi];
          uint32_t cm = (x >> 4) & 0xFu;
          while (cm) {
            const int b = __ffs(cm) - 1;
            cm &= cm - 1u;
            const uint4 uj = p.su[row_slot(sg, CELL_ALIGN * gi + b)];
            const float r2 = pred_r2((float)wrap23(uj.x, ui.x), (float)wrap23(uj.y, ui.y),
                                     (float)wrap23(uj.z, ui.z), p.hp);
            if (!(r2 < p.rc2p[spi * p.ns + (int)(uj.w >> SU_SP_SHIFT)])) x &= ~(0x10u << b);
          }
          gb[gi] = (unsigned char)x;
        }
      }
      __syncwarp();
    }
    // ---- shell counts of the rows r = g, g + 4, ...; the atom's core list -----
    int my_total = 0, mycore = 0;
    if (!over) {
      for (int r = g; r < nr; r += TPA) {
        const int ng = rgo[warp][r + 1] - rgo[warp][r];
        const uint32_t *wp = reinterpret_cast<const uint32_t *>(&gres[a][rbo[warp][r]]);
        int cnt = 0, cc = 0;
        for (int w = 0; 4 * w < ng; w++) {
          uint32_t x = wp[w];
          if (ng - 4 * w < 4) x &= (1u << (8 * (ng - 4 * w))) - 1u;   // groups past the row
          const uint32_t cm = (x >> 4) & 0x0F0F0F0Fu;
          cnt += __popc(x & 0x0F0F0F0Fu & ~cm);
          cc += __popc(cm);
        }
        scnt[a][r] = (unsigned char)min(cnt, 255);
        if (BUILD) ccnt[a][r] = (unsigned char)min(cc, 255);
        my_total += cnt;
        mycore += cc;
      }
    }
    if constexpr (BUILD) {
      // ---- kept lists: each thread writes the members of its rows at the
      // row's offset in the canonical order (prefix of the row counts) -------
      int nb = my_total, na = mycore;
#pragma unroll
      for (int o = 1; o < TPA; o <<= 1) {
        nb += __shfl_xor_sync(0xffffffffu, nb, o, TPA);
        na += __shfl_xor_sync(0xffffffffu, na, o, TPA);
      }
      const bool ok = active && !over && na <= RBSOG_MAX_CORE && nb <= RBSOG_MAX_KEPT;
      if (active && g == 0 && !ok) atomicOr(p.err, over ? ERR_CELL_SHELL_CAP : ERR_KEPT_CAP);
      __syncwarp();
      if (ok) {
        int accB = 0, accA = 0;
        for (int q = 0; q < g && q < nr; q++) {
          accB += scnt[a][q];
          accA += ccnt[a][q];
        }
        int *dA = p.lA + (int64_t)slot * RBSOG_MAX_CORE;
        int *dB = p.lB + (int64_t)slot * RBSOG_MAX_KEPT;
        unsigned short *dB16 = p.lB16 + (int64_t)slot * RBSOG_MAX_KEPT;
        const int M = p.cell_start[p.ncell];
        bool fits = true;
        for (int r = g; r < nr; r += TPA) {
          const int ng = rgo[warp][r + 1] - rgo[warp][r];
          const int4 sg = rseg[warp][r];
          const uint32_t *wp = reinterpret_cast<const uint32_t *>(&gres[a][rbo[warp][r]]);
          for (int w = 0; 4 * w < ng; w++) {
            uint32_t x = wp[w];
            if (ng - 4 * w < 4) x &= (1u << (8 * (ng - 4 * w))) - 1u;
            uint32_t cm = (x >> 4) & 0x0F0F0F0Fu;
            uint32_t sm = x & 0x0F0F0F0Fu & ~cm;
            while (cm) {
              const int b = __ffs(cm) - 1;
              cm &= cm - 1u;
              dA[accA++] = row_slot(sg, 16 * w + 4 * (b >> 3) + (b & 3));
            }
            while (sm) {
              const int b = __ffs(sm) - 1;
              sm &= sm - 1u;
              const int j = row_slot(sg, 16 * w + 4 * (b >> 3) + (b & 3));
              unsigned short e;
              fits &= kept_b16_encode(j, slot, M, e);
              dB16[accB] = e;
              dB[accB++] = j;
            }
          }
          for (int q = r + 1; q < min(r + TPA, nr); q++) {
            accB += scnt[a][q];
            accA += ccnt[a][q];
          }
        }
        if (!fits) atomicOr(p.b16_over, 1);
      }
      if (active && g == 0) p.nAB[slot] = ok ? make_int2(na, nb) : make_int2(0, 0);
      return;
    }
    if (!active) { my_total = 0; mycore = 0; over = false; }
    int cbase = mycore;                          // this thread's offset in the atom's core list
#pragma unroll
    for (int o = 1; o < TPA; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, cbase, o, TPA);
      if (g >= o) cbase += y;
    }
    const int ncore = __shfl_sync(0xffffffffu, cbase, TPA - 1, TPA);
    cbase -= mycore;
    if (active && !over && ncore <= RBSOG_MAX_CORE) {
      for (int r = g; r < nr; r += TPA) {
        const int ng = rgo[warp][r + 1] - rgo[warp][r];
        const uint32_t *wp = reinterpret_cast<const uint32_t *>(&gres[a][rbo[warp][r]]);
        for (int w = 0; 4 * w < ng; w++) {
          uint32_t x = wp[w];
          if (ng - 4 * w < 4) x &= (1u << (8 * (ng - 4 * w))) - 1u;
          uint32_t cm = (x >> 4) & 0x0F0F0F0Fu;
          while (cm) {
            const int b = __ffs(cm) - 1;
            cm &= cm - 1u;
            score[a][cbase++] = (unsigned short)((r << 7) | (16 * w + 4 * (b >> 3) + (b & 3)));
          }
        }
      }
    }
    if (active && ncore > RBSOG_MAX_CORE) over = true;
    if (over) atomicOr(p.err, (active && ncore > RBSOG_MAX_CORE) ? ERR_CORE_CAP : ERR_CELL_SHELL_CAP);
    // ---- pass 2: prefix of the row counts, Floyd's draw ---------------------------
    int nshell = my_total;
#pragma unroll
    for (int o = 1; o < TPA; o <<= 1) nshell += __shfl_xor_sync(0xffffffffu, nshell, o, TPA);
    const bool take_all = p.whole_shell || nshell <= p.P_R;
    const bool sampled = active && !take_all && nshell <= SHELL_BITS;
    if (active && !take_all && nshell > SHELL_BITS && g == 0) atomicOr(p.err, ERR_CELL_SHELL_CAP);
    const int PR = p.P_R;
    __syncwarp();
    if (sampled) {
      int acc = 0;
      for (int q = 0; q < g; q++) acc += scnt[a][q];
      for (int r = g; r < nr; r += TPA) {
        spre[a][r] = (unsigned short)acc;
        for (int q = r; q < min(r + TPA, nr); q++) acc += scnt[a][q];
      }
      if (g == 0) spre[a][nr] = (unsigned short)nshell;
      for (int w = g; w < ((nshell + 31) >> 5); w += TPA) bmask[a][w] = 0u;
      const uint32_t id = ui.w & SU_ID_MASK;
      for (int d = g; 2 * d < PR; d += TPA) {     // Philox word d serves samples 2d, 2d + 1
        const uint4 w4 = draw(p.seed, s, id, 0u, (uint32_t)d);
        const unsigned long long U0 = ((unsigned long long)w4.y << 32) | w4.x;
        const unsigned long long U1 = ((unsigned long long)w4.w << 32) | w4.z;
        const int r0 = 2 * d;
        stsel[a][r0] = (unsigned short)__umul64hi(U0, (unsigned long long)(nshell - PR + r0) + 1ull);
        if (r0 + 1 < PR)
          stsel[a][r0 + 1] = (unsigned short)__umul64hi(U1, (unsigned long long)(nshell - PR + r0 + 1) + 1ull);
      }
    }
    __syncwarp();
    if (sampled && g == 0) {
      uint32_t *bm = bmask[a];
      for (int r = 0; r < PR; r++) {
        uint32_t t = stsel[a][r];
        if ((bm[t >> 5] >> (t & 31)) & 1u) t = (uint32_t)(nshell - PR + r);
        bm[t >> 5] |= 1u << (t & 31);
        stsel[a][r] = (unsigned short)t;
      }
    }
    __syncwarp();
    Acc<R> fc, fs;
    R wgt = 1;
    if (sampled) wgt = (R)nshell / (R)PR;
    // shell member position of row r -> slot; the shell bits of gres word x
    auto shell_bits = [&](int r, int w, int ng) -> uint32_t {
      uint32_t x = reinterpret_cast<const uint32_t *>(&gres[a][rbo[warp][r]])[w];
      if (ng - 4 * w < 4) x &= (1u << (8 * (ng - 4 * w))) - 1u;
      return x & 0x0F0F0F0Fu & ~((x >> 4) & 0x0F0F0F0Fu);
    };
    if (active) {
      if (sampled) {
        // ---- pass 3: the sampled shell members, four at a time per thread ------
        for (int k0 = g; k0 < PR; k0 += 4 * TPA) {
          int js[4];
#pragma unroll
          for (int i = 0; i < 4; i++) {
            const int k = k0 + TPA * i;
            js[i] = -1;
            if (k < PR) {
              const int t = stsel[a][k];
              int lo = 0, hi = nr - 1;            // last row with prefix <= t
              while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (spre[a][mid] <= t) lo = mid; else hi = mid - 1;
              }
              int rank = t - spre[a][lo];
              const int ng = rgo[warp][lo + 1] - rgo[warp][lo];
              for (int w = 0; 4 * w < ng; w++) {
                const uint32_t m = shell_bits(lo, w, ng);
                const int c = __popc(m);
                if (rank < c) {
                  const int b = select_bit(m, rank);
                  js[i] = row_slot(rseg[warp][lo], 16 * w + 4 * (b >> 3) + (b & 3));
                  break;
                }
                rank -= c;
              }
            }
          }
          uint4 uj[4];
#pragma unroll
          for (int i = 0; i < 4; i++) uj[i] = p.su[max(js[i], 0)];
#pragma unroll
          for (int i = 0; i < 4; i++)
            if (js[i] >= 0) add_pair<R, ENERGY>(p, spf, spd, sg4, swa, sw, sh2, spi, ui, uj[i], fs);
        }
      } else if (take_all && !over) {
        // whole shell, weight 1: every shell member of the thread's rows (a
        // chunk rejected for overlong rows has no shell bits: its rows may
        // reach past gres; the overflow is reported through p.err)
        for (int r = g; r < nr; r += TPA) {
          const int ng = rgo[warp][r + 1] - rgo[warp][r];
          const int4 sg = rseg[warp][r];
          for (int w = 0; 4 * w < ng; w++) {
            uint32_t m = shell_bits(r, w, ng);
            while (m) {
              const int b = __ffs(m) - 1;
              m &= m - 1u;
              add_pair<R, ENERGY>(p, spf, spd, sg4, swa, sw, sh2, spi, ui,
                                  p.su[row_slot(sg, 16 * w + 4 * (b >> 3) + (b & 3))], fs);
            }
          }
        }
      }
    }
    // ---- pass 4: exact core sum, the atom's core list dealt over its threads ----
    __syncwarp();
    if (active && ncore <= RBSOG_MAX_CORE) {
      for (int e0 = g; e0 < ncore; e0 += 4 * TPA) {
        int js[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
          const int e = e0 + TPA * i;
          js[i] = -1;
          if (e < ncore) {
            const int code = score[a][e];
            js[i] = row_slot(rseg[warp][code >> 7], code & 127);
          }
        }
        uint4 uj[4];
#pragma unroll
        for (int i = 0; i < 4; i++) uj[i] = p.su[max(js[i], 0)];
#pragma unroll
        for (int i = 0; i < 4; i++)
          if (js[i] >= 0) add_pair<R, ENERGY>(p, spf, spd, sg4, swa, sw, sh2, spi, ui, uj[i], fc);
      }
    }
    combine_atom<R, ENERGY>(p, fc, fs, wgt, active, g, ui, part);
  }
  if constexpr (BUILD) return;
  // ---- partials of sum F_N and of the pair energy, one per warp (FP32 sums of
  // the warp's eight atoms in mixed precision, FP64 otherwise) ----------------
  warp_partials<MIX, ENERGY ? NEAR_NPART : 4>(p, part, bid * NEAR_WARPS + warp, lane);
}

template <typename R, bool WRAP, bool ENERGY, bool BUILD>
__global__ void __launch_bounds__(NEAR_BLOCK, 4) k_near(View p, int step_off) {
  near_body<R, WRAP, ENERGY, BUILD>(p, step_off, blockIdx.x, gridDim.x);
}
template <bool WRAP, bool BUILD>
__global__ void __launch_bounds__(NEAR_BLOCK, 4) kp_near(Pack pk, int step_off) {
  RB_PACK_PROLOGUE(pk);
  near_body<float, WRAP, false, BUILD>(sv, step_off, bid, nb);
}

void launch_near(const View &v, cudaStream_t st, int step_off, bool energy) {
  const dim3 g(v.nblk_near), b(NEAR_BLOCK);  // one warp per chunk
#define RB_NEAR(R, WR, EN) k_near<R, WR, EN, false><<<g, b, 0, st>>>(v, step_off)
  if (v.prec == RBSOG_MIXED) {
    if (v.wrap) { if (energy) RB_NEAR(float, true, true); else RB_NEAR(float, true, false); }
    else { if (energy) RB_NEAR(float, false, true); else RB_NEAR(float, false, false); }
  } else {
    if (v.wrap) { if (energy) RB_NEAR(double, true, true); else RB_NEAR(double, true, false); }
    else { if (energy) RB_NEAR(double, false, true); else RB_NEAR(double, false, false); }
  }
#undef RB_NEAR
}

void launch_build_lists(const View &v, cudaStream_t st) {
  const dim3 g(v.nblk_near), b(NEAR_BLOCK);
  if (v.wrap) k_near<float, true, false, true><<<g, b, 0, st>>>(v, 0);
  else k_near<float, false, false, true><<<g, b, 0, st>>>(v, 0);
}

// ---------------------------------------------------------------------------
// Near field with kept lists (Sec. 2.2 over the lists of the last build):
// one warp per run of NEAR_CHUNK consecutive slots of that build, TPA threads
// per atom.  A is summed exactly; B by Floyd's P_R of |B| (Philox stream 0,
// as the per-step batch) with weight |B| / P_R, or whole with weight 1 when
// |B| <= P_R; every term carries the indicator r < r_shell, the FP32 list
// predicate on the current minimum-image 23-bit differences.

// the list predicate between two current fixed-point positions
__device__ __forceinline__ bool in_shell(const View &p, uint4 ui, uint4 uj) {
  return pred_r2((float)wrap23(uj.x, ui.x), (float)wrap23(uj.y, ui.y), (float)wrap23(uj.z, ui.z), p.hp) <
         p.rs2f;
}

// Pair force with the mixed pair record read from the block's shared copy
// of the table (three 16-byte words per species pair).
template <bool ENERGY>
__device__ __forceinline__ void add_pair_sh(const View &p, const float4 *spf4, const float4 *sg, int spi,
                                            uint4 ui, uint4 uj, Acc<float> &a) {
  const int spj = (int)(uj.w >> SU_SP_SHIFT);
  const float4 *src = spf4 + 3 * (spi * p.ns + spj);
  const float4 r0 = src[0], r1 = src[1], r2 = src[2];
  PairF q;
  q.kqq = r0.x; q.Ar = r0.y; q.lr = r0.z; q.sig = r0.w;
  q.C6 = r1.x; q.D8 = r1.y; q.A = r1.z; q.C = r1.w;
  q.D = r2.x;
  float a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  pair_mixed<ENERGY>(p, q, sg, ui, uj, a0, a1, a2, a3, a.w);
  a.x += a0; a.y += a1; a.z += a2; a.e += a3;
}

// KB batch members in flight per thread (TPA * KB = 20 = P_R of the
// benchmark: one pass with every lane busy).
constexpr int KB = 5;

// The shell batch of every slot with kept lists (Sec. 2.2, F*_shell): Floyd's
// P_R of |B| from the slot's Philox words (the same draws and resolution as
// floyd()), the drawn members' slots written to bsel[slot][r] in draw order.
// The batch depends on the step, the caller id and the lists, not on the
// positions, so it is drawn in a kernel of its own ahead of the pair sums.
// Same block layout as the pair kernel: a warp per run of APW slots, TPA
// threads per atom (the Philox words in parallel, the resolution by the
// first); each thread then gathers its SB_LOADS drawn entries with all loads
// in flight before any store (the list is read-only here).
constexpr int SB_LOADS = 8;
__device__ __forceinline__ void sample_batch_body(const View &p, int step_off, int bid) {
  __shared__ unsigned short stsel[APB][RBSOG_MAX_PR + 2];
  __shared__ uint32_t bmask[APB][RBSOG_MAX_KEPT / 32 + 1];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int a = warp * APW + lane / TPA, g = lane % TPA;
  const long long s = *p.step + step_off;
  const int nslot = p.cell_start[p.ncell];
  const int slot = (bid * NEAR_WARPS + warp) * APW + lane / TPA;
  // the slot record and the counts are read for any slot within the slot
  // buffers' capacity, together with the slot count that masks them (three
  // loads in flight instead of one after another)
  const bool cap = slot < p.nslot;
  const uint32_t w0 = cap ? p.su[slot].w : SU_PAD;
  const int nB0 = cap ? p.nAB[slot].y : 0;
  const uint32_t w = slot < nslot ? w0 : SU_PAD;
  const bool active = w != SU_PAD;
  const int nB = active ? nB0 : 0, PR = p.P_R;
  const bool sampled = active && !p.whole_shell && nB > PR;
  const bool b16 = !p.kept_wide && *p.b16_over == 0;   // every offset of the last build fits 16 bits
  if (sampled) {
    for (int q = g; q < ((nB + 31) >> 5); q += TPA) bmask[a][q] = 0u;
    const uint32_t id = w & SU_ID_MASK;
    for (int d = g; 2 * d < PR; d += TPA) {     // Philox word d serves draws 2d, 2d + 1
      const uint4 w4 = draw(p.seed, s, id, 0u, (uint32_t)d);
      const unsigned long long U0 = ((unsigned long long)w4.y << 32) | w4.x;
      const unsigned long long U1 = ((unsigned long long)w4.w << 32) | w4.z;
      const int r0 = 2 * d;
      stsel[a][r0] = (unsigned short)__umul64hi(U0, (unsigned long long)(nB - PR + r0) + 1ull);
      if (r0 + 1 < PR)
        stsel[a][r0 + 1] = (unsigned short)__umul64hi(U1, (unsigned long long)(nB - PR + r0 + 1) + 1ull);
    }
  }
  __syncwarp();                                  // this warp's draws
  if (sampled && g == 0) {
    uint32_t *bm = bmask[a];
    for (int r = 0; r < PR; r++) {
      uint32_t t = stsel[a][r];
      if ((bm[t >> 5] >> (t & 31)) & 1u) t = (uint32_t)(nB - PR + r);
      bm[t >> 5] |= 1u << (t & 31);
      stsel[a][r] = (unsigned short)t;
    }
  }
  __syncwarp();
  if (sampled) {
    int *out = p.bsel + (int64_t)slot * PR;
    if (b16) {                                   // half the bytes of B's row per draw
      const unsigned short *lb = p.lB16 + (int64_t)slot * RBSOG_MAX_KEPT;
      for (int k0 = g; k0 < PR; k0 += TPA * SB_LOADS) {
        unsigned short e[SB_LOADS];
#pragma unroll
        for (int i = 0; i < SB_LOADS; i++) {
          const int k = k0 + TPA * i;
          e[i] = k < PR ? __ldg(lb + stsel[a][k]) : (unsigned short)0;
        }
#pragma unroll
        for (int i = 0; i < SB_LOADS; i++)
          if (k0 + TPA * i < PR) out[k0 + TPA * i] = kept_b16_decode(e[i], slot, nslot);
      }
    } else {
      const int *lb = p.lB + (int64_t)slot * RBSOG_MAX_KEPT;
      for (int k0 = g; k0 < PR; k0 += TPA * SB_LOADS) {
        int e[SB_LOADS];
#pragma unroll
        for (int i = 0; i < SB_LOADS; i++) {
          const int k = k0 + TPA * i;
          e[i] = k < PR ? __ldg(lb + stsel[a][k]) : 0;
        }
#pragma unroll
        for (int i = 0; i < SB_LOADS; i++)
          if (k0 + TPA * i < PR) out[k0 + TPA * i] = e[i];
      }
    }
  }
}
__global__ void __launch_bounds__(NEAR_BLOCK) k_sample_batch(View p, int step_off) {
  sample_batch_body(p, step_off, blockIdx.x);
}
__global__ void __launch_bounds__(NEAR_BLOCK) kp_sample_batch(Pack pk, int step_off) {
  RB_PACK_PROLOGUE_REF(pk);
  (void)nb;
  sample_batch_body(sv, step_off, bid);
}
void launch_sample_batch(const View &v, cudaStream_t st, int step_off) {
  k_sample_batch<<<v.nblk_near, NEAR_BLOCK, 0, st>>>(v, step_off);
}

template <typename R, bool ENERGY, bool WIDE, bool CAPPED>
__device__ __forceinline__ void near_kept_body(const View &p, int step_off, int bid, int nbk) {
  constexpr bool MIX = sizeof(R) == 4;
  __shared__ float4 spf4[MIX ? 3 * RBSOG_MAX_SPECIES * RBSOG_MAX_SPECIES : 1];
  const PairD *spd = p.pd;
  const float4 *sg4 = p.gtab;
  const double *swa = p.sog_wa, *sw = p.sog_w, *sh2 = p.sog_h;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane % TPA;
  (void)step_off;                                // the batch of this step is drawn by k_sample_batch
  const int nslot = p.cell_start[p.ncell];       // in flight while the pair table is staged
  if (MIX) {
    const float4 *src = reinterpret_cast<const float4 *>(p.pf);
    for (int e = tid; e < 3 * p.ns * p.ns; e += NEAR_BLOCK) spf4[e] = __ldg(src + e);
  }
  const int PR = p.P_R;
  bool first = true;
  // one warp per run of APW slots; a grid smaller than nblk_near (a capped
  // number of resident blocks) takes the runs in a grid-stride loop (every
  // warp of a block makes the same number of passes, at least one)
  for (int wc = bid * NEAR_WARPS + warp; wc < p.nblk_near * NEAR_WARPS; wc += nbk * NEAR_WARPS) {
  const int slot = wc * APW + lane / TPA;
  const bool inrange = slot < nslot;
  // the slot record, the counts, the batch row and the first round of A's
  // row are all issued at once (the rows' addresses depend on the slot only:
  // rows of the last build, valid memory for every slot); the counts mask
  // them below
  const int cs = inrange ? slot : 0;
  const uint4 ui = inrange ? p.su[cs] : make_uint4(0u, 0u, 0u, SU_PAD);
  const int2 nab0 = inrange ? p.nAB[cs] : make_int2(0, 0);
  const int *la = p.lA + (int64_t)cs * RBSOG_MAX_CORE;
  int jbs[KB], ja0[4];
#pragma unroll
  for (int i = 0; i < KB; i++) {
    const int k = g + TPA * i;
    jbs[i] = (inrange && k < PR) ? __ldg(p.bsel + (int64_t)cs * PR + k) : -1;
  }
#pragma unroll
  for (int i = 0; i < 4; i++) ja0[i] = inrange ? __ldg(la + g + TPA * i) : -1;
  if (MIX && first) __syncthreads();             // the pair table (these loads in flight meanwhile)
  first = false;
  const bool active = ui.w != SU_PAD;
  const int2 nab = active ? nab0 : make_int2(0, 0);
  const int spi = active ? (int)(ui.w >> SU_SP_SHIFT) : 0;
  double part[NEAR_NPART] = {};
  Acc<R> fa, fb;
  // ---- the batch (drawn by k_sample_batch) or all of B ----------------------
  const int nB = nab.y;
  const bool sampled = active && !p.whole_shell && nB > PR;
  const R wgt = sampled ? (R)nB / (R)PR : (R)1;
  const int *lb = sampled ? p.bsel + (int64_t)cs * PR : p.lB + (int64_t)cs * RBSOG_MAX_KEPT;
  const int nb = sampled ? PR : nB;
  int jb[KB];
#pragma unroll
  for (int i = 0; i < KB; i++) {
    const int k = g + TPA * i;
    jb[i] = sampled ? jbs[i] : (k < nb ? lb[k] : -1);
  }
  // ---- A, exactly, dealt round-robin over the atom's threads; the
  // indicator r < r_shell is 1 for every member of A when r_core + skin lies
  // well inside r_shell (no atom moves by more than skin/2 between builds) -----
  const bool acheck = !p.a_inside;
  int a_from = g, b_from = 0;                    // where the loops below start
  if (WIDE) {
    // a thread's first eight members of A and its first batch members are all
    // gathered before any pair is evaluated (13 independent loads in flight);
    // the members are visited in the same order as below, so the sums are
    // the same bit for bit
    int jsA[8];
#pragma unroll
    for (int i = 0; i < 8; i++) jsA[i] = (g + TPA * i < nab.x) ? la[g + TPA * i] : -1;
    uint4 uA[8], uB[KB];
#pragma unroll
    for (int i = 0; i < 8; i++) uA[i] = p.su[max(jsA[i], 0)];
#pragma unroll
    for (int i = 0; i < KB; i++) uB[i] = p.su[max(jb[i], 0)];
#pragma unroll
    for (int i = 0; i < 8; i++)
      if (jsA[i] >= 0 && (!acheck || in_shell(p, ui, uA[i]))) {
        if constexpr (MIX) add_pair_sh<ENERGY>(p, spf4, sg4, spi, ui, uA[i], fa);
        else add_pair<R, ENERGY>(p, nullptr, spd, sg4, swa, sw, sh2, spi, ui, uA[i], fa);
      }
#pragma unroll
    for (int i = 0; i < KB; i++)
      if (jb[i] >= 0 && in_shell(p, ui, uB[i])) {
        if constexpr (MIX) add_pair_sh<ENERGY>(p, spf4, sg4, spi, ui, uB[i], fb);
        else add_pair<R, ENERGY>(p, nullptr, spd, sg4, swa, sw, sh2, spi, ui, uB[i], fb);
      }
    a_from = g + 8 * TPA;
    b_from = TPA * KB;
#pragma unroll
    for (int i = 0; i < KB; i++) {
      const int k = b_from + g + TPA * i;
      jb[i] = k < nb ? lb[k] : -1;
    }
  }
  for (int e0 = a_from; e0 < nab.x; e0 += 4 * TPA) {
    int js[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
      const int e = e0 + TPA * i;
      js[i] = e < nab.x ? ((!WIDE && e0 == g) ? ja0[i] : la[e]) : -1;   // the first round was issued above
    }
    uint4 uj[4];
#pragma unroll
    for (int i = 0; i < 4; i++) uj[i] = p.su[max(js[i], 0)];
#pragma unroll
    for (int i = 0; i < 4; i++)
      if (js[i] >= 0 && (!acheck || in_shell(p, ui, uj[i]))) {
        if constexpr (MIX) add_pair_sh<ENERGY>(p, spf4, sg4, spi, ui, uj[i], fa);
        else add_pair<R, ENERGY>(p, nullptr, spd, sg4, swa, sw, sh2, spi, ui, uj[i], fa);
      }
  }
  // ---- the batch of B (or all of it) ---------------------------------------
  for (int k0 = b_from;; k0 += TPA * KB) {
    if (WIDE && k0 >= nb) break;
    uint4 uj[KB];
#pragma unroll
    for (int i = 0; i < KB; i++) uj[i] = p.su[max(jb[i], 0)];
#pragma unroll
    for (int i = 0; i < KB; i++)
      if (jb[i] >= 0 && in_shell(p, ui, uj[i])) {
        if constexpr (MIX) add_pair_sh<ENERGY>(p, spf4, sg4, spi, ui, uj[i], fb);
        else add_pair<R, ENERGY>(p, nullptr, spd, sg4, swa, sw, sh2, spi, ui, uj[i], fb);
      }
    if (k0 + TPA * KB >= nb) break;             // rare: P_R or |B| above TPA * KB
#pragma unroll
    for (int i = 0; i < KB; i++) {
      const int k = k0 + TPA * KB + g + TPA * i;
      jb[i] = k < nb ? lb[k] : -1;
    }
  }
  combine_atom<R, ENERGY>(p, fa, fb, wgt, active, g, ui, part);
  warp_partials<MIX, ENERGY ? NEAR_NPART : 4>(p, part, wc, lane);
  if (!CAPPED) break;                            // a warp per run: one pass
  }
}

// FP32 pair math: registers bounded for 7 resident blocks per SM (64 in the
// default form, no spills); FP64: 4 (its pair terms need more registers)
template <typename R, bool ENERGY, bool WIDE, bool CAPPED>
__global__ void __launch_bounds__(NEAR_BLOCK, sizeof(R) == 4 ? 7 : 4) k_near_kept(View p, int step_off) {
  near_kept_body<R, ENERGY, WIDE, CAPPED>(p, step_off, blockIdx.x, gridDim.x);
}
template <bool WIDE>
__global__ void __launch_bounds__(NEAR_BLOCK, 4) kp_near_kept(Pack pk, int step_off) {
  RB_PACK_PROLOGUE(pk);
  near_kept_body<float, false, WIDE, false>(sv, step_off, bid, nb);
}

void launch_near_kept(const View &v, cudaStream_t st, int step_off, bool energy) {
  // near_bps > 0: at most that many resident blocks per SM, looping over the
  // runs, so that the far-field branch always finds free slots
  const int nb = v.near_bps > 0 ? std::min(v.nblk_near, v.near_bps * v.nsm) : v.nblk_near;
  const dim3 g(nb), b(NEAR_BLOCK);
  const bool cap = v.near_bps > 0;
#define RB_KEPT(R, EN, WI)                                                    \
  do {                                                                        \
    if (cap) k_near_kept<R, EN, WI, true><<<g, b, 0, st>>>(v, step_off);      \
    else k_near_kept<R, EN, WI, false><<<g, b, 0, st>>>(v, step_off);         \
  } while (0)
  if (v.prec == RBSOG_MIXED) {
    if (energy) RB_KEPT(float, true, false);
    else if (v.near_wide) RB_KEPT(float, false, true);
    else RB_KEPT(float, false, false);
  } else {
    if (energy) RB_KEPT(double, true, false);
    else RB_KEPT(double, false, false);
  }
#undef RB_KEPT
}

// Parity hook: the kept lists of selected atoms (caller ids, canonical order)
// and the batch the current step draws from B (same Floyd routine).
__global__ void k_kept_lists(View p, int step_off, const long long *sel, int nsel, int cap_a, int cap_b,
                             int *A, int *nA, int *B, int *nB, int *batch, int *nbatch, double *weight) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nsel) return;
  const long long s = *p.step + step_off;
  const int slot = p.slot_of[sel[q]];
  const int2 nab = p.nAB[slot];
  const int *la = p.lA + (int64_t)slot * RBSOG_MAX_CORE;
  const int *lb = p.lB + (int64_t)slot * RBSOG_MAX_KEPT;
  for (int k = 0; k < nab.x && k < cap_a; k++) A[(long long)q * cap_a + k] = p.perm[la[k]];
  for (int k = 0; k < nab.y && k < cap_b; k++) B[(long long)q * cap_b + k] = p.perm[lb[k]];
  nA[q] = nab.x;
  nB[q] = nab.y;
  if (batch) {
    const bool take_all = p.whole_shell || nab.y <= p.P_R;
    int t[RBSOG_MAX_PR];
    const int m = take_all ? nab.y : p.P_R;
    if (!take_all) floyd(p, s, sel[q], nab.y, t);
    for (int k = 0; k < m && k < p.P_R; k++) batch[(long long)q * p.P_R + k] = p.perm[lb[take_all ? k : t[k]]];
    nbatch[q] = m;
    weight[q] = take_all ? 1.0 : (double)nab.y / (double)p.P_R;
  }
}

// Parity hook: the batch the last evaluation's pair sums read (bsel) of
// selected atoms, as caller ids; -1 rows for atoms that took all of B.
__global__ void k_kept_batch_used(View p, const long long *sel, int nsel, int *batch) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nsel) return;
  const int slot = p.slot_of[sel[q]];
  const int nB = p.nAB[slot].y, PR = p.P_R;
  if (p.whole_shell || nB <= PR) return;
  for (int r = 0; r < PR; r++) batch[(long long)q * PR + r] = p.perm[p.bsel[(int64_t)slot * PR + r]];
}
void launch_kept_batch_used(const View &v, cudaStream_t st, const long long *sel, int nsel, int *batch) {
  const int b = 64, g = (nsel + b - 1) / b;
  k_kept_batch_used<<<g, b, 0, st>>>(v, sel, nsel, batch);
}

void launch_kept_lists(const View &v, cudaStream_t st, int step_off, const long long *sel, int nsel,
                       int cap_a, int cap_b, int *A, int *nA, int *B, int *nB, int *batch, int *nbatch,
                       double *weight) {
  const int b = 64, g = (nsel + b - 1) / b;
  k_kept_lists<<<g, b, 0, st>>>(v, step_off, sel, nsel, cap_a, cap_b, A, nA, B, nB, batch, nbatch, weight);
}

// ---------------------------------------------------------------------------
// Parity hook: the lists of selected atoms, through the same stencil walk,
// predicate and canonical order as k_near.
template <bool SMALL>
__global__ void k_lists(View p, int step_off, const long long *sel, int nsel, int cap_core,
                        int cap_shell, int *core, int *ncore, int *shell, int *nshell, int *batch,
                        int *nbatch, double *weight) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nsel) return;
  const long long s = *p.step + step_off;
  const int slot = p.slot_of[sel[q]];
  const float3 me = make_float3(p.sx[slot], p.sy[slot], p.sz[slot]);
  const uint4 ui = p.su[slot];
  const Axis ax = make_axis(cell_of(ui.x, p.nc[0]), p.nc[0]);
  const Axis ay = make_axis(cell_of(ui.y, p.nc[1]), p.nc[1]);
  const Axis az = make_axis(cell_of(ui.z, p.nc[2]), p.nc[2]);
  const int nkx = axis_count(ax, SMALL), nky = axis_count(ay, SMALL), nkz = axis_count(az, SMALL);
  int nc = 0, ns = 0;
  for (int kz = 0; kz < nkz; kz++) {
    float shz;
    const int cz = axis_cell(az, kz, SMALL, shz);
    for (int ky = 0; ky < nky; ky++) {
      float shy;
      const int cy = axis_cell(ay, ky, SMALL, shy);
      for (int kx = 0; kx < nkx; kx++) {
        float shx;
        const int cx = axis_cell(ax, kx, SMALL, shx);
        const int cell = cx + p.nc[0] * (cy + p.nc[1] * cz);
        for (int j = p.cell_start[cell]; j < p.cell_start[cell + 1]; j++) {
          if (j == slot) continue;
          const float r2 = cand_r2<SMALL>(p, j, me.x - shx, me.y - shy, me.z - shz, ui);
          // core: inside the largest radius and (species-dependent radii) the pair's own
          const bool in_core = r2 < p.rc2f &&
                               (!p.core_pair ||
                                r2 < p.rc2p[(int)(ui.w >> SU_SP_SHIFT) * p.ns + (int)(p.su[j].w >> SU_SP_SHIFT)]);
          if (in_core) {
            if (nc < cap_core) core[(long long)q * cap_core + nc] = p.perm[j];
            nc++;
          } else if (r2 < p.rs2f) {
            if (ns < cap_shell) shell[(long long)q * cap_shell + ns] = p.perm[j];
            ns++;
          }
        }
      }
    }
  }
  ncore[q] = nc;
  nshell[q] = ns;
  if (batch) {
    const bool take_all = p.whole_shell || ns <= p.P_R;
    int t[RBSOG_MAX_PR];
    const int nb = take_all ? ns : p.P_R;
    if (!take_all) floyd(p, s, ui.w & SU_ID_MASK, ns, t);
    for (int k = 0; k < nb && k < p.P_R; k++) {
      const int pos = take_all ? k : t[k];
      batch[(long long)q * p.P_R + k] = (pos < cap_shell) ? shell[(long long)q * cap_shell + pos] : -1;
    }
    nbatch[q] = nb;
    weight[q] = take_all ? 1.0 : (double)ns / (double)p.P_R;
  }
}

void launch_lists(const View &v, cudaStream_t st, int step_off, const long long *sel, int nsel,
                  int cap_core, int cap_shell, int *core, int *ncore, int *shell, int *nshell,
                  int *batch, int *nbatch, double *weight) {
  const int b = 64, g = (nsel + b - 1) / b;
  if (v.small)
    k_lists<true><<<g, b, 0, st>>>(v, step_off, sel, nsel, cap_core, cap_shell, core, ncore, shell,
                                   nshell, batch, nbatch, weight);
  else
    k_lists<false><<<g, b, 0, st>>>(v, step_off, sel, nsel, cap_core, cap_shell, core, ncore, shell,
                                    nshell, batch, nbatch, weight);
}

// Packed launches of an ensemble (mixed precision, step evaluations).
void pack_near(const PackPlan &q, cudaStream_t st, int step_off) {
  if (q.total[PK_NEAR_W0]) kp_near<false, false><<<q.total[PK_NEAR_W0], NEAR_BLOCK, 0, st>>>(q.pack(PK_NEAR_W0), step_off);
  if (q.total[PK_NEAR_W1]) kp_near<true, false><<<q.total[PK_NEAR_W1], NEAR_BLOCK, 0, st>>>(q.pack(PK_NEAR_W1), step_off);
}
void pack_build_lists(const PackPlan &q, cudaStream_t st) {
  if (q.total[PK_NEAR_W0]) kp_near<false, true><<<q.total[PK_NEAR_W0], NEAR_BLOCK, 0, st>>>(q.pack(PK_NEAR_W0), 0);
  if (q.total[PK_NEAR_W1]) kp_near<true, true><<<q.total[PK_NEAR_W1], NEAR_BLOCK, 0, st>>>(q.pack(PK_NEAR_W1), 0);
}
void pack_sample_batch(const PackPlan &q, cudaStream_t st, int step_off) {
  kp_sample_batch<<<q.total[PK_NEAR], NEAR_BLOCK, 0, st>>>(q.pack(PK_NEAR), step_off);
}
void pack_near_kept(const PackPlan &q, cudaStream_t st, int step_off) {
  if (q.near_wide) kp_near_kept<true><<<q.total[PK_NEAR], NEAR_BLOCK, 0, st>>>(q.pack(PK_NEAR), step_off);
  else kp_near_kept<false><<<q.total[PK_NEAR], NEAR_BLOCK, 0, st>>>(q.pack(PK_NEAR), step_off);
}

}  // namespace rb
