// Stages (a2), (b), (c): one fused kernel per step builds the random batch list
// and evaluates the near field (Sec. 2.2).  One thread per atom in cell-sorted
// order:
//   pass 1  scan the 5x5x5 cell stencil in canonical order (cells ascending by
//           linear index, atoms ascending by caller index) with the FP32
//           predicate; core neighbours (r < r_core) go to a per-thread list,
//           shell neighbours (r_core <= r < r_shell) are only counted per cell;
//   pass 2  Floyd's P_R-of-N_shell draw without replacement (Philox stream 0);
//   pass 3  walk the per-cell counts, rescan only the cells holding sampled
//           positions and add their pair forces with weight N_shell / P_R;
//   pass 4  exact core sum.
// The pair force is Eq. (Fshort) (SOG residual + BMH, k_e on Coulomb): FP32
// with the SOG sum tabulated (mixed) or analytic FP64 over m = 0..M.  The
// block's FP64 partial sums of F_N feed the momentum correction F^corr.
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

template <bool ENERGY>
__device__ __forceinline__ void pair_mixed(const View &p, const PairF &q, const float4 *gt,
                                           uint4 ui, uint4 uj, float &fx, float &fy, float &fz,
                                           float &e) {
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
  }
}

template <bool ENERGY>
__device__ __forceinline__ void pair_fp64(const View &p, const PairD &q, const double *wa,
                                          const double *w, const double *h2, uint4 ui, uint4 uj,
                                          double &fx, double &fy, double &fz, double &e) {
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
  if (ENERGY) e += q.kqq * (1.0 / r - fsum) + rep - q.C / r6 - q.D / r8;
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

// ---------------------------------------------------------------------------
// Conservative cell culling: gap (23-bit units) between v_i and the image of
// cell c of an axis with cell width cw = 2^23 / n, widened by 4 units so that
// rounding of the cell bounds can only keep a cell, never drop one.
__device__ __forceinline__ float cell_gap(float vi, int c, float shift, float cw) {
  const float lo = __fmaf_rn((float)c, cw, shift) - 4.0f;
  const float hi = __fmaf_rn((float)(c + 1), cw, shift) + 4.0f;
  return fmaxf(0.0f, fmaxf(lo - vi, vi - hi));
}

template <typename R>
struct Acc {
  R x = 0, y = 0, z = 0, e = 0;
};

// Pair force of atom i with the sorted candidate uj (species in its top bits).
template <typename R, bool ENERGY>
__device__ __forceinline__ void add_pair(const View &p, const PairF *spf, const PairD *spd,
                                         const float4 *sg, const double *swa, const double *sw,
                                         const double *sh2, int spi, uint4 ui, uint4 uj, Acc<R> &a) {
  const int spj = (int)(uj.w >> SU_SP_SHIFT);
  if (sizeof(R) == 4) {
    float a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    pair_mixed<ENERGY>(p, spf[spi * p.ns + spj], sg, ui, uj, a0, a1, a2, a3);
    a.x += a0; a.y += a1; a.z += a2; a.e += a3;
  } else {
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    pair_fp64<ENERGY>(p, spd[spi * p.ns + spj], swa, sw, sh2, ui, uj, a0, a1, a2, a3);
    a.x += a0; a.y += a1; a.z += a2; a.e += a3;
  }
}

// One warp per chunk of NEAR_CHUNK = 8 consecutive sorted atoms of one row of
// cells (fixed y, z); TPA = 4 threads per atom.  Pass 1 has two forms:
//  - lockstep (the union of the chunk's x-stencils is at most WMAX cells and
//    narrower than the box): the warp first caches the candidate ranges of
//    the 25 rows x W union cells in shared memory; thread g of every atom
//    walks stencil rows g, g + 4, ... and, in each, the union cells in
//    ascending index order, so all 8 atoms test the same candidates in the
//    same order (uniform loops, broadcast loads, four loads in flight); each
//    atom files a candidate under its own stencil position;
//  - per atom (otherwise): the atom's own 125 cells dealt round-robin, with
//    conservative culling of cells beyond r_shell.
// Both fill the same per-atom state in shared memory: per-cell shell counts
// (canonical order) and per-thread core lists coded (stencil cell << 8 |
// offset in cell).  Floyd's set is a bitmask over canonical positions; the
// sorted samples are mapped to (cell, rank) by one sweep of the counts.
constexpr int TPA = 4;
constexpr int APW = NEAR_CHUNK;              // atoms per warp
constexpr int APB = NEAR_WARPS * NEAR_CHUNK; // atoms per block
constexpr int CORE_T = 40;                   // core neighbours per thread
constexpr int SHELL_BITS = 1024;             // canonical shell positions held by the bitmask
constexpr int WMAX = 8;                      // union x-cells of a lockstep chunk
static_assert(TPA * NEAR_CHUNK == 32 && NEAR_WARPS * 32 == NEAR_BLOCK, "near-field block layout");

// stencil position (0..4, ascending cell order) of cell x on an axis of n >= 5
// cells as seen from cell ci, or -1 when x is not among ci's five neighbours
__device__ __forceinline__ int stencil_pos(int x, const Axis &ax) {
  int o = x - ax.ci;
  if (o > ax.n / 2) o -= ax.n;
  if (o < -(ax.n / 2)) o += ax.n;
  if (o < -2 || o > 2) return -1;
  int k = o + 2 - ax.rot;
  return k < 0 ? k + STENCIL : k;
}

template <typename R, bool SMALL, bool ENERGY>
__global__ void __launch_bounds__(NEAR_BLOCK, 4) k_near(View p, int step_off) {
  constexpr bool MIX = sizeof(R) == 4;
  __shared__ uint32_t smk[125][APB];         // shell members of each stencil cell (bits over its slots)
  __shared__ unsigned char scell[APB][RBSOG_MAX_PR];
  __shared__ unsigned char srank[APB][RBSOG_MAX_PR];
  __shared__ unsigned short stsel[APB][RBSOG_MAX_PR];
  __shared__ uint32_t bmask[APB][SHELL_BITS / 32];
  __shared__ unsigned short score[NEAR_BLOCK][CORE_T];
  __shared__ int2 crange[NEAR_WARPS][STENCIL * STENCIL][WMAX];
  __shared__ PairF spf[MIX ? RBSOG_MAX_SPECIES * RBSOG_MAX_SPECIES : 1];
  __shared__ PairD spd[MIX ? 1 : RBSOG_MAX_SPECIES * RBSOG_MAX_SPECIES];
  __shared__ double red[4][NEAR_WARPS];
  const int tid = threadIdx.x;
  const int nsp2 = p.ns * p.ns;
  for (int k = tid; k < nsp2; k += NEAR_BLOCK) {
    if (MIX) spf[k] = p.pf[k]; else spd[k] = p.pd[k];
  }
  // SOG tables (FP32 cubic or FP64 coefficients) through the read-only cache
  const float4 *sg = p.gtab;
  const double *swa = p.sog_wa, *sw = p.sog_w, *sh2 = p.sog_h;
  __syncthreads();
  const long long s = *p.step + step_off;
  const int warp = tid >> 5, lane = tid & 31;
  const int a = warp * APW + lane / TPA;      // atom row of the shared arrays
  const int g = lane % TPA;
  const int nrow = p.nc[1] * p.nc[2];
  const int chunk = blockIdx.x * NEAR_WARPS + warp;
  double part[4] = {0.0, 0.0, 0.0, 0.0};
  if (chunk < p.row_chunk[nrow]) {
    // ---- the chunk's row of cells and atoms ------------------------------
    int lo = 0, hi = nrow - 1;  // last row with row_chunk[row] <= chunk
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (p.row_chunk[mid] <= chunk) lo = mid; else hi = mid - 1;
    }
    const int row = lo;
    const int rbeg = p.cell_start[row * p.nc[0]], rend = p.cell_start[(row + 1) * p.nc[0]];
    const int base = rbeg + (chunk - p.row_chunk[row]) * APW;
    const int cend = min(base + APW, rend);
    const int slot = base + lane / TPA;
    const uint4 u0 = p.su[min(slot, cend - 1)];
    const bool active = slot < cend && u0.w != SU_PAD;
    const uint4 ui = active ? u0 : p.su[base];   // the first slot of a chunk is an atom
    const float3 me = active ? make_float3(p.sx[slot], p.sy[slot], p.sz[slot]) : make_float3(0.f, 0.f, 0.f);
    const int spi = (int)(ui.w >> SU_SP_SHIFT);
    const int cyr = row % p.nc[1], czr = row / p.nc[1];
    const int cxi = cell_of(ui.x, p.nc[0]);
    const Axis ax = make_axis(cxi, p.nc[0]);
    const Axis ay = make_axis(cyr, p.nc[1]), az = make_axis(czr, p.nc[2]);
    const int nkx = axis_count(ax, SMALL), nky = axis_count(ay, SMALL), nkz = axis_count(az, SMALL);
    const int cx_lo = __reduce_min_sync(0xffffffffu, cxi), cx_hi = __reduce_max_sync(0xffffffffu, cxi);
    const int W = cx_hi - cx_lo + STENCIL;     // union x-cells of the chunk
    const bool lock = !SMALL && W <= WMAX && W <= p.nc[0];
    const int xs = cx_lo - 2;                  // first union cell (may be < 0)
    Acc<R> fc, fs;
    R wgt = 1;
    int my_total = 0, ncore = 0;
    bool over = false;
    if (lock) {
      // ---- candidate ranges of the union cells, cached per warp --------------
      for (int it = lane; it < STENCIL * STENCIL * W; it += 32) {
        const int r = it / W, ux = it - r * W;
        const int kz = r / STENCIL, ky = r - kz * STENCIL;
        float sh;
        const int cz = axis_cell(az, kz, false, sh);
        const int cy = axis_cell(ay, ky, false, sh);
        int x = xs + ux;
        x = x < 0 ? x + p.nc[0] : (x >= p.nc[0] ? x - p.nc[0] : x);
        const int cell = x + p.nc[0] * (cy + p.nc[1] * cz);
        crange[warp][r][ux] = make_int2(p.cell_start[cell], p.cell_start[cell + 1]);
      }
      // the atom's stencil position of every union cell, 3 bits each (kx + 1, 0 = none)
      int kxcode = 0;
      for (int ux = 0; ux < W; ux++) {
        int x = xs + ux;
        x = x < 0 ? x + p.nc[0] : (x >= p.nc[0] ? x - p.nc[0] : x);
        kxcode |= (stencil_pos(x, ax) + 1) << (3 * ux);
      }
      __syncwarp();
      // ---- pass 1, lockstep form ---------------------------------------------
      // Branch-free counts per cell: n(r < r_shell) and n(r < r_core) (the
      // atom itself, r = 0, is in both, so shell = difference), core hits as a
      // bit mask over the cell's slots, expanded into the core list per cell.
      const int rot = xs < 0 ? -xs : (cx_hi + 2 >= p.nc[0] ? W - (cx_hi + 2 - p.nc[0] + 1) : 0);
      for (int r = g; r < STENCIL * STENCIL; r += TPA) {
        const int kz = r / STENCIL, ky = r - kz * STENCIL;
        float shz, shy;
        axis_cell(az, kz, false, shz);
        axis_cell(ay, ky, false, shy);
        const float iy = me.y - shy, iz = me.z - shz;
        for (int k = 0; k < W; k++) {
          int ux = k + rot;
          ux = ux >= W ? ux - W : ux;           // union index, ascending cell order
          const int u = xs + ux;
          const float shx = u < 0 ? -8388608.0f : (u >= p.nc[0] ? 8388608.0f : 0.0f);
          const int kx = ((kxcode >> (3 * ux)) & 7) - 1;
          const int2 be = crange[warp][r][ux];
          const PredX4 pc = pred_x4_setup(me.x - shx, iy, iz, p.hp);
          const float rs2 = p.rs2f, rc2 = p.rc2f;
          uint32_t smask = 0u, cmask = 0u, bit = 1u;
          for (int j0 = be.x; j0 < be.y; j0 += CELL_ALIGN) {
            float r2v[4];
            pred_r2_x4(p.sx, p.sy, p.sz, j0, pc, r2v);
#pragma unroll
            for (int t = 0; t < 4; t++) {
              smask |= (r2v[t] < rs2) ? bit : 0u;
              cmask |= (r2v[t] < rc2) ? bit : 0u;
              bit <<= 1;
            }
          }
          if (slot >= be.x && slot < be.y) cmask &= ~(1u << ((slot - be.x) & 31));
          smask &= ~cmask;                        // shell = inside r_shell, not core, not self
          if (slot >= be.x && slot < be.y) smask &= ~(1u << ((slot - be.x) & 31));
          if (kx >= 0) {
            const int q = (kz * STENCIL + ky) * STENCIL + kx;
            const int c = __popc(smask);
            if (be.y - be.x > 32) over = true;
            smk[q][a] = smask;
            my_total += c;
            while (cmask) {
              const int b = __ffs(cmask) - 1;
              cmask &= cmask - 1u;
              if (ncore < CORE_T) score[tid][ncore] = (unsigned short)((q << 8) | b);
              else over = true;
              ncore++;
            }
          } else if ((smask | cmask) && active) {
            over = true;   // impossible: beyond the atom's stencil is beyond r_shell
          }
        }
      }
      if (!active) { my_total = 0; ncore = 0; over = false; }
    } else {
      // ---- pass 1, per-atom form ---------------------------------------------
      const float cw[3] = {8388608.0f / (float)p.nc[0], 8388608.0f / (float)p.nc[1], 8388608.0f / (float)p.nc[2]};
      const float cull = p.rs2f * (1.0f + 1.0f / 1024.0f);
      for (int q = g; q < STENCIL * STENCIL * STENCIL; q += TPA) {
        const int kz = q / 25, ky = (q / 5) % 5, kx = q % 5;
        uint32_t m = 0u;
        if (kz < nkz && ky < nky && kx < nkx) {
          float shx, shy, shz;
          const int cz = axis_cell(az, kz, SMALL, shz);
          const int cy = axis_cell(ay, ky, SMALL, shy);
          const int cx = axis_cell(ax, kx, SMALL, shx);
          bool keep = true;
          if (!SMALL) {
            const float gx = cell_gap(me.x, cx, shx, cw[0]) * p.hp[0];
            const float gy = cell_gap(me.y, cy, shy, cw[1]) * p.hp[1];
            const float gz = cell_gap(me.z, cz, shz, cw[2]) * p.hp[2];
            keep = __fmaf_rn(gz, gz, __fmaf_rn(gy, gy, gx * gx)) < cull;
          }
          if (keep) {
            const int cell = cx + p.nc[0] * (cy + p.nc[1] * cz);
            const int b = p.cell_start[cell], e = p.cell_start[cell + 1];
            const float ix = me.x - shx, iy = me.y - shy, iz = me.z - shz;
            if (e - b > 32) over = true;
            for (int j = b; j < e; j++) {
              const float r2 = cand_r2<SMALL>(p, j, ix, iy, iz, ui);
              if (r2 < p.rs2f && j != slot && active) {
                if (r2 < p.rc2f) {
                  if (ncore < CORE_T) score[tid][ncore] = (unsigned short)((q << 8) | ((j - b) & 255));
                  else over = true;
                  ncore++;
                } else {
                  m |= 1u << ((j - b) & 31);
                }
              }
            }
          }
        }
        smk[q][a] = m;
        my_total += __popc(m);
      }
    }
    if (over) atomicOr(p.err, ncore > CORE_T ? ERR_CORE_CAP : ERR_CELL_SHELL_CAP);
    ncore = min(ncore, CORE_T);
    // ---- group total of shell counts ------------------------------------
    int nshell = my_total;
#pragma unroll
    for (int o = 1; o < TPA; o <<= 1) nshell += __shfl_xor_sync(0xffffffffu, nshell, o, TPA);
    const bool take_all = p.whole_shell || nshell <= p.P_R;
    const bool sampled = active && !take_all && nshell <= SHELL_BITS;
    if (active && !take_all && nshell > SHELL_BITS && g == 0) atomicOr(p.err, ERR_CELL_SHELL_CAP);
    // ---- pass 2: Floyd's draw by the group's first thread -------------------
    if (sampled) {
      const int nw = (nshell + 31) >> 5;
      for (int w = g; w < nw; w += TPA) bmask[a][w] = 0u;
      for (int k = g; k < RBSOG_MAX_PR; k += TPA) scell[a][k] = 0xFF;
    }
    __syncwarp();
    if (sampled && g == 0) {
      uint32_t *bm = bmask[a];
      const int PR = p.P_R;
      const uint32_t id = ui.w & SU_ID_MASK;
      uint4 w4 = make_uint4(0, 0, 0, 0);
      for (int r = 0; r < PR; r++) {
        if ((r & 1) == 0) w4 = draw(p.seed, s, id, 0u, (uint32_t)(r >> 1));
        const unsigned long long U = (r & 1) ? (((unsigned long long)w4.w << 32) | w4.z)
                                             : (((unsigned long long)w4.y << 32) | w4.x);
        const uint32_t J = (uint32_t)(nshell - PR + r);
        uint32_t t = (uint32_t)__umul64hi(U, (unsigned long long)J + 1ull);
        if ((bm[t >> 5] >> (t & 31)) & 1u) t = J;
        bm[t >> 5] |= 1u << (t & 31);
      }
      int k = 0;
      const int nw = (nshell + 31) >> 5;
      for (int w = 0; w < nw; w++) {
        uint32_t bits = bm[w];
        while (bits) {
          stsel[a][k++] = (unsigned short)(32 * w + __ffs(bits) - 1);
          bits &= bits - 1u;
        }
      }
      k = 0;
      int cum = 0;
      for (int q = 0; q < STENCIL * STENCIL * STENCIL && k < PR; q++) {
        const int cn = __popc(smk[q][a]);
        while (k < PR && stsel[a][k] < cum + cn) {
          scell[a][k] = (unsigned char)q;
          srank[a][k] = (unsigned char)(stsel[a][k] - cum);
          k++;
        }
        cum += cn;
      }
    }
    if (sampled) wgt = (R)nshell / (R)p.P_R;
    __syncwarp();
    // candidate range and image shift of the atom's stencil cell q
    auto cell_range = [&](int q, float &shx, float &shy, float &shz) -> int2 {
      const int kz = q / 25, ky = (q / 5) % 5, kx = q % 5;
      const int cz = axis_cell(az, kz, SMALL, shz);
      const int cy = axis_cell(ay, ky, SMALL, shy);
      const int cx = axis_cell(ax, kx, SMALL, shx);
      if (lock) {
        int ux = cx - xs;
        if (ux < 0) ux += p.nc[0];
        if (ux >= p.nc[0]) ux -= p.nc[0];
        return crange[warp][kz * STENCIL + ky][ux];
      }
      const int cell = cx + p.nc[0] * (cy + p.nc[1] * cz);
      return make_int2(p.cell_start[cell], p.cell_start[cell + 1]);
    };
    if (active) {
      if (sampled) {
        // ---- pass 3: sampled shell members, spread over the group ---------
        for (int k = g; k < p.P_R; k += TPA) {
          const int q = scell[a][k], rank = srank[a][k];
          const int kz = q / 25, ky = (q / 5) % 5, kx = q % 5;
          if (q >= 125 || kz >= nkz || ky >= nky || kx >= nkx) continue;  // only after an overflow
          float shx, shy, shz;
          const int2 be = cell_range(q, shx, shy, shz);
          // the rank-th set bit of the cell's shell mask
          uint32_t m = smk[q][a];
          for (int t = 0; t < rank; t++) m &= m - 1u;
          if (m) add_pair<R, ENERGY>(p, spf, spd, sg, swa, sw, sh2, spi, ui, p.su[be.x + __ffs(m) - 1], fs);
        }
      } else if (take_all) {
        // whole shell, weight 1: every shell member of the thread's quarter of cells
        for (int q = g; q < STENCIL * STENCIL * STENCIL; q += TPA) {
          uint32_t m = smk[q][a];
          if (m == 0u) continue;
          float shx, shy, shz;
          const int b = cell_range(q, shx, shy, shz).x;
          while (m) {
            const int t = __ffs(m) - 1;
            m &= m - 1u;
            add_pair<R, ENERGY>(p, spf, spd, sg, swa, sw, sh2, spi, ui, p.su[b + t], fs);
          }
        }
      }
      // ---- pass 4: exact core sum; the group's core lists are dealt out
      // round-robin over its threads (entry e of the concatenated list) ----------
    }
    {
      int cbase = ncore;                         // exclusive prefix of the group's list lengths
#pragma unroll
      for (int o = 1; o < TPA; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, cbase, o, TPA);
        if (g >= o) cbase += y;
      }
      const int ctot = __shfl_sync(0xffffffffu, cbase, TPA - 1, TPA);
      cbase -= ncore;
      int off[TPA];
#pragma unroll
      for (int t = 0; t < TPA; t++) off[t] = __shfl_sync(0xffffffffu, cbase, t, TPA);
      __syncwarp();
      if (active) {
        const int tid0 = tid - g;                // first thread of the group
        for (int e = g; e < ctot; e += TPA) {
          int owner = 0;
#pragma unroll
          for (int t = 1; t < TPA; t++) owner += (e >= off[t]);
          const int code = score[tid0 + owner][e - off[owner]];
          float shx, shy, shz;
          const int j = cell_range(code >> 8, shx, shy, shz).x + (code & 255);
          add_pair<R, ENERGY>(p, spf, spd, sg, swa, sw, sh2, spi, ui, p.su[j], fc);
        }
      }
    }
    // ---- combine the group ----------------------------------------------
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
      }
    }
    if (active && g == 0) {
      const R Fx = fc.x + wgt * fs.x, Fy = fc.y + wgt * fs.y, Fz = fc.z + wgt * fs.z;
      const int64_t id = ui.w & SU_ID_MASK, n = p.n;
      if (MIX) {
        p.FNf[id] = (float)Fx; p.FNf[n + id] = (float)Fy; p.FNf[2 * n + id] = (float)Fz;
      } else {
        p.FNd[id] = (double)Fx; p.FNd[n + id] = (double)Fy; p.FNd[2 * n + id] = (double)Fz;
      }
      part[0] = (double)Fx; part[1] = (double)Fy; part[2] = (double)Fz;
      part[3] = (double)((R)0.5 * (fc.e + wgt * fs.e));
    }
  }
  // ---- FP64 block partials of sum F_N and of the pair energy ------------
#pragma unroll
  for (int c = 0; c < 4; c++) {
    for (int o = 16; o > 0; o >>= 1) part[c] += __shfl_down_sync(0xffffffffu, part[c], o);
    if (lane == 0) red[c][warp] = part[c];
  }
  __syncthreads();
  if (tid < 4) {
    double t = 0.0;
    for (int w = 0; w < NEAR_WARPS; w++) t += red[tid][w];
    p.near_part[4 * blockIdx.x + tid] = t;
  }
}

void launch_near(const View &v, cudaStream_t st, int step_off, bool energy) {
  const dim3 g(v.nblk_near), b(NEAR_BLOCK);  // nblk_near = ceil(ncell / cells per block)
#define RB_NEAR(R, SM, EN) k_near<R, SM, EN><<<g, b, 0, st>>>(v, step_off)
  if (v.prec == RBSOG_MIXED) {
    if (v.small) { if (energy) RB_NEAR(float, true, true); else RB_NEAR(float, true, false); }
    else { if (energy) RB_NEAR(float, false, true); else RB_NEAR(float, false, false); }
  } else {
    if (v.small) { if (energy) RB_NEAR(double, true, true); else RB_NEAR(double, true, false); }
    else { if (energy) RB_NEAR(double, false, true); else RB_NEAR(double, false, false); }
  }
#undef RB_NEAR
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
          if (r2 < p.rc2f) {
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

}  // namespace rb
