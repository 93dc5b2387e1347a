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
    return pred_r2((float)wrap23(uj.x, ui.x), (float)wrap23(uj.y, ui.y), (float)wrap23(uj.z, ui.z), p.hp);
  } else {
    const float4 o = p.sv[j];
    return pred_r2(o.x - ix, o.y - iy, o.z - iz, p.hp);
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
  const float r = sqrtf(x);
  const float rinv = 1.0f / r;
  const float rinv2 = rinv * rinv;
  const float t = x * p.tscale;
  const int it = min((int)t, NT_TAB - 1);
  const float f = t - (float)it;
  const float4 c = gt[it];
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
template <typename R, bool SMALL, bool ENERGY>
__global__ void __launch_bounds__(NEAR_BLOCK, 4) k_near(View p, int step_off) {
  __shared__ unsigned char cnt[125][NEAR_BLOCK];
  __shared__ float4 sg[NT_TAB];
  __shared__ PairF spf[RBSOG_MAX_SPECIES * RBSOG_MAX_SPECIES];
  __shared__ PairD spd[RBSOG_MAX_SPECIES * RBSOG_MAX_SPECIES];
  __shared__ double swa[RBSOG_MAX_M + 1], sw[RBSOG_MAX_M + 1], sh2[RBSOG_MAX_M + 1];
  __shared__ double red[4][NEAR_BLOCK / 32];
  constexpr bool MIX = sizeof(R) == 4;
  const int tid = threadIdx.x;
  const int nsp2 = p.ns * p.ns;
  for (int k = tid; k < nsp2; k += NEAR_BLOCK) {
    if (MIX) spf[k] = p.pf[k]; else spd[k] = p.pd[k];
  }
  if (MIX) {
    for (int k = tid; k < NT_TAB; k += NEAR_BLOCK) sg[k] = p.gtab[k];
  } else {
    for (int k = tid; k < p.G; k += NEAR_BLOCK) {
      swa[k] = p.sog_wa[k];
      sw[k] = p.sog_w[k];
      sh2[k] = p.sog_h[k];
    }
  }
  __syncthreads();
  const long long s = *p.step + step_off;
  const int slot = blockIdx.x * NEAR_BLOCK + tid;
  R fcx = 0, fcy = 0, fcz = 0, ec = 0;   // core
  R fsx = 0, fsy = 0, fsz = 0, es = 0;   // shell batch (unweighted)
  R wgt = 1;
  if (slot < p.n) {
    const float4 me = p.sv[slot];
    const uint4 ui = p.su[slot];
    const int spi = __float_as_int(me.w);
    const Axis ax = make_axis(cell_of(ui.x, p.nc[0]), p.nc[0]);
    const Axis ay = make_axis(cell_of(ui.y, p.nc[1]), p.nc[1]);
    const Axis az = make_axis(cell_of(ui.z, p.nc[2]), p.nc[2]);
    const int nkx = axis_count(ax, SMALL), nky = axis_count(ay, SMALL), nkz = axis_count(az, SMALL);
    int core[RBSOG_MAX_CORE];
    int ncore = 0;
    int nshell = 0;
    bool over = false;
    // ---- pass 1 -------------------------------------------------------
    for (int kz = 0; kz < STENCIL; kz++) {
      float shz;
      const int cz = axis_cell(az, kz, SMALL, shz);
      for (int ky = 0; ky < STENCIL; ky++) {
        float shy;
        const int cy = axis_cell(ay, ky, SMALL, shy);
        const int rowbase = p.nc[0] * (cy + p.nc[1] * cz);
        const float iy = me.y - shy, iz = me.z - shz;
        for (int kx = 0; kx < STENCIL; kx++) {
          const int cidx = (kz * STENCIL + ky) * STENCIL + kx;
          if (kz >= nkz || ky >= nky || kx >= nkx) {
            cnt[cidx][tid] = 0;
            continue;
          }
          float shx;
          const int cx = axis_cell(ax, kx, SMALL, shx);
          const int cell = rowbase + cx;
          const int b = p.cell_start[cell], e = p.cell_start[cell + 1];
          const float ix = me.x - shx;
          int c = 0;
          for (int j = b; j < e; j++) {
            if (j == slot) continue;
            const float r2 = cand_r2<SMALL>(p, j, ix, iy, iz, ui);
            if (r2 < p.rs2f) {
              if (r2 < p.rc2f) {
                if (ncore < RBSOG_MAX_CORE) core[ncore] = j;
                ncore++;
              } else {
                c++;
              }
            }
          }
          if (c > RBSOG_MAX_CELL_SHELL) over = true;
          cnt[cidx][tid] = (unsigned char)min(c, RBSOG_MAX_CELL_SHELL);
          nshell += c;
        }
      }
    }
    if (ncore > RBSOG_MAX_CORE) {
      atomicOr(p.err, ERR_CORE_CAP);
      ncore = RBSOG_MAX_CORE;
    }
    if (over) atomicOr(p.err, ERR_CELL_SHELL_CAP);
    // ---- pass 2 -------------------------------------------------------
    const bool take_all = p.whole_shell || nshell <= p.P_R;
    int tsel[RBSOG_MAX_PR];
    const int nb = take_all ? nshell : p.P_R;
    if (!take_all) {
      floyd(p, s, ui.w, nshell, tsel);
      wgt = (R)nshell / (R)p.P_R;
    }
    // ---- pass 3 -------------------------------------------------------
    int cum = 0, ptr = 0;
    for (int cidx = 0; cidx < STENCIL * STENCIL * STENCIL; cidx++) {
      const int k = cnt[cidx][tid];
      if (k == 0) continue;
      if (take_all || (ptr < nb && tsel[ptr] < cum + k)) {
        const int kz = cidx / 25, ky = (cidx / 5) % 5, kx = cidx % 5;
        float shx, shy, shz;
        const int cz = axis_cell(az, kz, SMALL, shz);
        const int cy = axis_cell(ay, ky, SMALL, shy);
        const int cx = axis_cell(ax, kx, SMALL, shx);
        const int cell = cx + p.nc[0] * (cy + p.nc[1] * cz);
        const int b = p.cell_start[cell], e = p.cell_start[cell + 1];
        const float ix = me.x - shx, iy = me.y - shy, iz = me.z - shz;
        int ord = cum;
        for (int j = b; j < e; j++) {
          if (j == slot) continue;
          const float r2 = cand_r2<SMALL>(p, j, ix, iy, iz, ui);
          if (r2 < p.rs2f && !(r2 < p.rc2f)) {
            if (take_all || tsel[ptr] == ord) {
              const uint4 uj = p.su[j];
              const int spj = __float_as_int(p.sv[j].w);
              if (MIX) {
                float a0 = 0, a1 = 0, a2 = 0, a3 = 0;
                pair_mixed<ENERGY>(p, spf[spi * p.ns + spj], sg, ui, uj, a0, a1, a2, a3);
                fsx += a0; fsy += a1; fsz += a2; es += a3;
              } else {
                double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
                pair_fp64<ENERGY>(p, spd[spi * p.ns + spj], swa, sw, sh2, ui, uj, a0, a1, a2, a3);
                fsx += a0; fsy += a1; fsz += a2; es += a3;
              }
              if (!take_all) {
                ptr++;
                if (ptr >= nb || tsel[ptr] >= cum + k) break;
              }
            }
            ord++;
          }
        }
      }
      cum += k;
    }
    // ---- pass 4 -------------------------------------------------------
    for (int k = 0; k < ncore; k++) {
      const int j = core[k];
      const uint4 uj = p.su[j];
      const int spj = __float_as_int(p.sv[j].w);
      if (MIX) {
        float a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        pair_mixed<ENERGY>(p, spf[spi * p.ns + spj], sg, ui, uj, a0, a1, a2, a3);
        fcx += a0; fcy += a1; fcz += a2; ec += a3;
      } else {
        double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        pair_fp64<ENERGY>(p, spd[spi * p.ns + spj], swa, sw, sh2, ui, uj, a0, a1, a2, a3);
        fcx += a0; fcy += a1; fcz += a2; ec += a3;
      }
    }
    const R Fx = fcx + wgt * fsx, Fy = fcy + wgt * fsy, Fz = fcz + wgt * fsz;
    const int64_t id = ui.w, n = p.n;
    if (MIX) {
      p.FNf[id] = (float)Fx; p.FNf[n + id] = (float)Fy; p.FNf[2 * n + id] = (float)Fz;
    } else {
      p.FNd[id] = (double)Fx; p.FNd[n + id] = (double)Fy; p.FNd[2 * n + id] = (double)Fz;
    }
    fcx = Fx; fcy = Fy; fcz = Fz;
    ec = (R)0.5 * (ec + wgt * es);
  }
  // ---- FP64 block partials of sum F_N and of the pair energy ------------
  double v[4] = {(double)fcx, (double)fcy, (double)fcz, (double)ec};
#pragma unroll
  for (int a = 0; a < 4; a++) {
    for (int o = 16; o > 0; o >>= 1) v[a] += __shfl_down_sync(0xffffffffu, v[a], o);
    if ((tid & 31) == 0) red[a][tid >> 5] = v[a];
  }
  __syncthreads();
  if (tid < 4) {
    double t = 0.0;
    for (int w = 0; w < NEAR_BLOCK / 32; w++) t += red[tid][w];
    p.near_part[4 * blockIdx.x + tid] = t;
  }
}

void launch_near(const View &v, cudaStream_t st, int step_off, bool energy) {
  const dim3 g(v.nblk_near), b(NEAR_BLOCK);
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
  const float4 me = p.sv[slot];
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
    if (!take_all) floyd(p, s, ui.w, ns, t);
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
