// Stage (a) and the integrator's first half, plus the k-batch draw of stage (d):
//   k_prepare   per atom: [half kick, drift / BAOAB B-A-O-A (Sec. 2.3)], 32-bit
//               fixed-point coordinates, cell index, cell and row histograms
//               (with kept lists between builds: the slot's coordinates and
//               the displacement check instead of the histograms).
//   k_ksample   the P_F k-vectors from P(k) (Eq. (Pk)), one warp per sample.
//   k_rowscan   row ranges (rows of cells padded to a multiple of 4 slots),
//               padding slots, near-field chunk offsets (one block).
//   k_cellstart cell ranges inside each row (one warp per row).
//   k_scatter   counting-sort scatter (slot claimed by atomicAdd).
//   k_rank      per atom: rank in its cell by (u_x, caller id), the canonical
//               order of the list -> sorted slot; write the SoA arrays.
#include "nh.cuh"

namespace rb {

// ---------------------------------------------------------------------------
// k-batch: exact i.i.d. draw from the mixture form of P(k) = k^2 Fhat(k)/S,
// one warp per sample.  U0 picks the (Gaussian g, axis d) component, U1
// picks m_d from the k^2-weighted 1-D CDF, U2/U3 pick the other two axes
// (ascending axis order) from the plain 1-D CDFs; c_p = S / (P_F |k_p|^2).
__device__ void ksample_warp(const View &p, int q, long long s, int lane) {
  if (q >= p.P_F || p.fixed_k) return;
  const uint4 w0 = draw(p.seed, s, (uint32_t)q, 1u, 0u);
  const uint4 w1 = draw(p.seed, s, (uint32_t)q, 1u, 1u);
  const unsigned long long U0 = ((unsigned long long)w0.y << 32) | w0.x;
  const unsigned long long U1 = ((unsigned long long)w0.w << 32) | w0.z;
  const unsigned long long U2 = ((unsigned long long)w1.y << 32) | w1.x;
  const unsigned long long U3 = ((unsigned long long)w1.w << 32) | w1.z;
  const int c = cdf_pick_warp(p.cmix, 3 * p.G, U0, lane);
  const int d = c % 3;
  const int g = c / 3;
  int m[3];
  {
    const int nm = p.cdf_nmax[c];
    m[d] = cdf_pick_warp(p.cdf + p.cdf_off2[c], 2 * nm + 1, U1, lane) - nm;
  }
  const unsigned long long Uo[2] = {U2, U3};
  int o = 0;
  for (int e = 0; e < 3; e++) {
    if (e == d) continue;
    const int ce = 3 * g + e;
    const int nm = p.cdf_nmax[ce];
    m[e] = cdf_pick_warp(p.cdf + p.cdf_off0[ce], 2 * nm + 1, Uo[o++], lane) - nm;
  }
  if (lane == 0) {
    double k2 = 0.0;
    for (int e = 0; e < 3; e++) {
      const double k = 2.0 * 3.141592653589793 * (double)m[e] / p.L[e];
      k2 += k * k;
    }
    p.km[q] = make_int4(m[0], m[1], m[2], 0);
    p.kc[q] = p.S / ((double)p.P_F * k2);
  }
}

// Component a of the O-step's Gaussian triple: Box-Muller on Philox stream 2,
// block 0, words (x, y, z, w) -> uniforms u0..u3 in (0, 1):
// (g0, g1) = sqrt(-2 ln u0) (cos, sin)(2 pi u1), g2 = sqrt(-2 ln u2) cos(2 pi u3).
// FP64 (noise1); mixed precision in FP32 on 24-bit uniforms (noise1f: FP64
// transcendental throughput is low on this part, the noise needs no more).
__device__ __forceinline__ double noise1(const View &p, long long s, uint32_t i, int a) {
  const uint4 w = draw(p.seed, s, i, 2u, 0u);
  const uint32_t wu = a < 2 ? w.x : w.z, wa = a < 2 ? w.y : w.w;
  const double u0 = ((double)wu + 0.5) * 2.3283064365386963e-10;
  const double u1 = ((double)wa + 0.5) * 2.3283064365386963e-10;
  const double r = sqrt(-2.0 * log(u0));
  double sn, cs;
  sincospi(2.0 * u1, &sn, &cs);
  return a == 1 ? r * sn : r * cs;
}
__device__ __forceinline__ double noise1f(const View &p, long long s, uint32_t i, int a) {
  const uint4 w = draw(p.seed, s, i, 2u, 0u);
  const uint32_t wu = a < 2 ? w.x : w.z, wa = a < 2 ? w.y : w.w;
  const float u0 = ((float)(wu >> 8) + 0.5f) * 5.9604645e-08f;
  const float u1 = ((float)(wa >> 8) + 0.5f) * 5.9604645e-08f;
  const float r = sqrtf(-2.0f * logf(u0));
  float sn, cs;
  sincospif(2.0f * u1, &sn, &cs);
  return a == 1 ? r * sn : r * cs;
}

// Cell and row histograms; lanes of one warp that share a cell (or row) add once.
__device__ __forceinline__ void histogram_add(const View &p, int cell) {
  const unsigned act = __activemask();
  const unsigned pc = __match_any_sync(act, cell);
  if ((threadIdx.x & 31) == __ffs(pc) - 1) atomicAdd(p.cell_count + cell, __popc(pc));
  const int row = cell / p.nc[0];
  const unsigned pr = __match_any_sync(act, row);
  if ((threadIdx.x & 31) == __ffs(pr) - 1) atomicAdd(p.row_count + row, __popc(pr));
}

// With automatic kept lists the binning kernels stay in every step's graph
// and return at once unless this step rebuilds the lists.
__device__ __forceinline__ bool skip_binning(const View &p) {
  return p.auto_lists && *(volatile const int *)p.lflag == 0;
}

// Three threads per atom, one per Cartesian component: the block takes
// PREP_ATOMS atoms, component-major (threads [c PREP_ATOMS, (c + 1)
// PREP_ATOMS) take component c), so the integrator's FP64 chain and the fixed
// point run on three times the warps of one thread per atom (the FP64 pipe is
// this kernel's busiest unit; the extra warps help it share the SMs with the
// far-field branch); the atom's first thread then gathers the components
// (cell, slot refresh, displacement check in the fixed order x, y, z,
// histograms).
constexpr int PREP_ATOMS = 128;

template <int MODE>
__device__ __forceinline__ void prepare_body(const View &p, int step_off, int bid) {
  __shared__ uint32_t su3[3][PREP_ATOMS];
  __shared__ double sq3[3][PREP_ATOMS];
  const long long s = *p.step + step_off;
  const int c = threadIdx.x / PREP_ATOMS, li = threadIdx.x % PREP_ATOMS;
  const int64_t i = (int64_t)bid * PREP_ATOMS + li;
  const int64_t n = p.n;
  // Nose-Hoover: the opening half step of the chain, every block alike
  const double s_open = (MODE == 1 && p.integ == RBSOG_NOSE_HOOVER) ? nh_open(p) : 1.0;
  const bool act = i < n;
  // the fixed-point F_N totals of this evaluation start at zero (the near
  // field adds to them after this kernel; k_finish of the last evaluation
  // has read them)
  if (bid == 0 && threadIdx.x < 3 * CORR_COPIES && p.npart == 4)
    p.corr_acc[16 * (threadIdx.x / 3) + threadIdx.x % 3] = 0ull;
  const bool keep_check = p.kept && (p.auto_lists || !p.build);   // displacement since the last build
  if (act) {
    const int sp = p.spc[i];
    double x = p.x[c * n + i];
    if (MODE != 0) {
      double v = p.v[c * n + i];
      const double F = p.prec == RBSOG_FP64 ? p.Fd[c * n + i] : (double)p.Ff[c * n + i];
      v = v * s_open + p.kick[sp] * F;
      if (MODE == 1) {
        x += p.dt * v;
      } else {
        const double g = p.prec == RBSOG_FP64 ? noise1(p, s, (uint32_t)i, c) : noise1f(p, s, (uint32_t)i, c);
        const double h = 0.5 * p.dt, so = p.sig_ou[sp];
        x += h * v;
        v = p.c1 * v + so * g;
        x += h * v;
      }
      p.x[c * n + i] = x;
      p.v[c * n + i] = v;
    }
    su3[c][li] = fixed_point(x, p.invL[c]);
    if (keep_check) {
      const double d = __dadd_rn(x, -p.xb[c * n + i]);
      sq3[c][li] = __dmul_rn(d, d);
    }
  }
  __syncthreads();
  if (c != 0 || !act) return;
  const int sp = p.spc[i];
  const uint32_t u[3] = {su3[0][li], su3[1][li], su3[2][li]};
  const int cell = cell_of(u[0], p.nc[0]) + p.nc[0] * (cell_of(u[1], p.nc[1]) + p.nc[1] * cell_of(u[2], p.nc[2]));
  p.ua[i] = make_uint4(u[0], u[1], u[2], (uint32_t)sp);
  p.cellid[i] = cell;
  if (p.kept) {
    // |x - x_build|^2 in the order x, y, z without contraction (the oracle's)
    const double d2 = keep_check ? __dadd_rn(__dadd_rn(sq3[0][li], sq3[1][li]), sq3[2][li]) : 0.0;
    if (p.auto_lists) {
      // refresh the slot of the last build (unless the host asked for a build:
      // then there may be none yet) and raise the build flag when this atom
      // has moved by more than skin/2 since then; the histograms follow, the
      // binning kernels run only if the flag is up
      if (*(volatile int *)p.lflag == 0)
        p.su[p.slot_of[i]] = make_uint4(u[0], u[1], u[2], (uint32_t)i | ((uint32_t)sp << SU_SP_SHIFT));
      const unsigned far = __ballot_sync(__activemask(), d2 > p.half_skin2);
      if (far && (threadIdx.x & 31) == __ffs(far) - 1) atomicOr(p.lflag, 1);   // one lane per warp
    } else if (!p.build) {
      // the lists and slots of the last build are kept: refresh this atom's
      // coordinates in its slot and check that it stayed within skin/2
      p.su[p.slot_of[i]] = make_uint4(u[0], u[1], u[2], (uint32_t)i | ((uint32_t)sp << SU_SP_SHIFT));
      if (d2 > p.half_skin2) atomicOr(p.err, ERR_SKIN);
      return;                      // no binning in this evaluation
    }
  }
  histogram_add(p, cell);
}

template <int MODE>
__global__ void __launch_bounds__(3 * PREP_ATOMS) k_prepare(View p, int step_off) {
  prepare_body<MODE>(p, step_off, blockIdx.x);
}
template <int MODE>
__global__ void __launch_bounds__(3 * PREP_ATOMS) kp_prepare(Pack pk, int step_off) {
  RB_PACK_PROLOGUE(pk);
  (void)nb;
  prepare_body<MODE>(sv, step_off, bid);
}

// Block-wide exclusive scan of one value per thread (1024 threads).
__device__ __forceinline__ int block_exclusive_scan(int v, int *wsum) {
  const int t = threadIdx.x, nt = blockDim.x;
  int incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if ((t & 31) >= o) incl += y;
  }
  __syncthreads();
  if ((t & 31) == 31) wsum[t >> 5] = incl;
  __syncthreads();
  if (t < 32) {
    int w = (t < (nt >> 5)) ? wsum[t] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (t >= o) w += y;
    }
    wsum[t] = w;
  }
  __syncthreads();
  return incl - v + ((t >> 5) ? wsum[(t >> 5) - 1] : 0);
}

// Row ranges: every row of cells (fixed y, z) is padded to a multiple of
// CELL_ALIGN slots (padding slots at FAR_AWAY, su.w = SU_PAD, written here);
// row_start[r] (exclusive scan of the padded row totals, cell_start[ncell] =
// all slots) and the near-field chunks: each row's slots cut into runs of
// NEAR_CHUNK from its start, row_chunk[r] = first chunk of row r.  One block;
// the row totals come from the binning's atomic counts.
__device__ __forceinline__ void rowscan_body(const View &p) {
  __shared__ int wsum[32];
  if (skip_binning(p)) return;
  const int nt = blockDim.x, t = threadIdx.x;
  if (t == 0 && p.b16_over) *p.b16_over = 0;     // a kept-list build follows: its own 16-bit check
  const int nrow = p.nc[1] * p.nc[2];
  const int per = (nrow + nt - 1) / nt;
  const int rb = min(t * per, nrow), re = min(rb + per, nrow);
  int local = 0, lchunk = 0;
  for (int r = rb; r < re; r++) {
    const int padded = (p.row_count[r] + CELL_ALIGN - 1) & ~(CELL_ALIGN - 1);
    local += padded;
    lchunk += (padded + NEAR_CHUNK - 1) / NEAR_CHUNK;
  }
  int run = block_exclusive_scan(local, wsum);
  int crun = block_exclusive_scan(lchunk, wsum);
  for (int r = rb; r < re; r++) {
    const int tot = p.row_count[r];
    const int padded = (tot + CELL_ALIGN - 1) & ~(CELL_ALIGN - 1);
    p.row_start[r] = run;
    for (int k = run + tot; k < run + padded; k++) {
      p.perm[k] = -1;
      p.sx[k] = FAR_AWAY;
      p.sy[k] = FAR_AWAY;
      p.sz[k] = FAR_AWAY;
      p.su[k] = make_uint4(0u, 0u, 0u, SU_PAD);
    }
    run += padded;
    p.row_chunk[r] = crun;
    crun += (padded + NEAR_CHUNK - 1) / NEAR_CHUNK;
  }
  if (t == nt - 1) {
    p.cell_start[p.ncell] = run;
    p.row_chunk[nrow] = crun;
  }
}
__global__ void __launch_bounds__(1024) k_rowscan(View p) { rowscan_body(p); }
__global__ void __launch_bounds__(1024) kp_rowscan(Pack pk) {
  RB_PACK_PROLOGUE_REF(pk);
  (void)bid; (void)nb;
  rowscan_body(sv);
}

// Cell ranges inside each row: one warp per row, an inclusive warp scan of
// the cell counts (32 cells per round) on top of the row's start.
__device__ __forceinline__ void cellstart_body(const View &p, int bid) {
  if (skip_binning(p)) return;
  const int nrow = p.nc[1] * p.nc[2], nc0 = p.nc[0];
  const int r = (int)(((int64_t)bid * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= nrow) return;
  int base = p.row_start[r];
  for (int c0 = 0; c0 < nc0; c0 += 32) {
    const int c = c0 + lane;
    const int cnt = c < nc0 ? p.cell_count[r * nc0 + c] : 0;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (c < nc0) {
      p.cell_start[r * nc0 + c] = base + incl - cnt;
      p.cell_cursor[r * nc0 + c] = base + incl - cnt;
    }
    base += __shfl_sync(0xffffffffu, incl, 31);
  }
}
__global__ void __launch_bounds__(256) k_cellstart(View p) { cellstart_body(p, blockIdx.x); }
__global__ void __launch_bounds__(256) kp_cellstart(Pack pk) {
  RB_PACK_PROLOGUE_REF(pk);
  (void)nb;
  cellstart_body(sv, bid);
}

__device__ __forceinline__ void scatter_body(const View &p, int bid) {
  const int64_t i = (int64_t)bid * blockDim.x + threadIdx.x;
  if (i >= p.n || skip_binning(p)) return;
  const int slot = atomicAdd(p.cell_cursor + p.cellid[i], 1);
  p.perm_tmp[slot] = (int)i;
  p.key_tmp[slot] = p.ua[i].x;
}
__global__ void __launch_bounds__(256) k_scatter(View p) { scatter_body(p, blockIdx.x); }
__global__ void __launch_bounds__(256) kp_scatter(Pack pk) {
  RB_PACK_PROLOGUE_REF(pk);
  (void)nb;
  scatter_body(sv, bid);
}

// One thread per atom: its rank in its cell under the canonical order
// (fixed-point x coordinate, caller id), so every row of cells is sorted by x;
// writes the sorted SoA arrays and the near-field chunk table.
__device__ __forceinline__ void rank_body(const View &p, int bid) {
  const int64_t i = (int64_t)bid * blockDim.x + threadIdx.x;
  if (i >= p.n || skip_binning(p)) return;
  if (p.kept)                      // positions of this build, for the displacement check
    for (int a = 0; a < 3; a++) p.xb[a * p.n + i] = p.x[a * p.n + i];
  const int c = p.cellid[i];
  const int b = p.cell_start[c], cnt = p.cell_count[c];
  const uint4 u = p.ua[i];
  int rank = 0;
  for (int k = b; k < b + cnt; k++) {
    const int j = p.perm_tmp[k];
    const uint32_t xj = p.key_tmp[k];
    rank += (xj < u.x || (xj == u.x && j < (int)i)) ? 1 : 0;
  }
  const int slot = b + rank;
  p.perm[slot] = (int)i;
  p.slot_of[i] = slot;
  p.sx[slot] = (float)(u.x >> 9);
  p.sy[slot] = (float)(u.y >> 9);
  p.sz[slot] = (float)(u.z >> 9);
  p.su[slot] = make_uint4(u.x, u.y, u.z, (uint32_t)i | (u.w << SU_SP_SHIFT));
  // the near-field chunks (runs of NEAR_CHUNK slots from the start of the row
  // of cells) that begin at this slot; padding only ends a row, so every run
  // begins at an atom
  const int row = c / p.nc[0];
  const int rbeg = p.cell_start[row * p.nc[0]];
  if (((slot - rbeg) & (NEAR_CHUNK - 1)) == 0)
    p.chunk_info[p.row_chunk[row] + (slot - rbeg) / NEAR_CHUNK] = make_int2(row, slot);
}
__global__ void __launch_bounds__(256) k_rank(View p) { rank_body(p, blockIdx.x); }
__global__ void __launch_bounds__(256) kp_rank(Pack pk) {
  RB_PACK_PROLOGUE_REF(pk);
  (void)nb;
  rank_body(sv, bid);
}

// The k-batch, one warp per sample (needs only the step counter).
__global__ void __launch_bounds__(256) k_ksample(View p, int step_off) {
  const long long s = *p.step + step_off;
  ksample_warp(p, (int)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), s, threadIdx.x & 31);
}
__global__ void __launch_bounds__(256) kp_ksample(Pack pk, int step_off) {
  RB_PACK_PROLOGUE_REF(pk);
  (void)nb;
  const long long s = *sv.step + step_off;
  ksample_warp(sv, bid * (blockDim.x >> 5) + (threadIdx.x >> 5), s, threadIdx.x & 31);
}

void launch_ksample(const View &v, cudaStream_t st, int step_off) {
  if (!v.fixed_k) k_ksample<<<v.nblk_kq, 256, 0, st>>>(v, step_off);
}

// The cell and row histograms start at zero: cleared at set-up and, after
// every use, by the near-field kernel (clear_counts) or by the caller.
void launch_prepare(const View &v, cudaStream_t st, int mode, int step_off) {
  const int blocks = (int)((v.n + PREP_ATOMS - 1) / PREP_ATOMS);
  if (mode == 0) k_prepare<0><<<blocks, 3 * PREP_ATOMS, 0, st>>>(v, step_off);
  else if (mode == 1) k_prepare<1><<<blocks, 3 * PREP_ATOMS, 0, st>>>(v, step_off);
  else k_prepare<2><<<blocks, 3 * PREP_ATOMS, 0, st>>>(v, step_off);
}

void launch_bin(const View &v, cudaStream_t st) {
  k_rowscan<<<1, 1024, 0, st>>>(v);
  k_cellstart<<<(unsigned)(((int64_t)v.nc[1] * v.nc[2] * 32 + 255) / 256), 256, 0, st>>>(v);
  k_scatter<<<(unsigned)((v.n + 255) / 256), 256, 0, st>>>(v);
  k_rank<<<(unsigned)((v.n + 255) / 256), 256, 0, st>>>(v);
}

// ---------------------------------------------------------------------------
// Packed launches of an ensemble (one grid over every replica; the block
// counts per replica are the prefix tables of PackPlan).
void pack_ksample(const PackPlan &q, cudaStream_t st, int step_off) {
  kp_ksample<<<q.total[PK_KSAMPLE], 256, 0, st>>>(q.pack(PK_KSAMPLE), step_off);
}
void pack_prepare(const PackPlan &q, cudaStream_t st, int mode, int step_off) {
  const int g = q.total[PK_PREP];
  if (mode == 1) kp_prepare<1><<<g, 3 * PREP_ATOMS, 0, st>>>(q.pack(PK_PREP), step_off);
  else kp_prepare<2><<<g, 3 * PREP_ATOMS, 0, st>>>(q.pack(PK_PREP), step_off);
}
void pack_bin(const PackPlan &q, cudaStream_t st) {
  kp_rowscan<<<q.total[PK_ONE], 1024, 0, st>>>(q.pack(PK_ONE));
  kp_cellstart<<<q.total[PK_ROWS], 256, 0, st>>>(q.pack(PK_ROWS));
  kp_scatter<<<q.total[PK_ATOM256], 256, 0, st>>>(q.pack(PK_ATOM256));
  kp_rank<<<q.total[PK_ATOM256], 256, 0, st>>>(q.pack(PK_ATOM256));
}

// ---------------------------------------------------------------------------
// Layout conversions between the ABI's [n][3] FP64 and the internal [3][n].
__global__ void k_aos_to_soa(const double *aos, double *soa, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int a = 0; a < 3; a++) soa[a * n + i] = aos[3 * i + a];
}
template <typename T>
__global__ void k_soa_to_aos(const T *soa, double *aos, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int a = 0; a < 3; a++) aos[3 * i + a] = (double)soa[a * n + i];
}
void launch_aos_to_soa(const double *aos, double *soa, int64_t n, cudaStream_t st) {
  k_aos_to_soa<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(aos, soa, n);
}
// The same conversion of new positions, which also sets the step counter
// (a kernel argument instead of a copy from host memory).
__global__ void k_aos_to_soa_step(const double *aos, double *soa, int64_t n, long long *step, long long s) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *step = s;
  if (i >= n) return;
  for (int a = 0; a < 3; a++) soa[a * n + i] = aos[3 * i + a];
}
void launch_aos_to_soa_step(const double *aos, double *soa, int64_t n, long long *step, long long s,
                            cudaStream_t st) {
  k_aos_to_soa_step<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(aos, soa, n, step, s);
}
void launch_soa_to_aos_d(const double *soa, double *aos, int64_t n, cudaStream_t st) {
  k_soa_to_aos<double><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(soa, aos, n);
}
void launch_soa_to_aos_f(const float *soa, double *aos, int64_t n, cudaStream_t st) {
  k_soa_to_aos<float><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(soa, aos, n);
}

}  // namespace rb
