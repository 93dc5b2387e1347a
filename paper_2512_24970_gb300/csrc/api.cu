// C ABI of the library (include/rbsog.h): context and device memory, system
// set-up, the force evaluation sequence, the CUDA-graph-captured MD step,
// state I/O and the parity hooks.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ctx_internal.h"
#include "rbsog_internal.cuh"
#include "setup.h"

using rb::View;

struct rbsog_ctx {
  int dev = 0;
  int nsm = 0;
  cudaStream_t user = nullptr;  // caller's stream (may be the legacy stream)
  cudaStream_t st = nullptr;    // library stream (capturable)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::string err;
  bool has_system = false;
  bool forces_valid = false;
  rbsog_params prm{};
  int64_t n = 0;
  int ns = 0;
  std::vector<double> charge, mass, bmh;
  rb::SogParams sog;
  rb::Sampler samp;
  double self_energy = 0.0;
  View v{};                    // device view (evaluation)
  std::vector<void *> allocs;  // system-lifetime device buffers
  int Pmax = 0;
  double *stage = nullptr;     // [n][3] FP64 staging
  cudaGraphExec_t gexec = nullptr;       // step graph (with kept lists: the build variant)
  cudaGraphExec_t gexec_keep = nullptr;  // kept lists: the variant that reuses them
  cudaGraph_t gstep = nullptr;           // the captured step graph behind gexec (ensemble child graphs)
  cudaGraphExec_t geval[2] = {};         // force-only evaluation graphs, by the view's build flag
  bool eval_ok[2] = {false, false};
  uint64_t graph_gen = 0;                // bumped at every capture
  bool graph_ok = false;
  bool lists_valid = false;              // kept lists built since the last set_system / set_state
  bool origin_pending = false;           // the next build uses x_origin (rbsog_set_list_origin)
  double *x_origin = nullptr;            // [3][n] positions for that build
  double *x_save = nullptr;              // [3][n] the current positions meanwhile
  bool nh_primed = false;                // Nose-Hoover: 2K of the current velocities is in the chain state
  int64_t host_step = 0;                 // mirror of the device step counter
  bool own_stream = false;
  bool profiling = false;
  cudaStream_t st2 = nullptr;                   // side stream of the structure-factor branch
  cudaStream_t st2_hi = nullptr;                // the same at the device's greatest priority
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_fork0 = nullptr;
  cudaEvent_t ev_copy = nullptr;                // rbsog_move_atoms: the host data has been read
  cudaEvent_t prof[12] = {};  // stage boundaries, see rbsog_get_stage_times
  int rho_bps = 2;            // mixed structure factor: resident blocks per SM the tiling aims at
  rbsog_schedule sched{0, 2, 2, 4, 1, 0, 0, 0, 0};  // far-field launch shapes (rbsog_set_schedule)
};

namespace {

int fail(rbsog_ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg;
  return code;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(ctx, RBSOG_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
int dalloc(rbsog_ctx *ctx, T **p, size_t count) {
  void *q = nullptr;
  if (count == 0) count = 1;
  CK(cudaMalloc(&q, sizeof(T) * count));
  ctx->allocs.push_back(q);
  *p = (T *)q;
  return RBSOG_OK;
}

// Every captured graph holds the context's view by value: any change of the
// view (or of what run_force launches) drops them.
void invalidate_graphs(rbsog_ctx *ctx) {
  ctx->graph_ok = false;
  ctx->eval_ok[0] = ctx->eval_ok[1] = false;
}

void free_system(rbsog_ctx *ctx) {
  for (int k = 0; k < 2; k++) {
    if (ctx->geval[k]) cudaGraphExecDestroy(ctx->geval[k]);
    ctx->geval[k] = nullptr;
    ctx->eval_ok[k] = false;
  }
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->gexec_keep) cudaGraphExecDestroy(ctx->gexec_keep);
  if (ctx->gstep) cudaGraphDestroy(ctx->gstep);
  ctx->gstep = nullptr;
  ctx->graph_gen++;
  ctx->gexec = nullptr;
  ctx->gexec_keep = nullptr;
  invalidate_graphs(ctx);
  ctx->lists_valid = false;
  ctx->origin_pending = false;
  ctx->x_origin = ctx->x_save = nullptr;
  for (void *p : ctx->allocs) cudaFree(p);
  ctx->allocs.clear();
  ctx->has_system = false;
  ctx->forces_valid = false;
}

// With a library-owned stream, order its work after the caller's (legacy)
// stream and the caller's after ours; with a caller stream nothing to do.
int enter(rbsog_ctx *ctx) {
  CK(cudaSetDevice(ctx->dev));
  if (ctx->own_stream) {
    CK(cudaEventRecord(ctx->ev_in, ctx->user));
    CK(cudaStreamWaitEvent(ctx->st, ctx->ev_in, 0));
  }
  return RBSOG_OK;
}
int leave(rbsog_ctx *ctx) {
  if (ctx->own_stream) {
    CK(cudaEventRecord(ctx->ev_out, ctx->st));
    CK(cudaStreamWaitEvent(ctx->user, ctx->ev_out, 0));
  }
  return RBSOG_OK;
}

int check_launch(rbsog_ctx *ctx) {
  CK(cudaGetLastError());
  return RBSOG_OK;
}

// One force evaluation; mode 0 = evaluate, 1 = VV step, 2 = BAOAB step.
// Two branches (of the captured step graph): the k-batch draw needs only the
// step counter, the structure factor and the far-field force only the
// prepared coordinates and the k-batch, so they run on a side stream,
// concurrently with the integrator, the binning and the near field; the
// branches join for the total force and the closing half kick.  With kept
// lists, v.build selects binning + list build + evaluation, else the
// evaluation of the last build's lists alone.
int run_force(rbsog_ctx *ctx, const View &v0, int mode, int step_off, bool energy) {
  View v = v0;                     // energy evaluations also carry the virial partials
  v.npart = energy ? rb::NEAR_NPART : 4;
  v.want_vir = energy ? 1 : 0;
  // the longer branch first (priorities are kept as node priorities in the
  // graph).  FP64: the far field (its FP64 sines); measured on one box with
  // kept lists, both branches at the same priority were 17 % slower per step.
  // Mixed: the two branches are about as long; the far field first was 0.7 %
  // slower than the same priority, the near field first 10 %.
  cudaStream_t st = ctx->st, st2 = v.prec == RBSOG_FP64 ? ctx->st2_hi : ctx->st2;
  const bool pr = ctx->profiling;
  // inside stream capture the stage events must become event-record nodes
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(st, &cap));
  const unsigned evflag = (cap == cudaStreamCaptureStatusActive) ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (pr) CK(cudaEventRecordWithFlags(ctx->prof[0], st, evflag));
  CK(cudaEventRecord(ctx->ev_fork0, st));
  CK(cudaStreamWaitEvent(st2, ctx->ev_fork0, 0));
  if (pr) CK(cudaEventRecordWithFlags(ctx->prof[3], st2, evflag));
  rb::launch_ksample(v, st2, step_off);
  rb::launch_prepare(v, st, mode, step_off);
  if (pr) CK(cudaEventRecordWithFlags(ctx->prof[1], st, evflag));
  CK(cudaEventRecord(ctx->ev_fork, st));
  CK(cudaStreamWaitEvent(st2, ctx->ev_fork, 0));
  // side branch: structure factor, its reduction, far-field force
  if (pr) CK(cudaEventRecordWithFlags(ctx->prof[9], st2, evflag));
  rb::launch_rho(v, st2);
  if (pr) CK(cudaEventRecordWithFlags(ctx->prof[10], st2, evflag));
  rb::launch_rhosum(v, st2, energy);
  if (pr) CK(cudaEventRecordWithFlags(ctx->prof[11], st2, evflag));
  rb::launch_farforce(v, st2);
  if (pr) CK(cudaEventRecordWithFlags(ctx->prof[4], st2, evflag));
  CK(cudaEventRecord(ctx->ev_join, st2));
  // main branch: binning, near field, F^corr
  if (!v.kept || v.build) rb::launch_bin(v, st);
  if (pr) CK(cudaEventRecordWithFlags(ctx->prof[2], st, evflag));
  if (!v.kept) {
    rb::launch_near(v, st, step_off, energy);
  } else {
    if (v.build) rb::launch_build_lists(v, st);
    rb::launch_sample_batch(v, st, step_off);
    rb::launch_near_kept(v, st, step_off, energy);
  }
  if (pr) CK(cudaEventRecordWithFlags(ctx->prof[7], st, evflag));
  rb::launch_corr(v, st, step_off);
  if (pr) CK(cudaEventRecordWithFlags(ctx->prof[5], st, evflag));
  CK(cudaStreamWaitEvent(st, ctx->ev_join, 0));
  if (pr) CK(cudaEventRecordWithFlags(ctx->prof[6], st, evflag));
  rb::launch_finish(v, st, mode);
  if (mode != 0 && v.integ == RBSOG_NOSE_HOOVER) rb::launch_nh_close(v, st);
  if (pr) CK(cudaEventRecordWithFlags(ctx->prof[8], st, evflag));
  return check_launch(ctx);
}

// The view of a one-off evaluation: kept lists that are not valid are built
// (automatic lists: by raising the device flag the binning kernels check).
// Kept lists from the positions of rbsog_set_list_origin: one evaluation that
// bins and builds at those positions (its forces are discarded), then the
// current positions back.  The lists, slots and build positions are then those
// of a build at the origin, whatever the current positions are.
int build_at_origin(rbsog_ctx *ctx) {
  View &v = ctx->v;
  const size_t bytes = sizeof(double) * 3 * (size_t)ctx->n;
  CK(cudaMemcpyAsync(ctx->x_save, v.x, bytes, cudaMemcpyDeviceToDevice, ctx->st));
  CK(cudaMemcpyAsync(v.x, ctx->x_origin, bytes, cudaMemcpyDeviceToDevice, ctx->st));
  View vb = v;
  vb.build = 1;
  if (v.auto_lists) CK(cudaMemsetAsync(v.lflag, 0x01, sizeof(int), ctx->st));
  int rc = run_force(ctx, vb, 0, 0, false);
  CK(cudaMemcpyAsync(v.x, ctx->x_save, bytes, cudaMemcpyDeviceToDevice, ctx->st));
  if (rc) return rc;
  ctx->origin_pending = false;
  ctx->lists_valid = true;
  return RBSOG_OK;
}

int eval_view(rbsog_ctx *ctx, View &vv) {
  if (ctx->origin_pending && !ctx->lists_valid) {
    const int rc = build_at_origin(ctx);
    if (rc) return rc;
  }
  vv = ctx->v;
  vv.build = (ctx->lists_valid && !ctx->v.auto_lists) ? 0 : 1;
  if (ctx->v.auto_lists && !ctx->lists_valid) CK(cudaMemsetAsync(ctx->v.lflag, 0x01, sizeof(int), ctx->st));
  return RBSOG_OK;
}

int read_err(rbsog_ctx *ctx) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, ctx->v.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (e) {
    CK(cudaMemsetAsync(ctx->v.err, 0, sizeof(int), ctx->st));
    std::string m;
    if (e & rb::ERR_SKIN) m += " an atom moved by more than skin/2 since the last build of the kept lists "
                               "(rebuild more often or widen the skin);";
    if (e & rb::ERR_CORE_CAP) m += " core list > RBSOG_MAX_CORE;";
    if (e & rb::ERR_CELL_SHELL_CAP) m += " stencil row > RBSOG_MAX_ROW_SLOTS slots or shell > RBSOG_MAX_SHELL;";
    if (e & rb::ERR_PR_CAP) m += " P_R;";
    if (e & rb::ERR_KEPT_CAP) m += " kept list: |A| > RBSOG_MAX_CORE or |B| > RBSOG_MAX_KEPT;";
    const bool cap = (e & ~rb::ERR_SKIN) != 0;
    return fail(ctx, cap ? RBSOG_E_CAP_OVERFLOW : RBSOG_E_SKIN, (cap ? "device capacity overflow:" : "kept lists:") + m);
  }
  return RBSOG_OK;
}

// Copy [n][3] FP64 from the caller into the SoA array dst.
int import_aos(rbsog_ctx *ctx, const double *src, double *dst, int kind) {
  const int64_t n = ctx->n;
  if (kind == RBSOG_PTR_HOST) {
    CK(cudaMemcpyAsync(ctx->stage, src, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, ctx->st));
    rb::launch_aos_to_soa(ctx->stage, dst, n, ctx->st);
  } else {
    rb::launch_aos_to_soa(src, dst, n, ctx->st);
  }
  return check_launch(ctx);
}

// Copy an SoA FP64/FP32 array to the caller as [n][3] FP64.  A host copy is
// complete on return unless sync is false (the caller then synchronizes the
// stream before it returns, e.g. through read_err).
int export_aos(rbsog_ctx *ctx, const double *srcd, const float *srcf, double *dst, int kind, bool sync = true) {
  const int64_t n = ctx->n;
  double *out = (kind == RBSOG_PTR_HOST) ? ctx->stage : dst;
  if (srcd) rb::launch_soa_to_aos_d(srcd, out, n, ctx->st);
  else rb::launch_soa_to_aos_f(srcf, out, n, ctx->st);
  int rc = check_launch(ctx);
  if (rc) return rc;
  if (kind == RBSOG_PTR_HOST) {
    CK(cudaMemcpyAsync(dst, ctx->stage, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, ctx->st));
    if (sync) CK(cudaStreamSynchronize(ctx->st));
  }
  return RBSOG_OK;
}

// Host copy of a caller array (host or device pointer).
template <typename T>
int fetch(rbsog_ctx *ctx, const T *src, size_t count, int kind, std::vector<T> &out) {
  out.resize(count);
  if (count == 0) return RBSOG_OK;
  if (kind == RBSOG_PTR_HOST) {
    std::memcpy(out.data(), src, sizeof(T) * count);
  } else {
    CK(cudaMemcpy(out.data(), src, sizeof(T) * count, cudaMemcpyDeviceToHost));
  }
  return RBSOG_OK;
}

int ensure_kcap(rbsog_ctx *ctx, int P) {
  View &v = ctx->v;
  if (P <= ctx->Pmax) return RBSOG_OK;
  int rc;
  if ((rc = dalloc(ctx, &v.km, P)) || (rc = dalloc(ctx, &v.kc, P)) ||
      (rc = dalloc(ctx, &v.rho, 2 * (size_t)P)) || (rc = dalloc(ctx, &v.uf, P)) ||
      (rc = dalloc(ctx, &v.kpair, (size_t)P / 2 + 1)) ||
      (rc = dalloc(ctx, &v.kfd, 5 * (size_t)P)) ||
      (rc = dalloc(ctx, &v.rho_part, 2 * (size_t)P * (size_t)v.ntile)) || (rc = dalloc(ctx, &v.vf, P)))
    return rc;
  ctx->Pmax = P;
  return RBSOG_OK;
}

// Structure-factor tiles: enough blocks for rho_bps resident blocks per SM
// (or, with the schedule's rho_tile_atoms, that many atoms per tile)
// (mixed: the block shape of the schedule's rho_variant; FP64: blocks of
// RHO_BLOCK threads), at least 32 atoms per tile.
void set_rho_tiling(rbsog_ctx *ctx, int P) {
  View &v = ctx->v;
  const int nky = (P + rb::RHO_BLOCK * rb::RHO_KPT - 1) / (rb::RHO_BLOCK * rb::RHO_KPT);
  const int target = (v.prec == RBSOG_MIXED ? ctx->rho_bps : 4) * ctx->nsm;
  int64_t nt = (target + nky - 1) / nky;
  if (v.prec == RBSOG_MIXED && ctx->sched.rho_tile_atoms > 0)
    nt = (ctx->n + ctx->sched.rho_tile_atoms - 1) / ctx->sched.rho_tile_atoms;
  nt = std::min<int64_t>(nt, (ctx->n + 31) / 32);
  nt = std::max<int64_t>(nt, 1);
  v.tile_atoms = (int)((ctx->n + nt - 1) / nt);
  v.ntile = (int)((ctx->n + v.tile_atoms - 1) / v.tile_atoms);
}

}  // namespace

// ===========================================================================
// Internal interface of a context for the ensemble (ctx_internal.h).
namespace rb {

int ctx_prepare_step(rbsog_ctx *ctx) {
  int rc;
  if (!ctx->forces_valid) {
    View vv;
    if ((rc = eval_view(ctx, vv))) return rc;
    if ((rc = run_force(ctx, vv, 0, 0, false))) return rc;
    ctx->forces_valid = true;
    ctx->lists_valid = true;
  }
  if (!ctx->graph_ok) {
    // velocity Verlet (Nose-Hoover: with the chain's half steps) or BAOAB
    const int mode = ctx->prm.integrator == RBSOG_LANGEVIN_BAOAB ? 2 : 1;
    // variant 0 bins and builds (per-step lists: the only one); variant 1
    // evaluates the kept lists of the last build
    for (int var = 0; var < ((ctx->v.kept && !ctx->v.auto_lists) ? 2 : 1); var++) {
      View vs = ctx->v;
      vs.build = var == 0 ? 1 : 0;
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal));
      rc = run_force(ctx, vs, mode, 1, false);
      cudaError_t e = cudaStreamEndCapture(ctx->st, &g);
      if (rc) { if (g) cudaGraphDestroy(g); return rc; }
      if (e != cudaSuccess) return fail(ctx, RBSOG_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      cudaGraphExec_t &ge = var == 0 ? ctx->gexec : ctx->gexec_keep;
      if (ge) cudaGraphExecDestroy(ge);
      ge = nullptr;
      e = cudaGraphInstantiate(&ge, g, cudaGraphInstantiateFlagUseNodePriority);
      if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(ctx, RBSOG_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
      }
      if (var == 0) {                          // kept for an ensemble's graph
        if (ctx->gstep) cudaGraphDestroy(ctx->gstep);
        ctx->gstep = g;
      } else {
        cudaGraphDestroy(g);
      }
    }
    ctx->graph_gen++;
    ctx->graph_ok = true;
  }
  if (ctx->prm.integrator == RBSOG_NOSE_HOOVER && !ctx->nh_primed) {
    rb::launch_nh_prime(ctx->v, ctx->st);   // 2K of the velocities the first half step sees
    if ((rc = check_launch(ctx))) return rc;
    ctx->nh_primed = true;
  }
  return RBSOG_OK;
}

bool ctx_single_graph(const rbsog_ctx *ctx) { return !ctx->v.kept || ctx->v.auto_lists; }

cudaGraph_t ctx_step_graph(const rbsog_ctx *ctx, uint64_t *gen) {
  if (gen) *gen = ctx->graph_gen;
  return ctx->graph_ok ? ctx->gstep : nullptr;
}

void ctx_advance(rbsog_ctx *ctx, int64_t nsteps) { ctx->host_step += nsteps; }

void ctx_step_view(const rbsog_ctx *ctx, View *out, int *mode, bool *profiling) {
  View v = ctx->v;
  v.npart = 4;                     // as run_force sets them for a step
  v.want_vir = 0;
  v.build = 1;                     // per-step lists, or automatic kept lists (one graph)
  *out = v;
  *mode = ctx->prm.integrator == RBSOG_LANGEVIN_BAOAB ? 2 : (ctx->prm.integrator == RBSOG_NVE_VV ? 1 : 0);
  *profiling = ctx->profiling;
}

}  // namespace rb

// ===========================================================================
extern "C" {

int rbsog_create(rbsog_ctx **out, int cuda_device, void *cuda_stream) {
  rbsog_ctx *ctx = nullptr;
  if (!out) return RBSOG_E_INVAL;
  *out = nullptr;
  ctx = new rbsog_ctx();
  ctx->dev = cuda_device;
  ctx->user = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaSetDevice(cuda_device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, cuda_device);
  if (ctx->user) {
    ctx->st = ctx->user;
  } else if (e == cudaSuccess) {
    e = cudaStreamCreateWithFlags(&ctx->st, cudaStreamNonBlocking);
    ctx->own_stream = (e == cudaSuccess);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming);
  for (int k = 0; k < 12 && e == cudaSuccess; k++) e = cudaEventCreate(&ctx->prof[k]);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->st2, cudaStreamNonBlocking);
  int prio_least = 0, prio_greatest = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ctx->st2_hi, cudaStreamNonBlocking, prio_greatest);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork0, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_copy, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    rbsog_destroy(ctx);
    return RBSOG_E_CUDA;
  }
  *out = ctx;
  return RBSOG_OK;
}

void rbsog_destroy(rbsog_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->dev);
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  if (ctx->st2) cudaStreamSynchronize(ctx->st2);
  if (ctx->st2_hi) cudaStreamSynchronize(ctx->st2_hi);
  free_system(ctx);
  if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
  if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
  for (int k = 0; k < 12; k++)
    if (ctx->prof[k]) cudaEventDestroy(ctx->prof[k]);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->ev_fork0) cudaEventDestroy(ctx->ev_fork0);
  if (ctx->ev_copy) cudaEventDestroy(ctx->ev_copy);
  if (ctx->st2) cudaStreamDestroy(ctx->st2);
  if (ctx->st2_hi) cudaStreamDestroy(ctx->st2_hi);
  if (ctx->st && ctx->own_stream) cudaStreamDestroy(ctx->st);
  delete ctx;
}

const char *rbsog_last_error(const rbsog_ctx *ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

int rbsog_set_system(rbsog_ctx *ctx, int64_t n, const double *pos, const int32_t *species,
                     int32_t n_species, const double *charge, const double *mass,
                     const double *bmh, const double box[3], const rbsog_params *params,
                     int ptr_kind) {
  if (!ctx) return RBSOG_E_INVAL;
  if (!pos || !species || !charge || !mass || !bmh || !box || !params)
    return fail(ctx, RBSOG_E_INVAL, "null argument");
  if (ptr_kind != RBSOG_PTR_HOST && ptr_kind != RBSOG_PTR_DEVICE)
    return fail(ctx, RBSOG_E_INVAL, "bad ptr_kind");
  const rbsog_params P = *params;
  if (n < 2 || n > (int64_t)rb::SU_ID_MASK) return fail(ctx, RBSOG_E_INVAL, "n out of range (2 .. 2^28 - 1)");
  if (n_species < 1 || n_species > RBSOG_MAX_SPECIES) return fail(ctx, RBSOG_E_INVAL, "n_species out of range");
  if (!(P.b > 1.0) || P.M < 1 || P.M > RBSOG_MAX_M) return fail(ctx, RBSOG_E_INVAL, "SOG b/M out of range");
  if (!(P.r_core > 0.0) || !(P.r_shell > P.r_core)) return fail(ctx, RBSOG_E_INVAL, "need 0 < r_core < r_shell");
  if (P.P_R < 1 || P.P_R > RBSOG_MAX_PR) return fail(ctx, RBSOG_E_INVAL, "P_R out of range");
  if (P.P_F < 1) return fail(ctx, RBSOG_E_INVAL, "P_F out of range");
  if (P.precision != RBSOG_FP64 && P.precision != RBSOG_MIXED) return fail(ctx, RBSOG_E_INVAL, "bad precision");
  if (P.integrator != RBSOG_NVE_VV && P.integrator != RBSOG_LANGEVIN_BAOAB && P.integrator != RBSOG_NOSE_HOOVER)
    return fail(ctx, RBSOG_E_INVAL, "bad integrator");
  if (P.integrator == RBSOG_NOSE_HOOVER &&
      (!(P.tdamp > 0.0) || P.nh_chain < 1 || P.nh_chain > RBSOG_MAX_NH_CHAIN || !(P.T > 0.0)))
    return fail(ctx, RBSOG_E_INVAL, "Nose-Hoover needs tdamp > 0, T > 0 and 1 <= nh_chain <= RBSOG_MAX_NH_CHAIN");
  if (P.list_every < RBSOG_LISTS_AUTO) return fail(ctx, RBSOG_E_INVAL, "list_every must be >= -1");
  if (P.list_every != 0 && !(P.skin >= 0.0)) return fail(ctx, RBSOG_E_INVAL, "skin must be >= 0");
  const bool kept = P.list_every != 0;
  const double r_list = P.r_shell + (kept ? P.skin : 0.0);  // outer radius of the lists
  std::vector<double> hb(3);
  int rc;
  if ((rc = fetch(ctx, box, 3, RBSOG_PTR_HOST, hb))) return rc;
  for (int a = 0; a < 3; a++) {
    if (!(hb[a] > 0.0)) return fail(ctx, RBSOG_E_INVAL, "box must be positive");
    if (hb[a] < 2.0 * r_list) return fail(ctx, RBSOG_E_BOX_TOO_SMALL, "box length < 2 (r_shell + skin)");
  }
  std::vector<double> hpos, hq, hm, hbmh;
  std::vector<int32_t> hsp;
  if ((rc = fetch(ctx, pos, 3 * (size_t)n, ptr_kind, hpos)) || (rc = fetch(ctx, species, (size_t)n, ptr_kind, hsp)) ||
      (rc = fetch(ctx, charge, (size_t)n_species, ptr_kind, hq)) || (rc = fetch(ctx, mass, (size_t)n_species, ptr_kind, hm)) ||
      (rc = fetch(ctx, bmh, 5 * (size_t)n_species * n_species, ptr_kind, hbmh)))
    return rc;
  double qsum = 0.0;
  for (int64_t i = 0; i < n; i++) {
    if (hsp[i] < 0 || hsp[i] >= n_species) return fail(ctx, RBSOG_E_INVAL, "species out of range");
    qsum += hq[hsp[i]];
  }
  if (std::fabs(qsum) > 1e-10) return fail(ctx, RBSOG_E_NONNEUTRAL, "system is not charge neutral");
  for (int a = 0; a < n_species; a++) {
    if (!(hm[a] > 0.0)) return fail(ctx, RBSOG_E_INVAL, "mass must be positive");
    for (int b = 0; b < n_species; b++)
      for (int k = 0; k < 5; k++)
        if (hbmh[5 * (a * n_species + b) + k] != hbmh[5 * (b * n_species + a) + k])
          return fail(ctx, RBSOG_E_INVAL, "BMH table not symmetric");
    for (int b = 0; b < n_species; b++)
      if (!(hbmh[5 * (a * n_species + b) + 2] > 0.0)) return fail(ctx, RBSOG_E_INVAL, "BMH rho must be positive");
  }
  // --- SOG parameters (Sec. 2.1) ------------------------------------------
  rb::SogParams sog;
  if (P.s <= 0.0 || P.w0 <= 0.0) {
    if ((rc = rb::sog_solve(P.b, P.M, P.r_shell, sog)) != RBSOG_OK)
      return fail(ctx, rc, "no C1 SOG bandwidth in [r_c/6, r_c/2]");
  } else {
    rb::sog_fill(P.b, P.M, P.s, P.w0, sog);
  }
  rb::Sampler samp;
  rb::sampler_build(sog, hb.data(), samp);
  std::vector<float> gt, ft;
  rb::sog_tables(sog, P.r_shell * P.r_shell, rb::NT_TAB, gt, ft);

  // --- (re)allocate ----------------------------------------------------------
  if ((rc = enter(ctx))) return rc;
  CK(cudaStreamSynchronize(ctx->st));
  free_system(ctx);
  ctx->prm = P;
  ctx->n = n;
  ctx->ns = n_species;
  ctx->charge = hq;
  ctx->mass = hm;
  ctx->bmh = hbmh;
  ctx->sog = sog;
  ctx->samp = samp;
  ctx->Pmax = 0;
  View &v = ctx->v;
  v = View{};
  v.n = n;
  v.ns = n_species;
  v.M = P.M;
  v.G = P.M + 1;
  v.prec = P.precision;
  v.whole_shell = 0;
  v.P_R = P.P_R;
  v.P_F = P.P_F;
  v.P = P.P_F;
  v.fixed_k = 0;
  v.integ = P.integrator;
  v.seed = P.seed;
  v.V = hb[0] * hb[1] * hb[2];
  for (int a = 0; a < 3; a++) {
    v.L[a] = hb[a];
    v.invL[a] = 1.0 / hb[a];
    v.hp[a] = (float)(hb[a] * 0x1p-23);
    v.hf[a] = (float)(hb[a] * 0x1p-32);
    v.hd[a] = hb[a] * 0x1p-32;
    v.kunit[a] = 2.0 * M_PI / hb[a];
    v.nc[a] = rb::cell_count(hb[a], r_list);
  }
  v.rc2f = (float)(P.r_core * P.r_core);
  v.rs2f = (float)(P.r_shell * P.r_shell);
  v.kept = kept ? 1 : 0;
  v.auto_lists = P.list_every == RBSOG_LISTS_AUTO ? 1 : 0;
  v.build = 0;
  v.rl2f = (float)(r_list * r_list);
  v.a_inside = (kept && (P.r_core + P.skin) * (P.r_core + P.skin) < 0.98 * P.r_shell * P.r_shell) ? 1 : 0;
  // an atom may move by skin/2 (pair distances by skin): shaded by 2^-10 so
  // that the FP32 predicate's rounding stays inside the margin
  v.half_skin2 = 0.25 * P.skin * P.skin * (1.0 - 1.0 / 1024.0);
  v.ncell = v.nc[0] * v.nc[1] * v.nc[2];
  v.small = (v.nc[0] < rb::STENCIL || v.nc[1] < rb::STENCIL || v.nc[2] < rb::STENCIL) ? 1 : 0;
  // the near field's union of a chunk's x-stencils (<= 8 cells) may meet
  // itself on short rows: there it takes whole rows and minimum images
  v.wrap = (v.small || v.nc[0] < 8) ? 1 : 0;
  v.tscale = (float)(rb::NT_TAB / (P.r_shell * P.r_shell));
  v.S = samp.S;
  v.dt = P.dt;
  v.c1 = std::exp(-P.gamma * P.dt);
  for (int a = 0; a < n_species; a++) {
    v.qs[a] = hq[a];
    v.kick[a] = 0.5 * P.dt * rb::FCONV / hm[a];
    v.qfar[a] = -rb::KE * hq[a] / v.V;
    v.sig_ou[a] = std::sqrt(std::max(0.0, (1.0 - v.c1 * v.c1) * rb::KBOLTZ * P.T * rb::FCONV / hm[a]));
    v.massv[a] = hm[a];
  }
  v.nh_M = P.integrator == RBSOG_NOSE_HOOVER ? P.nh_chain : 1;
  v.nh_nblk = (int)((n + rb::PREP_BLOCK - 1) / rb::PREP_BLOCK);
  v.nh_kT = rb::KBOLTZ * P.T;
  v.nh_g = 3.0 * (double)n - 3.0;
  for (int j = 0; j < RBSOG_MAX_NH_CHAIN; j++)
    v.nh_Q[j] = (j == 0 ? v.nh_g : 1.0) * v.nh_kT * P.tdamp * P.tdamp;
  v.nblk_atoms = (int)((n + 255) / 256);
  v.nblk_kq = (P.P_F + 7) / 8;   // one warp per sample
  // chunks <= n / NEAR_CHUNK + rows; one warp per chunk
  // chunks (8 padded slots) <= nslot / 8 + rows; one warp per chunk
  v.nblk_near = (int)(((n + 3 * (int64_t)v.ncell + rb::NEAR_CHUNK - 1) / rb::NEAR_CHUNK + (int64_t)v.nc[1] * v.nc[2] +
                       rb::NEAR_WARPS - 1) / rb::NEAR_WARPS);
  v.far_A = ctx->sched.far_atoms_per_thread;
  v.far_S = ctx->sched.far_segments;
  v.rho_var = ctx->sched.rho_variant;
  v.far_packed = ctx->sched.far_packed;
  v.near_bps = ctx->sched.near_blocks_per_sm;
  v.near_wide = ctx->sched.near_wide;
  v.rho_reduce = ctx->sched.rho_reduce;
  v.nsm = ctx->nsm;
  ctx->rho_bps = ctx->sched.rho_blocks_per_sm;
  set_rho_tiling(ctx, P.P_F);
  // self term U_F^self = k_e/2 sum_i q_i^2 F(0)
  double F0 = 0.0, q2 = 0.0;
  for (int m = 0; m <= P.M; m++) F0 += sog.w[m];
  for (int64_t i = 0; i < n; i++) q2 += hq[hsp[i]] * hq[hsp[i]];
  ctx->self_energy = 0.5 * rb::KE * q2 * F0;

  const size_t N = (size_t)n;
  v.nslot = (int)(N + (size_t)(rb::CELL_ALIGN - 1) * (size_t)v.ncell);
  const size_t NS = (size_t)v.nslot;
  int *spc_d = nullptr;
  rb::PairF *pf = nullptr;
  rb::PairD *pd = nullptr;
  double *wa = nullptr, *w = nullptr, *h2 = nullptr;
  float4 *gtab = nullptr, *ftab = nullptr;
  unsigned long long *cmix = nullptr, *cdf = nullptr;
  int *off0 = nullptr, *off2 = nullptr, *nmax = nullptr;
  if ((rc = dalloc(ctx, &v.x, 3 * N)) || (rc = dalloc(ctx, &v.v, 3 * N)) ||
      (rc = dalloc(ctx, &v.Ff, 3 * N)) || (rc = dalloc(ctx, &v.FNf, 3 * N)) || (rc = dalloc(ctx, &v.FFf, 3 * N)) ||
      (rc = dalloc(ctx, &v.Fd, 3 * N)) || (rc = dalloc(ctx, &v.FNd, 3 * N)) || (rc = dalloc(ctx, &v.FFd, 3 * N)) ||
      (rc = dalloc(ctx, &spc_d, N)) || (rc = dalloc(ctx, &v.ua, N)) || (rc = dalloc(ctx, &v.cellid, N)) ||
      (rc = dalloc(ctx, &v.cell_count, (size_t)v.ncell + (size_t)v.nc[1] * v.nc[2])) ||
      (rc = dalloc(ctx, &v.row_start, (size_t)v.nc[1] * v.nc[2])) || (rc = dalloc(ctx, &v.key_tmp, NS)) || (rc = dalloc(ctx, &v.cell_start, (size_t)v.ncell + 1)) ||
      (rc = dalloc(ctx, &v.cell_cursor, (size_t)v.ncell)) || (rc = dalloc(ctx, &v.perm_tmp, NS)) ||
      (rc = dalloc(ctx, &v.perm, NS)) || (rc = dalloc(ctx, &v.slot_of, N)) ||
      (rc = dalloc(ctx, &v.row_chunk, (size_t)v.nc[1] * v.nc[2] + 1)) ||
      (rc = dalloc(ctx, &v.chunk_info, (size_t)v.nblk_near * rb::NEAR_WARPS)) || (rc = dalloc(ctx, &v.sx, NS)) ||
      (rc = dalloc(ctx, &v.sy, NS)) || (rc = dalloc(ctx, &v.sz, NS)) || (rc = dalloc(ctx, &v.su, NS)) || (rc = dalloc(ctx, &v.near_part, (size_t)rb::NEAR_NPART * v.nblk_near * rb::NEAR_WARPS)) ||
      (rc = dalloc(ctx, &v.corr_part, (size_t)rb::NEAR_NPART * 64)) || (rc = dalloc(ctx, &v.corr_ticket, 1)) || (rc = dalloc(ctx, &v.corr_acc, 16 * (size_t)rb::CORR_COPIES)) ||
      (rc = dalloc(ctx, &v.red, 24)) || (rc = dalloc(ctx, &v.err, 1)) || (rc = dalloc(ctx, &v.step, 1)) ||
      (rc = dalloc(ctx, &pf, (size_t)n_species * n_species)) || (rc = dalloc(ctx, &pd, (size_t)n_species * n_species)) ||
      (rc = dalloc(ctx, &wa, (size_t)v.G)) || (rc = dalloc(ctx, &w, (size_t)v.G)) || (rc = dalloc(ctx, &h2, (size_t)v.G)) ||
      (rc = dalloc(ctx, &gtab, rb::NT_TAB)) || (rc = dalloc(ctx, &ftab, rb::NT_TAB)) ||
      (rc = dalloc(ctx, &cmix, samp.cmix.size())) || (rc = dalloc(ctx, &cdf, samp.cdf.size())) ||
      (rc = dalloc(ctx, &off0, samp.off0.size())) || (rc = dalloc(ctx, &off2, samp.off2.size())) ||
      (rc = dalloc(ctx, &nmax, samp.nmax.size())) || (rc = dalloc(ctx, &ctx->stage, 3 * N)) ||
      (rc = ensure_kcap(ctx, P.P_F))) {
    free_system(ctx);
    return rc;
  }
  if ((rc = dalloc(ctx, &v.lflag, 1)) || (rc = dalloc(ctx, &v.nbuild, 1)) ||
      (rc = dalloc(ctx, &v.nh, rb::NH_STATE)) || (rc = dalloc(ctx, &v.ke_part, (size_t)v.nh_nblk)) ||
      (rc = dalloc(ctx, &v.kin_part, 6 * (size_t)v.nh_nblk)) || (rc = dalloc(ctx, &v.kin, 6)) ||
      (kept && ((rc = dalloc(ctx, &v.lA, NS * RBSOG_MAX_CORE)) || (rc = dalloc(ctx, &v.lB, NS * RBSOG_MAX_KEPT)) ||
                (rc = dalloc(ctx, &v.nAB, NS)) || (rc = dalloc(ctx, &v.bsel, NS * (size_t)P.P_R)) ||
                (rc = dalloc(ctx, &v.lB16, NS * RBSOG_MAX_KEPT)) || (rc = dalloc(ctx, &v.b16_over, 1)) || (rc = dalloc(ctx, &v.xb, 3 * N))))) {
    free_system(ctx);
    return rc;
  }
  v.row_count = v.cell_count + v.ncell;
  v.spc = spc_d;
  v.pf = pf;
  v.pd = pd;
  v.sog_wa = wa;
  v.sog_w = w;
  v.sog_h = h2;
  v.gtab = gtab;
  v.ftab = ftab;
  v.cmix = cmix;
  v.cdf = cdf;
  v.cdf_off0 = off0;
  v.cdf_off2 = off2;
  v.cdf_nmax = nmax;
  // pair records
  std::vector<rb::PairF> hpf((size_t)n_species * n_species);
  std::vector<rb::PairD> hpd((size_t)n_species * n_species);
  const double LOG2E = 1.4426950408889634;
  for (int a = 0; a < n_species; a++)
    for (int b = 0; b < n_species; b++) {
      const double *t = &hbmh[5 * (a * n_species + b)];
      const double A = t[0], sig = t[1], rho = t[2], C = t[3], D = t[4];
      const double kqq = rb::KE * hq[a] * hq[b];
      rb::PairF f{};
      f.kqq = (float)kqq; f.Ar = (float)(A / rho); f.lr = (float)(LOG2E / rho); f.sig = (float)sig;
      f.C6 = (float)(6.0 * C); f.D8 = (float)(8.0 * D); f.A = (float)A; f.C = (float)C; f.D = (float)D;
      hpf[a * n_species + b] = f;
      hpd[a * n_species + b] = rb::PairD{kqq, A, sig, rho, C, D};
    }
  std::vector<double> hwa(v.G), hw(v.G), hh2(v.G);
  for (int m = 0; m < v.G; m++) {
    hwa[m] = sog.w[m] / sog.a[m];
    hw[m] = sog.w[m];
    hh2[m] = 1.0 / (2.0 * sog.a[m]);
  }
  // positions [n][3] -> SoA
  std::vector<double> soa(3 * N);
  for (size_t i = 0; i < N; i++)
    for (int a = 0; a < 3; a++) soa[a * N + i] = hpos[3 * i + a];
  auto up = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->st);
  };
  CK(up(v.x, soa.data(), sizeof(double) * 3 * N));
  CK(cudaMemsetAsync(v.v, 0, sizeof(double) * 3 * N, ctx->st));
  CK(cudaMemsetAsync(v.Ff, 0, sizeof(float) * 3 * N, ctx->st));
  CK(cudaMemsetAsync(v.Fd, 0, sizeof(double) * 3 * N, ctx->st));
  CK(up(spc_d, hsp.data(), sizeof(int) * N));
  CK(up(pf, hpf.data(), sizeof(rb::PairF) * hpf.size()));
  CK(up(pd, hpd.data(), sizeof(rb::PairD) * hpd.size()));
  CK(up(wa, hwa.data(), sizeof(double) * v.G));
  CK(up(w, hw.data(), sizeof(double) * v.G));
  CK(up(h2, hh2.data(), sizeof(double) * v.G));
  CK(up(gtab, gt.data(), sizeof(float) * gt.size()));
  CK(up(ftab, ft.data(), sizeof(float) * ft.size()));
  CK(up(cmix, samp.cmix.data(), sizeof(unsigned long long) * samp.cmix.size()));
  CK(up(cdf, samp.cdf.data(), sizeof(unsigned long long) * samp.cdf.size()));
  CK(up(off0, samp.off0.data(), sizeof(int) * samp.off0.size()));
  CK(up(off2, samp.off2.data(), sizeof(int) * samp.off2.size()));
  CK(up(nmax, samp.nmax.data(), sizeof(int) * samp.nmax.size()));
  CK(cudaMemsetAsync(v.err, 0, sizeof(int), ctx->st));
  CK(cudaMemsetAsync(v.step, 0, sizeof(long long), ctx->st));
  CK(cudaMemsetAsync(v.red, 0, sizeof(double) * 24, ctx->st));
  CK(cudaMemsetAsync(v.cell_count, 0, sizeof(int) * ((size_t)v.ncell + (size_t)v.nc[1] * v.nc[2]), ctx->st));
  CK(cudaMemsetAsync(v.corr_ticket, 0, sizeof(unsigned), ctx->st));
  if (v.b16_over) CK(cudaMemsetAsync(v.b16_over, 0, sizeof(int), ctx->st));
  CK(cudaMemsetAsync(v.lflag, 0, sizeof(int), ctx->st));
  CK(cudaMemsetAsync(v.nh, 0, sizeof(double) * rb::NH_STATE, ctx->st));   // the chain at rest
  CK(cudaMemsetAsync(v.nbuild, 0, sizeof(unsigned long long), ctx->st));
  CK(cudaMemsetAsync(v.slot_of, 0, sizeof(int) * N, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));  // host vectors go out of scope
  ctx->has_system = true;
  ctx->forces_valid = false;
  ctx->lists_valid = false;
  ctx->nh_primed = false;
  ctx->host_step = 0;
  return leave(ctx);
}

int rbsog_set_core_radii(rbsog_ctx *ctx, const double *r_core_pair) {
  if (!ctx) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  View &v = ctx->v;
  if (!r_core_pair) {
    v.core_pair = 0;
  } else {
    const int ns = v.ns;
    for (int a = 0; a < ns; a++)
      for (int b = 0; b < ns; b++) {
        const double r = r_core_pair[a * ns + b];
        if (!(r > 0.0) || r > ctx->prm.r_core) return fail(ctx, RBSOG_E_INVAL, "core radii must lie in (0, r_core]");
        if (r != r_core_pair[b * ns + a]) return fail(ctx, RBSOG_E_INVAL, "core radii must be symmetric");
        v.rc2p[a * ns + b] = (float)(r * r);
      }
    v.core_pair = 1;
  }
  invalidate_graphs(ctx);
  ctx->forces_valid = false;
  ctx->lists_valid = false;
  return RBSOG_OK;
}

int rbsog_set_velocities(rbsog_ctx *ctx, const double *vel, int ptr_kind) {
  if (!ctx) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  if (!vel) return fail(ctx, RBSOG_E_INVAL, "null velocities");
  int rc;
  if ((rc = enter(ctx))) return rc;
  if ((rc = import_aos(ctx, vel, ctx->v.v, ptr_kind))) return rc;
  if (ptr_kind == RBSOG_PTR_HOST) CK(cudaStreamSynchronize(ctx->st));
  ctx->nh_primed = false;
  return leave(ctx);
}

// A force-only evaluation: replays a captured graph (one launch instead of a
// dozen kernel launches from the host), captured on first use.
static int eval_forces_graph(rbsog_ctx *ctx, const View &vv) {
  int rc;
  const int key = vv.build ? 1 : 0;
  if (!ctx->eval_ok[key]) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal));
    rc = run_force(ctx, vv, 0, 0, false);
    cudaError_t e = cudaStreamEndCapture(ctx->st, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return fail(ctx, RBSOG_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    if (ctx->geval[key]) cudaGraphExecDestroy(ctx->geval[key]);
    ctx->geval[key] = nullptr;
    e = cudaGraphInstantiate(&ctx->geval[key], g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(ctx, RBSOG_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    ctx->eval_ok[key] = true;
  }
  CK(cudaGraphLaunch(ctx->geval[key], ctx->st));
  return RBSOG_OK;
}

int rbsog_compute_forces(rbsog_ctx *ctx, double *forces, double *energy, double *virial,
                         int ptr_kind) {
  if (!ctx) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  int rc;
  const bool ev = energy != nullptr || virial != nullptr;
  if ((rc = enter(ctx))) return rc;
  View vv;
  if ((rc = eval_view(ctx, vv))) return rc;
  if (ev) {
    if ((rc = run_force(ctx, vv, 0, 0, true))) return rc;
  } else {
    if ((rc = eval_forces_graph(ctx, vv))) return rc;
  }
  ctx->forces_valid = true;
  ctx->lists_valid = true;
  if (forces) {
    // host forces: the copy completes with read_err's synchronization below
    const bool sync = !(ptr_kind == RBSOG_PTR_HOST && !ev);
    if (ctx->v.prec == RBSOG_FP64) rc = export_aos(ctx, ctx->v.Fd, nullptr, forces, ptr_kind, sync);
    else rc = export_aos(ctx, nullptr, ctx->v.Ff, forces, ptr_kind, sync);
    if (rc) return rc;
  }
  if (ev) {
    double red[24];
    CK(cudaMemcpyAsync(red, ctx->v.red, sizeof(red), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    const double e[4] = {red[3], red[4], ctx->self_energy, red[3] + red[4] - ctx->self_energy};
    double w[6];
    for (int c = 0; c < 6; c++) w[c] = red[5 + c] + red[11 + c];   // W_N + W_F*
    if (energy) {
      if (ptr_kind == RBSOG_PTR_HOST) std::memcpy(energy, e, sizeof(e));
      else CK(cudaMemcpyAsync(energy, e, sizeof(e), cudaMemcpyHostToDevice, ctx->st));
    }
    if (virial) {
      if (ptr_kind == RBSOG_PTR_HOST) std::memcpy(virial, w, sizeof(w));
      else CK(cudaMemcpyAsync(virial, w, sizeof(w), cudaMemcpyHostToDevice, ctx->st));
    }
    if (ptr_kind != RBSOG_PTR_HOST) CK(cudaStreamSynchronize(ctx->st));   // e, w are on this stack
  }
  if (ptr_kind == RBSOG_PTR_HOST || ev) {
    if ((rc = read_err(ctx))) return rc;
  }
  return leave(ctx);
}

int rbsog_step(rbsog_ctx *ctx, int64_t nsteps) {
  if (!ctx) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  if (nsteps < 0) return fail(ctx, RBSOG_E_INVAL, "negative step count");
  if (!(ctx->prm.dt > 0.0)) return fail(ctx, RBSOG_E_INVAL, "dt must be positive");
  int rc;
  if ((rc = enter(ctx))) return rc;
  if ((rc = rb::ctx_prepare_step(ctx))) return rc;
  // kept lists are rebuilt at the steps that are multiples of list_every
  const int64_t every = ctx->prm.list_every;
  for (int64_t k = 0; k < nsteps; k++) {
    const int64_t next = ctx->host_step + 1;
    const bool build = !ctx->v.kept || ctx->v.auto_lists || next % every == 0;
    CK(cudaGraphLaunch(build ? ctx->gexec : ctx->gexec_keep, ctx->st));
    ctx->host_step = next;
  }
  return leave(ctx);
}

int rbsog_get_state(rbsog_ctx *ctx, double *pos, double *vel, int64_t *step, int ptr_kind) {
  if (!ctx) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  int rc;
  if ((rc = enter(ctx))) return rc;
  if (pos && (rc = export_aos(ctx, ctx->v.x, nullptr, pos, ptr_kind))) return rc;
  if (vel && (rc = export_aos(ctx, ctx->v.v, nullptr, vel, ptr_kind))) return rc;
  if (step) {
    long long s = 0;
    CK(cudaMemcpyAsync(&s, ctx->v.step, sizeof(s), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    *step = (int64_t)s;
  }
  return leave(ctx);
}

int rbsog_set_state(rbsog_ctx *ctx, const double *pos, const double *vel, int64_t step,
                    int ptr_kind) {
  if (!ctx) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  if (step < 0) return fail(ctx, RBSOG_E_INVAL, "negative step");
  int rc;
  if ((rc = enter(ctx))) return rc;
  if (pos && (rc = import_aos(ctx, pos, ctx->v.x, ptr_kind))) return rc;
  if (pos && ptr_kind == RBSOG_PTR_HOST) CK(cudaStreamSynchronize(ctx->st));
  if (vel && (rc = import_aos(ctx, vel, ctx->v.v, ptr_kind))) return rc;
  long long s = step;
  CK(cudaMemcpyAsync(ctx->v.step, &s, sizeof(s), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  ctx->forces_valid = false;
  ctx->lists_valid = false;
  ctx->nh_primed = false;
  ctx->host_step = step;
  return leave(ctx);
}

int rbsog_move_atoms(rbsog_ctx *ctx, const double *pos, int64_t step, int ptr_kind) {
  if (!ctx || !pos) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  if (step < 0) return fail(ctx, RBSOG_E_INVAL, "negative step");
  int rc;
  if ((rc = enter(ctx))) return rc;
  long long s = step;
  if (ptr_kind == RBSOG_PTR_HOST) {
    // the caller's positions and s are read by the copies; the return waits
    // for those only, the layout conversion runs on while the caller goes on
    CK(cudaMemcpyAsync(ctx->stage, pos, sizeof(double) * 3 * (size_t)ctx->n, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->v.step, &s, sizeof(s), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaEventRecord(ctx->ev_copy, ctx->st));
    rb::launch_aos_to_soa(ctx->stage, ctx->v.x, ctx->n, ctx->st);
    if ((rc = check_launch(ctx))) return rc;
    CK(cudaEventSynchronize(ctx->ev_copy));
  } else {
    if ((rc = import_aos(ctx, pos, ctx->v.x, ptr_kind))) return rc;
    CK(cudaMemcpyAsync(ctx->v.step, &s, sizeof(s), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));          // s is on this stack
  }
  ctx->forces_valid = false;                   // the kept lists stay; the next evaluation checks them
  ctx->host_step = step;
  return leave(ctx);
}

int rbsog_forces_at(rbsog_ctx *ctx, const double *pos, int64_t step, double *forces, int ptr_kind) {
  if (!ctx || !pos || !forces) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  if (step < 0) return fail(ctx, RBSOG_E_INVAL, "negative step");
  if (ptr_kind != RBSOG_PTR_HOST && ptr_kind != RBSOG_PTR_DEVICE) return fail(ctx, RBSOG_E_INVAL, "bad ptr_kind");
  int rc;
  if ((rc = enter(ctx))) return rc;
  // the positions (through the staging buffer for host memory) and the step
  // counter, as rbsog_move_atoms; nothing waits here: for host buffers the
  // single synchronization at the end covers both copies
  const bool host = ptr_kind == RBSOG_PTR_HOST;
  if (host)
    CK(cudaMemcpyAsync(ctx->stage, pos, sizeof(double) * 3 * (size_t)ctx->n, cudaMemcpyHostToDevice, ctx->st));
  rb::launch_aos_to_soa_step(host ? ctx->stage : pos, ctx->v.x, ctx->n, ctx->v.step, (long long)step, ctx->st);
  if ((rc = check_launch(ctx))) return rc;
  ctx->forces_valid = false;
  ctx->host_step = step;
  // the force-only evaluation of rbsog_compute_forces
  View vv;
  if ((rc = eval_view(ctx, vv))) return rc;
  if ((rc = eval_forces_graph(ctx, vv))) return rc;
  ctx->forces_valid = true;
  ctx->lists_valid = true;
  if (ctx->v.prec == RBSOG_FP64) rc = export_aos(ctx, ctx->v.Fd, nullptr, forces, ptr_kind, false);
  else rc = export_aos(ctx, nullptr, ctx->v.Ff, forces, ptr_kind, false);
  if (rc) return rc;
  if (host && (rc = read_err(ctx))) return rc;   // synchronizes the stream
  return leave(ctx);
}

int rbsog_get_list_origin(rbsog_ctx *ctx, double *pos_b, int ptr_kind) {
  if (!ctx || !pos_b) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  if (!ctx->v.kept) return fail(ctx, RBSOG_E_INVAL, "no kept lists (list_every = 0)");
  if (!ctx->lists_valid) return fail(ctx, RBSOG_E_INVAL, "no kept lists yet: evaluate forces first");
  int rc;
  if ((rc = enter(ctx))) return rc;
  if ((rc = export_aos(ctx, ctx->v.xb, nullptr, pos_b, ptr_kind))) return rc;
  return leave(ctx);
}

int rbsog_set_list_origin(rbsog_ctx *ctx, const double *pos_b, int ptr_kind) {
  if (!ctx || !pos_b) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  if (!ctx->v.kept) return fail(ctx, RBSOG_E_INVAL, "no kept lists (list_every = 0)");
  int rc;
  if ((rc = enter(ctx))) return rc;
  if (!ctx->x_origin && ((rc = dalloc(ctx, &ctx->x_origin, 3 * (size_t)ctx->n)) ||
                         (rc = dalloc(ctx, &ctx->x_save, 3 * (size_t)ctx->n))))
    return rc;
  if ((rc = import_aos(ctx, pos_b, ctx->x_origin, ptr_kind))) return rc;
  if (ptr_kind == RBSOG_PTR_HOST) CK(cudaStreamSynchronize(ctx->st));   // the staging buffer is reused
  ctx->origin_pending = true;
  ctx->lists_valid = false;
  ctx->forces_valid = false;
  return leave(ctx);
}

int rbsog_sync(rbsog_ctx *ctx) {
  if (!ctx) return RBSOG_E_INVAL;
  CK(cudaSetDevice(ctx->dev));
  CK(cudaStreamSynchronize(ctx->st));
  if (!ctx->has_system) return RBSOG_OK;
  return read_err(ctx);
}

int rbsog_get_kinetic_tensor(rbsog_ctx *ctx, double *K, int ptr_kind) {
  if (!ctx || !K) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  if (ptr_kind != RBSOG_PTR_HOST && ptr_kind != RBSOG_PTR_DEVICE) return fail(ctx, RBSOG_E_INVAL, "bad ptr_kind");
  int rc;
  if ((rc = enter(ctx))) return rc;
  rb::launch_kinetic_tensor(ctx->v, ctx->st);
  if ((rc = check_launch(ctx))) return rc;
  if (ptr_kind == RBSOG_PTR_HOST) {
    CK(cudaMemcpyAsync(K, ctx->v.kin, 6 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
  } else {
    CK(cudaMemcpyAsync(K, ctx->v.kin, 6 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
  }
  return leave(ctx);
}

int rbsog_get_thermostat(rbsog_ctx *ctx, double *eta, double *v_eta) {
  if (!ctx) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  if (ctx->prm.integrator != RBSOG_NOSE_HOOVER) return fail(ctx, RBSOG_E_INVAL, "not a Nose-Hoover run");
  double h[rb::NH_STATE];
  CK(cudaSetDevice(ctx->dev));
  CK(cudaMemcpyAsync(h, ctx->v.nh, sizeof(h), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  for (int j = 0; j < ctx->v.nh_M; j++) {
    if (eta) eta[j] = h[rb::NH_A_ETA + j];
    if (v_eta) v_eta[j] = h[rb::NH_A_V + j];
  }
  return RBSOG_OK;
}

int rbsog_set_thermostat(rbsog_ctx *ctx, const double *eta, const double *v_eta) {
  if (!ctx) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  if (ctx->prm.integrator != RBSOG_NOSE_HOOVER) return fail(ctx, RBSOG_E_INVAL, "not a Nose-Hoover run");
  if (!eta || !v_eta) return fail(ctx, RBSOG_E_INVAL, "null argument");
  double h[rb::NH_STATE];
  CK(cudaSetDevice(ctx->dev));
  CK(cudaMemcpyAsync(h, ctx->v.nh, sizeof(h), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  for (int j = 0; j < ctx->v.nh_M; j++) {
    h[rb::NH_A_ETA + j] = eta[j];
    h[rb::NH_A_V + j] = v_eta[j];
  }
  CK(cudaMemcpyAsync(ctx->v.nh, h, sizeof(h), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  ctx->nh_primed = false;
  return RBSOG_OK;
}

int rbsog_get_list_builds(rbsog_ctx *ctx, int64_t *builds) {
  if (!ctx || !builds) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  unsigned long long b = 0;
  CK(cudaSetDevice(ctx->dev));
  CK(cudaMemcpyAsync(&b, ctx->v.nbuild, sizeof(b), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  *builds = (int64_t)b;
  return RBSOG_OK;
}

int rbsog_get_sog(rbsog_ctx *ctx, double *s, double *w, double *S) {
  if (!ctx) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  if (s) *s = ctx->sog.s;
  if (w) std::memcpy(w, ctx->sog.w.data(), sizeof(double) * ctx->sog.w.size());
  if (S) *S = ctx->samp.S;
  return RBSOG_OK;
}

int rbsog_debug_get_lists(rbsog_ctx *ctx, const int64_t *sel, int64_t nsel, int32_t cap_core,
                          int32_t cap_shell, int32_t *core, int32_t *ncore, int32_t *shell,
                          int32_t *nshell, int32_t *batch, int32_t *nbatch, double *weight) {
  if (!ctx) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  if (!sel || nsel <= 0 || cap_core < 1 || cap_shell < 1 || !core || !ncore || !shell || !nshell)
    return fail(ctx, RBSOG_E_INVAL, "bad list arguments");
  for (int64_t q = 0; q < nsel; q++)
    if (sel[q] < 0 || sel[q] >= ctx->n) return fail(ctx, RBSOG_E_INVAL, "selected atom out of range");
  if (ctx->v.kept) return fail(ctx, RBSOG_E_INVAL, "kept lists in use: see rbsog_debug_get_kept_lists");
  int rc;
  if ((rc = enter(ctx))) return rc;
  View &v = ctx->v;
  rb::launch_prepare(v, ctx->st, 0, 0);
  rb::launch_bin(v, ctx->st);
  // the near field is not run here: clear the binning's histograms ourselves
  CK(cudaMemsetAsync(v.cell_count, 0, sizeof(int) * ((size_t)v.ncell + (size_t)v.nc[1] * v.nc[2]), ctx->st));
  const size_t k = (size_t)nsel;
  long long *dsel;
  int *dcore, *dnc, *dshell, *dns, *dbatch = nullptr, *dnb = nullptr;
  double *dw = nullptr;
  CK(cudaMalloc(&dsel, sizeof(long long) * k));
  CK(cudaMalloc(&dcore, sizeof(int) * k * cap_core));
  CK(cudaMalloc(&dnc, sizeof(int) * k));
  CK(cudaMalloc(&dshell, sizeof(int) * k * cap_shell));
  CK(cudaMalloc(&dns, sizeof(int) * k));
  if (batch) {
    CK(cudaMalloc(&dbatch, sizeof(int) * k * v.P_R));
    CK(cudaMalloc(&dnb, sizeof(int) * k));
    CK(cudaMalloc(&dw, sizeof(double) * k));
  }
  CK(cudaMemsetAsync(dcore, 0xFF, sizeof(int) * k * cap_core, ctx->st));   // pad rows with -1
  CK(cudaMemsetAsync(dshell, 0xFF, sizeof(int) * k * cap_shell, ctx->st));
  if (batch) CK(cudaMemsetAsync(dbatch, 0xFF, sizeof(int) * k * v.P_R, ctx->st));
  std::vector<long long> hs(sel, sel + k);
  CK(cudaMemcpyAsync(dsel, hs.data(), sizeof(long long) * k, cudaMemcpyHostToDevice, ctx->st));
  rb::launch_lists(v, ctx->st, 0, dsel, (int)nsel, cap_core, cap_shell, dcore, dnc, dshell, dns, dbatch,
                   dnb, dw);
  if ((rc = check_launch(ctx))) return rc;
  CK(cudaMemcpyAsync(core, dcore, sizeof(int) * k * cap_core, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(ncore, dnc, sizeof(int) * k, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(shell, dshell, sizeof(int) * k * cap_shell, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(nshell, dns, sizeof(int) * k, cudaMemcpyDeviceToHost, ctx->st));
  if (batch) {
    CK(cudaMemcpyAsync(batch, dbatch, sizeof(int) * k * v.P_R, cudaMemcpyDeviceToHost, ctx->st));
    if (nbatch) CK(cudaMemcpyAsync(nbatch, dnb, sizeof(int) * k, cudaMemcpyDeviceToHost, ctx->st));
    if (weight) CK(cudaMemcpyAsync(weight, dw, sizeof(double) * k, cudaMemcpyDeviceToHost, ctx->st));
  }
  CK(cudaStreamSynchronize(ctx->st));
  cudaFree(dsel); cudaFree(dcore); cudaFree(dnc); cudaFree(dshell); cudaFree(dns);
  if (batch) { cudaFree(dbatch); cudaFree(dnb); cudaFree(dw); }
  return leave(ctx);
}

int rbsog_debug_get_kept_lists(rbsog_ctx *ctx, const int64_t *sel, int64_t nsel, int32_t cap_a,
                               int32_t cap_b, int32_t *A, int32_t *nA, int32_t *B, int32_t *nB,
                               int32_t *batch, int32_t *nbatch, double *weight) {
  if (!ctx) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  if (!ctx->v.kept) return fail(ctx, RBSOG_E_INVAL, "per-step lists in use (list_every = 0)");
  if (!ctx->lists_valid) return fail(ctx, RBSOG_E_INVAL, "no kept lists yet: evaluate forces first");
  if (!sel || nsel <= 0 || cap_a < 1 || cap_b < 1 || !A || !nA || !B || !nB ||
      (batch && (!nbatch || !weight)))
    return fail(ctx, RBSOG_E_INVAL, "bad list arguments");
  for (int64_t q = 0; q < nsel; q++)
    if (sel[q] < 0 || sel[q] >= ctx->n) return fail(ctx, RBSOG_E_INVAL, "selected atom out of range");
  int rc;
  if ((rc = enter(ctx))) return rc;
  const View &v = ctx->v;
  const size_t k = (size_t)nsel;
  long long *dsel;
  int *dA, *dnA, *dB, *dnB, *dbatch = nullptr, *dnb = nullptr;
  double *dw = nullptr;
  CK(cudaMalloc(&dsel, sizeof(long long) * k));
  CK(cudaMalloc(&dA, sizeof(int) * k * cap_a));
  CK(cudaMalloc(&dnA, sizeof(int) * k));
  CK(cudaMalloc(&dB, sizeof(int) * k * cap_b));
  CK(cudaMalloc(&dnB, sizeof(int) * k));
  if (batch) {
    CK(cudaMalloc(&dbatch, sizeof(int) * k * v.P_R));
    CK(cudaMalloc(&dnb, sizeof(int) * k));
    CK(cudaMalloc(&dw, sizeof(double) * k));
    CK(cudaMemsetAsync(dbatch, 0xFF, sizeof(int) * k * v.P_R, ctx->st));
  }
  CK(cudaMemsetAsync(dA, 0xFF, sizeof(int) * k * cap_a, ctx->st));   // pad rows with -1
  CK(cudaMemsetAsync(dB, 0xFF, sizeof(int) * k * cap_b, ctx->st));
  std::vector<long long> hs(sel, sel + k);
  CK(cudaMemcpyAsync(dsel, hs.data(), sizeof(long long) * k, cudaMemcpyHostToDevice, ctx->st));
  rb::launch_kept_lists(v, ctx->st, 0, dsel, (int)nsel, cap_a, cap_b, dA, dnA, dB, dnB, dbatch, dnb, dw);
  if ((rc = check_launch(ctx))) return rc;
  CK(cudaMemcpyAsync(A, dA, sizeof(int) * k * cap_a, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(nA, dnA, sizeof(int) * k, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(B, dB, sizeof(int) * k * cap_b, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(nB, dnB, sizeof(int) * k, cudaMemcpyDeviceToHost, ctx->st));
  if (batch) {
    CK(cudaMemcpyAsync(batch, dbatch, sizeof(int) * k * v.P_R, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(nbatch, dnb, sizeof(int) * k, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(weight, dw, sizeof(double) * k, cudaMemcpyDeviceToHost, ctx->st));
  }
  CK(cudaStreamSynchronize(ctx->st));
  cudaFree(dsel); cudaFree(dA); cudaFree(dnA); cudaFree(dB); cudaFree(dnB);
  if (batch) { cudaFree(dbatch); cudaFree(dnb); cudaFree(dw); }
  return leave(ctx);
}

int rbsog_debug_get_kept_batch_used(rbsog_ctx *ctx, const int64_t *sel, int64_t nsel, int32_t *batch) {
  if (!ctx) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  if (!ctx->v.kept) return fail(ctx, RBSOG_E_INVAL, "per-step lists in use (list_every = 0)");
  if (!ctx->lists_valid) return fail(ctx, RBSOG_E_INVAL, "no force evaluation with kept lists yet");
  if (!sel || nsel <= 0 || !batch) return fail(ctx, RBSOG_E_INVAL, "bad batch arguments");
  for (int64_t q = 0; q < nsel; q++)
    if (sel[q] < 0 || sel[q] >= ctx->n) return fail(ctx, RBSOG_E_INVAL, "selected atom out of range");
  int rc;
  if ((rc = enter(ctx))) return rc;
  const View &v = ctx->v;
  const size_t k = (size_t)nsel;
  long long *dsel;
  int *db;
  CK(cudaMalloc(&dsel, sizeof(long long) * k));
  CK(cudaMalloc(&db, sizeof(int) * k * v.P_R));
  CK(cudaMemsetAsync(db, 0xFF, sizeof(int) * k * v.P_R, ctx->st));
  std::vector<long long> hs(sel, sel + k);
  CK(cudaMemcpyAsync(dsel, hs.data(), sizeof(long long) * k, cudaMemcpyHostToDevice, ctx->st));
  rb::launch_kept_batch_used(v, ctx->st, dsel, (int)nsel, db);
  if ((rc = check_launch(ctx))) return rc;
  CK(cudaMemcpyAsync(batch, db, sizeof(int) * k * v.P_R, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  cudaFree(dsel); cudaFree(db);
  return leave(ctx);
}

int rbsog_debug_kept_b16(rbsog_ctx *ctx, int force_wide, int32_t *fits) {
  if (!ctx) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  if (!ctx->v.kept) return fail(ctx, RBSOG_E_INVAL, "per-step lists in use (list_every = 0)");
  int rc;
  if ((rc = enter(ctx))) return rc;
  if (ctx->v.kept_wide != (force_wide != 0)) {
    ctx->v.kept_wide = force_wide != 0;
    invalidate_graphs(ctx);                      // the step graph holds the view by value
  }
  if (fits) {
    int h = 1;
    CK(cudaMemcpyAsync(&h, ctx->v.b16_over, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    *fits = h == 0;
  }
  return leave(ctx);
}

int rbsog_debug_get_kbatch(rbsog_ctx *ctx, int32_t *m, double *c) {
  if (!ctx) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  int rc;
  if ((rc = enter(ctx))) return rc;
  const int P = ctx->v.P;
  if (m) {
    std::vector<int4> hm(P);
    CK(cudaMemcpyAsync(hm.data(), ctx->v.km, sizeof(int4) * P, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    for (int k = 0; k < P; k++) { m[3 * k] = hm[k].x; m[3 * k + 1] = hm[k].y; m[3 * k + 2] = hm[k].z; }
  }
  if (c) {
    CK(cudaMemcpyAsync(c, ctx->v.kc, sizeof(double) * P, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
  }
  return leave(ctx);
}

int rbsog_debug_set_kbatch(rbsog_ctx *ctx, int32_t P, const int32_t *m, const double *c) {
  if (!ctx) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  if (P < 0 || (P > 0 && (!m || !c))) return fail(ctx, RBSOG_E_INVAL, "bad k list");
  int rc;
  if ((rc = enter(ctx))) return rc;
  CK(cudaStreamSynchronize(ctx->st));
  View &v = ctx->v;
  if (P == 0) {
    v.fixed_k = 0;
    v.P = v.P_F;
  } else {
    set_rho_tiling(ctx, P);
    if (P > ctx->Pmax || true) {
      ctx->Pmax = 0;  // re-size per-k buffers for the new tiling
      if ((rc = ensure_kcap(ctx, std::max(P, v.P_F)))) return rc;
    }
    std::vector<int4> hm(P);
    for (int k = 0; k < P; k++) hm[k] = make_int4(m[3 * k], m[3 * k + 1], m[3 * k + 2], 0);
    CK(cudaMemcpyAsync(v.km, hm.data(), sizeof(int4) * P, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(v.kc, c, sizeof(double) * P, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    v.fixed_k = 1;
    v.P = P;
  }
  if (P == 0) {
    set_rho_tiling(ctx, v.P_F);
    ctx->Pmax = 0;
    if ((rc = ensure_kcap(ctx, v.P_F))) return rc;
  }
  invalidate_graphs(ctx);
  ctx->forces_valid = false;
  return leave(ctx);
}

int rbsog_debug_get_parts(rbsog_ctx *ctx, double *near, double *far, double *fcorr,
                          double *rho) {
  if (!ctx) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  int rc;
  if ((rc = enter(ctx))) return rc;
  const View &v = ctx->v;
  const bool d = v.prec == RBSOG_FP64;
  if (near && (rc = export_aos(ctx, d ? v.FNd : nullptr, d ? nullptr : v.FNf, near, RBSOG_PTR_HOST))) return rc;
  if (far && (rc = export_aos(ctx, d ? v.FFd : nullptr, d ? nullptr : v.FFf, far, RBSOG_PTR_HOST))) return rc;
  if (fcorr) {
    CK(cudaMemcpyAsync(fcorr, v.red, sizeof(double) * 3, cudaMemcpyDeviceToHost, ctx->st));
  }
  if (rho) {
    CK(cudaMemcpyAsync(rho, v.rho, sizeof(double) * 2 * v.P, cudaMemcpyDeviceToHost, ctx->st));
  }
  CK(cudaStreamSynchronize(ctx->st));
  return leave(ctx);
}

int rbsog_debug_set_whole_shell(rbsog_ctx *ctx, int flag) {
  if (!ctx) return RBSOG_E_INVAL;
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  ctx->v.whole_shell = flag ? 1 : 0;
  invalidate_graphs(ctx);
  ctx->forces_valid = false;
  return RBSOG_OK;
}

int rbsog_debug_sincos(rbsog_ctx *ctx, int64_t n, const uint32_t *th, float *s, float *c) {
  if (!ctx || n < 1 || !th || !s || !c) return fail(ctx, RBSOG_E_INVAL, "bad sincos arguments");
  CK(cudaSetDevice(ctx->dev));
  uint32_t *dt = nullptr;
  float *ds = nullptr, *dc = nullptr;
  CK(cudaMalloc(&dt, sizeof(uint32_t) * n));
  CK(cudaMalloc(&ds, sizeof(float) * n));
  CK(cudaMalloc(&dc, sizeof(float) * n));
  CK(cudaMemcpyAsync(dt, th, sizeof(uint32_t) * n, cudaMemcpyHostToDevice, ctx->st));
  rb::launch_sincos(n, dt, ds, dc, ctx->st);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(s, ds, sizeof(float) * n, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(c, dc, sizeof(float) * n, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  cudaFree(dt); cudaFree(ds); cudaFree(dc);
  return RBSOG_OK;
}

int rbsog_structure_factor_static(rbsog_ctx *ctx, int32_t P, const int32_t *m, double *rho) {
  if (!ctx) return RBSOG_E_INVAL;
  if (P < 0 || P > RBSOG_SF_STATIC_PMAX) return fail(ctx, RBSOG_E_INVAL, "P out of range (0 .. RBSOG_SF_STATIC_PMAX)");
  if (!ctx->has_system) return fail(ctx, RBSOG_E_NO_SYSTEM, "no system");
  if (P == 0) return RBSOG_OK;
  if (!m || !rho) return fail(ctx, RBSOG_E_INVAL, "null argument");
  CK(cudaSetDevice(ctx->dev));
  for (const void *q : {(const void *)m, (const void *)rho}) {
    cudaPointerAttributes at{};
    CK(cudaPointerGetAttributes(&at, q));
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
      return fail(ctx, RBSOG_E_INVAL, "m and rho must be device pointers");
    if (at.type == cudaMemoryTypeDevice && at.device != ctx->dev)
      return fail(ctx, RBSOG_E_INVAL, "m and rho must be memory of the context's device");
  }
  void *scratch = nullptr;
  CK(rb::sf_static_scratch(ctx->dev, &scratch));
  int rc;
  if ((rc = enter(ctx))) return rc;
  rb::launch_sf_static(ctx->v, P, m, rho, scratch, ctx->st);
  if ((rc = check_launch(ctx))) return rc;
  return leave(ctx);
}

int rbsog_set_schedule(rbsog_ctx *ctx, const rbsog_schedule *sched) {
  if (!ctx) return RBSOG_E_INVAL;
  if (!sched) return fail(ctx, RBSOG_E_INVAL, "null schedule");
  const rbsog_schedule q = *sched;
  const int A = q.far_atoms_per_thread, S = q.far_segments;
  if (q.rho_variant < 0 || q.rho_variant > 9 || q.far_packed < 0 || q.far_packed > 2 ||
      q.near_blocks_per_sm < 0 || q.near_blocks_per_sm > 16 ||
      (q.rho_tile_atoms != 0 && (q.rho_tile_atoms < 32 || q.rho_tile_atoms > 65536)) ||
      (q.near_wide != 0 && q.near_wide != 1) || q.rho_reduce < 0 || q.rho_reduce > 2 || q.rho_blocks_per_sm < 1 || q.rho_blocks_per_sm > 8 ||
      (A != 1 && A != 2 && A != 4) ||
      (S != 1 && S != 2 && S != 4 && S != 8))
    return fail(ctx, RBSOG_E_INVAL, "schedule out of range");
  ctx->sched = q;
  if (!ctx->has_system) return RBSOG_OK;
  int rc;
  if ((rc = enter(ctx))) return rc;
  CK(cudaStreamSynchronize(ctx->st));
  View &v = ctx->v;
  v.far_A = A;
  v.far_S = S;
  v.rho_var = q.rho_variant;
  v.far_packed = q.far_packed;
  v.near_bps = q.near_blocks_per_sm;
  v.near_wide = q.near_wide;
  v.rho_reduce = q.rho_reduce;
  ctx->rho_bps = q.rho_blocks_per_sm;
  set_rho_tiling(ctx, v.P);
  ctx->Pmax = 0;                               // tile partials for the new tiling
  if ((rc = ensure_kcap(ctx, std::max(v.P, v.P_F)))) return rc;
  invalidate_graphs(ctx);
  return leave(ctx);
}

int rbsog_get_schedule(rbsog_ctx *ctx, rbsog_schedule *sched) {
  if (!ctx || !sched) return RBSOG_E_INVAL;
  *sched = ctx->sched;
  return RBSOG_OK;
}

int rbsog_set_profiling(rbsog_ctx *ctx, int on) {
  if (!ctx) return RBSOG_E_INVAL;
  if (ctx->profiling != (on != 0)) {
    ctx->profiling = on != 0;
    invalidate_graphs(ctx);
  }
  return RBSOG_OK;
}

int rbsog_get_stage_times(rbsog_ctx *ctx, float *ms, int32_t nstage) {
  if (!ctx || !ms || nstage < 1) return RBSOG_E_INVAL;
  if (!ctx->profiling) return fail(ctx, RBSOG_E_INVAL, "profiling is off");
  CK(cudaSetDevice(ctx->dev));
  CK(cudaEventSynchronize(ctx->prof[8]));
  // (start, end) event of each stage: prepare, bin, near, far branch (k-batch, structure factor,
  // its reduction, far force; side stream), F^corr, finish (after the join), total, and inside
  // the far branch the structure-factor kernel and the far-force kernel alone
  static const int b[RBSOG_NSTAGE] = {0, 1, 2, 3, 7, 6, 0, 9, 11};
  static const int e[RBSOG_NSTAGE] = {1, 2, 7, 4, 5, 8, 8, 10, 4};
  for (int k = 0; k < nstage && k < RBSOG_NSTAGE; k++)
    CK(cudaEventElapsedTime(ms + k, ctx->prof[b[k]], ctx->prof[e[k]]));
  return RBSOG_OK;
}

int rbsog_get_stage_marks(rbsog_ctx *ctx, float *ms, int32_t nmark) {
  if (!ctx || !ms || nmark < 1) return RBSOG_E_INVAL;
  if (!ctx->profiling) return fail(ctx, RBSOG_E_INVAL, "profiling is off");
  CK(cudaSetDevice(ctx->dev));
  CK(cudaEventSynchronize(ctx->prof[8]));
  CK(cudaEventSynchronize(ctx->prof[4]));
  // the marks in the order of RBSOG_NMARK, as events of run_force
  static const int ev[RBSOG_NMARK] = {0, 1, 2, 7, 5, 6, 8, 3, 9, 10, 11, 4};
  for (int k = 0; k < nmark && k < RBSOG_NMARK; k++) CK(cudaEventElapsedTime(ms + k, ctx->prof[0], ctx->prof[ev[k]]));
  return RBSOG_OK;
}

}  // extern "C"
