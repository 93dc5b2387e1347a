// Ensemble of independent replicas (include/rbsog.h, "ensemble"): one full
// context per replica.  Packed mode (the default where the replicas allow
// it): a step of the ensemble is one CUDA graph of the step's stages, each a
// single kernel launch over the blocks of every replica (a prefix table per
// launch shape maps a block to its replica and its block there; the kernels
// are the single-system ones, on a shared-memory copy of the replica's view),
// in the two branches of a single system's step.  Otherwise: one CUDA graph
// with every replica's step graph as a child node (no edges between them),
// and replicas whose kept lists follow a fixed rebuild schedule launch their
// own graphs on their own streams.  Both are rebuilt when a replica captures
// its graph again.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "ctx_internal.h"
#include "rbsog.h"
#include "rbsog_internal.cuh"

struct rbsog_ensemble {
  int dev = 0;
  cudaStream_t user = nullptr;             // the ensemble's stream (may be the legacy stream)
  int32_t cap = 0;
  std::vector<rbsog_ctx *> rep;
  std::vector<cudaStream_t> st;            // one stream per replica
  std::vector<cudaEvent_t> done;           // end of a replica's latest work
  cudaEvent_t start = nullptr;
  cudaGraphExec_t gexec = nullptr;         // one step of every replica
  std::vector<uint64_t> gen;               // the replicas' graph generations gexec was built from
  std::string err;
  // packed mode
  int mode = RBSOG_ENSEMBLE_PACKED;        // requested
  int groups = 1;                          // packed: groups of replicas, each packed, run as parallel branches
  int used = -1;                           // what the last step ran
  cudaStream_t cs = nullptr;               // capture origin
  cudaEvent_t pf_origin = nullptr;
  struct Branch {                          // capture streams and events of one group
    cudaStream_t st = nullptr, st2 = nullptr, st2hi = nullptr;
    cudaEvent_t f0 = nullptr, f1 = nullptr, join = nullptr, done = nullptr;
  };
  std::vector<Branch> br;
  cudaGraphExec_t pexec = nullptr;
  std::vector<uint64_t> pgen;
  int pgroups = 0;                         // groups pexec was built with
  void *dbuf = nullptr;                    // the plans' device views and block tables
};

namespace {
int efail(rbsog_ensemble *e, int code, const std::string &msg) {
  if (e) e->err = msg;
  return code;
}
}  // namespace

extern "C" {

int rbsog_ensemble_create(rbsog_ensemble **out, int cuda_device, void *cuda_stream,
                          int32_t max_replicas) {
  if (!out || max_replicas < 1) return RBSOG_E_INVAL;
  *out = nullptr;
  rbsog_ensemble *e = new rbsog_ensemble();
  e->dev = cuda_device;
  e->user = (cudaStream_t)cuda_stream;
  e->cap = max_replicas;
  cudaError_t c = cudaSetDevice(cuda_device);
  if (c == cudaSuccess) c = cudaEventCreateWithFlags(&e->start, cudaEventDisableTiming);
  if (c == cudaSuccess) c = cudaStreamCreateWithFlags(&e->cs, cudaStreamNonBlocking);
  if (c == cudaSuccess) c = cudaEventCreateWithFlags(&e->pf_origin, cudaEventDisableTiming);
  if (c != cudaSuccess) {
    rbsog_ensemble_destroy(e);
    return RBSOG_E_CUDA;
  }
  *out = e;
  return RBSOG_OK;
}

void rbsog_ensemble_destroy(rbsog_ensemble *e) {
  if (!e) return;
  cudaSetDevice(e->dev);
  for (rbsog_ctx *c : e->rep) rbsog_destroy(c);
  for (cudaStream_t s : e->st) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  for (cudaEvent_t v : e->done) cudaEventDestroy(v);
  if (e->start) cudaEventDestroy(e->start);
  if (e->gexec) cudaGraphExecDestroy(e->gexec);
  if (e->pexec) cudaGraphExecDestroy(e->pexec);
  if (e->cs) cudaStreamDestroy(e->cs);
  if (e->pf_origin) cudaEventDestroy(e->pf_origin);
  for (auto &b : e->br) {
    for (cudaStream_t q : {b.st, b.st2, b.st2hi})
      if (q) cudaStreamDestroy(q);
    for (cudaEvent_t q : {b.f0, b.f1, b.join, b.done})
      if (q) cudaEventDestroy(q);
  }
  if (e->dbuf) cudaFree(e->dbuf);
  delete e;
}

int rbsog_ensemble_add(rbsog_ensemble *e, int64_t n, const double *pos, const int32_t *species,
                       int32_t n_species, const double *charge, const double *mass,
                       const double *bmh, const double box[3], const rbsog_params *params,
                       int ptr_kind, int32_t *replica) {
  if (!e) return RBSOG_E_INVAL;
  if ((int32_t)e->rep.size() >= e->cap) return efail(e, RBSOG_E_INVAL, "ensemble is full");
  if (cudaSetDevice(e->dev) != cudaSuccess) return efail(e, RBSOG_E_CUDA, "cudaSetDevice");
  cudaStream_t s = nullptr;
  cudaEvent_t v = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
    return efail(e, RBSOG_E_CUDA, "stream creation");
  if (cudaEventCreateWithFlags(&v, cudaEventDisableTiming) != cudaSuccess) {
    cudaStreamDestroy(s);
    return efail(e, RBSOG_E_CUDA, "event creation");
  }
  rbsog_ctx *c = nullptr;
  int rc = rbsog_create(&c, e->dev, (void *)s);
  if (rc == RBSOG_OK) {
    // the replica's set-up is ordered after the ensemble's stream
    cudaEventRecord(e->start, e->user);
    cudaStreamWaitEvent(s, e->start, 0);
    rc = rbsog_set_system(c, n, pos, species, n_species, charge, mass, bmh, box, params, ptr_kind);
    if (rc != RBSOG_OK) e->err = std::string("replica set-up: ") + rbsog_last_error(c);
  }
  if (rc != RBSOG_OK) {
    if (c) rbsog_destroy(c);
    cudaStreamDestroy(s);
    cudaEventDestroy(v);
    return rc;
  }
  e->rep.push_back(c);
  e->st.push_back(s);
  e->done.push_back(v);
  if (replica) *replica = (int32_t)e->rep.size() - 1;
  return RBSOG_OK;
}

rbsog_ctx *rbsog_ensemble_replica(rbsog_ensemble *e, int32_t r) {
  if (!e || r < 0 || r >= (int32_t)e->rep.size()) return nullptr;
  return e->rep[r];
}

namespace {
// The ensemble graph for the replicas' current step graphs (rebuilt when any
// of them was captured again).
int ensure_graph(rbsog_ensemble *e) {
  const size_t R = e->rep.size();
  bool stale = e->gexec == nullptr || e->gen.size() != R;
  std::vector<cudaGraph_t> child(R);
  std::vector<uint64_t> gen(R);
  for (size_t r = 0; r < R; r++) {
    child[r] = rb::ctx_step_graph(e->rep[r], &gen[r]);
    if (!child[r]) return efail(e, RBSOG_E_INVAL, "replica without a step graph");
    if (!stale && gen[r] != e->gen[r]) stale = true;
  }
  if (!stale) return RBSOG_OK;
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return efail(e, RBSOG_E_CUDA, "graph creation");
  for (size_t r = 0; r < R; r++) {
    cudaGraphNode_t node;
    if (cudaGraphAddChildGraphNode(&node, g, nullptr, 0, child[r]) != cudaSuccess) {
      cudaGraphDestroy(g);
      return efail(e, RBSOG_E_CUDA, "child graph node");
    }
  }
  if (e->gexec) cudaGraphExecDestroy(e->gexec);
  e->gexec = nullptr;
  const cudaError_t c = cudaGraphInstantiate(&e->gexec, g, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(g);
  if (c != cudaSuccess) return efail(e, RBSOG_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(c));
  e->gen = gen;
  return RBSOG_OK;
}
}  // namespace

namespace {
// Whether every replica can run in one packed graph: mixed precision, one
// integrator (velocity Verlet or BAOAB), per-step lists or automatically
// rebuilt kept lists for all, one far-field schedule, no profiling.
bool packable(rbsog_ensemble *e, std::vector<rb::View> &views, int *mode, bool *kept) {
  const size_t R = e->rep.size();
  views.resize(R);
  for (size_t r = 0; r < R; r++) {
    int m = 0;
    bool prof = false;
    rb::ctx_step_view(e->rep[r], &views[r], &m, &prof);
    const rb::View &v = views[r];
    if (prof || m == 0 || v.prec != RBSOG_MIXED || (v.kept && !v.auto_lists)) return false;
    if (r == 0) {
      *mode = m;
      *kept = v.kept != 0;
      continue;
    }
    const rb::View &v0 = views[0];
    if (m != *mode || (v.kept != 0) != *kept || v.rho_var != v0.rho_var || v.far_A != v0.far_A ||
        v.far_S != v0.far_S || v.far_packed != v0.far_packed || v.near_wide != v0.near_wide)
      return false;
  }
  return R > 0;
}

// Streams and events of `n` capture branches.
int ensure_branches(rbsog_ensemble *e, size_t n) {
  int prio_least = 0, prio_greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess)
    return efail(e, RBSOG_E_CUDA, "stream priorities");
  while (e->br.size() < n) {
    rbsog_ensemble::Branch b;
    cudaError_t c = cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking);
    if (c == cudaSuccess) c = cudaStreamCreateWithFlags(&b.st2, cudaStreamNonBlocking);
    if (c == cudaSuccess) c = cudaStreamCreateWithPriority(&b.st2hi, cudaStreamNonBlocking, prio_greatest);
    for (cudaEvent_t *q : {&b.f0, &b.f1, &b.join, &b.done})
      if (c == cudaSuccess) c = cudaEventCreateWithFlags(q, cudaEventDisableTiming);
    e->br.push_back(b);
    if (c != cudaSuccess) return efail(e, RBSOG_E_CUDA, "branch streams");
  }
  return RBSOG_OK;
}

// The packed step graph for the replicas' current views (rebuilt when any
// replica was captured again or the grouping changed): the replicas dealt
// into `groups` groups of about equal atoms (largest first, each to the
// lightest group), each group's stages one packed launch each, the groups as
// parallel branches.  Returns RBSOG_OK, or RBSOG_E_INVAL when the replicas
// cannot be packed.
int ensure_packed(rbsog_ensemble *e) {
  const size_t R = e->rep.size();
  std::vector<uint64_t> gen(R);
  for (size_t r = 0; r < R; r++)
    if (!rb::ctx_step_graph(e->rep[r], &gen[r])) return efail(e, RBSOG_E_INVAL, "replica without a step graph");
  const size_t G = std::max<size_t>(1, std::min<size_t>((size_t)e->groups, R));
  if (e->pexec && gen == e->pgen && (int)G == e->pgroups) return RBSOG_OK;
  std::vector<rb::View> views;
  int mode = 0;
  bool kept = false;
  if (!packable(e, views, &mode, &kept)) return RBSOG_E_INVAL;
  // groups of about equal atoms
  std::vector<size_t> order(R);
  for (size_t r = 0; r < R; r++) order[r] = r;
  std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return views[a].n > views[b].n; });
  std::vector<std::vector<size_t>> grp(G);
  std::vector<int64_t> load(G, 0);
  for (size_t r : order) {
    const size_t g = (size_t)(std::min_element(load.begin(), load.end()) - load.begin());
    grp[g].push_back(r);
    load[g] += views[r].n;
  }
  for (auto &g : grp) std::sort(g.begin(), g.end());
  // device copies: each group's views, then its block tables
  size_t bytes = 0;
  std::vector<size_t> voff(G), toff(G);
  for (size_t g = 0; g < G; g++) {
    voff[g] = bytes;
    bytes += sizeof(rb::View) * grp[g].size();
    toff[g] = bytes;
    bytes += sizeof(int) * (grp[g].size() + 1) * rb::PK_KINDS;
    bytes = (bytes + 255) & ~(size_t)255;
  }
  std::vector<char> host(bytes);
  std::vector<rb::PackPlan> plans(G);
  for (size_t g = 0; g < G; g++) {
    const size_t Rg = grp[g].size();
    rb::View *hv = reinterpret_cast<rb::View *>(host.data() + voff[g]);
    int *tab = reinterpret_cast<int *>(host.data() + toff[g]);
    for (size_t j = 0; j < Rg; j++) hv[j] = views[grp[g][j]];
    rb::PackPlan &q = plans[g];
    for (int k = 0; k < rb::PK_KINDS; k++) {
      int *t = tab + (Rg + 1) * k;
      t[0] = 0;
      for (size_t j = 0; j < Rg; j++) t[j + 1] = t[j] + rb::pack_blocks(hv[j], k);
      q.total[k] = t[Rg];
    }
    q.R = (int)Rg;
    q.rho_var = views[0].rho_var;
    q.far_A = views[0].far_A;
    q.far_packed = views[0].far_packed;
    q.near_wide = views[0].near_wide;
  }
  if (e->dbuf) cudaFree(e->dbuf);
  e->dbuf = nullptr;
  if (cudaMalloc(&e->dbuf, bytes) != cudaSuccess) return efail(e, RBSOG_E_CUDA, "packed plan allocation");
  if (cudaMemcpy(e->dbuf, host.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess)
    return efail(e, RBSOG_E_CUDA, "packed plan upload");
  for (size_t g = 0; g < G; g++) {
    plans[g].views = reinterpret_cast<const rb::View *>((char *)e->dbuf + voff[g]);
    for (int k = 0; k < rb::PK_KINDS; k++)
      plans[g].b0[k] = reinterpret_cast<const int *>((char *)e->dbuf + toff[g]) + (grp[g].size() + 1) * k;
  }
  int rc = ensure_branches(e, G);
  if (rc != RBSOG_OK) return rc;
  // one step of every replica: per group the stages of a single system's step
  // (two branches: far field on the side stream, at the greatest priority
  // with kept lists, where it is the longer branch), the groups in parallel
  cudaGraph_t gr = nullptr;
  if (cudaStreamBeginCapture(e->cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return efail(e, RBSOG_E_CUDA, "packed capture");
  cudaEventRecord(e->pf_origin, e->cs);
  for (size_t g = 0; g < G; g++) {
    const rb::PackPlan &q = plans[g];
    const rbsog_ensemble::Branch &b = e->br[g];
    cudaStream_t st = b.st, st2 = kept ? b.st2hi : b.st2;
    cudaStreamWaitEvent(st, e->pf_origin, 0);
    cudaEventRecord(b.f0, st);
    cudaStreamWaitEvent(st2, b.f0, 0);
    rb::pack_ksample(q, st2, 1);
    rb::pack_prepare(q, st, mode, 1);
    cudaEventRecord(b.f1, st);
    cudaStreamWaitEvent(st2, b.f1, 0);
    rb::pack_rho(q, st2);
    rb::pack_rhosum(q, st2);
    rb::pack_farforce(q, st2);
    cudaEventRecord(b.join, st2);
    rb::pack_bin(q, st);
    if (kept) {
      rb::pack_build_lists(q, st);
      rb::pack_sample_batch(q, st, 1);
      rb::pack_near_kept(q, st, 1);
    } else {
      rb::pack_near(q, st, 1);
    }
    cudaStreamWaitEvent(st, b.join, 0);
    rb::pack_finish(q, st);
    cudaEventRecord(b.done, st);
    cudaStreamWaitEvent(e->cs, b.done, 0);
  }
  const cudaError_t le = cudaGetLastError();
  cudaError_t c = cudaStreamEndCapture(e->cs, &gr);
  if (le != cudaSuccess || c != cudaSuccess) {
    if (gr) cudaGraphDestroy(gr);
    return efail(e, RBSOG_E_CUDA, std::string("packed capture: ") + cudaGetErrorString(le != cudaSuccess ? le : c));
  }
  if (e->pexec) cudaGraphExecDestroy(e->pexec);
  e->pexec = nullptr;
  c = cudaGraphInstantiate(&e->pexec, gr, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(gr);
  if (c != cudaSuccess) return efail(e, RBSOG_E_CUDA, std::string("packed instantiate: ") + cudaGetErrorString(c));
  e->pgen = gen;
  e->pgroups = (int)G;
  return RBSOG_OK;
}
}  // namespace

int rbsog_ensemble_set_mode(rbsog_ensemble *e, int32_t mode) {
  if (!e || (mode != RBSOG_ENSEMBLE_PACKED && mode != RBSOG_ENSEMBLE_GRAPHS)) return RBSOG_E_INVAL;
  e->mode = mode;
  return RBSOG_OK;
}

int rbsog_ensemble_set_groups(rbsog_ensemble *e, int32_t groups) {
  if (!e || groups < 1) return RBSOG_E_INVAL;
  e->groups = groups;
  return RBSOG_OK;
}

int rbsog_ensemble_get_mode(rbsog_ensemble *e, int32_t *used) {
  if (!e || !used) return RBSOG_E_INVAL;
  *used = e->used;
  return RBSOG_OK;
}

int rbsog_ensemble_step(rbsog_ensemble *e, int64_t nsteps) {
  if (!e) return RBSOG_E_INVAL;
  if (nsteps < 0) return efail(e, RBSOG_E_INVAL, "negative step count");
  if (cudaSetDevice(e->dev) != cudaSuccess) return efail(e, RBSOG_E_CUDA, "cudaSetDevice");
  const size_t R = e->rep.size();
  if (R == 0 || nsteps == 0) return RBSOG_OK;
  if (cudaEventRecord(e->start, e->user) != cudaSuccess) return efail(e, RBSOG_E_CUDA, "fork event");
  for (size_t r = 0; r < R; r++)
    if (cudaStreamWaitEvent(e->st[r], e->start, 0) != cudaSuccess) return efail(e, RBSOG_E_CUDA, "fork wait");
  bool single = true;
  for (size_t r = 0; r < R; r++) single = single && rb::ctx_single_graph(e->rep[r]);
  if (single) {
    // each replica's pending work (stale forces, graph capture, chain priming)
    // on its own stream, then every step as one graph on the ensemble's stream
    for (size_t r = 0; r < R; r++) {
      const int rc = rb::ctx_prepare_step(e->rep[r]);
      if (rc != RBSOG_OK)
        return efail(e, rc, "replica " + std::to_string(r) + ": " + rbsog_last_error(e->rep[r]));
    }
    cudaGraphExec_t gx = nullptr;
    if (e->mode == RBSOG_ENSEMBLE_PACKED) {
      const int prc = ensure_packed(e);
      if (prc == RBSOG_OK) gx = e->pexec;
      else if (prc != RBSOG_E_INVAL) return prc;     // a CUDA failure, not a mix the packing cannot take
    }
    if (!gx) {
      const int rc = ensure_graph(e);
      if (rc != RBSOG_OK) return rc;
      gx = e->gexec;
    }
    e->used = gx == e->pexec ? RBSOG_ENSEMBLE_PACKED : RBSOG_ENSEMBLE_GRAPHS;
    for (size_t r = 0; r < R; r++)
      if (cudaEventRecord(e->done[r], e->st[r]) != cudaSuccess || cudaStreamWaitEvent(e->user, e->done[r], 0) != cudaSuccess)
        return efail(e, RBSOG_E_CUDA, "join");
    for (int64_t k = 0; k < nsteps; k++)
      if (cudaGraphLaunch(gx, e->user) != cudaSuccess) return efail(e, RBSOG_E_CUDA, "graph launch");
    for (size_t r = 0; r < R; r++) rb::ctx_advance(e->rep[r], nsteps);
    // later calls on a replica's own stream come after the ensemble's steps
    if (cudaEventRecord(e->start, e->user) != cudaSuccess) return efail(e, RBSOG_E_CUDA, "fork event");
    for (size_t r = 0; r < R; r++)
      if (cudaStreamWaitEvent(e->st[r], e->start, 0) != cudaSuccess) return efail(e, RBSOG_E_CUDA, "fork wait");
    return RBSOG_OK;
  }
  // one step of every replica per round, so all streams have work queued early
  e->used = RBSOG_ENSEMBLE_GRAPHS;
  for (int64_t k = 0; k < nsteps; k++)
    for (size_t r = 0; r < R; r++) {
      const int rc = rbsog_step(e->rep[r], 1);
      if (rc != RBSOG_OK)
        return efail(e, rc, "replica " + std::to_string(r) + ": " + rbsog_last_error(e->rep[r]));
    }
  for (size_t r = 0; r < R; r++) {
    if (cudaEventRecord(e->done[r], e->st[r]) != cudaSuccess ||
        cudaStreamWaitEvent(e->user, e->done[r], 0) != cudaSuccess)
      return efail(e, RBSOG_E_CUDA, "join");
  }
  return RBSOG_OK;
}

int rbsog_ensemble_sync(rbsog_ensemble *e) {
  if (!e) return RBSOG_E_INVAL;
  for (size_t r = 0; r < e->rep.size(); r++) {
    const int rc = rbsog_sync(e->rep[r]);
    if (rc != RBSOG_OK) return efail(e, rc, "replica " + std::to_string(r) + ": " + rbsog_last_error(e->rep[r]));
  }
  return RBSOG_OK;
}

const char *rbsog_ensemble_last_error(const rbsog_ensemble *e) {
  if (!e) return "null ensemble";
  return e->err.c_str();
}

}  // extern "C"
