// Ensemble of independent replicas (include/rbsog.h, "ensemble"): one full
// context per replica.  A step of the ensemble is one CUDA graph with every
// replica's step graph as a child node (no edges between them, so the
// replicas' kernels share the device as it frees up), launched once on the
// ensemble's stream; it is rebuilt when a replica captures its graph again.
// Replicas whose kept lists follow a fixed rebuild schedule need the host's
// choice of graph at every step: then each replica launches its own graphs on
// its own stream.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "ctx_internal.h"
#include "rbsog.h"

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
    int rc = ensure_graph(e);
    if (rc != RBSOG_OK) return rc;
    for (size_t r = 0; r < R; r++)
      if (cudaEventRecord(e->done[r], e->st[r]) != cudaSuccess || cudaStreamWaitEvent(e->user, e->done[r], 0) != cudaSuccess)
        return efail(e, RBSOG_E_CUDA, "join");
    for (int64_t k = 0; k < nsteps; k++)
      if (cudaGraphLaunch(e->gexec, e->user) != cudaSuccess) return efail(e, RBSOG_E_CUDA, "graph launch");
    for (size_t r = 0; r < R; r++) rb::ctx_advance(e->rep[r], nsteps);
    // later calls on a replica's own stream come after the ensemble's steps
    if (cudaEventRecord(e->start, e->user) != cudaSuccess) return efail(e, RBSOG_E_CUDA, "fork event");
    for (size_t r = 0; r < R; r++)
      if (cudaStreamWaitEvent(e->st[r], e->start, 0) != cudaSuccess) return efail(e, RBSOG_E_CUDA, "fork wait");
    return RBSOG_OK;
  }
  // one step of every replica per round, so all streams have work queued early
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
