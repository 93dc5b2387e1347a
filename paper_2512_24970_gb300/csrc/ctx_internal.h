// Internal interface of a context (api.cu) used by the replica ensemble
// (ensemble.cu): the same preparation rbsog_step makes before it launches its
// step graph, and the captured graph itself, so that an ensemble can launch
// all its replicas' steps as one graph.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rbsog.h"

namespace rb {

// Evaluate the forces if they are stale, (re)capture the step graph, prime
// the Nose-Hoover chain; work on the context's stream.  Returns an RBSOG code.
int ctx_prepare_step(rbsog_ctx *ctx);
// True when one graph serves every step (no fixed rebuild schedule of kept lists).
bool ctx_single_graph(const rbsog_ctx *ctx);
// The captured (not instantiated) step graph, owned by the context, and its
// generation, which changes whenever the graph is captured again.
cudaGraph_t ctx_step_graph(const rbsog_ctx *ctx, uint64_t *gen);
// The host's copy of the step counter after nsteps launches of the graph.
void ctx_advance(rbsog_ctx *ctx, int64_t nsteps);

struct View;
// The view a step of the context evaluates with (the device view with the
// step's settings: no energy or virial partials; with kept lists, the build
// variant's flags), its integrator mode (1 velocity Verlet, 2 BAOAB, 0 other)
// and whether the context is profiling.
void ctx_step_view(const rbsog_ctx *ctx, View *out, int *mode, bool *profiling);

}  // namespace rb
