// Batched CG for many independent seeded systems on one or several gauge
// fields (phase B of the solver; the seedcg_batch_solve entry point).
#pragma once

#include <vector>

#include "handle.cuh"

namespace seedcg {

// the systems of one gauge field: b^j and x^j in the internal FP64 layout,
// [nsys][12 V] each; x holds the start guess on entry and the solution on exit
struct CgGroup {
    seedcg_handle* h;
    int nsys;
    const double2* b64;
    double2* x64;
};

struct CgResult {
    // per group, per system
    std::vector<std::vector<int>> iters, ru, notconv;
    std::vector<std::vector<double>> true_resid;
    int reliable_updates = 0;
    int graph_chunks = 0;
    int rpb = 0;          // the operator's launch shape chosen by the autotuner (warps per
                          // 32-site tile, or TB * 1000 + groups for the brick kernel)
};

// Run CG on every system of every group until ||b - M x|| <= tol ||b|| in FP64.
// R is the working precision of the iteration; reliable_delta (mixed) triggers
// an FP64 residual recomputation when the iterated residual fell by that factor
// (0 = only at convergence).  `ws` holds the engine's device workspace.
template <typename R>
void batched_cg(std::vector<CgGroup>& groups, double tol, double reliable_delta, int maxiter,
                int poll, bool use_graph, DevBuf& ws, void* pinned, CgResult& out,
                cudaStream_t st);

}  // namespace seedcg
