// The opaque seedcg_handle: one gauge field, its internal link copies, and the
// workspaces of the last solve (kept between solves so that repeated solves
// on the same field do not pay for allocation again).
#pragma once

#include <string>
#include <vector>

#include "internal.cuh"

struct seedcg_handle {
    seedcg::Geom g;
    double kappa = 0.0;
    seedcg_options opt;
    int device = 0;
    seedcg::DevBuf u64, u32;      // links [4][9][V] double2 / float2
    // workspaces
    seedcg::DevBuf vbasis;        // stored Krylov basis V, m_cap rows
    int vbasis_prec = -1;         // precision mode V was written in
    int vbasis_m = 0;             // rows of V valid after the last solve
    seedcg::DevBuf lz_scalars;    // LzCtl + alpha/beta/... arrays
    seedcg::DevBuf red;           // reduction partials + counters
    seedcg::DevBuf work;          // working vectors of the solve
    seedcg::DevBuf coef;          // projection coefficients / gemm split scratch
    seedcg::DevBuf staging;       // complex128 staging of host B / X
    seedcg::DevBuf tcbuf;         // tensor-core projection: bf16 B operand + FP32 partials
    seedcg::DevBuf cgbuf;         // batched CG engine workspace
    std::vector<double> alpha, beta, delta;  // Lanczos scalars of the last solve
    int last_m = 0;
    int last_m_conv = 0, last_po_count = 0, last_lz_status = 0;
    float last_ms_lanczos = 0.f, last_ms_po = 0.f, last_ms_seed = 0.f;
    std::string err;
    void* pinned = nullptr;       // small pinned host buffer for flag polls
};

namespace seedcg {
seedcg_status batch_solve_impl(seedcg_handle** hs, int nf, const int* nrhs, const double* const* B,
                               double* const* X, double tol, int extra_iters, int reorth_period,
                               seedcg_info* infos, cudaStream_t st);
seedcg_status project_basis_impl(seedcg_handle* h, int rows, int nvec, const double* X,
                                 double* C, int use_tc, cudaStream_t st);
seedcg_status solve_impl(seedcg_handle* h, int nrhs, const double* B, double* X, double tol,
                         int extra_iters, int reorth_period, seedcg_info* info, cudaStream_t st);
}
