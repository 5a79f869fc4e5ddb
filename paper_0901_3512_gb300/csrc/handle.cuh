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
    seedcg::DevBuf hostio;        // device copies of host B / X passed to seedcg_solve
    std::vector<double> alpha, beta, delta;  // Lanczos scalars of the last solve
    int last_m = 0;
    int last_m_conv = 0, last_po_count = 0, last_lz_status = 0;
    float last_ms_lanczos = 0.f, last_ms_po = 0.f, last_ms_seed = 0.f;
    std::string err;
    void* pinned = nullptr;       // small pinned host buffer for flag polls
    void* guess = nullptr;        // learned initial guess: weights, Adam state, buffers
    bool force_x0 = false;        // this solve starts from X (set when the guess supplied x_0)
    bool eo_active = false;       // the running solve is on the even-odd system (half vectors)
    bool vbasis_eo = false;       // the stored basis holds half vectors of the even-odd system
};

namespace seedcg {
// learned initial guess (guess.cu); B, X internal FP64 [n][12 V]
void guess_set_weights(seedcg_handle* h, const double* w, cudaStream_t st);
void guess_get_weights(seedcg_handle* h, double* w, cudaStream_t st);
double guess_loss_grad(seedcg_handle* h, int npairs, const double2* B, const double2* X,
                       double* grad_out, cudaStream_t st);
double guess_train(seedcg_handle* h, int npairs, const double2* B, const double2* X, int epochs,
                   int batch, double lr, cudaStream_t st);
void guess_predict(seedcg_handle* h, int n_fields, const double2* B, double2* X0, cudaStream_t st);
void guess_free(seedcg_handle* h);
bool guess_ready(const seedcg_handle* h);

seedcg_status batch_solve_impl(seedcg_handle** hs, int nf, const int* nrhs, const double* const* B,
                               double* const* X, double tol, int extra_iters, int reorth_period,
                               seedcg_info* infos, cudaStream_t st);
void tridiag_lowest(int m, const double* a, const double* b, int nev, double* theta, double* S);
seedcg_status deflate_impl(seedcg_handle* h, int nev, int nr, const double* B, double* X0, double* theta_out,
                           cudaStream_t st);
seedcg_status project_basis_impl(seedcg_handle* h, int rows, int nvec, const double* X,
                                 double* C, int use_tc, cudaStream_t st);
seedcg_status solve_impl(seedcg_handle* h, int nrhs, const double* B, double* X, double tol,
                         int extra_iters, int reorth_period, seedcg_info* info, cudaStream_t st);
seedcg_status solve_eo_impl(seedcg_handle* h, int nrhs, const double* E, double* X, double tol,
                            int extra_iters, int reorth_period, seedcg_info* info, cudaStream_t st);
}
