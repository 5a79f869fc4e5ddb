// Declarations of the solver's kernel launchers (implemented in blas.cu and
// lanczos.cu) and of the device-side control block of one solve.
#pragma once

#include "internal.cuh"

namespace seedcg {

// Device control block of the first-RHS Lanczos run (Algorithm 1).  The
// scalars of T live on the device for the whole run; the host only polls
// `m` (the current target dimension) every few iterations.
struct LzCtl {
    int m;            // target m: m_max until convergence, then the past-convergence m
    int m_conv;       // first i with beta_i |zeta_i / delta_i| <= tol ||b^1||
    int status;       // SEEDCG_OK / SEEDCG_ERR_BREAKDOWN / SEEDCG_ERR_NAN
    int breakdown;    // 1: beta_i ~ 0 ended the run (invariant subspace)
    int po_count;
    int m_max;
    int extra_iters;
    int guard;        // 1: the step-8 guard may end the run (seedcg_options.po_guard)
    double beta0;     // ||r_0^1||
    double bnorm1;    // ||b^1||
    double tol;
    double past_factor;
    double nv;        // scratch: norm of v_i during re-orthogonalisation
    double2 dvf;      // scratch: v_i^dag f during re-orthogonalisation
};

struct LzDev {
    LzCtl* ctl;
    double* alpha;    // [m_max]  alpha_i at [i-1]
    double* beta;     // [m_max]  beta_i  at [i-1]
    double* delta;    // [m_max]
    double* gamma;    // [m_max]  gamma_i at [i-1]
    double* zeta;     // [m_max]
    double2* eta;     // [nrhs]   eta^j (literal seeding), j >= 2 at [j-2]
    double* partials; // reduction scratch
    unsigned* counters;
};

// counters[] slots used by the Lanczos kernels
enum { CTR_B = 0, CTR_D, CTR_PO1, CTR_PO2, CTR_PO3, CTR_PO4, CTR_NORM, CTR_ETA0, CTR_COUNT = 64 };

// ----- generic reductions (blas.cu) -----
// res[0] = sum conj(a) b over n complex entries (a, b flat internal vectors)
template <typename R>
void dot(const cx_t<R>* a, const cx_t<R>* b, long n, double* partials, unsigned* ctr,
         double2* res, cudaStream_t s);

// C[a][b] = sum_e conj(A[a][e]) B[b][e] for a < na, b < nb (A rows of type AT,
// B rows of cx_t<R>); C is double2 [na][ldc].  scratch holds the split partials.
template <typename R, typename AT>
void gemm_t(const AT* A, long lda, int na, const cx_t<R>* B, long ldb, int nb, long n,
            double2* C, int ldc, double2* scratch, size_t scratch_elems, cudaStream_t s);

// Same product, streaming form for few vectors (the re-orthogonalisation):
// V read once, X staged per block in shared memory, FP64 partials per block.
template <typename R, typename AT>
void proj(const AT* A, long lda, int na, const cx_t<R>* X, long ldx, int nx, long n, double2* C,
          int ldc, double2* scratch, size_t scratch_elems, cudaStream_t s);
template <typename R, typename AT>
size_t proj_scratch_elems(long n, int na);

// Y[b][e] += sign * sum_a A[a][e] C[a][b]  (accumulated in R, added in Y's type)
template <typename R, typename AT, typename YT>
void gemm_n(const AT* A, long lda, int na, const double2* C, int ldc, int nb, YT* Y, long ldy,
            long n, double sign, cudaStream_t s);

// y = b - y (FP64, flat)
void axpby_f64(const double2* b, double2* y, long n, cudaStream_t s);
// *out = ||x|| (FP64, deterministic; partials holds >= 1216 doubles, ctr one zero counter)
void k_norm2_public(const double2* x, long n, double* partials, unsigned* ctr, double* out,
                    cudaStream_t s);

// convert / copy flat vectors between storage types
template <typename ST, typename DT>
void convert(const ST* src, DT* dst, long n, cudaStream_t s);

}  // namespace seedcg
