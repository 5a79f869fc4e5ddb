// Even-odd (red-black) preconditioning of the Wilson operator, the setup the
// paper solves (Section 3).  With the sites split by parity (x + y + z + t even
// or odd), D = [[1, -kappa H_eo], [-kappa H_oe, 1]], and eliminating the even
// sites leaves the odd-site Schur complement
//
//     A = 1 - kappa^2 H_oe H_eo,   A x_o = phi = eta_o + kappa H_oe eta_e,
//
// after which x_e = eta_e + kappa H_eo x_o.  A^dag = gamma5 A gamma5 uses the
// hops of D^dag.  A half-lattice vector holds the sites of one parity in
// lexicographic order; with every extent even, half index h and full site s
// satisfy h = s >> 1, because each pair of sites (2h, 2h + 1) holds one site of
// each parity.  Half vectors use the same internal spinor layout as full ones,
// with V/2 sites.
#include <cmath>
#include <complex>
#include <vector>

#include "handle.cuh"
#include "internal.cuh"
#include "eo.cuh"
#include "kernels.cuh"
#include "wilson.cuh"

namespace seedcg {
namespace {

// out[h] = c_diag same[h] + c_hop (H other)(x), x the parity-p_out site of h;
// H is the hopping term of D = 1 - kappa H (DAG: of D^dag), with the
// antiperiodic sign on hops that wrap t.  `other` holds the opposite parity.
template <typename R, int DAG>
__global__ void __launch_bounds__(128)
k_eo_hop(Geom g, const cx_t<R>* __restrict__ u, int p_out, const cx_t<R>* __restrict__ other,
         const cx_t<R>* __restrict__ same, R c_diag, R c_hop, cx_t<R>* __restrict__ out) {
    const int vh = g.vol / 2;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= vh) return;
    Spinor<R> acc;
    eo_site_apply<R, DAG>(g, u, p_out, h, other, same, c_diag, c_hop, acc);
    store_spinor(out, vh, h, acc);
}

// half[h] = full at the parity-p site of h (scatter = 0) or the reverse (scatter = 1)
template <typename T>
__global__ void k_eo_move(Geom g, int p, int scatter, T* __restrict__ full, T* __restrict__ half) {
    const int vh = g.vol / 2;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= vh) return;
    const int s = eo_site(g, h, p);
#pragma unroll
    for (int k = 0; k < 12; k++) {
        if (scatter)
            full[sidx(k, s, g.vol)] = half[sidx(k, h, vh)];
        else
            half[sidx(k, h, vh)] = full[sidx(k, s, g.vol)];
    }
}

inline int eo_blocks(const Geom& g) { return (g.vol / 2 + 127) / 128; }

template <typename R>
void eo_hop(const Geom& g, const cx_t<R>* u, int dag, int p_out, const cx_t<R>* other,
            const cx_t<R>* same, R c_diag, R c_hop, cx_t<R>* out, cudaStream_t st) {
    if (dag)
        k_eo_hop<R, 1><<<eo_blocks(g), 128, 0, st>>>(g, u, p_out, other, same, c_diag, c_hop, out);
    else
        k_eo_hop<R, 0><<<eo_blocks(g), 128, 0, st>>>(g, u, p_out, other, same, c_diag, c_hop, out);
    SEEDCG_CHECK_LAUNCH();
}

// y_o = A x_o (dag = 0) or A^dag x_o (dag = 1), one half vector; t: even-site scratch
template <typename R>
void apply_a(const Geom& g, const cx_t<R>* u, double kappa, int dag, const cx_t<R>* x, cx_t<R>* t,
             cx_t<R>* y, cudaStream_t st) {
    eo_hop<R>(g, u, dag, 0, x, nullptr, R(0), R(1), t, st);                              // H_eo x
    eo_hop<R>(g, u, dag, 1, t, x, R(1), (R)(-kappa * kappa), y, st);                     // x - k^2 H_oe t
}

}  // namespace

// out_r = A^dag A x_r for n FP64 half vectors (te: one even half vector, y: one odd)
void eo_apply_mdag_m_f64(const Geom& g, const double2* u, double kappa, int n, const double2* x,
                         double2* te, double2* y, double2* out, cudaStream_t st) {
    const size_t hf = (size_t)g.vol / 2 * 12;
    for (int r = 0; r < n; r++) {
        apply_a<double>(g, u, kappa, 0, x + r * hf, te, y, st);
        apply_a<double>(g, u, kappa, 1, y, te, out + r * hf, st);
    }
}

// phi = eta_o + kappa H_oe eta_e and b = A^dag phi for n full FP64 fields
// (internal layout); phi, b: half vectors; ee, eo, te: half scratch
void eo_rhs_f64(const Geom& g, const double2* u, double kappa, int n, const double2* eta, double2* phi,
                double2* b, double2* ee, double2* eo, double2* te, cudaStream_t st) {
    const size_t hf = (size_t)g.vol / 2 * 12, ff = (size_t)g.vol * 12;
    for (int r = 0; r < n; r++) {
        k_eo_move<double2><<<eo_blocks(g), 128, 0, st>>>(g, 0, 0, const_cast<double2*>(eta) + r * ff, ee);
        SEEDCG_CHECK_LAUNCH();
        k_eo_move<double2><<<eo_blocks(g), 128, 0, st>>>(g, 1, 0, const_cast<double2*>(eta) + r * ff, eo);
        SEEDCG_CHECK_LAUNCH();
        eo_hop<double>(g, u, 0, 1, ee, eo, 1.0, kappa, phi + r * hf, st);
        apply_a<double>(g, u, kappa, 1, phi + r * hf, te, b + r * hf, st);
    }
}

void eo_gather_f64(const Geom& g, int p, int n, const double2* full, double2* half, cudaStream_t st) {
    const size_t hf = (size_t)g.vol / 2 * 12, ff = (size_t)g.vol * 12;
    for (int r = 0; r < n; r++) {
        k_eo_move<double2><<<eo_blocks(g), 128, 0, st>>>(g, p, 0, const_cast<double2*>(full) + r * ff, half + r * hf);
        SEEDCG_CHECK_LAUNCH();
    }
}

// x = [x_e, x_o] with x_e = eta_e + kappa H_eo x_o for n fields (x: full; ee, xe: half scratch)
void eo_reconstruct_f64(const Geom& g, const double2* u, double kappa, int n, const double2* x_odd,
                        const double2* eta, double2* x, double2* ee, double2* xe, cudaStream_t st) {
    const size_t hf = (size_t)g.vol / 2 * 12, ff = (size_t)g.vol * 12;
    for (int r = 0; r < n; r++) {
        k_eo_move<double2><<<eo_blocks(g), 128, 0, st>>>(g, 0, 0, const_cast<double2*>(eta) + r * ff, ee);
        SEEDCG_CHECK_LAUNCH();
        eo_hop<double>(g, u, 0, 0, x_odd + r * hf, ee, 1.0, kappa, xe, st);
        k_eo_move<double2><<<eo_blocks(g), 128, 0, st>>>(g, 0, 1, x + r * ff, xe);
        SEEDCG_CHECK_LAUNCH();
        k_eo_move<double2><<<eo_blocks(g), 128, 0, st>>>(g, 1, 1, x + r * ff, const_cast<double2*>(x_odd) + r * hf);
        SEEDCG_CHECK_LAUNCH();
    }
}

namespace {

bool eo_dims_ok(const Geom& g) {
    for (int mu = 0; mu < 4; mu++)
        if (g.L[mu] % 2) return false;
    return true;
}

template <typename R>
void apply_eo_impl(seedcg_handle* h, int op, int n, const double* in, double* out, cudaStream_t st) {
    const Geom& g = h->g;
    const int vh = g.vol / 2;
    const size_t hf = (size_t)vh * 12;
    const cx_t<R>* u = sizeof(R) == 8 ? reinterpret_cast<const cx_t<R>*>(h->u64.p)
                                      : reinterpret_cast<const cx_t<R>*>(h->u32.p);
    DevBuf buf;
    buf.ensure((3 * (size_t)n + 1) * hf * sizeof(cx_t<R>));
    cx_t<R>* X = buf.as<cx_t<R>>();
    cx_t<R>* Y = X + (size_t)n * hf;
    cx_t<R>* Z = Y + (size_t)n * hf;
    cx_t<R>* T = Z + (size_t)n * hf;
    if (sizeof(R) == 8) to_internal_f64(in, reinterpret_cast<double2*>(X), vh, n, st);
    else to_internal_f32(in, reinterpret_cast<float2*>(X), vh, n, st);
    cx_t<R>* res = Y;
    for (int r = 0; r < n; r++) {
        const cx_t<R>* x = X + (size_t)r * hf;
        cx_t<R>* y = Y + (size_t)r * hf;
        if (op == 0) {
            apply_a<R>(g, u, h->kappa, 0, x, T, y, st);
        } else if (op == 1) {
            apply_a<R>(g, u, h->kappa, 1, x, T, y, st);
        } else {
            apply_a<R>(g, u, h->kappa, 0, x, T, y, st);
            apply_a<R>(g, u, h->kappa, 1, y, T, Z + (size_t)r * hf, st);
            res = Z;
        }
    }
    if (sizeof(R) == 8) from_internal_f64(reinterpret_cast<double2*>(res), out, vh, n, st);
    else from_internal_f32(reinterpret_cast<float2*>(res), out, vh, n, st);
    SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
}

bool is_dev(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

seedcg_status check_eo(seedcg_handle* h, int n, std::initializer_list<const void*> ptrs) {
    if (!h) return SEEDCG_ERR_ARG;
    if (n < 1) {
        h->err = "n must be >= 1";
        return SEEDCG_ERR_ARG;
    }
    if (!eo_dims_ok(h->g)) {
        h->err = "even-odd preconditioning needs every lattice extent even";
        return SEEDCG_ERR_ARG;
    }
    for (const void* p : ptrs)
        if (!p || !is_dev(p)) {
            h->err = "even-odd calls take device pointers";
            return SEEDCG_ERR_ARG;
        }
    return SEEDCG_OK;
}

}  // namespace
}  // namespace seedcg

using seedcg::DevBuf;
using seedcg::Error;

extern "C" seedcg_status seedcg_apply_eo(seedcg_handle* h, int op, int prec, int n, const double* in,
                                         double* out, void* stream) {
    seedcg_status c = seedcg::check_eo(h, n, {in, out});
    if (c != SEEDCG_OK) return c;
    if (op < 0 || op > 2 || prec < 0 || prec > 1 || in == out) {
        h->err = "bad op / prec, or in and out alias";
        return SEEDCG_ERR_ARG;
    }
    try {
        SEEDCG_CUDA_TRY(cudaSetDevice(h->device));
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        if (prec == 0) seedcg::apply_eo_impl<double>(h, op, n, in, out, st);
        else seedcg::apply_eo_impl<float>(h, op, n, in, out, st);
        return SEEDCG_OK;
    } catch (const Error& e) {
        h->err = e.msg;
        return e.code;
    }
}

extern "C" seedcg_status seedcg_eo_source(seedcg_handle* h, int n, const double* eta, double* phi,
                                          void* stream) {
    seedcg_status c = seedcg::check_eo(h, n, {eta, phi});
    if (c != SEEDCG_OK) return c;
    try {
        SEEDCG_CUDA_TRY(cudaSetDevice(h->device));
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        const seedcg::Geom& g = h->g;
        const int vh = g.vol / 2;
        const size_t hf = (size_t)vh * 12, ff = (size_t)g.vol * 12;
        DevBuf buf;
        buf.ensure(((size_t)n * ff + (size_t)n * hf + 2 * hf) * sizeof(double2));
        double2* E = buf.as<double2>();
        double2* P = E + (size_t)n * ff;
        double2* Ee = P + (size_t)n * hf;
        double2* Eo = Ee + hf;
        seedcg::to_internal_f64(eta, E, g.vol, n, st);
        for (int r = 0; r < n; r++) {
            seedcg::k_eo_move<double2><<<seedcg::eo_blocks(g), 128, 0, st>>>(g, 0, 0, E + (size_t)r * ff, Ee);
            SEEDCG_CHECK_LAUNCH();
            seedcg::k_eo_move<double2><<<seedcg::eo_blocks(g), 128, 0, st>>>(g, 1, 0, E + (size_t)r * ff, Eo);
            SEEDCG_CHECK_LAUNCH();
            // phi = eta_o + kappa H_oe eta_e
            seedcg::eo_hop<double>(g, h->u64.as<double2>(), 0, 1, Ee, Eo, 1.0, h->kappa, P + (size_t)r * hf, st);
        }
        seedcg::from_internal_f64(P, phi, vh, n, st);
        SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
        return SEEDCG_OK;
    } catch (const Error& e) {
        h->err = e.msg;
        return e.code;
    }
}

extern "C" seedcg_status seedcg_eo_reconstruct(seedcg_handle* h, int n, const double* x_odd,
                                               const double* eta, double* x, void* stream) {
    seedcg_status c = seedcg::check_eo(h, n, {x_odd, eta, x});
    if (c != SEEDCG_OK) return c;
    try {
        SEEDCG_CUDA_TRY(cudaSetDevice(h->device));
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        const seedcg::Geom& g = h->g;
        const int vh = g.vol / 2;
        const size_t hf = (size_t)vh * 12, ff = (size_t)g.vol * 12;
        DevBuf buf;
        buf.ensure((2 * (size_t)n * ff + (size_t)n * hf + 2 * hf) * sizeof(double2));
        double2* E = buf.as<double2>();
        double2* F = E + (size_t)n * ff;
        double2* Xo = F + (size_t)n * ff;
        double2* Ee = Xo + (size_t)n * hf;
        double2* Xe = Ee + hf;
        seedcg::to_internal_f64(eta, E, g.vol, n, st);
        seedcg::to_internal_f64(x_odd, Xo, vh, n, st);
        for (int r = 0; r < n; r++) {
            double2* fr = F + (size_t)r * ff;
            double2* xo = Xo + (size_t)r * hf;
            seedcg::k_eo_move<double2><<<seedcg::eo_blocks(g), 128, 0, st>>>(g, 0, 0, E + (size_t)r * ff, Ee);
            SEEDCG_CHECK_LAUNCH();
            // x_e = eta_e + kappa H_eo x_o
            seedcg::eo_hop<double>(g, h->u64.as<double2>(), 0, 0, xo, Ee, 1.0, h->kappa, Xe, st);
            seedcg::k_eo_move<double2><<<seedcg::eo_blocks(g), 128, 0, st>>>(g, 0, 1, fr, Xe);
            SEEDCG_CHECK_LAUNCH();
            seedcg::k_eo_move<double2><<<seedcg::eo_blocks(g), 128, 0, st>>>(g, 1, 1, fr, xo);
            SEEDCG_CHECK_LAUNCH();
        }
        seedcg::from_internal_f64(F, x, g.vol, n, st);
        SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
        return SEEDCG_OK;
    } catch (const Error& e) {
        h->err = e.msg;
        return e.code;
    }
}

extern "C" seedcg_status seedcg_solve_eo(seedcg_handle* h, int nrhs, const double* eta, double* x, double tol,
                                         int extra_iters, int reorth_period, seedcg_info* info, void* stream) {
    seedcg_status c = seedcg::check_eo(h, nrhs, {eta, x});
    if (c != SEEDCG_OK) return c;
    if (!(tol > 0.0) || !(tol < 1.0) || extra_iters < 0 || reorth_period < 0 || nrhs > 256 || eta == x) {
        h->err = "bad tol, extra_iters, reorth_period or nrhs, or eta and x alias";
        return SEEDCG_ERR_ARG;
    }
    if (h->opt.use_guess || h->opt.resid_mode != 0) {
        h->err = "seedcg_solve_eo: use_guess and resid_mode = 1 are full-lattice options (the original "
                 "system's residual is reported in info->true_resid_D)";
        return SEEDCG_ERR_ARG;
    }
    try {
        SEEDCG_CUDA_TRY(cudaSetDevice(h->device));
        return seedcg::solve_eo_impl(h, nrhs, eta, x, tol, extra_iters, reorth_period, info,
                                     reinterpret_cast<cudaStream_t>(stream));
    } catch (const Error& e) {
        h->err = e.msg;
        return e.code;
    }
}
