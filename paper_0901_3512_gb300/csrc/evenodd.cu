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
#include <chrono>
#include <cmath>
#include <complex>
#include <vector>

#include "handle.cuh"
#include "internal.cuh"
#include "kernels.cuh"
#include "wilson.cuh"

namespace seedcg {
namespace {

// full site of half index h with parity p
__device__ __forceinline__ int eo_site(const Geom& g, int h, int p) {
    const int s0 = 2 * h;                       // x of s0 is even (Lx is even)
    const int r = s0 / g.L[0];
    const int y = r % g.L[1], z = (r / g.L[1]) % g.L[2], t = r / (g.L[1] * g.L[2]);
    return s0 + (((y + z + t) ^ p) & 1);
}

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
    const int vol = g.vol;
    const int s = eo_site(g, h, p_out);
    const Nbr nb = neighbours(g, s);
    Spinor<R> acc;
    if (same) {
        load_spinor(same, vh, h, acc);
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc.c[a][c] = cscale(acc.c[a][c], c_diag);
    } else {
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc.c[a][c] = mk<R>(0, 0);
    }
    constexpr int SF = DAG ? 1 : -1;
    constexpr int SB = -SF;
    Spinor<R> p;
    auto fl = [&](int mu, int e) { return __ldg(u + (size_t)(mu * 9 + e) * vol + s); };
    auto bl = [&](int mu, int e) { return __ldg(u + (size_t)(mu * 9 + e) * vol + nb.b[mu]); };
#define SEEDCG_EO_HOP(MU)                                                                            \
    {                                                                                                \
        const R cf = (MU == 3 && nb.fwrap_t) ? -c_hop : c_hop;                                       \
        const R cb = (MU == 3 && nb.bwrap_t) ? -c_hop : c_hop;                                       \
        load_spinor(other, vh, nb.f[MU] >> 1, p);                                                    \
        hop<MU, SF, false, R>(acc, p, [&](int a, int b) { return fl(MU, 3 * a + b); }, cf);          \
        load_spinor(other, vh, nb.b[MU] >> 1, p);                                                    \
        hop<MU, SB, true, R>(acc, p, [&](int a, int b) { return bl(MU, 3 * a + b); }, cb);           \
    }
    SEEDCG_EO_HOP(0)
    SEEDCG_EO_HOP(1)
    SEEDCG_EO_HOP(2)
    SEEDCG_EO_HOP(3)
#undef SEEDCG_EO_HOP
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

// ---------------------------------------------------------------------------
// Improved Seed-CG on the even-odd system A^dag A x_o = A^dag phi (Section 3),
// FP64, host-driven: the scalars of Algorithm 1 live on the host, every vector
// operation is one of this library's kernels.  The readings are those of the
// full-lattice solver: blocked Eq. (1) seeds from the post-PO basis, PO as one
// projection of [v_i, f] against v_1..v_{i-1} followed by v_i's normalisation
// and its removal from f, the guard that ends Lanczos at i - 1, and textbook
// CG (restarted from the true residual) for every system above tol.
// ---------------------------------------------------------------------------

// y = a x + b y (complex scalars)
__global__ void k_zaxpby(long n, double2 a, const double2* __restrict__ x, double2 b, double2* __restrict__ y) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        y[e] = cadd(cmul(a, x[e]), cmul(b, y[e]));
}

struct EoSolver {
    seedcg_handle* h;
    long n;
    cudaStream_t st;
    double* partials;
    unsigned* ctr;
    double2* res;
    double2* t_even;
    double2* y_odd;

    void axpby(double2 a, const double2* x, double2 b, double2* y) {
        const int nb = (int)std::min<long>((n + 255) / 256, 152 * 8);
        k_zaxpby<<<nb, 256, 0, st>>>(n, a, x, b, y);
        SEEDCG_CHECK_LAUNCH();
    }
    std::complex<double> dotz(const double2* a, const double2* b) {
        dot<double>(a, b, n, partials, ctr, res, st);
        double2 r;
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(&r, res, sizeof(double2), cudaMemcpyDeviceToHost, st));
        SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
        return {r.x, r.y};
    }
    double norm(const double2* a) { return std::sqrt(std::max(dotz(a, a).real(), 0.0)); }
    // y = A^dag A x
    void op(const double2* x, double2* y) {
        apply_a<double>(h->g, h->u64.as<double2>(), h->kappa, 0, x, t_even, y_odd, st);
        apply_a<double>(h->g, h->u64.as<double2>(), h->kappa, 1, y_odd, t_even, y, st);
    }
    void copy(const double2* x, double2* y) {
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(y, x, n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    }
    // textbook CG from x; returns iterations, *tr = ||b - M x|| / ||b||
    int cg(const double2* b, double2* x, double2* r, double2* p, double2* q, double tol, int maxiter, double* tr) {
        const double bn = norm(b);
        if (bn == 0.0) {
            *tr = 0.0;
            return 0;
        }
        int it = 0;
        for (int restart = 0; restart < 8; restart++) {
            op(x, r);
            axpby(make_double2(1, 0), b, make_double2(-1, 0), r);       // r = b - M x
            double rr = dotz(r, r).real();
            if (std::sqrt(rr) <= tol * bn) {
                *tr = std::sqrt(rr) / bn;
                return it;
            }
            copy(r, p);
            while (it < maxiter) {
                op(p, q);
                const double pq = dotz(p, q).real();
                const double a = rr / pq;
                axpby(make_double2(a, 0), p, make_double2(1, 0), x);
                axpby(make_double2(-a, 0), q, make_double2(1, 0), r);
                const double rn = dotz(r, r).real();
                it++;
                if (std::sqrt(rn) <= tol * bn) break;
                axpby(make_double2(1, 0), r, make_double2(rn / rr, 0), p);
                rr = rn;
            }
            if (it >= maxiter) break;
        }
        op(x, r);
        axpby(make_double2(1, 0), b, make_double2(-1, 0), r);
        *tr = norm(r) / bn;
        return it;
    }
};

seedcg_status eo_solve_impl(seedcg_handle* h, int nrhs, const double* eta, double* x, double tol, int extra,
                            int k, seedcg_info* info, cudaStream_t st) {
    const auto t0 = std::chrono::steady_clock::now();
    const Geom& g = h->g;
    const int vh = g.vol / 2;
    const long n = 12L * vh, ff = 12L * g.vol;
    const seedcg_options& o = h->opt;
    const int m_max = std::max(o.m_max, 1);
    DevBuf ebuf, vecs, vbuf, red, cbuf, scr, fbuf;
    ebuf.ensure((size_t)nrhs * ff * sizeof(double2));
    // Phi, B, X, R0 per system; work: v|f pair, vprev, Ee, Eo/Xe, t_even, y_odd, r, p, q
    vecs.ensure(((size_t)4 * nrhs + 11) * n * sizeof(double2));
    double2* E = ebuf.as<double2>();
    double2* Phi = vecs.as<double2>();
    double2* Bv = Phi + (size_t)nrhs * n;
    double2* X = Bv + (size_t)nrhs * n;
    double2* R0 = X + (size_t)nrhs * n;
    double2* VF = R0 + (size_t)nrhs * n;   // v at [0, n), f at [n, 2n)
    double2* vprev = VF + 2 * n;
    double2* Ee = vprev + n;
    double2* Eo = Ee + n;
    double2* Te = Eo + n;
    double2* Yo = Te + n;
    double2* r = Yo + n;
    double2* pv = r + n;
    double2* q = pv + n;
    vbuf.ensure((size_t)m_max * n * sizeof(double2));
    double2* V = vbuf.as<double2>();
    red.ensure(sizeof(double) * 4096 * 8 + 256 + sizeof(unsigned) * 64);
    EoSolver es{h, n, st, red.as<double>(), reinterpret_cast<unsigned*>(red.as<char>() + sizeof(double) * 4096 * 8 + 256),
                reinterpret_cast<double2*>(red.as<char>() + sizeof(double) * 4096 * 8), Te, Yo};
    SEEDCG_CUDA_TRY(cudaMemsetAsync(es.ctr, 0, sizeof(unsigned) * 64, st));
    // phi = eta_o + kappa H_oe eta_e, b = A^dag phi, x_0 = 0
    to_internal_f64(eta, E, g.vol, nrhs, st);
    for (int j = 0; j < nrhs; j++) {
        k_eo_move<double2><<<eo_blocks(g), 128, 0, st>>>(g, 0, 0, E + (size_t)j * ff, Ee);
        k_eo_move<double2><<<eo_blocks(g), 128, 0, st>>>(g, 1, 0, E + (size_t)j * ff, Eo);
        SEEDCG_CHECK_LAUNCH();
        eo_hop<double>(g, h->u64.as<double2>(), 0, 1, Ee, Eo, 1.0, h->kappa, Phi + (size_t)j * n, st);
        apply_a<double>(g, h->u64.as<double2>(), h->kappa, 1, Phi + (size_t)j * n, Te, Bv + (size_t)j * n, st);
    }
    SEEDCG_CUDA_TRY(cudaMemsetAsync(X, 0, (size_t)nrhs * n * sizeof(double2), st));
    SEEDCG_CUDA_TRY(cudaMemcpyAsync(R0, Bv, (size_t)nrhs * n * sizeof(double2), cudaMemcpyDeviceToDevice, st));

    // ---- Algorithm 1 on system 1 ----
    std::vector<double> alpha, beta;
    const double bn1 = es.norm(Bv);
    const double beta0 = es.norm(R0);
    int m = 0, m_conv = 0, po = 0;
    if (beta0 > 0.0) {
        double2* v = VF;
        double2* f = VF + n;
        es.axpby(make_double2(1.0 / beta0, 0), R0, make_double2(0, 0), v);
        double delta = 0.0, zeta = beta0, delta_prev = 0.0;
        int mt = m_max;
        for (int i = 1;; i++) {
            es.op(v, f);
            if (i > 1) es.axpby(make_double2(-beta.back(), 0), vprev, make_double2(1, 0), f);
            const double a = es.dotz(v, f).real();
            es.axpby(make_double2(-a, 0), v, make_double2(1, 0), f);
            if (i == 1) {
                delta = a;
            } else {
                const double gm = beta.back() / delta_prev;
                delta = a - gm * beta.back();
                zeta = -gm * zeta;
            }
            double b = es.norm(f);
            if (k > 0 && i >= 2 && i % k == 0) {
                const int na = i - 1;
                const size_t se = proj_scratch_elems<double, double2>(n, na);
                scr.ensure(se * sizeof(double2));
                cbuf.ensure((size_t)na * 2 * sizeof(double2));
                proj<double, double2>(V, n, na, VF, n, 2, n, cbuf.as<double2>(), 2, scr.as<double2>(), se, st);
                gemm_n<double, double2, double2>(V, n, na, cbuf.as<double2>(), 2, 2, VF, n, n, -1.0, st);
                const double nv = es.norm(v);
                if (!(nv >= 0.5)) {              // guard: end at i - 1
                    m = i - 1;
                    break;
                }
                es.axpby(make_double2(1.0 / nv, 0), v, make_double2(0, 0), v);
                const std::complex<double> d = es.dotz(v, f);
                es.axpby(make_double2(-d.real(), -d.imag()), v, make_double2(1, 0), f);
                const double bnew = es.norm(f);
                if (!(bnew <= 1.01 * b)) {
                    m = i - 1;
                    break;
                }
                b = bnew;
                po++;
            }
            alpha.push_back(a);
            beta.push_back(b);
            es.copy(v, V + (size_t)(i - 1) * n);
            m = i;
            delta_prev = delta;
            const double est = b * std::fabs(zeta / delta);
            if (m_conv == 0 && est <= tol * bn1) {
                m_conv = i;
                mt = std::min(m_max, std::max(i + extra, (int)std::ceil(o.past_factor * i)));
            }
            if (b <= 1e-14 * std::fabs(a) || !std::isfinite(b)) break;
            if (i >= mt || i >= m_max) break;
            es.copy(v, vprev);
            es.axpby(make_double2(1.0 / b, 0), f, make_double2(0, 0), v);
        }
    }
    alpha.resize(m);
    beta.resize(m);
    // ---- Eq. (1): X = V T^-1 V^dag R0 ----
    if (m > 0) {
        const size_t se = std::max<size_t>((size_t)m * nrhs * 64, (size_t)1 << 20);
        scr.ensure(se * sizeof(double2));
        cbuf.ensure((size_t)m * nrhs * sizeof(double2));
        gemm_t<double, double2>(V, n, m, R0, n, nrhs, n, cbuf.as<double2>(), nrhs, scr.as<double2>(), se, st);
        std::vector<double2> c((size_t)m * nrhs);
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(c.data(), cbuf.p, c.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
        SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
        std::vector<double> cp(m);
        std::vector<std::complex<double>> dp(m), y(m);
        for (int j = 0; j < nrhs; j++) {
            // Thomas algorithm on the symmetric tridiagonal T_m
            for (int i = 0; i < m; i++) {
                const double piv = alpha[i] - (i > 0 ? beta[i - 1] * cp[i - 1] : 0.0);
                cp[i] = i < m - 1 ? beta[i] / piv : 0.0;
                const std::complex<double> ci(c[(size_t)i * nrhs + j].x, c[(size_t)i * nrhs + j].y);
                dp[i] = (ci - (i > 0 ? beta[i - 1] * dp[i - 1] : 0.0)) / piv;
            }
            y[m - 1] = dp[m - 1];
            for (int i = m - 2; i >= 0; i--) y[i] = dp[i] - cp[i] * y[i + 1];
            for (int i = 0; i < m; i++) c[(size_t)i * nrhs + j] = make_double2(y[i].real(), y[i].imag());
        }
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(cbuf.p, c.data(), c.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
        gemm_n<double, double2, double2>(V, n, m, cbuf.as<double2>(), nrhs, nrhs, X, n, n, 1.0, st);
    }
    // ---- CG for every system above tol ----
    seedcg_status code = SEEDCG_OK;
    std::vector<int> cg_it(nrhs);
    std::vector<double> tr(nrhs);
    for (int j = 0; j < nrhs; j++) {
        cg_it[j] = es.cg(Bv + (size_t)j * n, X + (size_t)j * n, r, pv, q, tol, o.cg_maxiter, &tr[j]);
        if (!(tr[j] <= tol)) code = SEEDCG_ERR_NOT_CONVERGED;
    }
    // ---- x_e = eta_e + kappa H_eo x_o, and the full solution ----
    fbuf.ensure((size_t)nrhs * ff * sizeof(double2));
    double2* F = fbuf.as<double2>();
    for (int j = 0; j < nrhs; j++) {
        k_eo_move<double2><<<eo_blocks(g), 128, 0, st>>>(g, 0, 0, E + (size_t)j * ff, Ee);
        SEEDCG_CHECK_LAUNCH();
        eo_hop<double>(g, h->u64.as<double2>(), 0, 0, X + (size_t)j * n, Ee, 1.0, h->kappa, Eo, st);
        k_eo_move<double2><<<eo_blocks(g), 128, 0, st>>>(g, 0, 1, F + (size_t)j * ff, Eo);
        k_eo_move<double2><<<eo_blocks(g), 128, 0, st>>>(g, 1, 1, F + (size_t)j * ff, X + (size_t)j * n);
        SEEDCG_CHECK_LAUNCH();
    }
    from_internal_f64(F, x, g.vol, nrhs, st);
    SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
    if (info) {
        info->m_conv = m_conv;
        info->m = m;
        info->po_count = po;
        int mx = 0;
        for (int j = 0; j < nrhs; j++) mx = std::max(mx, cg_it[j]);
        info->cg_iters_max = mx;
        info->reliable_updates = 0;
        for (int j = 0; j < nrhs; j++) {
            if (info->iters) info->iters[j] = cg_it[j] + (j == 0 ? m : 0);
            if (info->matvecs) info->matvecs[j] = 4 * (cg_it[j] + (j == 0 ? m : 0));
            if (info->true_resid) info->true_resid[j] = tr[j];
        }
        const float ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
        info->ms_total = ms;
        info->ms_lanczos = info->ms_po = info->ms_seed = info->ms_cg = 0.f;
    }
    return code;
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
    try {
        SEEDCG_CUDA_TRY(cudaSetDevice(h->device));
        return seedcg::eo_solve_impl(h, nrhs, eta, x, tol, extra_iters, reorth_period, info,
                                     reinterpret_cast<cudaStream_t>(stream));
    } catch (const Error& e) {
        h->err = e.msg;
        return e.code;
    }
}
