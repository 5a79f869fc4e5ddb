// The C ABI (include/seedcg.h): argument checks, host/device staging, and
// the dispatch to the solver and the dslash kernels.  No exception crosses
// the ABI: every entry point converts failures into a seedcg_status and a
// message kept in the handle.
#include <cstring>
#include <new>
#include <vector>

#include "handle.cuh"
#include "kernels.cuh"

using seedcg::Error;

namespace seedcg {
std::atomic<unsigned long long> g_kernel_launches{0};
}

namespace {

constexpr size_t kPinnedBytes = 64 * 1024;

thread_local std::string g_create_error;

seedcg_status fail(seedcg_handle* h, seedcg_status code, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool valid_options(const seedcg_options& o, std::string& why) {
    if (o.m_max < 1) { why = "m_max must be >= 1"; return false; }
    if (!(o.past_factor >= 1.0)) { why = "past_factor must be >= 1"; return false; }
    if (o.precision < 0 || o.precision > 2) { why = "unknown precision mode"; return false; }
    if (!(o.reliable_delta > 0.0 && o.reliable_delta < 1.0)) { why = "reliable_delta must be in (0,1)"; return false; }
    if (o.po_passes < 1 || o.po_passes > 2) { why = "po_passes must be 1 or 2"; return false; }
    if (o.seed_mode < 0 || o.seed_mode > 3) { why = "seed_mode must be 0, 1, 2 or 3"; return false; }
    if (o.seed_mode == 0 && o.precision != SEEDCG_FP64) { why = "literal seeding (seed_mode 0) needs precision FP64"; return false; }
    if (o.cg_maxiter < 1) { why = "cg_maxiter must be >= 1"; return false; }
    if (o.poll_every < 1) { why = "poll_every must be >= 1"; return false; }
    if (o.use_tensor_cores < 0 || o.use_tensor_cores > 2) { why = "use_tensor_cores must be 0, 1 or 2"; return false; }
    if (o.use_guess < 0 || o.use_guess > 1) { why = "use_guess must be 0 or 1"; return false; }
    if (o.resid_mode < 0 || o.resid_mode > 1) { why = "resid_mode must be 0 or 1"; return false; }
    if (o.po_guard < 0 || o.po_guard > 1) { why = "po_guard must be 0 or 1"; return false; }
    return true;
}

}  // namespace

extern "C" {

void seedcg_default_options(seedcg_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->m_max = 4000;
    opt->past_factor = 1.0;
    opt->precision = SEEDCG_FP64;
    opt->reliable_delta = 0.1;
    opt->po_passes = 1;
    opt->seed_mode = 1;
    opt->x0_given = 0;
    opt->cg_maxiter = 20000;
    opt->stop_after_seed = 0;
    opt->poll_every = 32;
    opt->use_tensor_cores = 1;
    opt->use_guess = 0;
    opt->resid_mode = 0;
    opt->po_guard = 1;
}

seedcg_status seedcg_create(seedcg_handle** out, const int dims[4], const double* gauge,
                            double kappa, const seedcg_options* opt) {
    if (!out) return fail(nullptr, SEEDCG_ERR_ARG, "h is NULL");
    *out = nullptr;
    if (!dims || !gauge) return fail(nullptr, SEEDCG_ERR_ARG, "dims or gauge is NULL");
    long vol = 1;
    for (int i = 0; i < 4; i++) {
        if (dims[i] < 2 || (dims[i] & 1))
            return fail(nullptr, SEEDCG_ERR_ARG, "every lattice extent must be even and >= 2");
        vol *= dims[i];
    }
    if (vol * 12 > (1L << 31) - 1) return fail(nullptr, SEEDCG_ERR_ARG, "lattice too large");
    if (!(kappa == kappa)) return fail(nullptr, SEEDCG_ERR_ARG, "kappa is NaN");
    seedcg_options o;
    seedcg_default_options(&o);
    if (opt) o = *opt;
    std::string why;
    if (!valid_options(o, why)) return fail(nullptr, SEEDCG_ERR_ARG, why);
    seedcg_handle* h = new (std::nothrow) seedcg_handle();
    if (!h) return fail(nullptr, SEEDCG_ERR_OOM, "host allocation failed");
    try {
        h->g = seedcg::make_geom(dims);
        h->kappa = kappa;
        h->opt = o;
        SEEDCG_CUDA_TRY(cudaGetDevice(&h->device));
        SEEDCG_CUDA_TRY(cudaMallocHost(&h->pinned, kPinnedBytes));
        const size_t nl = (size_t)vol * 36;
        h->u64.ensure(nl * sizeof(double2));
        h->u32.ensure(nl * sizeof(float2));
        const double* src = gauge;
        seedcg::DevBuf tmp;
        if (!is_device_ptr(gauge)) {
            tmp.ensure(nl * sizeof(double2));
            SEEDCG_CUDA_TRY(cudaMemcpy(tmp.p, gauge, nl * sizeof(double2), cudaMemcpyHostToDevice));
            src = tmp.as<double>();
        }
        seedcg::gauge_to_internal(src, h->u64.as<double2>(), h->u32.as<float2>(), (int)vol, 0);
        SEEDCG_CUDA_TRY(cudaDeviceSynchronize());
        tmp.release();
    } catch (const Error& e) {
        g_create_error = e.msg;
        seedcg_destroy(h);
        return e.code;
    }
    *out = h;
    return SEEDCG_OK;
}

seedcg_status seedcg_set_options(seedcg_handle* h, const seedcg_options* opt) {
    if (!h || !opt) return fail(h, SEEDCG_ERR_ARG, "h or opt is NULL");
    std::string why;
    if (!valid_options(*opt, why)) return fail(h, SEEDCG_ERR_ARG, why);
    h->opt = *opt;
    return SEEDCG_OK;
}

seedcg_status seedcg_solve(seedcg_handle* h, int nrhs, const double* B, double* X, double tol,
                           int extra_iters, int reorth_period, seedcg_info* info, void* stream) {
    if (!h) return fail(nullptr, SEEDCG_ERR_ARG, "h is NULL");
    if (nrhs < 1 || nrhs > 256) return fail(h, SEEDCG_ERR_ARG, "nrhs must be in [1, 256]");
    if (!B || !X) return fail(h, SEEDCG_ERR_ARG, "B or X is NULL");
    if (!(tol > 0.0) || !(tol < 1.0)) return fail(h, SEEDCG_ERR_ARG, "tol must be in (0, 1)");
    if (extra_iters < 0 || reorth_period < 0)
        return fail(h, SEEDCG_ERR_ARG, "extra_iters and reorth_period must be >= 0");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    try {
        SEEDCG_CUDA_TRY(cudaSetDevice(h->device));
        const size_t bytes = (size_t)nrhs * h->g.vol * 12 * sizeof(double2);
        const bool bd = is_device_ptr(B), xd = is_device_ptr(X);
        // device copies of host B / X live in the handle (kept between solves)
        if (!bd || !xd) h->hostio.ensure(2 * bytes + 512);
        const double* Bd = B;
        double* Xd = X;
        if (!bd) {
            SEEDCG_CUDA_TRY(cudaMemcpyAsync(h->hostio.p, B, bytes, cudaMemcpyHostToDevice, st));
            Bd = h->hostio.as<double>();
        }
        if (!xd) {
            double* hx = h->hostio.as<double>() + 2 * (bytes / sizeof(double2));
            if (h->opt.x0_given)
                SEEDCG_CUDA_TRY(cudaMemcpyAsync(hx, X, bytes, cudaMemcpyHostToDevice, st));
            Xd = hx;
        }
        seedcg_status code = seedcg::solve_impl(h, nrhs, Bd, Xd, tol, extra_iters, reorth_period,
                                                info, st);
        if (!xd) {
            SEEDCG_CUDA_TRY(cudaMemcpyAsync(X, Xd, bytes, cudaMemcpyDeviceToHost, st));
            SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
        }
        if (code != SEEDCG_OK) {
            const char* what = code == SEEDCG_ERR_NOT_CONVERGED ? "a system did not converge"
                             : code == SEEDCG_ERR_BREAKDOWN ? "delta_i = 0 in the LU of T (M not HPD?)"
                             : code == SEEDCG_ERR_NAN ? "NaN/Inf in a Lanczos scalar"
                             : code == SEEDCG_ERR_TIMEOUT ? "a bounded device wait expired"
                             : "solve failed";
            h->err = what;
        }
        return code;
    } catch (const Error& e) {
        return fail(h, e.code, e.msg);
    }
}

seedcg_status seedcg_batch_solve(seedcg_handle** hs, int nfields, const int* nrhs,
                                 const double* const* B, double* const* X, double tol,
                                 int extra_iters, int reorth_period, seedcg_info* infos,
                                 void* stream) {
    if (!hs || nfields < 1 || nfields > 16 || !nrhs || !B || !X)
        return fail(nullptr, SEEDCG_ERR_ARG, "batch: need 1..16 handles and per-field nrhs, B, X");
    seedcg_handle* h0 = hs[0];
    if (!h0) return fail(nullptr, SEEDCG_ERR_ARG, "batch: NULL handle");
    if (!(tol > 0.0) || !(tol < 1.0)) return fail(h0, SEEDCG_ERR_ARG, "tol must be in (0, 1)");
    if (extra_iters < 0 || reorth_period < 0)
        return fail(h0, SEEDCG_ERR_ARG, "extra_iters and reorth_period must be >= 0");
    int total = 0;
    for (int f = 0; f < nfields; f++) {
        if (!hs[f] || !B[f] || !X[f]) return fail(h0, SEEDCG_ERR_ARG, "batch: NULL handle, B or X");
        if (nrhs[f] < 1 || nrhs[f] > 256) return fail(h0, SEEDCG_ERR_ARG, "batch: nrhs must be in [1, 256]");
        if (hs[f]->opt.precision != h0->opt.precision || hs[f]->device != h0->device)
            return fail(h0, SEEDCG_ERR_ARG, "batch: all handles need the same precision and device");
        if (hs[f]->opt.resid_mode != 0)
            return fail(h0, SEEDCG_ERR_ARG, "batch: resid_mode = 1 is supported by seedcg_solve only");
        if (hs[f]->opt.seed_mode > 1)
            return fail(h0, SEEDCG_ERR_ARG, "batch: seed_mode 2 and 3 are supported by seedcg_solve only");
        for (int g = 0; g < f; g++)
            if (hs[g] == hs[f]) return fail(h0, SEEDCG_ERR_ARG, "batch: a handle appears twice");
        total += nrhs[f];
    }
    if (total > 512) return fail(h0, SEEDCG_ERR_ARG, "batch: at most 512 systems");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    try {
        SEEDCG_CUDA_TRY(cudaSetDevice(h0->device));
        std::vector<seedcg::DevBuf> hb(nfields), hx(nfields);
        std::vector<const double*> Bd(nfields);
        std::vector<double*> Xd(nfields);
        std::vector<bool> xhost(nfields, false);
        for (int f = 0; f < nfields; f++) {
            const size_t bytes = (size_t)nrhs[f] * hs[f]->g.vol * 12 * sizeof(double2);
            Bd[f] = B[f];
            Xd[f] = X[f];
            if (!is_device_ptr(B[f])) {
                hb[f].ensure(bytes);
                SEEDCG_CUDA_TRY(cudaMemcpyAsync(hb[f].p, B[f], bytes, cudaMemcpyHostToDevice, st));
                Bd[f] = hb[f].as<double>();
            }
            if (!is_device_ptr(X[f])) {
                xhost[f] = true;
                hx[f].ensure(bytes);
                if (hs[f]->opt.x0_given)
                    SEEDCG_CUDA_TRY(cudaMemcpyAsync(hx[f].p, X[f], bytes, cudaMemcpyHostToDevice, st));
                Xd[f] = hx[f].as<double>();
            }
        }
        seedcg_status code = seedcg::batch_solve_impl(hs, nfields, nrhs, Bd.data(), Xd.data(), tol,
                                                      extra_iters, reorth_period, infos, st);
        for (int f = 0; f < nfields; f++)
            if (xhost[f])
                SEEDCG_CUDA_TRY(cudaMemcpyAsync(X[f], Xd[f], (size_t)nrhs[f] * hs[f]->g.vol * 12 * sizeof(double2),
                                                cudaMemcpyDeviceToHost, st));
        SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
        if (code != SEEDCG_OK) h0->err = "batch: a system did not converge or a Lanczos run failed";
        return code;
    } catch (const Error& e) {
        return fail(h0, e.code, e.msg);
    }
}

seedcg_status seedcg_apply(seedcg_handle* h, int op, int prec, int multi, int n, const double* in,
                           double* out, void* stream) {
    if (!h) return fail(nullptr, SEEDCG_ERR_ARG, "h is NULL");
    if (op < 0 || op > 2 || prec < 0 || prec > 1 || n < 0)
        return fail(h, SEEDCG_ERR_ARG, "bad op/prec/n");
    if (n == 0) return SEEDCG_OK;
    if (!in || !out || in == out) return fail(h, SEEDCG_ERR_ARG, "in/out NULL or aliased");
    if (!is_device_ptr(in) || !is_device_ptr(out))
        return fail(h, SEEDCG_ERR_ARG, "seedcg_apply takes device pointers");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    try {
        SEEDCG_CUDA_TRY(cudaSetDevice(h->device));
        const int vol = h->g.vol;
        const size_t nf = (size_t)n * vol * 12;
        const size_t esz = prec == 0 ? sizeof(double2) : sizeof(float2);
        seedcg::DevBuf buf;
        buf.ensure(3 * nf * esz + 512);
        char* b0 = buf.as<char>();
        void* A = b0;
        void* Bv = b0 + nf * esz;
        void* Cv = b0 + 2 * nf * esz;
        if (prec == 0) {
            seedcg::to_internal_f64(in, (double2*)A, vol, n, st);
            auto apply = [&](int dag, const double2* x, double2* y) {
                if (multi) seedcg::dslash_mrhs_f64(h->g, h->u64.as<double2>(), h->kappa, dag, n, x, y, st);
                else
                    for (int r = 0; r < n; r++)
                        seedcg::dslash_f64(h->g, h->u64.as<double2>(), h->kappa, dag,
                                           x + (size_t)r * 12 * vol, y + (size_t)r * 12 * vol, st);
            };
            const double2* res = nullptr;
            if (op == 0) { apply(0, (double2*)A, (double2*)Bv); res = (double2*)Bv; }
            else if (op == 1) { apply(1, (double2*)A, (double2*)Bv); res = (double2*)Bv; }
            else { apply(0, (double2*)A, (double2*)Bv); apply(1, (double2*)Bv, (double2*)Cv); res = (double2*)Cv; }
            seedcg::from_internal_f64(res, out, vol, n, st);
        } else {
            seedcg::to_internal_f32(in, (float2*)A, vol, n, st);
            const float k = (float)h->kappa;
            auto apply = [&](int dag, const float2* x, float2* y) {
                if (multi) seedcg::dslash_mrhs_f32(h->g, h->u32.as<float2>(), k, dag, n, x, y, st);
                else
                    for (int r = 0; r < n; r++)
                        seedcg::dslash_f32(h->g, h->u32.as<float2>(), k, dag,
                                           x + (size_t)r * 12 * vol, y + (size_t)r * 12 * vol, st);
            };
            const float2* res = nullptr;
            if (op == 0) { apply(0, (float2*)A, (float2*)Bv); res = (float2*)Bv; }
            else if (op == 1) { apply(1, (float2*)A, (float2*)Bv); res = (float2*)Bv; }
            else { apply(0, (float2*)A, (float2*)Bv); apply(1, (float2*)Bv, (float2*)Cv); res = (float2*)Cv; }
            seedcg::from_internal_f32(res, out, vol, n, st);
        }
        SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
        return SEEDCG_OK;
    } catch (const Error& e) {
        return fail(h, e.code, e.msg);
    }
}

seedcg_status seedcg_get_lanczos(const seedcg_handle* h, int cap, double* alpha, double* beta,
                                 double* delta, int* m_out) {
    if (!h) return SEEDCG_ERR_ARG;
    const int m = h->last_m;
    if (m_out) *m_out = m;
    const int c = cap < m ? cap : m;
    for (int i = 0; i < c; i++) {
        if (alpha) alpha[i] = h->alpha[i];
        if (beta) beta[i] = h->beta[i];
        if (delta) delta[i] = h->delta[i];
    }
    return SEEDCG_OK;
}

seedcg_status seedcg_get_basis(seedcg_handle* h, int first, int count, double* out) {
    if (!h || !out) return fail(h, SEEDCG_ERR_ARG, "h or out is NULL");
    if (first < 0 || count < 0 || first + count > h->vbasis_m)
        return fail(h, SEEDCG_ERR_ARG, "requested rows are outside the stored basis");
    if (count == 0) return SEEDCG_OK;
    try {
        // rows of an even-odd solve are odd-site half vectors
        const int vol = h->vbasis_eo ? h->g.vol / 2 : h->g.vol;
        const long n = 12L * vol;
        const size_t bytes = (size_t)count * n * sizeof(double2);
        seedcg::DevBuf wide, canon;
        wide.ensure(bytes);
        double2* w = wide.as<double2>();
        const size_t off = (size_t)first * n;
        if (h->vbasis_prec == SEEDCG_FP64)
            seedcg::convert<double2, double2>(h->vbasis.as<double2>() + off, w, count * n, 0);
        else if (h->vbasis_prec == SEEDCG_MIXED_V32)
            seedcg::convert<float2, double2>(h->vbasis.as<float2>() + off, w, count * n, 0);
        else
            seedcg::convert<__nv_bfloat162, double2>(h->vbasis.as<__nv_bfloat162>() + off, w, count * n, 0);
        const bool od = is_device_ptr(out);
        double* dst = out;
        if (!od) {
            canon.ensure(bytes);
            dst = canon.as<double>();
        }
        seedcg::from_internal_f64(w, dst, vol, count, 0);
        if (!od) SEEDCG_CUDA_TRY(cudaMemcpy(out, dst, bytes, cudaMemcpyDeviceToHost));
        SEEDCG_CUDA_TRY(cudaDeviceSynchronize());
        return SEEDCG_OK;
    } catch (const Error& e) {
        return fail(h, e.code, e.msg);
    }
}

seedcg_status seedcg_tridiag_lowest(int m, const double* alpha, const double* beta, int nev, double* theta,
                                   double* S) {
    if (m < 1 || nev < 1 || nev > m || !alpha || (m > 1 && !beta) || !theta || !S) return SEEDCG_ERR_ARG;
    try {
        seedcg::tridiag_lowest(m, alpha, beta, nev, theta, S);
        return SEEDCG_OK;
    } catch (...) {
        return SEEDCG_ERR_ARG;
    }
}

seedcg_status seedcg_deflate_guess(seedcg_handle* h, int nev, int nr, const double* B, double* X0,
                                   double* ritz_values, void* stream) {
    if (!h || !B || !X0) return fail(h, SEEDCG_ERR_ARG, "h, B or X0 is NULL");
    if (h->vbasis_m < 1) return fail(h, SEEDCG_ERR_ARG, "no stored basis: run seedcg_solve first");
    if (h->vbasis_eo) return fail(h, SEEDCG_ERR_ARG, "the stored basis is of the even-odd system (half vectors)");
    if (nev < 1 || nev > 64 || nev > h->vbasis_m || nr < 1 || nr > 256)
        return fail(h, SEEDCG_ERR_ARG, "nev must be in [1, min(64, basis size)], nr in [1, 256]");
    if (!is_device_ptr(B) || !is_device_ptr(X0)) return fail(h, SEEDCG_ERR_ARG, "B and X0 must be device pointers");
    try {
        SEEDCG_CUDA_TRY(cudaSetDevice(h->device));
        seedcg_status c = seedcg::deflate_impl(h, nev, nr, B, X0, ritz_values,
                                               reinterpret_cast<cudaStream_t>(stream));
        if (c == SEEDCG_ERR_BREAKDOWN) h->err = "the Ritz Gram matrix Y^dag M Y is not positive definite";
        else if (c == SEEDCG_ERR_ARG) h->err = "bad nev or basis";
        return c;
    } catch (const Error& e) {
        return fail(h, e.code, e.msg);
    }
}

seedcg_status seedcg_project_basis(seedcg_handle* h, int rows, int nvec, const double* X,
                                   double* C, int use_tensor_cores, void* stream) {
    if (!h || !X || !C) return fail(h, SEEDCG_ERR_ARG, "h, X or C is NULL");
    if (rows < 1 || rows > h->vbasis_m || nvec < 1 || nvec > 32)
        return fail(h, SEEDCG_ERR_ARG, "rows must be in [1, stored basis size], nvec in [1, 32]");
    if (!is_device_ptr(X)) return fail(h, SEEDCG_ERR_ARG, "X must be a device pointer");
    if (h->vbasis_eo) return fail(h, SEEDCG_ERR_ARG, "the stored basis is of the even-odd system (half vectors)");
    try {
        SEEDCG_CUDA_TRY(cudaSetDevice(h->device));
        seedcg_status c = seedcg::project_basis_impl(h, rows, nvec, X, C, use_tensor_cores ? 1 : 0,
                                                     reinterpret_cast<cudaStream_t>(stream));
        if (c != SEEDCG_OK) h->err = "a bounded device wait expired";
        return c;
    } catch (const Error& e) {
        return fail(h, e.code, e.msg);
    }
}

namespace {
// stage n canonical complex128 fields (host or device) into the internal FP64 layout
void stage_in(seedcg_handle* h, int n, const double* src, seedcg::DevBuf& dst, cudaStream_t st) {
    const int vol = h->g.vol;
    const size_t bytes = (size_t)n * vol * 12 * sizeof(double2);
    dst.ensure(bytes);
    const double* d = src;
    seedcg::DevBuf tmp;
    if (!is_device_ptr(src)) {
        tmp.ensure(bytes);
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(tmp.p, src, bytes, cudaMemcpyHostToDevice, st));
        d = tmp.as<double>();
    }
    seedcg::to_internal_f64(d, dst.as<double2>(), vol, n, st);
    SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
}
}  // namespace

seedcg_status seedcg_guess_set_weights(seedcg_handle* h, const double* w) {
    if (!h || !w) return fail(h, SEEDCG_ERR_ARG, "h or w is NULL");
    try {
        SEEDCG_CUDA_TRY(cudaSetDevice(h->device));
        seedcg::guess_set_weights(h, w, 0);
        return SEEDCG_OK;
    } catch (const Error& e) {
        return fail(h, e.code, e.msg);
    }
}

seedcg_status seedcg_guess_get_weights(seedcg_handle* h, double* w) {
    if (!h || !w) return fail(h, SEEDCG_ERR_ARG, "h or w is NULL");
    try {
        seedcg::guess_get_weights(h, w, 0);
        return SEEDCG_OK;
    } catch (const Error& e) {
        return fail(h, e.code, e.msg);
    }
}

seedcg_status seedcg_guess_loss_grad(seedcg_handle* h, int npairs, const double* B, const double* X,
                                     double* loss, double* grad, void* stream) {
    if (!h || !B || !X || !loss || npairs < 1) return fail(h, SEEDCG_ERR_ARG, "bad guess arguments");
    if (!seedcg::guess_ready(h)) return fail(h, SEEDCG_ERR_ARG, "set the guess weights first");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    try {
        SEEDCG_CUDA_TRY(cudaSetDevice(h->device));
        seedcg::DevBuf b, x;
        stage_in(h, npairs, B, b, st);
        stage_in(h, npairs, X, x, st);
        *loss = seedcg::guess_loss_grad(h, npairs, b.as<double2>(), x.as<double2>(), grad, st);
        return SEEDCG_OK;
    } catch (const Error& e) {
        return fail(h, e.code, e.msg);
    }
}

seedcg_status seedcg_guess_train(seedcg_handle* h, int npairs, const double* B, const double* X,
                                 int epochs, int batch, double lr, double* final_loss, void* stream) {
    if (!h || !B || !X || npairs < 1 || epochs < 1 || batch < 1 || !(lr > 0.0))
        return fail(h, SEEDCG_ERR_ARG, "bad guess training arguments");
    if (!seedcg::guess_ready(h)) return fail(h, SEEDCG_ERR_ARG, "set the initial guess weights first");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    try {
        SEEDCG_CUDA_TRY(cudaSetDevice(h->device));
        seedcg::DevBuf b, x;
        stage_in(h, npairs, B, b, st);
        stage_in(h, npairs, X, x, st);
        const double l = seedcg::guess_train(h, npairs, b.as<double2>(), x.as<double2>(), epochs,
                                             batch, lr, st);
        if (final_loss) *final_loss = l;
        return SEEDCG_OK;
    } catch (const Error& e) {
        return fail(h, e.code, e.msg);
    }
}

seedcg_status seedcg_guess_predict(seedcg_handle* h, int n, const double* B, double* X0, void* stream) {
    if (!h || !B || !X0 || n < 1) return fail(h, SEEDCG_ERR_ARG, "bad guess arguments");
    if (!seedcg::guess_ready(h)) return fail(h, SEEDCG_ERR_ARG, "set the guess weights first");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    try {
        SEEDCG_CUDA_TRY(cudaSetDevice(h->device));
        const int vol = h->g.vol;
        const size_t bytes = (size_t)n * vol * 12 * sizeof(double2);
        seedcg::DevBuf b, x, c;
        stage_in(h, n, B, b, st);
        x.ensure(bytes);
        seedcg::guess_predict(h, n, b.as<double2>(), x.as<double2>(), st);
        const bool xd = is_device_ptr(X0);
        double* dst = X0;
        if (!xd) {
            c.ensure(bytes);
            dst = c.as<double>();
        }
        seedcg::from_internal_f64(x.as<double2>(), dst, vol, n, st);
        if (!xd) SEEDCG_CUDA_TRY(cudaMemcpyAsync(X0, dst, bytes, cudaMemcpyDeviceToHost, st));
        SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
        return SEEDCG_OK;
    } catch (const Error& e) {
        return fail(h, e.code, e.msg);
    }
}

seedcg_status seedcg_time_dslash(seedcg_handle* h, int prec, int n, int reps, int flush_l2,
                                float* ms_per_launch, void* stream) {
    if (!h || !ms_per_launch) return fail(h, SEEDCG_ERR_ARG, "h or ms_per_launch is NULL");
    if (prec < 0 || prec > 1 || n < 1 || reps < 1) return fail(h, SEEDCG_ERR_ARG, "bad prec/n/reps");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    try {
        SEEDCG_CUDA_TRY(cudaSetDevice(h->device));
        const int vol = h->g.vol;
        const size_t nf = (size_t)n * vol * 12;
        const size_t esz = prec == 0 ? sizeof(double2) : sizeof(float2);
        seedcg::DevBuf buf, flush;
        buf.ensure(2 * nf * esz + 512);
        SEEDCG_CUDA_TRY(cudaMemsetAsync(buf.p, 0, 2 * nf * esz, st));
        const size_t fbytes = (size_t)512 << 20;  // 4x the 129 MB L2
        if (flush_l2) flush.ensure(fbytes);
        char* b0 = buf.as<char>();
        cudaEvent_t e0, e1;
        SEEDCG_CUDA_TRY(cudaEventCreate(&e0));
        SEEDCG_CUDA_TRY(cudaEventCreate(&e1));
        float tot = 0.f;
        for (int r = 0; r < reps + 1; r++) {
            if (flush_l2) SEEDCG_CUDA_TRY(cudaMemsetAsync(flush.p, r & 0xff, fbytes, st));
            SEEDCG_CUDA_TRY(cudaEventRecord(e0, st));
            if (prec == 0)
                seedcg::dslash_mrhs_f64(h->g, h->u64.as<double2>(), h->kappa, 0, n,
                                        (const double2*)b0, (double2*)(b0 + nf * esz), st);
            else
                seedcg::dslash_mrhs_f32(h->g, h->u32.as<float2>(), (float)h->kappa, 0, n,
                                        (const float2*)b0, (float2*)(b0 + nf * esz), st);
            SEEDCG_CUDA_TRY(cudaEventRecord(e1, st));
            SEEDCG_CUDA_TRY(cudaEventSynchronize(e1));
            float t = 0.f;
            SEEDCG_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
            if (r > 0) tot += t;  // the first launch is a warm-up
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        *ms_per_launch = tot / reps;
        return SEEDCG_OK;
    } catch (const Error& e) {
        return fail(h, e.code, e.msg);
    }
}

unsigned long long seedcg_kernel_launches(void) {
    return seedcg::g_kernel_launches.load(std::memory_order_relaxed);
}

const char* seedcg_last_error(const seedcg_handle* h) {
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

void seedcg_destroy(seedcg_handle* h) {
    if (!h) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    h->u64.release();
    h->u32.release();
    h->vbasis.release();
    h->lz_scalars.release();
    h->red.release();
    h->work.release();
    h->coef.release();
    h->tcbuf.release();
    h->cgbuf.release();
    h->hostio.release();
    seedcg::guess_free(h);
    h->staging.release();
    if (h->pinned) cudaFreeHost(h->pinned);
    cudaSetDevice(prev);
    delete h;
}

}  // extern "C"
