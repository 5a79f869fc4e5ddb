// Improved Seed-CG on the device (paper, Section 2, Algorithm 1):
//   phase A  Lanczos for RHS 1 past convergence, with the LU of T (Eq. 2) kept
//            on the device, periodic re-orthogonalisation every k iterations,
//            and (literal mode) the per-iteration seed updates of steps 3-7;
//   phase S  (blocked mode) the Galerkin seeds of Eq. (1) from the stored V;
//   phase B  CG for every system whose FP64 true residual exceeds tol, all
//            systems batched through the multi-RHS dslash, with FP64
//            reliable updates in the mixed-precision modes.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstddef>
#include <cstring>
#include <vector>

#include "cg_batch.cuh"
#include "eo.cuh"
#include "handle.cuh"
#include "kernels.cuh"
#include "reduce.cuh"
#include "tc_proj.cuh"
#include "wilson.cuh"

#include <type_traits>

namespace seedcg {

namespace {

inline int red_blocks(long n) {
    long b = (n + kRedThreads * 4 - 1) / (kRedThreads * 4);
    if (b < 1) b = 1;
    return (int)std::min<long>(b, 152 * 8);
}

// blocks for a kernel whose thread handles one 16-byte group of entries (n / w
// groups), in equal rounds of at most kMaxRedBlocks blocks
inline int vec_blocks(long n, int w) {
    long b = (n / w + kRedThreads - 1) / kRedThreads;
    if (b < 1) b = 1;
    const long rounds = (b + kMaxRedBlocks - 1) / kMaxRedBlocks;
    return (int)((b + rounds - 1) / rounds);
}

inline int site_blocks(int vol) { return (vol + kRedThreads - 1) / kRedThreads; }

// The single-RHS operator kernels of the Lanczos loop (one thread per site) run in
// blocks of 128 with at most 72 registers in FP32: 7 blocks per SM then hold a
// 16^3x32 lattice in one wave, where 256-thread blocks at 77 registers need 1.12
// waves (16.4 -> 14.6 us for D with the L2 warm)
constexpr int kSiteThreads = 128;
inline int site_blocks_lz(int vol) { return (vol + kSiteThreads - 1) / kSiteThreads; }

// blocks for a streaming pass that ends in one grid reduction: two per SM.  Every
// block takes the reduction's atomic ticket, and thousands of tickets on one
// counter cost more than the pass's loads (the 16^3x32 Lanczos update: 23 us at
// 304 blocks against 35 us at 3072)
inline int lean_blocks(long n, int w) { return std::min(vec_blocks(n, w), 2 * 152); }

// ===========================================================================
// phase A kernels.  Every kernel of iteration i returns at once when i
// exceeds the current target m (uniformly for the whole grid), so the host
// may queue iterations ahead of its next poll.
// ===========================================================================

// Algorithm 1 step 9 bookkeeping after beta_i is final.
__device__ void lz_after_beta(const LzDev& L, int i) {
    LzCtl* c = L.ctl;
    const double b = L.beta[i - 1], a = L.alpha[i - 1];
    const double d = L.delta[i - 1], z = L.zeta[i - 1];
    if (!isfinite(b) || !isfinite(d) || !isfinite(a)) {
        c->status = SEEDCG_ERR_NAN;
        c->m = i;
        return;
    }
    const double est = b * fabs(z / d);
    if (c->m_conv == 0 && est <= c->tol * c->bnorm1) {
        c->m_conv = i;
        int m1 = i + c->extra_iters;
        int m2 = (int)ceil(c->past_factor * (double)i);
        int m = m1 > m2 ? m1 : m2;
        c->m = m < c->m_max ? m : c->m_max;
    }
    if (b <= 1e-14 * fabs(a)) {
        c->breakdown = 1;
        c->m = i;
    }
}

// alpha_i is final: the LU recurrence of T (Algorithm 1 steps 3 and 6, Eq. 2)
__device__ __forceinline__ void lz_alpha_fin(const LzDev& L, int i, double a) {
    L.alpha[i - 1] = a;
    if (i == 1) {
        L.delta[0] = a;
        L.zeta[0] = L.ctl->beta0;
    } else {
        const double bp = L.beta[i - 2];
        const double gm = bp / L.delta[i - 2];
        L.gamma[i - 2] = gm;
        L.delta[i - 1] = a - gm * bp;
        L.zeta[i - 1] = -gm * L.zeta[i - 2];
    }
    if (L.delta[i - 1] == 0.0) {
        L.ctl->status = SEEDCG_ERR_BREAKDOWN;
        L.ctl->m = i;
    }
}

// v_1 = r_0^1 / beta_0 (step 2); beta_0 already in ctl
template <typename R>
__global__ void k_lz_start(const cx_t<R>* __restrict__ r0, cx_t<R>* __restrict__ v, long n,
                           LzDev L) {
    const double inv = 1.0 / L.ctl->beta0;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
        cx_t<R> z = r0[e];
        v[e] = mk<R>((R)(z.x * inv), (R)(z.y * inv));
    }
}

// t = D v_i
template <typename R>
__global__ void __launch_bounds__(kSiteThreads, sizeof(R) == 4 ? 7 : 4)
k_lz_D(Geom g, const cx_t<R>* __restrict__ u, R kappa, const cx_t<R>* __restrict__ v,
       cx_t<R>* __restrict__ t, int i, LzDev L) {
    if (i > L.ctl->m) return;
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.vol) return;
    const int vol = g.vol;
    Nbr n = neighbours(g, s);
    Spinor<R> res;
    auto load = [&](int y, Spinor<R>& p) { load_spinor(v, vol, y, p); };
    auto fl = [&](int mu, int e) { return __ldg(u + (size_t)(mu * 9 + e) * vol + s); };
    auto bl = [&](int mu, int e) { return __ldg(u + (size_t)(mu * 9 + e) * vol + n.b[mu]); };
    wilson_site<0, R>(n, s, load, fl, bl, kappa, res);
    store_spinor(t, vol, s, res);
}

// Step 5 (and 2): f = D^dag t - beta_{i-1} v_{i-1}; alpha_i = Re v_i^dag f.
// Step 6 scalars (and 3): gamma_{i-1}, delta_i, zeta_i.
template <typename R>
__global__ void __launch_bounds__(kSiteThreads, sizeof(R) == 4 ? 7 : 4)
k_lz_Ddag(Geom g, const cx_t<R>* __restrict__ u, R kappa, const cx_t<R>* __restrict__ t,
          const cx_t<R>* __restrict__ v, const cx_t<R>* __restrict__ vprev,
          cx_t<R>* __restrict__ f, int i, LzDev L) {
    if (i > L.ctl->m) return;
    const int vol = g.vol;
    const R bprev = i > 1 ? (R)L.beta[i - 2] : R(0);
    double red[1] = {0.0};
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < vol) {
        Nbr n = neighbours(g, s);
        Spinor<R> res;
        auto load = [&](int y, Spinor<R>& p) { load_spinor(t, vol, y, p); };
        auto fl = [&](int mu, int e) { return __ldg(u + (size_t)(mu * 9 + e) * vol + s); };
        auto bl = [&](int mu, int e) { return __ldg(u + (size_t)(mu * 9 + e) * vol + n.b[mu]); };
        wilson_site<1, R>(n, s, load, fl, bl, kappa, res);
        R part = 0;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            cx_t<R> fv = res.c[k / 3][k % 3];
            const size_t ix = sidx(k, s, vol);
            cx_t<R> vv = v[ix];
            if (i > 1) {
                cx_t<R> pv = vprev[ix];
                fv.x -= bprev * pv.x;
                fv.y -= bprev * pv.y;
            }
            f[ix] = fv;
            part += vv.x * fv.x + vv.y * fv.y;
        }
        red[0] = (double)part;
    }
    grid_sum<1>(red, L.partials, L.counters + CTR_B, [&](double* tot) { lz_alpha_fin(L, i, tot[0]); });
}

// Even-odd system (Section 3): M = A^dag A on odd-site half vectors, A = 1 - kappa^2 H_oe H_eo,
// applied in four parity-restricted hops per Lanczos iteration:
//   STAGE 0  e = H_eo v                 (even sites)
//   STAGE 1  y = v - kappa^2 H_oe e     (A v)
//   STAGE 2  e = H^dag_eo y
//   STAGE 3  f = y - kappa^2 H^dag_oe e - beta_{i-1} v_{i-1};  alpha_i = Re v_i^dag f
//            (the hops of D^dag give A^dag = g5 A g5), with the LU finaliser of k_lz_Ddag.
template <typename R, int STAGE>
__global__ void __launch_bounds__(kRedThreads)
k_lz_eo(Geom g, const cx_t<R>* __restrict__ u, R kk, const cx_t<R>* __restrict__ other,
        const cx_t<R>* __restrict__ same, cx_t<R>* __restrict__ out, const cx_t<R>* __restrict__ v,
        const cx_t<R>* __restrict__ vprev, int i, LzDev L) {
    constexpr int DAG = STAGE >= 2 ? 1 : 0;
    constexpr int POUT = (STAGE & 1) ? 1 : 0;
    if (i > L.ctl->m) return;
    const int vh = g.vol / 2;
    const int hh = blockIdx.x * blockDim.x + threadIdx.x;
    double red[1] = {0.0};
    if (hh < vh) {
        Spinor<R> acc;
        eo_site_apply<R, DAG>(g, u, POUT, hh, other, POUT ? same : nullptr, R(1), POUT ? -kk : R(1), acc);
        if (STAGE < 3) {
            store_spinor(out, vh, hh, acc);
        } else {
            const R bprev = i > 1 ? (R)L.beta[i - 2] : R(0);
            R part = 0;
#pragma unroll
            for (int k = 0; k < 12; k++) {
                cx_t<R> fv = acc.c[k / 3][k % 3];
                const size_t ix = sidx(k, hh, vh);
                const cx_t<R> vv = v[ix];
                if (i > 1) {
                    const cx_t<R> pv = vprev[ix];
                    fv.x -= bprev * pv.x;
                    fv.y -= bprev * pv.y;
                }
                out[ix] = fv;
                part += vv.x * fv.x + vv.y * fv.y;
            }
            red[0] = (double)part;
        }
    }
    if (STAGE == 3)
        grid_sum<1>(red, L.partials, L.counters + CTR_B, [&](double* tot) { lz_alpha_fin(L, i, tot[0]); });
}

// Steps 4 and 7 (literal seeding): eta^j = v_i^dag r_0^j - gamma_{i-1} eta^j for
// j = j0 .. j0+NE-1 (r_0^j at r0 + (j-1) * n).
template <typename R, int NE>
__global__ void __launch_bounds__(kRedThreads)
k_lz_eta(const cx_t<R>* __restrict__ v, const cx_t<R>* __restrict__ r0, long n, int j0, int ne,
         int i, LzDev L, unsigned* ctr) {
    if (i > L.ctl->m) return;
    double red[2 * NE];
    R acc[2 * NE];
#pragma unroll
    for (int k = 0; k < 2 * NE; k++) acc[k] = 0;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
        cx_t<R> a = v[e];
#pragma unroll
        for (int q = 0; q < NE; q++) {
            if (q < ne) {
                cx_t<R> b = r0[(size_t)(j0 + q - 1) * n + e];
                acc[2 * q] += a.x * b.x + a.y * b.y;
                acc[2 * q + 1] += a.x * b.y - a.y * b.x;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 2 * NE; k++) red[k] = (double)acc[k];
    grid_sum<2 * NE>(red, L.partials, ctr, [&](double* tot) {
        const double gm = i > 1 ? L.gamma[i - 2] : 0.0;
        for (int q = 0; q < ne; q++) {
            double2 old = L.eta[j0 + q - 2];
            double2 nw;
            nw.x = tot[2 * q] - (i > 1 ? gm * old.x : 0.0);
            nw.y = tot[2 * q + 1] - (i > 1 ? gm * old.y : 0.0);
            L.eta[j0 + q - 2] = nw;
        }
    });
}

// Steps 5-7 vector part: f -= alpha_i v_i; beta_i = ||f|| (final unless PO
// follows).  LIT (the literal seeding of FP64 runs) also does, in R, steps 3 and
// 6-7: w_i = (v_i - beta_{i-1} w_{i-1}) / delta_i, x^1 += zeta_i w_i, x^j += eta^j w_i.
template <typename R, bool LIT>
__global__ void __launch_bounds__(kRedThreads)
k_lz_update(const cx_t<R>* __restrict__ v, cx_t<R>* __restrict__ f, cx_t<R>* __restrict__ w,
            cx_t<R>* __restrict__ X, int nrhs, long n, int i, int final_beta, LzDev L) {
    if (i > L.ctl->m) return;
    const R a = (R)L.alpha[i - 1];
    R dl = 0, bp = 0, zt = 0;
    if (LIT) {
        dl = (R)L.delta[i - 1];
        bp = i > 1 ? (R)L.beta[i - 2] : R(0);
        zt = (R)L.zeta[i - 1];
    }
    R part = 0;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
        cx_t<R> vv = v[e], fv = f[e];
        fv.x -= a * vv.x;
        fv.y -= a * vv.y;
        f[e] = fv;
        part += fv.x * fv.x + fv.y * fv.y;
        if (LIT) {
            cx_t<R> ww = i > 1 ? w[e] : mk<R>(0, 0);
            ww.x = (vv.x - bp * ww.x) / dl;
            ww.y = (vv.y - bp * ww.y) / dl;
            w[e] = ww;
            cx_t<R> x1 = X[e];
            x1.x += zt * ww.x;
            x1.y += zt * ww.y;
            X[e] = x1;
            for (int j = 1; j < nrhs; j++) {
                double2 et = L.eta[j - 1];
                cx_t<R> xj = X[(size_t)j * n + e];
                xj = cfma(mk<R>((R)et.x, (R)et.y), ww, xj);
                X[(size_t)j * n + e] = xj;
            }
        }
    }
    double red[1] = {(double)part};
    grid_sum<1>(red, L.partials, L.counters + CTR_D, [&](double* tot) {
        L.beta[i - 1] = sqrt(tot[0]);
        if (final_beta) lz_after_beta(L, i);
    });
}

// The blocked modes' pass with 16-byte accesses: a thread owns 16 / sizeof(cx_t<R>)
// consecutive complex entries (two in FP32, one in FP64; n is a multiple of 4).
// X1: also steps 3 and 6 for RHS 1, w_i = (v_i - beta_{i-1} w_{i-1}) / delta_i in R
// and x^1 += zeta_i w_i accumulated in FP64 (x1 = the FP64 solution of RHS 1; the
// systems j >= 2 take Eq. (1) after the run).  X1 = false: f -= alpha v and beta only.
template <typename R, bool X1>
__global__ void __launch_bounds__(kRedThreads)
k_lz_update_v(const cx_t<R>* __restrict__ v, cx_t<R>* __restrict__ f, cx_t<R>* __restrict__ w,
              double2* __restrict__ x1, long n, int i, int final_beta, LzDev L) {
    if (i > L.ctl->m) return;
    constexpr int W = 16 / (int)sizeof(cx_t<R>);
    const R a = (R)L.alpha[i - 1];
    R bp = 0, idl = 0;
    double zt = 0.0;
    if (X1) {
        bp = i > 1 ? (R)L.beta[i - 2] : R(0);
        idl = (R)(1.0 / L.delta[i - 1]);
        zt = L.zeta[i - 1];
    }
    R part = 0;
    const long ng = n / W;
    const long st = (long)gridDim.x * blockDim.x;
    // two 16-byte groups per thread and trip, every load of both issued before the
    // arithmetic: the grid is two blocks per SM, so each thread keeps more bytes in flight
    for (long g0 = blockIdx.x * (long)blockDim.x + threadIdx.x; g0 < ng; g0 += 2 * st) {
        const bool two = g0 + st < ng;
        cx_t<R> vv[2][W], fv[2][W], ww[2][W];
        double2 xv[2][W];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            if (h == 1 && !two) break;
            const long g = g0 + h * st;
            if (X1) {
                // the FP64 x^1 is the widest stream of the pass
#pragma unroll
                for (int k = 0; k < W; k++) xv[h][k] = __ldcs(x1 + g * W + k);
            }
            if constexpr (W == 2) {
                const float4 a4 = reinterpret_cast<const float4*>(v)[g];
                const float4 b4 = reinterpret_cast<const float4*>(f)[g];
                vv[h][0] = mk<R>(a4.x, a4.y); vv[h][1] = mk<R>(a4.z, a4.w);
                fv[h][0] = mk<R>(b4.x, b4.y); fv[h][1] = mk<R>(b4.z, b4.w);
                if (X1) {
                    const float4 c4 = i > 1 ? __ldcs(reinterpret_cast<const float4*>(w) + g) : make_float4(0, 0, 0, 0);
                    ww[h][0] = mk<R>(c4.x, c4.y); ww[h][1] = mk<R>(c4.z, c4.w);
                }
            } else {
                vv[h][0] = v[g];
                fv[h][0] = f[g];
                if (X1) ww[h][0] = i > 1 ? __ldcs(reinterpret_cast<const double2*>(w) + g) : mk<R>(0, 0);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            if (h == 1 && !two) break;
            const long g = g0 + h * st;
#pragma unroll
            for (int k = 0; k < W; k++) {
                fv[h][k].x -= a * vv[h][k].x;
                fv[h][k].y -= a * vv[h][k].y;
                part += fv[h][k].x * fv[h][k].x + fv[h][k].y * fv[h][k].y;
                if (X1) {
                    ww[h][k].x = (vv[h][k].x - bp * ww[h][k].x) * idl;
                    ww[h][k].y = (vv[h][k].y - bp * ww[h][k].y) * idl;
                }
            }
            // w and x^1 are streamed (evict-first): each is touched once per iteration, and
            // caching them would push the operator's links and vectors out of L2
            if constexpr (W == 2) {
                reinterpret_cast<float4*>(f)[g] = make_float4(fv[h][0].x, fv[h][0].y, fv[h][1].x, fv[h][1].y);
                if (X1) __stcs(reinterpret_cast<float4*>(w) + g, make_float4(ww[h][0].x, ww[h][0].y, ww[h][1].x, ww[h][1].y));
            } else {
                f[g] = fv[h][0];
                if (X1) __stcs(reinterpret_cast<double2*>(w) + g, make_double2(ww[h][0].x, ww[h][0].y));
            }
            if (X1) {
#pragma unroll
                for (int k = 0; k < W; k++) {
                    xv[h][k].x = fma(zt, (double)ww[h][k].x, xv[h][k].x);
                    xv[h][k].y = fma(zt, (double)ww[h][k].y, xv[h][k].y);
                    __stcs(x1 + g * W + k, xv[h][k]);
                }
            }
        }
    }
    double red[1] = {(double)part};
    grid_sum<1>(red, L.partials, L.counters + CTR_D, [&](double* tot) {
        L.beta[i - 1] = sqrt(tot[0]);
        if (final_beta) lz_after_beta(L, i);
    });
}

// ---- step 8: periodic re-orthogonalisation (classical Gram-Schmidt) ----
// [v, f] -= V_{1:i-1} c   with c = V^dag [v, f] already in coef (double2 [i-1][2]);
// the columns of coef follow the order of the two rows passed to gemm_t.

// av, af (W entries from e) += sum over rows [r0, r1) of V[a][e..] * c[a][0 / 1]:
// one 16-byte load per row and thread, coefficients of 256 rows at a time in
// shared memory.  Every thread of the block calls it (it synchronises);
// `live` marks threads that own entries.
template <typename R, typename VT>
__device__ __forceinline__ void po_accumulate(const VT* __restrict__ V, long ldv, int r0, int r1,
                                              const double2* __restrict__ coef, int cv, long e,
                                              bool live, cx_t<R> (&av)[VLoad<R, VT>::N],
                                              cx_t<R> (&af)[VLoad<R, VT>::N],
                                              cx_t<R> (*sc)[2]) {
    constexpr int W = VLoad<R, VT>::N;
    constexpr int CH = 256;
#pragma unroll
    for (int w = 0; w < W; w++) av[w] = af[w] = mk<R>(0, 0);
    for (int a0 = r0; a0 < r1; a0 += CH) {
        const int cnt = r1 - a0 < CH ? r1 - a0 : CH;
        __syncthreads();
        for (int k = threadIdx.x; k < 2 * CH; k += blockDim.x) {
            int a = k >> 1, c = k & 1;
            double2 z = a < cnt ? coef[(size_t)(a0 + a) * 2 + (c == 0 ? cv : 1 - cv)]
                                : make_double2(0.0, 0.0);
            sc[a][c] = mk<R>((R)z.x, (R)z.y);
        }
        __syncthreads();
        if (live) {
            const VT* col = V + (size_t)a0 * ldv + e;
#pragma unroll 8
            for (int a = 0; a < cnt; a++) {
                cx_t<R> x[W];
                VLoad<R, VT>::get(col + (size_t)a * ldv, x);
                const cx_t<R> c0 = sc[a][0], c1 = sc[a][1];
#pragma unroll
                for (int w = 0; w < W; w++) {
                    av[w] = cfma(x[w], c0, av[w]);
                    af[w] = cfma(x[w], c1, af[w]);
                }
            }
        }
    }
}

// after the subtraction: ||v_i|| decides whether the run goes on
__device__ __forceinline__ void po_check_nv(const LzDev& L, int i, double nv2) {
    const double nv = sqrt(nv2);
    L.ctl->nv = nv;
    // v_i is a unit vector; if the projection removed most of it the basis no
    // longer spans what the recurrence assumes (numerical invariant subspace or
    // a basis stored too coarsely): end the run at i - 1, before this vector.
    // Without the guard only a vanished (or non-finite) v_i ends it.
    if (L.ctl->guard ? !(nv >= 0.5) : !(nv > 0.0 && isfinite(nv))) {
        L.ctl->breakdown = 2;
        L.ctl->m = i - 1;
    }
}

// the whole subtraction in one pass: thread = W consecutive entries down all rows
// (n is a multiple of W, host-checked)
template <typename R, typename VT>
__global__ void __launch_bounds__(kRedThreads)
k_po_sub(const VT* __restrict__ V, long ldv, int na, const double2* __restrict__ coef, int cv,
         cx_t<R>* __restrict__ v, cx_t<R>* __restrict__ f, long n, int i, LzDev L) {
    if (i > L.ctl->m) return;
    constexpr int W = VLoad<R, VT>::N;
    __shared__ cx_t<R> sc[256][2];
    R part = 0;
    const long ng = n / W;
    for (long g0 = blockIdx.x * (long)blockDim.x; g0 < ng; g0 += (long)gridDim.x * blockDim.x) {
        const long g = g0 + threadIdx.x;
        const long e = g * W;
        cx_t<R> av[W], af[W];
        po_accumulate<R, VT>(V, ldv, 0, na, coef, cv, e, g < ng, av, af, sc);
        if (g < ng) {
#pragma unroll
            for (int w = 0; w < W; w++) {
                const cx_t<R> vv = csub(v[e + w], av[w]);
                v[e + w] = vv;
                f[e + w] = csub(f[e + w], af[w]);
                part += vv.x * vv.x + vv.y * vv.y;
            }
        }
    }
    double red[1] = {(double)part};
    grid_sum<1>(red, L.partials, L.counters + CTR_PO2, [&](double* tot) { po_check_nv(L, i, tot[0]); });
}

// the subtraction split over row segments (blockIdx.y = segment of `seg` rows)
// so that long bases fill the GPU in many even waves: segment s writes its sums
// to part[s][0 / 1][n]; k_po_sub_fin adds the segments in a fixed order.
template <typename R, typename VT>
__global__ void __launch_bounds__(kRedThreads)
k_po_sub_seg(const VT* __restrict__ V, long ldv, int na, int seg, const double2* __restrict__ coef,
             int cv, long n, cx_t<R>* __restrict__ part, int i, LzDev L) {
    if (i > L.ctl->m) return;
    constexpr int W = VLoad<R, VT>::N;
    __shared__ cx_t<R> sc[256][2];
    const long g = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const bool live = g < n / W;
    const long e = g * W;
    const int r0 = blockIdx.y * seg, r1 = r0 + seg < na ? r0 + seg : na;
    cx_t<R> av[W], af[W];
    po_accumulate<R, VT>(V, ldv, r0, r1, coef, cv, e, live, av, af, sc);
    if (live) {
        cx_t<R>* pv = part + (size_t)blockIdx.y * 2 * n + e;
#pragma unroll
        for (int w = 0; w < W; w++) {
            pv[w] = av[w];
            pv[n + w] = af[w];
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(kRedThreads)
k_po_sub_fin(const cx_t<R>* __restrict__ part, int nseg, cx_t<R>* __restrict__ v,
             cx_t<R>* __restrict__ f, long n, int i, LzDev L) {
    if (i > L.ctl->m) return;
    R acc = 0;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
        cx_t<R> sv = part[e], sf = part[n + e];
        for (int s = 1; s < nseg; s++) {
            sv = cadd(sv, part[(size_t)s * 2 * n + e]);
            sf = cadd(sf, part[(size_t)s * 2 * n + n + e]);
        }
        const cx_t<R> vv = csub(v[e], sv);
        v[e] = vv;
        f[e] = csub(f[e], sf);
        acc += vv.x * vv.x + vv.y * vv.y;
    }
    double red[1] = {(double)acc};
    grid_sum<1>(red, L.partials, L.counters + CTR_PO2, [&](double* tot) { po_check_nv(L, i, tot[0]); });
}

// v_i /= ||v_i||; dvf = v_i^dag f
template <typename R>
__global__ void __launch_bounds__(kRedThreads)
k_po_normalise(cx_t<R>* __restrict__ v, const cx_t<R>* __restrict__ f, long n, int i, LzDev L) {
    if (i > L.ctl->m) return;
    const R inv = (R)(1.0 / L.ctl->nv);
    R pr = 0, pi = 0;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
        cx_t<R> vv = cscale(v[e], inv);
        v[e] = vv;
        cx_t<R> fv = f[e];
        pr += vv.x * fv.x + vv.y * fv.y;
        pi += vv.x * fv.y - vv.y * fv.x;
    }
    double red[2] = {(double)pr, (double)pi};
    grid_sum<2>(red, L.partials, L.counters + CTR_PO3,
                [&](double* tot) { L.ctl->dvf = make_double2(tot[0], tot[1]); });
}

// f -= (v_i^dag f) v_i; beta_i = ||f||; step 9 bookkeeping
template <typename R>
__global__ void __launch_bounds__(kRedThreads)
k_po_finish(const cx_t<R>* __restrict__ v, cx_t<R>* __restrict__ f, long n, int i, LzDev L) {
    if (i > L.ctl->m) return;
    const double2 d = L.ctl->dvf;
    const cx_t<R> dc = mk<R>((R)d.x, (R)d.y);
    R part = 0;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
        cx_t<R> fv = csub(f[e], cmul(dc, v[e]));
        f[e] = fv;
        part += fv.x * fv.x + fv.y * fv.y;
    }
    double red[1] = {(double)part};
    grid_sum<1>(red, L.partials, L.counters + CTR_PO4, [&](double* tot) {
        const double bnew = sqrt(tot[0]);
        L.ctl->po_count += 1;
        // an orthogonal projection never lengthens f; growth means the stored
        // basis is far from orthonormal: end the run at i - 1
        if (L.ctl->guard ? !(bnew <= 1.01 * L.beta[i - 1]) : !isfinite(bnew)) {
            L.ctl->breakdown = 3;
            L.ctl->m = i - 1;
            return;
        }
        L.beta[i - 1] = bnew;
        lz_after_beta(L, i);
    });
}

// Step 9: store v_i into V (storage type VT); v_{i+1} = f / beta_i
// (FP32: a thread moves two complex entries, 16-byte loads of v and f)
template <typename R, typename VT>
__global__ void k_lz_advance(const cx_t<R>* __restrict__ v, const cx_t<R>* __restrict__ f,
                             cx_t<R>* __restrict__ vnext, VT* __restrict__ Vrow, long n, int i,
                             LzDev L) {
    if (i > L.ctl->m) return;
    const double b = L.beta[i - 1];
    const bool go = b > 0.0 && i < L.ctl->m;
    const R inv = go ? (R)(1.0 / b) : R(0);
    if constexpr (sizeof(R) == 4) {
        const long ng = n / 2;   // n = 12 * sites is even
        for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < ng;
             g += (long)gridDim.x * blockDim.x) {
            const float4 a = reinterpret_cast<const float4*>(v)[g];
            float4 c;
            if (go) c = reinterpret_cast<const float4*>(f)[g];
            st_cx(Vrow, 2 * g, make_float2(a.x, a.y));
            st_cx(Vrow, 2 * g + 1, make_float2(a.z, a.w));
            if (go) reinterpret_cast<float4*>(vnext)[g] = make_float4(c.x * inv, c.y * inv, c.z * inv, c.w * inv);
        }
    } else {
        for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
             e += (long)gridDim.x * blockDim.x) {
            cx_t<R> vv = v[e];
            st_cx(Vrow, e, vv);
            if (go) vnext[e] = cscale(f[e], inv);
        }
    }
}

// ||x||^2 of one flat vector into *out (FP64)
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
k_norm2(const T* __restrict__ x, long n, double* partials, unsigned* ctr, double* out) {
    double p = 0.0;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
        cx_t<double> z = ld_cx<double>(x, e);
        p += z.x * z.x + z.y * z.y;
    }
    double red[1] = {p};
    grid_sum<1>(red, partials, ctr, [&](double* tot) { *out = sqrt(tot[0]); });
}

// ===========================================================================
// phase S: Z = L^{-1} C, Y = U^{-1} Z column by column (Eq. 2 factors), in place
// on C [m][ldc] double2.  One thread per right-hand side.
// ===========================================================================
// The two triangular solves are sequential in i; a block takes 32 right-hand sides
// and walks the rows in chunks of SEED_CH: all threads stage a chunk of C and of the
// scalars in shared memory (coalesced), one warp runs the recurrences on it (lane =
// right-hand side), all threads write the chunk back.  Each step then waits on
// shared memory instead of a global load.
constexpr int SEED_CH = 64;
__global__ void __launch_bounds__(256) k_seed_tridiag(double2* C, int ldc, int nrhs, int m, LzDev L) {
    __shared__ double2 sc[SEED_CH][33];       // [row][rhs], padded against bank conflicts
    __shared__ double sg[SEED_CH], sd[SEED_CH], sb[SEED_CH];   // gamma_{i-1}, 1 / delta_i, beta_i
    const int j0 = blockIdx.x * 32;
    const int nj = nrhs - j0 < 32 ? nrhs - j0 : 32;
    if (nj <= 0 || m <= 0) return;
    const int lane = threadIdx.x & 31;
    const bool runner = threadIdx.x < 32 && lane < nj;
    auto load_chunk = [&](int i0, int cnt) {
        for (int k = threadIdx.x; k < cnt * 32; k += blockDim.x) {
            const int r = k / 32, c = k % 32;
            if (c < nj) sc[r][c] = C[(size_t)(i0 + r) * ldc + j0 + c];
        }
        for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
            const int i = i0 + r + 1;                  // 1-based row
            sg[r] = i >= 2 ? L.gamma[i - 2] : 0.0;     // gamma_{i-1}
            sd[r] = 1.0 / L.delta[i - 1];              // the chain then multiplies
            sb[r] = i <= m - 1 ? L.beta[i - 1] : 0.0;  // beta_i couples rows i and i+1
        }
    };
    auto store_chunk = [&](int i0, int cnt) {
        for (int k = threadIdx.x; k < cnt * 32; k += blockDim.x) {
            const int r = k / 32, c = k % 32;
            if (c < nj) C[(size_t)(i0 + r) * ldc + j0 + c] = sc[r][c];
        }
    };
    // forward: eta_1 = c_1, eta_i = c_i - gamma_{i-1} eta_{i-1}
    double2 prev = make_double2(0.0, 0.0);
    for (int i0 = 0; i0 < m; i0 += SEED_CH) {
        const int cnt = m - i0 < SEED_CH ? m - i0 : SEED_CH;
        __syncthreads();
        load_chunk(i0, cnt);
        __syncthreads();
        if (runner) {
            for (int r = 0; r < cnt; r++) {
                double2 c = sc[r][lane];
                if (i0 + r > 0) {
                    c.x -= sg[r] * prev.x;
                    c.y -= sg[r] * prev.y;
                }
                sc[r][lane] = c;
                prev = c;
            }
        }
        __syncthreads();
        store_chunk(i0, cnt);
    }
    // back substitution with U (delta on the diagonal, beta above it):
    // y_m = z_m / delta_m, y_i = (z_i - beta_i y_{i+1}) / delta_i
    double2 y = make_double2(0.0, 0.0);
    for (int iend = m; iend > 0; iend -= SEED_CH) {
        const int i0 = iend - SEED_CH > 0 ? iend - SEED_CH : 0;
        const int cnt = iend - i0;
        __syncthreads();
        load_chunk(i0, cnt);
        __syncthreads();
        if (runner) {
            for (int r = cnt - 1; r >= 0; r--) {
                double2 z = sc[r][lane];
                if (i0 + r < m - 1) {
                    z.x -= sb[r] * y.x;
                    z.y -= sb[r] * y.y;
                }
                z.x *= sd[r];
                z.y *= sd[r];
                sc[r][lane] = z;
                y = z;
            }
        }
        __syncthreads();
        store_chunk(i0, cnt);
    }
}

// M x for n FP64 fields in internal layout (D then D^dag) via the multi-RHS kernel
inline void apply_M64(seedcg_handle* h, int n, const double2* x, double2* tmp, double2* out,
                      cudaStream_t st) {
    dslash_mrhs_f64(h->g, h->u64.as<double2>(), h->kappa, 0, n, x, tmp, st);
    dslash_mrhs_f64(h->g, h->u64.as<double2>(), h->kappa, 1, n, tmp, out, st);
}

// bump allocator over one device buffer
struct Carve {
    char* base;
    size_t off = 0, cap;
    template <typename T> T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = reinterpret_cast<T*>(base + off);
        off += count * sizeof(T);
        if (off > cap) throw Error{SEEDCG_ERR_OOM, "workspace carve overflow"};
        return p;
    }
};

struct PhaseTimer {
    cudaEvent_t a = nullptr, b = nullptr;
    float ms = 0.f;
    void start(cudaStream_t s) {
        if (!a) { cudaEventCreate(&a); cudaEventCreate(&b); }
        cudaEventRecord(a, s);
    }
    void stop(cudaStream_t s) { cudaEventRecord(b, s); }
    float read() {
        if (!a) return 0.f;
        cudaEventSynchronize(b);
        float t = 0.f;
        cudaEventElapsedTime(&t, a, b);
        return t;
    }
    ~PhaseTimer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};


// r0 = b - mx (mx may be null), narrowed to R
template <typename R>
__global__ void k_resid_init(const double2* __restrict__ b, const double2* __restrict__ mx,
                             cx_t<R>* __restrict__ r0, long n) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
        double2 z = b[e];
        if (mx) {
            double2 w = mx[e];
            z.x -= w.x;
            z.y -= w.y;
        }
        r0[e] = mk<R>((R)z.x, (R)z.y);
    }
}

// ===========================================================================
// host driver, templated on working precision R and basis storage VT
// ===========================================================================
template <typename R, typename VT>
seedcg_status run_solve(seedcg_handle* h, int nrhs, const double2* B64, double2* X64,
                        double tol, int extra_iters, int k_po, seedcg_info* info,
                        cudaStream_t st, bool run_cg = true) {
    const seedcg_options& o = h->opt;
    const int vol = h->g.vol;
    // the even-odd system (Section 3) works on odd-site half vectors
    const bool eo = h->eo_active;
    const long n = 12L * (eo ? vol / 2 : vol);
    const bool fp64 = sizeof(R) == 8;
    const bool literal = (o.seed_mode == 0) && fp64;
    const int m_max = std::max(o.m_max, 1);
    const int poll = o.poll_every > 0 ? o.poll_every : 32;
    const R kap = (R)h->kappa;
    const cx_t<R>* U = fp64 ? reinterpret_cast<const cx_t<R>*>(h->u64.p)
                            : reinterpret_cast<const cx_t<R>*>(h->u32.p);

    // ---------------- workspaces ----------------
    const size_t cxR = sizeof(cx_t<R>);
    size_t need = 0;
    auto add = [&](size_t bytes) { need += ((bytes + 255) & ~(size_t)255); };
    for (int k = 0; k < 6; k++) add(n * cxR);                   // vA f vB t w e
    for (int k = 0; k < 6; k++) add((size_t)nrhs * n * cxR);    // R0 XR Rr P Q T
    for (int k = 0; k < 2; k++) add((size_t)nrhs * n * sizeof(double2));  // G MX
    add((size_t)std::max(nrhs, 2) * n * sizeof(double2));                 // T64
    h->work.ensure(need + 8192);
    Carve cv{h->work.as<char>(), 0, h->work.bytes};
    cx_t<R>* vA = cv.take<cx_t<R>>(n);
    cx_t<R>* fv = cv.take<cx_t<R>>(n);
    cx_t<R>* vB = cv.take<cx_t<R>>(n);
    cx_t<R>* tv = cv.take<cx_t<R>>(n);
    cx_t<R>* wv = cv.take<cx_t<R>>(n);
    cx_t<R>* ev = cv.take<cx_t<R>>(n);   // even-site intermediate of the even-odd operator
    cx_t<R>* R0 = cv.take<cx_t<R>>((size_t)nrhs * n);
    cx_t<R>* XR = cv.take<cx_t<R>>((size_t)nrhs * n);
    cx_t<R>* Rr = cv.take<cx_t<R>>((size_t)nrhs * n);
    cx_t<R>* Pv = cv.take<cx_t<R>>((size_t)nrhs * n);
    cx_t<R>* Qv = cv.take<cx_t<R>>((size_t)nrhs * n);
    cx_t<R>* Tv = cv.take<cx_t<R>>((size_t)nrhs * n);
    double2* G = cv.take<double2>((size_t)nrhs * n);
    double2* MX = cv.take<double2>((size_t)nrhs * n);
    double2* T64 = cv.take<double2>((size_t)std::max(nrhs, 2) * n);
    if (fv != vA + n || vB != fv + n)
        throw Error{SEEDCG_ERR_ARG, "internal: working vectors are not contiguous"};

    // Lanczos scalars
    const size_t ms = (size_t)m_max + 2;
    h->lz_scalars.ensure(sizeof(LzCtl) + 5 * sizeof(double) * ms + sizeof(double2) * (nrhs + 2) +
                         sizeof(double) * 8 * (nrhs + 2) + sizeof(int) * 8 * (nrhs + 2) + 8192);
    SEEDCG_CUDA_TRY(cudaMemsetAsync(h->lz_scalars.p, 0, h->lz_scalars.bytes, st));
    Carve cs{h->lz_scalars.as<char>(), 0, h->lz_scalars.bytes};
    LzDev L;
    L.ctl = cs.take<LzCtl>(1);
    L.alpha = cs.take<double>(ms);
    L.beta = cs.take<double>(ms);
    L.delta = cs.take<double>(ms);
    L.gamma = cs.take<double>(ms);
    L.zeta = cs.take<double>(ms);
    L.eta = cs.take<double2>(nrhs + 2);
    double* bnorm = cs.take<double>(nrhs + 2);
    double* tr_dev = cs.take<double>(nrhs + 2);
    const int rb = red_blocks(n);
    const size_t part_doubles = (size_t)std::max(kMaxRedBlocks, rb * (nrhs + 2)) * 64;
    h->red.ensure(part_doubles * sizeof(double) + 8192 * sizeof(unsigned));
    L.partials = h->red.as<double>();
    L.counters = reinterpret_cast<unsigned*>(h->red.as<double>() + part_doubles);
    SEEDCG_CUDA_TRY(cudaMemsetAsync(L.counters, 0, 8192 * sizeof(unsigned), st));
    // V basis and coefficient scratch
    const size_t vrow = (size_t)n * sizeof(VT);
    if (h->vbasis.bytes < vrow * (size_t)m_max) {
        // refuse a basis that cannot fit before allocating it (m_max rows of one vector each)
        size_t free_b = 0, total_b = 0;
        SEEDCG_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
        if (vrow * (size_t)m_max > free_b + h->vbasis.bytes) {
            char msg[256];
            snprintf(msg, sizeof(msg),
                     "the stored basis needs m_max x %zu B = %.1f GB of device memory, %.1f GB is free; "
                     "lower m_max or choose a narrower basis precision",
                     vrow, 1e-9 * (double)(vrow * (size_t)m_max), 1e-9 * (double)(free_b + h->vbasis.bytes));
            throw Error{SEEDCG_ERR_OOM, msg};
        }
    }
    h->vbasis.ensure(vrow * (size_t)m_max);
    VT* Vb = h->vbasis.as<VT>();
    h->vbasis_prec = o.precision;
    h->vbasis_eo = eo;
    h->vbasis_m = 0;
    const size_t cols = (size_t)std::max(nrhs, 2);
    const size_t coef_elems = ms * cols;
    const bool seeds_streamed = !fp64 && !(std::is_same<VT, __nv_bfloat162>::value && o.use_tensor_cores);
    // also room for three row segments of the PO subtraction (k_po_sub_seg partials)
    const size_t seg3 = 3 * 2 * (size_t)n * sizeof(cx_t<R>) / sizeof(double2);
    const size_t split_elems = std::max<size_t>(
        std::max<size_t>(std::max<size_t>(coef_elems * 48, (size_t)1 << 20), seg3),
        seeds_streamed ? proj_scratch_elems<R, VT>(n, m_max) : proj_scratch_elems<R, VT>(n, m_max) / 2);
    h->coef.ensure((coef_elems + split_elems) * sizeof(double2));
    double2* Cc = h->coef.as<double2>();
    double2* split = Cc + coef_elems;

    // pinned host scratch: [0,256) slot lists / flags, [256,512) system lists,
    // [512,1024) active flags, [1024] a zero, doubles from int 2048 on
    // tensor-core projections for the bf16 basis
    constexpr bool kBf16 = std::is_same<VT, __nv_bfloat162>::value;
    const bool use_tc = kBf16 && o.use_tensor_cores;
    __nv_bfloat162* Bm = nullptr;
    float* tpart = nullptr;
    const size_t tpart_elems = (size_t)4 << 20;
    if (use_tc) {
        const size_t bb = tc_b_bytes(n, std::min(std::max(nrhs, 2), 32));
        const size_t need_tc = ((bb + 1023) & ~(size_t)1023) + tpart_elems * sizeof(float);
        if (h->tcbuf.bytes < need_tc) {
            h->tcbuf.ensure(need_tc);
            SEEDCG_CUDA_TRY(cudaMemsetAsync(h->tcbuf.p, 0, need_tc, st));
        }
        Bm = h->tcbuf.as<__nv_bfloat162>();
        tpart = reinterpret_cast<float*>(h->tcbuf.as<char>() + ((bb + 1023) & ~(size_t)1023));
    }
    auto project = [&](int rows, const cx_t<R>* X, int nvec, int ldc) {
        if constexpr (kBf16) {
            if (use_tc && nvec <= 32 && (nvec > 2 || o.use_tensor_cores == 2)) {
                tc_project(Vb, m_max, rows, reinterpret_cast<const float2*>(X), n, nvec, n, Bm, tpart,
                           tpart_elems, Cc, ldc, &L.ctl->status, st);
                return;
            }
        }
        if (nvec <= 2 || seeds_streamed)
            proj<R, VT>(Vb, n, rows, X, n, nvec, n, Cc, ldc, split, split_elems, st);
        else
            gemm_t<R, VT>(Vb, n, rows, X, n, nvec, n, Cc, ldc, split, split_elems, st);
    };

    // [v, f] -= V c: one pass down all rows, or (long bases) row segments so
    // that the grid is many even waves, summed by k_po_sub_fin
    int nsm = 0;
    SEEDCG_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    static int seg_occ = 0;
    if (!seg_occ)
        SEEDCG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&seg_occ, k_po_sub_seg<R, VT>,
                                                                      kRedThreads, 0));
    constexpr int kW = 16 / (int)sizeof(VT);
    if (n % 4 != 0) throw Error{SEEDCG_ERR_ARG, "spinor length not a multiple of 4"};
    const long po_gb = (n / kW + kRedThreads - 1) / kRedThreads;
    const long seg_cap = (long)(split_elems * sizeof(double2) / (2 * (size_t)n * sizeof(cx_t<R>)));
    auto po_subtract = [&](int na, int cvcol, cx_t<R>* vv, cx_t<R>* ff, int i) {
        long nseg = 1;
        if (na >= 256) {
            const long resident = (long)nsm * std::max(seg_occ, 1);
            nseg = std::min<long>({8, (6 * resident + po_gb - 1) / po_gb, na / 128, seg_cap});
        }
        if (nseg <= 1) {
            k_po_sub<R, VT><<<vec_blocks(n, kW), kRedThreads, 0, st>>>(Vb, n, na, Cc, cvcol, vv, ff, n,
                                                                       i, L);
            SEEDCG_CHECK_LAUNCH();
            return;
        }
        const int seg = (int)((na + nseg - 1) / nseg);
        const int ns = (na + seg - 1) / seg;
        cx_t<R>* sp = reinterpret_cast<cx_t<R>*>(split);
        k_po_sub_seg<R, VT><<<dim3((unsigned)po_gb, ns), kRedThreads, 0, st>>>(Vb, n, na, seg, Cc, cvcol,
                                                                              n, sp, i, L);
        SEEDCG_CHECK_LAUNCH();
        k_po_sub_fin<R><<<rb, kRedThreads, 0, st>>>(sp, ns, vv, ff, n, i, L);
        SEEDCG_CHECK_LAUNCH();
    };

    int* pin = reinterpret_cast<int*>(h->pinned);
    double* pind = reinterpret_cast<double*>(pin + 2048);
    pin[1024] = 0;

    PhaseTimer t_all, t_lz, t_seed, t_cg;
    t_all.start(st);

    // ---------------- step 1: r_0^j = b^j - M x_0^j ----------------
    const int nbl = std::min<long>((n * nrhs + 255) / 256, 152 * 32);
    if (o.x0_given || h->force_x0) {
        if (eo)
            eo_apply_mdag_m_f64(h->g, h->u64.as<double2>(), h->kappa, nrhs, X64, T64, T64 + n, MX, st);
        else
            apply_M64(h, nrhs, X64, T64, MX, st);
        k_resid_init<R><<<nbl, 256, 0, st>>>(B64, MX, R0, n * nrhs);
    } else {
        k_resid_init<R><<<nbl, 256, 0, st>>>(B64, nullptr, R0, n * nrhs);
    }
    SEEDCG_CHECK_LAUNCH();
    for (int j = 0; j < nrhs; j++) {
        k_norm2<double2><<<rb, kRedThreads, 0, st>>>(B64 + (size_t)j * n, n, L.partials,
                                                     L.counters + CTR_NORM, bnorm + j);
        SEEDCG_CHECK_LAUNCH();
    }
    k_norm2<cx_t<R>><<<rb, kRedThreads, 0, st>>>(R0, n, L.partials, L.counters + CTR_NORM,
                                                  &L.ctl->beta0);
    SEEDCG_CHECK_LAUNCH();
    {
        LzCtl hc;
        memset(&hc, 0, sizeof(hc));
        hc.m = m_max;
        hc.m_max = m_max;
        hc.extra_iters = extra_iters;
        hc.tol = tol;
        hc.past_factor = o.past_factor;
        hc.guard = o.po_guard ? 1 : 0;
        // copy everything but beta0 / bnorm1 (set on the device)
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(L.ctl, &hc, offsetof(LzCtl, beta0), cudaMemcpyHostToDevice, st));
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(&L.ctl->tol, &hc.tol, sizeof(double) * 2, cudaMemcpyHostToDevice, st));
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(&L.ctl->bnorm1, bnorm, sizeof(double), cudaMemcpyDeviceToDevice, st));
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(pind, &L.ctl->beta0, sizeof(double), cudaMemcpyDeviceToHost, st));
        SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
    }
    const double beta0 = pind[0];

    // ---------------- phase A: Lanczos for RHS 1 ----------------
    t_lz.start(st);
    float ms_po = 0.f;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> po_ev;
    int m = 0, m_conv = 0, po_count = 0, lz_status = SEEDCG_OK, breakdown = 0;
    if (beta0 > 0.0) {
        const int sb = site_blocks(vol);
        k_lz_start<R><<<rb, kRedThreads, 0, st>>>(R0, vA, n, L);
        SEEDCG_CHECK_LAUNCH();
        cx_t<R>* v = vA;
        cx_t<R>* vprev = vB;
        int i = 1;
        const int sbh = site_blocks(vol / 2);
        const R kk = (R)(h->kappa * h->kappa);
        for (; i <= m_max; i++) {
            if (eo) {
                // f = A^dag A v - beta v_prev, alpha: four half-lattice hops
                k_lz_eo<R, 0><<<sbh, kRedThreads, 0, st>>>(h->g, U, kk, v, nullptr, ev, nullptr, nullptr, i, L);
                SEEDCG_CHECK_LAUNCH();
                k_lz_eo<R, 1><<<sbh, kRedThreads, 0, st>>>(h->g, U, kk, ev, v, tv, nullptr, nullptr, i, L);
                SEEDCG_CHECK_LAUNCH();
                k_lz_eo<R, 2><<<sbh, kRedThreads, 0, st>>>(h->g, U, kk, tv, nullptr, ev, nullptr, nullptr, i, L);
                SEEDCG_CHECK_LAUNCH();
                k_lz_eo<R, 3><<<sbh, kRedThreads, 0, st>>>(h->g, U, kk, ev, tv, fv, v, vprev, i, L);
                SEEDCG_CHECK_LAUNCH();
            } else {
                k_lz_D<R><<<site_blocks_lz(vol), kSiteThreads, 0, st>>>(h->g, U, kap, v, tv, i, L);
                SEEDCG_CHECK_LAUNCH();
                k_lz_Ddag<R><<<site_blocks_lz(vol), kSiteThreads, 0, st>>>(h->g, U, kap, tv, v, vprev, fv, i, L);
                SEEDCG_CHECK_LAUNCH();
            }
            if (literal) {
                for (int j0 = 2; j0 <= nrhs; j0 += 8) {
                    int ne = std::min(8, nrhs - j0 + 1);
                    k_lz_eta<R, 8><<<rb, kRedThreads, 0, st>>>(v, R0, n, j0, ne, i, L,
                                                                 L.counters + CTR_ETA0 + j0);
                    SEEDCG_CHECK_LAUNCH();
                }
            }
            const bool po_now = k_po > 0 && i >= 2 && (i % k_po) == 0;
            if (literal)
                k_lz_update<R, true><<<rb, kRedThreads, 0, st>>>(
                    v, fv, wv, reinterpret_cast<cx_t<R>*>(X64), nrhs, n, i, po_now ? 0 : 1, L);
            else
                k_lz_update_v<R, true><<<lean_blocks(n, 16 / (int)sizeof(cx_t<R>)), kRedThreads, 0, st>>>(
                    v, fv, wv, X64, n, i, po_now ? 0 : 1, L);
            SEEDCG_CHECK_LAUNCH();
            if (po_now) {
                cudaEvent_t e0, e1;
                cudaEventCreate(&e0);
                cudaEventCreate(&e1);
                cudaEventRecord(e0, st);
                const int na = i - 1;
                const cx_t<R>* Bst = (v == vA) ? vA : fv;  // rows [v, f] or [f, v]
                const int cvcol = (v == vA) ? 0 : 1;
                for (int pass = 0; pass < std::max(o.po_passes, 1); pass++) {
                    project(na, Bst, 2, 2);
                    po_subtract(na, cvcol, v, fv, i);
                }
                k_po_normalise<R><<<rb, kRedThreads, 0, st>>>(v, fv, n, i, L);
                SEEDCG_CHECK_LAUNCH();
                k_po_finish<R><<<rb, kRedThreads, 0, st>>>(v, fv, n, i, L);
                SEEDCG_CHECK_LAUNCH();
                cudaEventRecord(e1, st);
                po_ev.push_back({e0, e1});
            }
            k_lz_advance<R, VT><<<rb, kRedThreads, 0, st>>>(v, fv, vprev, Vb + (size_t)(i - 1) * n, n,
                                                           i, L);
            SEEDCG_CHECK_LAUNCH();
            std::swap(v, vprev);
            if (i % poll == 0 || i == m_max) {
                SEEDCG_CUDA_TRY(cudaMemcpyAsync(pin, L.ctl, sizeof(int) * 8, cudaMemcpyDeviceToHost, st));
                SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
                if (i >= pin[0] || pin[2] != 0) break;
            }
        }
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(pin, L.ctl, sizeof(int) * 8, cudaMemcpyDeviceToHost, st));
        SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
        m = std::min(pin[0], m_max);
        m_conv = pin[1];
        lz_status = pin[2];
        breakdown = pin[3];
        po_count = pin[4];
        for (auto& pe : po_ev) {
            float t = 0.f;
            cudaEventElapsedTime(&t, pe.first, pe.second);
            ms_po += t;
            cudaEventDestroy(pe.first);
            cudaEventDestroy(pe.second);
        }
        // keep the scalars of T for seedcg_get_lanczos
        h->alpha.assign(m, 0.0);
        h->beta.assign(m, 0.0);
        h->delta.assign(m, 0.0);
        if (m > 0) {
            SEEDCG_CUDA_TRY(cudaMemcpy(h->alpha.data(), L.alpha, sizeof(double) * m, cudaMemcpyDeviceToHost));
            SEEDCG_CUDA_TRY(cudaMemcpy(h->beta.data(), L.beta, sizeof(double) * m, cudaMemcpyDeviceToHost));
            SEEDCG_CUDA_TRY(cudaMemcpy(h->delta.data(), L.delta, sizeof(double) * m, cudaMemcpyDeviceToHost));
        }
    }
    h->last_m = m;
    h->vbasis_m = m;
    t_lz.stop(st);
    (void)breakdown;

    // ---------------- phase S: Galerkin seeds, Eq. (1) ----------------
    t_seed.start(st);
    // x^1 already holds steps 3 and 6 (the LU recurrence); Eq. (1) seeds j >= 2
    const int ns = nrhs - 1;
    if (!literal && m > 0 && ns > 0) {
        project(m, R0 + n, ns, ns);
        k_seed_tridiag<<<(ns + 31) / 32, 256, 0, st>>>(Cc, ns, ns, m, L);
        SEEDCG_CHECK_LAUNCH();
        gemm_n<R, VT, double2>(Vb, n, m, Cc, ns, ns, X64 + n, n, n, 1.0, st);
    }
    t_seed.stop(st);

    // ---------------- phase B: batched CG ----------------
    t_cg.start(st);
    CgResult cgr;
    const bool cg_now = run_cg && !o.stop_after_seed;
    if (cg_now) {
        std::vector<CgGroup> gs{{h, nrhs, B64, X64}};
        batched_cg<R>(gs, tol, fp64 ? 0.0 : o.reliable_delta, o.cg_maxiter, poll, true, h->cgbuf,
                      h->pinned, cgr, st);
    }
    t_cg.stop(st);
    t_all.stop(st);
    h->last_m_conv = m_conv;
    h->last_po_count = po_count;
    h->last_lz_status = lz_status;
    h->last_ms_lanczos = t_lz.read();
    h->last_ms_po = ms_po;
    h->last_ms_seed = t_seed.read();

    // ---------------- results ----------------
    seedcg_status code = SEEDCG_OK;
    if (lz_status == SEEDCG_ERR_NAN) code = SEEDCG_ERR_NAN;
    else if (lz_status == SEEDCG_ERR_TIMEOUT) code = SEEDCG_ERR_TIMEOUT;
    else if (lz_status == SEEDCG_ERR_BREAKDOWN) code = SEEDCG_ERR_BREAKDOWN;
    if (cg_now && code == SEEDCG_OK) {
        for (int j = 0; j < nrhs; j++)
            if (cgr.notconv[0][j] || !(cgr.true_resid[0][j] <= tol)) code = SEEDCG_ERR_NOT_CONVERGED;
    }
    if (info) {
        info->m_conv = m_conv;
        info->m = m;
        info->po_count = po_count;
        int mx = 0;
        for (int j = 0; j < nrhs; j++) mx = std::max(mx, cg_now ? cgr.iters[0][j] : 0);
        info->cg_iters_max = mx;
        info->reliable_updates = cgr.reliable_updates;
        for (int j = 0; j < nrhs; j++) {
            const int it = cg_now ? cgr.iters[0][j] : 0;
            const int ru = cg_now ? cgr.ru[0][j] : 0;
            if (info->iters) info->iters[j] = it + (j == 0 ? m : 0);
            if (info->matvecs) info->matvecs[j] = 2 * (it + ru) + (j == 0 ? 2 * m : 0) + ((o.x0_given || h->force_x0) ? 2 : 0);
            if (info->true_resid) info->true_resid[j] = cg_now ? cgr.true_resid[0][j] : 0.0;
        }
        info->ms_total = t_all.read();
        info->ms_lanczos = t_lz.read();
        info->ms_po = ms_po;
        info->ms_seed = t_seed.read();
        info->ms_cg = t_cg.read();
    }
    return code;
}

}  // namespace

// Several gauge fields: Lanczos + seeds per field, then ONE batched CG over the
// seeded systems of all fields (B, X device canonical complex128 per field).
seedcg_status batch_solve_impl(seedcg_handle** hs, int nf, const int* nrhs, const double* const* B,
                               double* const* X, double tol, int extra_iters, int reorth_period,
                               seedcg_info* infos, cudaStream_t st) {
    const int prec = hs[0]->opt.precision;
    std::vector<CgGroup> groups;
    std::vector<seedcg_status> lz(nf, SEEDCG_OK);
    std::vector<int> ms(nf, 0);
    for (int f = 0; f < nf; f++) {
        seedcg_handle* h = hs[f];
        const int vol = h->g.vol;
        const long n = 12L * vol;
        const size_t fb = (size_t)nrhs[f] * n * sizeof(double2);
        h->staging.ensure(2 * fb + 512);
        double2* B64 = h->staging.as<double2>();
        double2* X64 = B64 + (size_t)nrhs[f] * n;
        to_internal_f64(B[f], B64, vol, nrhs[f], st);
        if (h->opt.x0_given)
            to_internal_f64(X[f], X64, vol, nrhs[f], st);
        else
            SEEDCG_CUDA_TRY(cudaMemsetAsync(X64, 0, fb, st));
        seedcg_info* inf = infos ? &infos[f] : nullptr;
        switch (prec) {
            case SEEDCG_FP64:
                lz[f] = run_solve<double, double2>(h, nrhs[f], B64, X64, tol, extra_iters, reorth_period, inf, st, false);
                break;
            case SEEDCG_MIXED_V32:
                lz[f] = run_solve<float, float2>(h, nrhs[f], B64, X64, tol, extra_iters, reorth_period, inf, st, false);
                break;
            default:
                lz[f] = run_solve<float, __nv_bfloat162>(h, nrhs[f], B64, X64, tol, extra_iters, reorth_period, inf, st, false);
                break;
        }
        ms[f] = h->last_m;
        groups.push_back({h, nrhs[f], B64, X64});
    }
    CgResult cgr;
    PhaseTimer t;
    t.start(st);
    if (!hs[0]->opt.stop_after_seed) {
        const seedcg_options& o = hs[0]->opt;
        if (prec == SEEDCG_FP64)
            batched_cg<double>(groups, tol, 0.0, o.cg_maxiter, o.poll_every, true, hs[0]->cgbuf,
                               hs[0]->pinned, cgr, st);
        else
            batched_cg<float>(groups, tol, o.reliable_delta, o.cg_maxiter, o.poll_every, true,
                              hs[0]->cgbuf, hs[0]->pinned, cgr, st);
    }
    t.stop(st);
    const float ms_cg = t.read();
    seedcg_status code = SEEDCG_OK;
    for (int f = 0; f < nf; f++) {
        seedcg_handle* h = hs[f];
        if (lz[f] != SEEDCG_OK && lz[f] != SEEDCG_ERR_NOT_CONVERGED && code == SEEDCG_OK) code = lz[f];
        const bool ran = !hs[0]->opt.stop_after_seed;
        if (ran)
            for (int j = 0; j < nrhs[f]; j++)
                if (cgr.notconv[f][j] || !(cgr.true_resid[f][j] <= tol))
                    if (code == SEEDCG_OK) code = SEEDCG_ERR_NOT_CONVERGED;
        if (infos) {
            seedcg_info& inf = infos[f];
            int mx = 0;
            for (int j = 0; j < nrhs[f]; j++) {
                const int it = ran ? cgr.iters[f][j] : 0;
                const int ru = ran ? cgr.ru[f][j] : 0;
                mx = std::max(mx, it);
                if (inf.iters) inf.iters[j] = it + (j == 0 ? ms[f] : 0);
                if (inf.matvecs) inf.matvecs[j] = 2 * (it + ru) + (j == 0 ? 2 * ms[f] : 0);
                if (inf.true_resid) inf.true_resid[j] = ran ? cgr.true_resid[f][j] : 0.0;
            }
            inf.cg_iters_max = mx;
            inf.reliable_updates = cgr.reliable_updates;
            inf.ms_cg = ms_cg;
            inf.ms_total += ms_cg;
        }
        const double2* X64 = groups[f].x64;
        from_internal_f64(X64, X[f], h->g.vol, nrhs[f], st);
    }
    SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
    return code;
}

// ---------------------------------------------------------------------------
// Ritz pairs and deflated initial guesses from the stored basis (the premise of
// Sections 1-2: the subspace built past convergence holds accurate low
// eigenvectors of M).
// ---------------------------------------------------------------------------

// number of eigenvalues of the symmetric tridiagonal T below x (Sturm sequence
// of the LDL^T factorisation of T - x I)
static int sturm_count(int m, const double* a, const double* b, double x) {
    int c = 0;
    double d = 1.0;
    for (int i = 0; i < m; i++) {
        const double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
        d = (a[i] - x) - (i > 0 ? bb / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) c++;
    }
    return c;
}

void tridiag_lowest(int m, const double* a, const double* b, int nev, double* theta, double* S) {
    double lo = a[0], hi = a[0];
    for (int i = 0; i < m; i++) {
        const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i < m - 1 ? std::fabs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    const double scale = std::max(std::fabs(lo), std::fabs(hi));
    // eigenvalues by bisection: theta_k is where the count passes k
    for (int k = 0; k < nev; k++) {
        double l = lo, u = hi;
        for (int it = 0; it < 200 && u - l > 4e-16 * scale; it++) {
            const double mid = 0.5 * (l + u);
            if (sturm_count(m, a, b, mid) <= k) l = mid;
            else u = mid;
        }
        theta[k] = 0.5 * (l + u);
    }
    // eigenvectors by inverse iteration with a slightly shifted theta, then
    // Gram-Schmidt against the earlier vectors (clusters)
    std::vector<double> y(m), z(m), dd(m), cc(m);
    for (int k = 0; k < nev; k++) {
        const double sh = theta[k] - 1e-13 * scale;
        for (int i = 0; i < m; i++) y[i] = 1.0 / std::sqrt((double)m) * (1.0 + 0.01 * ((i * 7 + k * 13) % 11));
        for (int it = 0; it < 4; it++) {
            // solve (T - sh I) z = y by elimination without pivoting (tiny pivots floored)
            for (int i = 0; i < m; i++) {
                double piv = a[i] - sh - (i > 0 ? b[i - 1] * cc[i - 1] : 0.0);
                if (std::fabs(piv) < 1e-300) piv = 1e-300;
                cc[i] = i < m - 1 ? b[i] / piv : 0.0;
                dd[i] = (y[i] - (i > 0 ? b[i - 1] * dd[i - 1] : 0.0)) / piv;
            }
            z[m - 1] = dd[m - 1];
            for (int i = m - 2; i >= 0; i--) z[i] = dd[i] - cc[i] * z[i + 1];
            for (int j = 0; j < k; j++) {
                double p = 0.0;
                for (int i = 0; i < m; i++) p += S[(size_t)i * nev + j] * z[i];
                for (int i = 0; i < m; i++) z[i] -= p * S[(size_t)i * nev + j];
            }
            double nrm = 0.0;
            for (int i = 0; i < m; i++) nrm += z[i] * z[i];
            nrm = std::sqrt(nrm);
            for (int i = 0; i < m; i++) y[i] = z[i] / nrm;
        }
        for (int i = 0; i < m; i++) S[(size_t)i * nev + k] = y[i];
    }
}

seedcg_status deflate_impl(seedcg_handle* h, int nev, int nr, const double* B, double* X0, double* theta_out,
                           cudaStream_t st) {
    const int vol = h->g.vol;
    const long n = 12L * vol;
    const int m = std::min<int>(h->vbasis_m, (int)h->alpha.size());
    if (m < 1 || nev < 1 || nev > m || nev > 64 || nr < 1) return SEEDCG_ERR_ARG;
    std::vector<double> theta(nev), S((size_t)m * nev);
    tridiag_lowest(m, h->alpha.data(), h->beta.data(), nev, theta.data(), S.data());
    std::vector<double2> hc((size_t)m * nev);
    for (size_t i = 0; i < hc.size(); i++) hc[i] = make_double2(S[i], 0.0);
    DevBuf cbuf, ybuf, mybuf, tbuf, bbuf, gbuf, rbuf, xbuf, scr;
    cbuf.ensure(hc.size() * sizeof(double2));
    SEEDCG_CUDA_TRY(cudaMemcpyAsync(cbuf.p, hc.data(), hc.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
    const size_t fy = (size_t)nev * n * sizeof(double2);
    ybuf.ensure(fy);
    mybuf.ensure(fy);
    tbuf.ensure(fy);
    SEEDCG_CUDA_TRY(cudaMemsetAsync(ybuf.p, 0, fy, st));
    double2* Y = ybuf.as<double2>();
    // Ritz vectors Y = V S in FP64
    if (h->vbasis_prec == SEEDCG_FP64)
        gemm_n<double, double2, double2>(h->vbasis.as<double2>(), n, m, cbuf.as<double2>(), nev, nev, Y, n, n,
                                         1.0, st);
    else if (h->vbasis_prec == SEEDCG_MIXED_V32)
        gemm_n<float, float2, double2>(h->vbasis.as<float2>(), n, m, cbuf.as<double2>(), nev, nev, Y, n, n,
                                       1.0, st);
    else
        gemm_n<float, __nv_bfloat162, double2>(h->vbasis.as<__nv_bfloat162>(), n, m, cbuf.as<double2>(), nev,
                                               nev, Y, n, n, 1.0, st);
    apply_M64(h, nev, Y, tbuf.as<double2>(), mybuf.as<double2>(), st);
    const size_t split = std::max<size_t>((size_t)nev * std::max(nev, nr) * 64, (size_t)1 << 20);
    scr.ensure(split * sizeof(double2));
    gbuf.ensure((size_t)nev * nev * sizeof(double2));
    gemm_t<double, double2>(Y, n, nev, mybuf.as<double2>(), n, nev, n, gbuf.as<double2>(), nev, scr.as<double2>(),
                            split, st);                                          // G = Y^dag M Y
    bbuf.ensure((size_t)nr * n * sizeof(double2));
    to_internal_f64(B, bbuf.as<double2>(), vol, nr, st);
    rbuf.ensure((size_t)nev * nr * sizeof(double2));
    gemm_t<double, double2>(Y, n, nev, bbuf.as<double2>(), n, nr, n, rbuf.as<double2>(), nr, scr.as<double2>(),
                            split, st);                                          // R = Y^dag B
    std::vector<double2> G((size_t)nev * nev), Rh((size_t)nev * nr);
    SEEDCG_CUDA_TRY(cudaMemcpyAsync(G.data(), gbuf.p, G.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
    SEEDCG_CUDA_TRY(cudaMemcpyAsync(Rh.data(), rbuf.p, Rh.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
    SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
    // Cholesky G = L L^dag (Hermitian positive definite), then c = G^-1 R column by column
    using cd = std::complex<double>;
    std::vector<cd> L((size_t)nev * nev, cd(0, 0));
    for (int i = 0; i < nev; i++)
        for (int j = 0; j <= i; j++) {
            cd sum(G[(size_t)i * nev + j].x, G[(size_t)i * nev + j].y);
            for (int k = 0; k < j; k++) sum -= L[(size_t)i * nev + k] * std::conj(L[(size_t)j * nev + k]);
            if (i == j) {
                if (!(sum.real() > 0.0)) return SEEDCG_ERR_BREAKDOWN;
                L[(size_t)i * nev + i] = std::sqrt(sum.real());
            } else {
                L[(size_t)i * nev + j] = sum / L[(size_t)j * nev + j];
            }
        }
    std::vector<double2> hcoef((size_t)nev * nr);
    std::vector<cd> w(nev);
    for (int r = 0; r < nr; r++) {
        for (int i = 0; i < nev; i++) {
            cd sum(Rh[(size_t)i * nr + r].x, Rh[(size_t)i * nr + r].y);
            for (int k = 0; k < i; k++) sum -= L[(size_t)i * nev + k] * w[k];
            w[i] = sum / L[(size_t)i * nev + i];
        }
        for (int i = nev - 1; i >= 0; i--) {
            cd sum = w[i];
            for (int k = i + 1; k < nev; k++) sum -= std::conj(L[(size_t)k * nev + i]) * w[k];
            w[i] = sum / L[(size_t)i * nev + i];
        }
        for (int i = 0; i < nev; i++) hcoef[(size_t)i * nr + r] = make_double2(w[i].real(), w[i].imag());
    }
    DevBuf cc;
    cc.ensure(hcoef.size() * sizeof(double2));
    SEEDCG_CUDA_TRY(cudaMemcpyAsync(cc.p, hcoef.data(), hcoef.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
    xbuf.ensure((size_t)nr * n * sizeof(double2));
    SEEDCG_CUDA_TRY(cudaMemsetAsync(xbuf.p, 0, (size_t)nr * n * sizeof(double2), st));
    gemm_n<double, double2, double2>(Y, n, nev, cc.as<double2>(), nr, nr, xbuf.as<double2>(), n, n, 1.0, st);
    from_internal_f64(xbuf.as<double2>(), X0, vol, nr, st);
    SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
    if (theta_out)
        for (int k = 0; k < nev; k++) theta_out[k] = theta[k];
    return SEEDCG_OK;
}

seedcg_status project_basis_impl(seedcg_handle* h, int rows, int nvec, const double* X,
                                 double* C, int use_tc, cudaStream_t st) {
    const int vol = h->g.vol;
    const long n = 12L * vol;
    const int prec = h->vbasis_prec;
    DevBuf xb, cb, scr;
    const size_t cbytes = (size_t)rows * nvec * sizeof(double2);
    cb.ensure(cbytes + 256);
    const size_t split_elems = std::max<size_t>((size_t)rows * nvec * 64, (size_t)1 << 20);
    scr.ensure(split_elems * sizeof(double2));
    if (prec == SEEDCG_FP64) {
        xb.ensure((size_t)nvec * n * sizeof(double2));
        to_internal_f64(X, xb.as<double2>(), vol, nvec, st);
        gemm_t<double, double2>(h->vbasis.as<double2>(), n, rows, xb.as<double2>(), n, nvec, n,
                                cb.as<double2>(), nvec, scr.as<double2>(), split_elems, st);
    } else {
        xb.ensure((size_t)nvec * n * sizeof(float2));
        to_internal_f32(X, xb.as<float2>(), vol, nvec, st);
        if (prec == SEEDCG_MIXED_V32) {
            gemm_t<float, float2>(h->vbasis.as<float2>(), n, rows, xb.as<float2>(), n, nvec, n,
                                  cb.as<double2>(), nvec, scr.as<double2>(), split_elems, st);
        } else if (use_tc) {
            DevBuf bm, part, e;
            bm.ensure(tc_b_bytes(n, nvec));
            const size_t pe = (size_t)4 << 20;
            part.ensure(pe * sizeof(float));
            e.ensure(sizeof(int));
            SEEDCG_CUDA_TRY(cudaMemsetAsync(e.p, 0, sizeof(int), st));
            SEEDCG_CUDA_TRY(cudaMemsetAsync(bm.p, 0, tc_b_bytes(n, nvec), st));
            tc_project(h->vbasis.as<__nv_bfloat162>(), h->opt.m_max, rows, xb.as<float2>(), n, nvec,
                       n, bm.as<__nv_bfloat162>(), part.as<float>(), pe, cb.as<double2>(), nvec,
                       e.as<int>(), st);
            int herr = 0;
            SEEDCG_CUDA_TRY(cudaMemcpyAsync(&herr, e.p, sizeof(int), cudaMemcpyDeviceToHost, st));
            SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
            if (herr) return SEEDCG_ERR_TIMEOUT;
        } else {
            gemm_t<float, __nv_bfloat162>(h->vbasis.as<__nv_bfloat162>(), n, rows, xb.as<float2>(), n,
                                          nvec, n, cb.as<double2>(), nvec, scr.as<double2>(),
                                          split_elems, st);
        }
    }
    SEEDCG_CUDA_TRY(cudaMemcpyAsync(C, cb.p, cbytes, cudaMemcpyDeviceToHost, st));
    SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
    return SEEDCG_OK;
}

namespace {

// Classic repeated seeding (seed_mode 2, the comparison variant of Section 1):
// round j runs Lanczos on system j from its current guess, stopped at
// convergence, and seeds systems j+1.. by Eq. (1); then one batched CG finishes
// every system whose true residual is still above tol.
template <typename R, typename VT>
seedcg_status classic_rounds(seedcg_handle* h, int nrhs, double2* B64, double2* X64, double tol,
                             int k_po, seedcg_info* info, cudaStream_t st) {
    const long n = 12L * (h->eo_active ? h->g.vol / 2 : h->g.vol);
    const seedcg_options saved = h->opt;
    const bool x0 = saved.x0_given || h->force_x0;
    std::vector<int> lz(nrhs, 0);
    float ms_lz = 0.f, ms_po = 0.f, ms_seed = 0.f, ms_rounds = 0.f;
    int m_conv0 = 0, m0 = 0, po0 = 0;
    seedcg_status code = SEEDCG_OK;
    try {
        h->opt.past_factor = 1.0;
        h->opt.seed_mode = 1;
        h->opt.x0_given = 0;
        for (int j = 0; j < nrhs && code == SEEDCG_OK; j++) {
            h->force_x0 = x0 || j > 0;
            const int nr = nrhs - j;
            std::vector<int> it(nr), mv(nr);
            std::vector<double> tr(nr);
            seedcg_info ri{};
            ri.iters = it.data();
            ri.matvecs = mv.data();
            ri.true_resid = tr.data();
            code = run_solve<R, VT>(h, nr, B64 + (size_t)j * n, X64 + (size_t)j * n, tol, 0, k_po, &ri, st,
                                    false);
            lz[j] = ri.m;
            if (j == 0) {
                m_conv0 = ri.m_conv;
                m0 = ri.m;
                po0 = ri.po_count;
            }
            ms_lz += ri.ms_lanczos;
            ms_po += ri.ms_po;
            ms_seed += ri.ms_seed;
            ms_rounds += ri.ms_total;
        }
    } catch (...) {
        h->opt = saved;
        h->force_x0 = false;
        throw;
    }
    h->opt = saved;
    h->force_x0 = false;
    if (code != SEEDCG_OK) return code;
    CgResult cgr;
    PhaseTimer t_cg;
    t_cg.start(st);
    std::vector<CgGroup> gs{{h, nrhs, B64, X64}};
    const int poll = saved.poll_every > 0 ? saved.poll_every : 32;
    batched_cg<R>(gs, tol, sizeof(R) == 8 ? 0.0 : saved.reliable_delta, saved.cg_maxiter, poll, true,
                  h->cgbuf, h->pinned, cgr, st);
    t_cg.stop(st);
    for (int j = 0; j < nrhs; j++)
        if (cgr.notconv[0][j] || !(cgr.true_resid[0][j] <= tol)) code = SEEDCG_ERR_NOT_CONVERGED;
    if (info) {
        info->m_conv = m_conv0;
        info->m = m0;
        info->po_count = po0;
        int mx = 0;
        for (int j = 0; j < nrhs; j++) mx = std::max(mx, cgr.iters[0][j]);
        info->cg_iters_max = mx;
        info->reliable_updates = cgr.reliable_updates;
        for (int j = 0; j < nrhs; j++) {
            if (info->iters) info->iters[j] = lz[j] + cgr.iters[0][j];
            if (info->matvecs)
                info->matvecs[j] = 2 * lz[j] + ((x0 || j > 0) ? 2 : 0) + 2 * (cgr.iters[0][j] + cgr.ru[0][j]);
            if (info->true_resid) info->true_resid[j] = cgr.true_resid[0][j];
        }
        info->ms_lanczos = ms_lz;
        info->ms_po = ms_po;
        info->ms_seed = ms_seed;
        info->ms_cg = t_cg.read();
        info->ms_total = ms_rounds + info->ms_cg;
    }
    return code;
}

// No seeding (seed_mode 3): standard CG for every system from its x_0, all of
// them in the batched engine.  Section 3 measures the seeded systems against
// this baseline (standard CG from zero); it runs no Lanczos and stores no basis.
template <typename R>
seedcg_status cg_only(seedcg_handle* h, int nrhs, double2* B64, double2* X64, double tol,
                      seedcg_info* info, cudaStream_t st) {
    const seedcg_options& o = h->opt;
    const bool x0 = o.x0_given || h->force_x0;
    CgResult cgr;
    PhaseTimer t_cg;
    t_cg.start(st);
    std::vector<CgGroup> gs{{h, nrhs, B64, X64}};
    const int poll = o.poll_every > 0 ? o.poll_every : 32;
    batched_cg<R>(gs, tol, sizeof(R) == 8 ? 0.0 : o.reliable_delta, o.cg_maxiter, poll, true, h->cgbuf,
                  h->pinned, cgr, st);
    t_cg.stop(st);
    h->last_m = 0;
    h->vbasis_m = 0;
    h->alpha.clear();
    h->beta.clear();
    h->delta.clear();
    seedcg_status code = SEEDCG_OK;
    for (int j = 0; j < nrhs; j++)
        if (cgr.notconv[0][j] || !(cgr.true_resid[0][j] <= tol)) code = SEEDCG_ERR_NOT_CONVERGED;
    if (info) {
        info->m_conv = 0;
        info->m = 0;
        info->po_count = 0;
        int mx = 0;
        for (int j = 0; j < nrhs; j++) mx = std::max(mx, cgr.iters[0][j]);
        info->cg_iters_max = mx;
        info->reliable_updates = cgr.reliable_updates;
        for (int j = 0; j < nrhs; j++) {
            if (info->iters) info->iters[j] = cgr.iters[0][j];
            if (info->matvecs) info->matvecs[j] = 2 * (cgr.iters[0][j] + cgr.ru[0][j]) + (x0 ? 2 : 0);
            if (info->true_resid) info->true_resid[j] = cgr.true_resid[0][j];
        }
        info->ms_lanczos = info->ms_po = info->ms_seed = 0.f;
        info->ms_cg = t_cg.read();
        info->ms_total = info->ms_cg;
    }
    return code;
}

// ratio[j] = ||eta_j - D x_j|| / ||eta_j|| in FP64 (T: scratch of nrhs fields)
void d_residuals(seedcg_handle* h, int nrhs, const double2* E64, const double2* X64, double2* T64,
                 std::vector<double>& ratio, cudaStream_t st) {
    const long n = 12L * h->g.vol;
    dslash_mrhs_f64(h->g, h->u64.as<double2>(), h->kappa, 0, nrhs, X64, T64, st);
    DevBuf nr;
    nr.ensure(sizeof(double) * (4096 + 2 * nrhs) + sizeof(unsigned) * 64);
    double* part = nr.as<double>();
    double* norms = part + 4096;
    unsigned* ctr = reinterpret_cast<unsigned*>(norms + 2 * nrhs);
    SEEDCG_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(unsigned) * 64, st));
    for (int j = 0; j < nrhs; j++) {
        axpby_f64(E64 + (size_t)j * n, T64 + (size_t)j * n, n, st);  // T = eta - D x
        k_norm2_public(E64 + (size_t)j * n, n, part, ctr, norms + j, st);
        k_norm2_public(T64 + (size_t)j * n, n, part, ctr, norms + nrhs + j, st);
    }
    std::vector<double> hn(2 * nrhs);
    SEEDCG_CUDA_TRY(cudaMemcpyAsync(hn.data(), norms, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, st));
    SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
    ratio.assign(nrhs, 0.0);
    for (int j = 0; j < nrhs; j++) ratio[j] = hn[j] > 0.0 ? hn[nrhs + j] / hn[j] : 0.0;
}

// Original-system criterion (resid_mode 1): while some ||eta - D x|| / ||eta|| > tol,
// continue CG on those systems with an M tolerance tightened by the observed gap.
seedcg_status d_residual_rounds(seedcg_handle* h, int nrhs, const double2* E64, const double2* B64,
                                double2* X64, double2* T64, double tol, bool run_cg,
                                seedcg_status code, seedcg_info* info, cudaStream_t st) {
    const long n = 12L * h->g.vol;
    const seedcg_options& o = h->opt;
    std::vector<double> ratio;
    d_residuals(h, nrhs, E64, X64, T64, ratio, st);
    double tol_m = tol;
    for (int round = 0; run_cg && code == SEEDCG_OK && round < 6; round++) {
        std::vector<int> fail;
        double worst = 0.0;
        for (int j = 0; j < nrhs; j++)
            if (!(ratio[j] <= tol)) {
                fail.push_back(j);
                worst = std::max(worst, ratio[j]);
            }
        if (fail.empty() || !std::isfinite(worst)) break;
        tol_m *= std::max(0.01, 0.5 * tol / worst);
        const int nf = (int)fail.size();
        DevBuf gb, gx;
        gb.ensure((size_t)nf * n * sizeof(double2));
        gx.ensure((size_t)nf * n * sizeof(double2));
        for (int k = 0; k < nf; k++) {
            SEEDCG_CUDA_TRY(cudaMemcpyAsync(gb.as<double2>() + (size_t)k * n, B64 + (size_t)fail[k] * n,
                                            n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
            SEEDCG_CUDA_TRY(cudaMemcpyAsync(gx.as<double2>() + (size_t)k * n, X64 + (size_t)fail[k] * n,
                                            n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        }
        std::vector<CgGroup> gs{{h, nf, gb.as<double2>(), gx.as<double2>()}};
        CgResult cgr;
        if (o.precision == SEEDCG_FP64)
            batched_cg<double>(gs, tol_m, 0.0, o.cg_maxiter, o.poll_every, true, h->cgbuf, h->pinned, cgr, st);
        else
            batched_cg<float>(gs, tol_m, o.reliable_delta, o.cg_maxiter, o.poll_every, true, h->cgbuf,
                              h->pinned, cgr, st);
        for (int k = 0; k < nf; k++)
            SEEDCG_CUDA_TRY(cudaMemcpyAsync(X64 + (size_t)fail[k] * n, gx.as<double2>() + (size_t)k * n,
                                            n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        bool stuck = false;
        if (info) {
            info->reliable_updates += cgr.reliable_updates;
            for (int k = 0; k < nf; k++) {
                const int j = fail[k];
                if (info->iters) info->iters[j] += cgr.iters[0][k];
                if (info->matvecs) info->matvecs[j] += 2 * (cgr.iters[0][k] + cgr.ru[0][k]) + 2;
                if (info->true_resid) info->true_resid[j] = cgr.true_resid[0][k];
            }
        }
        for (int k = 0; k < nf; k++) stuck = stuck || cgr.notconv[0][k];
        d_residuals(h, nrhs, E64, X64, T64, ratio, st);
        if (stuck) break;
    }
    if (info) {
        int mx = info->cg_iters_max;
        if (info->iters)
            for (int j = 1; j < nrhs; j++) mx = std::max(mx, info->iters[j]);
        info->cg_iters_max = mx;
        if (info->true_resid_D)
            for (int j = 0; j < nrhs; j++) info->true_resid_D[j] = ratio[j];
    }
    if (run_cg && code == SEEDCG_OK)
        for (int j = 0; j < nrhs; j++)
            if (!(ratio[j] <= tol)) code = SEEDCG_ERR_NOT_CONVERGED;
    return code;
}

}  // namespace

namespace {
seedcg_status dispatch_solve(seedcg_handle* h, int nrhs, double2* B64, double2* X64, double tol,
                             int extra_iters, int reorth_period, seedcg_info* info, cudaStream_t st);
}

seedcg_status solve_impl(seedcg_handle* h, int nrhs, const double* B, double* X, double tol,
                         int extra_iters, int reorth_period, seedcg_info* info, cudaStream_t st) {
    // B, X: device canonical complex128 (the API layer stages host pointers)
    const int vol = h->g.vol;
    const long n = 12L * vol;
    const size_t fb = (size_t)nrhs * n * sizeof(double2);
    const bool dmode = h->opt.resid_mode == 1;
    h->staging.ensure((dmode ? 4 : 2) * fb + 512);
    double2* B64 = h->staging.as<double2>();
    double2* X64 = B64 + (size_t)nrhs * n;
    double2* E64 = dmode ? X64 + (size_t)nrhs * n : nullptr;   // eta of D x = eta
    double2* T64 = dmode ? E64 + (size_t)nrhs * n : nullptr;   // scratch
    if (dmode) {
        to_internal_f64(B, E64, vol, nrhs, st);
        dslash_mrhs_f64(h->g, h->u64.as<double2>(), h->kappa, 1, nrhs, E64, B64, st);  // b = D^dag eta
    } else {
        to_internal_f64(B, B64, vol, nrhs, st);
    }
    if (h->opt.x0_given)
        to_internal_f64(X, X64, vol, nrhs, st);
    else
        SEEDCG_CUDA_TRY(cudaMemsetAsync(X64, 0, fb, st));
    h->force_x0 = false;
    if (h->opt.use_guess && guess_ready(h)) {
        // x_0 = net(b); fall back to 0 where ||b - M x_0|| >= ||b||
        guess_predict(h, nrhs, B64, X64, st);
        DevBuf t1, t2, nr;
        t1.ensure(fb);
        t2.ensure(fb);
        nr.ensure(sizeof(double) * (4096 + 2 * nrhs) + sizeof(unsigned) * 64);
        dslash_mrhs_f64(h->g, h->u64.as<double2>(), h->kappa, 0, nrhs, X64, t1.as<double2>(), st);
        dslash_mrhs_f64(h->g, h->u64.as<double2>(), h->kappa, 1, nrhs, t1.as<double2>(), t2.as<double2>(), st);
        double* part = nr.as<double>();
        double* norms = part + 4096;
        unsigned* ctr = reinterpret_cast<unsigned*>(norms + 2 * nrhs);
        SEEDCG_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(unsigned) * 64, st));
        for (int j = 0; j < nrhs; j++) {
            axpby_f64(B64 + (size_t)j * n, t2.as<double2>() + (size_t)j * n, n, st);  // t2 = b - M x0
            k_norm2_public(B64 + (size_t)j * n, n, part, ctr, norms + j, st);
            k_norm2_public(t2.as<double2>() + (size_t)j * n, n, part, ctr, norms + nrhs + j, st);
        }
        std::vector<double> hn(2 * nrhs);
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(hn.data(), norms, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, st));
        SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
        for (int j = 0; j < nrhs; j++)
            if (!(hn[nrhs + j] < hn[j])) SEEDCG_CUDA_TRY(cudaMemsetAsync(X64 + (size_t)j * n, 0, n * sizeof(double2), st));
        h->force_x0 = true;
    }
    seedcg_status code = dispatch_solve(h, nrhs, B64, X64, tol, extra_iters, reorth_period, info, st);
    if (dmode)
        code = d_residual_rounds(h, nrhs, E64, B64, X64, T64, tol, !h->opt.stop_after_seed, code, info, st);
    from_internal_f64(X64, X, vol, nrhs, st);
    SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
    return code;
}

namespace {
// the method selected by the options on internal FP64 B64 / X64 (full or, with
// h->eo_active, odd-site half vectors)
seedcg_status dispatch_solve(seedcg_handle* h, int nrhs, double2* B64, double2* X64, double tol,
                             int extra_iters, int reorth_period, seedcg_info* info, cudaStream_t st) {
    seedcg_status code;
    if (h->opt.seed_mode == 3) {
        code = h->opt.precision == SEEDCG_FP64 ? cg_only<double>(h, nrhs, B64, X64, tol, info, st)
                                                : cg_only<float>(h, nrhs, B64, X64, tol, info, st);
    } else if (h->opt.seed_mode == 2) {
        switch (h->opt.precision) {
            case SEEDCG_FP64:
                code = classic_rounds<double, double2>(h, nrhs, B64, X64, tol, reorth_period, info, st);
                break;
            case SEEDCG_MIXED_V32:
                code = classic_rounds<float, float2>(h, nrhs, B64, X64, tol, reorth_period, info, st);
                break;
            default:
                code = classic_rounds<float, __nv_bfloat162>(h, nrhs, B64, X64, tol, reorth_period, info, st);
                break;
        }
    } else switch (h->opt.precision) {
        case SEEDCG_FP64:
            code = run_solve<double, double2>(h, nrhs, B64, X64, tol, extra_iters, reorth_period, info, st);
            break;
        case SEEDCG_MIXED_V32:
            code = run_solve<float, float2>(h, nrhs, B64, X64, tol, extra_iters, reorth_period, info, st);
            break;
        default:
            code = run_solve<float, __nv_bfloat162>(h, nrhs, B64, X64, tol, extra_iters, reorth_period, info, st);
            break;
    }
    return code;
}
}  // namespace

// Improved Seed-CG on the even-odd preconditioned system of Section 3,
// A^dag A x_o = A^dag phi with phi = eta_o + kappa H_oe eta_e, on the same
// device-resident engine as the full-lattice solve (every precision mode and
// seeding form), then x_e = eta_e + kappa H_eo x_o.  E, X: device canonical
// complex128 full fields.
seedcg_status solve_eo_impl(seedcg_handle* h, int nrhs, const double* E, double* X, double tol,
                            int extra_iters, int reorth_period, seedcg_info* info, cudaStream_t st) {
    const Geom& g = h->g;
    const long nh = 12L * (g.vol / 2), nf = 12L * g.vol;
    // staging: eta and the full solution (full), then phi, b, x_o (half), 3 half scratch
    const size_t full_b = (size_t)nrhs * nf * sizeof(double2), half_b = (size_t)nrhs * nh * sizeof(double2);
    h->staging.ensure(2 * full_b + 3 * half_b + 3 * (size_t)nh * sizeof(double2) + 1024);
    double2* E64 = h->staging.as<double2>();
    double2* F64 = E64 + (size_t)nrhs * nf;
    double2* Phi = F64 + (size_t)nrhs * nf;
    double2* B64 = Phi + (size_t)nrhs * nh;
    double2* X64 = B64 + (size_t)nrhs * nh;
    double2* s0 = X64 + (size_t)nrhs * nh;
    double2* s1 = s0 + nh;
    double2* s2 = s1 + nh;
    const double2* u = h->u64.as<double2>();
    to_internal_f64(E, E64, g.vol, nrhs, st);
    eo_rhs_f64(g, u, h->kappa, nrhs, E64, Phi, B64, s0, s1, s2, st);
    if (h->opt.x0_given) {
        to_internal_f64(X, F64, g.vol, nrhs, st);
        eo_gather_f64(g, 1, nrhs, F64, X64, st);
    } else {
        SEEDCG_CUDA_TRY(cudaMemsetAsync(X64, 0, half_b, st));
    }
    struct EoScope {
        seedcg_handle* h;
        ~EoScope() { h->eo_active = false; }
    } scope{h};
    h->eo_active = true;
    h->force_x0 = false;
    seedcg_status code = dispatch_solve(h, nrhs, B64, X64, tol, extra_iters, reorth_period, info, st);
    h->eo_active = false;
    eo_reconstruct_f64(g, u, h->kappa, nrhs, X64, E64, F64, s0, s1, st);
    if (info && info->true_resid_D) {
        // the residual of the original system D x = eta, as Section 3 monitors it
        DevBuf tb;
        tb.ensure(full_b);
        std::vector<double> ratio;
        d_residuals(h, nrhs, E64, F64, tb.as<double2>(), ratio, st);
        for (int j = 0; j < nrhs; j++) info->true_resid_D[j] = ratio[j];
    }
    from_internal_f64(F64, X, g.vol, nrhs, st);
    SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
    return code;
}

}  // namespace seedcg
