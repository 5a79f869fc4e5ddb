// Device-side Wilson hopping term, shared by the dslash kernels and the fused
// solver kernels.
//
//   (D psi)(x) = psi(x) - kappa sum_mu [ P-_mu U_mu(x) psi(x+mu) s_f
//                                      + P+_mu U_mu(x-mu)^dag psi(x-mu) s_b ]
//   P-_mu = 1 - g_mu,  P+_mu = 1 + g_mu,  s = -1 on hops that wrap t.
//   D^dag = g5 D g5 swaps P- and P+ (g5 anticommutes with every g_mu).
//
// Each projector has rank 2 in spin space, so a hop projects the 4-spinor to
// two colour vectors h0, h1, multiplies them by the link and rebuilds the
// other two spin components from them.  In the chiral basis
// g_k = [[0,-i s_k],[i s_k,0]], g_4 = [[0,1],[1,0]] the projections for
// P = 1 + S g_mu (S = +-1) are
//   mu=x: h0 = p0 - S i p3, h1 = p1 - S i p2;  full = (r0, r1,  S i r1,  S i r0)
//   mu=y: h0 = p0 - S   p3, h1 = p1 + S   p2;  full = (r0, r1,  S   r1, -S   r0)
//   mu=z: h0 = p0 - S i p2, h1 = p1 + S i p3;  full = (r0, r1,  S i r0, -S i r1)
//   mu=t: h0 = p0 + S   p2, h1 = p1 + S   p3;  full = (r0, r1,  S   r0,  S   r1)
#pragma once

#include "internal.cuh"

namespace seedcg {

template <typename R> struct Spinor { cx_t<R> c[4][3]; };

// h = (1 + S g_mu) p, two colour vectors
template <int MU, int S, typename R>
__device__ __forceinline__ void spin_project(const Spinor<R>& p, cx_t<R> h[2][3]) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (MU == 0) {
            h[0][a] = S > 0 ? csub(p.c[0][a], ci(p.c[3][a])) : cadd(p.c[0][a], ci(p.c[3][a]));
            h[1][a] = S > 0 ? csub(p.c[1][a], ci(p.c[2][a])) : cadd(p.c[1][a], ci(p.c[2][a]));
        } else if (MU == 1) {
            h[0][a] = S > 0 ? csub(p.c[0][a], p.c[3][a]) : cadd(p.c[0][a], p.c[3][a]);
            h[1][a] = S > 0 ? cadd(p.c[1][a], p.c[2][a]) : csub(p.c[1][a], p.c[2][a]);
        } else if (MU == 2) {
            h[0][a] = S > 0 ? csub(p.c[0][a], ci(p.c[2][a])) : cadd(p.c[0][a], ci(p.c[2][a]));
            h[1][a] = S > 0 ? cadd(p.c[1][a], ci(p.c[3][a])) : csub(p.c[1][a], ci(p.c[3][a]));
        } else {
            h[0][a] = S > 0 ? cadd(p.c[0][a], p.c[2][a]) : csub(p.c[0][a], p.c[2][a]);
            h[1][a] = S > 0 ? cadd(p.c[1][a], p.c[3][a]) : csub(p.c[1][a], p.c[3][a]);
        }
    }
}

// acc += coef * (full spinor rebuilt from r) for P = 1 + S g_mu
template <int MU, int S, typename R, bool SCALE = true>
__device__ __forceinline__ void spin_accum(Spinor<R>& acc, const cx_t<R> r[2][3], R coef) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        cx_t<R> r0 = SCALE ? cscale(r[0][a], coef) : r[0][a];
        cx_t<R> r1 = SCALE ? cscale(r[1][a], coef) : r[1][a];
        acc.c[0][a] = cadd(acc.c[0][a], r0);
        acc.c[1][a] = cadd(acc.c[1][a], r1);
        if (MU == 0) {
            acc.c[2][a] = S > 0 ? cadd(acc.c[2][a], ci(r1)) : csub(acc.c[2][a], ci(r1));
            acc.c[3][a] = S > 0 ? cadd(acc.c[3][a], ci(r0)) : csub(acc.c[3][a], ci(r0));
        } else if (MU == 1) {
            acc.c[2][a] = S > 0 ? cadd(acc.c[2][a], r1) : csub(acc.c[2][a], r1);
            acc.c[3][a] = S > 0 ? csub(acc.c[3][a], r0) : cadd(acc.c[3][a], r0);
        } else if (MU == 2) {
            acc.c[2][a] = S > 0 ? cadd(acc.c[2][a], ci(r0)) : csub(acc.c[2][a], ci(r0));
            acc.c[3][a] = S > 0 ? csub(acc.c[3][a], ci(r1)) : cadd(acc.c[3][a], ci(r1));
        } else {
            acc.c[2][a] = S > 0 ? cadd(acc.c[2][a], r0) : csub(acc.c[2][a], r0);
            acc.c[3][a] = S > 0 ? cadd(acc.c[3][a], r1) : csub(acc.c[3][a], r1);
        }
    }
}

// ||v||^2 at one site, in the working precision
template <typename R>
__device__ __forceinline__ R spinor_norm2(const Spinor<R>& v) {
    R a = 0;
#pragma unroll
    for (int k = 0; k < 12; k++) {
        const cx_t<R> z = v.c[k / 3][k % 3];
        a += z.x * z.x + z.y * z.y;
    }
    return a;
}

// ---------------------------------------------------------------------------
// spinor loads/stores in the internal layouts
// ---------------------------------------------------------------------------
// flat complex index of spinor element k (0..11) of site s
__host__ __device__ __forceinline__ size_t sidx(int k, int s, int vol) {
    return ((size_t)(k >> 1) * (size_t)vol + (size_t)s) * 2 + (size_t)(k & 1);
}

__device__ __forceinline__ void load_spinor(const float2* __restrict__ p, int vol, int s,
                                            Spinor<float>& out) {
    const float4* q = reinterpret_cast<const float4*>(p) + s;
#pragma unroll
    for (int c = 0; c < 6; c++) {
        const float4 z = __ldg(q + (size_t)c * vol);
        out.c[(2 * c) / 3][(2 * c) % 3] = make_float2(z.x, z.y);
        out.c[(2 * c + 1) / 3][(2 * c + 1) % 3] = make_float2(z.z, z.w);
    }
}
__device__ __forceinline__ void store_spinor(float2* __restrict__ p, int vol, int s,
                                             const Spinor<float>& v) {
    float4* q = reinterpret_cast<float4*>(p) + s;
#pragma unroll
    for (int c = 0; c < 6; c++) {
        const float2 a = v.c[(2 * c) / 3][(2 * c) % 3], b = v.c[(2 * c + 1) / 3][(2 * c + 1) % 3];
        q[(size_t)c * vol] = make_float4(a.x, a.y, b.x, b.y);
    }
}
// coherent loads, for a field that the same kernel writes back at the same site
__device__ __forceinline__ void load_spinor_rw(const float2* p, int vol, int s, Spinor<float>& out) {
    const float4* q = reinterpret_cast<const float4*>(p) + s;
#pragma unroll
    for (int c = 0; c < 6; c++) {
        const float4 z = q[(size_t)c * vol];
        out.c[(2 * c) / 3][(2 * c) % 3] = make_float2(z.x, z.y);
        out.c[(2 * c + 1) / 3][(2 * c + 1) % 3] = make_float2(z.z, z.w);
    }
}
__device__ __forceinline__ void load_spinor_rw(const double2* p, int vol, int s, Spinor<double>& out) {
#pragma unroll
    for (int k = 0; k < 12; k++) out.c[k / 3][k % 3] = p[sidx(k, s, vol)];
}
__device__ __forceinline__ void load_spinor(const double2* __restrict__ p, int vol, int s,
                                            Spinor<double>& out) {
#pragma unroll
    for (int k = 0; k < 12; k++) out.c[k / 3][k % 3] = __ldg(p + sidx(k, s, vol));
}
__device__ __forceinline__ void store_spinor(double2* __restrict__ p, int vol, int s,
                                             const Spinor<double>& v) {
#pragma unroll
    for (int k = 0; k < 12; k++) p[sidx(k, s, vol)] = v.c[k / 3][k % 3];
}

// ---------------------------------------------------------------------------
// neighbours
// ---------------------------------------------------------------------------
struct Nbr {
    int f[4], b[4];
    bool fwrap_t, bwrap_t;
};

__device__ __forceinline__ Nbr neighbours(const Geom& g, int s) {
    Nbr n;
    int c[4];
    int r = s;
    c[0] = r % g.L[0]; r /= g.L[0];
    c[1] = r % g.L[1]; r /= g.L[1];
    c[2] = r % g.L[2]; r /= g.L[2];
    c[3] = r;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        n.f[mu] = (c[mu] == g.L[mu] - 1) ? s - (g.L[mu] - 1) * g.stride[mu] : s + g.stride[mu];
        n.b[mu] = (c[mu] == 0) ? s + (g.L[mu] - 1) * g.stride[mu] : s - g.stride[mu];
    }
    n.fwrap_t = (c[3] == g.L[3] - 1);
    n.bwrap_t = (c[3] == 0);
    return n;
}

// ---------------------------------------------------------------------------
// one hop: acc += coef * P U psi_nbr  (forward: U = U_mu(x); backward: U = U_mu(x-mu)^dag)
// LinkAt(a, b) returns U[a][b] for the link in use.
// ---------------------------------------------------------------------------
template <int MU, int S, bool BACK, typename R, typename LinkAt, bool SCALE = true>
__device__ __forceinline__ void hop(Spinor<R>& acc, const Spinor<R>& nb, LinkAt link, R coef) {
    cx_t<R> h[2][3], r[2][3];
    spin_project<MU, S>(nb, h);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        cx_t<R> r0 = mk<R>(0, 0), r1 = mk<R>(0, 0);
#pragma unroll
        for (int b = 0; b < 3; b++) {
            if (!BACK) {
                cx_t<R> u = link(a, b);
                r0 = cfma(u, h[0][b], r0);
                r1 = cfma(u, h[1][b], r1);
            } else {
                cx_t<R> u = link(b, a);
                r0 = cfma_conj(u, h[0][b], r0);
                r1 = cfma_conj(u, h[1][b], r1);
            }
        }
        r[0][a] = r0;
        r[1][a] = r1;
    }
    spin_accum<MU, S, R, SCALE>(acc, r, coef);
}

// (D psi)(x) or (D^dag psi)(x) at one site, accumulated straight into `out`
// (out = psi(x), then out += -kappa * s * P U psi(y) hop by hop).
// Fwd(mu, e) / Bwd(mu, e) give element e = 3a+b of U_mu(x) / U_mu(x-mu);
// load(y, sp) loads the spinor at site y.
template <int DAG, typename R, typename LoadNbr, typename Fwd, typename Bwd>
__device__ __forceinline__ void wilson_site(const Nbr& n, int s, LoadNbr load, Fwd fl, Bwd bl,
                                            R kappa, Spinor<R>& out) {
    constexpr int SF = DAG ? 1 : -1;   // forward projector 1 - g (D) or 1 + g (D^dag)
    constexpr int SB = -SF;
    const R mk_ = -kappa;
    load(s, out);
    Spinor<R> nb;
    load(n.f[0], nb); hop<0, SF, false>(out, nb, [&](int a, int b) { return fl(0, 3 * a + b); }, mk_);
    load(n.b[0], nb); hop<0, SB, true>(out, nb, [&](int a, int b) { return bl(0, 3 * a + b); }, mk_);
    load(n.f[1], nb); hop<1, SF, false>(out, nb, [&](int a, int b) { return fl(1, 3 * a + b); }, mk_);
    load(n.b[1], nb); hop<1, SB, true>(out, nb, [&](int a, int b) { return bl(1, 3 * a + b); }, mk_);
    load(n.f[2], nb); hop<2, SF, false>(out, nb, [&](int a, int b) { return fl(2, 3 * a + b); }, mk_);
    load(n.b[2], nb); hop<2, SB, true>(out, nb, [&](int a, int b) { return bl(2, 3 * a + b); }, mk_);
    load(n.f[3], nb); hop<3, SF, false>(out, nb, [&](int a, int b) { return fl(3, 3 * a + b); }, n.fwrap_t ? kappa : mk_);
    load(n.b[3], nb); hop<3, SB, true>(out, nb, [&](int a, int b) { return bl(3, 3 * a + b); }, n.bwrap_t ? kappa : mk_);
}

// Same, with links that already carry -kappa and the boundary sign (staged
// that way by the multi-RHS kernel): out = psi(x) + sum of hops, no scaling.
template <int DAG, typename R, typename LoadNbr, typename Fwd, typename Bwd>
__device__ __forceinline__ void wilson_site_prescaled(const Nbr& n, int s, LoadNbr load, Fwd fl,
                                                      Bwd bl, Spinor<R>& out) {
    constexpr int SF = DAG ? 1 : -1;
    constexpr int SB = -SF;
    load(s, out);
    Spinor<R> nb;
#define SEEDCG_HOP(MU)                                                                          \
    {                                                                                           \
        auto lf = [&](int a, int b) { return fl(MU, 3 * a + b); };                              \
        auto lb = [&](int a, int b) { return bl(MU, 3 * a + b); };                              \
        load(n.f[MU], nb);                                                                      \
        hop<MU, SF, false, R, decltype(lf), false>(out, nb, lf, R(1));                          \
        load(n.b[MU], nb);                                                                      \
        hop<MU, SB, true, R, decltype(lb), false>(out, nb, lb, R(1));                           \
    }
    SEEDCG_HOP(0)
    SEEDCG_HOP(1)
    SEEDCG_HOP(2)
    SEEDCG_HOP(3)
#undef SEEDCG_HOP
}

// Same result as wilson_site_prescaled, written for a looser register budget:
// the forward and backward neighbours of each direction are loaded together and
// the next direction's pair is requested before the current one is consumed,
// so two to four spinors are in flight per thread instead of one.
template <int DAG, typename R, typename LoadNbr, typename Fwd, typename Bwd>
__device__ __forceinline__ void wilson_site_prescaled_pipe(const Nbr& n, int s, LoadNbr load, Fwd fl,
                                                           Bwd bl, Spinor<R>& out) {
    constexpr int SF = DAG ? 1 : -1;
    constexpr int SB = -SF;
    Spinor<R> pf, pb, qf, qb;
    load(n.f[0], pf);
    load(n.b[0], pb);
    load(s, out);
#define SEEDCG_HOP2(MU, CF, CB, NF, NB, NEXT)                                                   \
    {                                                                                           \
        auto lf = [&](int a, int b) { return fl(MU, 3 * a + b); };                              \
        auto lb = [&](int a, int b) { return bl(MU, 3 * a + b); };                              \
        if (NEXT) {                                                                             \
            load(n.f[(MU + 1) & 3], NF);                                                        \
            load(n.b[(MU + 1) & 3], NB);                                                        \
        }                                                                                       \
        hop<MU, SF, false, R, decltype(lf), false>(out, CF, lf, R(1));                          \
        hop<MU, SB, true, R, decltype(lb), false>(out, CB, lb, R(1));                           \
    }
    SEEDCG_HOP2(0, pf, pb, qf, qb, true)
    SEEDCG_HOP2(1, qf, qb, pf, pb, true)
    SEEDCG_HOP2(2, pf, pb, qf, qb, true)
    SEEDCG_HOP2(3, qf, qb, pf, pb, false)
#undef SEEDCG_HOP2
}

}  // namespace seedcg
