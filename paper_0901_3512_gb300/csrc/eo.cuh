// Even-odd (red-black) site indexing and the parity-restricted hopping term,
// shared by the even-odd operator kernels, the even-odd Lanczos kernels and the
// batched CG on half vectors (Section 3 solves the even-odd preconditioned
// system A^dag A x_o = A^dag phi, A = 1 - kappa^2 H_oe H_eo).
//
// A half-lattice vector holds the sites of one parity in lexicographic order.
// With every extent even, the pair of sites (2h, 2h + 1) holds one site of each
// parity, so half index h and full site s satisfy h = s >> 1.  Half vectors use
// the internal spinor layout of full ones with V/2 sites.
#pragma once

#include "internal.cuh"
#include "wilson.cuh"

namespace seedcg {

// full site of half index h with parity p (p = (x + y + z + t) mod 2)
__device__ __forceinline__ int eo_site(const Geom& g, int h, int p) {
    const int s0 = 2 * h;                       // x of s0 is even (Lx is even)
    const int r = s0 / g.L[0];
    const int y = r % g.L[1], z = (r / g.L[1]) % g.L[2], t = r / (g.L[1] * g.L[2]);
    return s0 + (((y + z + t) ^ p) & 1);
}

// acc += c_hop * (H other)(s): the eight hops of D = 1 - kappa H (DAG: of D^dag)
// from site s, whose neighbours all have the opposite parity and are read from
// the half vector `other` at index >> 1; the antiperiodic sign on hops that wrap t
template <typename R, int DAG>
__device__ __forceinline__ void eo_hops(const Geom& g, const cx_t<R>* __restrict__ u, int s, const Nbr& nb,
                                        const cx_t<R>* __restrict__ other, R c_hop, Spinor<R>& acc) {
    const int vol = g.vol, vh = g.vol / 2;
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
}

// acc += (H other)(s) with links that already carry the hop coefficient and the
// t-boundary sign (staged that way by the batched CG's tile kernels): no scaling.
// Fwd(mu, e) / Bwd(mu, e) give element e = 3a+b of U_mu(s) / U_mu(s - mu).
template <typename R, int DAG, typename Fwd, typename Bwd>
__device__ __forceinline__ void eo_hops_prescaled(const Nbr& nb, const cx_t<R>* __restrict__ other, int vh,
                                                  Fwd fl, Bwd bl, Spinor<R>& acc) {
    constexpr int SF = DAG ? 1 : -1;
    constexpr int SB = -SF;
    Spinor<R> p;
#define SEEDCG_EO_HOP_P(MU)                                                                          \
    {                                                                                                \
        auto lf = [&](int a, int b) { return fl(MU, 3 * a + b); };                                   \
        auto lb = [&](int a, int b) { return bl(MU, 3 * a + b); };                                   \
        load_spinor(other, vh, nb.f[MU] >> 1, p);                                                    \
        hop<MU, SF, false, R, decltype(lf), false>(acc, p, lf, R(1));                                \
        load_spinor(other, vh, nb.b[MU] >> 1, p);                                                    \
        hop<MU, SB, true, R, decltype(lb), false>(acc, p, lb, R(1));                                 \
    }
    SEEDCG_EO_HOP_P(0)
    SEEDCG_EO_HOP_P(1)
    SEEDCG_EO_HOP_P(2)
    SEEDCG_EO_HOP_P(3)
#undef SEEDCG_EO_HOP_P
}

// out(h) = c_diag same(h) + c_hop (H other)(x), x the parity-p_out site of half index h
// (same may be null: no diagonal term)
template <typename R, int DAG>
__device__ __forceinline__ void eo_site_apply(const Geom& g, const cx_t<R>* __restrict__ u, int p_out, int h,
                                              const cx_t<R>* __restrict__ other,
                                              const cx_t<R>* __restrict__ same, R c_diag, R c_hop,
                                              Spinor<R>& acc) {
    const int vh = g.vol / 2;
    const int s = eo_site(g, h, p_out);
    const Nbr nb = neighbours(g, s);
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
    eo_hops<R, DAG>(g, u, s, nb, other, c_hop, acc);
}

}  // namespace seedcg
