// Batched CG engine (the "standard CG" of Section 2 for every seeded system,
// run for all systems of all gauge fields at once).
//
// Every iteration is five launches whatever the number of fields or systems (seven
// for the even-odd system, whose operator is four parity-restricted hops):
//   1. one multi-field multi-RHS dslash  t = D p   (tiles of 32 sites of every
//      field; each tile stages its links once, scaled by -kappa and the
//      boundary sign, and applies them to all of the field's active systems),
//      with one share per warp of ||t||^2 = p^dag M p
//   2. alpha_j = ||r_j||^2 / ||D p_j||^2         (one block per system)
//   3. the same kernel for D^dag t, whose result q never leaves the registers:
//      r -= alpha q at the site, with one share per warp of the new ||r||^2
//   4. beta_j = ||r_j||^2 (new) / ||r_j||^2 (old) and the per-system flags
//   5. x += alpha p, p = r + beta p                (one pass over p for both)
// A chunk of `poll` iterations is captured once as a CUDA graph and replayed;
// the kernels read the active-system tables from device memory, so the graph
// stays valid while systems converge and are compacted away.  Between chunks
// the host reads the per-system flags, runs the FP64 reliable updates
// (x64 += x_R, r = b - M x64 in FP64) and compacts the active systems.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "cg_batch.cuh"
#include "eo.cuh"
#include "kernels.cuh"
#include "reduce.cuh"
#include "wilson.cuh"

namespace seedcg {

namespace {

constexpr int kMaxGroups = 16;
constexpr int TS = 32;       // sites per dslash tile (one warp per right-hand side)
// right-hand sides processed side by side per tile (warps per block): picked
// per batch by the autotuner below from {4, 8, 12}

// brick tiling of one field's lattice: Lx x by x bz sites at one t per tile
// (x neighbours always in the tile, most y and z neighbours too); n = 0 when
// the lattice admits no brick of that many sites
struct Brk {
    int bx, by, bz, ny, nz, n;
};

template <typename R>
struct GroupDev {
    Geom g;
    const cx_t<R>* u;   // links in the working precision
    R kappa;
    long n;             // 12 * sites (the volume, or half of it for the even-odd system)
    int eo;             // 1: M = A^dag A on odd-site half vectors (Section 3's system)
    cx_t<R>* e;         // [cap][n] even-site intermediate of the even-odd operator
    cx_t<R>* xr;        // [cap][n] iterate increments since the last reliable update
    cx_t<R>* r;
    cx_t<R>* p;
    cx_t<R>* t;
    double* part;       // [cap][ntiles] shares of ||D p||^2 = p^dag M p (||A p||^2 even-odd)
    double* part2;      // [cap][ntiles] shares of ||r||^2 after the update of step 3
    int ntiles;         // tiles of 32 (half-)sites; every share is one warp's sum
    int tile0;          // first tile of this group in the dslash grid
    Brk b64, b128;      // brick tilings of 64 and 128 sites (single-field full-lattice batches)
};

struct Rows {
    int* group;   // [rows_cap] group of the row, -1 when unused
    int* local;   // [rows_cap] system slot within its group
    int* nact;    // [kMaxGroups] active systems of each group (slots 0..nact-1)
    int* first;   // [kMaxGroups] row of slot 0 of each group (rows run in group order)
};

struct CgS {
    double* rr;
    double* rr_ru;
    double* alpha;
    double* beta;
    double* bn;
    int* active;
    int* flag;      // 0 none, 1 reliable update due, 2 converged (check), 3 stop
    int* iters;
    double* partials;
    unsigned* counters;
    double tol, delta2;
    int maxiter;
    int rows_cap;   // rows of every per-row array (grid of the per-row kernels)
};

__device__ __forceinline__ int find_group(int b, int ng, const int* tile0) {
    int f = 0;
    while (f + 1 < ng && b >= tile0[f + 1]) f++;
    return f;
}

// The two epilogues of the operator kernels (one thread = one site of one system):
// after D, the site's ||t||^2; after D^dag, r -= alpha q at the site and its new
// ||r||^2.  Each warp's sum (32 sites of one system) is one share, written to
// shares[slot * ntiles + tile32]; k_mf_alpha / k_mf_beta add a system's shares in
// a fixed order, so no block barrier is needed and the result is reproducible.
template <typename R>
__device__ __forceinline__ R r_update_site(cx_t<R>* rr, int vol, int s, const Spinor<R>& q, R a) {
    Spinor<R> v;
    load_spinor_rw(rr, vol, s, v);
    R acc = 0;
#pragma unroll
    for (int k = 0; k < 12; k++) {
        cx_t<R>& z = v.c[k / 3][k % 3];
        const cx_t<R> w = q.c[k / 3][k % 3];
        z.x -= a * w.x;
        z.y -= a * w.y;
        acc += z.x * z.x + z.y * z.y;
    }
    store_spinor(rr, vol, s, v);
    return acc;
}

__device__ __forceinline__ void put_share(double* shares, int ntiles, int slot, int tile32, float v) {
    const double d = (double)warp_sum_t(v);
    if ((threadIdx.x & 31) == 0) shares[(size_t)slot * ntiles + tile32] = d;
}
__device__ __forceinline__ void put_share(double* shares, int ntiles, int slot, int tile32, double v) {
    const double d = warp_sum_t(v);
    if ((threadIdx.x & 31) == 0) shares[(size_t)slot * ntiles + tile32] = d;
}

// ---------------------------------------------------------------------------
// 1/3: multi-field multi-RHS dslash (DAG = 0: t = D p and ||t||^2;
//      DAG = 1: q = D^dag t, r -= alpha q and ||r||^2)
// ---------------------------------------------------------------------------
template <typename R, int DAG, int RPB>
__global__ void __launch_bounds__(TS * RPB, (sizeof(R) == 4 ? (RPB <= 8 ? 3 : 2) : 1))
k_mf_dslash(const GroupDev<R>* __restrict__ G, int ng, Rows rows, CgS C) {
    __shared__ cx_t<R> sl[2][4][9][TS];
    __shared__ int sb[4][TS];
    __shared__ Nbr snb[TS];   // neighbours of the tile's sites (kept out of the registers)
    __shared__ R sgn[2][TS];
    __shared__ int s_tile0[kMaxGroups];
    if (threadIdx.x < ng) s_tile0[threadIdx.x] = G[threadIdx.x].tile0;
    __syncthreads();
    const int f = find_group(blockIdx.x, ng, s_tile0);
    const GroupDev<R>& gd = G[f];
    const int nsys = rows.nact[f];
    if (nsys == 0) return;
    const Geom g = gd.g;
    const int vol = g.vol;
    const int tile = blockIdx.x - gd.tile0;
    const int s0 = tile * TS;
    const R kappa = gd.kappa;
    if (threadIdx.x < TS) {
        const int s = s0 + threadIdx.x;
        if (s < vol) {
            Nbr nb = neighbours(g, s);
            snb[threadIdx.x] = nb;
#pragma unroll
            for (int mu = 0; mu < 4; mu++) sb[mu][threadIdx.x] = nb.b[mu];
            sgn[0][threadIdx.x] = nb.fwrap_t ? kappa : -kappa;
            sgn[1][threadIdx.x] = nb.bwrap_t ? kappa : -kappa;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 72 * TS; e += blockDim.x) {
        const int j = e % TS;
        const int c = (e / TS) % 9;
        const int mu = (e / (9 * TS)) % 4;
        const int dir = e / (36 * TS);
        const int s = s0 + j;
        cx_t<R> z = mk<R>(0, 0);
        if (s < vol) {
            z = __ldg(gd.u + (size_t)(mu * 9 + c) * vol + (dir ? sb[mu][j] : s));
            z = cscale(z, mu == 3 ? sgn[dir][j] : -kappa);
        }
        sl[dir][mu][c][j] = z;
    }
    __syncthreads();
    const int j = threadIdx.x % TS;   // lane = site of the tile
    const int qg = threadIdx.x / TS;  // warp = right-hand-side group
    const int s = s0 + j;
    const bool live = s < vol;
    const Nbr& nb = snb[j];
    auto fl = [&](int mu, int e) { return sl[0][mu][e][j]; };
    auto bl = [&](int mu, int e) { return sl[1][mu][e][j]; };
    const cx_t<R>* in = DAG ? gd.t : gd.p;
    for (int r = qg; r < nsys; r += RPB) {
        R dr = 0;
        if (live) {
            const cx_t<R>* inr = in + (size_t)r * gd.n;
            Spinor<R> res;
            auto load = [&](int y, Spinor<R>& sp) { load_spinor(inr, vol, y, sp); };
            wilson_site_prescaled<DAG, R>(nb, s, load, fl, bl, res);
            if (DAG) {
                dr = r_update_site(gd.r + (size_t)r * gd.n, vol, s, res, (R)C.alpha[rows.first[f] + r]);
            } else {
                dr = spinor_norm2(res);   // before the store: fewer live registers
                store_spinor(gd.t + (size_t)r * gd.n, vol, s, res);
            }
        }
        put_share(DAG ? gd.part2 : gd.part, gd.ntiles, r, tile, dr);
    }
}

// 1/3 for the even-odd system: M p = A^dag A p in four parity-restricted hops over
// every active system of every field (tiles of TS odd / even half sites):
//   STAGE 0  e = H_eo p;  1  t = p - kappa^2 H_oe e = A p, and ||A p||^2 = p^dag M p;
//   STAGE 2  e = H^dag_eo t;  3  q = t - kappa^2 H^dag_oe e, r -= alpha q and ||r||^2
// The tile's links (U_mu(x) and U_mu(x - mu) of its 32 sites of the output parity) are
// staged once in shared memory, times the hop coefficient (1, or -kappa^2 in stages 1
// and 3) and the t-boundary sign, and reused by every system of the tile.
template <typename R, int STAGE, int RPB>
__global__ void __launch_bounds__(TS * RPB, (sizeof(R) == 4 ? 2 : 1))
k_mf_eo(const GroupDev<R>* __restrict__ G, int ng, Rows rows, CgS C) {
    constexpr int DAG = STAGE >= 2 ? 1 : 0;
    constexpr int POUT = (STAGE & 1) ? 1 : 0;
    __shared__ cx_t<R> sl[2][4][9][TS];
    __shared__ int ssite[TS];
    __shared__ int sb[4][TS];                 // x - mu (full site)
    __shared__ Nbr snb[TS];                   // neighbours of the tile's sites
    __shared__ R sgn[2][TS];
    __shared__ int s_tile0[kMaxGroups];
    if (threadIdx.x < ng) s_tile0[threadIdx.x] = G[threadIdx.x].tile0;
    __syncthreads();
    const int f = find_group(blockIdx.x, ng, s_tile0);
    const GroupDev<R>& gd = G[f];
    const int nsys = rows.nact[f];
    if (nsys == 0) return;
    const Geom g = gd.g;
    const int vol = g.vol, vh = g.vol / 2;
    const int tile = blockIdx.x - gd.tile0;
    const R kk = gd.kappa * gd.kappa;
    const R chop = POUT ? -kk : R(1);
    if (threadIdx.x < TS) {
        const int h = tile * TS + threadIdx.x;
        if (h < vh) {
            const int s = eo_site(g, h, POUT);
            const Nbr nb = neighbours(g, s);
            ssite[threadIdx.x] = s;
            snb[threadIdx.x] = nb;
#pragma unroll
            for (int mu = 0; mu < 4; mu++) sb[mu][threadIdx.x] = nb.b[mu];
            sgn[0][threadIdx.x] = nb.fwrap_t ? -chop : chop;
            sgn[1][threadIdx.x] = nb.bwrap_t ? -chop : chop;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 72 * TS; e += blockDim.x) {
        const int j = e % TS;
        const int c = (e / TS) % 9;
        const int mu = (e / (9 * TS)) % 4;
        const int dir = e / (36 * TS);
        cx_t<R> z = mk<R>(0, 0);
        if (tile * TS + j < vh) {
            z = __ldg(gd.u + (size_t)(mu * 9 + c) * vol + (dir ? sb[mu][j] : ssite[j]));
            z = cscale(z, mu == 3 ? sgn[dir][j] : chop);
        }
        sl[dir][mu][c][j] = z;
    }
    __syncthreads();
    const int j = threadIdx.x % TS;
    const int qg = threadIdx.x / TS;
    const int hh = tile * TS + j;
    const bool live = hh < vh;
    const Nbr& nb = snb[j];
    auto fl = [&](int mu, int e) { return sl[0][mu][e][j]; };
    auto bl = [&](int mu, int e) { return sl[1][mu][e][j]; };
    const cx_t<R>* in = STAGE == 0 ? gd.p : STAGE == 2 ? gd.t : gd.e;
    const cx_t<R>* same = STAGE == 1 ? gd.p : STAGE == 3 ? gd.t : nullptr;
    cx_t<R>* out = (STAGE == 0 || STAGE == 2) ? gd.e : gd.t;   // STAGE 3 stores nothing
    for (int r = qg; r < nsys; r += RPB) {
        R dr = 0;
        if (live) {
            const size_t off = (size_t)r * gd.n;
            Spinor<R> acc;
            if (POUT) {
                load_spinor(same + off, vh, hh, acc);
            } else {
#pragma unroll
                for (int k = 0; k < 12; k++) acc.c[k / 3][k % 3] = mk<R>(0, 0);
            }
            eo_hops_prescaled<R, DAG>(nb, in + off, vh, fl, bl, acc);
            if (STAGE == 3) {
                dr = r_update_site(gd.r + off, vh, hh, acc, (R)C.alpha[rows.first[f] + r]);
            } else {
                if (STAGE == 1) dr = spinor_norm2(acc);
                store_spinor(out + off, vh, hh, acc);
            }
        }
        if (STAGE == 1 || STAGE == 3) put_share(STAGE == 1 ? gd.part : gd.part2, gd.ntiles, r, tile, dr);
    }
}

// 1/3 for a batch of one full-lattice field: the same two kernels over brick
// tiles of TB sites (TB / 32 warps per right-hand-side group, RPB groups per block).
// The brick's links (U_mu(x) and U_mu(x - mu), scaled by -kappa and the boundary
// sign) are staged once in shared memory and reused by every right-hand side;
// the neighbours in x (always) and mostly in y and z are sites of the same
// brick, so their spinor loads hit in L1.  The bricks tile the lattice, so the
// warps of brick b are the 32-site tiles b * TB / 32 ... of the shares.
template <typename R, int DAG, int TB, int RPB>
__global__ void __launch_bounds__(TB * RPB, (sizeof(R) == 4 && TB * RPB <= 256) ? 3 : 1)
k_mf_brick(const GroupDev<R>* __restrict__ G, Rows rows, CgS C) {
    extern __shared__ unsigned char smem_raw[];
    cx_t<R>* sl = reinterpret_cast<cx_t<R>*>(smem_raw);   // [2][4][9][TB]
    Nbr* snb = reinterpret_cast<Nbr*>(sl + 72 * TB);        // [TB] neighbours of the brick's sites
    int* ss = reinterpret_cast<int*>(snb + TB);             // [TB] site
    R* sg = reinterpret_cast<R*>(ss + TB);                  // [2][TB]
    const GroupDev<R>& gd = G[0];
    const int nsys = rows.nact[0];
    if (nsys == 0) return;
    const Brk br = TB == 64 ? gd.b64 : gd.b128;
    const Geom g = gd.g;
    const int vol = g.vol;
    const R kappa = gd.kappa;
    int b = blockIdx.x;
    const int iy = b % br.ny;
    b /= br.ny;
    const int iz = b % br.nz;
    const int t = b / br.nz;
    if (threadIdx.x < TB) {
        const int j = threadIdx.x;
        const int x = j % br.bx, dy = (j / br.bx) % br.by, dz = j / (br.bx * br.by);
        const int s = x + g.stride[1] * (iy * br.by + dy) + g.stride[2] * (iz * br.bz + dz) + g.stride[3] * t;
        ss[j] = s;
        const Nbr nb = neighbours(g, s);
        snb[j] = nb;
        sg[j] = nb.fwrap_t ? kappa : -kappa;
        sg[TB + j] = nb.bwrap_t ? kappa : -kappa;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 72 * TB; e += blockDim.x) {
        const int j = e % TB;
        const int c = (e / TB) % 9;
        const int mu = (e / (9 * TB)) % 4;
        const int dir = e / (36 * TB);
        const cx_t<R> z = __ldg(gd.u + (size_t)(mu * 9 + c) * vol + (dir ? snb[j].b[mu] : ss[j]));
        sl[e] = cscale(z, mu == 3 ? sg[dir * TB + j] : -kappa);
    }
    __syncthreads();
    const int j = threadIdx.x % TB;
    const int q = threadIdx.x / TB;
    const int s = ss[j];
    const int tile32 = blockIdx.x * (TB / 32) + (j >> 5);
    const Nbr& nb = snb[j];
    auto fl = [&](int mu, int e) { return sl[((0 * 4 + mu) * 9 + e) * TB + j]; };
    auto bl = [&](int mu, int e) { return sl[((1 * 4 + mu) * 9 + e) * TB + j]; };
    const cx_t<R>* in = DAG ? gd.t : gd.p;
    // a warp's 32 threads share one system: the loop bound is warp-uniform
    for (int r = q; r < nsys; r += RPB) {
        const cx_t<R>* inr = in + (size_t)r * gd.n;
        Spinor<R> res;
        auto load = [&](int y, Spinor<R>& sp) { load_spinor(inr, vol, y, sp); };
        wilson_site_prescaled<DAG, R>(nb, s, load, fl, bl, res);
        R dr;
        if (DAG) {
            dr = r_update_site(gd.r + (size_t)r * gd.n, vol, s, res, (R)C.alpha[rows.first[0] + r]);
        } else {
            dr = spinor_norm2(res);
            store_spinor(gd.t + (size_t)r * gd.n, vol, s, res);
        }
        put_share(DAG ? gd.part2 : gd.part, gd.ntiles, r, tile32, dr);
    }
}

// a row's shares, summed in a fixed order (one block per row); four independent
// partial sums per thread keep four loads in flight
__device__ __forceinline__ double row_shares(const double* __restrict__ sh, int ntiles) {
    const int bd = blockDim.x;
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
    int b = threadIdx.x;
    for (; b + 3 * bd < ntiles; b += 4 * bd) {
        v0 += sh[b];
        v1 += sh[b + bd];
        v2 += sh[b + 2 * bd];
        v3 += sh[b + 3 * bd];
    }
    for (; b < ntiles; b += bd) v0 += sh[b];
    double v[1] = {(v0 + v1) + (v2 + v3)};
    block_sum<1>(v);
    return v[0];
}

// 2: alpha = ||r||^2 / ||D p||^2 (one block per row)
template <typename R>
__global__ void __launch_bounds__(256)
k_mf_alpha(const GroupDev<R>* __restrict__ G, Rows rows, CgS C) {
    const int row = blockIdx.x;
    const int f = rows.group[row];
    if (f < 0) return;
    if (!C.active[row]) {
        // a system that stopped keeps its x and r: the updates of steps 3 and 5 add 0
        if (threadIdx.x == 0) C.alpha[row] = 0.0;
        return;
    }
    const GroupDev<R>& gd = G[f];
    const double den = row_shares(gd.part + (size_t)rows.local[row] * gd.ntiles, gd.ntiles);
    if (threadIdx.x == 0) C.alpha[row] = C.rr[row] / den;
}

// 4: beta = the new ||r||^2 over the old, and the per-row flags (one block per row)
template <typename R>
__global__ void __launch_bounds__(256)
k_mf_beta(const GroupDev<R>* __restrict__ G, Rows rows, CgS C) {
    const int row = blockIdx.x;
    const int f = rows.group[row];
    if (f < 0 || !C.active[row]) return;
    const GroupDev<R>& gd = G[f];
    const double rn = row_shares(gd.part2 + (size_t)rows.local[row] * gd.ntiles, gd.ntiles);
    if (threadIdx.x != 0) return;
    C.beta[row] = rn / C.rr[row];
    C.rr[row] = rn;
    C.iters[row] += 1;
    if (!isfinite(rn)) {
        C.flag[row] = 3;
        C.active[row] = 0;
    } else if (sqrt(rn) <= C.tol * C.bn[row]) {
        C.flag[row] = 2;
        C.active[row] = 0;
    } else if (C.iters[row] >= C.maxiter) {
        C.flag[row] = 3;
        C.active[row] = 0;
    } else if (C.delta2 > 0.0 && rn < C.delta2 * C.rr_ru[row]) {
        C.flag[row] = 1;
    }
}

// per-row grid reduction (grid = (blocks, rows); row = blockIdx.y)
template <int NV, typename Fin>
__device__ __forceinline__ void rowsum(double (&v)[NV], double* partials, unsigned* counters,
                                       Fin fin) {
    __shared__ bool s_last;
    block_sum<NV>(v);
    const unsigned nblk = gridDim.x, row = blockIdx.y;
    double* part = partials + (size_t)row * NV * nblk;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) part[(size_t)k * nblk + blockIdx.x] = v[k];
        __threadfence();
        unsigned t = atomicAdd(counters + row, 1u);
        s_last = (t == nblk - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double tot[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) tot[k] = 0.0;
    for (unsigned b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; k++) tot[k] += __ldcg(part + (size_t)k * nblk + b);
    block_sum<NV>(tot);
    if (threadIdx.x == 0) {
        fin(tot);
        counters[row] = 0u;
        __threadfence();
    }
}

// W consecutive complex entries in one 16-byte access (two in FP32, one in FP64;
// every vector length n = 12 * sites is even, and every vector starts 16-byte aligned)
template <typename R> struct Pack16;
template <> struct Pack16<float> {
    using T = float4;
    static constexpr int W = 2;
    __device__ __forceinline__ static void split(const float4& a, float2 (&o)[2]) {
        o[0] = make_float2(a.x, a.y);
        o[1] = make_float2(a.z, a.w);
    }
    __device__ __forceinline__ static float4 join(const float2 (&o)[2]) {
        return make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
    }
};
template <> struct Pack16<double> {
    using T = double2;
    static constexpr int W = 1;
    __device__ __forceinline__ static void split(const double2& a, double2 (&o)[1]) { o[0] = a; }
    __device__ __forceinline__ static double2 join(const double2 (&o)[1]) { return o[0]; }
};

// 5: x += alpha p and p = r + beta p in one pass over p.  Rows that stopped in
// this iteration's step 4 still take their last x update; rows stopped earlier
// have alpha = 0 (their p changes, but it is not used again).  16-byte accesses,
// two groups per thread and trip with all six loads issued first.
template <typename R>
__global__ void __launch_bounds__(kRedThreads)
k_mf_xp(const GroupDev<R>* __restrict__ G, Rows rows, CgS C) {
    using P = Pack16<R>;
    using T = typename P::T;
    constexpr int W = P::W;
    const int row = blockIdx.y;
    const int f = rows.group[row];
    if (f < 0) return;
    const GroupDev<R>& gd = G[f];
    const size_t off = (size_t)rows.local[row] * gd.n;
    T* __restrict__ x = reinterpret_cast<T*>(gd.xr + off);
    const T* __restrict__ r = reinterpret_cast<const T*>(gd.r + off);
    T* __restrict__ p = reinterpret_cast<T*>(gd.p + off);
    const R a = (R)C.alpha[row], b = (R)C.beta[row];
    const long ng = gd.n / W;
    const long st = (long)gridDim.x * blockDim.x;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < ng; e += 2 * st) {
        const long e2 = e + st;
        const bool two = e2 < ng;
        cx_t<R> pv[2][W], xv[2][W], rv[2][W];
        P::split(p[e], pv[0]);
        P::split(x[e], xv[0]);
        P::split(r[e], rv[0]);
        if (two) {
            P::split(p[e2], pv[1]);
            P::split(x[e2], xv[1]);
            P::split(r[e2], rv[1]);
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            if (h == 1 && !two) break;
#pragma unroll
            for (int k = 0; k < W; k++) {
                xv[h][k].x += a * pv[h][k].x;
                xv[h][k].y += a * pv[h][k].y;
                pv[h][k].x = rv[h][k].x + b * pv[h][k].x;
                pv[h][k].y = rv[h][k].y + b * pv[h][k].y;
            }
            x[h ? e2 : e] = P::join(xv[h]);
            p[h ? e2 : e] = P::join(pv[h]);
        }
    }
}

// reliable update of k = 0..nf-1 systems of one group: x64[sys] += x_R[slot]; x_R = 0;
// gather x64[sys] into Gx[k]
template <typename R>
__global__ void k_mf_ru_flush(const int* __restrict__ slot, const int* __restrict__ sys,
                              cx_t<R>* __restrict__ XR, double2* __restrict__ X64,
                              double2* __restrict__ Gx, long n) {
    const int k = blockIdx.y;
    cx_t<R>* xr = XR + (size_t)slot[k] * n;
    double2* x = X64 + (size_t)sys[k] * n;
    double2* gk = Gx + (size_t)k * n;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
        cx_t<R> d = xr[e];
        double2 xv = x[e];
        xv.x += (double)d.x;
        xv.y += (double)d.y;
        x[e] = xv;
        gk[e] = xv;
        xr[e] = mk<R>(0, 0);
    }
}

// r64 = b - (M x)[k]; r_R[slot] = r64; rr, rr_ru, true residual; active flag
template <typename R>
__global__ void __launch_bounds__(kRedThreads)
k_mf_ru_resid(const int* __restrict__ row_of, const int* __restrict__ slot,
              const int* __restrict__ sys, const double2* __restrict__ B64,
              const double2* __restrict__ MX, cx_t<R>* __restrict__ Rv, long n, CgS C,
              double* __restrict__ tr_out, double* partials, unsigned* counters) {
    const int k = blockIdx.y;
    const int row = row_of[k], q = slot[k], j = sys[k];
    const double2* b = B64 + (size_t)j * n;
    const double2* mx = MX + (size_t)k * n;
    cx_t<R>* r = Rv + (size_t)q * n;
    double part = 0.0;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
        double2 bv = b[e], mv = mx[e];
        double rx = bv.x - mv.x, ry = bv.y - mv.y;
        r[e] = mk<R>((R)rx, (R)ry);
        part += rx * rx + ry * ry;
    }
    double red[1] = {part};
    rowsum<1>(red, partials, counters, [&](double* tot) {
        const double rn = tot[0], bn = C.bn[row];
        C.rr[row] = rn;
        C.rr_ru[row] = rn;
        C.flag[row] = 0;
        // a non-finite b or residual is reported as such (never as converged) and the
        // system leaves the iteration: the caller sees it as not converged
        const bool finite = isfinite(rn) && isfinite(bn);
        tr_out[k] = !finite ? rn + bn : bn > 0.0 ? sqrt(rn) / bn : 0.0;
        C.active[row] = (finite && bn > 0.0 && sqrt(rn) > C.tol * bn) ? 1 : 0;
    });
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads)
k_norm_rows(const T* __restrict__ base, long n, double* partials, unsigned* counters,
            double* out) {
    const int k = blockIdx.y;
    const T* x = base + (size_t)k * n;
    double p = 0.0;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
        cx_t<double> z = ld_cx<double>(x, e);
        p += z.x * z.x + z.y * z.y;
    }
    double red[1] = {p};
    rowsum<1>(red, partials, counters, [&](double* tot) { out[k] = sqrt(tot[0]); });
}

// ---------------------------------------------------------------------------
// autotuner: the multi-field dslash's warps per tile (right-hand sides side by
// side) is timed with CUDA events on the batch's own vectors for each candidate
// and the fastest kept; results are cached in memory per batch signature and,
// when SEEDCG_TUNE_CACHE names a file, in that file ("key rpb" lines).
// ---------------------------------------------------------------------------
template <typename R>
void launch_mf(int rpb, int dag, int tiles, cudaStream_t s, const GroupDev<R>* gdev, int ng, Rows rows,
               const CgS& C) {
#define SEEDCG_MF(RP)                                                                          \
    if (dag) k_mf_dslash<R, 1, RP><<<tiles, TS * RP, 0, s>>>(gdev, ng, rows, C);               \
    else k_mf_dslash<R, 0, RP><<<tiles, TS * RP, 0, s>>>(gdev, ng, rows, C);
    if (rpb == 4) { SEEDCG_MF(4) }
    else if (rpb == 12) { SEEDCG_MF(12) }
    else { SEEDCG_MF(8) }
#undef SEEDCG_MF
    SEEDCG_CHECK_LAUNCH();
}

template <typename R>
void launch_mf_eo(int rpb, int stage, int tiles, cudaStream_t s, const GroupDev<R>* gdev, int ng, Rows rows,
                  const CgS& C) {
#define SEEDCG_MFE(RP)                                                                          \
    switch (stage) {                                                                           \
        case 0: k_mf_eo<R, 0, RP><<<tiles, TS * RP, 0, s>>>(gdev, ng, rows, C); break;         \
        case 1: k_mf_eo<R, 1, RP><<<tiles, TS * RP, 0, s>>>(gdev, ng, rows, C); break;         \
        case 2: k_mf_eo<R, 2, RP><<<tiles, TS * RP, 0, s>>>(gdev, ng, rows, C); break;         \
        default: k_mf_eo<R, 3, RP><<<tiles, TS * RP, 0, s>>>(gdev, ng, rows, C); break;        \
    }
    if (rpb == 4) { SEEDCG_MFE(4) }
    else if (rpb == 12) { SEEDCG_MFE(12) }
    else { SEEDCG_MFE(8) }
#undef SEEDCG_MFE
    SEEDCG_CHECK_LAUNCH();
}

template <typename R, int DAG, int TB, int RPB>
void brick_launch(int nb, cudaStream_t s, const GroupDev<R>* gdev, Rows rows, const CgS& C) {
    const size_t smem = (size_t)TB * (72 * sizeof(cx_t<R>) + sizeof(Nbr) + sizeof(int) + 2 * sizeof(R));
    static_assert(sizeof(Nbr) % 4 == 0 && (TB * (sizeof(Nbr) + sizeof(int))) % sizeof(R) == 0,
                  "brick shared-memory layout alignment");
    static bool attr = false;
    if (!attr) {
        SEEDCG_CUDA_TRY(cudaFuncSetAttribute(k_mf_brick<R, DAG, TB, RPB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    k_mf_brick<R, DAG, TB, RPB><<<nb, TB * RPB, smem, s>>>(gdev, rows, C);
    SEEDCG_CHECK_LAUNCH();
}

// Launch shape of the operator, chosen by the autotuner: codes 4, 8, 12 are the
// multi-field kernel with that many warps per tile of TS sites; code TB * 1000 +
// RPB is the brick kernel of TB sites with RPB right-hand-side groups (one field).
constexpr bool is_brick_code(int code) { return code >= 1000; }

// steps 1 and 3 of an iteration for every active system: 2 launches (D, D^dag)
// or 4 (even-odd hops); step 2 (alpha) runs between them in the iteration proper
template <typename R>
void launch_op(bool eo, int code, int tiles, const Brk& b64, const Brk& b128, cudaStream_t s,
               const GroupDev<R>* gdev, int ng, Rows rows, const CgS& C, bool with_alpha) {
    auto alpha = [&]() {
        if (!with_alpha) return;
        k_mf_alpha<R><<<C.rows_cap, 256, 0, s>>>(gdev, rows, C);
        SEEDCG_CHECK_LAUNCH();
    };
    if (eo) {
        for (int stage = 0; stage < 2; stage++) launch_mf_eo<R>(code, stage, tiles, s, gdev, ng, rows, C);
        alpha();
        for (int stage = 2; stage < 4; stage++) launch_mf_eo<R>(code, stage, tiles, s, gdev, ng, rows, C);
    } else if (is_brick_code(code)) {
#define SEEDCG_BRICK(TB, RP, BR)                                                               \
    brick_launch<R, 0, TB, RP>(BR.n, s, gdev, rows, C);                                        \
    alpha();                                                                                   \
    brick_launch<R, 1, TB, RP>(BR.n, s, gdev, rows, C);
        switch (code) {
            case 64004: SEEDCG_BRICK(64, 4, b64) break;
            case 64008: SEEDCG_BRICK(64, 8, b64) break;
            case 128002: SEEDCG_BRICK(128, 2, b128) break;
            default: SEEDCG_BRICK(128, 4, b128) break;
        }
#undef SEEDCG_BRICK
    } else {
        launch_mf<R>(code, 0, tiles, s, gdev, ng, rows, C);
        alpha();
        launch_mf<R>(code, 1, tiles, s, gdev, ng, rows, C);
    }
}

int largest_divisor_le(int L, int cap) {
    int best = 1;
    for (int d = 1; d <= L && d <= cap; d++)
        if (L % d == 0) best = d;
    return best;
}

// the brick of about `cap` sites for g: Lx x by x bz, by preferring a share of
// the y extent before z (n = 0 when it does not come to exactly TB sites)
Brk brick_for(const Geom& g, int tb) {
    Brk b{};
    b.bx = g.L[0];
    if (b.bx > 64 || b.bx > tb) return b;
    b.by = largest_divisor_le(g.L[1], (tb / 2 > b.bx ? tb / 2 : tb) / b.bx);
    b.bz = largest_divisor_le(g.L[2], tb / (b.bx * b.by));
    if (b.bx * b.by * b.bz != tb) return Brk{};
    b.ny = g.L[1] / b.by;
    b.nz = g.L[2] / b.bz;
    b.n = b.ny * b.nz * g.L[3];
    return b;
}

std::string tune_key(const std::vector<CgGroup>& groups, bool fp64) {
    std::string k = fp64 ? "mf_dslash f64" : "mf_dslash f32";
    if (!groups.empty() && groups[0].h->eo_active) k += " eo";
    for (auto& g : groups) {
        char b[96];
        snprintf(b, sizeof(b), " %dx%dx%dx%d:%d", g.h->g.L[0], g.h->g.L[1], g.h->g.L[2], g.h->g.L[3], g.nsys);
        k += b;
    }
    cudaDeviceProp p;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaGetDeviceProperties(&p, dev) == cudaSuccess) k += std::string(" ") + p.name;
    for (auto& c : k) if (c == ' ') c = '_';
    return k;
}

// the process-wide table of tuned warps per tile (guarded by tune_mutex); the
// optional SEEDCG_TUNE_CACHE file is shared with the brick-dslash tuner, so only
// its "mf_dslash..." lines are read here
std::mutex& tune_mutex() {
    static std::mutex m;
    return m;
}

std::vector<std::pair<std::string, int>>& tune_table() {
    static std::vector<std::pair<std::string, int>> t;
    static bool loaded = false;
    if (!loaded) {
        loaded = true;
        const char* path = getenv("SEEDCG_TUNE_CACHE");
        if (path) {
            FILE* f = fopen(path, "r");
            if (f) {
                char line[640], key[512];
                int v;
                while (fgets(line, sizeof(line), f))
                    if (sscanf(line, "%511s %d", key, &v) == 2 && strncmp(key, "mf_dslash", 9) == 0)
                        t.push_back({key, v});
                fclose(f);
            }
        }
    }
    return t;
}

template <typename R>
int autotune_rpb(const std::vector<CgGroup>& groups, int tiles, const Brk& b64, const Brk& b128,
                 const GroupDev<R>* gdev, int ng, Rows rows, const CgS& C, cudaStream_t st) {
    const std::string key = tune_key(groups, sizeof(R) == 8);
    {
        std::lock_guard<std::mutex> lk(tune_mutex());
        for (auto& e : tune_table())
            if (e.first == key) return e.second;
    }
    const bool eo = groups[0].h->eo_active;
    std::vector<int> cands{4, 8, 12};
    if (!eo && ng == 1) {
        if (b64.n) cands.insert(cands.end(), {64004, 64008});
        if (b128.n) cands.insert(cands.end(), {128002, 128004});
    }
    cudaEvent_t a, b;
    SEEDCG_CUDA_TRY(cudaEventCreate(&a));
    SEEDCG_CUDA_TRY(cudaEventCreate(&b));
    int best = 8;
    float best_ms = 1e30f;
    const bool tune_log = getenv("SEEDCG_TUNE_LOG") != nullptr;
    for (int c : cands) {
        // alpha is zero here: the D^dag kernel rewrites r unchanged, as it would for a
        // stopped system, so the candidates are timed on the whole of steps 1 and 3
        launch_op<R>(eo, c, tiles, b64, b128, st, gdev, ng, rows, C, false);  // warm-up
        SEEDCG_CUDA_TRY(cudaEventRecord(a, st));
        for (int r = 0; r < 3; r++) launch_op<R>(eo, c, tiles, b64, b128, st, gdev, ng, rows, C, false);
        SEEDCG_CUDA_TRY(cudaEventRecord(b, st));
        SEEDCG_CUDA_TRY(cudaEventSynchronize(b));
        float ms = 0.f;
        SEEDCG_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
        if (tune_log) fprintf(stderr, "seedcg tune %s: code %d: %.4f ms\n", key.c_str(), c, ms / 3);
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    std::lock_guard<std::mutex> lk(tune_mutex());
    tune_table().push_back({key, best});
    if (const char* path = getenv("SEEDCG_TUNE_CACHE")) {
        FILE* f = fopen(path, "a");
        if (f) {
            fprintf(f, "%s %d\n", key.c_str(), best);
            fclose(f);
        }
    }
    return best;
}

struct Carve2 {
    char* base;
    size_t off = 0;
    template <typename T> T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = reinterpret_cast<T*>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

}  // namespace

template <typename R>
void batched_cg(std::vector<CgGroup>& groups, double tol, double reliable_delta, int maxiter,
                int poll, bool use_graph, DevBuf& ws, void* pinned, CgResult& out,
                cudaStream_t st) {
    const int ng = (int)groups.size();
    if (ng < 1 || ng > kMaxGroups) throw Error{SEEDCG_ERR_ARG, "1..16 gauge fields per batch"};
    const bool fp64 = sizeof(R) == 8;
    const size_t cxR = sizeof(cx_t<R>);
    const bool eo = groups[0].h->eo_active;
    for (auto& gr : groups)
        if (gr.h->eo_active != eo) throw Error{SEEDCG_ERR_ARG, "a batch mixes even-odd and full systems"};
    // sites of a system's vectors: the lattice, or its odd half for the even-odd system
    auto nsites = [&](const CgGroup& gr) { return eo ? gr.h->g.vol / 2 : gr.h->g.vol; };
    int rows_cap = 0, tiles = 0, nsys_max = 0;
    long nmax = 0;
    for (auto& gr : groups) {
        rows_cap += gr.nsys;
        tiles += (nsites(gr) + TS - 1) / TS;
        nsys_max = std::max(nsys_max, gr.nsys);
        nmax = std::max(nmax, 12L * nsites(gr));
    }
    if (rows_cap > 512) throw Error{SEEDCG_ERR_ARG, "at most 512 systems per batch"};
    const int rblocks = (int)std::min<long>((nmax + kRedThreads * 4 - 1) / (kRedThreads * 4), 152 * 8);

    // ---- workspace ----
    size_t need = 1 << 16;
    auto add = [&](size_t b) { need += (b + 255) & ~(size_t)255; };
    for (auto& gr : groups) {
        const long n = 12L * nsites(gr);
        for (int k = 0; k < (eo ? 5 : 4); k++) add((size_t)gr.nsys * n * cxR);   // x_R, r, p, t (+ e)
        for (int k = 0; k < 2; k++) add((size_t)gr.nsys * n * sizeof(double2));
        add((size_t)std::max(gr.nsys, 2) * n * sizeof(double2));
        for (int k = 0; k < 2; k++) add((size_t)gr.nsys * ((nsites(gr) + TS - 1) / TS) * sizeof(double));
    }
    add(sizeof(int) * 2 * kMaxGroups);
    add(sizeof(GroupDev<R>) * kMaxGroups);
    add(sizeof(double) * 8 * rows_cap + sizeof(int) * 8 * rows_cap);
    const size_t part_doubles = (size_t)rblocks * (rows_cap + 2) * 2 + 4096;
    add(part_doubles * sizeof(double));
    add(sizeof(unsigned) * (rows_cap + 64));
    ws.ensure(need);
    Carve2 cv{ws.as<char>()};
    std::vector<GroupDev<R>> gd(ng);
    std::vector<double2*> Gx(ng), MX(ng), T64(ng);
    int tile0 = 0;
    for (int f = 0; f < ng; f++) {
        seedcg_handle* h = groups[f].h;
        const long n = 12L * nsites(groups[f]);
        const int ns = groups[f].nsys;
        gd[f].g = h->g;
        gd[f].u = fp64 ? reinterpret_cast<const cx_t<R>*>(h->u64.p) : reinterpret_cast<const cx_t<R>*>(h->u32.p);
        gd[f].kappa = (R)h->kappa;
        gd[f].n = n;
        gd[f].eo = eo ? 1 : 0;
        gd[f].xr = cv.take<cx_t<R>>((size_t)ns * n);
        gd[f].r = cv.take<cx_t<R>>((size_t)ns * n);
        gd[f].p = cv.take<cx_t<R>>((size_t)ns * n);
        gd[f].t = cv.take<cx_t<R>>((size_t)ns * n);
        gd[f].e = eo ? cv.take<cx_t<R>>((size_t)ns * n) : nullptr;
        Gx[f] = cv.take<double2>((size_t)ns * n);
        MX[f] = cv.take<double2>((size_t)ns * n);
        T64[f] = cv.take<double2>((size_t)std::max(ns, 2) * n);
        gd[f].ntiles = (nsites(groups[f]) + TS - 1) / TS;
        gd[f].b64 = (ng == 1 && !eo) ? brick_for(h->g, 64) : Brk{};
        gd[f].b128 = (ng == 1 && !eo) ? brick_for(h->g, 128) : Brk{};
        // the brick kernels write one share per warp of 32 sites: the bricks must tile
        // the lattice exactly, so that their warps are the ntiles site tiles
        if ((gd[f].b64.n && gd[f].b64.n * 2 != gd[f].ntiles) ||
            (gd[f].b128.n && gd[f].b128.n * 4 != gd[f].ntiles))
            throw Error{SEEDCG_ERR_ARG, "internal: bricks do not tile the lattice"};
        gd[f].part = cv.take<double>((size_t)ns * gd[f].ntiles);
        gd[f].part2 = cv.take<double>((size_t)ns * gd[f].ntiles);
        gd[f].tile0 = tile0;
        tile0 += gd[f].ntiles;
        SEEDCG_CUDA_TRY(cudaMemsetAsync(gd[f].xr, 0, (size_t)ns * n * cxR, st));
    }
    GroupDev<R>* gdev = cv.take<GroupDev<R>>(kMaxGroups);
    CgS C;
    C.rr = cv.take<double>(rows_cap);
    C.rr_ru = cv.take<double>(rows_cap);
    C.alpha = cv.take<double>(rows_cap);
    C.beta = cv.take<double>(rows_cap);
    C.bn = cv.take<double>(rows_cap);
    double* trd = cv.take<double>(rows_cap);
    C.active = cv.take<int>(rows_cap);
    C.flag = cv.take<int>(rows_cap);
    C.iters = cv.take<int>(rows_cap);
    Rows rows;
    rows.group = cv.take<int>(rows_cap);
    rows.local = cv.take<int>(rows_cap);
    rows.nact = cv.take<int>(kMaxGroups);
    rows.first = cv.take<int>(kMaxGroups);
    int* ru_row = cv.take<int>(rows_cap);
    int* ru_slot = cv.take<int>(rows_cap);
    int* ru_sys = cv.take<int>(rows_cap);
    C.partials = cv.take<double>(part_doubles);
    C.counters = cv.take<unsigned>(rows_cap + 64);
    C.tol = tol;
    C.delta2 = reliable_delta > 0.0 ? reliable_delta * reliable_delta : 0.0;
    C.maxiter = maxiter;
    C.rows_cap = rows_cap;
    SEEDCG_CUDA_TRY(cudaMemsetAsync(C.counters, 0, sizeof(unsigned) * (rows_cap + 64), st));
    SEEDCG_CUDA_TRY(cudaMemsetAsync(C.iters, 0, sizeof(int) * rows_cap, st));
    SEEDCG_CUDA_TRY(cudaMemsetAsync(C.flag, 0, sizeof(int) * rows_cap, st));
    SEEDCG_CUDA_TRY(cudaMemsetAsync(C.alpha, 0, sizeof(double) * rows_cap, st));   // the autotuner's runs
    SEEDCG_CUDA_TRY(cudaMemcpyAsync(gdev, gd.data(), sizeof(GroupDev<R>) * ng, cudaMemcpyHostToDevice, st));

    // pinned host scratch (ints)
    int* pin = reinterpret_cast<int*>(pinned);
    double* pind = reinterpret_cast<double*>(pin + 4096);

    // ---- host mirror of the active systems ----
    std::vector<std::vector<int>> sysmap(ng);   // group -> slot -> system
    out.iters.assign(ng, {});
    out.ru.assign(ng, {});
    out.notconv.assign(ng, {});
    out.true_resid.assign(ng, {});
    for (int f = 0; f < ng; f++) {
        sysmap[f].resize(groups[f].nsys);
        for (int j = 0; j < groups[f].nsys; j++) sysmap[f][j] = j;
        out.iters[f].assign(groups[f].nsys, 0);
        out.ru[f].assign(groups[f].nsys, 0);
        out.notconv[f].assign(groups[f].nsys, 0);
        out.true_resid[f].assign(groups[f].nsys, 0.0);
    }
    std::vector<int> row0(ng);
    auto upload_rows = [&]() {
        // rows in group order, slots 0..nact-1 of each group
        std::vector<int> rg(rows_cap, -1), rl(rows_cap, 0), na(kMaxGroups, 0), fr(kMaxGroups, 0);
        int r = 0;
        for (int f = 0; f < ng; f++) {
            row0[f] = r;
            fr[f] = r;
            na[f] = (int)sysmap[f].size();
            for (int l = 0; l < na[f]; l++, r++) {
                rg[r] = f;
                rl[r] = l;
            }
        }
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(rows.group, rg.data(), sizeof(int) * rows_cap, cudaMemcpyHostToDevice, st));
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(rows.local, rl.data(), sizeof(int) * rows_cap, cudaMemcpyHostToDevice, st));
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(rows.nact, na.data(), sizeof(int) * kMaxGroups, cudaMemcpyHostToDevice, st));
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(rows.first, fr.data(), sizeof(int) * kMaxGroups, cudaMemcpyHostToDevice, st));
        SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
        return r;
    };
    int nrows = upload_rows();

    // ||b|| per system
    for (int f = 0; f < ng; f++) {
        const long n = gd[f].n;
        dim3 gr(rblocks, groups[f].nsys);
        k_norm_rows<double2><<<gr, kRedThreads, 0, st>>>(groups[f].b64, n, C.partials, C.counters,
                                                          C.bn + row0[f]);
        SEEDCG_CHECK_LAUNCH();
    }

    // reliable update of a set of rows (grouped by field); returns nothing,
    // leaves the new active flags in pin[2048..]
    auto reliable = [&](const std::vector<int>& rset) {
        std::vector<std::vector<int>> byg(ng);
        for (int r : rset) {
            int f = 0;
            while (f + 1 < ng && r >= row0[f + 1]) f++;
            byg[f].push_back(r);
        }
        for (int f = 0; f < ng; f++) {
            const int nf = (int)byg[f].size();
            if (!nf) continue;
            const long n = gd[f].n;
            seedcg_handle* h = groups[f].h;
            for (int k = 0; k < nf; k++) {
                const int r = byg[f][k], l = r - row0[f];
                pin[k] = r;
                pin[512 + k] = l;
                pin[1024 + k] = sysmap[f][l];
            }
            SEEDCG_CUDA_TRY(cudaMemcpyAsync(ru_row, pin, sizeof(int) * nf, cudaMemcpyHostToDevice, st));
            SEEDCG_CUDA_TRY(cudaMemcpyAsync(ru_slot, pin + 512, sizeof(int) * nf, cudaMemcpyHostToDevice, st));
            SEEDCG_CUDA_TRY(cudaMemcpyAsync(ru_sys, pin + 1024, sizeof(int) * nf, cudaMemcpyHostToDevice, st));
            dim3 gr(rblocks, nf);
            k_mf_ru_flush<R><<<gr, kRedThreads, 0, st>>>(ru_slot, ru_sys, gd[f].xr, groups[f].x64, Gx[f], n);
            SEEDCG_CHECK_LAUNCH();
            if (eo) {
                eo_apply_mdag_m_f64(h->g, h->u64.as<double2>(), h->kappa, nf, Gx[f], T64[f], T64[f] + n,
                                    MX[f], st);
            } else {
                dslash_mrhs_f64(h->g, h->u64.as<double2>(), h->kappa, 0, nf, Gx[f], T64[f], st);
                dslash_mrhs_f64(h->g, h->u64.as<double2>(), h->kappa, 1, nf, T64[f], MX[f], st);
            }
            k_mf_ru_resid<R><<<gr, kRedThreads, 0, st>>>(ru_row, ru_slot, ru_sys, groups[f].b64, MX[f],
                                                         gd[f].r, n, C, trd, C.partials, C.counters);
            SEEDCG_CHECK_LAUNCH();
            SEEDCG_CUDA_TRY(cudaMemcpyAsync(pind, trd, sizeof(double) * nf, cudaMemcpyDeviceToHost, st));
            SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
            for (int k = 0; k < nf; k++) {
                const int l = byg[f][k] - row0[f];
                out.true_resid[f][sysmap[f][l]] = pind[k];
                out.ru[f][sysmap[f][l]] += 1;
                out.reliable_updates++;
            }
        }
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(pin + 2048, C.active, sizeof(int) * rows_cap, cudaMemcpyDeviceToHost, st));
        SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
    };

    // compact: keep the active rows of every group at the front of its slots
    auto compact = [&](const std::vector<int>& act) {
        std::vector<double> rr(rows_cap), rru(rows_cap), bn(rows_cap);
        std::vector<int> it(rows_cap);
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(rr.data(), C.rr, sizeof(double) * rows_cap, cudaMemcpyDeviceToHost, st));
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(rru.data(), C.rr_ru, sizeof(double) * rows_cap, cudaMemcpyDeviceToHost, st));
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(bn.data(), C.bn, sizeof(double) * rows_cap, cudaMemcpyDeviceToHost, st));
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(it.data(), C.iters, sizeof(int) * rows_cap, cudaMemcpyDeviceToHost, st));
        SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
        std::vector<double> nrr, nru, nbn;
        std::vector<std::vector<int>> nmap(ng);
        for (int f = 0; f < ng; f++) {
            const long n = gd[f].n;
            int k = 0;
            for (int l = 0; l < (int)sysmap[f].size(); l++) {
                const int r = row0[f] + l;
                out.iters[f][sysmap[f][l]] += it[r];
                if (!act[r]) continue;
                if (l != k) {
                    SEEDCG_CUDA_TRY(cudaMemcpyAsync(gd[f].xr + (size_t)k * n, gd[f].xr + (size_t)l * n, n * cxR, cudaMemcpyDeviceToDevice, st));
                    SEEDCG_CUDA_TRY(cudaMemcpyAsync(gd[f].r + (size_t)k * n, gd[f].r + (size_t)l * n, n * cxR, cudaMemcpyDeviceToDevice, st));
                    SEEDCG_CUDA_TRY(cudaMemcpyAsync(gd[f].p + (size_t)k * n, gd[f].p + (size_t)l * n, n * cxR, cudaMemcpyDeviceToDevice, st));
                }
                nmap[f].push_back(sysmap[f][l]);
                nrr.push_back(rr[r]);
                nru.push_back(rru[r]);
                nbn.push_back(bn[r]);
                k++;
            }
        }
        sysmap = nmap;
        const int nk = (int)nrr.size();
        std::vector<int> zeros(std::max(nk, 1), 0), ones(std::max(nk, 1), 1);
        if (nk > 0) {
            SEEDCG_CUDA_TRY(cudaMemcpyAsync(C.rr, nrr.data(), sizeof(double) * nk, cudaMemcpyHostToDevice, st));
            SEEDCG_CUDA_TRY(cudaMemcpyAsync(C.rr_ru, nru.data(), sizeof(double) * nk, cudaMemcpyHostToDevice, st));
            SEEDCG_CUDA_TRY(cudaMemcpyAsync(C.bn, nbn.data(), sizeof(double) * nk, cudaMemcpyHostToDevice, st));
            SEEDCG_CUDA_TRY(cudaMemcpyAsync(C.iters, zeros.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, st));
            SEEDCG_CUDA_TRY(cudaMemcpyAsync(C.flag, zeros.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, st));
            SEEDCG_CUDA_TRY(cudaMemcpyAsync(C.active, ones.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, st));
        }
        // rows past the active ones are switched off
        std::vector<int> off(rows_cap, 0);
        if (rows_cap > nk)
            SEEDCG_CUDA_TRY(cudaMemcpyAsync(C.active + nk, off.data(), sizeof(int) * (rows_cap - nk), cudaMemcpyHostToDevice, st));
        SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
        return upload_rows();
    };

    // ---- start: true residual of every seeded guess ----
    {
        std::vector<int> all(nrows);
        for (int r = 0; r < nrows; r++) all[r] = r;
        reliable(all);
        for (int f = 0; f < ng; f++)
            SEEDCG_CUDA_TRY(cudaMemcpyAsync(gd[f].p, gd[f].r, (size_t)groups[f].nsys * gd[f].n * cxR,
                                            cudaMemcpyDeviceToDevice, st));
        std::vector<int> act(pin + 2048, pin + 2048 + rows_cap);
        nrows = compact(act);
    }

    // ---- the iteration chunk (graph-captured) ----
    const int gx = rblocks;
    const Brk b64 = gd[0].b64, b128 = gd[0].b128;
    const int rpb = nrows > 0 ? autotune_rpb<R>(groups, tiles, b64, b128, gdev, ng, rows, C, st) : 8;
    out.rpb = rpb;
    auto chunk = [&](cudaStream_t s) {
        for (int it = 0; it < poll; it++) {
            launch_op<R>(eo, rpb, tiles, b64, b128, s, gdev, ng, rows, C, true);   // steps 1-3
            k_mf_beta<R><<<rows_cap, 256, 0, s>>>(gdev, rows, C);
            SEEDCG_CHECK_LAUNCH();
            k_mf_xp<R><<<dim3(gx, rows_cap), kRedThreads, 0, s>>>(gdev, rows, C);
            SEEDCG_CHECK_LAUNCH();
        }
    };
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cs = nullptr;
    if (use_graph && nrows > 0) {
        SEEDCG_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph;
        const unsigned long long before = g_kernel_launches.load();
        SEEDCG_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        chunk(cs);
        SEEDCG_CUDA_TRY(cudaStreamEndCapture(cs, &graph));
        g_kernel_launches.store(before);  // capturing launches nothing; replays are counted
        SEEDCG_CUDA_TRY(cudaGraphInstantiate(&gexec, graph, 0));
        SEEDCG_CUDA_TRY(cudaGraphDestroy(graph));
    }
    cudaEvent_t ev = nullptr;
    if (gexec) SEEDCG_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    while (nrows > 0) {
        if (gexec) {
            // keep stream order: st -> graph on cs -> st
            SEEDCG_CUDA_TRY(cudaEventRecord(ev, st));
            SEEDCG_CUDA_TRY(cudaStreamWaitEvent(cs, ev, 0));
            SEEDCG_CUDA_TRY(cudaGraphLaunch(gexec, cs));
            g_kernel_launches.fetch_add((unsigned long long)(eo ? 7 : 5) * poll, std::memory_order_relaxed);
            SEEDCG_CUDA_TRY(cudaEventRecord(ev, cs));
            SEEDCG_CUDA_TRY(cudaStreamWaitEvent(st, ev, 0));
            out.graph_chunks++;
        } else {
            chunk(st);
        }
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(pin, C.flag, sizeof(int) * rows_cap, cudaMemcpyDeviceToHost, st));
        SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
        std::vector<int> flags(pin, pin + rows_cap);
        // the device counts iterations since the last compaction; enforce the total cap here
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(pin + 3072, C.iters, sizeof(int) * rows_cap, cudaMemcpyDeviceToHost, st));
        SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
        for (int f = 0; f < ng; f++)
            for (int l = 0; l < (int)sysmap[f].size(); l++) {
                const int r = row0[f] + l;
                if (!flags[r] && out.iters[f][sysmap[f][l]] + pin[3072 + r] >= maxiter) flags[r] = 3;
            }
        std::vector<int> fl;
        for (int r = 0; r < nrows; r++)
            if (flags[r]) fl.push_back(r);
        if (fl.empty()) continue;
        reliable(fl);
        std::vector<int> act(pin + 2048, pin + 2048 + rows_cap);
        bool changed = false;
        for (int r : fl) {
            int f = 0;
            while (f + 1 < ng && r >= row0[f + 1]) f++;
            const int l = r - row0[f];
            if (flags[r] == 3) {
                out.notconv[f][sysmap[f][l]] = 1;
                act[r] = 0;
            } else if (flags[r] == 2 && act[r]) {
                // the iterated residual converged but the true one did not: restart
                SEEDCG_CUDA_TRY(cudaMemcpyAsync(gd[f].p + (size_t)l * gd[f].n, gd[f].r + (size_t)l * gd[f].n,
                                                gd[f].n * cxR, cudaMemcpyDeviceToDevice, st));
            }
        }
        for (int r = 0; r < nrows; r++) changed |= !act[r];
        if (changed) nrows = compact(act);
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (ev) cudaEventDestroy(ev);
    if (cs) cudaStreamDestroy(cs);
}

template void batched_cg<double>(std::vector<CgGroup>&, double, double, int, int, bool, DevBuf&, void*, CgResult&, cudaStream_t);
template void batched_cg<float>(std::vector<CgGroup>&, double, double, int, int, bool, DevBuf&, void*, CgResult&, cudaStream_t);

}  // namespace seedcg
