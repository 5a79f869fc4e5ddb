// Learned initial guess: a gauge-covariant nearest-neighbour network
//   out_co(x) = sum_ci [ W_0[co,ci] in_ci(x) + sum_{d=+-mu} W_d[co,ci] U(x,d) in_ci(x+d) ]
// (U(x,+mu) = U_mu(x), U(x,-mu) = U_mu(x-mu)^dag, antiperiodic-t sign as in D;
// W_d[co,ci] a complex 4x4 spin matrix; channels 1 -> 8 -> 8 -> 1; ReLU on real
// and imaginary parts after layers 1 and 2; input b/||b||, output times ||b||),
// with hand-written forward, backward and Adam kernels.
//
// Storage is bf16, accumulation FP32: activations, their gradients and the
// weights the layers read are bf16; Adam keeps an FP32 master copy of the
// weights and FP32 moments, and the weight gradient is summed in FP64.
//
// Layer 2 (8 -> 8) is a dense contraction with K = 9 directions x 8 channels x 4
// spins = 288 complex terms per output, run on the tcgen05 tensor cores as the
// real GEMM  D[site][n] = sum_k A[site][k] B[n][k]  per colour:
//   A = the link-transported neighbour activations of 128 sites (built by the CTA
//       in shared memory, one direction d per 64-wide K chunk),
//   B = the layer's weights in real form (64 x 64 bf16 per direction),
//   D = 128 x 64 FP32 accumulators in TMEM, one per colour.
// The backward pass through the data of layer 2 is the same GEMM with the
// adjoint transport and the adjoint weights.  Layers 1 and 3 (one channel on one
// side) and the weight gradients run on SIMT.
//
// Activations are bf16x2 [C][V][12] (entry k = 3 spin + colour of site x at
// (c V + x) 12 + k); weights of a layer are [9][CO][CI][4][4] complex, directions
// 0 (on site), +x,-x,+y,-y,+z,-z,+t,-t.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "handle.cuh"
#include "kernels.cuh"
#include "reduce.cuh"
#include "tc_common.cuh"
#include "wilson.cuh"

namespace seedcg {

namespace {

using bf2 = __nv_bfloat162;
constexpr int kG = 256;

// ---------------------------------------------------------------------------
// bf16 site records: the 12 complex entries of one channel at one site, 48 bytes
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 unpack_bf2(unsigned w) {
    bf2 b;
    memcpy(&b, &w, 4);
    return __bfloat1622float2(b);
}
__device__ __forceinline__ unsigned pack_bf2(float2 v) {
    const bf2 b = __float22bfloat162_rn(v);
    unsigned w;
    memcpy(&w, &b, 4);
    return w;
}
__device__ __forceinline__ void ld_site(const bf2* __restrict__ p, float2 (&o)[12]) {
    const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const uint4 a = __ldg(q + j);
        o[4 * j + 0] = unpack_bf2(a.x);
        o[4 * j + 1] = unpack_bf2(a.y);
        o[4 * j + 2] = unpack_bf2(a.z);
        o[4 * j + 3] = unpack_bf2(a.w);
    }
}
__device__ __forceinline__ void st_site(bf2* __restrict__ p, const float2 (&v)[12]) {
    uint4* q = reinterpret_cast<uint4*>(p);
#pragma unroll
    for (int j = 0; j < 3; j++)
        q[j] = make_uint4(pack_bf2(v[4 * j]), pack_bf2(v[4 * j + 1]), pack_bf2(v[4 * j + 2]), pack_bf2(v[4 * j + 3]));
}
__device__ __forceinline__ const bf2* site_ptr(const bf2* a, int ch, int vol, int x) {
    return a + ((size_t)ch * vol + x) * 12;
}
__device__ __forceinline__ bf2* site_ptr(bf2* a, int ch, int vol, int x) {
    return a + ((size_t)ch * vol + x) * 12;
}

// U(x,d) applied to colour vector v (3 complex), with the boundary sign
__device__ __forceinline__ void apply_link(const float2* __restrict__ u, int vol, int x, int d,
                                           const Nbr& nb, const float2 v[3], float2 o[3]) {
    const int mu = (d - 1) >> 1;
    const bool back = (d - 1) & 1;
    const float sg = (mu == 3 && (back ? nb.bwrap_t : nb.fwrap_t)) ? -1.f : 1.f;
    const int site = back ? nb.b[mu] : x;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < 3; b++) {
            if (!back) {
                const float2 uu = __ldg(u + (size_t)(mu * 9 + 3 * a + b) * vol + site);
                acc = cfma(uu, v[b], acc);
            } else {
                const float2 uu = __ldg(u + (size_t)(mu * 9 + 3 * b + a) * vol + site);
                acc = cfma_conj(uu, v[b], acc);
            }
        }
        o[a] = make_float2(sg * acc.x, sg * acc.y);
    }
}

// The adjoint transport used by the backward pass through the data: the
// contribution to site y of direction d comes from site z (y - mu for +mu,
// y + mu for -mu) and is carried by U_mu(z)^dag (+mu) or U_mu(y) (-mu), with the
// sign of the hop from z in direction d.
struct AdjHop {
    int z;
    float sg;
};
__device__ __forceinline__ AdjHop adj_hop(int y, int d, const Nbr& nb) {
    if (d == 0) return AdjHop{y, 1.f};
    const int mu = (d - 1) >> 1;
    const bool back = (d - 1) & 1;
    AdjHop h;
    h.z = back ? nb.f[mu] : nb.b[mu];
    h.sg = (mu == 3 && (back ? nb.fwrap_t : nb.bwrap_t)) ? -1.f : 1.f;
    return h;
}
__device__ __forceinline__ void apply_link_adj(const float2* __restrict__ u, int vol, int y, int d,
                                               const AdjHop& hp, const float2 v[3], float2 o[3]) {
    const int mu = (d - 1) >> 1;
    const bool back = (d - 1) & 1;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < 3; b++) {
            if (!back) {  // U_mu(z)^dag, z = y - mu
                const float2 uu = __ldg(u + (size_t)(mu * 9 + 3 * b + a) * vol + hp.z);
                acc = cfma_conj(uu, v[b], acc);
            } else {      // U_mu(y)
                const float2 uu = __ldg(u + (size_t)(mu * 9 + 3 * a + b) * vol + y);
                acc = cfma(uu, v[b], acc);
            }
        }
        o[a] = make_float2(hp.sg * acc.x, hp.sg * acc.y);
    }
}

// gathered input g_d(x) of one channel: 4 spins x 3 colours
__device__ __forceinline__ void gather(const float2* __restrict__ u, const bf2* __restrict__ in_ch, int vol,
                                       int x, int d, const Nbr& nb, float2 g[4][3]) {
    float2 v[12];
    if (d == 0) {
        ld_site(in_ch + (size_t)x * 12, v);
#pragma unroll
        for (int k = 0; k < 12; k++) g[k / 3][k % 3] = v[k];
        return;
    }
    const int mu = (d - 1) >> 1;
    const int y = ((d - 1) & 1) ? nb.b[mu] : nb.f[mu];
    ld_site(in_ch + (size_t)y * 12, v);
#pragma unroll
    for (int s = 0; s < 4; s++) apply_link(u, vol, x, d, nb, &v[3 * s], g[s]);
}

// ---------------------------------------------------------------------------
// SIMT layers (one channel on one side): forward, one thread per (site, co)
// ---------------------------------------------------------------------------
template <int CI, int CO>
__global__ void __launch_bounds__(kG)
k_g_fwd(Geom gm, const float2* __restrict__ u, const bf2* __restrict__ W, const bf2* __restrict__ in,
        bf2* __restrict__ z, bf2* __restrict__ h, int relu) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const int vol = gm.vol;
    if (t >= (long)vol * CO) return;
    const int co = (int)(t / vol), x = (int)(t % vol);
    const Nbr nb = neighbours(gm, x);
    float2 acc[4][3];
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
        for (int c = 0; c < 3; c++) acc[s][c] = make_float2(0.f, 0.f);
    for (int d = 0; d < 9; d++) {
        for (int ci = 0; ci < CI; ci++) {
            float2 g[4][3];
            gather(u, in + (size_t)ci * vol * 12, vol, x, d, nb, g);
            const bf2* w = W + (((size_t)d * CO + co) * CI + ci) * 16;
#pragma unroll
            for (int s = 0; s < 4; s++)
#pragma unroll
                for (int sp = 0; sp < 4; sp++) {
                    const float2 ww = __bfloat1622float2(w[4 * s + sp]);
#pragma unroll
                    for (int c = 0; c < 3; c++) acc[s][c] = cfma(ww, g[sp][c], acc[s][c]);
                }
        }
    }
    float2 v[12], r[12];
#pragma unroll
    for (int k = 0; k < 12; k++) {
        v[k] = acc[k / 3][k % 3];
        r[k] = make_float2(fmaxf(v[k].x, 0.f), fmaxf(v[k].y, 0.f));
    }
    st_site(site_ptr(z, co, vol, x), v);
    if (relu) st_site(site_ptr(h, co, vol, x), r);
}

// backward through the data of a layer with CO = 1: din[ci](y) = sum_d adjoint
// transport of W_d^dag dout (one thread per (site, ci)), times the ReLU mask of zprev
template <int CI, int CO>
__global__ void __launch_bounds__(kG)
k_g_bwd_data(Geom gm, const float2* __restrict__ u, const bf2* __restrict__ W, const bf2* __restrict__ dout,
             const bf2* __restrict__ zprev, bf2* __restrict__ din) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const int vol = gm.vol;
    if (t >= (long)vol * CI) return;
    const int ci = (int)(t / vol), y = (int)(t % vol);
    const Nbr nb = neighbours(gm, y);
    float2 acc[4][3];
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
        for (int c = 0; c < 3; c++) acc[s][c] = make_float2(0.f, 0.f);
    for (int d = 0; d < 9; d++) {
        const AdjHop hp = adj_hop(y, d, nb);
        float2 dg[4][3];
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < 3; c++) dg[s][c] = make_float2(0.f, 0.f);
        for (int co = 0; co < CO; co++) {
            float2 dv[12];
            ld_site(site_ptr(dout, co, vol, hp.z), dv);
            const bf2* w = W + (((size_t)d * CO + co) * CI + ci) * 16;
#pragma unroll
            for (int s = 0; s < 4; s++)
#pragma unroll
                for (int sp = 0; sp < 4; sp++) {
                    const float2 ww = __bfloat1622float2(w[4 * s + sp]);
#pragma unroll
                    for (int c = 0; c < 3; c++) dg[sp][c] = cfma_conj(ww, dv[3 * s + c], dg[sp][c]);
                }
        }
        if (d == 0) {
#pragma unroll
            for (int s = 0; s < 4; s++)
#pragma unroll
                for (int c = 0; c < 3; c++) acc[s][c] = cadd(acc[s][c], dg[s][c]);
        } else {
#pragma unroll
            for (int s = 0; s < 4; s++) {
                float2 o[3];
                apply_link_adj(u, vol, y, d, hp, dg[s], o);
#pragma unroll
                for (int c = 0; c < 3; c++) acc[s][c] = cadd(acc[s][c], o[c]);
            }
        }
    }
    float2 v[12], zz[12];
    ld_site(site_ptr(zprev, ci, vol, y), zz);
#pragma unroll
    for (int k = 0; k < 12; k++) {
        const float2 a = acc[k / 3][k % 3];
        v[k] = make_float2(zz[k].x > 0.f ? a.x : 0.f, zz[k].y > 0.f ? a.y : 0.f);
    }
    st_site(site_ptr(din, ci, vol, y), v);
}

// backward to the weights: dW[d][co][ci][s][s'] = sum_{x,c} dout[co](x)[s][c] conj(g_d(a_ci)(x)[s'][c])
// block (d, slice of sites); the slice's gathered inputs and output gradients are
// staged in shared memory 32 sites at a time; each thread owns output entries and
// accumulates over the slice; partials [slice][9][CO][CI][16]
template <int CI, int CO>
__global__ void __launch_bounds__(kG)
k_g_bwd_w(Geom gm, const float2* __restrict__ u, const bf2* __restrict__ a, const bf2* __restrict__ dout,
          int sites_per_slice, float2* __restrict__ part) {
    constexpr int S = 32;
    constexpr int NO = CO * CI * 16;
    __shared__ float2 sg[S][3][CI * 4];   // [site][colour][ci*4 + s']
    __shared__ float2 sd[S][3][CO * 4];   // [site][colour][co*4 + s]
    const int d = blockIdx.x;
    const int slice = blockIdx.y;
    const int vol = gm.vol;
    const int x0 = slice * sites_per_slice;
    const int x1 = min(x0 + sites_per_slice, vol);
    constexpr int PER = (NO + kG - 1) / kG;
    float2 acc[PER];
#pragma unroll
    for (int k = 0; k < PER; k++) acc[k] = make_float2(0.f, 0.f);
    for (int xs = x0; xs < x1; xs += S) {
        const int cnt = min(S, x1 - xs);
        __syncthreads();
        for (int w = threadIdx.x; w < S * (CI + CO); w += blockDim.x) {
            const int j = w % S, ch = w / S;
            const int x = xs + j;
            if (j >= cnt) continue;
            const Nbr nb = neighbours(gm, x);
            if (ch < CI) {
                float2 g[4][3];
                gather(u, a + (size_t)ch * vol * 12, vol, x, d, nb, g);
#pragma unroll
                for (int s = 0; s < 4; s++)
#pragma unroll
                    for (int c = 0; c < 3; c++) sg[j][c][ch * 4 + s] = g[s][c];
            } else {
                const int co = ch - CI;
                float2 dv[12];
                ld_site(site_ptr(dout, co, vol, x), dv);
#pragma unroll
                for (int k = 0; k < 12; k++) sd[j][k % 3][co * 4 + k / 3] = dv[k];
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; k++) {
            const int o = threadIdx.x + k * kG;
            if (o < NO) {
                // o = ((co*CI + ci)*4 + s)*4 + sp
                const int sp = o % 4, s = (o / 4) % 4, ci = (o / 16) % CI, co = o / (16 * CI);
                float2 v = acc[k];
                for (int j = 0; j < cnt; j++)
#pragma unroll
                    for (int c = 0; c < 3; c++)
                        v = cfma_conj(sg[j][c][ci * 4 + sp], sd[j][c][co * 4 + s], v);
                acc[k] = v;
            }
        }
    }
    float2* out = part + ((size_t)slice * 9 + d) * NO;
#pragma unroll
    for (int k = 0; k < PER; k++) {
        const int o = threadIdx.x + k * kG;
        if (o < NO) out[o] = acc[k];
    }
}

// grad[e] += sum over slices of part[slice][e]  (e over 9*NO entries), in FP64
__global__ void k_g_reduce_w(const float2* __restrict__ part, int nslice, int ne,
                             double2* __restrict__ grad) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    double re = 0.0, im = 0.0;
    for (int p = 0; p < nslice; p++) {
        const float2 z = part[(size_t)p * ne + e];
        re += z.x;
        im += z.y;
    }
    grad[e].x += re;
    grad[e].y += im;
}

// ---------------------------------------------------------------------------
// layer 2 on tcgen05 (see the file header).  One CTA = 128 sites, 256 threads.
// MODE 0 (forward):  A = U(x,d) h1_ci(x+d), B = W in real form; epilogue z2, h2 = ReLU(z2).
// MODE 1 (backward through the data): A = adjoint transport of d2_co, B = W^dag in
//        real form; epilogue d1 = D masked by z1 > 0 (real and imaginary parts).
// K of direction d: k = (ch * 4 + spin) * 2 + {re, im} over the 8 channels of the
// input side; N: n = (ch' * 4 + spin') * 2 + {re, im} over the output side.
// ---------------------------------------------------------------------------
constexpr int TC_SITES = 128;
constexpr uint32_t TC_A_BYTES = TC_SITES * 128;      // 128 rows x 64 bf16
constexpr uint32_t TC_B_BYTES = 64 * 128;            // 64 rows x 64 bf16
constexpr uint32_t TC_SMEM = 2 * 3 * TC_A_BYTES + 2 * TC_B_BYTES + 1024 + 256;
constexpr uint32_t TC_TMEM_COLS = 256;               // 3 colours x 64 columns

// byte offset of (row r, 16-byte chunk j) in a K-major 128-byte-swizzled tile
__device__ __forceinline__ uint32_t sw128(int r, int j) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) << 4));
}

template <int MODE>
__global__ void __launch_bounds__(256, 1)
k_g_tc(Geom gm, const float2* __restrict__ u, const bf2* __restrict__ in, const uint4* __restrict__ wimg,
       const bf2* __restrict__ zprev, bf2* __restrict__ out0, bf2* __restrict__ out1, int* __restrict__ err) {
    using namespace tc;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;                                   // [2 buffers][3 colours][TC_A_BYTES]
    uint8_t* sB = smem + 2 * 3 * TC_A_BYTES;              // [2 buffers][TC_B_BYTES]
    uint64_t* done = reinterpret_cast<uint64_t*>(sB + 2 * TC_B_BYTES);   // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 2);
    volatile int* s_fail = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int vol = gm.vol;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = blockIdx.x * TC_SITES;
    if (threadIdx.x == 0) {
        mbar_init(&done[0], 1);
        mbar_init(&done[1], 1);
        *s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem_d = *tmem_slot;

    // this thread's site and half of the input channels
    const int row = threadIdx.x & (TC_SITES - 1);
    const int half = threadIdx.x >> 7;
    const int x = x0 + row;
    const bool live = x < vol;
    Nbr nb;
    if (live) nb = neighbours(gm, x);
    int issued = 0;   // MMA groups committed (one per direction)
    for (int d = 0; d < 9; d++) {
        const int b = d & 1;
        if (d >= 2) {
            // the MMAs that read buffer b (direction d - 2) must be done before it is refilled
            if (!mbar_wait(&done[b], (uint32_t)((d - 2) >> 1) & 1u)) *s_fail = 1;
        }
        __syncthreads();
        if (*s_fail) break;
        // B: this direction's weights (a ready 128-byte-swizzled image)
        {
            const uint4* src = wimg + (size_t)d * (TC_B_BYTES / 16);
            uint4* dst = reinterpret_cast<uint4*>(sB + b * TC_B_BYTES);
            for (int i = threadIdx.x; i < (int)(TC_B_BYTES / 16); i += blockDim.x) dst[i] = __ldg(src + i);
        }
        // A: the transported activations of channels [4 half, 4 half + 4) at this site
        float2 lk[9];   // the link of this direction at this site (already with its sign)
        int src_site = x;
        float sgn = 1.f;
        bool dag = false;   // apply the link's adjoint
        if (live && d > 0) {
            const int mu = (d - 1) >> 1;
            const bool back = (d - 1) & 1;
            int lsite;
            if (MODE == 0) {
                src_site = back ? nb.b[mu] : nb.f[mu];
                lsite = back ? nb.b[mu] : x;
                dag = back;
                sgn = (mu == 3 && (back ? nb.bwrap_t : nb.fwrap_t)) ? -1.f : 1.f;
            } else {
                src_site = back ? nb.f[mu] : nb.b[mu];
                lsite = back ? x : nb.b[mu];
                dag = !back;
                sgn = (mu == 3 && (back ? nb.fwrap_t : nb.bwrap_t)) ? -1.f : 1.f;
            }
#pragma unroll
            for (int e = 0; e < 9; e++) lk[e] = __ldg(u + (size_t)(mu * 9 + e) * vol + lsite);
        }
#pragma unroll 1
        for (int q = 0; q < 4; q++) {
            const int ch = 4 * half + q;
            float2 v[12];
            if (live) {
                ld_site(site_ptr(in, ch, vol, src_site), v);
            } else {
#pragma unroll
                for (int k = 0; k < 12; k++) v[k] = make_float2(0.f, 0.f);
            }
            float2 g[4][3];
#pragma unroll
            for (int s = 0; s < 4; s++) {
                if (d == 0 || !live) {
#pragma unroll
                    for (int c = 0; c < 3; c++) g[s][c] = v[3 * s + c];
                } else {
#pragma unroll
                    for (int a = 0; a < 3; a++) {
                        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                        for (int c = 0; c < 3; c++)
                            acc = dag ? cfma_conj(lk[3 * c + a], v[3 * s + c], acc) : cfma(lk[3 * a + c], v[3 * s + c], acc);
                        g[s][a] = make_float2(sgn * acc.x, sgn * acc.y);
                    }
                }
            }
            // colour c of this (site, channel): 4 spins x (re, im) = 16 bytes, chunk ch of the row
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const uint4 w = make_uint4(pack_bf2(g[0][c]), pack_bf2(g[1][c]), pack_bf2(g[2][c]), pack_bf2(g[3][c]));
                *reinterpret_cast<uint4*>(sA + (b * 3 + c) * TC_A_BYTES + sw128(row, ch)) = w;
            }
        }
        // the tensor cores read shared memory through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            constexpr uint32_t idesc = umma_idesc_bf16(64, 128);
            const uint32_t b0 = smem_u32(sB + b * TC_B_BYTES);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const uint32_t a0 = smem_u32(sA + (b * 3 + c) * TC_A_BYTES);
#pragma unroll
                for (int kk = 0; kk < 4; kk++)
                    umma_bf16(tmem_d + (uint32_t)(c * 64), umma_desc_sw128(a0 + kk * 32), umma_desc_sw128(b0 + kk * 32),
                              idesc, (d > 0 || kk > 0) ? 1u : 0u);
            }
            umma_commit(&done[b]);
        }
        issued = d + 1;
    }
    // the last group's completion covers every earlier MMA of this CTA
    if (issued > 0) {
        const int dl = issued - 1;
        if (!mbar_wait(&done[dl & 1], (uint32_t)(dl >> 1) & 1u)) *s_fail = 1;
    }
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (*s_fail || issued < 9) {
        if (threadIdx.x == 0) atomicExch(err, SEEDCG_ERR_TIMEOUT);
    } else if (warp < 4) {
        // warp w reads TMEM lanes [32 w, 32 w + 32): the rows (sites) of its threads
        const int r = warp * 32 + lane;
        const int xs = x0 + r;
        for (int o = 0; o < 8; o++) {
            float cv[3][8];
#pragma unroll
            for (int c = 0; c < 3; c++)
                tmem_ld8(tmem_d + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 64 + o * 8), cv[c]);
            if (xs < vol) {
                float2 z[12];
#pragma unroll
                for (int s = 0; s < 4; s++)
#pragma unroll
                    for (int c = 0; c < 3; c++) z[3 * s + c] = make_float2(cv[c][2 * s], cv[c][2 * s + 1]);
                if (MODE == 0) {
                    float2 hr[12];
#pragma unroll
                    for (int k = 0; k < 12; k++) hr[k] = make_float2(fmaxf(z[k].x, 0.f), fmaxf(z[k].y, 0.f));
                    st_site(site_ptr(out0, o, vol, xs), z);
                    st_site(site_ptr(out1, o, vol, xs), hr);
                } else {
                    float2 zz[12];
                    ld_site(site_ptr(zprev, o, vol, xs), zz);
#pragma unroll
                    for (int k = 0; k < 12; k++)
                        z[k] = make_float2(zz[k].x > 0.f ? z[k].x : 0.f, zz[k].y > 0.f ? z[k].y : 0.f);
                    st_site(site_ptr(out0, o, vol, xs), z);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_d), "r"(TC_TMEM_COLS));
    }
}

// The B operands of layer 2 as 128-byte-swizzled bf16 images, one 64 x 64 tile per
// direction: forward B[n = (co,s,p)][k = (ci,s',q)] and adjoint B[n = (ci,s',p)][k = (co,s,q)]
// (p, q: 0 real, 1 imaginary), from the FP32 master weights W2[9][8][8][4][4].
__global__ void k_g_wform(const float2* __restrict__ W2, uint8_t* __restrict__ fwd, uint8_t* __restrict__ adj) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;   // one thread per (d, n, k)
    if (t >= 9 * 64 * 64) return;
    const int k = t % 64, n = (t / 64) % 64, d = t / 4096;
    const int q = k & 1, kk = k >> 1, p = n & 1, nn = n >> 1;
    // forward: n -> (co, s), k -> (ci, s')
    {
        const int co = nn >> 2, s = nn & 3, ci = kk >> 2, sp = kk & 3;
        const float2 w = W2[(((size_t)d * 8 + co) * 8 + ci) * 16 + s * 4 + sp];
        const float v = p == 0 ? (q == 0 ? w.x : -w.y) : (q == 0 ? w.y : w.x);
        *reinterpret_cast<unsigned short*>(fwd + (size_t)d * TC_B_BYTES + sw128(n, k >> 3) + (k & 7) * 2) =
            __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
    // adjoint: n -> (ci, s'), k -> (co, s); din = sum conj(W) dout'
    {
        const int ci = nn >> 2, sp = nn & 3, co = kk >> 2, s = kk & 3;
        const float2 w = W2[(((size_t)d * 8 + co) * 8 + ci) * 16 + s * 4 + sp];
        const float v = p == 0 ? (q == 0 ? w.x : w.y) : (q == 0 ? -w.y : w.x);
        *reinterpret_cast<unsigned short*>(adj + (size_t)d * TC_B_BYTES + sw128(n, k >> 3) + (k & 7) * 2) =
            __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
}

// ---------------------------------------------------------------------------
// input, output, loss, Adam
// ---------------------------------------------------------------------------
// internal paired-layout index of entry k of site s
__device__ __forceinline__ size_t pidx(int s, int k, int vol) {
    return ((size_t)(k >> 1) * vol + s) * 2 + (k & 1);
}

// a0 = b / ||b|| in bf16 [V][12]
__global__ void k_g_scale_in(const double2* __restrict__ b, const double* __restrict__ nb, bf2* __restrict__ a0,
                             int vol) {
    const double inv = 1.0 / *nb;
    for (long o = blockIdx.x * (long)blockDim.x + threadIdx.x; o < 12L * vol; o += (long)gridDim.x * blockDim.x) {
        const int s = (int)(o / 12), k = (int)(o % 12);
        const double2 z = b[pidx(s, k, vol)];
        a0[o] = __float22bfloat162_rn(make_float2((float)(z.x * inv), (float)(z.y * inv)));
    }
}

// x0 = ||b|| z3 (FP64 internal layout)
__global__ void k_g_scale_out(const bf2* __restrict__ z3, const double* __restrict__ nb, double2* __restrict__ x0,
                              int vol) {
    const double s = *nb;
    for (long o = blockIdx.x * (long)blockDim.x + threadIdx.x; o < 12L * vol; o += (long)gridDim.x * blockDim.x) {
        const int st = (int)(o / 12), k = (int)(o % 12);
        const float2 z = __bfloat1622float2(z3[o]);
        x0[pidx(st, k, vol)] = make_double2(s * z.x, s * z.y);
    }
}

// loss term ||y - x||^2 / ||x||^2 / nbatch with y = ||b|| z3, and dz3 = ||b|| * 2 (y - x) / ||x||^2 / nbatch
__global__ void __launch_bounds__(kRedThreads)
k_g_loss(const bf2* __restrict__ z3, const double2* __restrict__ x, const double* __restrict__ nb,
         const double* __restrict__ nx, double inv_batch, bf2* __restrict__ dz3, int vol,
         double* partials, unsigned* ctr, double* loss_acc) {
    const double s = *nb, xn2 = (*nx) * (*nx);
    double part = 0.0;
    for (long o = blockIdx.x * (long)blockDim.x + threadIdx.x; o < 12L * vol; o += (long)gridDim.x * blockDim.x) {
        const int st = (int)(o / 12), k = (int)(o % 12);
        const float2 z = __bfloat1622float2(z3[o]);
        const double2 xv = x[pidx(st, k, vol)];
        const double rx = s * z.x - xv.x, ry = s * z.y - xv.y;
        part += rx * rx + ry * ry;
        const double f = s * 2.0 * inv_batch / xn2;
        dz3[o] = __float22bfloat162_rn(make_float2((float)(f * rx), (float)(f * ry)));
    }
    double red[1] = {part};
    grid_sum<1>(red, partials, ctr, [&](double* tot) { *loss_acc += tot[0] / xn2 * inv_batch; });
}

// Adam on real and imaginary parts: FP32 master weights and moments, FP64 gradient;
// the bf16 copy the layers read is refreshed in the same pass
__global__ void k_g_adam(float2* __restrict__ W, bf2* __restrict__ Wb, const double2* __restrict__ g,
                         float2* __restrict__ m, float2* __restrict__ v, int ne, float lr, float b1, float b2,
                         float eps, float c1, float c2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const float gx = (float)g[e].x, gy = (float)g[e].y;
    float2 mm = m[e], vv = v[e], w = W[e];
    mm.x = b1 * mm.x + (1.f - b1) * gx;
    mm.y = b1 * mm.y + (1.f - b1) * gy;
    vv.x = b2 * vv.x + (1.f - b2) * gx * gx;
    vv.y = b2 * vv.y + (1.f - b2) * gy * gy;
    w.x -= lr * (mm.x / c1) / (sqrtf(vv.x / c2) + eps);
    w.y -= lr * (mm.y / c1) / (sqrtf(vv.y / c2) + eps);
    m[e] = mm;
    v[e] = vv;
    W[e] = w;
    Wb[e] = __float22bfloat162_rn(w);
}

__global__ void k_g_round(const float2* __restrict__ W, bf2* __restrict__ Wb, int ne) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < ne) Wb[e] = __float22bfloat162_rn(W[e]);
}

inline int gblocks(long n) { return (int)((n + kG - 1) / kG); }

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct GuessState {
    static constexpr int NW1 = 9 * 8 * 1 * 16, NW2 = 9 * 8 * 8 * 16, NW3 = 9 * 1 * 8 * 16;
    static constexpr int NW = NW1 + NW2 + NW3;
    DevBuf w;       // float2 [NW] master weights
    DevBuf wb;      // bf16x2 [NW] the weights the layers read
    DevBuf wimg;    // layer-2 B operands: forward and adjoint images, 9 x 8 KB each
    DevBuf adam;    // m, v float2 [NW] each
    DevBuf grad;    // double2 [NW]
    DevBuf act;     // activations and gradients (bf16)
    DevBuf part;    // weight-gradient partials
    DevBuf scal;    // norms, loss, the tensor-core error flag
    int steps = 0;
    bool have_weights = false;
};

GuessState* guess_state(seedcg_handle* h) {
    if (!h->guess) h->guess = new GuessState();
    return reinterpret_cast<GuessState*>(h->guess);
}

bool guess_ready(const seedcg_handle* h) {
    return h->guess && reinterpret_cast<const GuessState*>(h->guess)->have_weights;
}

void guess_free(seedcg_handle* h) {
    if (h->guess) {
        GuessState* g = reinterpret_cast<GuessState*>(h->guess);
        delete g;   // every DevBuf frees its allocation
        h->guess = nullptr;
    }
}

namespace {

struct Acts {
    bf2 *a0, *z1, *h1, *z2, *h2, *z3, *d3, *d2, *d1;
    double* nb;
    double* nx;
    double* loss;
    int* tc_err;
};

Acts carve_acts(GuessState* G, int vol) {
    const size_t site = (size_t)vol * 12;   // bf16x2 entries of one channel
    const size_t need = site * (1 + 8 * 4 + 1 + 1 + 8 * 2) * sizeof(bf2) + 4096;
    G->act.ensure(need);
    G->scal.ensure(64 * sizeof(double) + 8192 * sizeof(double) + 8192 * sizeof(unsigned));
    bf2* p = G->act.as<bf2>();
    Acts A;
    A.a0 = p; p += site;
    A.z1 = p; p += 8 * site;
    A.h1 = p; p += 8 * site;
    A.z2 = p; p += 8 * site;
    A.h2 = p; p += 8 * site;
    A.z3 = p; p += site;
    A.d3 = p; p += site;
    A.d2 = p; p += 8 * site;
    A.d1 = p; p += 8 * site;
    A.nb = G->scal.as<double>();
    A.nx = A.nb + 1;
    A.loss = A.nb + 2;
    A.tc_err = reinterpret_cast<int*>(A.nb + 3);
    return A;
}

// layer 2 on the tensor cores (mode 0 forward, 1 backward through the data)
void layer2_tc(seedcg_handle* h, GuessState* G, int mode, const bf2* in, const bf2* zprev, bf2* out0, bf2* out1,
               int* err, cudaStream_t st) {
    const Geom& gm = h->g;
    const int blocks = (gm.vol + TC_SITES - 1) / TC_SITES;
    const uint4* img = reinterpret_cast<const uint4*>(G->wimg.as<uint8_t>() + (mode ? 9 * TC_B_BYTES : 0));
    static bool attr[2] = {false, false};
    if (!attr[mode]) {
        if (mode == 0)
            SEEDCG_CUDA_TRY(cudaFuncSetAttribute(k_g_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
        else
            SEEDCG_CUDA_TRY(cudaFuncSetAttribute(k_g_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
        attr[mode] = true;
    }
    if (mode == 0)
        k_g_tc<0><<<blocks, 256, TC_SMEM, st>>>(gm, h->u32.as<float2>(), in, img, zprev, out0, out1, err);
    else
        k_g_tc<1><<<blocks, 256, TC_SMEM, st>>>(gm, h->u32.as<float2>(), in, img, zprev, out0, out1, err);
    SEEDCG_CHECK_LAUNCH();
}

// the bf16 weights and the layer-2 operand images from the master weights
void refresh_weight_forms(GuessState* G, cudaStream_t st) {
    uint8_t* img = G->wimg.as<uint8_t>();
    k_g_wform<<<(9 * 64 * 64 + 255) / 256, 256, 0, st>>>(G->w.as<float2>() + GuessState::NW1, img, img + 9 * TC_B_BYTES);
    SEEDCG_CHECK_LAUNCH();
}

void check_tc(const Acts& A, cudaStream_t st) {
    int e = 0;
    SEEDCG_CUDA_TRY(cudaMemcpyAsync(&e, A.tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
    if (e) throw Error{SEEDCG_ERR_TIMEOUT, "a tensor-core wait of the learned guess expired"};
}

void forward(seedcg_handle* h, GuessState* G, const Acts& A, const double2* b64, cudaStream_t st) {
    const Geom& gm = h->g;
    const long n = 12L * gm.vol;
    const float2* u = h->u32.as<float2>();
    const bf2* W = G->wb.as<bf2>();
    double* partials = A.nb + 64;
    unsigned* ctr = reinterpret_cast<unsigned*>(partials + 8192);
    k_norm2_public(b64, n, partials, ctr, A.nb, st);
    k_g_scale_in<<<std::min<long>((n + 255) / 256, 4096), 256, 0, st>>>(b64, A.nb, A.a0, gm.vol);
    SEEDCG_CHECK_LAUNCH();
    k_g_fwd<1, 8><<<gblocks(8L * gm.vol), kG, 0, st>>>(gm, u, W, A.a0, A.z1, A.h1, 1);
    SEEDCG_CHECK_LAUNCH();
    layer2_tc(h, G, 0, A.h1, nullptr, A.z2, A.h2, A.tc_err, st);
    k_g_fwd<8, 1><<<gblocks((long)gm.vol), kG, 0, st>>>(gm, u, W + GuessState::NW1 + GuessState::NW2, A.h2, A.z3,
                                                        A.z3, 0);
    SEEDCG_CHECK_LAUNCH();
}

template <int CI, int CO>
void weight_grad(seedcg_handle* h, GuessState* G, const bf2* a, const bf2* dout, double2* grad, cudaStream_t st) {
    const Geom& gm = h->g;
    const int per = 1024;
    const int nslice = (gm.vol + per - 1) / per;
    constexpr int NO = CO * CI * 16;
    const size_t ne = (size_t)9 * NO;
    G->part.ensure((size_t)nslice * ne * sizeof(float2));
    dim3 grid(9, nslice);
    k_g_bwd_w<CI, CO><<<grid, kG, 0, st>>>(gm, h->u32.as<float2>(), a, dout, per, G->part.as<float2>());
    SEEDCG_CHECK_LAUNCH();
    k_g_reduce_w<<<(int)((ne + 255) / 256), 256, 0, st>>>(G->part.as<float2>(), nslice, (int)ne, grad);
    SEEDCG_CHECK_LAUNCH();
}

// accumulate the loss and gradient of one pair into G->grad / A.loss
void backward_pair(seedcg_handle* h, GuessState* G, const Acts& A, const double2* x64, double inv_batch,
                   cudaStream_t st) {
    const Geom& gm = h->g;
    const long n = 12L * gm.vol;
    const float2* u = h->u32.as<float2>();
    const bf2* W = G->wb.as<bf2>();
    double2* grad = G->grad.as<double2>();
    double* partials = A.nb + 64;
    unsigned* ctr = reinterpret_cast<unsigned*>(partials + 8192);
    k_norm2_public(x64, n, partials, ctr, A.nx, st);
    k_g_loss<<<std::min<long>((n + 1023) / 1024, 1216), kRedThreads, 0, st>>>(A.z3, x64, A.nb, A.nx, inv_batch,
                                                                             A.d3, gm.vol, partials, ctr + 1, A.loss);
    SEEDCG_CHECK_LAUNCH();
    // layer 3 (8 -> 1)
    weight_grad<8, 1>(h, G, A.h2, A.d3, grad + GuessState::NW1 + GuessState::NW2, st);
    k_g_bwd_data<8, 1><<<gblocks(8L * gm.vol), kG, 0, st>>>(gm, u, W + GuessState::NW1 + GuessState::NW2, A.d3,
                                                            A.z2, A.d2);
    SEEDCG_CHECK_LAUNCH();
    // layer 2 (8 -> 8)
    weight_grad<8, 8>(h, G, A.h1, A.d2, grad + GuessState::NW1, st);
    layer2_tc(h, G, 1, A.d2, A.z1, A.d1, nullptr, A.tc_err, st);
    // layer 1 (1 -> 8): only the weight gradient is needed
    weight_grad<1, 8>(h, G, A.a0, A.d1, grad, st);
}

}  // namespace

void guess_set_weights(seedcg_handle* h, const double* w, cudaStream_t st) {
    GuessState* G = guess_state(h);
    G->w.ensure(GuessState::NW * sizeof(float2));
    G->wb.ensure(GuessState::NW * sizeof(bf2));
    G->wimg.ensure(2 * 9 * TC_B_BYTES);
    G->adam.ensure(2 * GuessState::NW * sizeof(float2));
    G->grad.ensure(GuessState::NW * sizeof(double2));
    std::vector<float2> hw(GuessState::NW);
    for (int e = 0; e < GuessState::NW; e++) hw[e] = make_float2((float)w[2 * e], (float)w[2 * e + 1]);
    SEEDCG_CUDA_TRY(cudaMemcpyAsync(G->w.p, hw.data(), GuessState::NW * sizeof(float2), cudaMemcpyHostToDevice, st));
    SEEDCG_CUDA_TRY(cudaMemsetAsync(G->adam.p, 0, 2 * GuessState::NW * sizeof(float2), st));
    k_g_round<<<(GuessState::NW + 255) / 256, 256, 0, st>>>(G->w.as<float2>(), G->wb.as<bf2>(), GuessState::NW);
    SEEDCG_CHECK_LAUNCH();
    refresh_weight_forms(G, st);
    SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
    G->steps = 0;
    G->have_weights = true;
}

void guess_get_weights(seedcg_handle* h, double* w, cudaStream_t st) {
    GuessState* G = guess_state(h);
    if (!G->have_weights) throw Error{SEEDCG_ERR_ARG, "no guess weights set"};
    std::vector<float2> hw(GuessState::NW);
    SEEDCG_CUDA_TRY(cudaMemcpyAsync(hw.data(), G->w.p, GuessState::NW * sizeof(float2), cudaMemcpyDeviceToHost, st));
    SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
    for (int e = 0; e < GuessState::NW; e++) {
        w[2 * e] = hw[e].x;
        w[2 * e + 1] = hw[e].y;
    }
}

// loss and gradient over npairs (B, X internal FP64 [npairs][n]); grad out in
// complex128 [NW] (host) if non-null; returns the loss
double guess_loss_grad(seedcg_handle* h, int npairs, const double2* B, const double2* X, double* grad_out,
                       cudaStream_t st) {
    GuessState* G = guess_state(h);
    if (!G->have_weights) throw Error{SEEDCG_ERR_ARG, "no guess weights set"};
    const long n = 12L * h->g.vol;
    Acts A = carve_acts(G, h->g.vol);
    SEEDCG_CUDA_TRY(cudaMemsetAsync(G->grad.p, 0, GuessState::NW * sizeof(double2), st));
    SEEDCG_CUDA_TRY(cudaMemsetAsync(A.nb, 0, G->scal.bytes, st));
    for (int k = 0; k < npairs; k++) {
        forward(h, G, A, B + (size_t)k * n, st);
        backward_pair(h, G, A, X + (size_t)k * n, 1.0 / npairs, st);
    }
    double loss = 0.0;
    SEEDCG_CUDA_TRY(cudaMemcpyAsync(&loss, A.loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (grad_out)
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(grad_out, G->grad.p, GuessState::NW * sizeof(double2), cudaMemcpyDeviceToHost, st));
    check_tc(A, st);
    return loss;
}

// Adam training over `epochs` passes of the pairs in order, mini-batches of `batch`
double guess_train(seedcg_handle* h, int npairs, const double2* B, const double2* X, int epochs, int batch,
                   double lr, cudaStream_t st) {
    GuessState* G = guess_state(h);
    double last = 0.0;
    for (int ep = 0; ep < epochs; ep++) {
        double tot = 0.0;
        for (int k0 = 0; k0 < npairs; k0 += batch) {
            const int nb = std::min(batch, npairs - k0);
            const double l = guess_loss_grad(h, nb, B + (size_t)k0 * 12 * h->g.vol, X + (size_t)k0 * 12 * h->g.vol,
                                             nullptr, st);
            tot += l * nb;
            G->steps++;
            const float b1 = 0.9f, b2 = 0.999f;
            const float c1 = 1.f - powf(b1, (float)G->steps), c2 = 1.f - powf(b2, (float)G->steps);
            float2* m = G->adam.as<float2>();
            k_g_adam<<<(GuessState::NW + 255) / 256, 256, 0, st>>>(G->w.as<float2>(), G->wb.as<bf2>(),
                                                                  G->grad.as<double2>(), m, m + GuessState::NW,
                                                                  GuessState::NW, (float)lr, b1, b2, 1e-8f, c1, c2);
            SEEDCG_CHECK_LAUNCH();
            refresh_weight_forms(G, st);
        }
        last = tot / npairs;
    }
    SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
    return last;
}

// x0 = net(b) for n fields (internal FP64 in/out)
void guess_predict(seedcg_handle* h, int n_fields, const double2* B, double2* X0, cudaStream_t st) {
    GuessState* G = guess_state(h);
    if (!G->have_weights) throw Error{SEEDCG_ERR_ARG, "no guess weights set"};
    const long n = 12L * h->g.vol;
    Acts A = carve_acts(G, h->g.vol);
    SEEDCG_CUDA_TRY(cudaMemsetAsync(A.nb, 0, G->scal.bytes, st));
    for (int k = 0; k < n_fields; k++) {
        forward(h, G, A, B + (size_t)k * n, st);
        k_g_scale_out<<<std::min<long>((n + 255) / 256, 4096), 256, 0, st>>>(A.z3, A.nb, X0 + (size_t)k * n,
                                                                            h->g.vol);
        SEEDCG_CHECK_LAUNCH();
    }
    check_tc(A, st);
}

}  // namespace seedcg
