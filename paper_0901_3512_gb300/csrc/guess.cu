// Learned initial guess: a gauge-covariant nearest-neighbour network
//   out_co(x) = sum_ci [ W_0[co,ci] in_ci(x) + sum_{d=+-mu} W_d[co,ci] U(x,d) in_ci(x+d) ]
// (U(x,+mu) = U_mu(x), U(x,-mu) = U_mu(x-mu)^dag, antiperiodic-t sign as in D;
// W_d[co,ci] a complex 4x4 spin matrix; channels 1 -> 8 -> 8 -> 1; ReLU on real
// and imaginary parts after layers 1 and 2; input b/||b||, output times ||b||),
// with hand-written forward, backward and Adam kernels.  FP32 activations and
// weights, FP32 accumulation, FP64 reductions.
//
// Activations are [C][12 V] complex in the paired spinor layout; weights of a
// layer are [9][CO][CI][4][4] complex, directions 0 (on site), +x,-x,+y,-y,
// +z,-z,+t,-t.
#include <algorithm>
#include <cmath>
#include <vector>

#include "handle.cuh"
#include "kernels.cuh"
#include "reduce.cuh"
#include "wilson.cuh"

namespace seedcg {

namespace {

constexpr int kG = 256;

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

// U(x,d)^dag-side adjoint used by the data backward: for the +mu gather the
// adjoint carries U_mu(y-mu)^dag from y-mu to y; for -mu it carries U_mu(y)
// from y+mu to y.  Here `z` is the site the contribution comes from.
__device__ __forceinline__ void apply_link_adj(const float2* __restrict__ u, int vol, int y, int z,
                                               int d, float sg, const float2 v[3], float2 o[3]) {
    const int mu = (d - 1) >> 1;
    const bool back = (d - 1) & 1;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < 3; b++) {
            if (!back) {  // U_mu(z)^dag, z = y - mu
                const float2 uu = __ldg(u + (size_t)(mu * 9 + 3 * b + a) * vol + z);
                acc = cfma_conj(uu, v[b], acc);
            } else {      // U_mu(y)
                const float2 uu = __ldg(u + (size_t)(mu * 9 + 3 * a + b) * vol + y);
                acc = cfma(uu, v[b], acc);
            }
        }
        o[a] = make_float2(sg * acc.x, sg * acc.y);
    }
}

// gathered input g_d(x) for channel ci: 4 spins x 3 colours
__device__ __forceinline__ void gather(const float2* __restrict__ u, const float2* __restrict__ in,
                                       int vol, int x, int d, const Nbr& nb, float2 g[4][3]) {
    if (d == 0) {
#pragma unroll
        for (int k = 0; k < 12; k++) g[k / 3][k % 3] = __ldg(in + sidx(k, x, vol));
        return;
    }
    const int mu = (d - 1) >> 1;
    const int y = ((d - 1) & 1) ? nb.b[mu] : nb.f[mu];
#pragma unroll
    for (int s = 0; s < 4; s++) {
        float2 v[3];
#pragma unroll
        for (int c = 0; c < 3; c++) v[c] = __ldg(in + sidx(3 * s + c, y, vol));
        apply_link(u, vol, x, d, nb, v, g[s]);
    }
}

// forward: one thread per (site, co)
template <int CI, int CO>
__global__ void __launch_bounds__(kG)
k_g_fwd(Geom gm, const float2* __restrict__ u, const float2* __restrict__ W,
        const float2* __restrict__ in, float2* __restrict__ z, float2* __restrict__ h, int relu) {
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
            gather(u, in + (size_t)ci * 12 * vol, vol, x, d, nb, g);
            const float2* w = W + (((size_t)d * CO + co) * CI + ci) * 16;
#pragma unroll
            for (int s = 0; s < 4; s++)
#pragma unroll
                for (int sp = 0; sp < 4; sp++) {
                    const float2 ww = __ldg(w + 4 * s + sp);
#pragma unroll
                    for (int c = 0; c < 3; c++) acc[s][c] = cfma(ww, g[sp][c], acc[s][c]);
                }
        }
    }
    float2* zo = z + (size_t)co * 12 * vol;
    float2* ho = h + (size_t)co * 12 * vol;
#pragma unroll
    for (int k = 0; k < 12; k++) {
        const float2 v = acc[k / 3][k % 3];
        zo[sidx(k, x, vol)] = v;
        if (relu) ho[sidx(k, x, vol)] = make_float2(fmaxf(v.x, 0.f), fmaxf(v.y, 0.f));
    }
}

// backward through the data: din[ci](y) = sum_d adjoint-gather of (W_d^dag dout)
// (one thread per (site, ci)); optionally times the ReLU mask of z_prev
template <int CI, int CO>
__global__ void __launch_bounds__(kG)
k_g_bwd_data(Geom gm, const float2* __restrict__ u, const float2* __restrict__ W,
             const float2* __restrict__ dout, const float2* __restrict__ zprev,
             float2* __restrict__ din) {
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
        // contribution comes from site zsite: y itself (d = 0), y - mu (+mu), y + mu (-mu)
        int zsite = y;
        float sg = 1.f;
        if (d > 0) {
            const int mu = (d - 1) >> 1;
            const bool back = (d - 1) & 1;
            zsite = back ? nb.f[mu] : nb.b[mu];
            // the sign of the hop from zsite in direction d
            if (mu == 3) sg = back ? (nb.fwrap_t ? -1.f : 1.f) : (nb.bwrap_t ? -1.f : 1.f);
        }
        // dg = sum_co W_d[co][ci]^dag dout[co](zsite)
        float2 dg[4][3];
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < 3; c++) dg[s][c] = make_float2(0.f, 0.f);
        for (int co = 0; co < CO; co++) {
            const float2* dz = dout + (size_t)co * 12 * vol;
            float2 dv[4][3];
#pragma unroll
            for (int k = 0; k < 12; k++) dv[k / 3][k % 3] = __ldg(dz + sidx(k, zsite, vol));
            const float2* w = W + (((size_t)d * CO + co) * CI + ci) * 16;
#pragma unroll
            for (int s = 0; s < 4; s++)
#pragma unroll
                for (int sp = 0; sp < 4; sp++) {
                    const float2 ww = __ldg(w + 4 * s + sp);
#pragma unroll
                    for (int c = 0; c < 3; c++) dg[sp][c] = cfma_conj(ww, dv[s][c], dg[sp][c]);
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
                apply_link_adj(u, vol, y, zsite, d, sg, dg[s], o);
#pragma unroll
                for (int c = 0; c < 3; c++) acc[s][c] = cadd(acc[s][c], o[c]);
            }
        }
    }
    float2* out = din + (size_t)ci * 12 * vol;
    const float2* zp = zprev ? zprev + (size_t)ci * 12 * vol : nullptr;
#pragma unroll
    for (int k = 0; k < 12; k++) {
        float2 v = acc[k / 3][k % 3];
        if (zp) {
            const float2 zz = __ldg(zp + sidx(k, y, vol));
            v.x = zz.x > 0.f ? v.x : 0.f;
            v.y = zz.y > 0.f ? v.y : 0.f;
        }
        out[sidx(k, y, vol)] = v;
    }
}

// backward to the weights: dW[d][co][ci][s][s'] = sum_{x,c} dout[co](x)[s][c] conj(g_d(a_ci)(x)[s'][c])
// block (d, slice of sites); the slice's gathered inputs and output gradients
// are staged in shared memory 32 sites at a time; each thread owns output
// entries and accumulates over the slice; partials [slice][9][CO][CI][16]
template <int CI, int CO>
__global__ void __launch_bounds__(kG)
k_g_bwd_w(Geom gm, const float2* __restrict__ u, const float2* __restrict__ a,
          const float2* __restrict__ dout, int sites_per_slice, float2* __restrict__ part) {
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
        // stage: threads (site j, channel) compute the gathers and copy dout
        for (int w = threadIdx.x; w < S * (CI + CO); w += blockDim.x) {
            const int j = w % S, ch = w / S;
            const int x = xs + j;
            if (j >= cnt) continue;
            const Nbr nb = neighbours(gm, x);
            if (ch < CI) {
                float2 g[4][3];
                gather(u, a + (size_t)ch * 12 * vol, vol, x, d, nb, g);
#pragma unroll
                for (int s = 0; s < 4; s++)
#pragma unroll
                    for (int c = 0; c < 3; c++) sg[j][c][ch * 4 + s] = g[s][c];
            } else {
                const int co = ch - CI;
                const float2* dz = dout + (size_t)co * 12 * vol;
#pragma unroll
                for (int k = 0; k < 12; k++) sd[j][k % 3][co * 4 + k / 3] = __ldg(dz + sidx(k, x, vol));
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

// a0 = b / ||b|| (FP32), nb read from device
__global__ void k_g_scale_in(const double2* __restrict__ b, const double* __restrict__ nb,
                             float2* __restrict__ a0, long n) {
    const double inv = 1.0 / *nb;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
        const double2 z = b[e];
        a0[e] = make_float2((float)(z.x * inv), (float)(z.y * inv));
    }
}

// x0 = ||b|| z3 (FP64 out)
__global__ void k_g_scale_out(const float2* __restrict__ z3, const double* __restrict__ nb,
                              double2* __restrict__ x0, long n) {
    const double s = *nb;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
        const float2 z = z3[e];
        x0[e] = make_double2(s * z.x, s * z.y);
    }
}

// loss term ||y - x||^2 / ||x||^2 / nbatch with y = ||b|| z3, and dz3 = ||b|| * 2 (y - x) / ||x||^2 / nbatch
__global__ void __launch_bounds__(kRedThreads)
k_g_loss(const float2* __restrict__ z3, const double2* __restrict__ x, const double* __restrict__ nb,
         const double* __restrict__ nx, double inv_batch, float2* __restrict__ dz3, long n,
         double* partials, unsigned* ctr, double* loss_acc) {
    const double s = *nb, xn2 = (*nx) * (*nx);
    double part = 0.0;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
        const float2 z = z3[e];
        const double2 xv = x[e];
        const double rx = s * z.x - xv.x, ry = s * z.y - xv.y;
        part += rx * rx + ry * ry;
        const double f = s * 2.0 * inv_batch / xn2;
        dz3[e] = make_float2((float)(f * rx), (float)(f * ry));
    }
    double red[1] = {part};
    grid_sum<1>(red, partials, ctr, [&](double* tot) { *loss_acc += tot[0] / xn2 * inv_batch; });
}

// Adam on real and imaginary parts; weights FP32, moments FP32, gradient FP64
__global__ void k_g_adam(float2* __restrict__ W, const double2* __restrict__ g, float2* __restrict__ m,
                         float2* __restrict__ v, int ne, float lr, float b1, float b2, float eps,
                         float c1, float c2) {
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
}

inline int gblocks(long n) { return (int)((n + kG - 1) / kG); }

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct GuessState {
    static constexpr int NW1 = 9 * 8 * 1 * 16, NW2 = 9 * 8 * 8 * 16, NW3 = 9 * 1 * 8 * 16;
    static constexpr int NW = NW1 + NW2 + NW3;
    DevBuf w;       // float2 [NW]
    DevBuf adam;    // m, v float2 [NW] each
    DevBuf grad;    // double2 [NW]
    DevBuf act;     // activations and gradients
    DevBuf part;    // weight-gradient partials
    DevBuf scal;    // norms, loss
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
        g->w.release(); g->adam.release(); g->grad.release(); g->act.release();
        g->part.release(); g->scal.release();
        delete g;
        h->guess = nullptr;
    }
}

namespace {

struct Acts {
    float2 *a0, *z1, *h1, *z2, *h2, *z3, *d3, *d2, *d1;
    double* nb;
    double* nx;
    double* loss;
};

Acts carve_acts(GuessState* G, long n) {
    const size_t need = (size_t)n * (1 + 8 * 4 + 1 + 1 + 8 * 2) * sizeof(float2) + 4096;
    G->act.ensure(need);
    G->scal.ensure(64 * sizeof(double) + 8192 * sizeof(double));
    float2* p = G->act.as<float2>();
    Acts A;
    A.a0 = p; p += n;
    A.z1 = p; p += 8 * n;
    A.h1 = p; p += 8 * n;
    A.z2 = p; p += 8 * n;
    A.h2 = p; p += 8 * n;
    A.z3 = p; p += n;
    A.d3 = p; p += n;
    A.d2 = p; p += 8 * n;
    A.d1 = p; p += 8 * n;
    A.nb = G->scal.as<double>();
    A.nx = A.nb + 1;
    A.loss = A.nb + 2;
    return A;
}

void forward(seedcg_handle* h, GuessState* G, const Acts& A, const double2* b64, cudaStream_t st) {
    const Geom& gm = h->g;
    const long n = 12L * gm.vol;
    const float2* u = h->u32.as<float2>();
    const float2* W = G->w.as<float2>();
    double* partials = A.nb + 64;
    unsigned* ctr = reinterpret_cast<unsigned*>(partials + 4096);
    k_norm2_public(b64, n, partials, ctr, A.nb, st);
    k_g_scale_in<<<std::min<long>((n + 255) / 256, 4096), 256, 0, st>>>(b64, A.nb, A.a0, n);
    SEEDCG_CHECK_LAUNCH();
    k_g_fwd<1, 8><<<gblocks(8L * gm.vol), kG, 0, st>>>(gm, u, W, A.a0, A.z1, A.h1, 1);
    SEEDCG_CHECK_LAUNCH();
    k_g_fwd<8, 8><<<gblocks(8L * gm.vol), kG, 0, st>>>(gm, u, W + GuessState::NW1, A.h1, A.z2, A.h2, 1);
    SEEDCG_CHECK_LAUNCH();
    k_g_fwd<8, 1><<<gblocks((long)gm.vol), kG, 0, st>>>(gm, u, W + GuessState::NW1 + GuessState::NW2,
                                                        A.h2, A.z3, A.z3, 0);
    SEEDCG_CHECK_LAUNCH();
}

template <int CI, int CO>
void weight_grad(seedcg_handle* h, GuessState* G, const float2* a, const float2* dout,
                 double2* grad, cudaStream_t st) {
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
void backward_pair(seedcg_handle* h, GuessState* G, const Acts& A, const double2* x64,
                   double inv_batch, cudaStream_t st) {
    const Geom& gm = h->g;
    const long n = 12L * gm.vol;
    const float2* u = h->u32.as<float2>();
    const float2* W = G->w.as<float2>();
    double2* grad = G->grad.as<double2>();
    double* partials = A.nb + 64;
    unsigned* ctr = reinterpret_cast<unsigned*>(partials + 4096);
    k_norm2_public(x64, n, partials, ctr, A.nx, st);
    k_g_loss<<<std::min<long>((n + 1023) / 1024, 1216), kRedThreads, 0, st>>>(
        A.z3, x64, A.nb, A.nx, inv_batch, A.d3, n, partials, ctr + 1, A.loss);
    SEEDCG_CHECK_LAUNCH();
    // layer 3 (8 -> 1)
    weight_grad<8, 1>(h, G, A.h2, A.d3, grad + GuessState::NW1 + GuessState::NW2, st);
    k_g_bwd_data<8, 1><<<gblocks(8L * gm.vol), kG, 0, st>>>(gm, u, W + GuessState::NW1 + GuessState::NW2,
                                                            A.d3, A.z2, A.d2);
    SEEDCG_CHECK_LAUNCH();
    // layer 2 (8 -> 8)
    weight_grad<8, 8>(h, G, A.h1, A.d2, grad + GuessState::NW1, st);
    k_g_bwd_data<8, 8><<<gblocks(8L * gm.vol), kG, 0, st>>>(gm, u, W + GuessState::NW1, A.d2, A.z1, A.d1);
    SEEDCG_CHECK_LAUNCH();
    // layer 1 (1 -> 8): only the weight gradient is needed
    weight_grad<1, 8>(h, G, A.a0, A.d1, grad, st);
}

}  // namespace

void guess_set_weights(seedcg_handle* h, const double* w, cudaStream_t st) {
    GuessState* G = guess_state(h);
    G->w.ensure(GuessState::NW * sizeof(float2));
    G->adam.ensure(2 * GuessState::NW * sizeof(float2));
    G->grad.ensure(GuessState::NW * sizeof(double2));
    std::vector<float2> hw(GuessState::NW);
    for (int e = 0; e < GuessState::NW; e++) hw[e] = make_float2((float)w[2 * e], (float)w[2 * e + 1]);
    SEEDCG_CUDA_TRY(cudaMemcpyAsync(G->w.p, hw.data(), GuessState::NW * sizeof(float2), cudaMemcpyHostToDevice, st));
    SEEDCG_CUDA_TRY(cudaMemsetAsync(G->adam.p, 0, 2 * GuessState::NW * sizeof(float2), st));
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
double guess_loss_grad(seedcg_handle* h, int npairs, const double2* B, const double2* X,
                       double* grad_out, cudaStream_t st) {
    GuessState* G = guess_state(h);
    if (!G->have_weights) throw Error{SEEDCG_ERR_ARG, "no guess weights set"};
    const long n = 12L * h->g.vol;
    Acts A = carve_acts(G, n);
    SEEDCG_CUDA_TRY(cudaMemsetAsync(G->grad.p, 0, GuessState::NW * sizeof(double2), st));
    SEEDCG_CUDA_TRY(cudaMemsetAsync(A.nb, 0, (64 + 4096) * sizeof(double) + 8192 * sizeof(unsigned), st));
    for (int k = 0; k < npairs; k++) {
        forward(h, G, A, B + (size_t)k * n, st);
        backward_pair(h, G, A, X + (size_t)k * n, 1.0 / npairs, st);
    }
    double loss = 0.0;
    SEEDCG_CUDA_TRY(cudaMemcpyAsync(&loss, A.loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (grad_out)
        SEEDCG_CUDA_TRY(cudaMemcpyAsync(grad_out, G->grad.p, GuessState::NW * sizeof(double2), cudaMemcpyDeviceToHost, st));
    SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
    return loss;
}

// Adam training over `epochs` passes of the pairs in order, mini-batches of `batch`
double guess_train(seedcg_handle* h, int npairs, const double2* B, const double2* X, int epochs,
                   int batch, double lr, cudaStream_t st) {
    GuessState* G = guess_state(h);
    double last = 0.0;
    for (int ep = 0; ep < epochs; ep++) {
        double tot = 0.0;
        for (int k0 = 0; k0 < npairs; k0 += batch) {
            const int nb = std::min(batch, npairs - k0);
            const double l = guess_loss_grad(h, nb, B + (size_t)k0 * 12 * h->g.vol,
                                             X + (size_t)k0 * 12 * h->g.vol, nullptr, st);
            tot += l * nb;
            G->steps++;
            const float b1 = 0.9f, b2 = 0.999f;
            const float c1 = 1.f - powf(b1, (float)G->steps), c2 = 1.f - powf(b2, (float)G->steps);
            float2* m = G->adam.as<float2>();
            k_g_adam<<<(GuessState::NW + 255) / 256, 256, 0, st>>>(G->w.as<float2>(), G->grad.as<double2>(), m,
                                                                  m + GuessState::NW, GuessState::NW, (float)lr,
                                                                  b1, b2, 1e-8f, c1, c2);
            SEEDCG_CHECK_LAUNCH();
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
    Acts A = carve_acts(G, n);
    SEEDCG_CUDA_TRY(cudaMemsetAsync(A.nb, 0, (64 + 4096) * sizeof(double) + 8192 * sizeof(unsigned), st));
    for (int k = 0; k < n_fields; k++) {
        forward(h, G, A, B + (size_t)k * n, st);
        k_g_scale_out<<<std::min<long>((n + 255) / 256, 4096), 256, 0, st>>>(A.z3, A.nb, X0 + (size_t)k * n, n);
        SEEDCG_CHECK_LAUNCH();
    }
    SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
}

}  // namespace seedcg
