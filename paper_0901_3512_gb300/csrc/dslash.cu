// Wilson dslash kernels (single- and multi-right-hand-side, FP64 and FP32)
// and the layout transforms between the boundary's complex128 AoS and the
// internal site-fastest layouts.
#include "internal.cuh"
#include "wilson.cuh"

namespace seedcg {

namespace {

constexpr int kThreads = 128;

inline int blocks_for(long n, int threads) { return (int)((n + threads - 1) / threads); }

// ---------------------------------------------------------------------------
// layout transforms
// ---------------------------------------------------------------------------
__global__ void k_to_internal_f64(const double2* __restrict__ in, double2* __restrict__ out,
                                  int vol, int n) {
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)vol * n) return;
    int r = (int)(t / vol), s = (int)(t % vol);
    const double2* src = in + ((size_t)r * vol + s) * 12;
    double2* dst = out + (size_t)r * 12 * vol + s;
#pragma unroll
    for (int k = 0; k < 12; k++) dst[(size_t)k * vol] = src[k];
}

__global__ void k_from_internal_f64(const double2* __restrict__ in, double2* __restrict__ out,
                                    int vol, int n) {
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)vol * n) return;
    int r = (int)(t / vol), s = (int)(t % vol);
    const double2* src = in + (size_t)r * 12 * vol + s;
    double2* dst = out + ((size_t)r * vol + s) * 12;
#pragma unroll
    for (int k = 0; k < 12; k++) dst[k] = src[(size_t)k * vol];
}

__global__ void k_to_internal_f32(const double2* __restrict__ in, float2* __restrict__ out,
                                  int vol, int n) {
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)vol * n) return;
    int r = (int)(t / vol), s = (int)(t % vol);
    const double2* src = in + ((size_t)r * vol + s) * 12;
    float2* dst = out + (size_t)r * 12 * vol + s;
#pragma unroll
    for (int k = 0; k < 12; k++) dst[(size_t)k * vol] = make_float2((float)src[k].x, (float)src[k].y);
}

__global__ void k_from_internal_f32(const float2* __restrict__ in, double2* __restrict__ out,
                                    int vol, int n) {
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)vol * n) return;
    int r = (int)(t / vol), s = (int)(t % vol);
    const float2* src = in + (size_t)r * 12 * vol + s;
    double2* dst = out + ((size_t)r * vol + s) * 12;
#pragma unroll
    for (int k = 0; k < 12; k++) {
        float2 q = src[(size_t)k * vol];
        dst[k] = make_double2(q.x, q.y);
    }
}

__global__ void k_gauge_to_internal(const double2* __restrict__ in, double2* __restrict__ u64,
                                    float2* __restrict__ u32, int vol) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= vol) return;
    const double2* src = in + (size_t)s * 36;
#pragma unroll
    for (int e = 0; e < 36; e++) {  // e = mu*9 + 3a + b
        double2 z = src[e];
        u64[(size_t)e * vol + s] = z;
        u32[(size_t)e * vol + s] = make_float2((float)z.x, (float)z.y);
    }
}

// ---------------------------------------------------------------------------
// single right-hand side: one thread per site, links and neighbours from
// global memory (coalesced: neighbouring threads read neighbouring sites)
// ---------------------------------------------------------------------------
template <typename R, int DAG>
__global__ void __launch_bounds__(kThreads)
k_dslash(Geom g, const cx_t<R>* __restrict__ u, R kappa, const cx_t<R>* __restrict__ in,
         cx_t<R>* __restrict__ out) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.vol) return;
    const int vol = g.vol;
    Nbr n = neighbours(g, s);
    Spinor<R> acc, self, res;
    auto load = [&](int y, Spinor<R>& p) { load_spinor(in, vol, y, p); };
    auto fl = [&](int mu, int e) { return __ldg(u + (size_t)(mu * 9 + e) * vol + s); };
    auto bl = [&](int mu, int e) { return __ldg(u + (size_t)(mu * 9 + e) * vol + n.b[mu]); };
    hopping_sum<DAG, R>(n, load, fl, bl, acc);
    load_spinor(in, vol, s, self);
    wilson_combine(self, acc, kappa, res);
    store_spinor(out, vol, s, res);
}

// ---------------------------------------------------------------------------
// multi right-hand side: a block owns TS consecutive sites and all n
// right-hand sides.  The 8 links each site needs (U_mu(x) and U_mu(x-mu)) are
// staged once in shared memory and reused for every right-hand side.
// blockDim = TS * RPB; thread (site j, group q) handles rhs q, q+RPB, ...
// ---------------------------------------------------------------------------
template <typename R, int DAG, int TS>
__global__ void k_dslash_mrhs(Geom g, const cx_t<R>* __restrict__ u, R kappa, int n,
                              const cx_t<R>* __restrict__ in, cx_t<R>* __restrict__ out) {
    extern __shared__ unsigned char smem_raw[];
    cx_t<R>* sl = reinterpret_cast<cx_t<R>*>(smem_raw);  // [2][4][9][TS]
    const int vol = g.vol;
    const int s0 = blockIdx.x * TS;
    const int nthr = blockDim.x;
    // stage links: entry e = ((dir*4 + mu)*9 + c)*TS + j
    for (int e = threadIdx.x; e < 2 * 4 * 9 * TS; e += nthr) {
        int j = e % TS;
        int rest = e / TS;
        int c = rest % 9;
        int mu = (rest / 9) % 4;
        int dir = rest / 36;
        int s = s0 + j;
        cx_t<R> z = mk<R>(0, 0);
        if (s < vol) {
            int y = s;
            if (dir) {
                int cm = (s / g.stride[mu]) % g.L[mu];
                y = (cm == 0) ? s + (g.L[mu] - 1) * g.stride[mu] : s - g.stride[mu];
            }
            z = __ldg(u + (size_t)(mu * 9 + c) * vol + y);
        }
        sl[e] = z;
    }
    __syncthreads();
    const int j = threadIdx.x % TS;
    const int q = threadIdx.x / TS;
    const int rpb = nthr / TS;
    const int s = s0 + j;
    if (s >= vol) return;
    Nbr nb = neighbours(g, s);
    auto fl = [&](int mu, int e) { return sl[((0 * 4 + mu) * 9 + e) * TS + j]; };
    auto bl = [&](int mu, int e) { return sl[((1 * 4 + mu) * 9 + e) * TS + j]; };
    for (int r = q; r < n; r += rpb) {
        const cx_t<R>* inr = in + (size_t)r * 12 * vol;
        cx_t<R>* outr = out + (size_t)r * 12 * vol;
        Spinor<R> acc, self, res;
        auto load = [&](int y, Spinor<R>& p) { load_spinor(inr, vol, y, p); };
        hopping_sum<DAG, R>(nb, load, fl, bl, acc);
        load_spinor(inr, vol, s, self);
        wilson_combine(self, acc, kappa, res);
        store_spinor(outr, vol, s, res);
    }
}

template <typename R>
void launch_dslash(const Geom& g, const cx_t<R>* u, R kappa, int dag, const cx_t<R>* in,
                   cx_t<R>* out, cudaStream_t st) {
    int nb = blocks_for(g.vol, kThreads);
    if (dag)
        k_dslash<R, 1><<<nb, kThreads, 0, st>>>(g, u, kappa, in, out);
    else
        k_dslash<R, 0><<<nb, kThreads, 0, st>>>(g, u, kappa, in, out);
    SEEDCG_CHECK_LAUNCH();
}

template <typename R>
void launch_dslash_mrhs(const Geom& g, const cx_t<R>* u, R kappa, int dag, int n,
                        const cx_t<R>* in, cx_t<R>* out, cudaStream_t st) {
    if (n <= 0) return;
    constexpr int TS = 32;
    int rpb = n < 8 ? n : 8;
    int threads = TS * rpb;
    size_t smem = sizeof(cx_t<R>) * 2 * 4 * 9 * TS;
    int nb = blocks_for(g.vol, TS);
    if (dag)
        k_dslash_mrhs<R, 1, TS><<<nb, threads, smem, st>>>(g, u, kappa, n, in, out);
    else
        k_dslash_mrhs<R, 0, TS><<<nb, threads, smem, st>>>(g, u, kappa, n, in, out);
    SEEDCG_CHECK_LAUNCH();
}

}  // namespace

void to_internal_f64(const double* in, double2* out, int vol, int n, cudaStream_t s) {
    if ((long)vol * n == 0) return;
    k_to_internal_f64<<<blocks_for((long)vol * n, 256), 256, 0, s>>>(
        reinterpret_cast<const double2*>(in), out, vol, n);
    SEEDCG_CHECK_LAUNCH();
}
void from_internal_f64(const double2* in, double* out, int vol, int n, cudaStream_t s) {
    if ((long)vol * n == 0) return;
    k_from_internal_f64<<<blocks_for((long)vol * n, 256), 256, 0, s>>>(
        in, reinterpret_cast<double2*>(out), vol, n);
    SEEDCG_CHECK_LAUNCH();
}
void to_internal_f32(const double* in, float2* out, int vol, int n, cudaStream_t s) {
    if ((long)vol * n == 0) return;
    k_to_internal_f32<<<blocks_for((long)vol * n, 256), 256, 0, s>>>(
        reinterpret_cast<const double2*>(in), out, vol, n);
    SEEDCG_CHECK_LAUNCH();
}
void from_internal_f32(const float2* in, double* out, int vol, int n, cudaStream_t s) {
    if ((long)vol * n == 0) return;
    k_from_internal_f32<<<blocks_for((long)vol * n, 256), 256, 0, s>>>(
        in, reinterpret_cast<double2*>(out), vol, n);
    SEEDCG_CHECK_LAUNCH();
}
void gauge_to_internal(const double* in, double2* u64, float2* u32, int vol, cudaStream_t s) {
    k_gauge_to_internal<<<blocks_for(vol, 256), 256, 0, s>>>(
        reinterpret_cast<const double2*>(in), u64, u32, vol);
    SEEDCG_CHECK_LAUNCH();
}

void dslash_f64(const Geom& g, const double2* u, double kappa, int dag, const double2* in,
                double2* out, cudaStream_t s) {
    launch_dslash<double>(g, u, kappa, dag, in, out, s);
}
void dslash_f32(const Geom& g, const float2* u, float kappa, int dag, const float2* in,
                float2* out, cudaStream_t s) {
    launch_dslash<float>(g, u, kappa, dag, in, out, s);
}
void dslash_mrhs_f64(const Geom& g, const double2* u, double kappa, int dag, int n,
                     const double2* in, double2* out, cudaStream_t s) {
    launch_dslash_mrhs<double>(g, u, kappa, dag, n, in, out, s);
}
void dslash_mrhs_f32(const Geom& g, const float2* u, float kappa, int dag, int n,
                     const float2* in, float2* out, cudaStream_t s) {
    launch_dslash_mrhs<float>(g, u, kappa, dag, n, in, out, s);
}

}  // namespace seedcg
