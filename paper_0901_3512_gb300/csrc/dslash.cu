// Wilson dslash kernels (single- and multi-right-hand-side, FP64 and FP32)
// and the layout transforms between the boundary's complex128 AoS and the
// internal site-fastest layouts.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>

#include "internal.cuh"
#include "wilson.cuh"
#include "reduce.cuh"

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
    double2* dst = out + (size_t)r * 12 * vol;
#pragma unroll
    for (int k = 0; k < 12; k++) dst[sidx(k, s, vol)] = src[k];
}

__global__ void k_from_internal_f64(const double2* __restrict__ in, double2* __restrict__ out,
                                    int vol, int n) {
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)vol * n) return;
    int r = (int)(t / vol), s = (int)(t % vol);
    const double2* src = in + (size_t)r * 12 * vol;
    double2* dst = out + ((size_t)r * vol + s) * 12;
#pragma unroll
    for (int k = 0; k < 12; k++) dst[k] = src[sidx(k, s, vol)];
}

__global__ void k_to_internal_f32(const double2* __restrict__ in, float2* __restrict__ out,
                                  int vol, int n) {
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)vol * n) return;
    int r = (int)(t / vol), s = (int)(t % vol);
    const double2* src = in + ((size_t)r * vol + s) * 12;
    float2* dst = out + (size_t)r * 12 * vol;
#pragma unroll
    for (int k = 0; k < 12; k++) dst[sidx(k, s, vol)] = make_float2((float)src[k].x, (float)src[k].y);
}

__global__ void k_from_internal_f32(const float2* __restrict__ in, double2* __restrict__ out,
                                    int vol, int n) {
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)vol * n) return;
    int r = (int)(t / vol), s = (int)(t % vol);
    const float2* src = in + (size_t)r * 12 * vol;
    double2* dst = out + ((size_t)r * vol + s) * 12;
#pragma unroll
    for (int k = 0; k < 12; k++) {
        float2 q = src[sidx(k, s, vol)];
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
    Spinor<R> res;
    auto load = [&](int y, Spinor<R>& p) { load_spinor(in, vol, y, p); };
    auto fl = [&](int mu, int e) { return __ldg(u + (size_t)(mu * 9 + e) * vol + s); };
    auto bl = [&](int mu, int e) { return __ldg(u + (size_t)(mu * 9 + e) * vol + n.b[mu]); };
    wilson_site<DAG, R>(n, s, load, fl, bl, kappa, res);
    store_spinor(out, vol, s, res);
}

// ---------------------------------------------------------------------------
// multi right-hand side: a block owns TS consecutive sites and all n
// right-hand sides.  The 8 links each site needs (U_mu(x) and U_mu(x-mu)) are
// staged once in shared memory and reused for every right-hand side.
// blockDim = TS * RPB; thread (site j, group q) handles rhs q, q+RPB, ...
// ---------------------------------------------------------------------------
template <typename R, int DAG, int TS>
__global__ void __launch_bounds__(384, (sizeof(R) == 4 ? 2 : 1))
k_dslash_mrhs(Geom g, const cx_t<R>* __restrict__ u, R kappa, int n,
              const cx_t<R>* __restrict__ in, cx_t<R>* __restrict__ out) {
    // links of the tile, already multiplied by -kappa and the t-boundary sign
    __shared__ cx_t<R> sl[2][4][9][TS];   // [fwd/bwd][mu][3a+b][site]
    __shared__ int sb[4][TS];              // x - mu for each tile site
    __shared__ R sgn[2][TS];               // -kappa * sign of the forward / backward t hop
    const int vol = g.vol;
    const int s0 = blockIdx.x * TS;
    const int nthr = blockDim.x;
    if (threadIdx.x < TS) {
        const int s = s0 + threadIdx.x;
        if (s < vol) {
            Nbr nb = neighbours(g, s);
#pragma unroll
            for (int mu = 0; mu < 4; mu++) sb[mu][threadIdx.x] = nb.b[mu];
            sgn[0][threadIdx.x] = nb.fwrap_t ? kappa : -kappa;
            sgn[1][threadIdx.x] = nb.bwrap_t ? kappa : -kappa;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * 4 * 9 * TS; e += nthr) {
        const int j = e % TS;
        const int c = (e / TS) % 9;
        const int mu = (e / (9 * TS)) % 4;
        const int dir = e / (36 * TS);
        const int s = s0 + j;
        cx_t<R> z = mk<R>(0, 0);
        if (s < vol) {
            z = __ldg(u + (size_t)(mu * 9 + c) * vol + (dir ? sb[mu][j] : s));
            z = cscale(z, mu == 3 ? sgn[dir][j] : -kappa);
        }
        sl[dir][mu][c][j] = z;
    }
    __syncthreads();
    const int j = threadIdx.x % TS;
    const int q = threadIdx.x / TS;
    const int rpb = nthr / TS;
    const int s = s0 + j;
    if (s >= vol) return;
    Nbr nb = neighbours(g, s);
    auto fl = [&](int mu, int e) { return sl[0][mu][e][j]; };
    auto bl = [&](int mu, int e) { return sl[1][mu][e][j]; };
    for (int r = q; r < n; r += rpb) {
        const cx_t<R>* inr = in + (size_t)r * 12 * vol;
        cx_t<R>* outr = out + (size_t)r * 12 * vol;
        Spinor<R> res;
        auto load = [&](int y, Spinor<R>& p) { load_spinor(inr, vol, y, p); };
        wilson_site_prescaled<DAG, R>(nb, s, load, fl, bl, res);
        store_spinor(outr, vol, s, res);
    }
}

// ---------------------------------------------------------------------------
// multi right-hand side, brick tiling: a block owns a Bx x By x Bz brick of
// sites at one t (Bx = Lx), so the x, y and z neighbours of most sites are
// sites of the same block and hit in L1; its links (scaled by -kappa and the
// boundary sign) are staged once in dynamic shared memory and reused for every
// right-hand side.  blockDim = TB * rpb, TB = Bx*By*Bz a multiple of 32.
// ---------------------------------------------------------------------------
struct Brick {
    int bx, by, bz, tb;     // brick extents and sites per brick
    int ny, nz;             // bricks along y and z
};

// PIPE: at most 256 threads and up to 128 registers per thread, spent on
// keeping more neighbour spinors in flight (wilson_site_prescaled_pipe)
template <typename R, int DAG, int TB, bool PIPE = false>
__global__ void __launch_bounds__(PIPE ? 256 : 384, (sizeof(R) == 4 ? 2 : 1))
k_dslash_brick(Geom g, Brick br, const cx_t<R>* __restrict__ u, R kappa, int n,
               const cx_t<R>* __restrict__ in, cx_t<R>* __restrict__ out) {
    extern __shared__ unsigned char smem_raw[];
    cx_t<R>* sl = reinterpret_cast<cx_t<R>*>(smem_raw);            // [2][4][9][TB]
    int* ss = reinterpret_cast<int*>(sl + 72 * TB);                  // [TB] site index
    int* sbk = ss + TB;                                              // [4][TB] x - mu
    R* sg = reinterpret_cast<R*>(sbk + 4 * TB);                      // [2][TB]
    const int vol = g.vol;
    int b = blockIdx.x;
    const int iy = b % br.ny; b /= br.ny;
    const int iz = b % br.nz;
    const int t = b / br.nz;
    if (threadIdx.x < TB) {
        const int j = threadIdx.x;
        const int x = j % br.bx, dy = (j / br.bx) % br.by, dz = j / (br.bx * br.by);
        const int s = x + g.stride[1] * (iy * br.by + dy) + g.stride[2] * (iz * br.bz + dz) + g.stride[3] * t;
        ss[j] = s;
        Nbr nb = neighbours(g, s);
#pragma unroll
        for (int mu = 0; mu < 4; mu++) sbk[mu * TB + j] = nb.b[mu];
        sg[j] = nb.fwrap_t ? kappa : -kappa;
        sg[TB + j] = nb.bwrap_t ? kappa : -kappa;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 72 * TB; e += blockDim.x) {
        const int j = e % TB;
        const int c = (e / TB) % 9;
        const int mu = (e / (9 * TB)) % 4;
        const int dir = e / (36 * TB);
        cx_t<R> z = __ldg(u + (size_t)(mu * 9 + c) * vol + (dir ? sbk[mu * TB + j] : ss[j]));
        sl[e] = cscale(z, mu == 3 ? sg[dir * TB + j] : -kappa);
    }
    __syncthreads();
    const int j = threadIdx.x % TB;
    const int q = threadIdx.x / TB;
    const int rpb = blockDim.x / TB;
    const int s = ss[j];
    Nbr nb = neighbours(g, s);
    auto fl = [&](int mu, int e) { return sl[((0 * 4 + mu) * 9 + e) * TB + j]; };
    auto bl = [&](int mu, int e) { return sl[((1 * 4 + mu) * 9 + e) * TB + j]; };
    for (int r = q; r < n; r += rpb) {
        const cx_t<R>* inr = in + (size_t)r * 12 * vol;
        cx_t<R>* outr = out + (size_t)r * 12 * vol;
        Spinor<R> res;
        auto load = [&](int y, Spinor<R>& p) { load_spinor(inr, vol, y, p); };
        if constexpr (PIPE)
            wilson_site_prescaled_pipe<DAG, R>(nb, s, load, fl, bl, res);
        else
            wilson_site_prescaled<DAG, R>(nb, s, load, fl, bl, res);
        store_spinor(outr, vol, s, res);
    }
}

int largest_divisor_at_most(int L, int cap) {
    int best = 1;
    for (int d = 1; d <= L && d <= cap; d++)
        if (L % d == 0) best = d;
    return best;
}

bool make_brick(const Geom& g, Brick& br, int cap = 128) {
    br.bx = g.L[0];
    if (br.bx > 64 || br.bx > cap) return false;
    br.by = largest_divisor_at_most(g.L[1], (cap / 2 > br.bx ? cap / 2 : cap) / br.bx);
    br.bz = largest_divisor_at_most(g.L[2], cap / (br.bx * br.by));
    br.tb = br.bx * br.by * br.bz;
    br.ny = g.L[1] / br.by;
    br.nz = g.L[2] / br.bz;
    return br.tb % 32 == 0 && br.tb <= 128;
}

// one launch of a brick kernel; the dynamic shared memory limit is raised once
// per instantiation (each has its own static flag)
template <typename R, int DAG, int TB, bool PIPE = false>
void brick_go(int nb, int threads, size_t smem, cudaStream_t st, const Geom& g, const Brick& br,
              const cx_t<R>* u, R kappa, int n, const cx_t<R>* in, cx_t<R>* out) {
    static bool attr = false;
    if (!attr) {
        SEEDCG_CUDA_TRY(cudaFuncSetAttribute(k_dslash_brick<R, DAG, TB, PIPE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
        attr = true;
    }
    k_dslash_brick<R, DAG, TB, PIPE><<<nb, threads, smem, st>>>(g, br, u, kappa, n, in, out);
    SEEDCG_CHECK_LAUNCH();
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

// ---------------------------------------------------------------------------
// autotuner of the brick kernel: sites per brick (64 / 128) and right-hand
// sides side by side per block, timed with CUDA events on the caller's own
// buffers at the first call for a (lattice, n, precision, D or D^dag) and kept
// for the process (and in SEEDCG_TUNE_CACHE when set).
// ---------------------------------------------------------------------------
struct BrickChoice {
    int cap;
    int rpb;    // 0 = balanced default
    int pipe;   // 1 = the register-pipelined site kernel (<= 256 threads)
};

template <typename R>
void launch_dslash_mrhs(const Geom& g, const cx_t<R>* u, R kappa, int dag, int n,
                        const cx_t<R>* in, cx_t<R>* out, cudaStream_t st,
                        const BrickChoice* force = nullptr);

template <typename R>
BrickChoice tuned_brick(const Geom& g, const cx_t<R>* u, R kappa, int dag, int n, const cx_t<R>* in,
                        cx_t<R>* out, cudaStream_t st) {
    static std::mutex mu;
    static std::map<std::string, BrickChoice> cache;
    char key[160];
    snprintf(key, sizeof(key), "brick_%s_%dx%dx%dx%d_n%d_dag%d", sizeof(R) == 8 ? "f64" : "f32",
             g.L[0], g.L[1], g.L[2], g.L[3], n, dag);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
        if (const char* path = getenv("SEEDCG_TUNE_CACHE")) {
            FILE* f = fopen(path, "r");
            if (f) {
                // the file is shared with the batched-CG tuner: read only full brick lines
                char line[640], k[512];
                int a, b, c;
                while (fgets(line, sizeof(line), f))
                    if (sscanf(line, "%511s %d %d %d", k, &a, &b, &c) == 4 && std::string(k) == key)
                        cache[key] = BrickChoice{a, b, c};
                fclose(f);
                it = cache.find(key);
                if (it != cache.end()) return it->second;
            }
        }
    }
    cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cap_status);
    if (cap_status != cudaStreamCaptureStatusNone) return BrickChoice{128, 0, 0};  // no timing inside a capture
    const BrickChoice cands[] = {{128, 0, 0}, {128, 2, 0}, {128, 1, 0}, {64, 0, 0}, {64, 4, 0},
                                 {64, 3, 0},  {128, 2, 1}, {128, 1, 1}, {64, 4, 1}, {64, 2, 1}};
    const bool tune_log = getenv("SEEDCG_TUNE_LOG") != nullptr;
    cudaEvent_t a, b;
    SEEDCG_CUDA_TRY(cudaEventCreate(&a));
    SEEDCG_CUDA_TRY(cudaEventCreate(&b));
    BrickChoice best{128, 0};
    float best_ms = 1e30f;
    for (const BrickChoice& c : cands) {
        Brick br;
        if (!make_brick(g, br, c.cap) || !(br.tb == 64 || br.tb == 96 || br.tb == 128)) continue;
        launch_dslash_mrhs<R>(g, u, kappa, dag, n, in, out, st, &c);
        SEEDCG_CUDA_TRY(cudaEventRecord(a, st));
        for (int r = 0; r < 3; r++)
            launch_dslash_mrhs<R>(g, u, kappa, dag, n, in, out, st, &c);
        SEEDCG_CUDA_TRY(cudaEventRecord(b, st));
        SEEDCG_CUDA_TRY(cudaEventSynchronize(b));
        float ms = 0.f;
        SEEDCG_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
        if (tune_log)
            fprintf(stderr, "seedcg tune %s: cap %d rpb %d pipe %d: %.4f ms\n", key, c.cap, c.rpb, c.pipe,
                    ms / 3);
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = best;
    if (const char* path = getenv("SEEDCG_TUNE_CACHE")) {
        FILE* f = fopen(path, "a");
        if (f) {
            fprintf(f, "%s %d %d %d\n", key, best.cap, best.rpb, best.pipe);
            fclose(f);
        }
    }
    return best;
}

template <typename R>
void launch_dslash_mrhs(const Geom& g, const cx_t<R>* u, R kappa, int dag, int n,
                        const cx_t<R>* in, cx_t<R>* out, cudaStream_t st,
                        const BrickChoice* force) {
    if (n <= 0) return;
    Brick br;
    BrickChoice ch{128, 0, 0};
    if (force) ch = *force;
    else ch = tuned_brick<R>(g, u, kappa, dag, n, in, out, st);
    if (make_brick(g, br, ch.cap) && (br.tb == 64 || br.tb == 96 || br.tb == 128)) {
        const int maxr = (ch.pipe ? 256 : 384) / br.tb;
        const int passes = (n + maxr - 1) / maxr;
        const int rpb = ch.rpb > 0 ? std::min(ch.rpb, maxr) : (n + passes - 1) / passes;
        const int threads = br.tb * rpb;
        const size_t smem = (size_t)br.tb * (72 * sizeof(cx_t<R>) + 5 * sizeof(int) + 2 * sizeof(R));
        const int nb = br.ny * br.nz * g.L[3];
        if (ch.pipe && br.tb == 128) {
            if (dag) brick_go<R, 1, 128, true>(nb, threads, smem, st, g, br, u, kappa, n, in, out);
            else brick_go<R, 0, 128, true>(nb, threads, smem, st, g, br, u, kappa, n, in, out);
        } else if (ch.pipe && br.tb == 64) {
            if (dag) brick_go<R, 1, 64, true>(nb, threads, smem, st, g, br, u, kappa, n, in, out);
            else brick_go<R, 0, 64, true>(nb, threads, smem, st, g, br, u, kappa, n, in, out);
        } else if (br.tb == 128) {
            if (dag) brick_go<R, 1, 128>(nb, threads, smem, st, g, br, u, kappa, n, in, out);
            else brick_go<R, 0, 128>(nb, threads, smem, st, g, br, u, kappa, n, in, out);
        } else if (br.tb == 96) {
            if (dag) brick_go<R, 1, 96>(nb, threads, smem, st, g, br, u, kappa, n, in, out);
            else brick_go<R, 0, 96>(nb, threads, smem, st, g, br, u, kappa, n, in, out);
        } else {
            if (dag) brick_go<R, 1, 64>(nb, threads, smem, st, g, br, u, kappa, n, in, out);
            else brick_go<R, 0, 64>(nb, threads, smem, st, g, br, u, kappa, n, in, out);
        }
        return;
    }
    constexpr int TS = 32;
    // right-hand sides handled side by side per block: balanced passes of <= 12
    const int passes = (n + 11) / 12;
    const int rpb = (n + passes - 1) / passes;
    const int threads = TS * rpb;
    const int nb = blocks_for(g.vol, TS);
    if (dag)
        k_dslash_mrhs<R, 1, TS><<<nb, threads, 0, st>>>(g, u, kappa, n, in, out);
    else
        k_dslash_mrhs<R, 0, TS><<<nb, threads, 0, st>>>(g, u, kappa, n, in, out);
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
void dslash_mrhs_fixed_f64(const Geom& g, const double2* u, double kappa, int dag, int n,
                           const double2* in, double2* out, cudaStream_t s) {
    const BrickChoice c{128, 0};
    launch_dslash_mrhs<double>(g, u, kappa, dag, n, in, out, s, &c);
}
void dslash_mrhs_fixed_f32(const Geom& g, const float2* u, float kappa, int dag, int n,
                           const float2* in, float2* out, cudaStream_t s) {
    const BrickChoice c{128, 0};
    launch_dslash_mrhs<float>(g, u, kappa, dag, n, in, out, s, &c);
}
}  // namespace seedcg
