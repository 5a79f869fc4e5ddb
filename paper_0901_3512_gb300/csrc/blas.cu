// BLAS-1 reductions and the SIMT projections against the stored basis:
//   gemm_t:  C = A^dag B   (V^dag [v, f] for re-orthogonalisation, V^dag R_0 for seeds)
//   gemm_n:  Y += A C      (the Gram-Schmidt subtraction, X = X_0 + V Y)
// Vectors are flat arrays of complex entries in the internal order; inner
// products do not depend on that order.
#include <cstdint>
#include <cstring>
#include <type_traits>

#include "kernels.cuh"
#include "reduce.cuh"

namespace seedcg {

namespace {

inline int nblocks(long n, int per_block, int cap) {
    long b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    return (int)(b < cap ? b : cap);
}

template <typename R>
__global__ void __launch_bounds__(kRedThreads)
k_dot(const cx_t<R>* __restrict__ a, const cx_t<R>* __restrict__ b, long n, double* partials,
      unsigned* ctr, double2* res) {
    double v[2] = {0.0, 0.0};
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
        cx_t<R> x = a[e], y = b[e];
        v[0] += (double)x.x * y.x + (double)x.y * y.y;
        v[1] += (double)x.x * y.y - (double)x.y * y.x;
    }
    grid_sum<2>(v, partials, ctr, [&](double* t) { *res = make_double2(t[0], t[1]); });
}

// ---------------------------------------------------------------------------
// gemm_t: block (tile of TA rows of A) x (slice of the entries); every thread
// keeps TA x NB complex accumulators in R, the block reduces them in FP64 and
// writes one partial per (slice, row, column); k_gemm_t_fin sums the slices
// in a fixed order.
// ---------------------------------------------------------------------------
template <typename R, typename AT, int TA, int NB>
__global__ void __launch_bounds__(kRedThreads)
k_gemm_t(const AT* __restrict__ A, long lda, int na, const cx_t<R>* __restrict__ B, long ldb,
         int nb, long n, double2* __restrict__ part) {
    const int a0 = blockIdx.x * TA;
    const int b0 = blockIdx.z * NB;
    const long slice = (n + gridDim.y - 1) / gridDim.y;
    const long e0 = blockIdx.y * slice;
    const long e1 = e0 + slice < n ? e0 + slice : n;
    cx_t<R> acc[TA][NB];
#pragma unroll
    for (int t = 0; t < TA; t++)
#pragma unroll
        for (int c = 0; c < NB; c++) acc[t][c] = mk<R>(0, 0);
    for (long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        cx_t<R> bv[NB];
#pragma unroll
        for (int c = 0; c < NB; c++)
            bv[c] = (b0 + c < nb) ? B[(size_t)(b0 + c) * ldb + e] : mk<R>(0, 0);
#pragma unroll
        for (int t = 0; t < TA; t++) {
            if (a0 + t < na) {
                cx_t<R> av = ld_cx<R>(A, (size_t)(a0 + t) * lda + e);
#pragma unroll
                for (int c = 0; c < NB; c++) acc[t][c] = cfma_conj(av, bv[c], acc[t][c]);
            }
        }
    }
    double v[2 * TA * NB];
#pragma unroll
    for (int t = 0; t < TA; t++)
#pragma unroll
        for (int c = 0; c < NB; c++) {
            v[2 * (t * NB + c)] = acc[t][c].x;
            v[2 * (t * NB + c) + 1] = acc[t][c].y;
        }
    block_sum<2 * TA * NB>(v);
    // part layout [slice][a][b] with b over the full nb
    for (int k = threadIdx.x; k < TA * NB; k += blockDim.x) {
        int t = k / NB, c = k % NB;
        if (a0 + t < na && b0 + c < nb)
            part[((size_t)blockIdx.y * na + a0 + t) * nb + b0 + c] =
                make_double2(v[2 * k], v[2 * k + 1]);
    }
}

__global__ void k_gemm_t_fin(const double2* __restrict__ part, int nsplit, int na, int nb,
                             double2* __restrict__ C, int ldc) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na * nb) return;
    int a = k / nb, b = k % nb;
    double2 s = make_double2(0.0, 0.0);
    for (int p = 0; p < nsplit; p++) {
        double2 z = part[((size_t)p * na + a) * nb + b];
        s.x += z.x;
        s.y += z.y;
    }
    C[(size_t)a * ldc + b] = s;
}

// ---------------------------------------------------------------------------
// gemm_n: one thread per entry, loops over the rows of A (coalesced across the
// warp for every row); the coefficients are staged in shared memory.
// ---------------------------------------------------------------------------
template <typename R, typename AT, typename YT, int NB>
__global__ void __launch_bounds__(256)
k_gemm_n(const AT* __restrict__ A, long lda, int na, const double2* __restrict__ C, int ldc,
         int nb, int b0, YT* __restrict__ Y, long ldy, long n, double sign) {
    constexpr int CH = 128;
    __shared__ cx_t<R> sc[CH][NB];
    for (long base = blockIdx.x * (long)blockDim.x; base < n; base += (long)gridDim.x * blockDim.x) {
        const long e = base + threadIdx.x;
        cx_t<R> acc[NB];
#pragma unroll
        for (int c = 0; c < NB; c++) acc[c] = mk<R>(0, 0);
        for (int a0 = 0; a0 < na; a0 += CH) {
            int cnt = na - a0 < CH ? na - a0 : CH;
            __syncthreads();
            for (int k = threadIdx.x; k < CH * NB; k += blockDim.x) {
                int a = k / NB, c = k % NB;
                double2 z = (a < cnt && b0 + c < nb) ? C[(size_t)(a0 + a) * ldc + b0 + c]
                                                     : make_double2(0.0, 0.0);
                sc[a][c] = mk<R>((R)(sign * z.x), (R)(sign * z.y));
            }
            __syncthreads();
            if (e < n) {
#pragma unroll 8
                for (int a = 0; a < cnt; a++) {
                    cx_t<R> av = ld_cx<R>(A, (size_t)(a0 + a) * lda + e);
#pragma unroll
                    for (int c = 0; c < NB; c++) acc[c] = cfma(av, sc[a][c], acc[c]);
                }
            }
        }
        if (e < n) {
#pragma unroll
            for (int c = 0; c < NB; c++) {
                if (b0 + c < nb) {
                    size_t idx = (size_t)(b0 + c) * ldy + e;
                    cx_t<double> y = ld_cx<double>(Y, idx);
                    st_cx(Y, idx, make_double2(y.x + (double)acc[c].x, y.y + (double)acc[c].y));
                }
            }
        }
    }
}

// Two consecutive complex entries of a basis row in one load (8 bytes of bf16x2,
// 16 of complex64), widened to cx_t<R>; FP64 rows take one entry per load.
template <typename R, typename AT> struct Row2;
template <typename R> struct Row2<R, __nv_bfloat162> {
    static constexpr int W = 2;
    __device__ __forceinline__ static void get(const __nv_bfloat162* p, cx_t<R> (&o)[2]) {
        const uint2 z = __ldcs(reinterpret_cast<const uint2*>(p));
        __nv_bfloat162 b0, b1;
        memcpy(&b0, &z.x, 4);
        memcpy(&b1, &z.y, 4);
        const float2 f0 = __bfloat1622float2(b0), f1 = __bfloat1622float2(b1);
        o[0] = mk<R>((R)f0.x, (R)f0.y);
        o[1] = mk<R>((R)f1.x, (R)f1.y);
    }
};
template <typename R> struct Row2<R, float2> {
    static constexpr int W = 2;
    __device__ __forceinline__ static void get(const float2* p, cx_t<R> (&o)[2]) {
        const float4 z = __ldcs(reinterpret_cast<const float4*>(p));
        o[0] = mk<R>((R)z.x, (R)z.y);
        o[1] = mk<R>((R)z.z, (R)z.w);
    }
};
template <typename R> struct Row2<R, double2> {
    static constexpr int W = 1;
    __device__ __forceinline__ static void get(const double2* p, cx_t<R> (&o)[1]) {
        const double2 z = __ldcs(p);
        o[0] = mk<R>((R)z.x, (R)z.y);
    }
};

// Y[:, b0 .. b0+NB) += A C[:, b0 ..] for up to NB = 12 columns in ONE pass over the rows
// of A (the seeds X += V Y of Eq. (1) read the stored basis once): a thread owns W
// consecutive entries (one 8- or 16-byte load per row), the coefficients of CH rows
// at a time sit in shared memory; Y is FP64 (double2).  n and lda are multiples of W.
template <typename R, typename AT, int NB>
__global__ void __launch_bounds__(256)
k_gemm_n_wide(const AT* __restrict__ A, long lda, int na, const double2* __restrict__ C, int ldc,
              int nb, int b0, double2* __restrict__ Y, long ldy, long n, double sign) {
    constexpr int CH = 64;
    constexpr int W = Row2<R, AT>::W;
    __shared__ cx_t<R> sc[CH][NB];
    const long ng = n / W;
    for (long base = blockIdx.x * (long)blockDim.x; base < ng; base += (long)gridDim.x * blockDim.x) {
        const long g = base + threadIdx.x;
        cx_t<R> acc[W][NB];
#pragma unroll
        for (int w = 0; w < W; w++)
#pragma unroll
            for (int c = 0; c < NB; c++) acc[w][c] = mk<R>(0, 0);
        for (int a0 = 0; a0 < na; a0 += CH) {
            const int cnt = na - a0 < CH ? na - a0 : CH;
            __syncthreads();
            for (int k = threadIdx.x; k < CH * NB; k += blockDim.x) {
                const int a = k / NB, c = k % NB;
                const double2 z = (a < cnt && b0 + c < nb) ? C[(size_t)(a0 + a) * ldc + b0 + c]
                                                           : make_double2(0.0, 0.0);
                sc[a][c] = mk<R>((R)(sign * z.x), (R)(sign * z.y));
            }
            __syncthreads();
            if (g < ng) {
#pragma unroll 4
                for (int a = 0; a < cnt; a++) {
                    cx_t<R> av[W];
                    Row2<R, AT>::get(A + (size_t)(a0 + a) * lda + g * W, av);
#pragma unroll
                    for (int c = 0; c < NB; c++) {
                        const cx_t<R> cc = sc[a][c];
#pragma unroll
                        for (int w = 0; w < W; w++) acc[w][c] = cfma(av[w], cc, acc[w][c]);
                    }
                }
            }
        }
        if (g < ng) {
#pragma unroll
            for (int c = 0; c < NB; c++) {
                if (b0 + c < nb) {
#pragma unroll
                    for (int w = 0; w < W; w++) {
                        const size_t idx = (size_t)(b0 + c) * ldy + g * W + w;
                        double2 y = Y[idx];
                        y.x += (double)acc[w][c].x;
                        y.y += (double)acc[w][c].y;
                        Y[idx] = y;
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// proj: the split-K projection C = V^dag X for NV <= 4 vectors, the shape of the
// re-orthogonalisation (NV = 2: [v_i, f]).  A block owns CHUNK consecutive
// entries: it stages X there in shared memory once, then its warps sweep the
// rows of V (RPW rows per pass, coalesced 256-byte row segments), reduce each
// row with warp shuffles and write one FP64 partial per (block, row, vector).
// V is read exactly once from HBM.
// ---------------------------------------------------------------------------
template <typename R, typename VT, int NV, int RPW, int CHUNK>
__global__ void __launch_bounds__(256, (sizeof(R) == 4 && NV == 2) ? 4 : 1)
k_proj_partial(const VT* __restrict__ V, long ldv, int na, const cx_t<R>* __restrict__ X,
               long ldx, int nv, long n, int chunk, int rg, double2* __restrict__ part) {
    // block (x, y): one chunk of entries (X chunk staged in shared memory)
    // against the rows of group y (rg rows); warp: RPW rows at a time; lane: W
    // consecutive entries per 16-byte load.  chunk and n are multiples of W
    // (host-checked).
    constexpr int W = VLoad<R, VT>::N;
    // X chunk in shared memory, component-major: entry e at sx[j][e % W][e / W], so
    // that the lanes of a warp (W consecutive entries each) read consecutive words
    __shared__ __align__(16) cx_t<R> sx[NV][W][CHUNK / W];
    const long e0 = (long)blockIdx.x * chunk;
    const int cnt = (int)(n - e0 < chunk ? n - e0 : chunk);
    for (int k = threadIdx.x; k < NV * chunk; k += blockDim.x) {
        const int j = k / chunk, e = k % chunk;
        sx[j][e % W][e / W] = (j < nv && e < cnt) ? X[(size_t)j * ldx + e0 + e] : mk<R>(0, 0);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    double2* out = part + (size_t)blockIdx.x * na * NV;
    const int rbeg = blockIdx.y * rg, rend = rbeg + rg < na ? rbeg + rg : na;
    for (int a0 = rbeg + warp * RPW; a0 < rend; a0 += nw * RPW) {
        cx_t<R> acc[RPW][NV];
#pragma unroll
        for (int r = 0; r < RPW; r++)
#pragma unroll
            for (int j = 0; j < NV; j++) acc[r][j] = mk<R>(0, 0);
        const VT* rows[RPW];
#pragma unroll
        for (int r = 0; r < RPW; r++) rows[r] = V + (size_t)(a0 + r < rend ? a0 + r : a0) * ldv + e0;
#pragma unroll 2
        for (int e = lane * W; e < cnt; e += 32 * W) {
            cx_t<R> a[RPW][W];
#pragma unroll
            for (int r = 0; r < RPW; r++) VLoad<R, VT>::get(rows[r] + e, a[r]);
#pragma unroll
            for (int w = 0; w < W; w++) {
#pragma unroll
                for (int j = 0; j < NV; j++) {
                    const cx_t<R> xv = sx[j][w][e / W];
#pragma unroll
                    for (int r = 0; r < RPW; r++) acc[r][j] = cfma_conj(a[r][w], xv, acc[r][j]);
                }
            }
        }
        // lane sums -> warp sum in the working precision (FP64 arithmetic is a
        // scarce pipe on this GPU; the partials over blocks are summed in FP64)
#pragma unroll
        for (int r = 0; r < RPW; r++) {
#pragma unroll
            for (int j = 0; j < NV; j++) {
                R re = acc[r][j].x, im = acc[r][j].y;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    re += __shfl_down_sync(0xffffffffu, re, o);
                    im += __shfl_down_sync(0xffffffffu, im, o);
                }
                if (lane == 0 && a0 + r < rend && j < nv)
                    out[(size_t)(a0 + r) * NV + j] = make_double2((double)re, (double)im);
            }
        }
    }
}

// C[a][j] = sum over blocks of part[b][a][j]: one warp per output, lanes stride
// over the blocks, then a fixed shuffle tree (deterministic)
template <int NV>
__global__ void k_proj_reduce(const double2* __restrict__ part, int nblk, int na, int nv,
                              double2* __restrict__ C, int ldc, int c0) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= na * nv) return;
    const int a = w / nv, j = w % nv;
    double re = 0.0, im = 0.0;
    for (int b = lane; b < nblk; b += 32) {
        const double2 z = part[((size_t)b * na + a) * NV + j];
        re += z.x;
        im += z.y;
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) C[(size_t)a * ldc + c0 + j] = make_double2(re, im);
}

__global__ void __launch_bounds__(kRedThreads)
k_nrm2(const double2* __restrict__ x, long n, double* partials, unsigned* ctr, double* out) {
    double p = 0.0;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
        const double2 z = x[e];
        p += z.x * z.x + z.y * z.y;
    }
    double red[1] = {p};
    grid_sum<1>(red, partials, ctr, [&](double* tot) { *out = sqrt(tot[0]); });
}

// y = b - y (FP64)
__global__ void k_bmy(const double2* __restrict__ b, double2* __restrict__ y, long n) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
        const double2 bb = b[e], yy = y[e];
        y[e] = make_double2(bb.x - yy.x, bb.y - yy.y);
    }
}

template <typename ST, typename DT>
__global__ void k_convert(const ST* __restrict__ src, DT* __restrict__ dst, long n) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
        cx_t<double> z = ld_cx<double>(src, e);
        st_cx(dst, e, z);
    }
}

}  // namespace

void axpby_f64(const double2* b, double2* y, long n, cudaStream_t s) {
    k_bmy<<<nblocks(n, 256, 152 * 16), 256, 0, s>>>(b, y, n);
    SEEDCG_CHECK_LAUNCH();
}

void k_norm2_public(const double2* x, long n, double* partials, unsigned* ctr, double* out,
                    cudaStream_t s) {
    k_nrm2<<<nblocks(n, kRedThreads * 8, 1216), kRedThreads, 0, s>>>(x, n, partials, ctr, out);
    SEEDCG_CHECK_LAUNCH();
}

template <typename R>
void dot(const cx_t<R>* a, const cx_t<R>* b, long n, double* partials, unsigned* ctr,
         double2* res, cudaStream_t s) {
    int nb = nblocks(n, kRedThreads * 8, kMaxRedBlocks);
    k_dot<R><<<nb, kRedThreads, 0, s>>>(a, b, n, partials, ctr, res);
    SEEDCG_CHECK_LAUNCH();
}

template <typename R, typename AT>
void gemm_t(const AT* A, long lda, int na, const cx_t<R>* B, long ldb, int nb, long n,
            double2* C, int ldc, double2* scratch, size_t scratch_elems, cudaStream_t s) {
    if (na <= 0 || nb <= 0) return;
    constexpr int TA = sizeof(R) == 8 ? 4 : 8;
    constexpr int NB = 2;
    int tiles = (na + TA - 1) / TA;
    int ctiles = (nb + NB - 1) / NB;
    // enough blocks for ~4 waves on 152 SMs, each slice >= 4096 entries
    long want = 2048 / ((long)tiles * ctiles) + 1;
    long maxs = n / 4096 + 1;
    long nsplit = want < maxs ? want : maxs;
    long cap = (long)(scratch_elems / ((size_t)na * nb));
    if (nsplit > cap) nsplit = cap;
    if (nsplit < 1) nsplit = 1;
    if (nsplit > 65535) nsplit = 65535;
    dim3 grid(tiles, (unsigned)nsplit, ctiles);
    k_gemm_t<R, AT, TA, NB><<<grid, kRedThreads, 0, s>>>(A, lda, na, B, ldb, nb, n, scratch);
    SEEDCG_CHECK_LAUNCH();
    int tot = na * nb;
    k_gemm_t_fin<<<(tot + 255) / 256, 256, 0, s>>>(scratch, (int)nsplit, na, nb, C, ldc);
    SEEDCG_CHECK_LAUNCH();
}

// staged entries per block: 32 KB of shared memory for the NV vectors
template <typename R, int NV> constexpr int proj_chunk() { return 32768 / (NV * (int)sizeof(cx_t<R>)); }

// entries per block: enough blocks to fill 152 SMs twice, at most the staging capacity
inline int proj_chunk_for(long n, int cap) {
    long c = (n + 303) / 304;
    c = (c + 127) / 128 * 128;   // whole 16-byte vectors per lane
    if (c < 256) c = 256;
    if (c > cap) c = cap;
    return (int)c;
}

template <typename R, typename AT>
size_t proj_scratch_elems(long n, int na) {
    const long c2 = proj_chunk_for(n, proj_chunk<R, 2>());
    const long c4 = proj_chunk_for(n, proj_chunk<R, 4>());
    const size_t a = (size_t)((n + c2 - 1) / c2) * 2, b = (size_t)((n + c4 - 1) / c4) * 4;
    return (a > b ? a : b) * (size_t)na;
}

template <typename R, typename AT>
void proj(const AT* A, long lda, int na, const cx_t<R>* X, long ldx, int nx, long n, double2* C,
          int ldc, double2* scratch, size_t scratch_elems, cudaStream_t s) {
    if (na <= 0 || nx <= 0) return;
    constexpr int W = 16 / (int)sizeof(AT);
    if (n % W != 0 || lda % W != 0 || (reinterpret_cast<uintptr_t>(A) & 15) != 0)
        throw Error{SEEDCG_ERR_ARG, "proj: basis rows must be 16-byte aligned whole vectors"};
    for (int c0 = 0; c0 < nx; c0 += 4) {
        const int nv = nx - c0 < 4 ? nx - c0 : 4;
        const cx_t<R>* Xc = X + (size_t)c0 * ldx;
        if (nv <= 2) {
            constexpr int CH = proj_chunk<R, 2>();
            const int ch = proj_chunk_for(n, CH);
            const int nblk = (int)((n + ch - 1) / ch);
            if ((size_t)nblk * na * 2 > scratch_elems) throw Error{SEEDCG_ERR_OOM, "proj scratch"};
            constexpr int RG = 8 * 4 * 4;
            k_proj_partial<R, AT, 2, 4, CH><<<dim3(nblk, (na + RG - 1) / RG), 256, 0, s>>>(
                A, lda, na, Xc, ldx, nv, n, ch, RG, scratch);
            SEEDCG_CHECK_LAUNCH();
            k_proj_reduce<2><<<(na * nv + 7) / 8, 256, 0, s>>>(scratch, nblk, na, nv, C, ldc, c0);
        } else {
            constexpr int CH = proj_chunk<R, 4>();
            const int ch = proj_chunk_for(n, CH);
            const int nblk = (int)((n + ch - 1) / ch);
            if ((size_t)nblk * na * 4 > scratch_elems) throw Error{SEEDCG_ERR_OOM, "proj scratch"};
            constexpr int RG = 8 * 2 * 4;
            k_proj_partial<R, AT, 4, 2, CH><<<dim3(nblk, (na + RG - 1) / RG), 256, 0, s>>>(
                A, lda, na, Xc, ldx, nv, n, ch, RG, scratch);
            SEEDCG_CHECK_LAUNCH();
            k_proj_reduce<4><<<(na * nv + 7) / 8, 256, 0, s>>>(scratch, nblk, na, nv, C, ldc, c0);
        }
        SEEDCG_CHECK_LAUNCH();
    }
}

template <typename R, typename AT, typename YT>
void gemm_n(const AT* A, long lda, int na, const double2* C, int ldc, int nb, YT* Y, long ldy,
            long n, double sign, cudaStream_t s) {
    if (na <= 0 || nb <= 0 || n <= 0) return;
    int blocks = nblocks(n, 256, 152 * 16);
    if (nb <= 2) {
        k_gemm_n<R, AT, YT, 2><<<blocks, 256, 0, s>>>(A, lda, na, C, ldc, nb, 0, Y, ldy, n, sign);
        SEEDCG_CHECK_LAUNCH();
        return;
    }
    constexpr int W = Row2<R, AT>::W;
    if constexpr (std::is_same<YT, double2>::value) {
        if (n % W == 0 && lda % W == 0 && (reinterpret_cast<uintptr_t>(A) & (W * sizeof(AT) - 1)) == 0) {
            // one pass over A per 12 columns (the 11 seeds of the twelve-source workload)
            const int wblocks = nblocks(n / W, 256, 152 * 8);
            for (int b0 = 0; b0 < nb; b0 += 12) {
                k_gemm_n_wide<R, AT, 12><<<wblocks, 256, 0, s>>>(A, lda, na, C, ldc, nb, b0, Y, ldy, n, sign);
                SEEDCG_CHECK_LAUNCH();
            }
            return;
        }
    }
    for (int b0 = 0; b0 < nb; b0 += 8) {
        k_gemm_n<R, AT, YT, 8><<<blocks, 256, 0, s>>>(A, lda, na, C, ldc, nb, b0, Y, ldy, n, sign);
        SEEDCG_CHECK_LAUNCH();
    }
}

template <typename ST, typename DT>
void convert(const ST* src, DT* dst, long n, cudaStream_t s) {
    if (n <= 0) return;
    k_convert<ST, DT><<<nblocks(n, 256, 152 * 32), 256, 0, s>>>(src, dst, n);
    SEEDCG_CHECK_LAUNCH();
}

// explicit instantiations
template void dot<double>(const double2*, const double2*, long, double*, unsigned*, double2*, cudaStream_t);
template void dot<float>(const float2*, const float2*, long, double*, unsigned*, double2*, cudaStream_t);

template void gemm_t<double, double2>(const double2*, long, int, const double2*, long, int, long, double2*, int, double2*, size_t, cudaStream_t);
template void gemm_t<float, float2>(const float2*, long, int, const float2*, long, int, long, double2*, int, double2*, size_t, cudaStream_t);
template void gemm_t<float, __nv_bfloat162>(const __nv_bfloat162*, long, int, const float2*, long, int, long, double2*, int, double2*, size_t, cudaStream_t);

template void proj<double, double2>(const double2*, long, int, const double2*, long, int, long, double2*, int, double2*, size_t, cudaStream_t);
template void proj<float, float2>(const float2*, long, int, const float2*, long, int, long, double2*, int, double2*, size_t, cudaStream_t);
template void proj<float, __nv_bfloat162>(const __nv_bfloat162*, long, int, const float2*, long, int, long, double2*, int, double2*, size_t, cudaStream_t);
template size_t proj_scratch_elems<double, double2>(long, int);
template size_t proj_scratch_elems<float, float2>(long, int);
template size_t proj_scratch_elems<float, __nv_bfloat162>(long, int);

template void gemm_n<double, double2, double2>(const double2*, long, int, const double2*, int, int, double2*, long, long, double, cudaStream_t);
template void gemm_n<float, float2, float2>(const float2*, long, int, const double2*, int, int, float2*, long, long, double, cudaStream_t);
template void gemm_n<float, float2, double2>(const float2*, long, int, const double2*, int, int, double2*, long, long, double, cudaStream_t);
template void gemm_n<float, __nv_bfloat162, float2>(const __nv_bfloat162*, long, int, const double2*, int, int, float2*, long, long, double, cudaStream_t);
template void gemm_n<float, __nv_bfloat162, double2>(const __nv_bfloat162*, long, int, const double2*, int, int, double2*, long, long, double, cudaStream_t);

template void convert<double2, double2>(const double2*, double2*, long, cudaStream_t);
template void convert<float2, double2>(const float2*, double2*, long, cudaStream_t);
template void convert<double2, float2>(const double2*, float2*, long, cudaStream_t);
template void convert<__nv_bfloat162, double2>(const __nv_bfloat162*, double2*, long, cudaStream_t);
template void convert<float2, float2>(const float2*, float2*, long, cudaStream_t);
template void convert<float2, __nv_bfloat162>(const float2*, __nv_bfloat162*, long, cudaStream_t);

}  // namespace seedcg
