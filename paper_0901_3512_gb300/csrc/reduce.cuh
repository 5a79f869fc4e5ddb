// Deterministic block and grid reductions in FP64.
//
// Every reducing kernel writes one partial per block into a fixed slot; the
// last block to finish (elected through an atomic ticket) sums the slots in
// a fixed order and runs the finalisation on one thread.  The result does not
// depend on block scheduling, so repeated runs are bitwise identical.
#pragma once

#include "internal.cuh"

namespace seedcg {

constexpr int kRedThreads = 256;  // every reducing kernel uses this block size
constexpr int kMaxRedBlocks = 4096;

// warp sum in the value's own precision (FP32 sums stay off the scarce FP64 pipe)
template <typename T> __device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum v[k] over the block; on return every thread holds the block totals.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double sh[NV][kRedThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double t = warp_sum(v[k]);
        if (lane == 0) sh[k][warp] = t;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) {
            double t = lane < nw ? sh[k][lane] : 0.0;
            t = warp_sum(t);
            if (lane == 0) sh[k][0] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = sh[k][0];
    __syncthreads();
}

// Grid-wide sum over a 1-D or 2-D grid.  partials holds NV * nblocks doubles,
// counter one unsigned that is zero on entry (it is reset on exit).  fin(tot)
// runs once, on thread 0 of the last block, with the grid totals.
template <int NV, typename Fin>
__device__ __forceinline__ void grid_sum(double (&v)[NV], double* partials, unsigned* counter,
                                         Fin fin) {
    __shared__ bool s_last;
    block_sum<NV>(v);
    const unsigned nblk = gridDim.x * gridDim.y;
    const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) partials[(size_t)k * nblk + bid] = v[k];
        __threadfence();
        unsigned t = atomicAdd(counter, 1u);
        s_last = (t == nblk - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double tot[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) tot[k] = 0.0;
    for (unsigned b = threadIdx.x; b < nblk; b += blockDim.x) {
#pragma unroll
        for (int k = 0; k < NV; k++) tot[k] += __ldcg(partials + (size_t)k * nblk + b);
    }
    block_sum<NV>(tot);
    if (threadIdx.x == 0) {
        fin(tot);
        *counter = 0u;
        __threadfence();
    }
}

// ---------------------------------------------------------------------------
// loads of one complex entry from the three storage types, widened to R
// ---------------------------------------------------------------------------
template <typename R> __device__ __forceinline__ cx_t<R> ld_cx(const double2* p, size_t i) {
    double2 z = __ldg(p + i); return mk<R>((R)z.x, (R)z.y);
}
template <typename R> __device__ __forceinline__ cx_t<R> ld_cx(const float2* p, size_t i) {
    float2 z = __ldg(p + i); return mk<R>((R)z.x, (R)z.y);
}
template <typename R> __device__ __forceinline__ cx_t<R> ld_cx(const __nv_bfloat162* p, size_t i) {
    float2 z = __bfloat1622float2(p[i]); return mk<R>((R)z.x, (R)z.y);
}
__device__ __forceinline__ void st_cx(double2* p, size_t i, double2 z) { p[i] = z; }
__device__ __forceinline__ void st_cx(double2* p, size_t i, float2 z) { p[i] = make_double2(z.x, z.y); }
__device__ __forceinline__ void st_cx(float2* p, size_t i, double2 z) { p[i] = make_float2((float)z.x, (float)z.y); }
__device__ __forceinline__ void st_cx(float2* p, size_t i, float2 z) { p[i] = z; }
__device__ __forceinline__ void st_cx(__nv_bfloat162* p, size_t i, float2 z) { p[i] = __float22bfloat162_rn(z); }
__device__ __forceinline__ void st_cx(__nv_bfloat162* p, size_t i, double2 z) {
    p[i] = __float22bfloat162_rn(make_float2((float)z.x, (float)z.y));
}

// One 16-byte load of consecutive complex elements of type VT (1 double2,
// 2 float2 or 4 bf16x2), widened to cx_t<R>; marked streaming (evict-first):
// the stored basis is read once per use and should not push the iteration
// vectors out of L2.  p must be 16-byte aligned.
template <typename R, typename VT> struct VLoad;
template <typename R> struct VLoad<R, double2> {
    static constexpr int N = 1;
    __device__ __forceinline__ static void get(const double2* p, cx_t<R> (&o)[1]) {
        const double2 z = __ldcs(p);
        o[0] = mk<R>((R)z.x, (R)z.y);
    }
};
template <typename R> struct VLoad<R, float2> {
    static constexpr int N = 2;
    __device__ __forceinline__ static void get(const float2* p, cx_t<R> (&o)[2]) {
        const float4 z = __ldcs(reinterpret_cast<const float4*>(p));
        o[0] = mk<R>((R)z.x, (R)z.y);
        o[1] = mk<R>((R)z.z, (R)z.w);
    }
};
template <typename R> struct VLoad<R, __nv_bfloat162> {
    static constexpr int N = 4;
    __device__ __forceinline__ static void get(const __nv_bfloat162* p, cx_t<R> (&o)[4]) {
        const uint4 z = __ldcs(reinterpret_cast<const uint4*>(p));
        const unsigned w[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            __nv_bfloat162 b;
            memcpy(&b, &w[k], 4);
            const float2 f = __bfloat1622float2(b);
            o[k] = mk<R>((R)f.x, (R)f.y);
        }
    }
};

}  // namespace seedcg
