// Internal declarations shared by the library's translation units.
//
// Device data layout (GB300: 32-wide warps, 128-byte lines; every kernel
// below maps one thread to one lattice site so that neighbouring threads
// touch neighbouring addresses):
//   spinor       element k = 3*spin + colour (0..11) of site s at flat complex index
//                ((k/2)*V + s)*2 + k%2: six "pair" planes, each site's two complex
//                entries of a plane adjacent (one 16-byte load in FP32, 32 bytes in FP64);
//                the same flat order in FP64 (double2) and FP32 (float2)
//   links        T2      [4][9][V]    U_mu(x)[a][b] at [(mu*9 + 3a + b)*V + s]
// A basis vector of V is one spinor in the same flat order, in the storage
// type of the precision mode (double2, float2 or bf16x2 per complex entry).
#pragma once

#include <atomic>

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>
#include <string>

#include "../../include/seedcg.h"

namespace seedcg {

// ----------------------------------------------------------------------------
// errors
// ----------------------------------------------------------------------------
struct Error {
    seedcg_status code;
    std::string msg;
};

#define SEEDCG_CUDA_TRY(expr)                                                              \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            throw ::seedcg::Error{e_ == cudaErrorMemoryAllocation ? SEEDCG_ERR_OOM         \
                                                                  : SEEDCG_ERR_CUDA,       \
                                  std::string(#expr) + ": " + cudaGetErrorString(e_)};     \
        }                                                                                  \
    } while (0)

// every kernel launch site ends with this: it checks the launch and counts it
extern std::atomic<unsigned long long> g_kernel_launches;
#define SEEDCG_CHECK_LAUNCH()                                                              \
    do {                                                                                   \
        ::seedcg::g_kernel_launches.fetch_add(1, std::memory_order_relaxed);               \
        SEEDCG_CUDA_TRY(cudaGetLastError());                                               \
    } while (0)

// ----------------------------------------------------------------------------
// complex helpers on CUDA vector types
// ----------------------------------------------------------------------------
template <typename R> struct Cx;
template <> struct Cx<double> { using T = double2; };
template <> struct Cx<float> { using T = float2; };
template <typename R> using cx_t = typename Cx<R>::T;

template <typename R> __host__ __device__ __forceinline__ cx_t<R> mk(R re, R im) {
    cx_t<R> z; z.x = re; z.y = im; return z;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
// a * b
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    C z; z.x = a.x * b.x - a.y * b.y; z.y = a.x * b.y + a.y * b.x; return z;
}
// acc + a * b
template <typename C> __host__ __device__ __forceinline__ C cfma(C a, C b, C acc) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
    return acc;
}
// acc + conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cfma_conj(C a, C b, C acc) {
    acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
    return acc;
}
// i * a
template <typename C> __host__ __device__ __forceinline__ C ci(C a) { C z; z.x = -a.y; z.y = a.x; return z; }
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) { a.x *= s; a.y *= s; return a; }

// ----------------------------------------------------------------------------
// lattice geometry
// ----------------------------------------------------------------------------
struct Geom {
    int L[4];        // Lx, Ly, Lz, Lt
    int vol;         // sites
    int stride[4];   // 1, Lx, Lx*Ly, Lx*Ly*Lz
};

inline Geom make_geom(const int dims[4]) {
    Geom g;
    for (int i = 0; i < 4; i++) g.L[i] = dims[i];
    g.stride[0] = 1;
    g.stride[1] = dims[0];
    g.stride[2] = dims[0] * dims[1];
    g.stride[3] = dims[0] * dims[1] * dims[2];
    g.vol = g.stride[3] * dims[3];
    return g;
}

// ----------------------------------------------------------------------------
// device buffers
// ----------------------------------------------------------------------------
// Owning device allocation: freed by the destructor (or release()); move-only.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes) {
        o.p = nullptr;
        o.bytes = 0;
    }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p;
            bytes = o.bytes;
            o.p = nullptr;
            o.bytes = 0;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void ensure(size_t n) {
        if (n <= bytes) return;
        release();
        SEEDCG_CUDA_TRY(cudaMalloc(&p, n));
        bytes = n;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

// ----------------------------------------------------------------------------
// launchers implemented in dslash.cu
// ----------------------------------------------------------------------------
// canonical complex128 AoS [n][V][12] <-> internal
void to_internal_f64(const double* in, double2* out, int vol, int n, cudaStream_t s);
void from_internal_f64(const double2* in, double* out, int vol, int n, cudaStream_t s);
void to_internal_f32(const double* in, float2* out, int vol, int n, cudaStream_t s);
void from_internal_f32(const float2* in, double* out, int vol, int n, cudaStream_t s);
void gauge_to_internal(const double* in, double2* u64, float2* u32, int vol, cudaStream_t s);

// out = D in (dag = 0) or D^dag in (dag = 1); single right-hand side
void dslash_f64(const Geom& g, const double2* u, double kappa, int dag, const double2* in,
                double2* out, cudaStream_t s);
void dslash_f32(const Geom& g, const float2* u, float kappa, int dag, const float2* in,
                float2* out, cudaStream_t s);
// n right-hand sides at in + r*12*V; links staged once per tile of sites
void dslash_mrhs_f64(const Geom& g, const double2* u, double kappa, int dag, int n,
                     const double2* in, double2* out, cudaStream_t s);
void dslash_mrhs_f32(const Geom& g, const float2* u, float kappa, int dag, int n,
                     const float2* in, float2* out, cudaStream_t s);

// even-odd preconditioned system (evenodd.cu), FP64 half vectors in the internal layout:
// out_r = A^dag A x_r, A = 1 - kappa^2 H_oe H_eo (te, y: one even / odd half scratch each)
void eo_apply_mdag_m_f64(const Geom& g, const double2* u, double kappa, int n, const double2* x,
                         double2* te, double2* y, double2* out, cudaStream_t st);
// phi = eta_o + kappa H_oe eta_e and b = A^dag phi for n full fields eta
void eo_rhs_f64(const Geom& g, const double2* u, double kappa, int n, const double2* eta, double2* phi,
                double2* b, double2* ee, double2* eo, double2* te, cudaStream_t st);
// half[r] = the parity-p sites of full[r] for n fields
void eo_gather_f64(const Geom& g, int p, int n, const double2* full, double2* half, cudaStream_t st);
// full x from x_o: x_e = eta_e + kappa H_eo x_o
void eo_reconstruct_f64(const Geom& g, const double2* u, double kappa, int n, const double2* x_odd,
                        const double2* eta, double2* x, double2* ee, double2* xe, cudaStream_t st);

// the multi-RHS kernel with its default tile shape, never timing alternatives
void dslash_mrhs_fixed_f64(const Geom& g, const double2* u, double kappa, int dag, int n,
                           const double2* in, double2* out, cudaStream_t s);
void dslash_mrhs_fixed_f32(const Geom& g, const float2* u, float kappa, int dag, int n,
                           const float2* in, float2* out, cudaStream_t s);

}  // namespace seedcg
