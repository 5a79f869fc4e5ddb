// Tensor-core projection against the stored basis (bf16 V), sm_103a:
//
//   C = V^dag X   for a few complex vectors X (the re-orthogonalisation's
//                 [v_i, f] of Algorithm 1 step 8, or R_0 for the Eq. (1) seeds)
//
// as a real GEMM  D[a][c] = sum_k A[a][k] B[c][k]  with
//   A = V viewed as bf16 [rows][K = 2N] (each basis vector one row, re/im interleaved),
//   B = [Re-column, Im-column] per complex vector x: (xr, xi) and (xi, -xr) interleaved,
//       rounded to bf16, so that D[a][2j] = Re(v_a^dag x_j), D[a][2j+1] = Im(v_a^dag x_j).
// One CTA owns R tiles of 128 rows of V and a range of K (split-K); per stage
// TMA streams KC 64-wide K chunks of each of its R row tiles (128x64 boxes)
// and of B (NBx64 boxes) into a shared-memory ring (128-byte swizzle), so one
// B chunk serves R row tiles and each row is read in runs of KC x 128 bytes;
// one thread issues tcgen05.mma (M=128, N=NB, K=16, bf16 -> fp32) into R TMEM
// accumulators; after the K range four warps read the accumulators back with
// tcgen05.ld and write FP32 partials, which a second kernel sums over the
// splits in FP64 (fixed order: deterministic).
//
// Every wait on an mbarrier is bounded (1 s of globaltimer); on expiry the
// kernel records an error code, stops issuing work, waits (bounded) for the
// copies it already issued, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "kernels.cuh"
#include "reduce.cuh"
#include "tc_proj.cuh"
#include "tc_common.cuh"

#include <algorithm>
#include <cstdio>
#include <cstdlib>

namespace seedcg {

namespace {

using namespace tc;

constexpr int BM = 128;
constexpr int BK = 64;          // bf16 elements per 128-byte swizzle row
constexpr uint32_t A_BOX_BYTES = BM * BK * 2;  // 16 KB
// shared memory per CTA: two CTAs per SM when a stage is small, one otherwise
constexpr uint32_t smem_budget(uint32_t stage) { return stage <= 40 * 1024 ? 108 * 1024 : 200 * 1024; }

template <int NB, int R, int KC>
struct TcSmem {
    static constexpr uint32_t B_BOX = ((NB * BK * 2) + 1023) & ~1023u;
    static constexpr uint32_t A_STAGE = R * KC * A_BOX_BYTES;
    static constexpr uint32_t B_STAGE = KC * B_BOX;
    static constexpr int STAGES_RAW = (int)(smem_budget(A_STAGE + B_STAGE) / (A_STAGE + B_STAGE));
    static constexpr int STAGES = STAGES_RAW > 8 ? 8 : STAGES_RAW;
    static_assert(STAGES >= 2, "tensor-core projection stage too large");
    static constexpr uint32_t BYTES = STAGES * (A_STAGE + B_STAGE) + 1024 + 256;
    static constexpr uint32_t TMEM_COLS = R * NB <= 32 ? 32 : (R * NB <= 64 ? 64 : (R * NB <= 128 ? 128 : 256));
};

// NB: columns of B (multiple of 16, <= 64).  part: float [nsplit][rows_valid][NB].
// blockIdx.x = group of R row tiles, blockIdx.y = K split of kb_per_split
// 64-wide chunks (a multiple of KC).
template <int NB, int R, int KC>
__global__ void __launch_bounds__(128, 1)
k_tc_proj(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
          int nkb, int kb_per_split, int rows_valid, float* __restrict__ part,
          int* __restrict__ err) {
    using SM = TcSmem<NB, R, KC>;
    constexpr int STAGES = SM::STAGES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + STAGES * SM::A_STAGE;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + STAGES * SM::B_STAGE);
    uint64_t* empty = full + STAGES;
    uint64_t* done = empty + STAGES;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* s_fail = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kb0 = blockIdx.y * kb_per_split;
    // chunks of this split (past nkb the loads read zeros, so whole stages are fine)
    const int kb1 = min(kb0 + kb_per_split, ((nkb + KC - 1) / KC) * KC);
    const int nst = kb1 > kb0 ? (kb1 - kb0) / KC : 0;
    constexpr uint32_t TMEM_COLS = SM::TMEM_COLS;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem_d = *tmem_slot;
    const int tile0 = blockIdx.x * R;
    // row tiles of this CTA that hold valid rows (the others are neither loaded nor multiplied)
    const int tiles_valid = (rows_valid + BM - 1) / BM;
    const int nt = tiles_valid - tile0 < R ? tiles_valid - tile0 : R;

    int issued = 0;  // TMA stages issued by the producer
    if (nst > 0) {
        if (warp == 0 && lane == 0) {
            // producer: TMA loads of V (R row tiles) and B, KC chunks per stage
            for (int it = 0; it < nst; it++) {
                const int s = it % STAGES;
                const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u) || *s_fail) {
                    *s_fail = 1;
                    break;
                }
                mbar_expect_tx(&full[s], (uint32_t)nt * KC * A_BOX_BYTES + KC * NB * BK * 2);
#pragma unroll
                for (int c = 0; c < KC; c++) {
                    const int x = (kb0 + it * KC + c) * BK;
#pragma unroll
                    for (int t = 0; t < R; t++)
                        if (t < nt)
                            tma_load_2d(sA + s * SM::A_STAGE + (t * KC + c) * A_BOX_BYTES, &tmA, &full[s], x,
                                        (tile0 + t) * BM);
                    tma_load_2d(sB + s * SM::B_STAGE + c * SM::B_BOX, &tmB, &full[s], x, 0);
                }
                issued = it + 1;
            }
        } else if (warp == 1 && lane == 0) {
            // MMA issuer: R accumulators, NB columns apart in TMEM
            constexpr uint32_t idesc = umma_idesc_bf16(NB);
            for (int it = 0; it < nst; it++) {
                const int s = it % STAGES;
                const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                if (!mbar_wait(&full[s], ph) || *s_fail) {
                    *s_fail = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int c = 0; c < KC; c++) {
                    const uint32_t b0 = smem_u32(sB + s * SM::B_STAGE + c * SM::B_BOX);
#pragma unroll
                    for (int kk = 0; kk < BK / 16; kk++) {
                        const uint64_t db = umma_desc_sw128(b0 + kk * 32);
#pragma unroll
                        for (int t = 0; t < R; t++) {
                            if (t >= nt) continue;
                            const uint32_t a0 = smem_u32(sA + s * SM::A_STAGE + (t * KC + c) * A_BOX_BYTES);
                            const uint64_t da = umma_desc_sw128(a0 + kk * 32);
                            umma_bf16(tmem_d + (uint32_t)(t * NB), da, db, idesc,
                                      (it > 0 || c > 0 || kk > 0) ? 1u : 0u);
                        }
                    }
                }
                umma_commit(&empty[s]);
            }
            umma_commit(done);
        }
        // everyone waits for the accumulator (bounded)
        if (!mbar_wait(done, 0)) *s_fail = 1;
    }
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    const bool failed = *s_fail != 0;
    if (failed) {
        if (threadIdx.x == 0) atomicExch(err, SEEDCG_ERR_TIMEOUT);
        // drain the copies this CTA issued (bounded), so none lands after exit
        if (warp == 0 && lane == 0) {
            for (int it = 0; it < issued; it++) {
                const int s = it % STAGES;
                mbar_wait(&full[s], (uint32_t)(it / STAGES) & 1u);
            }
        }
    } else {
        // epilogue: warp w owns TMEM lanes [32w, 32w + 32) = rows of each tile
#pragma unroll
        for (int t = 0; t < R; t++) {
            if (t >= nt) continue;
            const int row = (tile0 + t) * BM + warp * 32 + lane;
            float* out = part + ((size_t)blockIdx.y * rows_valid + row) * NB;
#pragma unroll
            for (int c0 = 0; c0 < NB; c0 += 16) {
                float v[16];
                if (nst > 0) {
                    tmem_ld16<NB>(tmem_d + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * NB + c0), v);
                } else {
#pragma unroll
                    for (int k = 0; k < 16; k++) v[k] = 0.f;
                }
                if (row < rows_valid) {
#pragma unroll
                    for (int k = 0; k < 16; k += 4)
                        *reinterpret_cast<float4*>(out + c0 + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_d),
                     "r"(TMEM_COLS));
    }
}

// C[a][j] (complex, double2) = sum over splits of part[split][a][2j] + i part[..][2j+1];
// one warp per output, lanes stride over the splits, fixed shuffle tree
__global__ void k_tc_reduce(const float* __restrict__ part, int nsplit, int rows, int nb_cols,
                            int nvec, double2* __restrict__ C, int ldc) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= rows * nvec) return;
    const int a = w / nvec, j = w % nvec;
    double re = 0.0, im = 0.0;
    for (int p = lane; p < nsplit; p += 32) {
        const float* q = part + ((size_t)p * rows + a) * nb_cols;
        re += q[2 * j];
        im += q[2 * j + 1];
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) C[(size_t)a * ldc + j] = make_double2(re, im);
}

// B[2j][2e..2e+1] = (xr, xi), B[2j+1][2e..2e+1] = (xi, -xr) in bf16, for x_j = X + j*ldx
__global__ void k_tc_build_b(const float2* __restrict__ X, long ldx, int nvec, long n,
                             __nv_bfloat162* __restrict__ Bm) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
        for (int j = 0; j < nvec; j++) {
            float2 x = X[(size_t)j * ldx + e];
            Bm[(size_t)(2 * j) * n + e] = __floats2bfloat162_rn(x.x, x.y);
            Bm[(size_t)(2 * j + 1) * n + e] = __floats2bfloat162_rn(x.y, -x.x);
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        SEEDCG_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                         cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !p)
            throw Error{SEEDCG_ERR_CUDA, "cuTensorMapEncodeTiled is not available"};
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D bf16 tensor map over [rows][k_elems] with a box of [box_rows][64]
CUtensorMap make_map(const void* base, uint64_t k_elems, uint64_t rows, uint32_t box_rows) {
    CUtensorMap m;
    cuuint64_t dims[2] = {k_elems, rows};
    cuuint64_t strides[1] = {k_elems * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
    cuuint32_t es[2] = {1, 1};
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (strides[0] & 15))
        throw Error{SEEDCG_ERR_ARG, "tensor map base/stride not 16-byte aligned"};
    CUresult r = get_encode()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                              strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error{SEEDCG_ERR_CUDA, "cuTensorMapEncodeTiled failed"};
    return m;
}

template <int NB, int R, int KC>
void launch_tc_shape(const CUtensorMap& ma, const CUtensorMap& mb, int rows, long kelems, float* part,
                     size_t part_elems, int* err, int* nsplit_out, cudaStream_t st) {
    using SM = TcSmem<NB, R, KC>;
    const int nkb = (int)((kelems + BK - 1) / BK);
    const int tiles = (rows + BM - 1) / BM;
    const int groups = (tiles + R - 1) / R;
    static int occ = 0, nsm = 0;
    if (!occ) {
        SEEDCG_CUDA_TRY(cudaFuncSetAttribute(k_tc_proj<NB, R, KC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::BYTES));
        int dev = 0;
        SEEDCG_CUDA_TRY(cudaGetDevice(&dev));
        SEEDCG_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        SEEDCG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tc_proj<NB, R, KC>, 128,
                                                                      SM::BYTES));
        if (occ < 1) throw Error{SEEDCG_ERR_CUDA, "tensor-core projection does not fit on an SM"};
    }
    // whole waves (two by default; SEEDCG_TC_WAVES overrides): as many K splits
    // as keep groups * nsplit within waves x the resident CTAs, each split at
    // least 16 chunks long and a multiple of KC chunks
    int waves = 2;
    if (const char* e = getenv("SEEDCG_TC_WAVES")) waves = std::max(1, std::min(8, atoi(e)));
    const int resident = nsm * occ * waves;
    int nsplit = resident / groups;
    if (nsplit < 1) nsplit = 1;
    const int maxs = nkb / 16 > 0 ? nkb / 16 : 1;
    if (nsplit > maxs) nsplit = maxs;
    long cap = (long)(part_elems / ((size_t)rows * NB));
    if (nsplit > cap) nsplit = (int)cap;
    if (nsplit < 1) throw Error{SEEDCG_ERR_OOM, "tensor-core projection: partial buffer too small"};
    int per = (nkb + nsplit - 1) / nsplit;
    per = (per + KC - 1) / KC * KC;
    nsplit = (nkb + per - 1) / per;
    dim3 grid(groups, nsplit);
    k_tc_proj<NB, R, KC><<<grid, 128, SM::BYTES, st>>>(ma, mb, nkb, per, rows, part, err);
    SEEDCG_CHECK_LAUNCH();
    *nsplit_out = nsplit;
}

// row tiles per CTA (R) and K chunks per stage (KC); SEEDCG_TC_SHAPE="R,KC"
// overrides the default for measurements
void tc_shape(int& r, int& kc) {
    r = 4;
    kc = 1;
    if (const char* e = getenv("SEEDCG_TC_SHAPE")) {
        int a = 0, b = 0;
        if (sscanf(e, "%d,%d", &a, &b) == 2 && (a == 1 || a == 2 || a == 4) && (b == 1 || b == 2 || b == 4)) {
            r = a;
            kc = b;
        }
    }
}

template <int NB>
void launch_tc(const CUtensorMap& ma, const CUtensorMap& mb, int rows, long kelems, float* part,
               size_t part_elems, int* err, int* nsplit_out, cudaStream_t st) {
    int r, kc;
    tc_shape(r, kc);
#define SEEDCG_TC(RR, KK)                                                                             \
    if (r == RR && kc == KK) {                                                                        \
        launch_tc_shape<NB, RR, KK>(ma, mb, rows, kelems, part, part_elems, err, nsplit_out, st);   \
        return;                                                                                       \
    }
    SEEDCG_TC(1, 1)
    SEEDCG_TC(2, 1)
    SEEDCG_TC(2, 2)
    SEEDCG_TC(1, 2)
    SEEDCG_TC(1, 4)
#undef SEEDCG_TC
    launch_tc_shape<NB, 4, 1>(ma, mb, rows, kelems, part, part_elems, err, nsplit_out, st);
}

// Failure-detection self-check: one thread waits on an mbarrier that nothing
// arrives at, through the bounded wait every tensor-core kernel uses; the wait
// must give up after limit_ns and the kernel report SEEDCG_ERR_TIMEOUT.
__global__ void k_wait_selftest(unsigned long long limit_ns, int* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) *status = mbar_wait_for(&bar, 0u, limit_ns) ? SEEDCG_OK : SEEDCG_ERR_TIMEOUT;
}

}  // namespace

size_t tc_b_bytes(long n, int nvec) {
    int nb = tc_cols(nvec);
    return (size_t)nb * n * sizeof(__nv_bfloat162);
}

int tc_cols(int nvec) {
    int c = 2 * nvec;
    return c <= 16 ? 16 : (c <= 32 ? 32 : (c <= 48 ? 48 : 64));
}

void tc_project(const __nv_bfloat162* V, int rows_alloc, int rows, const float2* X, long ldx,
                int nvec, long n, __nv_bfloat162* Bm, float* part, size_t part_elems,
                double2* C, int ldc, int* err, cudaStream_t st) {
    if (rows <= 0 || nvec <= 0) return;
    if (nvec > 32) throw Error{SEEDCG_ERR_ARG, "tensor-core projection takes at most 32 vectors"};
    const int nb = tc_cols(nvec);
    const long kel = 2 * n;  // bf16 elements per basis vector
    {
        int blocks = (int)std::min<long>((n + 255) / 256, 152 * 16);
        k_tc_build_b<<<blocks, 256, 0, st>>>(X, ldx, nvec, n, Bm);
        SEEDCG_CHECK_LAUNCH();
    }
    CUtensorMap ma = make_map(V, (uint64_t)kel, (uint64_t)rows_alloc, BM);
    CUtensorMap mb = make_map(Bm, (uint64_t)kel, (uint64_t)nb, (uint32_t)nb);
    int nsplit = 0;
    switch (nb) {
        case 16: launch_tc<16>(ma, mb, rows, kel, part, part_elems, err, &nsplit, st); break;
        case 32: launch_tc<32>(ma, mb, rows, kel, part, part_elems, err, &nsplit, st); break;
        case 48: launch_tc<48>(ma, mb, rows, kel, part, part_elems, err, &nsplit, st); break;
        default: launch_tc<64>(ma, mb, rows, kel, part, part_elems, err, &nsplit, st); break;
    }
    const int tot = rows * nvec;
    k_tc_reduce<<<(tot + 7) / 8, 256, 0, st>>>(part, nsplit, rows, nb, nvec, C, ldc);
    SEEDCG_CHECK_LAUNCH();
}

}  // namespace seedcg

extern "C" seedcg_status seedcg_selftest_bounded_wait(double limit_ms, int* kernel_status) {
    if (!kernel_status || !(limit_ms > 0.0) || limit_ms > 1000.0) return SEEDCG_ERR_ARG;
    int* d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return SEEDCG_ERR_OOM;
    const int init = 1;
    cudaMemcpy(d, &init, sizeof(int), cudaMemcpyHostToDevice);
    seedcg::k_wait_selftest<<<1, 32>>>((unsigned long long)(limit_ms * 1e6), d);
    seedcg::g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(kernel_status, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? SEEDCG_OK : SEEDCG_ERR_CUDA;
}
