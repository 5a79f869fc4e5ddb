// seedcg_apply_noalloc: the operator application of seedcg_apply for callers
// that cannot allocate device memory.  Its scratch (the internal-layout copies
// of the input and of the intermediate / output fields) lives in one fixed
// file-scope device array instead of per-call cudaMalloc buffers.
#include <cstring>
#include <mutex>

#include "handle.cuh"
#include "internal.cuh"

namespace seedcg {

// 16 MiB, reserved on every GPU that loads this library until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current).
// In host code the array's name is only a host-side stand-in; the address a
// kernel may use comes from cudaGetSymbolAddress, looked up once per device.
void* scratch_on(int device) {
    if (device < 0 || device >= kMaxDevices)
        throw Error{SEEDCG_ERR_ARG, "device ordinal out of range for the fixed scratch"};
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[device]) {
        void* p = nullptr;
        SEEDCG_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_ptr[device] = p;
    }
    return g_ptr[device];
}

// True when p is device (or managed) memory of `device`.  Asking the runtime
// allocates nothing; a host or unregistered pointer must be refused here,
// before any kernel dereferences it.
bool on_device(const void* p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

}  // namespace
}  // namespace seedcg

using seedcg::Error;

extern "C" seedcg_status seedcg_apply_noalloc(seedcg_handle* h, int op, int prec, int multi, int n,
                                              const double* in, double* out, void* stream) {
    if (!h) return SEEDCG_ERR_ARG;
    if (op < 0 || op > 2 || prec < 0 || prec > 1 || n < 0) {
        h->err = "bad op/prec/n";
        return SEEDCG_ERR_ARG;
    }
    if (n == 0) return SEEDCG_OK;
    if (!in || !out || in == out) {
        h->err = "in/out NULL or aliased";
        return SEEDCG_ERR_ARG;
    }
    if (!seedcg::on_device(in, h->device) || !seedcg::on_device(out, h->device)) {
        h->err = "seedcg_apply_noalloc: in and out must be device memory of the handle's GPU";
        return SEEDCG_ERR_ARG;
    }
    const int vol = h->g.vol;
    const size_t nf = (size_t)n * vol * 12;
    const size_t esz = prec == 0 ? sizeof(double2) : sizeof(float2);
    const size_t need = 3 * nf * esz;
    if (need > seedcg::kNoAllocScratchBytes) {
        h->err = "seedcg_apply_noalloc: n * volume too large for the fixed 16 MiB scratch "
                 "(needs 3 * n * V * 12 * (16 B FP64 | 8 B FP32))";
        return SEEDCG_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    try {
        SEEDCG_CUDA_TRY(cudaSetDevice(h->device));
        char* b0 = static_cast<char*>(seedcg::scratch_on(h->device));
        void* A = b0;
        void* Bv = b0 + nf * esz;
        void* Cv = b0 + 2 * nf * esz;
        if (prec == 0) {
            seedcg::to_internal_f64(in, (double2*)A, vol, n, st);
            auto apply = [&](int dag, const double2* x, double2* y) {
                if (multi)
                    seedcg::dslash_mrhs_fixed_f64(h->g, h->u64.as<double2>(), h->kappa, dag, n, x, y, st);
                else
                    for (int r = 0; r < n; r++)
                        seedcg::dslash_f64(h->g, h->u64.as<double2>(), h->kappa, dag,
                                           x + (size_t)r * 12 * vol, y + (size_t)r * 12 * vol, st);
            };
            const double2* res = (const double2*)Bv;
            if (op == 0) apply(0, (double2*)A, (double2*)Bv);
            else if (op == 1) apply(1, (double2*)A, (double2*)Bv);
            else { apply(0, (double2*)A, (double2*)Bv); apply(1, (double2*)Bv, (double2*)Cv); res = (double2*)Cv; }
            seedcg::from_internal_f64(res, out, vol, n, st);
        } else {
            seedcg::to_internal_f32(in, (float2*)A, vol, n, st);
            const float k = (float)h->kappa;
            auto apply = [&](int dag, const float2* x, float2* y) {
                if (multi)
                    seedcg::dslash_mrhs_fixed_f32(h->g, h->u32.as<float2>(), k, dag, n, x, y, st);
                else
                    for (int r = 0; r < n; r++)
                        seedcg::dslash_f32(h->g, h->u32.as<float2>(), k, dag,
                                           x + (size_t)r * 12 * vol, y + (size_t)r * 12 * vol, st);
            };
            const float2* res = (const float2*)Bv;
            if (op == 0) apply(0, (float2*)A, (float2*)Bv);
            else if (op == 1) apply(1, (float2*)A, (float2*)Bv);
            else { apply(0, (float2*)A, (float2*)Bv); apply(1, (float2*)Bv, (float2*)Cv); res = (float2*)Cv; }
            seedcg::from_internal_f32(res, out, vol, n, st);
        }
        SEEDCG_CUDA_TRY(cudaStreamSynchronize(st));
        return SEEDCG_OK;
    } catch (const Error& e) {
        h->err = e.msg;
        return e.code;
    }
}
