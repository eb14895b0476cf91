// Dose tally that allocates no memory, for callers that must not call
// cudaMalloc: code inside a framework whose caching allocator owns the
// device memory (a raw cudaMalloc can fail against memory the allocator has
// reserved, and it synchronises the device), and real-time or embedded
// callers that forbid allocation after start-up.  The regular doctors_dose
// stages the conversion-factor table in a device buffer it allocates per
// call; this variant stages it in a fixed file-scope device array instead
// and writes only into the caller's device buffer.
//
// The array is part of the library's device image, so every GPU that loads
// the library holds it until the process exits.  All calls share it: a call
// overwrites the whole table it uses before launching, so nothing has to
// start at zero, and calls that overlap on the GPU (different streams or
// problems at the same time) race on its contents.
#include <cmath>
#include <mutex>
#include <string>

#include "doctors_internal.h"

namespace doctors {

// n_mat * G conversion factors, FP64 (8 materials x 32 groups)
constexpr int kNoAllocFactors = 256;

static __device__ __align__(256) double g_noalloc_factors[kNoAllocFactors];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_symbol_mu;
double* g_symbol_ptr[kMaxDevices] = {};

// Device address of the factor array on the current device, looked up once
// per device (with that device current) and cached for the life of the
// process: the cache assumes one context per device (a cudaDeviceReset would
// leave a stale address).
cudaError_t factor_table_address(int device, double** out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_symbol_mu);
    if (!g_symbol_ptr[device]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_factors);
        if (e != cudaSuccess) return e;
        g_symbol_ptr[device] = static_cast<double*>(ptr);
    }
    *out = g_symbol_ptr[device];
    return cudaSuccess;
}

}  // namespace
}  // namespace doctors

using namespace doctors;

extern "C" int doctors_dose_noalloc(doctors_problem* p, const double* k, double* dose) {
    if (!p) {
        set_error("null problem");
        return DOCTORS_ERR_INVALID_ARG;
    }
    if (!k || !dose) {
        set_error("null argument");
        return DOCTORS_ERR_INVALID_ARG;
    }
    if (p->have_mat && p->nmat * p->G > kNoAllocFactors) {
        set_error("doctors_dose_noalloc: n_mat * groups = " + std::to_string(p->nmat * p->G) +
                  " exceeds the fixed factor table of " + std::to_string(kNoAllocFactors) + " entries");
        return DOCTORS_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaSetDevice(p->device);
    if (e != cudaSuccess) {
        set_error(std::string("cudaSetDevice: ") + cudaGetErrorString(e));
        return DOCTORS_ERR_CUDA;
    }
    if (!p->solved) {
        set_error("no solution: call doctors_solve first");
        return DOCTORS_ERR_STATE;
    }
    const int n = p->nmat * p->G;
    for (int q = 0; q < n; ++q)
        if (!std::isfinite(k[q])) {
            set_error("k must be finite");
            return DOCTORS_ERR_INVALID_ARG;
        }
    double* table = nullptr;
    e = factor_table_address(p->device, &table);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(table, k, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess)
        e = launch_dose(p->V, p->G, p->M, p->d_mat, p->d_rho, table, p->d_phiu, p->d_mom, dose, p->stream);
    if (e != cudaSuccess) {
        set_error(std::string("doctors_dose_noalloc: ") + cudaGetErrorString(e));
        return DOCTORS_ERR_CUDA;
    }
    return DOCTORS_OK;
}
