// Region-of-interest dose and the two ROI terms of its gradient, in FP64 on
// the device (Sec. II.A, III.A: the dose tally D(v) = rho(v) sum_g
// k[mat v][g] (phi_u + phi_c)[g](v), here summed with voxel weights roi(v)).
//
//   J          = sum_v roi(v) D(v)                       (k_roi_dose + k_sum_partials)
//   r[g][v]    = roi(v) k[mat v][g] rho(v)                (k_roi_response: dJ/dphi[g](v),
//                                                          the adjoint's source)
//   dJ/drho(v) at fixed fluence = roi(v) sum_g k[mat v][g] phi[g](v)
//                                                         (k_roi_explicit, added to the
//                                                          transport part of the gradient)
//
// J is summed in a fixed order (a fixed grid of per-block partial sums, then
// one block sums those in a fixed tree), so it is reproducible bit for bit.
#include <algorithm>

#include "doctors_internal.h"

namespace doctors {

namespace {

constexpr int kRoiThreads = 256;

__device__ __forceinline__ double voxel_dose(size_t V, int G, int M, int m, float rho, const double* k,
                                             const float* phi_u, const float* mom, size_t v) {
    double acc = 0.0;
    for (int g = 0; g < G; ++g) {
        const double phi = (double)phi_u[(size_t)g * V + v] + (double)mom[((size_t)g * V + v) * M];
        acc += k[m * G + g] * phi;
    }
    return acc * (double)rho;
}

// block sum of x into out (thread 0 writes)
__device__ __forceinline__ void block_sum(double x, double* out) {
    __shared__ double red[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        double y = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) y += __shfl_down_sync(0xffffffffu, y, off);
        if (threadIdx.x == 0) *out = y;
    }
}

__global__ void __launch_bounds__(kRoiThreads) k_roi_dose(size_t V, int G, int M, const uint8_t* mat,
                                                          const float* rho, const double* k, const double* roi,
                                                          const float* phi_u, const float* mom, double* dose,
                                                          double* partial) {
    double x = 0.0;
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (size_t)gridDim.x * blockDim.x) {
        const double d = voxel_dose(V, G, M, mat[v], rho[v], k, phi_u, mom, v);
        if (dose) dose[v] = d;
        x += roi[v] * d;
    }
    block_sum(x, partial + blockIdx.x);
}

// one block: out = sum of n partials, in a fixed order
__global__ void __launch_bounds__(kRoiThreads) k_sum_partials(const double* partial, int n, double* out) {
    double x = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) x += partial[q];
    block_sum(x, out);
}

__global__ void __launch_bounds__(kRoiThreads) k_roi_response(size_t V, int G, const uint8_t* mat, const float* rho,
                                                              const double* k, const double* roi, double* r,
                                                              float* rf) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= V * G) return;
    const size_t g = t / V, v = t - g * V;
    const double x = roi[v] * k[mat[v] * G + g] * (double)rho[v];
    r[t] = x;
    rf[t] = (float)x;
}

__global__ void __launch_bounds__(kRoiThreads) k_roi_explicit(size_t V, int G, int M, const uint8_t* mat,
                                                              const double* k, const double* roi,
                                                              const float* phi_u, const float* mom, double* grad) {
    const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    grad[v] += roi[v] * voxel_dose(V, G, M, mat[v], 1.0f, k, phi_u, mom, v);
}

unsigned blocks_of(size_t n) { return (unsigned)((n + kRoiThreads - 1) / kRoiThreads); }

}  // namespace

cudaError_t launch_roi_dose(size_t V, int G, int M, const uint8_t* mat, const float* rho, const double* k,
                            const double* roi, const float* phi_u, const float* mom, double* dose,
                            double* partial, double* J, cudaStream_t s) {
    const unsigned nb = (unsigned)std::min<size_t>(kRoiPartials, std::max<size_t>(1, blocks_of(V)));
    k_roi_dose<<<nb, kRoiThreads, 0, s>>>(V, G, M, mat, rho, k, roi, phi_u, mom, dose, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sum_partials<<<1, kRoiThreads, 0, s>>>(partial, (int)nb, J);
    return cudaGetLastError();
}

cudaError_t launch_roi_response(size_t V, int G, const uint8_t* mat, const float* rho, const double* k,
                                const double* roi, double* r, float* rf, cudaStream_t s) {
    k_roi_response<<<blocks_of(V * G), kRoiThreads, 0, s>>>(V, G, mat, rho, k, roi, r, rf);
    return cudaGetLastError();
}

cudaError_t launch_roi_explicit(size_t V, int G, int M, const uint8_t* mat, const double* k, const double* roi,
                                const float* phi_u, const float* mom, double* grad, cudaStream_t s) {
    k_roi_explicit<<<blocks_of(V), kRoiThreads, 0, s>>>(V, G, M, mat, k, roi, phi_u, mom, grad);
    return cudaGetLastError();
}

}  // namespace doctors
