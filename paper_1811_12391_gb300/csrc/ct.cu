// CT numbers -> materials and densities (Sec. II.B: the geometry input is a
// reconstructed CT image whose numbers are converted to dosimetrically
// equivalent materials through a calibration; the paper cites a
// stoichiometric calibration and does not print it).  Any piecewise
// calibration of that form is applied here: a material per CT-number bin
// between ascending thresholds, and a density piecewise linear in the CT
// number through ascending knots, constant beyond the end knots.
//
// One thread per voxel (grid-stride over a resident grid); the calibration
// is a kernel parameter, read through the constant bank.  The density is
// formed with explicitly rounded FP32 operations in a fixed order, so a
// plain FP32 evaluation of the same steps gives the same bits.  HBM-bound:
// 4 bytes read and 5 written per voxel.
#include <cmath>
#include <string>

#include "doctors_internal.h"

namespace doctors {
namespace {

constexpr int kCtMaxThresholds = 31;   // at most 32 bins
constexpr int kCtMaxKnots = 32;

struct CtCalib {
    int nt, nk;
    float t[kCtMaxThresholds];          // bin thresholds, ascending
    unsigned char m[kCtMaxThresholds + 1];   // material of each bin
    float hk[kCtMaxKnots], rk[kCtMaxKnots];  // density knots (CT number, density)
};

__global__ void __launch_bounds__(256) k_ct_to_materials(const float* __restrict__ hu, size_t n, const CtCalib c,
                                                         uint8_t* __restrict__ mat, float* __restrict__ rho) {
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x) {
        const float h = hu[v];
        // bin: the number of thresholds at or below h (NaN: bin 0)
        int b = 0;
        for (int i = 0; i < c.nt; ++i) b += c.t[i] <= h ? 1 : 0;
        // density: the number of knots at or below h picks the segment
        int k = 0;
        for (int i = 0; i < c.nk; ++i) k += c.hk[i] <= h ? 1 : 0;
        float r;
        if (k == 0) {
            r = c.rk[0];                       // below the first knot, or NaN
        } else if (k == c.nk) {
            r = c.rk[c.nk - 1];                // at or beyond the last knot
        } else {
            const int s = k - 1;               // hk[s] <= h < hk[s + 1]
            const float t = __fdiv_rn(__fsub_rn(h, c.hk[s]), __fsub_rn(c.hk[s + 1], c.hk[s]));
            r = __fadd_rn(c.rk[s], __fmul_rn(t, __fsub_rn(c.rk[s + 1], c.rk[s])));
        }
        mat[v] = c.m[b];
        rho[v] = r;
    }
}

int fail(int code, const std::string& msg) {
    set_error(msg);
    return code;
}

}  // namespace
}  // namespace doctors

using namespace doctors;

extern "C" int doctors_ct_to_materials(const float* hu, size_t n, int n_thresholds, const float* thresholds,
                                       const uint8_t* bin_material, int n_knots, const float* hu_knots,
                                       const float* rho_knots, uint8_t* mat_out, float* rho_out, int mem,
                                       void* cuda_stream) {
    if (mem != DOCTORS_MEM_HOST && mem != DOCTORS_MEM_DEVICE) return fail(DOCTORS_ERR_INVALID_ARG, "bad mem");
    if (n_thresholds < 0 || n_thresholds > kCtMaxThresholds)
        return fail(DOCTORS_ERR_INVALID_ARG, "n_thresholds must be 0..31");
    if (n_knots < 1 || n_knots > kCtMaxKnots) return fail(DOCTORS_ERR_INVALID_ARG, "n_knots must be 1..32");
    if ((n_thresholds > 0 && !thresholds) || !bin_material || !hu_knots || !rho_knots)
        return fail(DOCTORS_ERR_INVALID_ARG, "null calibration table");
    if (n > 0 && (!hu || !mat_out || !rho_out)) return fail(DOCTORS_ERR_INVALID_ARG, "null voxel array");
    CtCalib c{};
    c.nt = n_thresholds;
    c.nk = n_knots;
    for (int i = 0; i < n_thresholds; ++i) {
        if (!std::isfinite(thresholds[i])) return fail(DOCTORS_ERR_INVALID_ARG, "thresholds must be finite");
        if (i > 0 && !(thresholds[i] > thresholds[i - 1]))
            return fail(DOCTORS_ERR_INVALID_ARG, "thresholds must be strictly ascending");
        c.t[i] = thresholds[i];
    }
    for (int i = 0; i <= n_thresholds; ++i) c.m[i] = bin_material[i];
    for (int i = 0; i < n_knots; ++i) {
        if (!std::isfinite(hu_knots[i]) || !std::isfinite(rho_knots[i]) || rho_knots[i] < 0.0f)
            return fail(DOCTORS_ERR_INVALID_ARG, "knots must be finite with densities >= 0");
        if (i > 0 && !(hu_knots[i] > hu_knots[i - 1]))
            return fail(DOCTORS_ERR_INVALID_ARG, "knot CT numbers must be strictly ascending");
        c.hk[i] = hu_knots[i];
        c.rk[i] = rho_knots[i];
    }
    if (n == 0) return DOCTORS_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(DOCTORS_ERR_CUDA, std::string("doctors_ct_to_materials: ") + cudaGetErrorString(e));
    const size_t want = (n + 255) / 256, cap = (size_t)nsm * 8;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    if (mem == DOCTORS_MEM_DEVICE) {
        k_ct_to_materials<<<grid, 256, 0, s>>>(hu, n, c, mat_out, rho_out);
        e = cudaGetLastError();
        if (e != cudaSuccess)
            return fail(DOCTORS_ERR_CUDA, std::string("doctors_ct_to_materials: ") + cudaGetErrorString(e));
        return DOCTORS_OK;
    }
    // host arrays: staged through device buffers, synchronises
    float* d_hu = nullptr;
    float* d_rho = nullptr;
    uint8_t* d_mat = nullptr;
    e = cudaMalloc(&d_hu, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&d_rho, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&d_mat, n);
    if (e != cudaSuccess) {
        cudaFree(d_hu);
        cudaFree(d_rho);
        cudaFree(d_mat);
        cudaGetLastError();
        return fail(DOCTORS_ERR_OOM, "doctors_ct_to_materials: device buffers");
    }
    e = cudaMemcpyAsync(d_hu, hu, n * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_ct_to_materials<<<grid, 256, 0, s>>>(d_hu, n, c, d_mat, d_rho);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(mat_out, d_mat, n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rho_out, d_rho, n * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_hu);
    cudaFree(d_rho);
    cudaFree(d_mat);
    if (e != cudaSuccess) return fail(DOCTORS_ERR_CUDA, std::string("doctors_ct_to_materials: ") + cudaGetErrorString(e));
    return DOCTORS_OK;
}
