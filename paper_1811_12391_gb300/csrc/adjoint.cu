// Gradient kernels of the discrete adjoint (the paper has no adjoint; these
// differentiate the forward operator of Eq. 2 with the first-collision
// source of Sec. II.A).  For J = sum_{g,v} r[g][v] phi[g][v]:
//   * the adjoint moments Z solve Z = D L^-T M (4 pi r delta_00 + S^T Z)
//     (the same sweep with directions reversed and scattering transposed);
//   * T = S^T Z gives dJ/dU = (2l+1)/(4 pi) T for the uncollided moments U,
//     so each point source's uncollided fluence has importance
//     imp = r + sum_lm (2l+1)/(4 pi) R_lm(Omega_source->v) T_lm;
//   * the density enters through sigma_t in the sweep (angular product of the
//     forward and adjoint fluences), sigma_s in the scattering source
//     (moments) and the attenuation of the uncollided rays (back-projection).
#include "doctors_internal.h"

namespace doctors {
namespace {

template <int M>
__device__ __forceinline__ void harmonics_scaled(float x, float y, float z, float (&R)[M]) {
    // Schmidt semi-normalised real harmonics times (2l+1)/(4 pi)
    const float c0 = 0.07957747154594767f, c1 = 3.0f * c0, c2 = 5.0f * c0, c3 = 7.0f * c0;
    R[0] = c0;
    if constexpr (M > 1) { R[1] = c1 * y; R[2] = c1 * z; R[3] = c1 * x; }
    if constexpr (M > 4) {
        const float s3 = 1.7320508075688772f;
        R[4] = c2 * s3 * x * y; R[5] = c2 * s3 * y * z; R[6] = c2 * 0.5f * (3.0f * z * z - 1.0f);
        R[7] = c2 * s3 * x * z; R[8] = c2 * 0.5f * s3 * (x * x - y * y);
    }
    if constexpr (M > 9) {
        const float ca = 0.7905694150420949f, cb = 3.872983346207417f, cc = 0.6123724356957945f;
        R[9] = c3 * ca * y * (3.0f * x * x - y * y); R[10] = c3 * cb * x * y * z;
        R[11] = c3 * cc * y * (5.0f * z * z - 1.0f); R[12] = c3 * 0.5f * z * (5.0f * z * z - 3.0f);
        R[13] = c3 * cc * x * (5.0f * z * z - 1.0f); R[14] = c3 * 0.5f * cb * z * (x * x - y * y);
        R[15] = c3 * ca * x * (x * x - 3.0f * y * y);
    }
}

// a voxel's M moments as 16-byte vector loads (records are 16-byte aligned when M % 4 == 0)
template <int M>
__device__ __forceinline__ void load_record(const float* p, float (&t)[M]) {
    if constexpr (M % 4 == 0) {
#pragma unroll
        for (int q = 0; q < M / 4; ++q) {
            const float4 v4 = __ldg(reinterpret_cast<const float4*>(p) + q);
            t[4 * q] = v4.x; t[4 * q + 1] = v4.y; t[4 * q + 2] = v4.z; t[4 * q + 3] = v4.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < M; ++q) t[q] = __ldg(p + q);
    }
}

template <int M>
__global__ void __launch_bounds__(256) k_source_grad(const SourceGradArgs a) {
    __shared__ double s_acc[kMaxG];
    for (int g = threadIdx.x; g < a.G; g += blockDim.x) s_acc[g] = 0.0;
    __syncthreads();
    const size_t V = (size_t)a.nx * a.ny * a.nz;
    const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = v < V;
    float R[M];
#pragma unroll
    for (int m = 0; m < M; ++m) R[m] = 0.0f;
    if (in) {
        const int i = (int)(v % a.nx);
        const int j = (int)((v / a.nx) % a.ny);
        const int k = (int)(v / ((size_t)a.nx * a.ny));
        float x = a.ox + (i + 0.5f) * a.dx - a.sx;
        float y = a.oy + (j + 0.5f) * a.dy - a.sy;
        float z = a.oz + (k + 0.5f) * a.dz - a.sz;
        const float rn = rsqrtf(x * x + y * y + z * z);
        harmonics_scaled<M>(x * rn, y * rn, z * rn, R);
    }
    float h[kMaxMat];
#pragma unroll
    for (int m = 0; m < kMaxMat; ++m) h[m] = 0.0f;
    // per group: this voxel's term, summed over the warp by shuffles and added
    // to the block's total by one shared-memory atomic per warp (every thread
    // of the block takes part in every shuffle)
    for (int g = 0; g < a.G; ++g) {
        double term = 0.0;
        const float u = in ? a.u[(size_t)g * V + v] : 0.0f;
        if (u != 0.0f) {
            float t[M];
            load_record<M>(a.T + ((size_t)g * V + v) * M, t);
            float imp = 0.0f;
#pragma unroll
            for (int pm = 0; pm < M; ++pm) imp = fmaf(R[lm_of_pos(pm, M)], t[pm], imp);
            const double impd = a.r[(size_t)g * V + v] + (double)imp;
            term = (double)u * impd;
            if (a.H) {
                const float w = (float)impd * __ldg(a.emit + g) * u;
#pragma unroll
                for (int m = 0; m < kMaxMat; ++m)
                    if (m < a.nmat) h[m] = fmaf(__ldg(a.sigt + m * a.G + g), w, h[m]);
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) term += __shfl_down_sync(0xffffffffu, term, off);
        if ((threadIdx.x & 31) == 0 && term != 0.0) atomicAdd(&s_acc[g], term);
    }
    if (in && a.H)
#pragma unroll
        for (int m = 0; m < kMaxMat; ++m)
            if (m < a.nmat) a.H[(size_t)m * V + v] = h[m];
    __syncthreads();
    for (int g = threadIdx.x; g < a.G; g += blockDim.x)
        if (s_acc[g] != 0.0) atomicAdd(a.acc + g, s_acc[g]);
}

// one thread per voxel
__global__ void __launch_bounds__(256) k_density_grad(const DensityGradArgs a) {
    const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.V) return;
    const int m = __ldg(a.mat + v);
    const size_t VM = a.V * a.M;
    double acc = 0.0;
    for (int g = 0; g < a.G; ++g) {
        for (int lm = 0; lm < a.M; ++lm) {
            const int l = degree_of_lm(lm_of_pos(lm, a.M));
            const float zc = a.Z[g * VM + v * a.M + lm] * (float)(2 * l + 1) * 0.07957747154594767f;
            if (zc == 0.0f) continue;
            const float* tab = a.sigs + ((size_t)m * (a.L + 1) + l) * a.G * a.G;
            float s = 0.0f;
            for (int gp = 0; gp <= g; ++gp) {
                const size_t idx = gp * VM + v * a.M + lm;
                s = fmaf(__ldg(tab + gp * a.G + g), a.phic[idx] + a.U[idx], s);
            }
            acc += (double)zc * (double)s;
        }
        if (a.prod) acc -= (double)__ldg(a.sigt + m * a.G + g) * (double)a.prod[(size_t)g * a.V + v];
    }
    a.grad[v] += acc;
}

// The same density gradient with the scattering term laid out like the
// scattering source: one (voxel, moment) entry per thread in a resident grid,
// coalesced loads of every group's X = phi_c + U and Z at the entry, the
// (material, degree) blocks of sigma_s staged in shared memory (odd block
// pitch), the triangular sum over source groups in registers, and the
// voxel's M entries summed by a shuffle within their M-lane segment (M = 1, 4
// or 16 divides the warp); the collision term is added by the voxel's first
// lane.  Per entry: (2l+1)/(4 pi) sum_g Z_g sum_{g' <= g} sigma_s,l(g' -> g) X_g'.
constexpr int kGradThreads = 256;
constexpr size_t kGradTableSmem = 100 * 1024;
template <int GMAX>
__host__ __device__ constexpr int grad_block_pitch() { return GMAX * GMAX + 1; }

template <int GMAX, int M>
__global__ void __launch_bounds__(kGradThreads, GMAX <= 24 ? 3 : 1) k_density_grad_fast(const DensityGradArgs a) {
    extern __shared__ float tab_s[];
    const int G = a.G;
    constexpr int BP = grad_block_pitch<GMAX>();
    const int nblk = a.nmat * (a.L + 1);
    for (int e = threadIdx.x; e < nblk * BP; e += blockDim.x) {
        const int blk = e / BP, r = e % BP, i = r / GMAX, j = r % GMAX;
        tab_s[e] = (r < GMAX * GMAX && i < G && j < G) ? __ldg(a.sigs + ((size_t)blk * G + i) * G + j) : 0.0f;
    }
    __syncthreads();
    const unsigned V = (unsigned)a.V, VM = (unsigned)(a.V * M);
    const unsigned stride = gridDim.x * blockDim.x;               // a multiple of 32
    const unsigned tend = (VM + 31u) & ~31u;                      // whole warps iterate together
    const int L1 = a.L + 1;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < tend; t += stride) {
        const bool ok = t < VM;
        const unsigned tt = ok ? t : 0u;
        const unsigned v = tt / M;
        const int lm = (int)(tt - v * M);
        const int l = degree_of_lm(lm_of_pos(lm, M));
        const int m = __ldg(a.mat + v);
        float x[GMAX], z[GMAX];
#pragma unroll
        for (int g = 0; g < GMAX; ++g) {
            const size_t o = (size_t)(g < G ? g : G - 1) * VM + tt;
            const float xp = __ldg(a.phic + o) + __ldg(a.U + o);
            const float zz = __ldg(a.Z + o);
            x[g] = g < G ? xp : 0.0f;
            z[g] = g < G ? zz : 0.0f;
        }
        const float* ts = tab_s + (m * L1 + l) * BP;
        float acc = 0.0f;
#pragma unroll
        for (int g = 0; g < GMAX; ++g) {
            float sg = 0.0f;
#pragma unroll
            for (int gp = 0; gp <= g; ++gp) sg = fmaf(ts[gp * GMAX + g], x[gp], sg);
            acc = fmaf(z[g], sg, acc);
        }
        double part = ok ? (double)(acc * (float)(2 * l + 1) * 0.07957747154594767f) : 0.0;
#pragma unroll
        for (int off = M / 2; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off, M);
        if (ok && lm == 0) {
            if (a.prod)
                for (int g = 0; g < G; ++g)
                    part -= (double)__ldg(a.sigt + m * G + g) * (double)a.prod[(size_t)g * V + v];
            a.grad[v] += part;
        }
    }
}

template <int GMAX, int M>
cudaError_t launch_density_grad_fast(const DensityGradArgs& a, size_t smem, cudaStream_t s) {
    auto kern = k_density_grad_fast<GMAX, M>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int nb = 0, dev = 0, nsm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kGradThreads, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    size_t want = (a.V * M + kGradThreads - 1) / kGradThreads, cap = (size_t)nsm * (nb > 0 ? nb : 1);
    kern<<<(unsigned)(want < cap ? want : cap), kGradThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int GMAX>
cudaError_t launch_density_grad_g(const DensityGradArgs& a, cudaStream_t s) {
    const size_t smem = (size_t)a.nmat * (a.L + 1) * grad_block_pitch<GMAX>() * sizeof(float);
    if (smem > kGradTableSmem || a.V * a.M >= ((size_t)1 << 31)) return cudaErrorNotSupported;
    switch (a.M) {
        case 1: return launch_density_grad_fast<GMAX, 1>(a, smem, s);
        case 4: return launch_density_grad_fast<GMAX, 4>(a, smem, s);
        case 16: return launch_density_grad_fast<GMAX, 16>(a, smem, s);
        default: return cudaErrorNotSupported;
    }
}

__global__ void __launch_bounds__(256) k_sum00(size_t V, int M, const float* mom, double* out) {
    const int g = blockIdx.y;
    double x = 0.0;
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (size_t)gridDim.x * blockDim.x)
        x += (double)mom[((size_t)g * V + v) * M];
    __shared__ double red[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        double y = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) y += __shfl_down_sync(0xffffffffu, y, off);
        if (threadIdx.x == 0 && y != 0.0) atomicAdd(out + g, y);
    }
}

__global__ void k_to_float(size_t n, const double* in, float* out) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = (float)in[t];
}

unsigned nblocks(size_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

cudaError_t launch_source_grad(const SourceGradArgs& a, cudaStream_t s) {
    const size_t V = (size_t)a.nx * a.ny * a.nz;
    switch (a.M) {
        case 1: k_source_grad<1><<<nblocks(V, 256), 256, 0, s>>>(a); break;
        case 4: k_source_grad<4><<<nblocks(V, 256), 256, 0, s>>>(a); break;
        case 9: k_source_grad<9><<<nblocks(V, 256), 256, 0, s>>>(a); break;
        case 16: k_source_grad<16><<<nblocks(V, 256), 256, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_density_grad(const DensityGradArgs& a, cudaStream_t s) {
    cudaError_t e = cudaErrorNotSupported;
    if (a.G <= 8) e = launch_density_grad_g<8>(a, s);
    else if (a.G <= 16) e = launch_density_grad_g<16>(a, s);
    else if (a.G <= 20) e = launch_density_grad_g<20>(a, s);
    else if (a.G <= 24) e = launch_density_grad_g<24>(a, s);
    if (e != cudaErrorNotSupported) return e;
    // M = 9, more groups or larger tables: the voxel-per-thread form
    k_density_grad<<<nblocks(a.V, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sum00(size_t V, int G, int M, const float* mom, double* out, cudaStream_t s) {
    size_t b = nblocks(V, 256);
    if (b > 296) b = 296;
    dim3 grid((unsigned)b, G);
    k_sum00<<<grid, 256, 0, s>>>(V, M, mom, out);
    return cudaGetLastError();
}

cudaError_t launch_to_float(size_t n, const double* in, float* out, cudaStream_t s) {
    k_to_float<<<nblocks(n, 256), 256, 0, s>>>(n, in, out);
    return cudaGetLastError();
}

}  // namespace doctors
