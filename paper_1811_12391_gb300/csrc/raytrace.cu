// Uncollided fluence by Siddon ray tracing (Sec. II.A: the uncollided
// photon transport equation has no scatter term, so its fluence is computed
// by ray tracing and then used to form the first-collision source).
//
// One thread per voxel centre T.  The ray from the source S to T is walked
// backward from T (parameter a = 1) toward S: at each step the next plane
// crossed is the one with the largest crossing parameter below the current
// one, with ties crossed in x, y, z order (zero-length segments dropped), and
// the walk stops when it leaves the mesh.  Plane p of axis q sits at
// o_q + p d_q and is crossed at a = (o_q + p d_q - S_q) / (T_q - S_q).  Every
// operation of the walk is an explicitly rounded FP32 operation (no FMA
// contraction), so the voxel index lists are reproducible bit for bit.
//
// Along the walk the density-weighted path length per material,
// Lambda_m = sum rho * length, is accumulated; then for every group
// tau_g = sum_m sigma_t[m][g] Lambda_m and
// phi_u[g] = weight * spectrum[g] * W * exp(-tau_g) / (4 pi r^2).
#include "doctors_internal.h"

namespace doctors {

namespace {

struct Walk {
    int cx, cy, cz;
    int stx, sty, stz;
    float ax, ay, az;       // next crossing parameter per axis
    float dirx, diry, dirz, norm, a;
};

__device__ __forceinline__ float plane_param(float o, int p, float d, float S, float dir) {
    return __fdiv_rn(__fsub_rn(__fadd_rn(o, __fmul_rn((float)p, d)), S), dir);
}

__device__ __forceinline__ void walk_init(const RayArgs& r, int i, int j, int k, Walk& w) {
    w.cx = i; w.cy = j; w.cz = k;
    const float tx = __fadd_rn(r.ox, __fmul_rn(__fadd_rn((float)i, 0.5f), r.dx));
    const float ty = __fadd_rn(r.oy, __fmul_rn(__fadd_rn((float)j, 0.5f), r.dy));
    const float tz = __fadd_rn(r.oz, __fmul_rn(__fadd_rn((float)k, 0.5f), r.dz));
    w.dirx = __fsub_rn(tx, r.sx);
    w.diry = __fsub_rn(ty, r.sy);
    w.dirz = __fsub_rn(tz, r.sz);
    w.norm = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(w.dirx, w.dirx), __fmul_rn(w.diry, w.diry)),
                                  __fmul_rn(w.dirz, w.dirz)));
    // axis x
    if (w.dirx > 0.0f) { w.stx = -1; w.ax = plane_param(r.ox, i, r.dx, r.sx, w.dirx); }
    else if (w.dirx < 0.0f) { w.stx = 1; w.ax = plane_param(r.ox, i + 1, r.dx, r.sx, w.dirx); }
    else { w.stx = 0; w.ax = -INFINITY; }
    if (w.diry > 0.0f) { w.sty = -1; w.ay = plane_param(r.oy, j, r.dy, r.sy, w.diry); }
    else if (w.diry < 0.0f) { w.sty = 1; w.ay = plane_param(r.oy, j + 1, r.dy, r.sy, w.diry); }
    else { w.sty = 0; w.ay = -INFINITY; }
    if (w.dirz > 0.0f) { w.stz = -1; w.az = plane_param(r.oz, k, r.dz, r.sz, w.dirz); }
    else if (w.dirz < 0.0f) { w.stz = 1; w.az = plane_param(r.oz, k + 1, r.dz, r.sz, w.dirz); }
    else { w.stz = 0; w.az = -INFINITY; }
    w.a = 1.0f;
}

// Walk the ray, calling emit(voxel, length) for every non-empty segment.
// The number of steps is bounded by the mesh size (each step leaves a voxel).
template <class F>
__device__ __forceinline__ void walk_ray(const RayArgs& r, int i, int j, int k, F&& emit) {
    Walk w;
    walk_init(r, i, j, k, w);
    const int max_steps = r.nx + r.ny + r.nz + 3;
    for (int it = 0; it < max_steps; ++it) {
        int q = 0;
        float an = w.ax;
        if (w.ay > an) { q = 1; an = w.ay; }
        if (w.az > an) { q = 2; an = w.az; }
        const float anext = an > 0.0f ? an : 0.0f;
        const float seg = __fsub_rn(w.a, anext);
        if (seg > 0.0f)
            emit((w.cz * r.ny + w.cy) * r.nx + w.cx, __fmul_rn(seg, w.norm));
        if (an <= 0.0f) break;
        w.a = anext;
        if (q == 0) {
            w.cx += w.stx;
            if (w.cx < 0 || w.cx >= r.nx) break;
            w.ax = plane_param(r.ox, w.stx < 0 ? w.cx : w.cx + 1, r.dx, r.sx, w.dirx);
        } else if (q == 1) {
            w.cy += w.sty;
            if (w.cy < 0 || w.cy >= r.ny) break;
            w.ay = plane_param(r.oy, w.sty < 0 ? w.cy : w.cy + 1, r.dy, r.sy, w.diry);
        } else {
            w.cz += w.stz;
            if (w.cz < 0 || w.cz >= r.nz) break;
            w.az = plane_param(r.oz, w.stz < 0 ? w.cz : w.cz + 1, r.dz, r.sz, w.dirz);
        }
    }
}

// Rectangular fan x cone collimator, decided in FP32 in a fixed order.
__device__ __forceinline__ bool lit(const RayArgs& r, float ux, float uy, float uz) {
    if (r.lit_all) return true;
    const float along = __fadd_rn(__fadd_rn(__fmul_rn(ux, r.ax), __fmul_rn(uy, r.ay)), __fmul_rn(uz, r.az));
    const float across = __fadd_rn(__fadd_rn(__fmul_rn(ux, r.px), __fmul_rn(uy, r.py)), __fmul_rn(uz, r.pz));
    const float vert = __fadd_rn(__fadd_rn(__fmul_rn(ux, r.ux), __fmul_rn(uy, r.uy)), __fmul_rn(uz, r.uz));
    return along > 0.0f && fabsf(across) <= __fmul_rn(r.tan_half, along) &&
           fabsf(vert) <= __fmul_rn(r.z_slope, along);
}

__global__ void __launch_bounds__(256) k_raytrace(const RayArgs r) {
    extern __shared__ float s_sigt[];   // [nmat][G]
    for (int t = threadIdx.x; t < r.nmat * r.G; t += blockDim.x) s_sigt[t] = r.sigt[t];
    __syncthreads();
    const size_t V = (size_t)r.nx * r.ny * r.nz;
    const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const int i = (int)(v % r.nx);
    const int j = (int)((v / r.nx) % r.ny);
    const int k = (int)(v / ((size_t)r.nx * r.ny));
    const float ux = __fsub_rn(__fadd_rn(r.ox, __fmul_rn(__fadd_rn((float)i, 0.5f), r.dx)), r.sx);
    const float uy = __fsub_rn(__fadd_rn(r.oy, __fmul_rn(__fadd_rn((float)j, 0.5f), r.dy)), r.sy);
    const float uz = __fsub_rn(__fadd_rn(r.oz, __fmul_rn(__fadd_rn((float)k, 0.5f), r.dz)), r.sz);
    if (!lit(r, ux, uy, uz)) {
        for (int g = 0; g < r.G; ++g) r.phi_src[(size_t)g * V + v] = 0.0f;
        return;
    }
    float lam[kMaxMat];
#pragma unroll
    for (int m = 0; m < kMaxMat; ++m) lam[m] = 0.0f;
    walk_ray(r, i, j, k, [&](int u, float len) {
        const int mu = __ldg(r.mat + u);
        const float pl = __ldg(r.rho + u) * len;
#pragma unroll
        for (int m = 0; m < kMaxMat; ++m) lam[m] += (mu == m) ? pl : 0.0f;
    });
    const float r2 = ux * ux + uy * uy + uz * uz;
    const float inv = 1.0f / (4.0f * 3.14159265358979f * r2);
    for (int g = 0; g < r.G; ++g) {
        float tau = 0.0f;
#pragma unroll
        for (int m = 0; m < kMaxMat; ++m)
            if (m < r.nmat) tau = fmaf(s_sigt[m * r.G + g], lam[m], tau);
        const float phi = __ldg(r.emit + g) * expf(-tau) * inv;
        r.phi_src[(size_t)g * V + v] = phi;
        if (r.phi_tot) r.phi_tot[(size_t)g * V + v] += phi;
    }
}

// Density gradient of the uncollided fluence, back-projected along the rays:
// d phi_u[g](t) / d rho_u = -sigma_t[mat u][g] * length(u on ray t) * phi_u[g](t),
// so grad[u] -= length * H[mat u][t] with H[m][t] = sum_g sigma_t[m][g] *
// dJ/dphi_u[g](t) * phi_u[g](t).  One thread per target voxel t; FP64 atomics.
__global__ void __launch_bounds__(256) k_backproject(const RayArgs r, const float* H, double* grad) {
    const size_t V = (size_t)r.nx * r.ny * r.nz;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= V) return;
    float h[kMaxMat];
    bool any = false;
#pragma unroll
    for (int m = 0; m < kMaxMat; ++m) {
        h[m] = m < r.nmat ? H[(size_t)m * V + t] : 0.0f;
        any |= h[m] != 0.0f;
    }
    if (!any) return;
    const int i = (int)(t % r.nx);
    const int j = (int)((t / r.nx) % r.ny);
    const int k = (int)(t / ((size_t)r.nx * r.ny));
    walk_ray(r, i, j, k, [&](int u, float len) {
        const int mu = __ldg(r.mat + u);
        float hm = 0.0f;
#pragma unroll
        for (int m = 0; m < kMaxMat; ++m) hm = (mu == m) ? h[m] : hm;
        if (hm != 0.0f) atomicAdd(grad + u, -(double)len * (double)hm);
    });
}

__global__ void k_debug_ray(const RayArgs r, int voxel, int32_t* idx, float* len, int cap, int* count) {
    const int i = voxel % r.nx;
    const int j = (voxel / r.nx) % r.ny;
    const int k = voxel / (r.nx * r.ny);
    int n = 0;
    walk_ray(r, i, j, k, [&](int u, float l) {
        if (n < cap) { idx[n] = u; len[n] = l; }
        ++n;
    });
    *count = n;
}

// Uncollided angular fluence is a delta in the direction source -> voxel, so
// its moments are phi_u * R_lm(that direction) (first-collision source).  One
// thread per voxel; a voxel's moments of a group are one record of M floats,
// written as 16-byte vectors when M is a multiple of 4 (the first source
// stores, later sources of a superposed scan add).  HBM-bound: the record is
// written (and, when adding, read) once per group.
template <int M, bool ACC>
__global__ void __launch_bounds__(256) k_uncollided_moments(const MomentArgs a) {
    const size_t V = (size_t)a.nx * a.ny * a.nz;
    const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const int i = (int)(v % a.nx);
    const int j = (int)((v / a.nx) % a.ny);
    const int k = (int)(v / ((size_t)a.nx * a.ny));
    float x = a.ox + (i + 0.5f) * a.dx - a.sx;
    float y = a.oy + (j + 0.5f) * a.dy - a.sy;
    float z = a.oz + (k + 0.5f) * a.dz - a.sz;
    const float rn = rsqrtf(x * x + y * y + z * z);
    x *= rn; y *= rn; z *= rn;
    float R[16];
    R[0] = 1.0f;
    if (M > 1) { R[1] = y; R[2] = z; R[3] = x; }
    if (M > 4) {
        const float s3 = 1.7320508075688772f;
        R[4] = s3 * x * y; R[5] = s3 * y * z; R[6] = 0.5f * (3.0f * z * z - 1.0f);
        R[7] = s3 * x * z; R[8] = 0.5f * s3 * (x * x - y * y);
    }
    if (M > 9) {
        const float ca = 0.7905694150420949f, cb = 3.872983346207417f, cc = 0.6123724356957945f;
        R[9] = ca * y * (3.0f * x * x - y * y); R[10] = cb * x * y * z;
        R[11] = cc * y * (5.0f * z * z - 1.0f); R[12] = 0.5f * z * (5.0f * z * z - 3.0f);
        R[13] = cc * x * (5.0f * z * z - 1.0f); R[14] = 0.5f * cb * z * (x * x - y * y);
        R[15] = ca * x * (x * x - 3.0f * y * y);
    }
    for (int g = 0; g < a.G; ++g) {
        const float p = a.phi_src[(size_t)g * V + v];
        float* u = a.U + ((size_t)g * V + v) * M;
        if constexpr (M % 4 == 0) {
            float4* u4 = reinterpret_cast<float4*>(u);
#pragma unroll
            for (int c = 0; c < M / 4; ++c) {
                float4 w = make_float4(p * R[lm_of_pos(4 * c, M)], p * R[lm_of_pos(4 * c + 1, M)],
                                       p * R[lm_of_pos(4 * c + 2, M)], p * R[lm_of_pos(4 * c + 3, M)]);
                if (ACC) {
                    const float4 o = u4[c];
                    w.x += o.x; w.y += o.y; w.z += o.z; w.w += o.w;
                }
                u4[c] = w;
            }
        } else {
#pragma unroll
            for (int m = 0; m < M; ++m) u[m] = ACC ? u[m] + p * R[lm_of_pos(m, M)] : p * R[lm_of_pos(m, M)];
        }
    }
}

}  // namespace

cudaError_t launch_raytrace(const RayArgs& a, cudaStream_t s) {
    const size_t V = (size_t)a.nx * a.ny * a.nz;
    const int bs = 256;
    const unsigned grid = (unsigned)((V + bs - 1) / bs);
    k_raytrace<<<grid, bs, sizeof(float) * a.nmat * a.G, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_backproject(const RayArgs& a, const float* H, double* grad, cudaStream_t s) {
    const size_t V = (size_t)a.nx * a.ny * a.nz;
    const int bs = 256;
    k_backproject<<<(unsigned)((V + bs - 1) / bs), bs, 0, s>>>(a, H, grad);
    return cudaGetLastError();
}

cudaError_t launch_debug_ray(const RayArgs& a, int voxel, int32_t* idx, float* len, int cap, int* count,
                             cudaStream_t s) {
    k_debug_ray<<<1, 1, 0, s>>>(a, voxel, idx, len, cap, count);
    return cudaGetLastError();
}

cudaError_t launch_uncollided_moments(const MomentArgs& a, cudaStream_t s) {
    const size_t V = (size_t)a.nx * a.ny * a.nz;
    const int bs = 256;
    const unsigned grid = (unsigned)((V + bs - 1) / bs);
    const bool acc = a.accumulate != 0;
    switch (a.M) {
        case 1: acc ? k_uncollided_moments<1, true><<<grid, bs, 0, s>>>(a) : k_uncollided_moments<1, false><<<grid, bs, 0, s>>>(a); break;
        case 4: acc ? k_uncollided_moments<4, true><<<grid, bs, 0, s>>>(a) : k_uncollided_moments<4, false><<<grid, bs, 0, s>>>(a); break;
        case 9: acc ? k_uncollided_moments<9, true><<<grid, bs, 0, s>>>(a) : k_uncollided_moments<9, false><<<grid, bs, 0, s>>>(a); break;
        case 16: acc ? k_uncollided_moments<16, true><<<grid, bs, 0, s>>>(a) : k_uncollided_moments<16, false><<<grid, bs, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace doctors
