// Step-differenced discrete-ordinates sweep (Eq. 2, vacuum boundaries) as
// diagonal wavefronts over the eight octants.
//
// For a direction Omega_n of octant o and group g, the step scheme sets the
// outgoing face fluxes of a cell equal to its cell-average angular fluence:
//   psi = (q_n + c_x psi_x + c_y psi_y + c_z psi_z) / (sigma_t + c_x + c_y + c_z),
//   c_q = |Omega_q| / d_q,  q_n = sum_lm (2l+1)/(4 pi) R_lm(Omega_n) s_lm,
// with psi_q the fluence of the upwind neighbour along q (0 outside the mesh).
// A cell depends only on its three upwind neighbours, so all cells on a
// hyperplane i' + j' + k' = h (indices reflected into the octant's sweep
// order) are independent.
//
// Decomposition (one launch per tile diagonal, all octants and groups in the
// launch):
//   * the mesh is cut into tiles of tx x ty columns spanning all of z; tiles
//     on one anti-diagonal of the octant's reflected tile grid form a stage;
//   * a CTA owns one (tile, group, octant, block of `ab` directions); thread
//     (li, lj) owns column (li, lj) of the tile and walks it in z;
//   * inside the CTA the hyperplane h = li + lj + k' advances one step per
//     __syncthreads(); the x/y upwind fluxes of the previous step come from a
//     double-buffered shared-memory plane, the z upwind flux stays in a
//     register, and the cell's source moments are prefetched one step ahead;
//   * fluxes leaving the tile through its downwind x/y faces go to global
//     face buffers; the next stage loads its incoming face strips into
//     shared memory once, before its first step;
//   * the group is the slowest grid dimension, so the CTAs resident at one
//     time work on few groups and their moment slabs stay in L2;
//   * each thread accumulates the moments sum_n w_n R_lm(Omega_n) psi_n of
//     its cell over its directions (Eq. 3 for lm = 00) and adds them to the
//     global moments with one vector atomic per 4 moments;
//   * outgoing current through the mesh boundary is accumulated in FP64 for
//     the balance check.
#pragma once

#include "doctors_internal.h"

namespace doctors {

// 1 / x by the hardware's approximate reciprocal (relative error about one
// unit in the last place; x here is a positive total cross section plus the
// step coefficients, far from the denormal and overflow ranges)
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <int M>
__device__ __forceinline__ void load_moments(const float* p, float (&s)[M]) {
    if constexpr (M % 4 == 0) {
        const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
        for (int q = 0; q < M / 4; ++q) {
            const float4 t = __ldg(p4 + q);
            s[4 * q] = t.x; s[4 * q + 1] = t.y; s[4 * q + 2] = t.z; s[4 * q + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < M; ++q) s[q] = __ldg(p + q);
    }
}

// The stored angular fluence of the stage, chained and tensor-core kernels
// (modes 1 and 2) is [G][V][A]: a voxel's directions are contiguous, so the
// thread that sweeps a cell writes, and later reads, one contiguous run of
// its block's directions (16-byte vectors when the block is a multiple of 4
// directions, which then also starts on a 16-byte boundary).
template <int AB>
__device__ __forceinline__ void psi_store_run(float* rec, const float (&psi)[AB]) {
    if constexpr (AB % 4 == 0) {
#pragma unroll
        for (int c4 = 0; c4 < AB / 4; ++c4)
            reinterpret_cast<float4*>(rec)[c4] = make_float4(psi[4 * c4], psi[4 * c4 + 1], psi[4 * c4 + 2], psi[4 * c4 + 3]);
    } else {
#pragma unroll
        for (int q = 0; q < AB; ++q) rec[q] = psi[q];
    }
}
// sum_q w_q psi_q stored_q over the run
template <int AB>
__device__ __forceinline__ float psi_product_run(const float* rec, const float (&wpsi)[AB]) {
    float pacc = 0.0f;
    if constexpr (AB % 4 == 0) {
#pragma unroll
        for (int c4 = 0; c4 < AB / 4; ++c4) {
            const float4 t4 = __ldg(reinterpret_cast<const float4*>(rec) + c4);
            pacc = fmaf(wpsi[4 * c4], t4.x, pacc);
            pacc = fmaf(wpsi[4 * c4 + 1], t4.y, pacc);
            pacc = fmaf(wpsi[4 * c4 + 2], t4.z, pacc);
            pacc = fmaf(wpsi[4 * c4 + 3], t4.w, pacc);
        }
    } else {
#pragma unroll
        for (int q = 0; q < AB; ++q) pacc = fmaf(wpsi[q], __ldg(rec + q), pacc);
    }
    return pacc;
}

// one float added with a reduction that returns nothing
__device__ __forceinline__ void red_add_f32(float* p, float x) {
    asm volatile("red.global.add.f32 [%0], %1;\n" ::"l"(p), "f"(x) : "memory");
}

// moments added with reductions that return nothing (red, not atom): the
// thread never waits for them
template <int M>
__device__ __forceinline__ void add_moments(float* p, const float (&a)[M]) {
    if constexpr (M % 4 == 0) {
#pragma unroll
        for (int q = 0; q < M / 4; ++q)
            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"l"(p + 4 * q), "f"(a[4 * q]),
                         "f"(a[4 * q + 1]), "f"(a[4 * q + 2]), "f"(a[4 * q + 3])
                         : "memory");
    } else {
#pragma unroll
        for (int q = 0; q < M; ++q) asm volatile("red.global.add.f32 [%0], %1;\n" ::"l"(p + q), "f"(a[q]) : "memory");
    }
}

// Direction tables shared by every problem: R_lm(Omega_n) (Schmidt real
// harmonics, 16 per direction, l <= 3) and w_n of every supported S_N set,
// concatenated (S2, S4, S6, S8, S12, S16: 616 directions).  They depend only
// on N, so they are uploaded once per device; each CTA copies the rows of its
// directions into shared memory (re-read after every barrier, so the compiler
// keeps them out of registers).
constexpr int kTableDirs = 616;
__constant__ float c_R[kTableDirs * 16];
__constant__ float c_w[kTableDirs];

// MODE 0: plain sweep.  MODE 1: also store every angular fluence psi[g][n][v]
// (forward fluence kept for the density gradient).  MODE 2: also accumulate
// prod[g][v] += sum_n w_n psi_n psi_store[g][n][v] (adjoint sweep against the
// stored forward fluence).
template <int AB, int M, int MODE>
__global__ void __launch_bounds__(256, 2) k_sweep(const SweepArgs a) {
    // float4 arrays first: the dynamic shared block is 16-byte aligned
    extern __shared__ float4 sm4[];
    const int T = a.tx * a.ty;
    float4* coef_s = sm4;                   // [AB]: cx, cy, cz, cx+cy+cz
    float4* R_s = coef_s + AB;              // [AB][4]: R_lm, 16 per direction
    float* buf = reinterpret_cast<float*>(R_s + 4 * AB);   // [2][AB][T] previous/current hyperplane
    float* xin = buf + 2 * AB * T;          // [AB][ty][nz]  incoming x-face strip
    float* yin = xin + AB * a.ty * a.nz;    // [AB][tx][nz]  incoming y-face strip
    float* w_s = yin + AB * a.tx * a.nz;    // [AB]
    float* sigt_s = w_s + AB;               // [nmat]

    if (a.skip && *a.skip) return;         // retired instance of a batched loop
    const int g = a.g0 + blockIdx.z;               // group slowest: resident CTAs share a few groups in L2
    const int o = blockIdx.y / a.nab;       // sweep octant
    const int blk = blockIdx.y % a.nab;
    const int a_lo = max(0, a.stage - (a.nty - 1));
    const int at = a_lo + blockIdx.x;       // reflected tile coordinates
    const int bt = a.stage - at;
    const int sx = (o & 1) ? -1 : 1, sy = (o & 2) ? -1 : 1, sz = (o & 4) ? -1 : 1;
    // the adjoint sweeps direction n along -Omega_n
    const int nbase = (a.reverse ? (o ^ 7) : o) * a.A8 + blk * AB;
    const int tb = a.table_base + nbase;    // row of direction nbase in the constant tables
    const int slot0 = blk * AB;             // direction slot within the octant (face buffers)
    const size_t xf_stride = (size_t)(a.ntx > 1 ? a.ntx - 1 : 0) * a.ny * a.nz;
    const size_t yf_stride = (size_t)(a.nty > 1 ? a.nty - 1 : 0) * a.nx * a.nz;

    for (int t = threadIdx.x; t < AB; t += blockDim.x) {
        const float* c = a.coef + (size_t)(nbase + t) * 8;
        coef_s[t] = make_float4(c[0], c[1], c[2], c[3]);
        w_s[t] = c_w[tb + t];
    }
    for (int t = threadIdx.x; t < 4 * AB; t += blockDim.x) {
        const float* r = c_R + (size_t)(tb + t / 4) * 16;
        const int p0 = 4 * (t % 4);
        R_s[t] = make_float4(r[lm_of_pos(p0, M)], r[lm_of_pos(p0 + 1, M)], r[lm_of_pos(p0 + 2, M)],
                             r[lm_of_pos(p0 + 3, M)]);
    }
    for (int t = threadIdx.x; t < a.nmat; t += blockDim.x) sigt_s[t] = a.sigt[t * a.G + g];
    // incoming face strips (contiguous in the face buffers), zero on the mesh boundary
    {
        const int nxs = AB * a.ty * a.nz;
        for (int t = threadIdx.x; t < nxs; t += blockDim.x) {
            const int q = t / (a.ty * a.nz), r = t % (a.ty * a.nz);
            const int jr = bt * a.ty + r / a.nz;
            float val = 0.0f;
            if (at > 0 && jr < a.ny) {
                const size_t fb = (((size_t)o * a.A8 + slot0 + q) * a.G + g) * xf_stride;
                val = a.xface[fb + (size_t)(at - 1) * a.ny * a.nz + (size_t)bt * a.ty * a.nz + r];
            }
            xin[t] = val;
        }
        const int nys = AB * a.tx * a.nz;
        for (int t = threadIdx.x; t < nys; t += blockDim.x) {
            const int q = t / (a.tx * a.nz), r = t % (a.tx * a.nz);
            const int ir = at * a.tx + r / a.nz;
            float val = 0.0f;
            if (bt > 0 && ir < a.nx) {
                const size_t fb = (((size_t)o * a.A8 + slot0 + q) * a.G + g) * yf_stride;
                val = a.yface[fb + (size_t)(bt - 1) * a.nx * a.nz + (size_t)at * a.tx * a.nz + r];
            }
            yin[t] = val;
        }
    }
    __syncthreads();

    const int tid = threadIdx.x;
    // threads own the tile's columns in diagonal order (li + lj ascending):
    // the columns active at a hyperplane step are then a contiguous range of
    // threads, so warps are either busy or skip the step entirely
    int li = 0, lj = 0;
    {
        int base = 0;
        for (int d = 0; d <= a.tx + a.ty - 2; ++d) {
            const int lo = d > a.ty - 1 ? d - (a.ty - 1) : 0;
            const int hi = d < a.tx - 1 ? d : a.tx - 1;
            const int cnt = hi - lo + 1;
            if (tid < base + cnt) {
                li = lo + (tid - base);
                lj = d - li;
                break;
            }
            base += cnt;
        }
    }
    const int col_id = lj * a.tx + li;          // column slot in the plane buffers
    const int ir = at * a.tx + li, jr = bt * a.ty + lj;
    const bool col = ir < a.nx && jr < a.ny;
    const int i = sx > 0 ? ir : a.nx - 1 - ir;
    const int j = sy > 0 ? jr : a.ny - 1 - jr;
    const size_t V = (size_t)a.nx * a.ny * a.nz;
    const size_t gV = (size_t)g * V;
    const size_t plane = (size_t)a.nx * a.ny;
    const size_t vcol = (size_t)j * a.nx + i;      // voxel index of k = 0 in this column
    const bool xout = li == a.tx - 1 && at < a.ntx - 1;
    const bool yout = lj == a.ty - 1 && bt < a.nty - 1;
    const bool xleak = ir == a.nx - 1, yleak = jr == a.ny - 1;
    float* xo = a.xface + (((size_t)o * a.A8 + slot0) * a.G + g) * xf_stride + ((size_t)at * a.ny + jr) * a.nz;
    float* yo = a.yface + (((size_t)o * a.A8 + slot0) * a.G + g) * yf_stride + ((size_t)bt * a.nx + ir) * a.nz;
    const size_t xo_q = (size_t)a.G * xf_stride, yo_q = (size_t)a.G * yf_stride;

    float zc[AB];
#pragma unroll
    for (int q = 0; q < AB; ++q) zc[q] = 0.0f;
    float lk = 0.0f;

    // software pipeline: the source moments and material of the next cell
    // are loaded one hyperplane step ahead
    float sn[M];
    float rho_n = 0.0f;       // density and material of the prefetched cell: the cross
    int mat_n = 0;            // section is looked up when the cell is swept, not at the load
    auto prefetch = [&](int kr) {
        if (col && kr >= 0 && kr < a.nz) {
            const int k = sz > 0 ? kr : a.nz - 1 - kr;
            const size_t v = (size_t)k * plane + vcol;
            load_moments<M>(a.src + (gV + v) * M, sn);
            rho_n = __ldg(a.rho + v);
            mat_n = __ldg(a.mat + v);
        }
    };
    prefetch(0);      // first cell of this column

    const int hmax = a.tx + a.ty + a.nz - 3;
    for (int h = 0; h <= hmax; ++h) {
        const int kr = h - li - lj;
        const int cb = h & 1, pb = cb ^ 1;
        const bool act = col && kr >= 0 && kr < a.nz;
        if (act) {
            float s[M];
            // (2l+1)/(4 pi) folded into the source moments
#pragma unroll
            for (int m = 0; m < M; ++m)
                s[m] = sn[m] * ((2 * degree_of_lm(lm_of_pos(m, M)) + 1) * 0.07957747154594767f);
            const float sig = rho_n * sigt_s[mat_n];
            prefetch(kr + 1);
            const int k = sz > 0 ? kr : a.nz - 1 - kr;
            const size_t v = (size_t)k * plane + vcol;
            // moments -> directions: AB independent dot products
            float psi[AB];
#pragma unroll
            for (int q = 0; q < AB; ++q) {
                float t0 = 0.0f, t1 = 0.0f, t2 = 0.0f, t3 = 0.0f;
#pragma unroll
                for (int m = 0; m < M; m += 4) {
                    const float4 R = R_s[4 * q + m / 4];
                    t0 = fmaf(R.x, s[m], t0);
                    if (m + 1 < M) t1 = fmaf(R.y, s[m + 1], t1);
                    if (m + 2 < M) t2 = fmaf(R.z, s[m + 2], t2);
                    if (m + 3 < M) t3 = fmaf(R.w, s[m + 3], t3);
                }
                psi[q] = (t0 + t1) + (t2 + t3);
            }
            // step-differenced cell solve per direction
#pragma unroll
            for (int q = 0; q < AB; ++q) {
                const float px = li > 0 ? buf[(pb * AB + q) * T + col_id - 1] : xin[(q * a.ty + lj) * a.nz + kr];
                const float py = lj > 0 ? buf[(pb * AB + q) * T + col_id - a.tx] : yin[(q * a.tx + li) * a.nz + kr];
                const float4 c = coef_s[q];
                const float num = fmaf(c.z, zc[q], fmaf(c.y, py, fmaf(c.x, px, psi[q])));
                psi[q] = __fdividef(num, sig + c.w);
                buf[(cb * AB + q) * T + col_id] = psi[q];
                zc[q] = psi[q];
            }
            if constexpr (MODE == 1) psi_store_run<AB>(a.psi + ((size_t)g * V + v) * a.A + nbase, psi);
            if constexpr (MODE == 2) {
                float wpsi[AB];
#pragma unroll
                for (int q = 0; q < AB; ++q) wpsi[q] = w_s[q] * psi[q];
                red_add_f32(a.prod + gV + v, psi_product_run<AB>(a.psi + ((size_t)g * V + v) * a.A + nbase, wpsi));
            }
            // faces leaving the tile and current leaving the mesh
            if (xout) {
#pragma unroll
                for (int q = 0; q < AB; ++q) xo[q * xo_q + kr] = psi[q];
            }
            if (yout) {
#pragma unroll
                for (int q = 0; q < AB; ++q) yo[q * yo_q + kr] = psi[q];
            }
            if (xleak || yleak || kr == a.nz - 1) {
#pragma unroll
                for (int q = 0; q < AB; ++q) {
                    const float* c = a.coef + (size_t)(nbase + q) * 8;
                    float f = 0.0f;
                    if (xleak) f += __ldg(c + 4);
                    if (yleak) f += __ldg(c + 5);
                    if (kr == a.nz - 1) f += __ldg(c + 6);
                    lk = fmaf(f, psi[q], lk);
                }
            }
            // directions -> moments (Eq. 3 for lm = 00)
            float acc[M];
#pragma unroll
            for (int m = 0; m < M; ++m) acc[m] = 0.0f;
#pragma unroll
            for (int q = 0; q < AB; ++q) {
                const float wp = w_s[q] * psi[q];
#pragma unroll
                for (int m = 0; m < M; m += 4) {
                    const float4 R = R_s[4 * q + m / 4];
                    acc[m] = fmaf(R.x, wp, acc[m]);
                    if (m + 1 < M) acc[m + 1] = fmaf(R.y, wp, acc[m + 1]);
                    if (m + 2 < M) acc[m + 2] = fmaf(R.z, wp, acc[m + 2]);
                    if (m + 3 < M) acc[m + 3] = fmaf(R.w, wp, acc[m + 3]);
                }
            }
            add_moments<M>(a.mom + (gV + v) * M, acc);
        }
        __syncthreads();
    }
    // boundary leakage of this CTA, reduced per full warp in FP64 (the last
    // warp of a block whose size is not a multiple of 32 adds lane by lane)
    double dl = (double)lk;
    if ((int)blockDim.x - (tid & ~31) >= 32) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) dl += __shfl_down_sync(0xffffffffu, dl, off);
        if ((tid & 31) == 0 && dl != 0.0) atomicAdd(a.leak + g, dl);
    } else if (dl != 0.0) {
        atomicAdd(a.leak + g, dl);
    }
}

inline size_t sweep_smem_bytes(int ab, int M, int tx, int ty, int nz, int nmat) {
    (void)M;
    return sizeof(float) * (size_t)(2 * ab * tx * ty + ab * (tx + ty) * nz + 4 * ab + 16 * ab + ab + nmat);
}

// upload the direction tables of this translation unit's constant bank
// (internal linkage, so that each unit's own copy is the one filled)
static cudaError_t upload_direction_tables(const float* R, const float* w) {
    cudaError_t e = cudaMemcpyToSymbol(c_R, R, sizeof(float) * kTableDirs * 16);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_w, w, sizeof(float) * kTableDirs);
    return e;
}

template <int M, int MODE>
cudaError_t launch_sweep_m(const SweepArgs& a, cudaStream_t s) {
    const int a_lo = a.stage - (a.nty - 1) > 0 ? a.stage - (a.nty - 1) : 0;
    const int a_hi = a.stage < a.ntx - 1 ? a.stage : a.ntx - 1;
    const int ntiles = a_hi - a_lo + 1;
    if (ntiles <= 0) return cudaSuccess;
    const int T = a.tx * a.ty;
    dim3 grid(ntiles, 8 * a.nab, a.gcount);
    const size_t smem = sweep_smem_bytes(a.ab, M, a.tx, a.ty, a.nz, a.nmat);
#define DOCTORS_SWEEP_CASE(AB)                                                                  \
    case AB: {                                                                                  \
        auto kern = k_sweep<AB, M, MODE>;                                                             \
        if (smem > 48 * 1024) {                                                                 \
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                                 (int)smem);                                    \
            if (e != cudaSuccess) return e;                                                     \
        }                                                                                       \
        kern<<<grid, T, smem, s>>>(a);                                                          \
        break;                                                                                  \
    }
    switch (a.ab) {
        DOCTORS_SWEEP_CASE(1)
        DOCTORS_SWEEP_CASE(2)
        DOCTORS_SWEEP_CASE(3)
        DOCTORS_SWEEP_CASE(4)
        DOCTORS_SWEEP_CASE(5)
        DOCTORS_SWEEP_CASE(6)
        DOCTORS_SWEEP_CASE(7)
        DOCTORS_SWEEP_CASE(9)
        DOCTORS_SWEEP_CASE(10)
        DOCTORS_SWEEP_CASE(12)
        default: return cudaErrorInvalidValue;
    }
#undef DOCTORS_SWEEP_CASE
    return cudaGetLastError();
}

}  // namespace doctors
