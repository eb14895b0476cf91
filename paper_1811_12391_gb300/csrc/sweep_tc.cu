// Step-differenced octant wavefront sweep for P3 (16 flux moments) with the
// moment <-> direction transforms on the tensor pipe.
//
// Same decomposition as sweep_impl.cuh (tiles of columns spanning z, one CTA
// per tile x group x octant x block of up to 16 directions, one hyperplane
// step per __syncthreads), but the work of a warp at a step is expressed as
// two small matrix products over its 32 cells:
//
//   Q[cell][n]   = sum_lm S[cell][lm] * (2l+1)/(4 pi) R_lm(Omega_n)     (Eq. 2's Legendre source)
//   Phi[cell][lm] += sum_n Psi[cell][n] * w_n R_lm(Omega_n)             (Eq. 3 moments)
//
// each as mma.sync m16n8k8 TF32 with the three-term split
// a*b ~ a_hi*b_hi + a_hi*b_lo + a_lo*b_hi (a_hi = tf32(a), a_lo = tf32(a - a_hi)),
// which keeps FP32-level accuracy with FP32 accumulation.
//
// Fragment layout (PTX m16n8k8, tf32; g = lane / 4, t = lane % 4):
//   A (16x8):  a0 = A[g][t]  a1 = A[g+8][t]  a2 = A[g][t+4]  a3 = A[g+8][t+4]
//   B (8x8):   b0 = B[t][g]  b1 = B[t+4][g]
//   C (16x8):  c0 = C[g][2t] c1 = C[g][2t+1] c2 = C[g+8][2t] c3 = C[g+8][2t+1]
// Rows are cells: lane (g, t) owns the fragment rows of cells g, g+8, 16+g,
// 24+g of its warp.  With the moment record stored in the transposed order
// of lm_of_pos(), a lane's A-fragment entries of one cell are one float4
// (positions 4t..4t+3), and so are its accumulator entries after the second
// product.  The step solve runs directly on the C fragment of the first
// product (cells x direction slots 2t, 2t+1, 8+2t, 9+2t), and that fragment
// is reused as the A operand of the second product by ordering the summed
// direction index as (2t, 2t+1) <-> (t, t+4).
#include <cstdint>

#include "doctors_internal.h"

namespace doctors {

constexpr int kTcDirs = 616;
__constant__ float tc_R[kTcDirs * 16];   // R_lm(Omega_n), (l, m) order, all S_N sets
__constant__ float tc_w[kTcDirs];        // w_n

namespace {

constexpr int kSlots = 16;               // direction slots per CTA (padded)
constexpr float kInv4Pi = 0.07957747154594767f;

__device__ __forceinline__ uint32_t tf32_of(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    hi = tf32_of(x);
    lo = tf32_of(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// d += a * b with the three-term TF32 split (a and b pre-split; b = {b0hi, b1hi, b0lo, b1lo})
__device__ __forceinline__ void mma_3xtf32(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                           const float4 b) {
    const uint32_t b0h = __float_as_uint(b.x), b1h = __float_as_uint(b.y);
    const uint32_t b0l = __float_as_uint(b.z), b1l = __float_as_uint(b.w);
    mma_tf32(d, al, b0h, b1h);
    mma_tf32(d, ah, b0l, b1l);
    mma_tf32(d, ah, b0h, b1h);
}

__device__ __forceinline__ float4 split_pair(float b0, float b1) {
    uint32_t h0, l0, h1, l1;
    split_tf32(b0, h0, l0);
    split_tf32(b1, h1, l1);
    return make_float4(__uint_as_float(h0), __uint_as_float(h1), __uint_as_float(l0), __uint_as_float(l1));
}

// MODE 0: plain; 1: store psi[g][n][v]; 2: prod[g][v] += sum_n w_n psi_n psi_stored_n
template <int MODE>
__global__ void __launch_bounds__(256, 2) k_sweep_tc(const SweepArgs a) {
    extern __shared__ float4 sm4[];
    const int T = a.tx * a.ty;
    const int SA = T + 4;                   // slot stride of the plane buffers (bank-conflict free)
    const int AB = a.ab;
    float4* tabM = sm4;                     // [2 kt][2 nt][32 lanes]  moments -> directions
    float4* tabD = tabM + 128;              // [2 kt][2 nt][32 lanes]  directions -> moments
    float4* coefs = tabD + 128;             // [16 slots]: cx, cy, cz, cx+cy+cz
    float4* leakc = coefs + kSlots;         // [16 slots]: leak_x, leak_y, leak_z, w
    float* buf = reinterpret_cast<float*>(leakc + kSlots);   // [2][16][SA]
    float* xin = buf + 2 * kSlots * SA;     // [AB][ty][nz]
    float* yin = xin + AB * a.ty * a.nz;    // [AB][tx][nz]
    float* sigt_s = yin + AB * a.tx * a.nz; // [nmat]

    if (a.skip && *a.skip) return;         // retired instance of a batched loop
    const int g = blockIdx.z;
    const int o = blockIdx.y / a.nab;
    const int blk = blockIdx.y % a.nab;
    const int a_lo = max(0, a.stage - (a.nty - 1));
    const int at = a_lo + blockIdx.x;
    const int bt = a.stage - at;
    const int sx = (o & 1) ? -1 : 1, sy = (o & 2) ? -1 : 1, sz = (o & 4) ? -1 : 1;
    const int nbase = (a.reverse ? (o ^ 7) : o) * a.A8 + blk * AB;
    const int tb = a.table_base + nbase;
    const int slot0 = blk * AB;
    const size_t xf_stride = (size_t)(a.ntx > 1 ? a.ntx - 1 : 0) * a.ny * a.nz;
    const size_t yf_stride = (size_t)(a.nty > 1 ? a.nty - 1 : 0) * a.nx * a.nz;

    // ---- tables in fragment order -------------------------------------------------
    for (int idx = threadIdx.x; idx < 128; idx += blockDim.x) {
        const int kt = idx >> 6, nt = (idx >> 5) & 1, ln = idx & 31;
        const int gq = ln >> 2, tq = ln & 3;
        // moments -> directions: B[k = lm][n = slot] = (2l+1)/(4 pi) R_lm(Omega_slot)
        {
            const int n = 8 * nt + gq;
            const int k0 = 8 * kt + tq, k1 = k0 + 4;
            float b0 = 0.0f, b1 = 0.0f;
            if (n < AB) {
                b0 = (2 * degree_of_lm(k0) + 1) * kInv4Pi * tc_R[(tb + n) * 16 + k0];
                b1 = (2 * degree_of_lm(k1) + 1) * kInv4Pi * tc_R[(tb + n) * 16 + k1];
            }
            tabM[idx] = split_pair(b0, b1);
        }
        // directions -> moments: B'[k' = (slot 8kt+2t, 8kt+2t+1) <-> (t, t+4)][n' = output column]
        {
            const int col = gq;                              // column within the n' tile
            const int lm = col / 2 + 4 * ((col & 1) + 2 * nt);
            const int s0 = 8 * kt + 2 * tq, s1 = s0 + 1;
            const float b0 = s0 < AB ? tc_w[tb + s0] * tc_R[(tb + s0) * 16 + lm] : 0.0f;
            const float b1 = s1 < AB ? tc_w[tb + s1] * tc_R[(tb + s1) * 16 + lm] : 0.0f;
            tabD[idx] = split_pair(b0, b1);
        }
    }
    for (int t = threadIdx.x; t < kSlots; t += blockDim.x) {
        if (t < AB) {
            const float* c = a.coef + (size_t)(nbase + t) * 8;
            coefs[t] = make_float4(c[0], c[1], c[2], c[3]);
            leakc[t] = make_float4(c[4], c[5], c[6], c[7]);
        } else {   // padded slot: psi = 0 whatever the cell
            coefs[t] = make_float4(0.0f, 0.0f, 0.0f, 1.0f);
            leakc[t] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
    }
    for (int t = threadIdx.x; t < a.nmat; t += blockDim.x) sigt_s[t] = a.sigt[t * a.G + g];
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

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gq = lane >> 2, tq = lane & 3;
    const size_t V = (size_t)a.nx * a.ny * a.nz;
    const size_t gV = (size_t)g * V;
    const size_t plane = (size_t)a.nx * a.ny;

    // the four cells (fragment rows gq, gq+8, 16+gq, 24+gq) of this lane
    int cc[4], li[4], lj[4], ir[4], jr[4];
    size_t vcol[4];
    bool colok[4];
#pragma unroll
    for (int ci = 0; ci < 4; ++ci) {
        cc[ci] = 32 * warp + gq + 8 * ci;
        li[ci] = cc[ci] % a.tx;
        lj[ci] = cc[ci] / a.tx;
        ir[ci] = at * a.tx + li[ci];
        jr[ci] = bt * a.ty + lj[ci];
        colok[ci] = ir[ci] < a.nx && jr[ci] < a.ny;
        const int i = sx > 0 ? ir[ci] : a.nx - 1 - ir[ci];
        const int j = sy > 0 ? jr[ci] : a.ny - 1 - jr[ci];
        vcol[ci] = colok[ci] ? (size_t)j * a.nx + i : 0;
    }
    // direction slot of fragment entry (nt, e): 8 nt + 2 tq + (e & 1); zc index si = 2 nt + (e & 1)
    float zc[4][4];
#pragma unroll
    for (int ci = 0; ci < 4; ++ci)
#pragma unroll
        for (int si = 0; si < 4; ++si) zc[ci][si] = 0.0f;
    float lk = 0.0f;

    const int hmax = a.tx + a.ty + a.nz - 3;
    for (int h = 0; h <= hmax; ++h) {
        const int cb = h & 1, pb = cb ^ 1;
        int kr[4];
        bool act[4];
        size_t v[4];
        float4 sv[4];
        float sig[4];
#pragma unroll
        for (int ci = 0; ci < 4; ++ci) {
            kr[ci] = h - li[ci] - lj[ci];
            act[ci] = colok[ci] && kr[ci] >= 0 && kr[ci] < a.nz;
            const int k = sz > 0 ? kr[ci] : a.nz - 1 - kr[ci];
            v[ci] = act[ci] ? (size_t)k * plane + vcol[ci] : 0;
            sv[ci] = act[ci] ? __ldg(reinterpret_cast<const float4*>(a.src + (gV + v[ci]) * 16) + tq)
                             : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            sig[ci] = act[ci] ? __ldg(a.rho + v[ci]) * sigt_s[__ldg(a.mat + v[ci])] : 1.0f;
        }
        // ---- moments -> directions ----------------------------------------------
        float q[2][2][4];
#pragma unroll
        for (int rt = 0; rt < 2; ++rt)
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) q[rt][nt][e] = 0.0f;
#pragma unroll
        for (int rt = 0; rt < 2; ++rt) {
            const float4 s0 = sv[2 * rt], s1 = sv[2 * rt + 1];
#pragma unroll
            for (int kt = 0; kt < 2; ++kt) {
                float af[4];
                af[0] = kt == 0 ? s0.x : s0.z;
                af[1] = kt == 0 ? s1.x : s1.z;
                af[2] = kt == 0 ? s0.y : s0.w;
                af[3] = kt == 0 ? s1.y : s1.w;
                uint32_t ah[4], al[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) split_tf32(af[e], ah[e], al[e]);
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) mma_3xtf32(q[rt][nt], ah, al, tabM[(kt * 2 + nt) * 32 + lane]);
            }
        }
        // ---- step-differenced cell solve on the fragment --------------------------
#pragma unroll
        for (int rt = 0; rt < 2; ++rt)
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int ci = 2 * rt + (e >> 1);
                    const int slot = 8 * nt + 2 * tq + (e & 1);
                    const int si = 2 * nt + (e & 1);
                    float psi = 0.0f;
                    if (act[ci]) {
                        const float px = li[ci] > 0 ? buf[(pb * kSlots + slot) * SA + cc[ci] - 1]
                                         : (slot < AB ? xin[(slot * a.ty + lj[ci]) * a.nz + kr[ci]] : 0.0f);
                        const float py = lj[ci] > 0 ? buf[(pb * kSlots + slot) * SA + cc[ci] - a.tx]
                                         : (slot < AB ? yin[(slot * a.tx + li[ci]) * a.nz + kr[ci]] : 0.0f);
                        const float4 cf = coefs[slot];
                        const float num = fmaf(cf.z, zc[ci][si], fmaf(cf.y, py, fmaf(cf.x, px, q[rt][nt][e])));
                        psi = __fdividef(num, sig[ci] + cf.w);
                    }
                    buf[(cb * kSlots + slot) * SA + cc[ci]] = psi;
                    zc[ci][si] = psi;
                    q[rt][nt][e] = psi;
                }
        // faces leaving the tile, current leaving the mesh, stored fluence: only
        // cells on a tile or mesh boundary (or in store mode) take this path
        {
            bool bnd[4];
            bool anyb = false;
#pragma unroll
            for (int ci = 0; ci < 4; ++ci) {
                bnd[ci] = act[ci] && (MODE == 1 || (li[ci] == a.tx - 1 && at < a.ntx - 1) ||
                                      (lj[ci] == a.ty - 1 && bt < a.nty - 1) || ir[ci] == a.nx - 1 ||
                                      jr[ci] == a.ny - 1 || kr[ci] == a.nz - 1);
                anyb |= bnd[ci];
            }
            if (__any_sync(0xffffffffu, anyb)) {
#pragma unroll
                for (int ci = 0; ci < 4; ++ci) {
                    if (!bnd[ci]) continue;
                    const int rt = ci >> 1;
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                        for (int b = 0; b < 2; ++b) {
                            const int slot = 8 * nt + 2 * tq + b;
                            if (slot >= AB) continue;
                            const float psi = q[rt][nt][2 * (ci & 1) + b];
                            if (li[ci] == a.tx - 1 && at < a.ntx - 1) {
                                const size_t fb = (((size_t)o * a.A8 + slot0 + slot) * a.G + g) * xf_stride;
                                a.xface[fb + ((size_t)at * a.ny + jr[ci]) * a.nz + kr[ci]] = psi;
                            }
                            if (lj[ci] == a.ty - 1 && bt < a.nty - 1) {
                                const size_t fb = (((size_t)o * a.A8 + slot0 + slot) * a.G + g) * yf_stride;
                                a.yface[fb + ((size_t)bt * a.nx + ir[ci]) * a.nz + kr[ci]] = psi;
                            }
                            if (ir[ci] == a.nx - 1 || jr[ci] == a.ny - 1 || kr[ci] == a.nz - 1) {
                                const float4 lc = leakc[slot];
                                float f = 0.0f;
                                if (ir[ci] == a.nx - 1) f += lc.x;
                                if (jr[ci] == a.ny - 1) f += lc.y;
                                if (kr[ci] == a.nz - 1) f += lc.z;
                                lk = fmaf(f, psi, lk);
                            }
                            if constexpr (MODE == 1) a.psi[((size_t)g * a.A + nbase + slot) * V + v[ci]] = psi;
                        }
                }
            }
        }
        if constexpr (MODE == 2) {
            // prod[g][v] += sum over this cell's real slots of w psi psi_stored
#pragma unroll
            for (int ci = 0; ci < 4; ++ci) {
                const int rt = ci >> 1;
                float pacc = 0.0f;
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int b = 0; b < 2; ++b) {
                        const int e = 2 * (ci & 1) + b;
                        const int slot = 8 * nt + 2 * tq + b;
                        if (act[ci] && slot < AB)
                            pacc = fmaf(leakc[slot].w * q[rt][nt][e],
                                        __ldg(a.psi + ((size_t)g * a.A + nbase + slot) * V + v[ci]), pacc);
                    }
                pacc += __shfl_xor_sync(0xffffffffu, pacc, 1);
                pacc += __shfl_xor_sync(0xffffffffu, pacc, 2);
                if (tq == 0 && act[ci]) atomicAdd(a.prod + gV + v[ci], pacc);
            }
        }
        // ---- directions -> moments ----------------------------------------------
#pragma unroll
        for (int rt = 0; rt < 2; ++rt) {
            float acc[2][4];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[nt][e] = 0.0f;
#pragma unroll
            for (int kt = 0; kt < 2; ++kt) {
                const float af[4] = {q[rt][kt][0], q[rt][kt][2], q[rt][kt][1], q[rt][kt][3]};
                uint32_t ah[4], al[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) split_tf32(af[e], ah[e], al[e]);
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) mma_3xtf32(acc[nt], ah, al, tabD[(kt * 2 + nt) * 32 + lane]);
            }
            const int c0 = 2 * rt, c1 = 2 * rt + 1;
            if (act[c0])
                atomicAdd(reinterpret_cast<float4*>(a.mom + (gV + v[c0]) * 16) + tq,
                          make_float4(acc[0][0], acc[0][1], acc[1][0], acc[1][1]));
            if (act[c1])
                atomicAdd(reinterpret_cast<float4*>(a.mom + (gV + v[c1]) * 16) + tq,
                          make_float4(acc[0][2], acc[0][3], acc[1][2], acc[1][3]));
        }
        __syncthreads();
    }
    double dl = (double)lk;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) dl += __shfl_down_sync(0xffffffffu, dl, off);
    if (lane == 0 && dl != 0.0) atomicAdd(a.leak + g, dl);
}

}  // namespace

size_t sweep_tc_smem_bytes(int ab, int tx, int ty, int nz, int nmat) {
    const int T = tx * ty;
    return sizeof(float4) * (256 + 2 * kSlots) +
           sizeof(float) * ((size_t)2 * kSlots * (T + 4) + (size_t)ab * (tx + ty) * nz + nmat);
}

bool sweep_tc_supported(int ab, int M, int tx, int ty) {
    return M == 16 && ab >= 1 && ab <= kSlots && (tx * ty) % 32 == 0 && tx * ty <= 256;
}

cudaError_t launch_sweep_tc(const SweepArgs& a, int mode, cudaStream_t s) {
    const int a_lo = a.stage - (a.nty - 1) > 0 ? a.stage - (a.nty - 1) : 0;
    const int a_hi = a.stage < a.ntx - 1 ? a.stage : a.ntx - 1;
    const int ntiles = a_hi - a_lo + 1;
    if (ntiles <= 0) return cudaSuccess;
    dim3 grid(ntiles, 8 * a.nab, a.G);
    const size_t smem = sweep_tc_smem_bytes(a.ab, a.tx, a.ty, a.nz, a.nmat);
    const int T = a.tx * a.ty;
    cudaError_t e = cudaSuccess;
    switch (mode) {
        case 0:
            e = cudaFuncSetAttribute(k_sweep_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) k_sweep_tc<0><<<grid, T, smem, s>>>(a);
            break;
        case 1:
            e = cudaFuncSetAttribute(k_sweep_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) k_sweep_tc<1><<<grid, T, smem, s>>>(a);
            break;
        case 2:
            e = cudaFuncSetAttribute(k_sweep_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) k_sweep_tc<2><<<grid, T, smem, s>>>(a);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t upload_tables_tc(const float* R, const float* w) {
    cudaError_t e = cudaMemcpyToSymbol(tc_R, R, sizeof(float) * kTcDirs * 16);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(tc_w, w, sizeof(float) * kTcDirs);
    return e;
}

}  // namespace doctors
