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
// Rows are cells: fragment row r of a warp is the cell of lane r, so lane
// (g, t) loads and accumulates the rows g, g+8, 16+g, 24+g.  With the moment
// record stored in the transposed order of lm_of_pos(), a lane's A-fragment
// entries of one cell are one float4 (positions 4t..4t+3), and so are its
// accumulator entries after the second product.  Between the two products a
// per-warp shared-memory block turns the C fragment (cells x direction slots)
// into one row per thread: each thread runs the step solve of its own cell
// (as in the CUDA-core sweep), writes its row of Psi back, and the second
// product reads the rows as A fragments with the summed direction index
// ordered as (2t, 2t+1) <-> (t, t+4).
#include <cstdint>

#include "doctors_internal.h"

namespace doctors {

constexpr int kTcDirs = 616;
__constant__ float tc_R[kTcDirs * 16];   // R_lm(Omega_n), (l, m) order, all S_N sets
__constant__ float tc_w[kTcDirs];        // w_n

namespace {

constexpr int kSlots = 16;               // direction slots per CTA (padded)
constexpr int kQS = 20;                  // row stride (floats) of the per-warp Q/Psi rows
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

// Split for the per-step operands: hi keeps the TF32 bits of x (truncated),
// lo = x - hi is exact in FP32 and is truncated to TF32 by the mma itself;
// the product error stays below ~2^-20 |a b|.
__device__ __forceinline__ void split_fast(float x, uint32_t& hi, uint32_t& lo) {
    hi = __float_as_uint(x) & 0xffffe000u;
    lo = __float_as_uint(x - __uint_as_float(hi));
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
// The upwind planes carry a one-column halo (x = -1, y = -1) that the
// boundary threads fill from the incoming face strips one step ahead, so the
// cell solve reads its x and y upwind values at fixed offsets.
template <int TX, int TY, int MODE>
__global__ void __launch_bounds__(TX * TY, 2) k_sweep_tc(const SweepArgs a) {
    if (a.skip && *a.skip) return;         // retired instance of a batched loop
    constexpr int T = TX * TY;              // columns = threads (multiple of 32)
    // plane pitch with the x halo, plus one spare column so that the stride
    // between consecutive diagonal-order threads (PX - 1) is odd: no bank conflicts
    constexpr int PX = TX + 2;
    constexpr int P = PX * (TY + 1);        // plane size with both halos
    extern __shared__ float4 sm4[];
    const int AB = a.ab;
    float4* tabM = sm4;                     // [2 kt][2 nt][32 lanes]  moments -> directions
    float4* tabD = tabM + 128;              // [2 kt][2 nt][32 lanes]  directions -> moments
    float4* coefs = tabD + 128;             // [16 slots]: cx, cy, cz, cx+cy+cz
    float4* leakc = coefs + kSlots;         // [16 slots]: leak_x, leak_y, leak_z, w
    float* qs = reinterpret_cast<float*>(leakc + kSlots);   // per warp [32 rows][kQS]: Q, then Psi
    float* buf = qs + T * kQS;              // [2][16 slots][P] previous/current hyperplane
    float* xin = buf + 2 * kSlots * P;      // [AB][TY][nz]
    float* yin = xin + AB * TY * a.nz;      // [AB][TX][nz]
    float* sigt_s = yin + AB * TX * a.nz;   // [nmat]

    const int g = a.g0 + blockIdx.z;
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
        {
            const int col = gq;
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
        } else {
            coefs[t] = make_float4(0.0f, 0.0f, 0.0f, 1.0f);
            leakc[t] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
    }
    for (int t = threadIdx.x; t < a.nmat; t += blockDim.x) sigt_s[t] = a.sigt[t * a.G + g];
    for (int t = threadIdx.x; t < 2 * kSlots * P; t += blockDim.x) buf[t] = 0.0f;
    {
        const int nxs = AB * TY * a.nz;
        for (int t = threadIdx.x; t < nxs; t += blockDim.x) {
            const int q = t / (TY * a.nz), r = t % (TY * a.nz);
            const int jr = bt * TY + r / a.nz;
            float val = 0.0f;
            if (at > 0 && jr < a.ny) {
                const size_t fb = (((size_t)o * a.A8 + slot0 + q) * a.G + g) * xf_stride;
                val = a.xface[fb + (size_t)(at - 1) * a.ny * a.nz + (size_t)bt * TY * a.nz + r];
            }
            xin[t] = val;
        }
        const int nys = AB * TX * a.nz;
        for (int t = threadIdx.x; t < nys; t += blockDim.x) {
            const int q = t / (TX * a.nz), r = t % (TX * a.nz);
            const int ir = at * TX + r / a.nz;
            float val = 0.0f;
            if (bt > 0 && ir < a.nx) {
                const size_t fb = (((size_t)o * a.A8 + slot0 + q) * a.G + g) * yf_stride;
                val = a.yface[fb + (size_t)(bt - 1) * a.nx * a.nz + (size_t)at * TX * a.nz + r];
            }
            yin[t] = val;
        }
    }
    __syncthreads();

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int gq = lane >> 2, tq = lane & 3;
    float* wq = qs + (tid >> 5) * 32 * kQS;        // this warp's Q/Psi rows
    // threads own the tile's columns in diagonal order (li + lj ascending)
    int li = 0, lj = 0;
    {
        int base = 0;
        for (int d = 0; d <= TX + TY - 2; ++d) {
            const int lo = d > TY - 1 ? d - (TY - 1) : 0;
            const int hi = d < TX - 1 ? d : TX - 1;
            const int cnt = hi - lo + 1;
            if (tid < base + cnt) {
                li = lo + (tid - base);
                lj = d - li;
                break;
            }
            base += cnt;
        }
    }
    const int pc = (lj + 1) * PX + (li + 1);       // plane cell of this column
    const int ir = at * TX + li, jr = bt * TY + lj;
    const bool col = ir < a.nx && jr < a.ny;
    const int i = sx > 0 ? ir : a.nx - 1 - ir;
    const int j = sy > 0 ? jr : a.ny - 1 - jr;
    const size_t V = (size_t)a.nx * a.ny * a.nz;
    const size_t gV = (size_t)g * V;
    const size_t plane = (size_t)a.nx * a.ny;
    const size_t vcol = (size_t)j * a.nx + i;
    const bool xout = li == TX - 1 && at < a.ntx - 1;
    const bool yout = lj == TY - 1 && bt < a.nty - 1;
    const bool xleak = ir == a.nx - 1, yleak = jr == a.ny - 1;
    float* xo = a.xface + (((size_t)o * a.A8 + slot0) * a.G + g) * xf_stride + ((size_t)at * a.ny + jr) * a.nz;
    float* yo = a.yface + (((size_t)o * a.A8 + slot0) * a.G + g) * yf_stride + ((size_t)bt * a.nx + ir) * a.nz;
    const size_t xo_q = (size_t)a.G * xf_stride, yo_q = (size_t)a.G * yf_stride;

    // halo values of step hh (incoming faces of the tile's first column/row)
    auto fill_halo = [&](int hh, float* dst) {
        if (li == 0) {
            const int kq = hh - lj;
            if (kq >= 0 && kq < a.nz)
                for (int s = 0; s < AB; ++s) dst[s * P + (lj + 1) * PX] = xin[(s * TY + lj) * a.nz + kq];
        }
        if (lj == 0) {
            const int kq = hh - li;
            if (kq >= 0 && kq < a.nz)
                for (int s = 0; s < AB; ++s) dst[s * P + li + 1] = yin[(s * TX + li) * a.nz + kq];
        }
    };
    fill_halo(0, buf + kSlots * P);                 // step 0 reads plane 1
    __syncthreads();

    float zc[kSlots];
#pragma unroll
    for (int q = 0; q < kSlots; ++q) zc[q] = 0.0f;
    float lk = 0.0f;

    const int hmax = TX + TY + a.nz - 3;
    for (int h = 0; h <= hmax; ++h) {
        const int kr = h - li - lj;
        const float* prev = buf + ((h & 1) ^ 1) * kSlots * P;
        float* cur = buf + (h & 1) * kSlots * P;
        const bool act = col && kr >= 0 && kr < a.nz;
        const unsigned amask = __ballot_sync(0xffffffffu, act);
        if (amask) {
            const int k = sz > 0 ? kr : a.nz - 1 - kr;
            const unsigned vme = act ? (unsigned)((size_t)k * plane + vcol) : 0u;   // V < 2^31
            unsigned vr[4];
            bool ar[4];
#pragma unroll
            for (int ci = 0; ci < 4; ++ci) {
                vr[ci] = __shfl_sync(0xffffffffu, vme, gq + 8 * ci);
                ar[ci] = (amask >> (gq + 8 * ci)) & 1u;
            }
            // ---- moments -> directions (3xTF32 mma) ---------------------------------
#pragma unroll
            for (int rt = 0; rt < 2; ++rt) {
                const float4 s0 = ar[2 * rt] ? __ldg(reinterpret_cast<const float4*>(a.src + (gV + vr[2 * rt]) * 16) + tq)
                                             : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                const float4 s1 = ar[2 * rt + 1]
                                      ? __ldg(reinterpret_cast<const float4*>(a.src + (gV + vr[2 * rt + 1]) * 16) + tq)
                                      : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                float q[2][4];
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) q[nt][e] = 0.0f;
#pragma unroll
                for (int kt = 0; kt < 2; ++kt) {
                    const float af[4] = {kt == 0 ? s0.x : s0.z, kt == 0 ? s1.x : s1.z,
                                         kt == 0 ? s0.y : s0.w, kt == 0 ? s1.y : s1.w};
                    uint32_t ah[4], al[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) split_fast(af[e], ah[e], al[e]);
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt) mma_3xtf32(q[nt], ah, al, tabM[(kt * 2 + nt) * 32 + lane]);
                }
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    const int c = 8 * nt + 2 * tq;
                    *reinterpret_cast<float2*>(wq + (16 * rt + gq) * kQS + c) = make_float2(q[nt][0], q[nt][1]);
                    *reinterpret_cast<float2*>(wq + (16 * rt + gq + 8) * kQS + c) = make_float2(q[nt][2], q[nt][3]);
                }
            }
            __syncwarp();
            // ---- step-differenced cell solve, one thread per column ---------------------
            float* my = wq + lane * kQS;
            if (act) {
                const float sig = __ldg(a.rho + vme) * sigt_s[__ldg(a.mat + vme)];
                float psi[kSlots];
#pragma unroll
                for (int c4 = 0; c4 < kSlots / 4; ++c4) {
                    const float4 t4 = *reinterpret_cast<const float4*>(my + 4 * c4);
                    psi[4 * c4] = t4.x; psi[4 * c4 + 1] = t4.y; psi[4 * c4 + 2] = t4.z; psi[4 * c4 + 3] = t4.w;
                }
                const float* px = prev + pc - 1;
                const float* py = prev + pc - PX;
                float* pw = cur + pc;
#pragma unroll
                for (int s = 0; s < kSlots; ++s) {
                    const float4 cf = coefs[s];
                    const float num = fmaf(cf.z, zc[s], fmaf(cf.y, py[s * P], fmaf(cf.x, px[s * P], psi[s])));
                    psi[s] = __fdividef(num, sig + cf.w);
                    pw[s * P] = psi[s];
                    zc[s] = psi[s];
                }
#pragma unroll
                for (int c4 = 0; c4 < kSlots / 4; ++c4)
                    *reinterpret_cast<float4*>(my + 4 * c4) =
                        make_float4(psi[4 * c4], psi[4 * c4 + 1], psi[4 * c4 + 2], psi[4 * c4 + 3]);
                // rare paths read this cell's Psi row back from shared memory
                if (xout)
                    for (int s = 0; s < AB; ++s) xo[s * xo_q + kr] = my[s];
                if (yout)
                    for (int s = 0; s < AB; ++s) yo[s * yo_q + kr] = my[s];
                if (xleak || yleak || kr == a.nz - 1) {
                    for (int s = 0; s < AB; ++s) {
                        const float4 lc = leakc[s];
                        float f = 0.0f;
                        if (xleak) f += lc.x;
                        if (yleak) f += lc.y;
                        if (kr == a.nz - 1) f += lc.z;
                        lk = fmaf(f, my[s], lk);
                    }
                }
                // stored angular fluence [G][V][A] (the stage kernels' layout)
                if constexpr (MODE == 1) {
                    float* rec = a.psi + ((size_t)g * V + vme) * a.A + nbase;
                    for (int s = 0; s < AB; ++s) rec[s] = my[s];
                }
                if constexpr (MODE == 2) {
                    const float* rec = a.psi + ((size_t)g * V + vme) * a.A + nbase;
                    float pacc = 0.0f;
                    for (int s = 0; s < AB; ++s) pacc = fmaf(leakc[s].w * my[s], __ldg(rec + s), pacc);
                    atomicAdd(a.prod + gV + vme, pacc);
                }
            } else {
#pragma unroll
                for (int c4 = 0; c4 < kSlots / 4; ++c4)
                    *reinterpret_cast<float4*>(my + 4 * c4) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
            __syncwarp();
            // ---- directions -> moments (3xTF32 mma) ---------------------------------
#pragma unroll
            for (int rt = 0; rt < 2; ++rt) {
                float acc[2][4];
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[nt][e] = 0.0f;
#pragma unroll
                for (int kt = 0; kt < 2; ++kt) {
                    const int c = 8 * kt + 2 * tq;
                    const float2 p0 = *reinterpret_cast<const float2*>(wq + (16 * rt + gq) * kQS + c);
                    const float2 p1 = *reinterpret_cast<const float2*>(wq + (16 * rt + gq + 8) * kQS + c);
                    const float af[4] = {p0.x, p1.x, p0.y, p1.y};
                    uint32_t ah[4], al[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) split_fast(af[e], ah[e], al[e]);
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt) mma_3xtf32(acc[nt], ah, al, tabD[(kt * 2 + nt) * 32 + lane]);
                }
                if (ar[2 * rt])
                    atomicAdd(reinterpret_cast<float4*>(a.mom + (gV + vr[2 * rt]) * 16) + tq,
                              make_float4(acc[0][0], acc[0][1], acc[1][0], acc[1][1]));
                if (ar[2 * rt + 1])
                    atomicAdd(reinterpret_cast<float4*>(a.mom + (gV + vr[2 * rt + 1]) * 16) + tq,
                              make_float4(acc[0][2], acc[0][3], acc[1][2], acc[1][3]));
            }
        }
        // incoming face values of the next step go into this step's plane
        fill_halo(h + 1, cur);
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
           sizeof(float) * ((size_t)T * kQS + (size_t)2 * kSlots * (tx + 2) * (ty + 1) + (size_t)ab * (tx + ty) * nz +
                            nmat);
}

bool sweep_tc_supported(int ab, int M, int tx, int ty) {
    const bool tile = (tx == 16 && ty == 16) || (tx == 32 && ty == 8) || (tx == 16 && ty == 8) || (tx == 8 && ty == 16) ||
                      (tx == 8 && ty == 8) || (tx == 8 && ty == 4);
    return M == 16 && ab >= 1 && ab <= kSlots && tile;
}

template <int TX, int TY>
cudaError_t launch_tc_tile(const SweepArgs& a, int mode, dim3 grid, size_t smem, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    switch (mode) {
        case 0:
            e = cudaFuncSetAttribute(k_sweep_tc<TX, TY, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) k_sweep_tc<TX, TY, 0><<<grid, TX * TY, smem, s>>>(a);
            break;
        case 1:
            e = cudaFuncSetAttribute(k_sweep_tc<TX, TY, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) k_sweep_tc<TX, TY, 1><<<grid, TX * TY, smem, s>>>(a);
            break;
        case 2:
            e = cudaFuncSetAttribute(k_sweep_tc<TX, TY, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) k_sweep_tc<TX, TY, 2><<<grid, TX * TY, smem, s>>>(a);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return e;
}

cudaError_t launch_sweep_tc(const SweepArgs& a, int mode, cudaStream_t s) {
    const int a_lo = a.stage - (a.nty - 1) > 0 ? a.stage - (a.nty - 1) : 0;
    const int a_hi = a.stage < a.ntx - 1 ? a.stage : a.ntx - 1;
    const int ntiles = a_hi - a_lo + 1;
    if (ntiles <= 0) return cudaSuccess;
    dim3 grid(ntiles, 8 * a.nab, a.gcount);
    const size_t smem = sweep_tc_smem_bytes(a.ab, a.tx, a.ty, a.nz, a.nmat);
    cudaError_t e;
    if (a.tx == 16 && a.ty == 16) e = launch_tc_tile<16, 16>(a, mode, grid, smem, s);
    else if (a.tx == 32 && a.ty == 8) e = launch_tc_tile<32, 8>(a, mode, grid, smem, s);
    else if (a.tx == 16 && a.ty == 8) e = launch_tc_tile<16, 8>(a, mode, grid, smem, s);
    else if (a.tx == 8 && a.ty == 16) e = launch_tc_tile<8, 16>(a, mode, grid, smem, s);
    else if (a.tx == 8 && a.ty == 8) e = launch_tc_tile<8, 8>(a, mode, grid, smem, s);
    else if (a.tx == 8 && a.ty == 4) e = launch_tc_tile<8, 4>(a, mode, grid, smem, s);
    else return cudaErrorInvalidValue;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t upload_tables_tc(const float* R, const float* w) {
    cudaError_t e = cudaMemcpyToSymbol(tc_R, R, sizeof(float) * kTcDirs * 16);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(tc_w, w, sizeof(float) * kTcDirs);
    return e;
}

}  // namespace doctors
