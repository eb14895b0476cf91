// The moment <-> direction transforms of the split dataflow sweep on the
// tensor cores: tcgen05.mma (kind::tf32) with the FP32 accumulator in tensor
// memory, as the three-term split-precision product (3xTF32).  Each operand
// x is split into hi = x rounded to TF32 and lo = x - hi (exact in FP32), and
// a.b ~ hi_a.hi_b + hi_a.lo_b + lo_a.hi_b; the dropped lo.lo term and the
// TF32 truncation of lo leave about 2^-21 of relative error.
//
// The transforms are the moment form of Eq. 2's scattering kernel and the
// quadrature sum of Eq. 3, for P3 (16 moments) and whole octants of S2-S8:
//
//   moments -> directions, k_m2d_tc: 128 rows (group, voxel) per tile,
//     Q[row][16 o + q] = sum_m S[row][m] B1[16 o + q][m],
//     B1[16 o + q][m] = s_o(m) (2l+1)/(4 pi) R_lm(Omega_q),
//   an M = 128, N = 128, K = 16 product (direction slots q >= AB are zero rows);
//   the epilogue writes each octant's angular-source record of ABP floats.
//
//   directions -> moments, k_d2m_tc: A[row][ABP o + q] = psi[g][o][v][q],
//     mom[row][m] = sum_k A[row][k] B2[m][k], B2[m][ABP o + q] = s_o(m) w_q R_lm(Omega_q),
//   an M = 128, N = 16, K = 8 ABP product.
//
// Omega_q is the first octant's direction q; octant o's directions are its
// reflections, and s_o(m) is the sign R_lm picks up under them.  Moments are
// in the library's storage order (position m holds lm = lm_of_pos(m, 16)).
//
// Shared-memory operands are K-major without swizzling: core matrices of 8
// rows x 16 bytes stored contiguously, [K/4][rows][4] floats, so the
// leading (K) byte offset between core matrices is rows * 16 and the stride
// (row-group) byte offset 128.  One CTA = 4 warps; warp w owns the tensor
// memory lanes 32 w .. 32 w + 31, i.e. rows 32 w .. 32 w + 31 of the tile.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "doctors_internal.h"

namespace doctors {

namespace {

constexpr int kTcThreads = 128;           // one row per thread
constexpr int kTcRows = 128;              // MMA M
constexpr long long kTcSpinLimit = 1LL << 26;

// TF32 round to nearest (ties away), as the hardware's cvt.rna.tf32.f32
__device__ __forceinline__ float tf32_hi(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// UMMA shared-memory descriptor, K-major, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;                  // descriptor version of this architecture
    return d;                                // base offset 0, layout type 0 (no swizzle)
}

// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// bounded wait for phase `parity` of an mbarrier; false if the bound ran out
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long long it = 0; it < kTcSpinLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 16 consecutive FP32 columns of this warp's 32 lanes: thread = lane = row
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// the same without the wait: the caller waits (tcgen05.wait::ld) before using v
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, float* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]),
          "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15])
        : "r"(taddr));
}

// allocate `cols` tensor-memory columns (one warp); the base address lands in *slot
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, int cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t base, int cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(base), "r"(cols) : "memory");
}

// split x into (hi, lo) and store both at float4 slot `at` of the hi and lo operands
__device__ __forceinline__ void store_split(float4* hi, float4* lo, int at, float4 x) {
    const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
    hi[at] = h;
    lo[at] = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
}

}  // namespace

// moments -> angular sources of all 8 octants.  Dynamic shared memory:
// A hi/lo [4][128][4] floats (8 KB each), B1 hi/lo [4][128][4] (8 KB each),
// mbarrier and tensor-memory slot; padded so that at most four CTAs share an
// SM (4 x 128 tensor-memory columns = all 512).
template <int AB>
__global__ void __launch_bounds__(kTcThreads) k_m2d_tc(const float* src, float* qang, const float* b1,
                                                       size_t V, int g0, int gcount, const int* skip, int* flag) {
    constexpr int ABP = (AB + 3) & ~3;
    constexpr int N = 128;
    extern __shared__ __align__(1024) float4 smq[];
    float4* a_hi = smq;                       // [4][128]
    float4* a_lo = a_hi + 4 * kTcRows;
    float4* b_hi = a_lo + 4 * kTcRows;        // [4][128]
    float4* b_lo = b_hi + 4 * N;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(b_lo + 4 * N);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    if (skip && *skip) return;
    const int tid = threadIdx.x, warp = tid >> 5;
    // B1 hi and lo, already in operand layout
    const float4* b4 = reinterpret_cast<const float4*>(b1);
    for (int e = tid; e < 8 * N; e += kTcThreads) b_hi[e] = b4[e];
    if (tid == 0) mbar_init(smem_u32(mbar), 1);
    if (warp == 0) tmem_alloc(tslot, N);
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = umma_idesc_tf32(kTcRows, N);
    const size_t rows = (size_t)gcount * V;
    const size_t tiles = (rows + kTcRows - 1) / kTcRows;
    uint32_t phase = 0;
    bool ok = true;
    for (size_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const size_t row = tile * kTcRows + tid;
        const bool live = row < rows;
        const size_t gv = live ? (size_t)g0 * V + row : 0;     // (g, v) as one index: g V + v
        const float4* s4 = reinterpret_cast<const float4*>(src + gv * 16);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            store_split(a_hi, a_lo, c * kTcRows + tid, live ? __ldg(s4 + c) : make_float4(0.f, 0.f, 0.f, 0.f));
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        if (tid == 0) {
            const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
            constexpr uint32_t lbo = kTcRows * 16, sbo = 128;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {                    // K = 16 in two steps of 8
                const uint32_t ko = ks * 2 * lbo;
                mma_tf32(tmem, umma_desc(ah + ko, lbo, sbo), umma_desc(bh + ko, N * 16, sbo), idesc, ks > 0);
                mma_tf32(tmem, umma_desc(ah + ko, lbo, sbo), umma_desc(bl + ko, N * 16, sbo), idesc, 1);
                mma_tf32(tmem, umma_desc(al + ko, lbo, sbo), umma_desc(bh + ko, N * 16, sbo), idesc, 1);
            }
            mma_commit(smem_u32(mbar));
        }
        if (!mbar_wait(smem_u32(mbar), phase)) {
            atomicExch(flag, 1);
            ok = false;
        }
        ok = __syncthreads_and(ok ? 1 : 0) != 0;     // one decision for the whole CTA
        phase ^= 1u;
        fence_after_sync();
        if (ok) {
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
            const size_t g = live ? gv / V : 0, v = live ? gv % V : 0;
            // two octants' columns per wait (registers for four CTAs per SM), then their records
#pragma unroll 1
            for (int o2 = 0; o2 < 8; o2 += 2) {
                float q[2][16];
                tmem_ld16_nowait(taddr + o2 * 16, q[0]);
                tmem_ld16_nowait(taddr + (o2 + 1) * 16, q[1]);
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                if (live) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        float4* out = reinterpret_cast<float4*>(qang + ((g * 8 + o2 + h) * V + v) * ABP);
#pragma unroll
                        for (int c4 = 0; c4 < ABP / 4; ++c4)
                            out[c4] = make_float4(q[h][4 * c4], q[h][4 * c4 + 1], q[h][4 * c4 + 2], q[h][4 * c4 + 3]);
                    }
                }
            }
        }
        fence_before_sync();
        __syncthreads();
    }
    fence_after_sync();
    if (warp == 0) tmem_free(tmem, N);
}

// angular fluence of all 8 octants -> moments.  Dynamic shared memory:
// A hi/lo [2 ABP][128][4] floats, B2 hi/lo [2 ABP][16][4], mbarrier, slot.
template <int AB>
__global__ void __launch_bounds__(kTcThreads) k_d2m_tc(const float* pang, float* mom, const float* b2, size_t V,
                                                       int g0, int gcount, const int* skip, int* flag) {
    constexpr int ABP = (AB + 3) & ~3;
    constexpr int KC = 2 * ABP;               // K / 4 core-matrix columns (K = 8 ABP)
    constexpr int N = 16;
    constexpr int TCOLS = 32;                 // smallest tensor-memory allocation
    extern __shared__ __align__(1024) float4 smd[];
    float4* a_hi = smd;                       // [KC][128]
    float4* a_lo = a_hi + KC * kTcRows;
    float4* b_hi = a_lo + KC * kTcRows;       // [KC][16]
    float4* b_lo = b_hi + KC * N;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(b_lo + KC * N);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    if (skip && *skip) return;
    const int tid = threadIdx.x, warp = tid >> 5;
    const float4* b4 = reinterpret_cast<const float4*>(b2);
    for (int e = tid; e < 2 * KC * N; e += kTcThreads) b_hi[e] = b4[e];
    if (tid == 0) mbar_init(smem_u32(mbar), 1);
    if (warp == 0) tmem_alloc(tslot, TCOLS);
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = umma_idesc_tf32(kTcRows, N);
    const size_t rows = (size_t)gcount * V;
    const size_t tiles = (rows + kTcRows - 1) / kTcRows;
    uint32_t phase = 0;
    bool ok = true;
    for (size_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const size_t row = tile * kTcRows + tid;
        const bool live = row < rows;
        const size_t gv = live ? (size_t)g0 * V + row : 0;
        const size_t g = gv / V, v = gv % V;
        // the row's 8 records: every load in flight before the first split
        float4 rec[8 * (ABP / 4)];
        if (live) {
            const float4* p4 = reinterpret_cast<const float4*>(pang + (g * 8 * V + v) * ABP);
            const size_t ostride = V * (ABP / 4);          // float4s between octant records
#pragma unroll
            for (int o = 0; o < 8; ++o)
#pragma unroll
                for (int c = 0; c < ABP / 4; ++c) rec[o * (ABP / 4) + c] = __ldg(p4 + o * ostride + c);
        } else {
#pragma unroll
            for (int e = 0; e < 8 * (ABP / 4); ++e) rec[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int e = 0; e < 8 * (ABP / 4); ++e) store_split(a_hi, a_lo, e * kTcRows + tid, rec[e]);
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        if (tid == 0) {
            const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
            constexpr uint32_t lbo_a = kTcRows * 16, lbo_b = N * 16, sbo = 128;
#pragma unroll 1
            for (int ks = 0; ks < KC / 2; ++ks) {              // K = 8 ABP in steps of 8
                const uint32_t ka = ks * 2 * lbo_a, kb = ks * 2 * lbo_b;
                mma_tf32(tmem, umma_desc(ah + ka, lbo_a, sbo), umma_desc(bh + kb, lbo_b, sbo), idesc, ks > 0);
                mma_tf32(tmem, umma_desc(ah + ka, lbo_a, sbo), umma_desc(bl + kb, lbo_b, sbo), idesc, 1);
                mma_tf32(tmem, umma_desc(al + ka, lbo_a, sbo), umma_desc(bh + kb, lbo_b, sbo), idesc, 1);
            }
            mma_commit(smem_u32(mbar));
        }
        if (!mbar_wait(smem_u32(mbar), phase)) {
            atomicExch(flag, 1);
            ok = false;
        }
        ok = __syncthreads_and(ok ? 1 : 0) != 0;     // one decision for the whole CTA
        phase ^= 1u;
        fence_after_sync();
        if (ok) {
            float m16[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16), m16);
            if (live) {
                float4* out = reinterpret_cast<float4*>(mom + gv * 16);
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4)
                    out[c4] = make_float4(m16[4 * c4], m16[4 * c4 + 1], m16[4 * c4 + 2], m16[4 * c4 + 3]);
            }
        }
        fence_before_sync();
        __syncthreads();
    }
    fence_after_sync();
    if (warp == 0) tmem_free(tmem, TCOLS);
}

namespace {

// TF32 round to nearest (ties away) of an FP32 value, on the host
float tf32_round_host(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

// sign of R_lm (storage position m of 16) in direction octant o
float octant_sign_host(int m, int o) {
    const int lm = lm_of_pos(m, 16);
    float r = 1.0f;
    if ((o & 1) && ((kOddX >> lm) & 1u)) r = -r;
    if ((o & 2) && ((kOddY >> lm) & 1u)) r = -r;
    if ((o & 4) && ((kOddZ >> lm) & 1u)) r = -r;
    return r;
}

// write x split into hi (first half of `out`) and lo (second half) at float index e
void put_split(std::vector<float>& out, size_t half, size_t e, float x) {
    const float h = tf32_round_host(x);
    out[e] = h;
    out[half + e] = x - h;
}

int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return sms;
}

// dynamic shared memory: operands, mbarrier and slot; the moment -> direction
// kernel is padded so that at most four CTAs (4 x 128 tensor-memory columns)
// share an SM
size_t m2d_smem() { return std::max<size_t>(4 * (2 * 128 + 2 * 128) * 16 + 16, 56 * 1024); }
size_t d2m_smem(int abp) { return (size_t)2 * abp * (2 * 128 + 2 * 16) * 16 + 16; }

}  // namespace

void build_tc_transform_tables(const ChainDirTable& dt, int AB, std::vector<float>& b1, std::vector<float>& b2) {
    const int abp = (AB + 3) & ~3;
    // B1: [4][128][4] floats, row n = 16 o + q, column k = m
    const size_t h1 = 4 * 128 * 4;
    b1.assign(2 * h1, 0.0f);
    for (int o = 0; o < 8; ++o)
        for (int q = 0; q < AB; ++q)
            for (int m = 0; m < 16; ++m) {
                const int n = 16 * o + q;
                put_split(b1, h1, ((size_t)(m / 4) * 128 + n) * 4 + m % 4, octant_sign_host(m, o) * dt.mop[q * 16 + m]);
            }
    // B2: [2 abp][16][4] floats, row n = m, column k = abp o + q
    const size_t h2 = (size_t)2 * abp * 16 * 4;
    b2.assign(2 * h2, 0.0f);
    for (int o = 0; o < 8; ++o)
        for (int q = 0; q < AB; ++q)
            for (int m = 0; m < 16; ++m) {
                const int k = abp * o + q;
                put_split(b2, h2, ((size_t)(k / 4) * 16 + m) * 4 + k % 4,
                          octant_sign_host(m, o) * dt.dop[m * kFlowMaxAB + q]);
            }
}

cudaError_t launch_m2d_tc(const SweepArgs& a, cudaStream_t s) {
    const size_t V = (size_t)a.nx * a.ny * a.nz;
    const size_t tiles = ((size_t)a.gcount * V + 127) / 128;
    const int sms = sm_count();
    if (sms <= 0) return cudaErrorInvalidDevice;
    const unsigned grid = (unsigned)std::min<size_t>(tiles, (size_t)4 * sms);
    const size_t smem = m2d_smem();
    cudaError_t e = cudaSuccess;
    auto go = [&](auto kern) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) kern<<<grid, 128, smem, s>>>(a.src, const_cast<float*>(a.qang), a.tc_b1, V, a.g0,
                                                           a.gcount, a.skip, a.flow + 2);
    };
    switch (a.ab) {
        case 1: go(k_m2d_tc<1>); break;
        case 3: go(k_m2d_tc<3>); break;
        case 6: go(k_m2d_tc<6>); break;
        case 10: go(k_m2d_tc<10>); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_d2m_tc(const SweepArgs& a, cudaStream_t s) {
    const size_t V = (size_t)a.nx * a.ny * a.nz;
    const size_t tiles = ((size_t)a.gcount * V + 127) / 128;
    const int sms = sm_count();
    if (sms <= 0) return cudaErrorInvalidDevice;
    const int abp = (a.ab + 3) & ~3;
    const size_t smem = d2m_smem(abp);
    const unsigned grid = (unsigned)std::min<size_t>(tiles, (size_t)2 * sms);
    cudaError_t e = cudaSuccess;
    auto go = [&](auto kern) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) kern<<<grid, 128, smem, s>>>(a.pang, a.mom, a.tc_b2, V, a.g0, a.gcount, a.skip,
                                                           a.flow + 2);
    };
    switch (a.ab) {
        case 1: go(k_d2m_tc<1>); break;
        case 3: go(k_d2m_tc<3>); break;
        case 6: go(k_d2m_tc<6>); break;
        case 10: go(k_d2m_tc<10>); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace doctors
