// Scattering-source update, FP64 reductions (residual, balance), dose tally
// and fluence extraction.
//
// Eq. 2's scattering term with the kernel as a Legendre expansion reduces, in
// moment form, to s_lm[g](v) = rho_v sum_{g'} sigma_s,l(g' -> g) phi_lm[g'](v)
// (downscatter only, self-scatter included).  The first-collision source is
// the same map applied to the uncollided moments (Sec. II.A).  Eq. 3's scalar
// fluence is the lm = 00 moment.  The dose tally multiplies the group fluence
// by group-wise conversion factors (Sec. II.A, III.A) and is accumulated in
// FP64, like the residual norm and the particle balance.
#include <mutex>
#include <string>
#include <vector>

#include "doctors_internal.h"

namespace doctors {

cudaError_t launch_sweep_m1_entry(const SweepArgs& a, int mode, cudaStream_t s);
cudaError_t launch_sweep_m4_entry(const SweepArgs& a, int mode, cudaStream_t s);
cudaError_t launch_sweep_m9_entry(const SweepArgs& a, int mode, cudaStream_t s);
cudaError_t launch_sweep_m16_entry(const SweepArgs& a, int mode, cudaStream_t s);

int sweep_chain_blocks_m1(int ab, bool ct, int threads, size_t smem);
int sweep_chain_blocks_m4(int ab, bool ct, int threads, size_t smem);
int sweep_chain_blocks_m9(int ab, bool ct, int threads, size_t smem);
int sweep_chain_blocks_m16(int ab, bool ct, int threads, size_t smem);

cudaError_t launch_sweep_flow_m1_entry(const SweepArgs& a, int mode, cudaStream_t s);
cudaError_t launch_sweep_flow_m4_entry(const SweepArgs& a, int mode, cudaStream_t s);
cudaError_t launch_sweep_flow_m9_entry(const SweepArgs& a, int mode, cudaStream_t s);
cudaError_t launch_sweep_flow_m16_entry(const SweepArgs& a, int mode, cudaStream_t s);
int sweep_flow_blocks_m1(int ab, int threads, size_t smem, bool split, bool dd, bool hw);
cudaError_t launch_split_sweep_m1_entry(const SweepArgs& a, cudaStream_t s, int* count);
int sweep_flow_blocks_m4(int ab, int threads, size_t smem, bool split, bool dd, bool hw);
cudaError_t launch_split_sweep_m4_entry(const SweepArgs& a, cudaStream_t s, int* count);
int sweep_flow_blocks_m9(int ab, int threads, size_t smem, bool split, bool dd, bool hw);
cudaError_t launch_split_sweep_m9_entry(const SweepArgs& a, cudaStream_t s, int* count);
int sweep_flow_blocks_m16(int ab, int threads, size_t smem, bool split, bool dd, bool hw);
cudaError_t launch_split_sweep_m16_entry(const SweepArgs& a, cudaStream_t s, int* count);

cudaError_t upload_tables_m1(const float* R, const float* w);
cudaError_t upload_tables_m4(const float* R, const float* w);
cudaError_t upload_tables_m9(const float* R, const float* w);
cudaError_t upload_tables_m16(const float* R, const float* w);

namespace {
std::mutex g_table_mu;
bool g_table_done[64] = {};
const int kOrders[6] = {2, 4, 6, 8, 12, 16};
}  // namespace

// The level-symmetric sets and their harmonics depend only on N, so one
// concatenated table (S2, S4, S6, S8, S12, S16) serves every problem.
cudaError_t ensure_direction_tables(int device, int N, int* base) {
    int off = 0, found = -1;
    for (int q = 0; q < 6; ++q) {
        if (kOrders[q] == N) found = off;
        off += kOrders[q] * (kOrders[q] + 2);
    }
    if (found < 0 || device < 0 || device >= 64) return cudaErrorInvalidValue;
    *base = found;
    std::lock_guard<std::mutex> lock(g_table_mu);
    if (g_table_done[device]) return cudaSuccess;
    std::vector<float> R, w;
    for (int q = 0; q < 6; ++q) {
        std::vector<double> dirs, wt;
        std::string err;
        if (!build_quadrature(kOrders[q], dirs, wt, err)) return cudaErrorInvalidValue;
        for (size_t n = 0; n < wt.size(); ++n) {
            double r[16];
            real_harmonics(3, dirs[3 * n], dirs[3 * n + 1], dirs[3 * n + 2], r);
            for (int m = 0; m < 16; ++m) R.push_back((float)r[m]);
            w.push_back((float)wt[n]);
        }
    }
    cudaError_t e = upload_tables_m1(R.data(), w.data());
    if (e == cudaSuccess) e = upload_tables_m4(R.data(), w.data());
    if (e == cudaSuccess) e = upload_tables_m9(R.data(), w.data());
    if (e == cudaSuccess) e = upload_tables_m16(R.data(), w.data());
    if (e == cudaSuccess) g_table_done[device] = true;
    return e;
}

bool sweep_supported(int ab, int M) {
    const int abs_ok[] = {1, 2, 3, 4, 5, 6, 7, 9, 10, 12};
    bool ok = false;
    for (int x : abs_ok) ok |= (x == ab);
    return ok && (M == 1 || M == 4 || M == 9 || M == 16);
}

int sweep_chain_blocks_per_sm(int ab, bool ct, int M, int threads, size_t smem) {
    switch (M) {
        case 1: return sweep_chain_blocks_m1(ab, ct, threads, smem);
        case 4: return sweep_chain_blocks_m4(ab, ct, threads, smem);
        case 9: return sweep_chain_blocks_m9(ab, ct, threads, smem);
        case 16: return sweep_chain_blocks_m16(ab, ct, threads, smem);
        default: return 0;
    }
}

int sweep_flow_blocks_per_sm(int ab, int M, int threads, size_t smem, bool split, bool dd, bool hw) {
    switch (M) {
        case 1: return sweep_flow_blocks_m1(ab, threads, smem, split, dd, hw);
        case 4: return sweep_flow_blocks_m4(ab, threads, smem, split, dd, hw);
        case 9: return sweep_flow_blocks_m9(ab, threads, smem, split, dd, hw);
        case 16: return sweep_flow_blocks_m16(ab, threads, smem, split, dd, hw);
        default: return 0;
    }
}

cudaError_t launch_split_sweep(const SweepArgs& a, int M, cudaStream_t s, int* count) {
    switch (M) {
        case 1: return launch_split_sweep_m1_entry(a, s, count);
        case 4: return launch_split_sweep_m4_entry(a, s, count);
        case 9: return launch_split_sweep_m9_entry(a, s, count);
        case 16: return launch_split_sweep_m16_entry(a, s, count);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sweep_flow(const SweepArgs& a, int M, int mode, cudaStream_t s) {
    switch (M) {
        case 1: return launch_sweep_flow_m1_entry(a, mode, s);
        case 4: return launch_sweep_flow_m4_entry(a, mode, s);
        case 9: return launch_sweep_flow_m9_entry(a, mode, s);
        case 16: return launch_sweep_flow_m16_entry(a, mode, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sweep_stage(const SweepArgs& a, int M, int mode, cudaStream_t s) {
    switch (M) {
        case 1: return launch_sweep_m1_entry(a, mode, s);
        case 4: return launch_sweep_m4_entry(a, mode, s);
        case 9: return launch_sweep_m9_entry(a, mode, s);
        case 16: return launch_sweep_m16_entry(a, mode, s);
        default: return cudaErrorInvalidValue;
    }
}

namespace {

// Threads stride over (voxel, moment) pairs, moment fastest, so that a warp reads and
// writes contiguous memory.  A thread loads the moments of every source group
// it needs into registers once (all loads in flight together) and forms each
// destination group's sum from them; the group loops are unrolled up to
// GMAX (>= G) so that the moments stay in registers.  The scattering table
// is staged in shared memory when it fits.  Blocks stride over the
// (voxel, moment) range, so each stages the table once.
constexpr int kScatterThreads = 256;
constexpr size_t kScatterTableSmem = 100 * 1024;  // largest staged table

// staged table: [nmat][L+1] blocks of [GMAX (from)][GMAX (to)], so that every
// entry a thread reads is at a compile-time offset from its (material, degree)
// block; the block pitch GMAX^2 + 1 is odd, so the lanes of a warp (two voxels,
// up to eight blocks) read distinct shared-memory banks
template <int GMAX>
__host__ __device__ constexpr int scatter_block_pitch() { return GMAX * GMAX + 1; }
template <int GMAX>
size_t scatter_table_bytes(const ScatterArgs& a) {
    return (size_t)a.nmat * (a.L + 1) * scatter_block_pitch<GMAX>() * sizeof(float);
}

template <int GMAX>
__global__ void __launch_bounds__(kScatterThreads, 3) k_scatter(const ScatterArgs a, int table_in_smem) {
    extern __shared__ float tab_s[];
    if (a.skip && *a.skip) return;
    const int G = a.G;
    if (table_in_smem) {
        constexpr int BP = scatter_block_pitch<GMAX>();
        const int nblk = a.nmat * (a.L + 1);
        for (int e = threadIdx.x; e < nblk * BP; e += blockDim.x) {
            const int blk = e / BP, r = e % BP, i = r / GMAX, j = r % GMAX;
            tab_s[e] = (r < GMAX * GMAX && i < G && j < G) ? __ldg(a.sigs + ((size_t)blk * G + i) * G + j) : 0.0f;
        }
        __syncthreads();
    }
    const size_t VM = a.V * a.M;
    const int g_beg = a.win ? a.win[0] : a.g0, g_end = a.win ? a.win[1] : (a.g1 > 0 ? a.g1 : G);
    // no barrier below: threads leave the grid-stride loop independently
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < VM; t += (size_t)gridDim.x * blockDim.x) {
        const size_t v = t / a.M;
        const int lm = (int)(t % a.M);
        const int l = degree_of_lm(lm_of_pos(lm, a.M));
        float ph[GMAX];
        float r = 0.0f;
        int mb = 0;
        if (a.phi) {
            mb = __ldg(a.mat + v) * (a.L + 1) + l;     // (material, degree) block of the table
            r = __ldg(a.rho + v);
            // every source group a destination group of the window needs
#pragma unroll
            for (int gp = 0; gp < GMAX; ++gp) {
                const bool need = a.transpose ? (gp >= g_beg && gp < G) : (gp < g_end);
                ph[gp] = need ? __ldg(a.phi + gp * VM + t) : 0.0f;
            }
        }
        // the fixed source of every destination group, also loaded up front
        float qb[GMAX];
#pragma unroll
        for (int g = 0; g < GMAX; ++g) qb[g] = (a.base && g >= g_beg && g < g_end) ? __ldg(a.base + g * VM + t) : 0.0f;
        const float* ts = tab_s + (size_t)mb * scatter_block_pitch<GMAX>();
        const float* tg = a.sigs + (size_t)mb * G * G;
#pragma unroll
        for (int g = 0; g < GMAX; ++g) {
            if (g < g_beg || g >= g_end) continue;
            float out = qb[g];
            if (lm == 0) {
                if (a.iso) out += __ldg(a.iso + g);
                if (a.iso_field) out += a.iso_field_scale * __ldg(a.iso_field + (size_t)g * a.V + v);
            }
            if (a.phi) {
                float acc = 0.0f;
                if (!a.transpose) {
                    // downscatter: g' <= g
                    if (table_in_smem) {
#pragma unroll
                        for (int gp = 0; gp <= g; ++gp) acc = fmaf(ts[gp * GMAX + g], ph[gp], acc);
                    } else {
#pragma unroll
                        for (int gp = 0; gp <= g; ++gp) acc = fmaf(__ldg(tg + gp * G + g), ph[gp], acc);
                    }
                } else {
                    // adjoint: g' >= g (zero padding beyond G in the staged table)
                    if (table_in_smem) {
#pragma unroll
                        for (int gp = g; gp < GMAX; ++gp) acc = fmaf(ts[g * GMAX + gp], ph[gp], acc);
                    } else {
#pragma unroll
                        for (int gp = g; gp < GMAX; ++gp)
                            if (gp < G) acc = fmaf(__ldg(tg + g * G + gp), ph[gp], acc);
                    }
                }
                out = fmaf(r, acc, out);
            }
            a.out[g * VM + t] = out;
        }
    }
}

// The iteration's form of the same map (a scattering term, no per-voxel
// isotropic field, fewer than 2^31 entries) with no branch in its group
// loops (ISO: the first-collision form, with the volume sources' isotropic
// term and no fixed source, added to the l = 0 entries): the
// direction of the sum (downscatter or its transpose) and the presence of a
// fixed source are template parameters, the group window only predicates the
// loads of the fixed source and the stores, and entry indices are 32-bit.  The
// inner sums are those of k_scatter term by term, so the two kernels give
// identical results.  Every source group below G is needed by some group of
// the window (the forward window only retires leading groups, the adjoint
// window trailing ones), so all G source moments are loaded; padding groups up
// to GMAX read group G-1's row again and are zeroed.
__device__ __forceinline__ float ldg_if(const float* p, bool pred) {
    float x = 0.0f;
    asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.global.nc.f32 %0, [%1];\n\t}"
        : "+f"(x)
        : "l"(p), "r"((unsigned)pred));
    return x;
}

// staged table of k_scatter_fast: per (material, degree) block GMAX rows of
// GMAX entries, row g holding the entries destination group g sums over in
// ascending source order (forward: sigma(g' -> g) for g' = 0..GMAX-1, the
// table's column g; adjoint: sigma(g -> g'), its row g), so that a thread
// reads them as 16-byte vectors.  The block pitch GMAX^2 + 4 is 4 or 20 mod
// 32 words for every GMAX used, so eight consecutive blocks (the degrees of
// two voxels of neighbouring materials, as one warp reads them) start in
// distinct 16-byte bank groups.
template <int GMAX>
__host__ __device__ constexpr int scatter_fast_pitch() { return GMAX * GMAX + 4; }
template <int GMAX>
size_t scatter_fast_table_bytes(const ScatterArgs& a) {
    return (size_t)a.nmat * (a.L + 1) * scatter_fast_pitch<GMAX>() * sizeof(float);
}

template <int GMAX, bool TR, bool HAS_BASE, bool ISO = false>
__global__ void __launch_bounds__(kScatterThreads, GMAX <= 24 ? 2 : 1) k_scatter_fast(const ScatterArgs a) {
    extern __shared__ float4 tab4_s[];
    float* tab_s = reinterpret_cast<float*>(tab4_s);
    static_assert(GMAX % 4 == 0, "rows of whole 16-byte vectors");
    if (a.skip && *a.skip) return;
    const int G = a.G;
    constexpr int BP = scatter_fast_pitch<GMAX>();
    const int nblk = a.nmat * (a.L + 1);
    for (int e = threadIdx.x; e < nblk * BP; e += blockDim.x) {
        const int blk = e / BP, r = e % BP, i = r / GMAX, j = r % GMAX;   // row i, entry j
        const int from = TR ? i : j, to = TR ? j : i;
        tab_s[e] = (r < GMAX * GMAX && i < G && j < G) ? __ldg(a.sigs + ((size_t)blk * G + from) * G + to) : 0.0f;
    }
    __syncthreads();
    const unsigned VM = (unsigned)(a.V * a.M), M = (unsigned)a.M;
    const int g_beg = a.win ? a.win[0] : a.g0, g_end = a.win ? a.win[1] : (a.g1 > 0 ? a.g1 : G);
    const int L1 = a.L + 1;
    // no barrier below: threads leave the grid-stride loop independently
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < VM; t += gridDim.x * blockDim.x) {
        const unsigned v = t / M;
        const int lm = (int)(t - v * M);
        const int mb = __ldg(a.mat + v) * L1 + degree_of_lm(lm_of_pos(lm, (int)M));
        const float r = __ldg(a.rho + v);
        float ph[GMAX];
        const float* pp = a.phi + t;
#pragma unroll
        for (int gp = 0; gp < GMAX; ++gp) {
            const float x = __ldg(pp + (size_t)(gp < G ? gp : G - 1) * VM);
            ph[gp] = gp < G ? x : 0.0f;
        }
        float qb[GMAX];
        const float* pb = a.base + t;
#pragma unroll
        for (int g = 0; g < GMAX; ++g) qb[g] = HAS_BASE ? ldg_if(pb + (size_t)g * VM, g >= g_beg && g < g_end) : 0.0f;
        if (ISO && lm == 0) {
#pragma unroll
            for (int g = 0; g < GMAX; ++g)
                if (g < G) qb[g] += __ldg(a.iso + g);
        }
        const float4* ts4 = reinterpret_cast<const float4*>(tab_s + mb * BP);
        float* po = a.out + t;
#pragma unroll
        for (int g = 0; g < GMAX; ++g) {
            // the same sums as k_scatter, source groups ascending: forward
            // g' = 0..g, adjoint g' = g..GMAX-1, read four entries at a time
            float acc = 0.0f;
            constexpr int R4 = GMAX / 4;
#pragma unroll
            for (int c = TR ? g / 4 : 0; c < (TR ? R4 : g / 4 + 1); ++c) {
                const float4 t4 = ts4[g * R4 + c];
                const float tv[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int gp = 4 * c + k;
                    if (TR ? gp >= g : gp <= g) acc = fmaf(tv[k], ph[gp], acc);
                }
            }
            const float out = fmaf(r, acc, qb[g]);
            if (g >= g_beg && g < g_end) po[(size_t)g * VM] = out;
        }
    }
}

template <int NV>
__device__ __forceinline__ void block_reduce_add(double (&x)[NV], double* dst) {
    __shared__ double red[NV][32];
#pragma unroll
    for (int q = 0; q < NV; ++q)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x[q] += __shfl_down_sync(0xffffffffu, x[q], off);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) red[q][wid] = x[q];
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double y = lane < nw ? red[q][lane] : 0.0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) y += __shfl_down_sync(0xffffffffu, y, off);
            if (lane == 0 && y != 0.0) atomicAdd(dst + q, y);
        }
    }
}

// grid: (blocks over V, G).  The four elements of one pass are differenced
// and squared in FP32 (a relative error near 1e-7 in a convergence norm that
// is compared against tolerances of 1e-6 and above); the passes, the threads
// and the blocks are summed in FP64, so that few FP64 operations are issued:
// their rate on this part is a small fraction of the FP32 rate.
// rho sigma_t of every cell and group, the product the sweep would form per cell step
__global__ void __launch_bounds__(256) k_total_xs(size_t V, int G, const uint8_t* mat, const float* rho,
                                                  const float* sigt, float* out) {
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (size_t)gridDim.x * blockDim.x) {
        const float r = rho[v];
        const int m = mat[v];
        for (int g = 0; g < G; ++g) out[(size_t)g * V + v] = r * __ldg(sigt + m * G + g);
    }
}

__global__ void __launch_bounds__(256) k_residual(size_t V, int M, const float* mom, float* prev,
                                                  double* res, const int* skip, int g0, const int* win) {
    if (skip && *skip) return;
    const int g = g0 + blockIdx.y;
    if (win && (g < win[0] || g >= win[1])) return;      // retired group (whole block)
    double x[2] = {0.0, 0.0};
    // four voxels per thread and pass, their loads issued together
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t v0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v0 < V; v0 += 4 * stride) {
        float cur[4], old[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const size_t v = v0 + u * stride;
            cur[u] = v < V ? mom[((size_t)g * V + v) * M] : 0.0f;
            old[u] = v < V ? prev[(size_t)g * V + v] : 0.0f;
        }
        float dd = 0.0f, cc = 0.0f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const size_t v = v0 + u * stride;
            if (v < V) {
                const float d = cur[u] - old[u];
                dd = fmaf(d, d, dd);
                cc = fmaf(cur[u], cur[u], cc);
                prev[(size_t)g * V + v] = cur[u];
            }
        }
        x[0] += (double)dd;
        x[1] += (double)cc;
    }
    block_reduce_add<2>(x, res + 2 * g);
}

__global__ void __launch_bounds__(256) k_balance(size_t V, int G, int M, const uint8_t* mat,
                                                 const float* rho, const float* sigt, const float* src,
                                                 const float* mom, double vol, double* bal) {
    const int g = blockIdx.y;
    double x[2] = {0.0, 0.0};
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (size_t)gridDim.x * blockDim.x) {
        const double s00 = src[((size_t)g * V + v) * M];
        const double p00 = mom[((size_t)g * V + v) * M];
        const double st = (double)rho[v] * (double)sigt[mat[v] * G + g];
        x[0] += vol * s00;
        x[1] += vol * st * p00;
    }
    block_reduce_add<2>(x, bal + 2 * g);
}

__global__ void __launch_bounds__(256) k_dose(size_t V, int G, int M, const uint8_t* mat, const float* rho,
                                              const double* k, const float* phi_u, const float* mom,
                                              double* dose) {
    const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const int m = mat[v];
    double acc = 0.0;
    for (int g = 0; g < G; ++g) {
        const double phi = (double)phi_u[(size_t)g * V + v] + (double)mom[((size_t)g * V + v) * M];
        acc += k[m * G + g] * phi;
    }
    dose[v] = acc * (double)rho[v];
}

__global__ void __launch_bounds__(256) k_extract(size_t V, int G, int M, int which, const float* phi_u,
                                                 const float* mom, float* out) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= V * G) return;
    float x = 0.0f;
    if (which & 1) x += phi_u[t];
    if (which & 2) x += mom[t * M];
    out[t] = x;
}

template <class T>
__global__ void __launch_bounds__(256) k_zero(T* p, size_t n, const int* skip) {
    if (skip && *skip) return;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        p[t] = T(0);
}

// One thread: update every live instance's iteration count and residual
// (max over groups of sqrt(sum (dphi)^2 / sum phi^2)), retire it when the
// relative change is below its tolerance or the cap is reached, and stop
// the graph's while loop once all instances are retired.
__global__ void k_decide(LoopCtl* ctl, int n, cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0) return;
    bool all = true;
    for (int q = 0; q < n; ++q) {
        LoopCtl& c = ctl[q];
        if (c.done) continue;
        double eps = 0.0;
        for (int g = 0; g < c.G; ++g) {
            const double num = c.res[2 * g], den = c.res[2 * g + 1];
            const double e = den > 0.0 ? sqrt(num / den) : 0.0;
            eps = e > eps || e != e ? e : eps;
        }
        c.iters += 1;
        c.resid = eps;
        c.group_sweeps += c.use_window ? c.win[1] - c.win[0] : c.G;
        if (eps < c.tol || c.iters >= c.max_iters) {
            c.done = 1;
        } else {
            all = false;
            // shrink the active group window as the host loop does: a group whose
            // relative change is below tol and whose sources are all final is
            // final too (forward: leading groups, adjoint: trailing groups)
            if (c.use_window) {
                auto eps_of = [&](int g) {
                    const double num = c.res[2 * g], den = c.res[2 * g + 1];
                    return den > 0.0 ? sqrt(num / den) : 0.0;
                };
                if (!c.reverse)
                    while (c.win[0] < c.win[1] - 1 && eps_of(c.win[0]) < c.tol) ++c.win[0];
                else
                    while (c.win[1] - 1 > c.win[0] && eps_of(c.win[1] - 1) < c.tol) --c.win[1];
            }
        }
    }
    if (all) cudaGraphSetConditional(h, 0);
}

template <class T>
__global__ void __launch_bounds__(256) k_zero_window(T* p, size_t per_group, const int* win, const int* skip) {
    if (skip && *skip) return;
    const size_t beg = (size_t)win[0] * per_group, end = (size_t)win[1] * per_group;
    for (size_t t = beg + (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < end; t += (size_t)gridDim.x * blockDim.x)
        p[t] = T(0);
}

unsigned blocks_for(size_t n, int bs, unsigned cap = 0) {
    size_t b = (n + bs - 1) / bs;
    if (cap && b > cap) b = cap;
    return (unsigned)(b ? b : 1);
}

}  // namespace

// one resident wave of k_scatter_fast
template <int GMAX, bool TR, bool HAS_BASE, bool ISO = false>
cudaError_t launch_scatter_fast(const ScatterArgs& a, size_t smem, cudaStream_t s) {
    auto kern = k_scatter_fast<GMAX, TR, HAS_BASE, ISO>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int nb = 0, dev = 0, nsm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kScatterThreads, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const unsigned grid = blocks_for(a.V * a.M, kScatterThreads, (unsigned)(nsm * (nb > 0 ? nb : 1)));
    kern<<<grid, kScatterThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int GMAX>
cudaError_t launch_scatter_g(const ScatterArgs& a, cudaStream_t s) {
    const size_t tab_bytes = scatter_table_bytes<GMAX>(a);
    const int staged = tab_bytes <= kScatterTableSmem ? 1 : 0;
    const size_t smem = staged ? tab_bytes : 0;
    const size_t fast_bytes = scatter_fast_table_bytes<GMAX>(a);
    const bool fast = fast_bytes <= kScatterTableSmem && a.phi && !a.iso_field && a.V * a.M < ((size_t)1 << 31);
    if (fast && a.iso && !a.transpose && !a.base)
        return launch_scatter_fast<GMAX, false, false, true>(a, fast_bytes, s);
    if (fast && !a.iso) {
        if (a.transpose)
            return a.base ? launch_scatter_fast<GMAX, true, true>(a, fast_bytes, s)
                          : launch_scatter_fast<GMAX, true, false>(a, fast_bytes, s);
        return a.base ? launch_scatter_fast<GMAX, false, true>(a, fast_bytes, s)
                      : launch_scatter_fast<GMAX, false, false>(a, fast_bytes, s);
    }
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_scatter<GMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_scatter<GMAX><<<blocks_for(a.V * a.M, kScatterThreads, 152 * 8), kScatterThreads, smem, s>>>(a, staged);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const ScatterArgs& a, cudaStream_t s) {
    if (a.G <= 8) return launch_scatter_g<8>(a, s);
    if (a.G <= 16) return launch_scatter_g<16>(a, s);
    if (a.G <= 20) return launch_scatter_g<20>(a, s);
    if (a.G <= 24) return launch_scatter_g<24>(a, s);
    if (a.G <= 32) return launch_scatter_g<32>(a, s);
    if (a.G <= 64) return launch_scatter_g<64>(a, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_residual(size_t V, int G, int M, const float* mom, float* prev, double* res,
                            cudaStream_t s, const int* skip, int g0, int gcount, const int* win) {
    // sixteen voxels per thread (four passes)
    dim3 grid(blocks_for((V + 15) / 16, 256, 152), gcount < 0 ? G : gcount);
    k_residual<<<grid, 256, 0, s>>>(V, M, mom, prev, res, skip, g0, win);
    return cudaGetLastError();
}

cudaError_t launch_total_xs(size_t V, int G, const uint8_t* mat, const float* rho, const float* sigt, float* out,
                            cudaStream_t s) {
    k_total_xs<<<blocks_for(V, 256, 152 * 16), 256, 0, s>>>(V, G, mat, rho, sigt, out);
    return cudaGetLastError();
}

cudaError_t launch_zero_window(float* p, size_t per_group, int G, const int* win, const int* skip, cudaStream_t s) {
    k_zero_window<float><<<blocks_for((per_group * G + 3) / 4, 256, 152 * 16), 256, 0, s>>>(p, per_group, win, skip);
    return cudaGetLastError();
}

cudaError_t launch_zero_window(double* p, size_t per_group, int G, const int* win, const int* skip, cudaStream_t s) {
    k_zero_window<double><<<blocks_for((per_group * G + 3) / 4, 256, 152 * 16), 256, 0, s>>>(p, per_group, win, skip);
    return cudaGetLastError();
}

cudaError_t launch_zero(float* p, size_t n, const int* skip, cudaStream_t s) {
    k_zero<float><<<blocks_for((n + 3) / 4, 256, 152 * 16), 256, 0, s>>>(p, n, skip);
    return cudaGetLastError();
}

cudaError_t launch_zero(double* p, size_t n, const int* skip, cudaStream_t s) {
    k_zero<double><<<blocks_for((n + 3) / 4, 256, 152 * 16), 256, 0, s>>>(p, n, skip);
    return cudaGetLastError();
}

cudaError_t launch_decide(LoopCtl* ctl, int n, unsigned long long cond_handle, cudaStream_t s) {
    k_decide<<<1, 32, 0, s>>>(ctl, n, (cudaGraphConditionalHandle)cond_handle);
    return cudaGetLastError();
}

cudaError_t launch_balance(size_t V, int G, int M, const uint8_t* mat, const float* rho, const float* sigt,
                           const float* src, const float* mom, double vol, double* bal, cudaStream_t s) {
    dim3 grid(blocks_for(V, 256, 296), G);
    k_balance<<<grid, 256, 0, s>>>(V, G, M, mat, rho, sigt, src, mom, vol, bal);
    return cudaGetLastError();
}

cudaError_t launch_dose(size_t V, int G, int M, const uint8_t* mat, const float* rho, const double* k,
                        const float* phi_u, const float* mom, double* dose, cudaStream_t s) {
    k_dose<<<blocks_for(V, 256), 256, 0, s>>>(V, G, M, mat, rho, k, phi_u, mom, dose);
    return cudaGetLastError();
}

cudaError_t launch_extract(size_t V, int G, int M, int which, const float* phi_u, const float* mom,
                           float* out, cudaStream_t s) {
    k_extract<<<blocks_for(V * G, 256), 256, 0, s>>>(V, G, M, which, phi_u, mom, out);
    return cudaGetLastError();
}

}  // namespace doctors
