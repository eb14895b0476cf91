// Chained octant wavefront sweep: the step-differenced cell update, tile
// stages and face buffers of k_sweep, with one change of schedule.
//
// In k_sweep a CTA owns one task (tile, octant, direction block, group) and
// its hyperplane pipeline fills and drains for every task: with a tx x ty
// tile the thread of column (li, lj) starts li + lj steps late, so a CTA runs
// nz + tx + ty - 2 steps for nz steps of work per thread.  Here a launch has
// at most as many CTAs as fit on the GPU at once, and each CTA runs a chain
// of tasks of the stage back to back: the thread of column (li, lj) works at
// step h on position u = h - li - lj of the concatenated z columns of its
// chain (task u / nz, plane u % nz).  Its upwind x and y neighbours worked on
// the same position one step earlier, so the double-buffered hyperplane needs
// no drain between tasks and the pipeline fills once per launch.  Tasks of
// one stage are independent, so CTAs never wait on one another.
//
// Incoming face fluxes reach the tile's first row and column through a halo
// of the plane buffers: the edge threads copy the value of their next cell
// with cp.async one step ahead (zero on the mesh boundary), so every upwind
// read is the same shared-memory load, without a branch.
//
// CT = true (a CTA sweeps whole octants of S2..S8): the first octant's
// moment-to-direction and direction-to-moment rows come from this unit's
// constant bank (c_Mop1, c_Dop1) and its step coefficients and weights from a
// kernel parameter (ChainDirTable), all read at compile-time offsets, so the
// transforms issue no shared-memory loads.  Another octant's directions are the first octant's
// reflected, which multiplies R_lm by -1 for every reflected axis in which it
// is odd: the kernel applies those signs to the source moments before the
// transform and to the accumulated moments after it.  CT = false: the rows
// of every chained task are staged in shared memory.
#pragma once

#include <type_traits>

#include "sweep_impl.cuh"

namespace doctors {

struct ChainNoTable {
    int unused;
};

// First-octant transform rows of the S2, S4, S6 and S8 sets (the sets a CTA
// can sweep as whole octants), natural (l, m) order: (2l+1)/(4 pi) R_lm for
// moments -> direction and w R_lm for direction -> moments.  They depend only
// on N, so they live in this translation unit's constant bank next to c_R,
// and the kernel reads them at compile-time offsets (row base fixed by AB).
constexpr int kChainRows = 1 + 3 + 6 + 10;
__constant__ float c_Mop1[kChainRows * 16];
__constant__ float c_Dop1[kChainRows * 16];

__host__ __device__ constexpr int chain_row_base(int ab) { return ab == 1 ? 0 : ab == 3 ? 1 : ab == 6 ? 4 : 10; }

// R, w: the concatenated direction tables (all octants of S2, S4, S6, S8,
// S12, S16, natural order) as uploaded to c_R and c_w.  Internal linkage:
// every translation unit including this header must fill its own copy of
// the constant arrays (a shared inline definition would fill only one).
static cudaError_t upload_chain_tables(const float* R, const float* w) {
    const int first_row[4] = {0, 8, 32, 80};     // first direction of S2, S4, S6, S8
    const int a8[4] = {1, 3, 6, 10};
    float mop[kChainRows * 16], dop[kChainRows * 16];
    int row = 0;
    for (int set = 0; set < 4; ++set)
        for (int j = 0; j < a8[set]; ++j, ++row)
            for (int lm = 0; lm < 16; ++lm) {
                const double r = R[(first_row[set] + j) * 16 + lm];
                mop[row * 16 + lm] = (float)((2 * degree_of_lm(lm) + 1) / (4.0 * 3.14159265358979323846) * r);
                dop[row * 16 + lm] = (float)((double)w[first_row[set] + j] * r);
            }
    cudaError_t e = cudaMemcpyToSymbol(c_Mop1, mop, sizeof(mop));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_Dop1, dop, sizeof(dop));
    return e;
}

// sign of R_lm (storage position m) under the reflections (fx, fy, fz) = +-1
template <int M>
__device__ __forceinline__ float octant_sign(int m, float fx, float fy, float fz) {
    const int lm = lm_of_pos(m, M);
    float r = 1.0f;
    if ((kOddX >> lm) & 1u) r *= fx;
    if ((kOddY >> lm) & 1u) r *= fy;
    if ((kOddZ >> lm) & 1u) r *= fz;
    return r;
}

__device__ __forceinline__ void cp_async_f32(float* dst_smem, const float* src_gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(dst_smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src_gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// task t of a stage with `ntiles` tiles: tile fastest, then direction block,
// octant, group
__device__ __forceinline__ void chain_decode(int t, int ntiles, int nab, int& ti, int& blk, int& o, int& gi) {
    ti = t % ntiles;
    int r = t / ntiles;
    blk = r % nab;
    r /= nab;
    o = r & 7;
    gi = r >> 3;
}

// field f of the direction table at index i (CT only; i and f compile-time
// in the unrolled loops, so this is a constant-bank operand)
template <bool CT, typename T>
__device__ __forceinline__ float dt_at(const T& dt, int f, int i) {
    if constexpr (CT) {
        switch (f) {
            case 2: return dt.cx[i];
            case 3: return dt.cy[i];
            case 4: return dt.cz[i];
            case 5: return dt.csum[i];
            case 6: return dt.lx[i];
            case 7: return dt.ly[i];
            case 8: return dt.lz[i];
            default: return dt.w[i];
        }
    } else {
        return 0.0f;
    }
}

template <int AB, int M, int MODE, bool CT>
__global__ void __launch_bounds__(256, 2)
    k_sweep_chain(const SweepArgs a, const std::conditional_t<CT, ChainDirTable, ChainNoTable> dt) {
    extern __shared__ float4 sm4[];
    if (a.skip && *a.skip) return;         // retired instance of a batched loop
    const int a_lo = max(0, a.stage - (a.nty - 1));
    const int a_hi = min(a.stage, a.ntx - 1);
    const int ntiles = a_hi - a_lo + 1;
    const int ntasks = ntiles * 8 * a.nab * a.gcount;
    const int grid = (int)gridDim.x;
    const int cmax = CT ? 0 : (ntasks + grid - 1) / grid;   // staged table rows (CT: none)
    const int nchain = (ntasks - (int)blockIdx.x + grid - 1) / grid;   // tasks of this CTA (grid <= ntasks)
    constexpr int RS = AB | 1;                  // floats per column record (odd: conflict-free)
    const int PX = chain_px(a.tx);              // row pitch in columns (even), halo column at 0
    const int P = PX * (a.ty + 1);              // columns per plane, halo row at 0

    float4* coef_s = sm4;                       // [cmax][AB]: cx, cy, cz, cx+cy+cz
    float4* R_s = coef_s + cmax * AB;           // [cmax][AB][4]: R_lm, 16 per direction
    double* leak_s = reinterpret_cast<double*>(R_s + 4 * cmax * AB);   // [gcount]
    float* buf = reinterpret_cast<float*>(leak_s + a.gcount);        // [2][P][RS]
    float* w_s = buf + 2 * P * RS;              // [cmax][AB]
    float* sigt_s = w_s + cmax * AB;            // [gcount][nmat]

    for (int e = threadIdx.x; e < (CT ? 0 : nchain * AB); e += blockDim.x) {
        const int cc = e / AB, q = e % AB;
        int ti, blk, o, gi;
        chain_decode((int)blockIdx.x + cc * grid, ntiles, a.nab, ti, blk, o, gi);
        const int n = (a.reverse ? (o ^ 7) : o) * a.A8 + blk * AB + q;   // adjoint: along -Omega_n
        const float* cf = a.coef + (size_t)n * 8;
        coef_s[e] = make_float4(cf[0], cf[1], cf[2], cf[3]);
        w_s[e] = c_w[a.table_base + n];
        const float* r = c_R + (size_t)(a.table_base + n) * 16;
#pragma unroll
        for (int p4 = 0; p4 < 4; ++p4)
            R_s[4 * e + p4] = make_float4(r[lm_of_pos(4 * p4, M)], r[lm_of_pos(4 * p4 + 1, M)],
                                          r[lm_of_pos(4 * p4 + 2, M)], r[lm_of_pos(4 * p4 + 3, M)]);
    }
    for (int e = threadIdx.x; e < a.gcount * a.nmat; e += blockDim.x)
        sigt_s[e] = a.sigt[(e % a.nmat) * a.G + a.g0 + e / a.nmat];
    for (int e = threadIdx.x; e < a.gcount; e += blockDim.x) leak_s[e] = 0.0;
    for (int e = threadIdx.x; e < 2 * P * RS; e += blockDim.x) buf[e] = 0.0f;
    __syncthreads();

    // threads own the tile's columns in diagonal order (li + lj ascending):
    // the columns active at a step are a contiguous range of threads
    const int tid = threadIdx.x;
    int li = 0, lj = 0;
    {
        int base = 0;
        for (int dd = 0; dd <= a.tx + a.ty - 2; ++dd) {
            const int lo = dd > a.ty - 1 ? dd - (a.ty - 1) : 0;
            const int hi = dd < a.tx - 1 ? dd : a.tx - 1;
            const int cnt = hi - lo + 1;
            if (tid < base + cnt) {
                li = lo + (tid - base);
                lj = dd - li;
                break;
            }
            base += cnt;
        }
    }
    const int d = li + lj;
    const int cs = (lj + 1) * PX + li + 1;      // this column's slot in the padded planes
    const int xs = (cs - 1) * RS, ys = (cs - PX) * RS, os = cs * RS;   // upwind x, upwind y, own record
    const size_t V = (size_t)a.nx * a.ny * a.nz;
    const size_t nxy = (size_t)a.nx * a.ny;
    const size_t xf_stride = (size_t)(a.ntx > 1 ? a.ntx - 1 : 0) * a.ny * a.nz;
    const size_t yf_stride = (size_t)(a.nty > 1 ? a.nty - 1 : 0) * a.nx * a.nz;
    const size_t xo_q = (size_t)a.G * xf_stride, yo_q = (size_t)a.G * yf_stride;

    // state of the task this thread works on (or starts next)
    int gi = 0, sz = 1, nb = 0, tab = 0;
    float fx = 1.0f, fy = 1.0f, fz = 1.0f;      // reflections of the task's directions (CT)
    size_t gV = 0, vcol = 0;
    bool col = false, xout = false, yout = false, xleak = false, yleak = false;
    float* xo = nullptr;
    float* yo = nullptr;
    const float* xi = nullptr;
    const float* yi = nullptr;
    auto begin_task = [&](int cc) {
        int ti, blk, o;
        chain_decode((int)blockIdx.x + cc * grid, ntiles, a.nab, ti, blk, o, gi);
        const int g = a.g0 + gi;
        const int at = a_lo + ti, bt = a.stage - at;
        const int sx = (o & 1) ? -1 : 1, sy = (o & 2) ? -1 : 1;
        sz = (o & 4) ? -1 : 1;
        const int oe = a.reverse ? (o ^ 7) : o;          // octant of the directions
        nb = oe * a.A8 + blk * AB;
        tab = cc * AB;
        fx = (oe & 1) ? -1.0f : 1.0f;
        fy = (oe & 2) ? -1.0f : 1.0f;
        fz = (oe & 4) ? -1.0f : 1.0f;
        const int ir = at * a.tx + li, jr = bt * a.ty + lj;
        col = ir < a.nx && jr < a.ny;
        const int i = sx > 0 ? ir : a.nx - 1 - ir;
        const int j = sy > 0 ? jr : a.ny - 1 - jr;
        vcol = (size_t)j * a.nx + i;
        gV = (size_t)g * V;
        xout = li == a.tx - 1 && at < a.ntx - 1;
        yout = lj == a.ty - 1 && bt < a.nty - 1;
        xleak = ir == a.nx - 1;
        yleak = jr == a.ny - 1;
        const size_t fq = ((size_t)o * a.A8 + blk * AB) * a.G + g;
        xo = a.xface + fq * xf_stride + ((size_t)at * a.ny + jr) * a.nz;
        yo = a.yface + fq * yf_stride + ((size_t)bt * a.nx + ir) * a.nz;
        xi = at > 0 ? a.xface + fq * xf_stride + ((size_t)(at - 1) * a.ny + jr) * a.nz : nullptr;
        yi = bt > 0 ? a.yface + fq * yf_stride + ((size_t)(bt - 1) * a.nx + ir) * a.nz : nullptr;
    };
    // incoming face values of plane kn of the current task into the halo of
    // hyperplane buffer `pl` (read by this thread one step later)
    auto fill_halo = [&](int pl, int kn) {
        if (!col) return;
        float* hb = buf + pl * P * RS;
        if (li == 0) {
            if (xi) {
#pragma unroll
                for (int q = 0; q < AB; ++q) cp_async_f32(hb + xs + q, xi + q * xo_q + kn);
            } else {
#pragma unroll
                for (int q = 0; q < AB; ++q) hb[xs + q] = 0.0f;
            }
        }
        if (lj == 0) {
            if (yi) {
#pragma unroll
                for (int q = 0; q < AB; ++q) cp_async_f32(hb + ys + q, yi + q * yo_q + kn);
            } else {
#pragma unroll
                for (int q = 0; q < AB; ++q) hb[ys + q] = 0.0f;
            }
        }
    };
    // source moments and total cross section of plane kn, one step ahead
    float sn[M];
#pragma unroll
    for (int m = 0; m < M; ++m) sn[m] = 0.0f;
    float rho_n = 0.0f;       // density and material of the prefetched cell: the cross
    int mat_n = 0;            // section is looked up when the cell is swept, not at the load
    auto prefetch = [&](int kn) {
        if (col) {
            const int k = sz > 0 ? kn : a.nz - 1 - kn;
            const size_t v = (size_t)k * nxy + vcol;
            load_moments<M>(a.src + (gV + v) * M, sn);
            rho_n = __ldg(a.rho + v);
            mat_n = __ldg(a.mat + v);
        }
    };

    int c = 0, kr = 0;
    begin_task(0);
    prefetch(0);
    if (d == 0) fill_halo(1, 0);                // read at step 0
    cp_async_wait_all();
    __syncthreads();

    float zc[AB];
#pragma unroll
    for (int q = 0; q < AB; ++q) zc[q] = 0.0f;
    float lk = 0.0f;

    const int hend = a.tx + a.ty - 2 + nchain * a.nz;
    for (int h = 0; h < hend; ++h) {
        const int cb = h & 1, pb = cb ^ 1;
        if (h + 1 == d) fill_halo(cb, 0);      // this thread's first cell comes next step
        if (h >= d && c < nchain) {
            const bool last = kr == a.nz - 1;
            if (col) {
                float s[M];
                // CT: reflection signs; otherwise (2l+1)/(4 pi) folded into the source moments
#pragma unroll
                for (int m = 0; m < M; ++m)
                    s[m] = CT ? sn[m] * octant_sign<M>(m, fx, fy, fz)
                              : sn[m] * ((2 * degree_of_lm(lm_of_pos(m, M)) + 1) * 0.07957747154594767f);
                const float sig = rho_n * sigt_s[gi * a.nmat + mat_n];
                const int k = sz > 0 ? kr : a.nz - 1 - kr;
                const size_t v = (size_t)k * nxy + vcol;
                const size_t mo = (gV + v) * M;
                if (!last) {
                    fill_halo(cb, kr + 1);
                    prefetch(kr + 1);
                }
                // moments -> directions: AB independent dot products
                float psi[AB];
#pragma unroll
                for (int q = 0; q < AB; ++q) {
                    float t0 = 0.0f, t1 = 0.0f, t2 = 0.0f, t3 = 0.0f;
#pragma unroll
                    for (int m = 0; m < M; m += 4) {
                        constexpr int rb = chain_row_base(AB) * 16;
                        const float4 R = CT ? make_float4(c_Mop1[rb + q * 16 + lm_of_pos(m, M)],
                                                          c_Mop1[rb + q * 16 + lm_of_pos(m + 1, M)],
                                                          c_Mop1[rb + q * 16 + lm_of_pos(m + 2, M)],
                                                          c_Mop1[rb + q * 16 + lm_of_pos(m + 3, M)])
                                            : R_s[4 * (tab + q) + m / 4];
                        t0 = fmaf(R.x, s[m], t0);
                        if (m + 1 < M) t1 = fmaf(R.y, s[m + 1], t1);
                        if (m + 2 < M) t2 = fmaf(R.z, s[m + 2], t2);
                        if (m + 3 < M) t3 = fmaf(R.w, s[m + 3], t3);
                    }
                    psi[q] = (t0 + t1) + (t2 + t3);
                }
                // step-differenced cell solve per direction (branch-free
                // upwind reads: the halo holds the incoming face values)
                const float* pv = buf + pb * P * RS;
                float* cv = buf + cb * P * RS;
#pragma unroll
                for (int q = 0; q < AB; ++q) {
                    const float px = pv[xs + q];
                    const float py = pv[ys + q];
                    const float4 cq = CT ? make_float4(dt_at<CT>(dt, 2, q), dt_at<CT>(dt, 3, q), dt_at<CT>(dt, 4, q),
                                                       dt_at<CT>(dt, 5, q))
                                         : coef_s[tab + q];
                    const float num = fmaf(cq.z, zc[q], fmaf(cq.y, py, fmaf(cq.x, px, psi[q])));
                    psi[q] = num * rcp_approx(sig + cq.w);
                    cv[os + q] = psi[q];
                    zc[q] = psi[q];
                }
                if constexpr (MODE == 1) psi_store_run<AB>(a.psi + ((size_t)(a.g0 + gi) * V + v) * a.A + nb, psi);
                if constexpr (MODE == 2) {
                    float wpsi[AB];
#pragma unroll
                    for (int q = 0; q < AB; ++q) wpsi[q] = (CT ? dt_at<CT>(dt, 9, q) : w_s[tab + q]) * psi[q];
                    red_add_f32(a.prod + gV + v,
                                psi_product_run<AB>(a.psi + ((size_t)(a.g0 + gi) * V + v) * a.A + nb, wpsi));
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
                if (xleak || yleak || last) {
#pragma unroll
                    for (int q = 0; q < AB; ++q) {
                        float f = 0.0f;
                        if constexpr (CT) {
                            if (xleak) f += dt_at<CT>(dt, 6, q);
                            if (yleak) f += dt_at<CT>(dt, 7, q);
                            if (last) f += dt_at<CT>(dt, 8, q);
                        } else {
                            const float* cf = a.coef + (size_t)(nb + q) * 8;
                            if (xleak) f += __ldg(cf + 4);
                            if (yleak) f += __ldg(cf + 5);
                            if (last) f += __ldg(cf + 6);
                        }
                        lk = fmaf(f, psi[q], lk);
                    }
                }
                // directions -> moments (Eq. 3 for lm = 00)
                float acc[M];
#pragma unroll
                for (int m = 0; m < M; ++m) acc[m] = 0.0f;
#pragma unroll
                for (int q = 0; q < AB; ++q) {
                    // CT: the table holds w R_lm
                    const float wp = CT ? psi[q] : w_s[tab + q] * psi[q];
#pragma unroll
                    for (int m = 0; m < M; m += 4) {
                        constexpr int rb = chain_row_base(AB) * 16;
                        const float4 R = CT ? make_float4(c_Dop1[rb + q * 16 + lm_of_pos(m, M)],
                                                          c_Dop1[rb + q * 16 + lm_of_pos(m + 1, M)],
                                                          c_Dop1[rb + q * 16 + lm_of_pos(m + 2, M)],
                                                          c_Dop1[rb + q * 16 + lm_of_pos(m + 3, M)])
                                            : R_s[4 * (tab + q) + m / 4];
                        acc[m] = fmaf(R.x, wp, acc[m]);
                        if (m + 1 < M) acc[m + 1] = fmaf(R.y, wp, acc[m + 1]);
                        if (m + 2 < M) acc[m + 2] = fmaf(R.z, wp, acc[m + 2]);
                        if (m + 3 < M) acc[m + 3] = fmaf(R.w, wp, acc[m + 3]);
                    }
                }
                if constexpr (CT) {
#pragma unroll
                    for (int m = 0; m < M; ++m) acc[m] *= octant_sign<M>(m, fx, fy, fz);
                }
                add_moments<M>(a.mom + mo, acc);
            }
            if (last) {                          // task done: next task of the chain
                if (lk != 0.0f) atomicAdd(leak_s + gi, (double)lk);
                lk = 0.0f;
#pragma unroll
                for (int q = 0; q < AB; ++q) zc[q] = 0.0f;
                kr = 0;
                ++c;
                if (c < nchain) {
                    begin_task(c);
                    fill_halo(cb, 0);
                    prefetch(0);
                }
            } else {
                ++kr;
            }
        }
        cp_async_wait_all();
        __syncthreads();
    }
    for (int e = threadIdx.x; e < a.gcount; e += blockDim.x)
        if (leak_s[e] != 0.0) atomicAdd(a.leak + a.g0 + e, leak_s[e]);
}

// CTAs of k_sweep_chain<AB, M, 0, CT> resident per SM at this shared-memory size
template <int M>
int sweep_chain_blocks_per_sm(int ab, bool ct, int threads, size_t smem) {
    int b = 0;
    cudaError_t e = cudaErrorInvalidValue;
    auto query = [&](auto kern) {
        e = smem > 48 * 1024 ? cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                             : cudaSuccess;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, smem);
    };
    if (ct) {
        switch (ab) {
            case 1: query(k_sweep_chain<1, M, 0, true>); break;
            case 3: query(k_sweep_chain<3, M, 0, true>); break;
            case 6: query(k_sweep_chain<6, M, 0, true>); break;
            case 10: query(k_sweep_chain<10, M, 0, true>); break;
            default: break;
        }
    } else {
        switch (ab) {
            case 1: query(k_sweep_chain<1, M, 0, false>); break;
            case 2: query(k_sweep_chain<2, M, 0, false>); break;
            case 3: query(k_sweep_chain<3, M, 0, false>); break;
            case 4: query(k_sweep_chain<4, M, 0, false>); break;
            case 5: query(k_sweep_chain<5, M, 0, false>); break;
            case 6: query(k_sweep_chain<6, M, 0, false>); break;
            case 7: query(k_sweep_chain<7, M, 0, false>); break;
            case 9: query(k_sweep_chain<9, M, 0, false>); break;
            case 10: query(k_sweep_chain<10, M, 0, false>); break;
            case 12: query(k_sweep_chain<12, M, 0, false>); break;
            default: break;
        }
    }
    return e == cudaSuccess ? b : 0;
}

template <int M, int MODE>
cudaError_t launch_sweep_chain_m(const SweepArgs& a, cudaStream_t s) {
    const int a_lo = a.stage - (a.nty - 1) > 0 ? a.stage - (a.nty - 1) : 0;
    const int a_hi = a.stage < a.ntx - 1 ? a.stage : a.ntx - 1;
    const int ntiles = a_hi - a_lo + 1;
    if (ntiles <= 0 || a.gcount <= 0) return cudaSuccess;
    const int ntasks = ntiles * 8 * a.nab * a.gcount;
    const int grid = ntasks < a.chain_slots ? ntasks : a.chain_slots;
    const bool ct = a.nab == 1 && chain_const_table_ab(a.ab) && a.dir_table != nullptr;
    const int cmax = ct ? 0 : (ntasks + grid - 1) / grid;
    const int T = a.tx * a.ty;
    const size_t smem = sweep_chain_smem_bytes(a.ab, a.tx, a.ty, cmax, a.gcount, a.nmat);
    cudaError_t e = cudaSuccess;
    auto launch = [&](auto kern, const auto& table) {
        if (smem > 48 * 1024) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) kern<<<grid, T, smem, s>>>(a, table);
    };
    if (ct) {
        const ChainDirTable& dt = *a.dir_table;
        switch (a.ab) {
            case 1: launch(k_sweep_chain<1, M, MODE, true>, dt); break;
            case 3: launch(k_sweep_chain<3, M, MODE, true>, dt); break;
            case 6: launch(k_sweep_chain<6, M, MODE, true>, dt); break;
            case 10: launch(k_sweep_chain<10, M, MODE, true>, dt); break;
            default: return cudaErrorInvalidValue;
        }
    } else {
        const ChainNoTable nt{0};
        switch (a.ab) {
            case 1: launch(k_sweep_chain<1, M, MODE, false>, nt); break;
            case 2: launch(k_sweep_chain<2, M, MODE, false>, nt); break;
            case 3: launch(k_sweep_chain<3, M, MODE, false>, nt); break;
            case 4: launch(k_sweep_chain<4, M, MODE, false>, nt); break;
            case 5: launch(k_sweep_chain<5, M, MODE, false>, nt); break;
            case 6: launch(k_sweep_chain<6, M, MODE, false>, nt); break;
            case 7: launch(k_sweep_chain<7, M, MODE, false>, nt); break;
            case 9: launch(k_sweep_chain<9, M, MODE, false>, nt); break;
            case 10: launch(k_sweep_chain<10, M, MODE, false>, nt); break;
            case 12: launch(k_sweep_chain<12, M, MODE, false>, nt); break;
            default: return cudaErrorInvalidValue;
        }
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace doctors
