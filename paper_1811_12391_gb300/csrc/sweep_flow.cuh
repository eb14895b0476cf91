// Dataflow octant wavefront sweep: the step-differenced cell update of
// k_sweep_chain (whole octants per CTA; the first octant's direction rows,
// coefficients and moment tables are kernel parameters, read through the
// constant bank at compile-time offsets) with the tile stages replaced by a
// task queue in one launch.  S12 and S16 run as whole octants (21 and 36
// directions per cell step); S16 also as three launches, one per block of
// 12 directions of every octant, each with that block's table.
//
// The tasks (tile, octant, group) are numbered stage by stage (the tile
// diagonal of the octant's reflected tile grid).  Each CTA takes the next
// task from a global counter, sweeps it through its hyperplane pipeline and
// takes another, until the queue is empty; there is one launch per sweep and
// no barrier between stages.  A task needs the fluxes leaving its upstream
// x and y tiles, which other CTAs may still be producing: every face record
// (the AB fluxes of one column face and plane) starts the sweep as NaN, the
// producer overwrites it with the fluxes, and the consumer's edge thread
// fetches it one step ahead with cp.async (L2, not L1), re-fetching while any
// value is still NaN.  Having used a record, the consumer writes NaN back, so
// the face buffers are ready for the next sweep without a reset pass.
//
// Waiting is bounded and cannot deadlock: a CTA holds one task at a time and
// waits only on tasks with smaller numbers, which are held by running CTAs
// (a task is taken only by a running CTA) and themselves wait only on smaller
// numbers.  A wait that exceeds kFlowSpinLimit polls records the failure in
// the problem's flag word, uses zero fluxes and goes on (later waits of the
// sweep then give up at once); the host turns the flag into
// DOCTORS_ERR_TIMEOUT and resets the buffers.
#pragma once

#include <algorithm>

#include "sweep_chain.cuh"

namespace doctors {

constexpr int kFlowSpinLimit = 1 << 18;

// floats per face record: AB fluxes padded to a multiple of 4 (16-byte copies)
__host__ __device__ constexpr int flow_abp(int ab) { return (ab + 3) & ~3; }

__device__ __forceinline__ void cp_async_cg16(void* dst_smem, const void* src_gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(dst_smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src_gmem) : "memory");
}

// tiles of stage s of an ntx x nty tile grid
__device__ __forceinline__ int flow_stage_tiles(int s, int ntx, int nty) {
    const int lo = s - (nty - 1) > 0 ? s - (nty - 1) : 0;
    const int hi = s < ntx - 1 ? s : ntx - 1;
    return hi - lo + 1;
}

// SPLIT = true: the transforms run in separate passes (k_split_m2d before,
// k_split_d2m after); the sweep reads each cell's angular-source record
// a.qang and writes its angular-fluence record a.pang, with no moments and
// no reductions (mode 0 only).
//
// HW = true: one more warp per CTA, the face warp, takes over the incoming
// face records: it fetches them ahead, waits until each is complete, moves
// it into the halo of the plane buffers and hands the record back as NaN.
// The column threads then run no face code at all (in the plain kernel the
// threads of the tile's first row and column do it, and their warps carry
// that code at every step).  Mode 0.
//
// DD = true: diamond differencing (no negative-flux fixup).  The direction
// table then holds 2 c_x, 2 c_y, 2 c_z and their sum, so the cell solve
// (q + sum 2 c psi_in) / (sigma + 2 sum c) is the step formula's; each face
// leaves with 2 psi - psi_in.  The x-going and y-going face fluxes of a cell
// differ, so they are kept in two planes (x: buf, y: bufy), and the face
// records and the leakage carry the face fluxes, not the cell flux.
template <int AB, int M, int MODE, bool SPLIT = false, bool DD = false, bool HW = false>
__global__ void __launch_bounds__(HW ? 288 : 256, AB > 12 ? 1 : ((!SPLIT && M % 4 == 0) ? 3 : 2))
    k_sweep_flow(const SweepArgs a, const ChainDirTable dt) {
    static_assert(!SPLIT || MODE == 0, "split transforms sweep in mode 0 only");
    static_assert(!DD || !SPLIT, "diamond differencing in the fused kernel only");
    static_assert(!HW || MODE == 0, "the face warp serves the mode-0 sweep");
    constexpr int ABP = flow_abp(AB);
    constexpr int RS = AB | 1;                // a column's record of fluxes (odd length)
    // Total cross section of a cell: in the plain and split step-differenced
    // kernels one load from the per-cell table dt.sig (rho sigma_t of every cell
    // and group, formed when the materials are set: one memory request per cell
    // step fewer, 5-7 % per sweep); the face-warp and diamond kernels keep the
    // density and material loads and the staged table (with the table load they
    // spill: the face warp's 72 registers at three 288-thread CTAs per SM)
    constexpr bool XS = !HW && !DD;
    // pipeline depths: face records are fetched PD steps before the step
    // that uses them, source values PDS steps (the split sweep's steps are
    // short, so one step does not cover the memory latency)
    constexpr int PD = 2;                     // face records
    constexpr int PDS = SPLIT ? 2 : 1;        // source values (registers)
    // fused kernel with moments in 16-byte quarters: the next cell's source
    // moments go to shared memory by cp.async (no registers held for them
    // across the step)
    constexpr bool SMEMPF = !SPLIT && M % 4 == 0;
    extern __shared__ float4 sm4[];
    if (a.skip && *a.skip) return;          // retired instance of a batched loop
    const int PX = chain_px(a.tx);
    const int P = PX * (a.ty + 1);
    float4* momst = sm4;                                      // [2][column threads][4] prefetched source moments
    const int T = a.tx * a.ty;                                // column threads
    float4* landx = momst + 2 * T * 4;                        // [PD][ty][ABP/4] fetched x-face records
    float4* landy = landx + PD * a.ty * (ABP / 4);            // [PD][tx][ABP/4] fetched y-face records
    double* leak_s = reinterpret_cast<double*>(landy + PD * a.tx * (ABP / 4));   // [gcount]
    float* buf = reinterpret_cast<float*>(leak_s + a.gcount);              // [2][P][RS]
    float* bufy = DD ? buf + 2 * P * RS : buf;                // [2][P][RS] y-going faces (diamond)
    float* sigt_s = buf + (DD ? 4 : 2) * P * RS;              // [gcount][nmat]
    int* task_s = reinterpret_cast<int*>(sigt_s + a.gcount * a.nmat);

    // groups swept: [g0, g0 + gcount), from device memory in a batched
    // graph loop (a.g0, a.gcount then size the buffers only)
    int g0 = a.g0, gcount = a.gcount;
    if (a.win) {
        g0 = a.win[0];
        gcount = a.win[1] - a.win[0];
    }
    if constexpr (!XS)   // rho sigma_t formed from the staged table
        for (int e = threadIdx.x; e < gcount * a.nmat; e += blockDim.x)
            sigt_s[e] = a.sigt[(e % a.nmat) * a.G + g0 + e / a.nmat];
    for (int e = threadIdx.x; e < gcount; e += blockDim.x) leak_s[e] = 0.0;
    for (int e = threadIdx.x; e < (DD ? 4 : 2) * P * RS; e += blockDim.x) buf[e] = 0.0f;

    // threads own the tile's columns in diagonal order (li + lj ascending)
    const int tid = threadIdx.x;
    // with the face warp: the warps after the column threads' warps
    const int ncw = (T + 31) / 32;
    const bool fw = HW && tid >= ncw * 32;
    const bool colthread = tid < T;
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
    const int cs = (lj + 1) * PX + li + 1;
    const int xs = (cs - 1) * RS, ys = (cs - PX) * RS, os = cs * RS;
    const size_t V = (size_t)a.nx * a.ny * a.nz;
    const size_t nxy = (size_t)a.nx * a.ny;
    const int nst = a.ntx + a.nty - 1;
    const int ntxf = a.ntx > 1 ? a.ntx - 1 : 0, ntyf = a.nty > 1 ? a.nty - 1 : 0;
    const size_t xslab = (size_t)a.ny * a.nz * ABP, yslab = (size_t)a.nx * a.nz * ABP;
    int ntasks = 0;
    for (int s = 0; s < nst; ++s) ntasks += flow_stage_tiles(s, a.ntx, a.nty) * 8 * gcount;
    // landing slot of the x (y) record of row (column) i used at step st; this thread's
    auto land_xr = [&](int st, int row) { return landx + ((st & (PD - 1)) * a.ty + row) * (ABP / 4); };
    auto land_yr = [&](int st, int cl) { return landy + ((st & (PD - 1)) * a.tx + cl) * (ABP / 4); };
    auto land_x = [&](int st) { return land_xr(st, lj); };
    auto land_y = [&](int st) { return land_yr(st, li); };
    const float qnan = __int_as_float(0x7fffffff);

    constexpr int NS = SPLIT ? ABP : M;       // prefetched source values per cell (register path)
    float sn[SMEMPF ? 1 : NS], sn2[PDS == 2 ? NS : 1];   // next cell; the cell after (depth 2)
#pragma unroll
    for (int m = 0; m < (SMEMPF ? 1 : NS); ++m) sn[m] = 0.0f;
    float rho_n = 0.0f, rho_n2 = 0.0f;        // density (XS: rho sigma_t) and material of the prefetched
    int mat_n = 0, mat_n2 = 0;                // cells; the cross section is formed when the cell is swept
    float zc[AB];                             // z inflow of the column's next cell
    float lk = 0.0f;

    for (;;) {
        __syncthreads();                        // previous task done with task_s and the planes
        if (threadIdx.x == 0) *task_s = atomicAdd(a.flow + 0, 1);
        __syncthreads();
        const int t = *task_s;
        if (t >= ntasks) break;
        const bool withhold = a.flow[3] == t + 1;   // test hook: this task owes no faces
        // task t: stage, then tile fastest, octant, group block
        int s = 0, r = t, ntiles = 1;
        for (; s < nst; ++s) {
            ntiles = flow_stage_tiles(s, a.ntx, a.nty);
            if (r < ntiles * 8 * gcount) break;
            r -= ntiles * 8 * gcount;
        }
        const int ti = r % ntiles;
        r /= ntiles;
        const int o = r & 7, gi = r >> 3;
        const int g = g0 + gi;
        const int at = max(0, s - (a.nty - 1)) + ti, bt = s - at;
        const int sx = (o & 1) ? -1 : 1, sy = (o & 2) ? -1 : 1, sz = (o & 4) ? -1 : 1;
        const int oe = a.reverse ? (o ^ 7) : o;     // octant of the directions
        const float fx = (oe & 1) ? -1.0f : 1.0f, fy = (oe & 2) ? -1.0f : 1.0f, fz = (oe & 4) ? -1.0f : 1.0f;
        const int ir = at * a.tx + li, jr = bt * a.ty + lj;
        const bool col = colthread && ir < a.nx && jr < a.ny;
        const int i = sx > 0 ? ir : a.nx - 1 - ir;
        const int j = sy > 0 ? jr : a.ny - 1 - jr;
        const size_t vcol = (size_t)j * a.nx + i;
        const size_t gV = (size_t)g * V;
        const bool xout = li == a.tx - 1 && at < a.ntx - 1 && !withhold;
        const bool yout = lj == a.ty - 1 && bt < a.nty - 1 && !withhold;
        const bool xleak = ir == a.nx - 1, yleak = jr == a.ny - 1;
        const size_t og = (size_t)o * a.G + g;
        float* const xo = a.xface + (og * ntxf + at) * xslab + (size_t)jr * a.nz * ABP;
        float* const yo = a.yface + (og * ntyf + bt) * yslab + (size_t)ir * a.nz * ABP;
        // incoming records (null on the mesh boundary: zero inflow)
        float* const xi = (li == 0 && at > 0) ? a.xface + (og * ntxf + at - 1) * xslab + (size_t)jr * a.nz * ABP : nullptr;
        float* const yi = (lj == 0 && bt > 0) ? a.yface + (og * ntyf + bt - 1) * yslab + (size_t)ir * a.nz * ABP : nullptr;
        // the column threads of the first row and column fetch and wait for the
        // incoming face records, unless the face warp does
        const bool xedge = !HW && col && li == 0, yedge = !HW && col && lj == 0;

        const size_t ang0 = ((size_t)g * 8 + oe) * V;       // angular records of (group, direction octant)
        // source values, density and material of plane kn into (dst, rho, mat);
        // with SMEMPF the moments go to shared memory
        auto fetch = [&](int kn, float* dst, float& rho, int& mt) {
            const int k = sz > 0 ? kn : a.nz - 1 - kn;
            const size_t v = (size_t)k * nxy + vcol;
            if constexpr (SPLIT) {
                const float4* r4 = reinterpret_cast<const float4*>(a.qang + (ang0 + v) * ABP);
#pragma unroll
                for (int c4 = 0; c4 < ABP / 4; ++c4) {
                    const float4 t4 = __ldg(r4 + c4);
                    dst[4 * c4] = t4.x; dst[4 * c4 + 1] = t4.y; dst[4 * c4 + 2] = t4.z; dst[4 * c4 + 3] = t4.w;
                }
            } else if constexpr (SMEMPF) {
                float4* slot = momst + ((kn & 1) * T + threadIdx.x) * 4;
                const float* srcm = a.src + (gV + v) * M;
#pragma unroll
                for (int c4 = 0; c4 < M / 4; ++c4) cp_async_cg16(slot + c4, srcm + 4 * c4);
                (void)dst;
            } else {
                float tmp[M];
                load_moments<M>(a.src + (gV + v) * M, tmp);
#pragma unroll
                for (int m = 0; m < M; ++m) dst[m] = tmp[m];
            }
            if constexpr (XS) {
                rho = __ldg(dt.sig + gV + v);
                (void)mt;
            } else {
                rho = __ldg(a.rho + v);
                mt = __ldg(a.mat + v);
            }
        };
        // register path: the cell after the one in (sn, rho_n, mat_n) moves up,
        // plane kn is fetched behind it
        auto prefetch = [&](int kn) {
            if constexpr (PDS == 2) {
#pragma unroll
                for (int m = 0; m < NS; ++m) sn[m] = sn2[m];
                rho_n = rho_n2;
                mat_n = mat_n2;
                if (kn < a.nz) fetch(kn, sn2, rho_n2, mat_n2);
            } else {
                if (kn < a.nz) fetch(kn, sn, rho_n, mat_n);
            }
        };
        if (col) {
            fetch(0, sn, rho_n, mat_n);
            if constexpr (PDS == 2) {
                if (a.nz > 1) fetch(1, sn2, rho_n2, mat_n2);
            }
        }
        if constexpr (SMEMPF) asm volatile("cp.async.commit_group;\n" ::: "memory");
#pragma unroll
        for (int q = 0; q < AB; ++q) zc[q] = 0.0f;

        // issue the fetch of the face records this thread uses at step st
        // (plane st - d): one commit group per step for every thread
        auto issue_faces = [&](int st) {
            const int kt = st - d;
            if (col && kt >= 0 && kt < a.nz) {
                if (xedge && xi) {
#pragma unroll
                    for (int c4 = 0; c4 < ABP / 4; ++c4)
                        cp_async_cg16(land_x(st) + c4, xi + (size_t)kt * ABP + 4 * c4);
                }
                if (yedge && yi) {
#pragma unroll
                    for (int c4 = 0; c4 < ABP / 4; ++c4)
                        cp_async_cg16(land_y(st) + c4, yi + (size_t)kt * ABP + 4 * c4);
                }
            }
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        };
        // the face warp's records: lane r owns x-face row r (r < ty: the
        // record entering column (0, r)) and y-face column r - ty (entering
        // column (r - ty, 0)), and again r + 32
        const int lane = threadIdx.x & 31;
        auto fw_rec = [&](int r, int& side, int& idx, bool& ok, float*& src) {
            if (r < a.ty) {
                side = 0;
                idx = r;
                const int jr2 = bt * a.ty + r;
                ok = jr2 < a.ny;
                src = at > 0 ? a.xface + (og * ntxf + at - 1) * xslab + (size_t)jr2 * a.nz * ABP : nullptr;
            } else {
                side = 1;
                idx = r - a.ty;
                const int ir2 = at * a.tx + idx;
                ok = ir2 < a.nx;
                src = bt > 0 ? a.yface + (og * ntyf + bt - 1) * yslab + (size_t)ir2 * a.nz * ABP : nullptr;
            }
        };
        // fetch the records used at step st (plane st - idx of each edge column)
        auto fw_issue = [&](int st) {
            for (int r = lane; r < a.tx + a.ty; r += 32) {
                int side, idx;
                bool ok;
                float* src;
                fw_rec(r, side, idx, ok, src);
                const int pf = st - idx;
                if (ok && src && pf >= 0 && pf < a.nz) {
                    float4* land = side == 0 ? land_xr(st, idx) : land_yr(st, idx);
                    const float* s0 = src + (size_t)pf * ABP;
#pragma unroll
                    for (int c4 = 0; c4 < ABP / 4; ++c4) cp_async_cg16(land + c4, s0 + 4 * c4);
                }
            }
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        };
        // the records of step st (fetched PD steps ago): wait until complete,
        // move into the halo of plane buffer cbf, hand back as NaN; zero
        // inflow on the mesh boundary
        auto fw_fill = [&](int st, int cbf) {
            for (int r = lane; r < a.tx + a.ty; r += 32) {
                int side, idx;
                bool ok;
                float* src;
                fw_rec(r, side, idx, ok, src);
                const int pf = st - idx;
                if (!ok || pf < 0 || pf >= a.nz) continue;
                const int hs = side == 0 ? (idx + 1) * PX * RS : (idx + 1) * RS;
                float* hb = (side == 0 ? buf : bufy) + cbf * P * RS;
                if (!src) {
#pragma unroll
                    for (int q = 0; q < AB; ++q) hb[hs + q] = 0.0f;
                    continue;
                }
                float4* land = side == 0 ? land_xr(st, idx) : land_yr(st, idx);
                const float* lf = reinterpret_cast<const float*>(land);
                float* s0 = src + (size_t)pf * ABP;
                bool got = false;
                for (int it = 0; it < kFlowSpinLimit; ++it) {
                    got = true;
#pragma unroll
                    for (int q = 0; q < AB; ++q) got = got && !isnan(lf[q]);
                    if (got) break;
                    if ((it & 63) == 63 && *reinterpret_cast<volatile int*>(a.flow + 2)) break;
                    __nanosleep(100);
#pragma unroll
                    for (int c4 = 0; c4 < ABP / 4; ++c4) cp_async_cg16(land + c4, s0 + 4 * c4);
                    cp_async_wait_all();
                }
                if (!got) atomicExch(a.flow + 2, 1);
#pragma unroll
                for (int q = 0; q < AB; ++q) hb[hs + q] = got ? lf[q] : 0.0f;
                float4* back = reinterpret_cast<float4*>(s0);
#pragma unroll
                for (int c4 = 0; c4 < ABP / 4; ++c4) back[c4] = make_float4(qnan, qnan, qnan, qnan);
            }
        };
        // steps -PD .. -1 only fetch the first records
        for (int st = 0; st < PD - 1; ++st) {
            if (HW && fw) fw_issue(st);
            else issue_faces(st);
        }
        const int hend = a.nz + a.tx + a.ty - 2;
#pragma unroll 1
        for (int h = -1; h < hend; ++h) {
            const int cb = h & 1, pb = cb ^ 1;
          if (HW && fw) {
            fw_issue(h + PD);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
            fw_fill(h + 1, cb);
          } else {
            float sig_cur = 0.0f;
            if constexpr (SMEMPF) {
                // this step's cross section, then the next cell's moments (their own
                // commit group, ahead of the face records of this step)
                const int kr0 = h - d;
                if (col && kr0 >= 0 && kr0 < a.nz) {
                    sig_cur = XS ? rho_n : rho_n * sigt_s[gi * a.nmat + mat_n];
                    if (kr0 + 1 < a.nz) fetch(kr0 + 1, sn, rho_n, mat_n);
                }
                asm volatile("cp.async.commit_group;\n" ::: "memory");
            }
            if constexpr (!HW) issue_faces(h + PD);
            const int kr = h - d;
            const bool act = col && h >= d && kr < a.nz;
            if (act) {
                const bool last = kr == a.nz - 1;
                const int k = sz > 0 ? kr : a.nz - 1 - kr;
                const size_t v = (size_t)k * nxy + vcol;
                float sig_reg = 0.0f;
                if constexpr (!SMEMPF) {
                    if constexpr (!SPLIT) {
#pragma unroll
                        for (int m = 0; m < NS; ++m) sn[m] *= octant_sign<M>(m, fx, fy, fz);
                    }
                    sig_reg = XS ? rho_n : rho_n * sigt_s[gi * a.nmat + mat_n];
                }
                float sreg[SMEMPF ? 1 : NS];
                if constexpr (!SMEMPF) {
#pragma unroll
                    for (int m = 0; m < NS; ++m) sreg[m] = sn[m];
                    if (!last) prefetch(kr + PDS);
                }
                const size_t mo = (gV + v) * M;
                float s[NS];
                float sig;
                if constexpr (SMEMPF) {
                    sig = sig_cur;
                    const float4* slot = momst + ((kr & 1) * T + threadIdx.x) * 4;
#pragma unroll
                    for (int c4 = 0; c4 < M / 4; ++c4) {
                        const float4 t4 = slot[c4];
                        s[4 * c4] = t4.x; s[4 * c4 + 1] = t4.y; s[4 * c4 + 2] = t4.z; s[4 * c4 + 3] = t4.w;
                    }
#pragma unroll
                    for (int m = 0; m + 1 < NS; m += 2) {
                        const float2 r2 = __fmul2_rn(make_float2(s[m], s[m + 1]),
                                                     make_float2(octant_sign<M>(m, fx, fy, fz),
                                                                 octant_sign<M>(m + 1, fx, fy, fz)));
                        s[m] = r2.x;
                        s[m + 1] = r2.y;
                    }
                    if constexpr (NS % 2 == 1) s[NS - 1] *= octant_sign<M>(NS - 1, fx, fy, fz);
                } else {
                    sig = sig_reg;
#pragma unroll
                    for (int m = 0; m < NS; ++m) s[m] = sreg[m];
                }
                // moments -> directions (split: the record already holds them)
                float psi[AB];
                if constexpr (SPLIT) {
#pragma unroll
                    for (int q = 0; q < AB; ++q) psi[q] = s[q];
                } else {
                    // even and odd moments in the two lanes of packed FMAs; the lane
                    // sums of directions q, q+1 in one packed add
                    auto msum = [&](int q) {
                        float2 t2 = make_float2(0.0f, 0.0f);
#pragma unroll
                        for (int m = 0; m + 1 < M; m += 2)
                            t2 = __ffma2_rn(make_float2(dt.mop[q * 16 + m], dt.mop[q * 16 + m + 1]),
                                            make_float2(s[m], s[m + 1]), t2);
                        if constexpr (M % 2 == 1) t2.x = fmaf(dt.mop[q * 16 + M - 1], s[M - 1], t2.x);
                        return t2;
                    };
#pragma unroll
                    for (int q = 0; q + 1 < AB; q += 2) {
                        const float2 ta = msum(q), tb = msum(q + 1);
                        const float2 p2 = __fadd2_rn(make_float2(ta.x, tb.x), make_float2(ta.y, tb.y));
                        psi[q] = p2.x;
                        psi[q + 1] = p2.y;
                    }
                    if constexpr (AB % 2 == 1) {
                        const float2 ta = msum(AB - 1);
                        psi[AB - 1] = ta.x + ta.y;
                    }
                }
                // step-differenced cell solve
                const float* pv = buf + pb * P * RS;
                float* cv = buf + cb * P * RS;
                const float* pvy = bufy + pb * P * RS;    // step: the same plane
                float* cvy = bufy + cb * P * RS;
                if constexpr (!DD) {
                    // two directions per packed operation
#pragma unroll
                    for (int q = 0; q + 1 < AB; q += 2) {
                        const float2 px2 = make_float2(pv[xs + q], pv[xs + q + 1]);
                        const float2 py2 = make_float2(pvy[ys + q], pvy[ys + q + 1]);
                        float2 n2 = __ffma2_rn(make_float2(dt.cx[q], dt.cx[q + 1]), px2, make_float2(psi[q], psi[q + 1]));
                        n2 = __ffma2_rn(make_float2(dt.cy[q], dt.cy[q + 1]), py2, n2);
                        n2 = __ffma2_rn(make_float2(dt.cz[q], dt.cz[q + 1]), make_float2(zc[q], zc[q + 1]), n2);
                        const float2 d2 = __fadd2_rn(make_float2(sig, sig), make_float2(dt.csum[q], dt.csum[q + 1]));
                        const float2 p2 = make_float2(n2.x * rcp_approx(d2.x), n2.y * rcp_approx(d2.y));
                        psi[q] = p2.x;
                        psi[q + 1] = p2.y;
                        cv[os + q] = p2.x;
                        cv[os + q + 1] = p2.y;
                        zc[q] = p2.x;
                        zc[q + 1] = p2.y;
                    }
                }
#pragma unroll
                for (int q = DD ? 0 : (AB & ~1); q < AB; ++q) {
                    const float px = pv[xs + q];
                    const float py = pvy[ys + q];
                    const float num = fmaf(dt.cz[q], zc[q], fmaf(dt.cy[q], py, fmaf(dt.cx[q], px, psi[q])));
                    psi[q] = num * rcp_approx(sig + dt.csum[q]);
                    if constexpr (DD) {
                        cv[os + q] = fmaf(2.0f, psi[q], -px);
                        cvy[os + q] = fmaf(2.0f, psi[q], -py);
                        zc[q] = fmaf(2.0f, psi[q], -zc[q]);
                    } else {
                        cv[os + q] = psi[q];
                        zc[q] = psi[q];
                    }
                }
                // stored angular fluence, laid out for this kernel as one 16-byte
                // aligned record of ABP floats per (group, voxel, direction octant,
                // direction block): [G][V][8][nab][ABP] (the stage kernels use [G][V][A])
                if constexpr (MODE == 1) {
                    float4* rec = reinterpret_cast<float4*>(a.psi + ((((size_t)g * V + v) * 8 + oe) * a.nab + a.blk) * ABP);
#pragma unroll
                    for (int c4 = 0; c4 < ABP / 4; ++c4)
                        rec[c4] = make_float4(4 * c4 < AB ? psi[4 * c4 < AB ? 4 * c4 : 0] : 0.0f,
                                              4 * c4 + 1 < AB ? psi[4 * c4 + 1 < AB ? 4 * c4 + 1 : 0] : 0.0f,
                                              4 * c4 + 2 < AB ? psi[4 * c4 + 2 < AB ? 4 * c4 + 2 : 0] : 0.0f,
                                              4 * c4 + 3 < AB ? psi[4 * c4 + 3 < AB ? 4 * c4 + 3 : 0] : 0.0f);
                }
                if constexpr (MODE == 2) {
                    const float4* rec =
                        reinterpret_cast<const float4*>(a.psi + ((((size_t)g * V + v) * 8 + oe) * a.nab + a.blk) * ABP);
                    float pacc = 0.0f;
#pragma unroll
                    for (int c4 = 0; c4 < ABP / 4; ++c4) {
                        const float4 t4 = __ldg(rec + c4);
                        const float st4[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (4 * c4 + e < AB) pacc = fmaf(dt.w[4 * c4 + e] * psi[4 * c4 + e < AB ? 4 * c4 + e : 0], st4[e], pacc);
                    }
                    red_add_f32(a.prod + gV + v, pacc);
                }
                // outgoing face records of plane kr
                if constexpr (DD) {
                    // the x and y face fluxes, read back from this thread's plane entries
                    const float* fxo = cv + os;
                    const float* fyo = cvy + os;
                    if (xout) {
                        float4* dst = reinterpret_cast<float4*>(xo + (size_t)kr * ABP);
#pragma unroll
                        for (int c4 = 0; c4 < ABP / 4; ++c4)
                            dst[c4] = make_float4(4 * c4 < AB ? fxo[4 * c4] : 0.0f, 4 * c4 + 1 < AB ? fxo[4 * c4 + 1] : 0.0f,
                                                  4 * c4 + 2 < AB ? fxo[4 * c4 + 2] : 0.0f,
                                                  4 * c4 + 3 < AB ? fxo[4 * c4 + 3] : 0.0f);
                    }
                    if (yout) {
                        float4* dst = reinterpret_cast<float4*>(yo + (size_t)kr * ABP);
#pragma unroll
                        for (int c4 = 0; c4 < ABP / 4; ++c4)
                            dst[c4] = make_float4(4 * c4 < AB ? fyo[4 * c4] : 0.0f, 4 * c4 + 1 < AB ? fyo[4 * c4 + 1] : 0.0f,
                                                  4 * c4 + 2 < AB ? fyo[4 * c4 + 2] : 0.0f,
                                                  4 * c4 + 3 < AB ? fyo[4 * c4 + 3] : 0.0f);
                    }
                    if (xleak || yleak || last) {
#pragma unroll
                        for (int q = 0; q < AB; ++q) {
                            if (xleak) lk = fmaf(dt.lx[q], fxo[q], lk);
                            if (yleak) lk = fmaf(dt.ly[q], fyo[q], lk);
                            if (last) lk = fmaf(dt.lz[q], zc[q], lk);
                        }
                    }
                } else {
                if (xout || yout) {
                    float4 rec[ABP / 4];
#pragma unroll
                    for (int c4 = 0; c4 < ABP / 4; ++c4)
                        rec[c4] = make_float4(4 * c4 < AB ? psi[4 * c4 < AB ? 4 * c4 : 0] : 0.0f,
                                              4 * c4 + 1 < AB ? psi[4 * c4 + 1 < AB ? 4 * c4 + 1 : 0] : 0.0f,
                                              4 * c4 + 2 < AB ? psi[4 * c4 + 2 < AB ? 4 * c4 + 2 : 0] : 0.0f,
                                              4 * c4 + 3 < AB ? psi[4 * c4 + 3 < AB ? 4 * c4 + 3 : 0] : 0.0f);
                    if (xout) {
                        float4* dst = reinterpret_cast<float4*>(xo + (size_t)kr * ABP);
#pragma unroll
                        for (int c4 = 0; c4 < ABP / 4; ++c4) dst[c4] = rec[c4];
                    }
                    if (yout) {
                        float4* dst = reinterpret_cast<float4*>(yo + (size_t)kr * ABP);
#pragma unroll
                        for (int c4 = 0; c4 < ABP / 4; ++c4) dst[c4] = rec[c4];
                    }
                }
                if (xleak || yleak || last) {
#pragma unroll
                    for (int q = 0; q < AB; ++q) {
                        float f = 0.0f;
                        if (xleak) f += dt.lx[q];
                        if (yleak) f += dt.ly[q];
                        if (last) f += dt.lz[q];
                        lk = fmaf(f, psi[q], lk);
                    }
                }
                }
                if constexpr (SPLIT) {
                    // the cell's angular fluence record, for k_split_d2m
                    float4* w4 = reinterpret_cast<float4*>(a.pang + (ang0 + v) * ABP);
#pragma unroll
                    for (int c4 = 0; c4 < ABP / 4; ++c4)
                        w4[c4] = make_float4(4 * c4 < AB ? psi[4 * c4 < AB ? 4 * c4 : 0] : 0.0f,
                                             4 * c4 + 1 < AB ? psi[4 * c4 + 1 < AB ? 4 * c4 + 1 : 0] : 0.0f,
                                             4 * c4 + 2 < AB ? psi[4 * c4 + 2 < AB ? 4 * c4 + 2 : 0] : 0.0f,
                                             4 * c4 + 3 < AB ? psi[4 * c4 + 3 < AB ? 4 * c4 + 3 : 0] : 0.0f);
                    (void)mo;
                } else {
                    // directions -> moments (Eq. 3 for lm = 00): table rows hold w R_lm
                    // even and odd directions in the two lanes of packed FMAs
                    float acc[M];
                    // sum over directions of moment m, even and odd directions in the two lanes
                    auto dsum = [&](int m) {
                        float2 t2 = make_float2(0.0f, 0.0f);
#pragma unroll
                        for (int q = 0; q + 1 < AB; q += 2)
                            t2 = __ffma2_rn(make_float2(dt.dop[m * kFlowMaxAB + q], dt.dop[m * kFlowMaxAB + q + 1]),
                                            make_float2(psi[q], psi[q + 1]), t2);
                        if constexpr (AB % 2 == 1) t2.x = fmaf(dt.dop[m * kFlowMaxAB + AB - 1], psi[AB - 1], t2.x);
                        return t2;
                    };
#pragma unroll
                    for (int m = 0; m + 1 < M; m += 2) {
                        // lane sums and octant signs of moments m, m+1 in one packed add and multiply
                        const float2 ta = dsum(m), tb = dsum(m + 1);
                        const float2 r2 = __fmul2_rn(__fadd2_rn(make_float2(ta.x, tb.x), make_float2(ta.y, tb.y)),
                                                     make_float2(octant_sign<M>(m, fx, fy, fz),
                                                                 octant_sign<M>(m + 1, fx, fy, fz)));
                        acc[m] = r2.x;
                        acc[m + 1] = r2.y;
                    }
                    if constexpr (M % 2 == 1) {
                        const float2 ta = dsum(M - 1);
                        acc[M - 1] = (ta.x + ta.y) * octant_sign<M>(M - 1, fx, fy, fz);
                    }
                    add_moments<M>(a.mom + mo, acc);
                }
                if (last && lk != 0.0f) {
                    atomicAdd(leak_s + gi, (double)lk);
                    lk = 0.0f;
                }
            }
            // incoming records of the plane swept next step (fetched PD steps
            // ago): wait until the producer has written every flux (no NaN
            // left), move them into the halo and hand the records back to the
            // next sweep as NaN; zero inflow on the mesh boundary
            const int pf = h + 1 - d;
            if constexpr (SMEMPF) {
                // the next cell's moments (and the faces fetched a step ago) have landed
                if constexpr (HW) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
                else asm volatile("cp.async.wait_group 1;\n" ::: "memory");
            }
            if (col && pf >= 0 && pf < a.nz && (xedge || yedge)) {
                if constexpr (PD == 2) {
                    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
                } else {
                    cp_async_wait_all();
                }
                float* hbx = buf + cb * P * RS;
                float* hby = bufy + cb * P * RS;
                {
                  for (int side = 0; side < 2; ++side) {
                    const bool edge = side == 0 ? xedge : yedge;
                    if (!edge) continue;
                    const int hs = side == 0 ? xs : ys;
                    float* hb = side == 0 ? hbx : hby;
                    float* src = side == 0 ? xi : yi;
                    if (!src) {
#pragma unroll
                        for (int q = 0; q < AB; ++q) hb[hs + q] = 0.0f;
                        continue;
                    }
                    float4* land = side == 0 ? land_x(h + 1) : land_y(h + 1);
                    const float* lf = reinterpret_cast<const float*>(land);
                    src += (size_t)pf * ABP;
                    bool ok = false;
                    for (int it = 0; it < kFlowSpinLimit; ++it) {
                        ok = true;
#pragma unroll
                        for (int q = 0; q < AB; ++q) ok = ok && !isnan(lf[q]);
                        if (ok) break;
                        // once any wait of this sweep has given up, give up at once
                        if ((it & 63) == 63 && *reinterpret_cast<volatile int*>(a.flow + 2)) break;
                        __nanosleep(100);
#pragma unroll
                        for (int c4 = 0; c4 < ABP / 4; ++c4) cp_async_cg16(land + c4, src + 4 * c4);
                        cp_async_wait_all();
                    }
                    if (!ok) atomicExch(a.flow + 2, 1);
#pragma unroll
                    for (int q = 0; q < AB; ++q) hb[hs + q] = ok ? lf[q] : 0.0f;
                    float4* back = reinterpret_cast<float4*>(src);
#pragma unroll
                    for (int c4 = 0; c4 < ABP / 4; ++c4) back[c4] = make_float4(qnan, qnan, qnan, qnan);
                  }
                }
            }
          }
            __syncthreads();
        }
    }
    for (int e = threadIdx.x; e < gcount; e += blockDim.x)
        if (leak_s[e] != 0.0) atomicAdd(a.leak + g0 + e, leak_s[e]);
    // the last CTA out resets the queue for the next sweep
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.flow + 1, 1) == (int)gridDim.x - 1) {
            a.flow[0] = 0;
            a.flow[1] = 0;
        }
    }
}

// Moments -> angular source of every direction of every octant (the
// transform taken out of the split sweep): q[g][o][v][j] =
// sum_lm (2l+1)/(4 pi) R_lm(Omega_{o,j}) s_lm[g][v], with R of octant o the
// first octant's times the reflection signs.  One thread per (group, voxel),
// records written as 16-byte vectors; HBM-bound.
template <int M, int AB>
__global__ void __launch_bounds__(256) k_split_m2d(const float* src, float* qang, size_t V, int g0, int gcount,
                                                  const int* skip) {
    constexpr int ABP = flow_abp(AB);
    constexpr int rb = chain_row_base(AB) * 16;
    if (skip && *skip) return;
    const size_t n = (size_t)gcount * V;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int g = g0 + (int)(e / V);
        const size_t v = e % V;
        float s[M];
        load_moments<M>(src + ((size_t)g * V + v) * M, s);
#pragma unroll 1
        for (int o = 0; o < 8; ++o) {
            const float fx = (o & 1) ? -1.0f : 1.0f, fy = (o & 2) ? -1.0f : 1.0f, fz = (o & 4) ? -1.0f : 1.0f;
            float so[M];
#pragma unroll
            for (int m = 0; m < M; ++m) so[m] = s[m] * octant_sign<M>(m, fx, fy, fz);
            float q[ABP];
#pragma unroll
            for (int j = 0; j < ABP; ++j) {
                float t = 0.0f;
                if (j < AB) {
#pragma unroll
                    for (int m = 0; m < M; ++m) t = fmaf(c_Mop1[rb + j * 16 + lm_of_pos(m, M)], so[m], t);
                }
                q[j] = t;
            }
            float4* out = reinterpret_cast<float4*>(qang + (((size_t)g * 8 + o) * V + v) * ABP);
#pragma unroll
            for (int c4 = 0; c4 < ABP / 4; ++c4) out[c4] = make_float4(q[4 * c4], q[4 * c4 + 1], q[4 * c4 + 2], q[4 * c4 + 3]);
        }
    }
}

// Angular fluence of every direction -> moments (Eq. 3 for lm = 00):
// mom[g][v][lm] = sum_o sum_j w_j R_lm(Omega_{o,j}) psi[g][o][v][j], written
// with plain stores (one thread per (group, voxel), no reductions).
template <int M, int AB>
__global__ void __launch_bounds__(256) k_split_d2m(const float* pang, float* mom, size_t V, int g0, int gcount,
                                                  const int* skip) {
    constexpr int ABP = flow_abp(AB);
    constexpr int rb = chain_row_base(AB) * 16;
    if (skip && *skip) return;
    const size_t n = (size_t)gcount * V;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int g = g0 + (int)(e / V);
        const size_t v = e % V;
        float acc[M];
#pragma unroll
        for (int m = 0; m < M; ++m) acc[m] = 0.0f;
#pragma unroll 1
        for (int o = 0; o < 8; ++o) {
            const float fx = (o & 1) ? -1.0f : 1.0f, fy = (o & 2) ? -1.0f : 1.0f, fz = (o & 4) ? -1.0f : 1.0f;
            const float4* in = reinterpret_cast<const float4*>(pang + (((size_t)g * 8 + o) * V + v) * ABP);
            float ps[ABP];
#pragma unroll
            for (int c4 = 0; c4 < ABP / 4; ++c4) {
                const float4 t4 = __ldg(in + c4);
                ps[4 * c4] = t4.x; ps[4 * c4 + 1] = t4.y; ps[4 * c4 + 2] = t4.z; ps[4 * c4 + 3] = t4.w;
            }
#pragma unroll
            for (int m = 0; m < M; ++m) {
                float b = 0.0f;
#pragma unroll
                for (int j = 0; j < AB; ++j) b = fmaf(c_Dop1[rb + j * 16 + lm_of_pos(m, M)], ps[j], b);
                acc[m] = fmaf(octant_sign<M>(m, fx, fy, fz), b, acc[m]);
            }
        }
        float* out = mom + ((size_t)g * V + v) * M;
        if constexpr (M % 4 == 0) {
            float4* o4 = reinterpret_cast<float4*>(out);
#pragma unroll
            for (int c4 = 0; c4 < M / 4; ++c4) o4[c4] = make_float4(acc[4 * c4], acc[4 * c4 + 1], acc[4 * c4 + 2], acc[4 * c4 + 3]);
        } else {
#pragma unroll
            for (int m = 0; m < M; ++m) out[m] = acc[m];
        }
    }
}

template <int M>
int sweep_flow_blocks_per_sm(int ab, int threads, size_t smem, bool split, bool dd, bool hw) {
    int b = 0;
    cudaError_t e = cudaErrorInvalidValue;
    auto query = [&](auto kern) {
        e = smem > 48 * 1024 ? cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                             : cudaSuccess;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, smem);
    };
#define DOCTORS_FLOW_OCC(AB)                                                            \
    case AB:                                                                            \
        if (split) query(k_sweep_flow<AB, M, 0, true>);                                  \
        else if (dd) query(k_sweep_flow<AB, M, 0, false, true>);                         \
        else if (hw) {                                                                  \
            if constexpr (M % 4 == 0) query(k_sweep_flow<AB, M, 0, false, false, true>); \
        } else query(k_sweep_flow<AB, M, 0>);                                            \
        break;
    switch (ab) {
        DOCTORS_FLOW_OCC(1)
        DOCTORS_FLOW_OCC(3)
        DOCTORS_FLOW_OCC(6)
        DOCTORS_FLOW_OCC(10)
        DOCTORS_FLOW_OCC(12)
        DOCTORS_FLOW_OCC(21)
        DOCTORS_FLOW_OCC(36)
        default: break;
    }
#undef DOCTORS_FLOW_OCC
    return e == cudaSuccess ? b : 0;
}

// m2d, split sweep, d2m: one full sweep with the transforms taken out
template <int M>
cudaError_t launch_split_sweep_m(const SweepArgs& a, cudaStream_t s, int* count) {
    *count = 0;
    if (a.gcount <= 0) return cudaSuccess;
    if (a.dir_table == nullptr || a.flow == nullptr || a.dir_table->sig == nullptr || a.nab != 1 || !a.qang ||
        !a.pang)
        return cudaErrorInvalidValue;
    const size_t V = (size_t)a.nx * a.ny * a.nz;
    const size_t n = (size_t)a.gcount * V;
    const unsigned tgrid = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 8);
    int ntasks = 0;
    for (int st = 0; st < a.ntx + a.nty - 1; ++st) {
        const int lo = st - (a.nty - 1) > 0 ? st - (a.nty - 1) : 0;
        const int hi = st < a.ntx - 1 ? st : a.ntx - 1;
        ntasks += (hi - lo + 1) * 8 * a.gcount;
    }
    // persistent CTAs: every resident slot, or its share when several instances sweep at once
    const int slots = std::max(1, a.chain_slots / std::max(1, a.slot_share));
    const int grid = ntasks < slots ? ntasks : slots;
    const int T = a.tx * a.ty;
    const size_t smem = sweep_flow_smem_bytes(a.ab, a.tx, a.ty, a.gcount, a.nmat);
    cudaError_t e = cudaSuccess;
    // P3: the transforms on the tensor cores when the problem holds their tables
    const bool tc = M == 16 && a.tc_b1 && a.tc_b2;
    auto run = [&](auto m2d, auto sweep, auto d2m) {
        if (tc) {
            e = launch_m2d_tc(a, s);
        } else {
            m2d<<<tgrid, 256, 0, s>>>(a.src, const_cast<float*>(a.qang), V, a.g0, a.gcount, a.skip);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && smem > 48 * 1024)
            e = cudaFuncSetAttribute(sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) {
            sweep<<<grid, T, smem, s>>>(a, *a.dir_table);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            if (tc) {
                e = launch_d2m_tc(a, s);
            } else {
                d2m<<<tgrid, 256, 0, s>>>(a.pang, a.mom, V, a.g0, a.gcount, a.skip);
                e = cudaGetLastError();
            }
        }
    };
    switch (a.ab) {
        case 1: run(k_split_m2d<M, 1>, k_sweep_flow<1, M, 0, true>, k_split_d2m<M, 1>); break;
        case 3: run(k_split_m2d<M, 3>, k_sweep_flow<3, M, 0, true>, k_split_d2m<M, 3>); break;
        case 6: run(k_split_m2d<M, 6>, k_sweep_flow<6, M, 0, true>, k_split_d2m<M, 6>); break;
        case 10: run(k_split_m2d<M, 10>, k_sweep_flow<10, M, 0, true>, k_split_d2m<M, 10>); break;
        default: return cudaErrorInvalidValue;
    }
    if (e == cudaSuccess) *count = 3;
    return e;
}

template <int M, int MODE>
cudaError_t launch_sweep_flow_m(const SweepArgs& a, cudaStream_t s) {
    if (a.gcount <= 0) return cudaSuccess;
    if (a.dir_table == nullptr || a.flow == nullptr || a.dir_table->sig == nullptr || a.blk < 0 || a.blk >= a.nab ||
        a.ab * a.nab != a.A8)
        return cudaErrorInvalidValue;
    const bool dd = a.dd != 0;
    int ntasks = 0;
    for (int st = 0; st < a.ntx + a.nty - 1; ++st) {
        const int lo = st - (a.nty - 1) > 0 ? st - (a.nty - 1) : 0;
        const int hi = st < a.ntx - 1 ? st : a.ntx - 1;
        ntasks += (hi - lo + 1) * 8 * a.gcount;
    }
    // persistent CTAs: every resident slot, or its share when several instances sweep at once
    const int slots = std::max(1, a.chain_slots / std::max(1, a.slot_share));
    const int grid = ntasks < slots ? ntasks : slots;
    const bool hw = MODE == 0 && a.hw != 0 && !dd && M % 4 == 0;
    // column threads, plus the face warp
    const int T = hw ? ((a.tx * a.ty + 31) / 32 + 1) * 32 : a.tx * a.ty;
    const size_t smem = sweep_flow_smem_bytes(a.ab, a.tx, a.ty, a.gcount, a.nmat, dd);
    cudaError_t e = cudaSuccess;
    auto launch = [&](auto kern) {
        if (smem > 48 * 1024) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) kern<<<grid, T, smem, s>>>(a, *a.dir_table);
    };
#define DOCTORS_FLOW_CASE(AB)                                                           \
    case AB:                                                                            \
        if (dd) {                                                                       \
            launch(k_sweep_flow<AB, M, MODE, false, true>);                              \
            break;                                                                      \
        }                                                                               \
        if constexpr (MODE == 0 && M % 4 == 0) {                                        \
            if (hw) {                                                                   \
                launch(k_sweep_flow<AB, M, 0, false, false, true>);                      \
                break;                                                                  \
            }                                                                           \
        }                                                                               \
        launch(k_sweep_flow<AB, M, MODE>);                                               \
        break;
    switch (a.ab) {
        DOCTORS_FLOW_CASE(1)
        DOCTORS_FLOW_CASE(3)
        DOCTORS_FLOW_CASE(6)
        DOCTORS_FLOW_CASE(10)
        DOCTORS_FLOW_CASE(12)
        DOCTORS_FLOW_CASE(21)
        DOCTORS_FLOW_CASE(36)
        default: return cudaErrorInvalidValue;
    }
#undef DOCTORS_FLOW_CASE
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace doctors
