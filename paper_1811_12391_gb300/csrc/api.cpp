// C-ABI entry points of libdoctors (declared in include/doctors.h).
//
// The handle owns the device state; every launch goes to the problem's
// stream.  Solve = ray trace + first-collision source (Sec. II.A), then
// source iteration of the collided problem (Eq. 2) with all groups per sweep
// (Jacobi in energy: same fixed point as solving the groups one after the
// other), stopped on the FP64 relative L2 change of the scalar fluence
// (Eq. 3) in every group.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "doctors_internal.h"

namespace doctors {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

}  // namespace doctors

using namespace doctors;

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));              \
            return DOCTORS_ERR_CUDA;                                                    \
        }                                                                               \
    } while (0)

#define CHECK_ARG(cond, msg)          \
    do {                              \
        if (!(cond)) {                \
            set_error(msg);           \
            return DOCTORS_ERR_INVALID_ARG; \
        }                             \
    } while (0)

namespace {

// default choice of the moment-transform path of the sweep for P3 problems
constexpr bool kDefaultChainedSweep = true;
constexpr bool kDefaultDataflowSweep = true;
constexpr bool kDefaultSplitSweep = false;
constexpr bool kDefaultFaceWarpSweep = true;

int dalloc(void** p, size_t bytes, const char* what) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        set_error(std::string("device allocation failed: ") + what + " (" + std::to_string(bytes) + " bytes)");
        return e == cudaErrorMemoryAllocation ? DOCTORS_ERR_OOM : DOCTORS_ERR_CUDA;
    }
    return DOCTORS_OK;
}

template <class T>
int dalloc_t(T** p, size_t count, const char* what) {
    return dalloc(reinterpret_cast<void**>(p), count * sizeof(T), what);
}

int default_ab(int A8, int kernel) {
    // the dataflow kernels (the default where they apply) sweep whole octants
    if ((kernel == 0 || kernel == 4 || kernel == 7) && flow_octant_ab(A8)) return A8;
    const int cand[] = {12, 10, 9, 7, 6, 5, 4, 3, 2, 1};
    for (int c : cand)
        if (A8 % c == 0) return c;
    return 1;
}

// Direction table of the first octant's directions j0 .. j0+n-1: step and
// boundary coefficients and weights (n <= kMaxA8) and, for the first
// kFlowMaxAB of them, the moment <-> direction rows.  Diamond differencing
// stores 2 c (the dataflow kernel's cell solve then has the step form).
ChainDirTable make_dir_table(const doctors_problem* p, int j0, int n) {
    ChainDirTable t{};
    t.sig = p->d_sig;
    const double dx = p->mesh.dx, dy = p->mesh.dy, dz = p->mesh.dz;
    const float cf = p->differencing == DOCTORS_DIFF_DIAMOND ? 2.0f : 1.0f;
    double Rb[16];
    for (int jl = 0; jl < n && jl < kMaxA8; ++jl) {
        const int j = j0 + jl;
        const double x = p->dirs[3 * j], y = p->dirs[3 * j + 1], z = p->dirs[3 * j + 2];
        const double ox = std::fabs(x), oy = std::fabs(y), oz = std::fabs(z), wj = p->w[j];
        if (jl < kFlowMaxAB) {
            real_harmonics(3, x, y, z, Rb);
            for (int m = 0; m < p->M; ++m) {
                const int lm = lm_of_pos(m, p->M);
                t.mop[jl * 16 + m] = (float)((2 * degree_of_lm(lm) + 1) / (4.0 * M_PI) * Rb[lm]);
                t.dop[m * kFlowMaxAB + jl] = (float)(wj * Rb[lm]);
            }
        }
        t.cx[jl] = cf * (float)(ox / dx);
        t.cy[jl] = cf * (float)(oy / dy);
        t.cz[jl] = cf * (float)(oz / dz);
        t.csum[jl] = cf * (float)(ox / dx + oy / dy + oz / dz);
        t.lx[jl] = (float)(wj * ox * dy * dz);
        t.ly[jl] = (float)(wj * oy * dx * dz);
        t.lz[jl] = (float)(wj * oz * dx * dy);
        t.w[jl] = (float)wj;
    }
    return t;
}

void free_problem(doctors_problem* p) {
    void* ptrs[] = {p->d_coef, p->d_mat, p->d_rho, p->d_sigt, p->d_sigs,
                    p->d_phiu_src, p->d_phiu, p->d_U, p->d_Q, p->d_mom, p->d_src, p->d_src2, p->d_prev,
                    p->d_emit, p->d_iso, p->d_xface, p->d_yface, p->d_red,
                    p->d_Z, p->d_Qa, p->d_T, p->d_rf, p->d_r, p->d_acc, p->d_grad, p->d_H,
                    p->d_ones, p->d_psi, p->d_prod, p->d_flow, p->d_qang, p->d_pang,
                    p->d_k, p->d_roi, p->d_part, p->d_tcb, p->d_emit_all, p->d_dose_stage, p->d_sig};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (p->h_red) cudaFreeHost(p->h_red);
    if (p->h_acc) cudaFreeHost(p->h_acc);
    if (p->d_acc_src) cudaFree(p->d_acc_src);
    if (p->h_acc_src) cudaFreeHost(p->h_acc_src);
    for (auto& e : p->ev)
        if (e) cudaEventDestroy(e);
}

// the (perp, up) frame of a collimated source: perp = (-a_y, a_x, 0)/|(a_x, a_y)|
// ((1,0,0) for an axis along z), up = axis x perp; FP64, then rounded to FP32.
void collimator_frame(const double a[3], double perp[3], double up[3]) {
    const double h = std::sqrt(a[0] * a[0] + a[1] * a[1]);
    if (h == 0.0) {
        perp[0] = 1.0; perp[1] = 0.0; perp[2] = 0.0;
    } else {
        perp[0] = -a[1] / h; perp[1] = a[0] / h; perp[2] = 0.0;
    }
    up[0] = a[1] * perp[2] - a[2] * perp[1];
    up[1] = a[2] * perp[0] - a[0] * perp[2];
    up[2] = a[0] * perp[1] - a[1] * perp[0];
}

RayArgs ray_args(const doctors_problem* p, const doctors_source& s, const float* emit) {
    RayArgs r{};
    r.nx = p->nx; r.ny = p->ny; r.nz = p->nz; r.G = p->G; r.nmat = p->nmat;
    r.ox = (float)p->mesh.origin[0]; r.oy = (float)p->mesh.origin[1]; r.oz = (float)p->mesh.origin[2];
    r.dx = (float)p->mesh.dx; r.dy = (float)p->mesh.dy; r.dz = (float)p->mesh.dz;
    r.sx = (float)s.pos[0]; r.sy = (float)s.pos[1]; r.sz = (float)s.pos[2];
    r.lit_all = s.kind == DOCTORS_SRC_POINT ? 1 : 0;
    double perp[3], up[3];
    collimator_frame(s.axis, perp, up);
    r.ax = (float)s.axis[0]; r.ay = (float)s.axis[1]; r.az = (float)s.axis[2];
    r.px = (float)perp[0]; r.py = (float)perp[1]; r.pz = (float)perp[2];
    r.ux = (float)up[0]; r.uy = (float)up[1]; r.uz = (float)up[2];
    r.tan_half = (float)std::tan(0.5 * s.fan_deg * (M_PI / 180.0));
    r.z_slope = (float)(s.z_half_iso / (s.iso_dist > 0 ? s.iso_dist : 1.0));
    r.mat = p->d_mat; r.rho = p->d_rho; r.sigt = p->d_sigt; r.emit = emit;
    r.phi_src = p->d_phiu_src; r.phi_tot = p->d_phiu;
    return r;
}

int check_problem(doctors_problem* p) {
    CHECK_ARG(p != nullptr, "null problem");
    cudaError_t e = cudaSetDevice(p->device);
    if (e != cudaSuccess) {
        set_error(std::string("cudaSetDevice: ") + cudaGetErrorString(e));
        return DOCTORS_ERR_CUDA;
    }
    return DOCTORS_OK;
}

// ray trace every point source and build the fixed (first-collision) source Q
int first_collision(doctors_problem* p) {
    const size_t GV = (size_t)p->G * p->V;
    CU(cudaMemsetAsync(p->d_phiu, 0, GV * sizeof(float), p->stream));
    // the first point source stores the uncollided moments, later ones add;
    // with volume sources only they stay zero
    bool any_point = false;
    for (const doctors_source& src : p->srcs) any_point = any_point || src.kind != DOCTORS_SRC_VOLUME;
    if (!any_point) CU(cudaMemsetAsync(p->d_U, 0, GV * p->M * sizeof(float), p->stream));
    bool first_point = true;
    std::vector<float> iso(p->G, 0.0f);
    std::vector<float> emit_all((size_t)p->srcs.size() * p->G);
    for (size_t s = 0; s < p->srcs.size(); ++s)
        for (int g = 0; g < p->G; ++g) emit_all[s * p->G + g] = (float)(p->srcs[s].weight * p->spectra[s][g]);
    // the emission table stays allocated between solves (grown when the
    // source list grows); copies from pageable host memory are staged before
    // they return, and the table is only read by launches on this stream
    if (p->emit_cap < emit_all.size()) {
        if (p->d_emit_all) {
            CU(cudaStreamSynchronize(p->stream));
            cudaFree(p->d_emit_all);
            p->d_emit_all = nullptr;
            p->emit_cap = 0;
        }
        int rc = dalloc_t(&p->d_emit_all, emit_all.size(), "source emission table");
        if (rc) return rc;
        p->emit_cap = emit_all.size();
    }
    float* d_emit_all = p->d_emit_all;
    cudaError_t e = cudaMemcpyAsync(d_emit_all, emit_all.data(), emit_all.size() * sizeof(float),
                                    cudaMemcpyHostToDevice, p->stream);
    for (size_t s = 0; s < p->srcs.size() && e == cudaSuccess; ++s) {
        const doctors_source& src = p->srcs[s];
        if (src.kind == DOCTORS_SRC_VOLUME) {
            for (int g = 0; g < p->G; ++g) iso[g] += (float)(src.weight * p->spectra[s][g]);
            continue;
        }
        RayArgs r = ray_args(p, src, d_emit_all + s * p->G);
        e = launch_raytrace(r, p->stream);
        if (e != cudaSuccess) break;
        ++p->launches;
        MomentArgs m{};
        m.nx = p->nx; m.ny = p->ny; m.nz = p->nz; m.G = p->G; m.M = p->M; m.L = p->L;
        m.ox = r.ox; m.oy = r.oy; m.oz = r.oz; m.dx = r.dx; m.dy = r.dy; m.dz = r.dz;
        m.sx = r.sx; m.sy = r.sy; m.sz = r.sz;
        m.phi_src = p->d_phiu_src;
        m.U = p->d_U;
        m.accumulate = first_point ? 0 : 1;
        first_point = false;
        e = launch_uncollided_moments(m, p->stream);
        ++p->launches;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->d_iso, iso.data(), p->G * sizeof(float), cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) {
        ScatterArgs sa{};
        sa.V = p->V; sa.G = p->G; sa.M = p->M; sa.L = p->L; sa.nmat = p->nmat; sa.transpose = 0;
        sa.mat = p->d_mat; sa.rho = p->d_rho; sa.sigs = p->d_sigs;
        sa.base = nullptr; sa.iso = p->d_iso; sa.phi = p->d_U; sa.out = p->d_Q;
        e = launch_scatter(sa, p->stream);
        ++p->launches;
    }
    if (e != cudaSuccess) {
        set_error(std::string("first-collision source: ") + cudaGetErrorString(e));
        return DOCTORS_ERR_CUDA;
    }
    return DOCTORS_OK;
}

SweepArgs sweep_args(const doctors_problem* p, int reverse, const float* src, float* mom) {
    SweepArgs a{};
    a.nx = p->nx; a.ny = p->ny; a.nz = p->nz; a.G = p->G; a.A8 = p->A8; a.ab = p->ab; a.nab = p->nab;
    a.nmat = p->nmat; a.tx = p->tx; a.ty = p->ty; a.ntx = p->ntx; a.nty = p->nty; a.reverse = reverse;
    a.mat = p->d_mat; a.rho = p->d_rho; a.sigt = p->d_sigt; a.src = src; a.mom = mom;
    a.table_base = p->table_base; a.coef = p->d_coef; a.xface = p->d_xface; a.yface = p->d_yface;
    a.leak = p->d_red;
    a.A = p->A;
    a.g0 = 0;
    a.gcount = p->G;
    a.chain_slots = p->chain_slots;
    a.dir_table = &p->dir_table;
    a.flow = (p->use_flow || p->use_split) ? p->d_flow : nullptr;
    a.qang = p->d_qang;
    a.pang = p->d_pang;
    a.hw = p->flow_hw ? 1 : 0;
    a.tc_b1 = (p->use_split && p->split_tc) ? p->d_tcb : nullptr;
    a.tc_b2 = (p->use_split && p->split_tc) ? p->d_tcb + p->tcb1_floats : nullptr;
    a.dd = p->differencing == DOCTORS_DIFF_DIAMOND ? 1 : 0;
    a.blk = 0;
    return a;
}

// One full sweep with the problem's chosen kernel: one launch per tile stage,
// or one dataflow launch.  Returns the kernels launched in *count.
cudaError_t launch_sweep(const doctors_problem* p, SweepArgs sw, int mode, cudaStream_t s, int* count) {
    if (p->use_split && mode == 0) return launch_split_sweep(sw, p->M, s, count);
    if (p->use_flow || p->use_split) {
        // modes 1 and 2 (stored / paired angular fluence) of the split and face-warp
        // paths use the plain dataflow kernel
        if (p->use_split || (mode != 0 && p->flow_hw)) sw.chain_slots = p->flow_slots;
        if (p->nab == 1) {
            *count = 1;
            return launch_sweep_flow(sw, p->M, mode, s);
        }
        // direction blocks (S16): one launch per block, each with its own table;
        // the blocks only share the moments (vector reductions) and the leakage
        *count = 0;
        for (int b = 0; b < p->nab; ++b) {
            sw.blk = b;
            sw.dir_table = &p->dir_blk[b];
            cudaError_t e = launch_sweep_flow(sw, p->M, mode, s);
            if (e != cudaSuccess) return e;
            ++*count;
        }
        return cudaSuccess;
    }
    *count = 0;
    for (int st = 0; st < p->ntx + p->nty - 1; ++st) {
        sw.stage = st;
        cudaError_t e = launch_sweep_stage(sw, p->M, mode, s);
        if (e != cudaSuccess) return e;
        ++*count;
    }
    return cudaSuccess;
}

// After a dataflow sweep: a face wait that timed out leaves the queue and the
// face records in an unknown state; reset them and report the failure.
int check_flow(doctors_problem* p) {
    if (!(p->use_flow || p->use_split) || !p->d_flow) return DOCTORS_OK;
    int h[4] = {0, 0, 0, 0};
    CU(cudaMemcpyAsync(h, p->d_flow, sizeof(h), cudaMemcpyDeviceToHost, p->stream));
    CU(cudaStreamSynchronize(p->stream));
    if (h[2] == 0) return DOCTORS_OK;
    CU(cudaMemsetAsync(p->d_flow, 0, 3 * sizeof(int), p->stream));
    CU(cudaMemsetAsync(p->d_xface, 0xff, p->xface_bytes, p->stream));
    CU(cudaMemsetAsync(p->d_yface, 0xff, p->yface_bytes, p->stream));
    CU(cudaStreamSynchronize(p->stream));
    set_error("dataflow sweep: a wait for an upstream face timed out");
    return DOCTORS_ERR_TIMEOUT;
}

// Source iteration: src = Q + S(mom); mom = sweep(src); residual.  `reverse`
// selects the adjoint: sweep directions reversed and scattering transposed.
int iterate(doctors_problem* p, int reverse, const float* Q, float* mom, doctors_result* info) {
    const size_t GVM = (size_t)p->G * p->V * p->M;
    const size_t VM = p->V * p->M;
    double* d_res = p->d_red + p->G;
    double* d_bal = p->d_red + 3 * p->G;
    CU(cudaMemsetAsync(mom, 0, GVM * sizeof(float), p->stream));
    CU(cudaMemsetAsync(p->d_prev, 0, (size_t)p->G * p->V * sizeof(float), p->stream));
    CU(cudaMemsetAsync(p->d_red, 0, 5 * (size_t)p->G * sizeof(double), p->stream));
    const double tol = std::max(p->opt.tol, kTolFloor);
    int it = 0;
    double resid = 0.0;
    double ms_sweep = 0.0;
    double updates = 0.0;
    bool conv = false;
    // Active group window [g0, g1).  A group whose relative change is below
    // tol and whose sources are all final is final itself: in the forward
    // problem (downscatter) the window's leading groups retire, in the adjoint
    // (transposed scattering, upward in energy) its trailing groups.
    int g0 = 0, g1 = p->G;
    std::vector<double> eps(p->G, 0.0);
    // The next iteration's scattering source is formed while the host reads
    // this iteration's residuals: it is launched right after the residual
    // copy, for the current window (a superset of the next one), into the
    // other source buffer; the host waits only for the copy.  After the last
    // iteration that launch is wasted, and the source of the last sweep stays
    // in its own buffer for the balance.
    float* srcs[2] = {p->d_src, p->d_src2};
    int cur = 0;
    SweepArgs sw = sweep_args(p, reverse, srcs[cur], mom);
    ScatterArgs sa{};
    sa.V = p->V; sa.G = p->G; sa.M = p->M; sa.L = p->L; sa.nmat = p->nmat; sa.transpose = reverse;
    sa.mat = p->d_mat; sa.rho = p->d_rho; sa.sigs = p->d_sigs;
    sa.base = Q; sa.phi = mom;
    CU(cudaMemcpyAsync(srcs[cur], Q, GVM * sizeof(float), cudaMemcpyDeviceToDevice, p->stream));
    while (it < p->opt.max_iters) {
        const int gc = g1 - g0;
        if (!p->use_split)   // the split path's d2m pass writes the window's moments
            CU(cudaMemsetAsync(mom + (size_t)g0 * VM, 0, (size_t)gc * VM * sizeof(float), p->stream));
        CU(cudaMemsetAsync(p->d_red + g0, 0, (size_t)gc * sizeof(double), p->stream));
        CU(cudaMemsetAsync(d_res + 2 * g0, 0, 2 * (size_t)gc * sizeof(double), p->stream));
        CU(cudaEventRecord(p->ev[3], p->stream));
        sw.src = srcs[cur];
        sw.g0 = g0;
        sw.gcount = gc;
        int nl = 0;
        CU(launch_sweep(p, sw, 0, p->stream, &nl));
        p->launches += nl;
        CU(cudaEventRecord(p->ev[4], p->stream));
        CU(launch_residual(p->V, p->G, p->M, mom, p->d_prev, d_res, p->stream, nullptr, g0, gc));
        ++p->launches;
        CU(cudaMemcpyAsync(p->h_red, p->d_red, 3 * (size_t)p->G * sizeof(double), cudaMemcpyDeviceToHost,
                           p->stream));
        CU(cudaEventRecord(p->ev[5], p->stream));
        const bool ahead = it + 1 < p->opt.max_iters;
        if (ahead) {
            sa.g0 = g0;
            sa.g1 = g1;
            sa.out = srcs[cur ^ 1];
            CU(launch_scatter(sa, p->stream));
            ++p->launches;
        }
        CU(cudaEventSynchronize(p->ev[5]));
        float ms = 0.0f;
        CU(cudaEventElapsedTime(&ms, p->ev[3], p->ev[4]));
        ms_sweep += ms;
        updates += (double)p->V * p->A * gc;
        ++it;
        resid = 0.0;
        for (int g = g0; g < g1; ++g) {
            const double num = p->h_red[p->G + 2 * g], den = p->h_red[p->G + 2 * g + 1];
            eps[g] = den > 0.0 ? std::sqrt(num / den) : 0.0;
            if (!std::isfinite(eps[g])) {
                CU(cudaStreamSynchronize(p->stream));
                set_error("source iteration produced a non-finite fluence");
                return DOCTORS_ERR_INVALID_ARG;
            }
            resid = std::max(resid, eps[g]);
        }
        if (resid < tol) {
            conv = true;
            break;
        }
        if (!ahead) break;
        if (!reverse)
            while (g0 < g1 - 1 && eps[g0] < tol) ++g0;
        else
            while (g1 - 1 > g0 && eps[g1 - 1] < tol) --g1;
        cur ^= 1;
    }
    // particle balance of the last sweep (FP64)
    const double vol = p->mesh.dx * p->mesh.dy * p->mesh.dz;
    CU(launch_balance(p->V, p->G, p->M, p->d_mat, p->d_rho, p->d_sigt, srcs[cur], mom, vol, d_bal,
                      p->stream));
    ++p->launches;
    CU(cudaMemcpyAsync(p->h_red, p->d_red, 5 * (size_t)p->G * sizeof(double), cudaMemcpyDeviceToHost,
                       p->stream));
    CU(cudaStreamSynchronize(p->stream));
    double gain = 0.0, loss = 0.0;
    for (int g = 0; g < p->G; ++g) {
        gain += p->h_red[3 * p->G + 2 * g];
        loss += p->h_red[3 * p->G + 2 * g + 1] + p->h_red[g];
    }
    if (info) {
        info->iterations = it;
        info->converged = conv ? 1 : 0;
        info->residual = resid;
        info->balance_rel = gain != 0.0 ? std::fabs(gain - loss) / std::fabs(gain) : 0.0;
        info->tol_used = tol;
        info->cell_updates = updates;
        info->ms_sweep = ms_sweep;
    }
    return conv ? DOCTORS_OK : DOCTORS_ERR_NOT_CONVERGED;
}




// Source iteration of n problems as one CUDA graph: a while node whose body
// holds every problem's iteration and a decision kernel that retires
// converged problems and ends the loop on the device.
int graph_iterate(doctors_problem** ps, int n, int reverse, const float* const* Qs, float* const* moms,
                  doctors_result* infos) {
    doctors_problem* p0 = ps[0];
    cudaStream_t s = p0->stream;
    std::vector<LoopCtl> ctl(n);
    for (int q = 0; q < n; ++q) {
        ctl[q].done = 0;
        ctl[q].iters = 0;
        ctl[q].max_iters = ps[q]->opt.max_iters;
        ctl[q].G = ps[q]->G;
        ctl[q].tol = std::max(ps[q]->opt.tol, kTolFloor);
        ctl[q].resid = 0.0;
        ctl[q].res = ps[q]->d_red + ps[q]->G;
        ctl[q].reverse = reverse;
        // the dataflow sweeps (and the scattering source, zeroing and residual
        // around them) follow a device-side active-group window; the other
        // sweep kernels sweep every group at every iteration
        ctl[q].use_window = ps[q]->use_flow ? 1 : 0;
        ctl[q].win[0] = 0;
        ctl[q].win[1] = ps[q]->G;
        ctl[q].group_sweeps = 0;
    }
    LoopCtl* d_ctl = nullptr;
    int rc = dalloc_t(&d_ctl, (size_t)n, "loop control");
    if (rc) return rc;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaMemcpyAsync(d_ctl, ctl.data(), n * sizeof(LoopCtl), cudaMemcpyHostToDevice, s);
    for (int q = 0; q < n && e == cudaSuccess; ++q) {
        e = cudaMemsetAsync(moms[q], 0, (size_t)ps[q]->G * ps[q]->V * ps[q]->M * sizeof(float), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(ps[q]->d_prev, 0, (size_t)ps[q]->G * ps[q]->V * sizeof(float), s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaGraphCreate(&graph, 0);
    cudaGraphConditionalHandle handle{};
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
    cudaGraph_t body = nullptr;
    if (e == cudaSuccess) {
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
        if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
    }
    long long per_iter_launches = 1;
    // independent instances run on parallel branches of the body: the
    // capture forks onto up to kBranches side streams and joins before the
    // decision kernel
    constexpr int kBranches = 8;
    const int nb = std::min(n, kBranches);
    cudaStream_t side[kBranches] = {};
    cudaEvent_t fork = nullptr, join[kBranches] = {};
    for (int b = 0; b < nb && e == cudaSuccess; ++b) {
        e = cudaStreamCreateWithFlags(&side[b], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        if (nb > 1) {
            e = cudaEventRecord(fork, cap);
            for (int b = 0; b < nb && e == cudaSuccess; ++b) e = cudaStreamWaitEvent(side[b], fork, 0);
        }
        for (int q = 0; q < n && e == cudaSuccess; ++q) {
            doctors_problem* p = ps[q];
            const int* skip = &d_ctl[q].done;
            cudaStream_t cs = nb > 1 ? side[q % nb] : cap;
            ScatterArgs sa{};
            sa.V = p->V; sa.G = p->G; sa.M = p->M; sa.L = p->L; sa.nmat = p->nmat; sa.transpose = reverse;
            sa.mat = p->d_mat; sa.rho = p->d_rho; sa.sigs = p->d_sigs;
            sa.base = Qs[q]; sa.phi = moms[q]; sa.out = p->d_src; sa.skip = skip;
            const int* win = p->use_flow ? d_ctl[q].win : nullptr;
            sa.win = win;
            e = launch_scatter(sa, cs);
            if (e == cudaSuccess && win)
                e = launch_zero_window(moms[q], (size_t)p->V * p->M, p->G, win, skip, cs);
            else if (e == cudaSuccess && !p->use_split)
                e = launch_zero(moms[q], (size_t)p->G * p->V * p->M, skip, cs);
            // leakage [G] (a retired group keeps its last sweep's, for the balance),
            // then the residual and balance sums [4G]
            if (e == cudaSuccess && win) e = launch_zero_window(p->d_red, 1, p->G, win, skip, cs);
            else if (e == cudaSuccess) e = launch_zero(p->d_red, (size_t)p->G, skip, cs);
            if (e == cudaSuccess) e = launch_zero(p->d_red + p->G, 4 * (size_t)p->G, skip, cs);
            SweepArgs sw = sweep_args(p, reverse, p->d_src, moms[q]);
            sw.skip = skip;
            sw.win = win;
            // two instances' dataflow sweeps share the resident CTA slots, so
            // one's wavefront fill and drain overlap the other's full stages
            // (measured on the axial-scan batch: sharing among 2, 4 and 8 took
            // 2025, 2058 and 2233 ms against 2038 ms without sharing; more
            // instances at once spill each other's working sets out of L2)
            sw.slot_share = std::min(nb, 2);
            int nl = 0;
            if (e == cudaSuccess) e = launch_sweep(p, sw, 0, cs, &nl);
            if (e == cudaSuccess)
                e = launch_residual(p->V, p->G, p->M, moms[q], p->d_prev, p->d_red + p->G, cs, skip, 0, -1, win);
            per_iter_launches += 4 + nl;
        }
        if (nb > 1) {
            for (int b = 0; b < nb && e == cudaSuccess; ++b) {
                e = cudaEventRecord(join[b], side[b]);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, join[b], 0);
            }
        }
        if (e == cudaSuccess) e = launch_decide(d_ctl, n, (unsigned long long)handle, cap);
        cudaGraph_t captured = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cap, &captured);
        if (e == cudaSuccess) e = e2;
    }
    for (int b = 0; b < nb; ++b) {
        if (join[b]) cudaEventDestroy(join[b]);
        if (side[b]) cudaStreamDestroy(side[b]);
    }
    if (fork) cudaEventDestroy(fork);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctl.data(), d_ctl, n * sizeof(LoopCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    cudaFree(d_ctl);
    if (e != cudaSuccess) {
        set_error(std::string("device-side iteration graph: ") + cudaGetErrorString(e));
        return DOCTORS_ERR_CUDA;
    }
    int worst = DOCTORS_OK;
    int max_it = 0;
    for (int q = 0; q < n; ++q) max_it = std::max(max_it, ctl[q].iters);
    for (int q = 0; q < n; ++q) {
        doctors_problem* p = ps[q];
        if (!std::isfinite(ctl[q].resid)) {
            set_error("source iteration produced a non-finite fluence");
            return DOCTORS_ERR_INVALID_ARG;
        }
        // particle balance of the last sweep (FP64)
        const double vol = p->mesh.dx * p->mesh.dy * p->mesh.dz;
        double* d_bal = p->d_red + 3 * p->G;
        CU(cudaMemsetAsync(d_bal, 0, 2 * (size_t)p->G * sizeof(double), s));
        CU(launch_balance(p->V, p->G, p->M, p->d_mat, p->d_rho, p->d_sigt, p->d_src, moms[q], vol, d_bal, s));
        CU(cudaMemcpyAsync(p->h_red, p->d_red, 5 * (size_t)p->G * sizeof(double), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        double gain = 0.0, loss = 0.0;
        for (int g = 0; g < p->G; ++g) {
            gain += p->h_red[3 * p->G + 2 * g];
            loss += p->h_red[3 * p->G + 2 * g + 1] + p->h_red[g];
        }
        const bool conv = ctl[q].resid < ctl[q].tol;
        if (infos) {
            doctors_result& r = infos[q];
            r.iterations = ctl[q].iters;
            r.converged = conv ? 1 : 0;
            r.residual = ctl[q].resid;
            r.balance_rel = gain != 0.0 ? std::fabs(gain - loss) / std::fabs(gain) : 0.0;
            r.tol_used = ctl[q].tol;
            r.cell_updates = (double)ctl[q].group_sweeps * (double)p->V * p->A;
            r.ms_sweep = -1.0;   // not separable inside the graph
        }
        p->launches += (long long)max_it * per_iter_launches / n + 1;
        if (!conv) worst = DOCTORS_ERR_NOT_CONVERGED;
    }
    return worst;
}

// (Re)install a sweep schedule: tile, directions per CTA, transform path.
int configure_sweep(doctors_problem* p, int tx, int ty, int ab, int kernel) {
    if (tx < 1 || ty < 1 || tx * ty > 256) {
        set_error("tile_x * tile_y must be 1..256");
        return DOCTORS_ERR_INVALID_ARG;
    }
    if (p->A8 % ab != 0 || !(sweep_supported(ab, p->M) || flow_block_ab(p->A8, ab))) {
        set_error("angles_per_block must divide N(N+2)/8 and be one of 1,2,3,4,5,6,7,9,10,12 "
                  "(or 21 at S12, 36 at S16: whole octants, dataflow sweep only)");
        return DOCTORS_ERR_INVALID_ARG;
    }
    if (kernel < 0 || kernel > 8 || kernel == 2 || kernel == 6) {
        set_error("sweep_kernel must be 0, 1, 3, 4, 5, 7 or 8 (2 and 6 are not offered: both measured slower "
                  "on every workload)");
        return DOCTORS_ERR_INVALID_ARG;
    }
    const bool whole_octant = p->A8 == ab && chain_const_table_ab(ab);   // S2..S8
    if ((kernel == 5 || kernel == 8) && !whole_octant) {
        set_error("the split dataflow sweeps (sweep_kernel 5, 8) need whole octants per CTA "
                  "(angles_per_block = N(N+2)/8) of S2, S4, S6 or S8");
        return DOCTORS_ERR_INVALID_ARG;
    }
    if ((kernel == 4 || kernel == 7) && !flow_block_ab(p->A8, ab)) {
        set_error("the dataflow sweep (sweep_kernel 4, 7) needs whole octants per CTA (angles_per_block = "
                  "N(N+2)/8) of S2, S4, S6, S8, S12 or S16, or blocks of 12 directions (S16)");
        return DOCTORS_ERR_INVALID_ARG;
    }
    if (kernel == 7 && p->M % 4 != 0) {
        set_error("the face-warp dataflow sweep (sweep_kernel 7) needs P1 or P3 (legendre 1 or 3)");
        return DOCTORS_ERR_INVALID_ARG;
    }
    if (kernel == 8 && p->M != 16) {
        set_error("the tensor-core transforms (sweep_kernel 8) need P3 (legendre 3)");
        return DOCTORS_ERR_INVALID_ARG;
    }
    if (kernel == 7 && tx + ty > 64) {
        set_error("the face-warp dataflow sweep (sweep_kernel 7) needs tile_x + tile_y <= 64");
        return DOCTORS_ERR_INVALID_ARG;
    }
    const bool dd = p->differencing == DOCTORS_DIFF_DIAMOND;
    if (dd) {
        // diamond differencing is built into the one-group dataflow kernel only
        if (kernel != 0 && kernel != 4) {
            set_error("diamond differencing runs on the dataflow sweep (sweep_kernel 0 or 4)");
            return DOCTORS_ERR_INVALID_ARG;
        }
        if (!(p->A8 == ab && flow_octant_ab(ab))) {
            set_error("diamond differencing needs the dataflow sweep: whole octants per CTA "
                      "(angles_per_block = N(N+2)/8) of S2, S4, S6, S8, S12 or S16");
            return DOCTORS_ERR_INVALID_ARG;
        }
        kernel = 4;
    }
    // the default (sweep_kernel 0) takes the dataflow kernels for whole octants
    // of S2..S8, S12 and S16 and for S16 in blocks of 12 directions
    const bool flow_ok = flow_block_ab(p->A8, ab);
    const bool use_split = kernel == 5 || kernel == 8 || (kernel == 0 && flow_ok && kDefaultSplitSweep);
    const bool split_tc = kernel == 8 && p->M == 16;
    const bool use_flow = !use_split && (kernel == 4 || kernel == 7 ||
                                         (kernel == 0 && flow_ok && kDefaultDataflowSweep));
    const bool hw = !dd && p->M % 4 == 0 && tx + ty <= 64 &&
                    (kernel == 7 || (kernel == 0 && use_flow && kDefaultFaceWarpSweep));
    const bool use_chain = !use_flow && !use_split && (kernel == 3 || (kernel == 0 && kDefaultChainedSweep));
    if (!use_flow && !use_split && !sweep_supported(ab, p->M)) {
        set_error("whole S12 or S16 octants (angles_per_block 21, 36) run on the dataflow sweep only "
                  "(sweep_kernel 0, 4, 7)");
        return DOCTORS_ERR_INVALID_ARG;
    }
    const int ntx = (p->nx + tx - 1) / tx, nty = (p->ny + ty - 1) / ty;
    int chain_slots = 0, flow_slots = 0;
    size_t smem = 0;
    if (use_flow || use_split) {
        int sms = 0;
        CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
        smem = sweep_flow_smem_bytes(ab, tx, ty, p->G, kMaxMat, dd);
        if (smem <= 227 * 1024) {
            const int per_sm = sweep_flow_blocks_per_sm(ab, p->M, tx * ty, smem, false, dd);
            const int hw_threads = ((tx * ty + 31) / 32 + 1) * 32;
            const int per_sm_main = use_split ? sweep_flow_blocks_per_sm(ab, p->M, tx * ty, smem, true)
                                  : hw ? sweep_flow_blocks_per_sm(ab, p->M, hw_threads, smem, false, false, true)
                                       : per_sm;
            if (per_sm < 1 || per_sm_main < 1) {
                set_error("dataflow sweep cannot be resident with this tile");
                return DOCTORS_ERR_INVALID_ARG;
            }
            chain_slots = sms * per_sm_main;
            flow_slots = sms * per_sm;
        }
    } else if (use_chain) {
        // CTA slots from the occupancy at the largest chain a stage can need
        // (every chain is at most ceil(tasks / SMs) long once there is at
        // least one CTA per SM)
        int sms = 0;
        CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
        const int max_tasks = std::min(ntx, nty) * 8 * (p->A8 / ab) * p->G;
        // whole octants per CTA: direction table in the constant bank, no staged rows
        const bool ct = p->A8 == ab && chain_const_table_ab(ab);
        const int cmax = ct ? 0 : (max_tasks + sms - 1) / sms;
        smem = sweep_chain_smem_bytes(ab, tx, ty, cmax, p->G, kMaxMat);
        if (smem <= 227 * 1024) {
            const int per_sm = sweep_chain_blocks_per_sm(ab, ct, p->M, tx * ty, smem);
            if (per_sm < 1) {
                set_error("chained sweep cannot be resident with this tile");
                return DOCTORS_ERR_INVALID_ARG;
            }
            chain_slots = sms * per_sm;
        }
    } else {
        smem = sizeof(float) * (size_t)(2 * ab * tx * ty + ab * (tx + ty) * p->nz + 21 * ab + kMaxMat);
    }
    if (smem > 227 * 1024) {
        set_error("sweep tile needs more than 227 KB of shared memory");
        return DOCTORS_ERR_INVALID_ARG;
    }
    // face buffers: [8][A/8][G][tiles-1][ny or nx][nz] per direction for the
    // staged kernels; [8][G][tiles-1][ny or nx][nz][A/8 padded to 4] records
    // for the dataflow kernel
    const size_t per_dir = std::max((size_t)p->A, (size_t)8 * flow_abp_host(p->A8));
    const size_t xf = per_dir * p->G * (ntx > 1 ? ntx - 1 : 0) * p->ny * p->nz;
    const size_t yf = per_dir * p->G * (nty > 1 ? nty - 1 : 0) * p->nx * p->nz;
    if (p->d_xface == nullptr || xf * sizeof(float) > p->xface_bytes) {
        float* nb = nullptr;
        int rc = dalloc_t(&nb, xf, "x face buffer");
        if (rc) return rc;
        if (p->d_xface) cudaFree(p->d_xface);
        p->d_xface = nb;
        p->xface_bytes = xf * sizeof(float);
    }
    if (p->d_yface == nullptr || yf * sizeof(float) > p->yface_bytes) {
        float* nb = nullptr;
        int rc = dalloc_t(&nb, yf, "y face buffer");
        if (rc) return rc;
        if (p->d_yface) cudaFree(p->d_yface);
        p->d_yface = nb;
        p->yface_bytes = yf * sizeof(float);
    }
    if (use_split) {
        // angular source and fluence records of every direction, group and voxel
        const size_t nang = (size_t)p->G * 8 * p->V * flow_abp_host(p->A8);
        if (p->ang_floats < nang) {
            if (p->d_qang) cudaFree(p->d_qang);
            if (p->d_pang) cudaFree(p->d_pang);
            p->d_qang = p->d_pang = nullptr;
            p->ang_floats = 0;
            int rc = dalloc_t(&p->d_qang, nang, "angular source");
            if (!rc) rc = dalloc_t(&p->d_pang, nang, "angular fluence");
            if (rc) return rc;
            p->ang_floats = nang;
        }
    }
    if (split_tc && !p->d_tcb) {
        // operand tables of the tensor-core transforms (the first octant's rows are fixed per problem)
        std::vector<float> b1, b2;
        build_tc_transform_tables(p->dir_table, p->A8, b1, b2);
        int rc = dalloc_t(&p->d_tcb, b1.size() + b2.size(), "tensor-core transform tables");
        if (rc) return rc;
        CU(cudaMemcpy(p->d_tcb, b1.data(), b1.size() * sizeof(float), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(p->d_tcb + b1.size(), b2.data(), b2.size() * sizeof(float), cudaMemcpyHostToDevice));
        p->tcb1_floats = b1.size();
    }
    if (use_flow || use_split) {
        // every face record starts as NaN (not yet written); the queue at zero
        if (!p->d_flow) {
            int rc = dalloc_t(&p->d_flow, 4, "dataflow queue");
            if (rc) return rc;
        }
        CU(cudaMemsetAsync(p->d_flow, 0, 4 * sizeof(int), p->stream));
        if (p->xface_bytes) CU(cudaMemsetAsync(p->d_xface, 0xff, p->xface_bytes, p->stream));
        if (p->yface_bytes) CU(cudaMemsetAsync(p->d_yface, 0xff, p->yface_bytes, p->stream));
    }
    p->tx = tx; p->ty = ty; p->ab = ab; p->nab = p->A8 / ab; p->ntx = ntx; p->nty = nty;
    p->dir_blk.clear();
    if (use_flow && p->nab > 1)
        for (int b = 0; b < p->nab; ++b) p->dir_blk.push_back(make_dir_table(p, b * ab, ab));
    p->use_flow = use_flow;
    p->use_split = use_split;
    p->split_tc = use_split && split_tc;
    p->flow_hw = use_flow && hw;
    p->chain_slots = chain_slots;
    p->flow_slots = flow_slots;
    return DOCTORS_OK;
}

struct TuneKey {
    int nx, ny, nz, N, L, G, differencing;
    bool operator<(const TuneKey& o) const {
        return std::tie(nx, ny, nz, N, L, G, differencing) < std::tie(o.nx, o.ny, o.nz, o.N, o.L, o.G, o.differencing);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, doctors_tuning> g_tune_cache;

}  // namespace

extern "C" {

const char* doctors_last_error(void) { return g_err.c_str(); }

int doctors_create_problem(const doctors_mesh* mesh, const doctors_options* opt, void* cuda_stream,
                           doctors_problem** out) {
    CHECK_ARG(mesh && opt && out, "null argument");
    CHECK_ARG(mesh->nx >= 1 && mesh->ny >= 1 && mesh->nz >= 1, "mesh dimensions must be >= 1");
    CHECK_ARG((double)mesh->nx * mesh->ny * mesh->nz < 2147483647.0, "mesh has too many voxels");
    CHECK_ARG(mesh->dx > 0 && mesh->dy > 0 && mesh->dz > 0, "voxel sizes must be > 0");
    CHECK_ARG(std::isfinite(mesh->origin[0]) && std::isfinite(mesh->origin[1]) && std::isfinite(mesh->origin[2]),
              "origin must be finite");
    CHECK_ARG(opt->groups >= 1 && opt->groups <= kMaxG, "groups must be 1..64");
    CHECK_ARG(opt->legendre >= 0 && opt->legendre <= 3, "legendre must be 0..3");
    CHECK_ARG(opt->tol > 0 && std::isfinite(opt->tol), "tol must be > 0");
    CHECK_ARG(opt->max_iters >= 1, "max_iters must be >= 1");
    CHECK_ARG(opt->differencing == DOCTORS_DIFF_STEP || opt->differencing == DOCTORS_DIFF_DIAMOND,
              "differencing must be DOCTORS_DIFF_STEP or DOCTORS_DIFF_DIAMOND");
    for (int r : opt->reserved) CHECK_ARG(r == 0, "reserved option fields must be zero");
    std::vector<double> dirs, w;
    std::string err;
    if (!build_quadrature(opt->sn_order, dirs, w, err)) {
        set_error(err);
        return DOCTORS_ERR_INVALID_ARG;
    }
    auto* p = new doctors_problem();
    p->mesh = *mesh;
    p->opt = *opt;
    p->nx = mesh->nx; p->ny = mesh->ny; p->nz = mesh->nz;
    p->V = (size_t)p->nx * p->ny * p->nz;
    p->G = opt->groups; p->N = opt->sn_order; p->L = opt->legendre; p->M = (p->L + 1) * (p->L + 1);
    p->A = (int)w.size(); p->A8 = p->A / 8;
    p->dirs = dirs; p->w = w;
    p->stream = (cudaStream_t)cuda_stream;
    p->differencing = opt->differencing;
    p->ab = opt->angles_per_block > 0 ? opt->angles_per_block : default_ab(p->A8, opt->sweep_kernel);
    // default tile: 8 x 8 for the dataflow sweep (whole octants of S2..S8 and
    // S12, S16, or S16 in blocks of 12), 16 x 16 for the stage kernels (the fastest
    // measured shapes)
    const bool flow_default = opt->sweep_kernel >= 4 || p->differencing == DOCTORS_DIFF_DIAMOND ||
                              (opt->sweep_kernel == 0 && kDefaultDataflowSweep && flow_block_ab(p->A8, p->ab));
    const int tdef = flow_default ? 8 : 16;
    p->tx = opt->tile_x > 0 ? opt->tile_x : std::min(tdef, p->nx);
    p->ty = opt->tile_y > 0 ? opt->tile_y : std::min(tdef, p->ny);
    auto fail = [&](int code, const std::string& msg) {
        if (!msg.empty()) set_error(msg);
        free_problem(p);
        delete p;
        return code;
    };
    if (p->tx * p->ty > 256 || p->tx < 1 || p->ty < 1) return fail(DOCTORS_ERR_INVALID_ARG, "tile_x * tile_y must be 1..256");
    if (p->A8 % p->ab != 0 || !(sweep_supported(p->ab, p->M) || flow_block_ab(p->A8, p->ab)))
        return fail(DOCTORS_ERR_INVALID_ARG, "angles_per_block must divide N(N+2)/8 and be one of "
                                             "1,2,3,4,5,6,7,9,10,12 (or 21 at S12, 36 at S16: whole octants, dataflow sweep only)");
    if ((opt->sweep_kernel == 1 || opt->sweep_kernel == 3) && !sweep_supported(p->ab, p->M))
        return fail(DOCTORS_ERR_INVALID_ARG,
                    "whole S12 or S16 octants (angles_per_block 21, 36) run on the dataflow sweep only "
                    "(sweep_kernel 0, 4, 7)");
    p->nab = p->A8 / p->ab;
    p->ntx = (p->nx + p->tx - 1) / p->tx;
    p->nty = (p->ny + p->ty - 1) / p->ty;
    if (opt->sweep_kernel < 0 || opt->sweep_kernel > 8)
        return fail(DOCTORS_ERR_INVALID_ARG, "sweep_kernel must be 0, 1, 3, 4, 5, 7 or 8");
    if (opt->sweep_kernel == 2 || opt->sweep_kernel == 6)
        return fail(DOCTORS_ERR_INVALID_ARG, "sweep_kernel 2 and 6 are not offered (both measured slower on every workload)");
    if (p->differencing == DOCTORS_DIFF_DIAMOND &&
        !((opt->sweep_kernel == 0 || opt->sweep_kernel == 4) && p->A8 == p->ab && flow_octant_ab(p->ab)))
        return fail(DOCTORS_ERR_INVALID_ARG,
                    "diamond differencing runs on the dataflow sweep: sweep_kernel 0 or 4, angles_per_block = "
                    "N(N+2)/8 and N <= 8, N = 12 or N = 16");
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) return fail(DOCTORS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));

    // sweep tables
    const int A = p->A, M = p->M;
    std::vector<float> coef((size_t)A * 8, 0.0f);
    const double dx = mesh->dx, dy = mesh->dy, dz = mesh->dz;
    for (int n = 0; n < A; ++n) {
        const double ox = std::fabs(dirs[3 * n]), oy = std::fabs(dirs[3 * n + 1]), oz = std::fabs(dirs[3 * n + 2]);
        coef[n * 8 + 0] = (float)(ox / dx);
        coef[n * 8 + 1] = (float)(oy / dy);
        coef[n * 8 + 2] = (float)(oz / dz);
        coef[n * 8 + 3] = (float)(ox / dx + oy / dy + oz / dz);
        coef[n * 8 + 4] = (float)(w[n] * ox * dy * dz);
        coef[n * 8 + 5] = (float)(w[n] * oy * dx * dz);
        coef[n * 8 + 6] = (float)(w[n] * oz * dx * dy);
        coef[n * 8 + 7] = (float)w[n];
    }
    // first-octant direction table of the chained sweep; check that every
    // octant's harmonics are the first octant's with the reflection signs
    {
        ChainDirTable& t = p->dir_table;
        double Rb[16], Rn[16];
        for (int n = 0; n < A; ++n) {
            const int o = n / p->A8, j = n % p->A8;
            real_harmonics(3, dirs[3 * j], dirs[3 * j + 1], dirs[3 * j + 2], Rb);
            real_harmonics(3, dirs[3 * n], dirs[3 * n + 1], dirs[3 * n + 2], Rn);
            for (int lm = 0; lm < 16; ++lm) {
                const bool flip = (((o & 1) && ((kOddX >> lm) & 1u)) != 0) ^ (((o & 2) && ((kOddY >> lm) & 1u)) != 0) ^
                                  (((o & 4) && ((kOddZ >> lm) & 1u)) != 0);
                if (std::fabs(Rn[lm] - (flip ? -Rb[lm] : Rb[lm])) > 1e-12)
                    return fail(DOCTORS_ERR_INVALID_ARG, "quadrature octants are not reflections of the first");
            }
        }
        t = make_dir_table(p, 0, p->A8);
    }
    const size_t GV = (size_t)p->G * p->V, GVM = GV * M;
    int rc = 0;
    rc = rc ? rc : dalloc_t(&p->d_coef, coef.size(), "tables");
    rc = rc ? rc : dalloc_t(&p->d_mat, p->V, "materials");
    rc = rc ? rc : dalloc_t(&p->d_rho, p->V, "densities");
    rc = rc ? rc : dalloc_t(&p->d_sig, (size_t)p->G * p->V, "total cross sections per cell");
    rc = rc ? rc : dalloc_t(&p->d_sigt, (size_t)kMaxMat * p->G, "sigma_t");
    rc = rc ? rc : dalloc_t(&p->d_sigs, (size_t)kMaxMat * (p->L + 1) * p->G * p->G, "sigma_s");
    rc = rc ? rc : dalloc_t(&p->d_phiu_src, GV, "uncollided (source)");
    rc = rc ? rc : dalloc_t(&p->d_phiu, GV, "uncollided");
    rc = rc ? rc : dalloc_t(&p->d_U, GVM, "uncollided moments");
    rc = rc ? rc : dalloc_t(&p->d_Q, GVM, "first-collision source");
    rc = rc ? rc : dalloc_t(&p->d_mom, GVM, "moments");
    rc = rc ? rc : dalloc_t(&p->d_src, GVM, "sweep source");
    rc = rc ? rc : dalloc_t(&p->d_src2, GVM, "sweep source (next iteration)");
    rc = rc ? rc : dalloc_t(&p->d_prev, GV, "previous scalar fluence");
    rc = rc ? rc : dalloc_t(&p->d_iso, (size_t)p->G, "volume source");
    p->dir_table.sig = p->d_sig;   // the whole-octant table also carries the per-cell cross sections
    rc = rc ? rc : configure_sweep(p, p->tx, p->ty, p->ab, opt->sweep_kernel);
    rc = rc ? rc : dalloc_t(&p->d_red, 5 * (size_t)p->G, "reductions");
    if (rc) return fail(rc, "");
    e = cudaMallocHost(&p->h_red, 5 * (size_t)p->G * sizeof(double));
    if (e != cudaSuccess) return fail(DOCTORS_ERR_OOM, "pinned host allocation failed");
    for (auto& ev : p->ev) {
        e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return fail(DOCTORS_ERR_CUDA, "cudaEventCreate failed");
    }
    e = ensure_direction_tables(p->device, p->N, &p->table_base);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->d_coef, coef.data(), coef.size() * sizeof(float), cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return fail(DOCTORS_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(e));
    *out = p;
    return DOCTORS_OK;
}

int doctors_set_materials(doctors_problem* p, int n_mat, const uint8_t* mat, const float* density,
                          const double* sigma_t, const double* sigma_s, int mem) {
    int rc = check_problem(p);
    if (rc) return rc;
    CHECK_ARG(n_mat >= 1 && n_mat <= kMaxMat, "n_mat must be 1..8");
    CHECK_ARG(mat && sigma_t && sigma_s, "null material table");
    CHECK_ARG(mem == DOCTORS_MEM_HOST || mem == DOCTORS_MEM_DEVICE, "mem must be DOCTORS_MEM_HOST or _DEVICE");
    const int G = p->G, L = p->L;
    for (int m = 0; m < n_mat; ++m)
        for (int g = 0; g < G; ++g) {
            const double st = sigma_t[m * G + g];
            CHECK_ARG(std::isfinite(st) && st >= 0, "sigma_t must be finite and >= 0");
            double out0 = 0.0;
            for (int l = 0; l <= L; ++l)
                for (int gt = 0; gt < G; ++gt) {
                    const double s = sigma_s[(((size_t)m * (L + 1) + l) * G + g) * G + gt];
                    CHECK_ARG(std::isfinite(s), "sigma_s must be finite");
                    if (gt < g) CHECK_ARG(s == 0.0, "sigma_s has upscatter (to < from)");
                    if (l == 0) {
                        CHECK_ARG(s >= 0.0, "sigma_s,0 must be >= 0");
                        out0 += s;
                    }
                }
            CHECK_ARG(out0 <= st * (1.0 + 1e-12), "sum of sigma_s,0 out of a group exceeds sigma_t");
        }
    // voxel arrays: validate on the host
    std::vector<uint8_t> hm(p->V);
    std::vector<float> hr(p->V, 1.0f);
    if (mem == DOCTORS_MEM_HOST) {
        std::memcpy(hm.data(), mat, p->V);
        if (density) std::memcpy(hr.data(), density, p->V * sizeof(float));
    } else {
        CU(cudaMemcpy(hm.data(), mat, p->V, cudaMemcpyDeviceToHost));
        if (density) CU(cudaMemcpy(hr.data(), density, p->V * sizeof(float), cudaMemcpyDeviceToHost));
    }
    for (size_t v = 0; v < p->V; ++v) {
        CHECK_ARG(hm[v] < n_mat, "material id out of range");
        CHECK_ARG(std::isfinite(hr[v]) && hr[v] >= 0.0f, "density must be finite and >= 0");
    }
    std::vector<float> st((size_t)n_mat * G), ss((size_t)n_mat * (L + 1) * G * G);
    for (size_t q = 0; q < st.size(); ++q) st[q] = (float)sigma_t[q];
    for (size_t q = 0; q < ss.size(); ++q) ss[q] = (float)sigma_s[q];
    CU(cudaMemcpyAsync(p->d_mat, hm.data(), p->V, cudaMemcpyHostToDevice, p->stream));
    CU(cudaMemcpyAsync(p->d_rho, hr.data(), p->V * sizeof(float), cudaMemcpyHostToDevice, p->stream));
    CU(cudaMemcpyAsync(p->d_sigt, st.data(), st.size() * sizeof(float), cudaMemcpyHostToDevice, p->stream));
    CU(cudaMemcpyAsync(p->d_sigs, ss.data(), ss.size() * sizeof(float), cudaMemcpyHostToDevice, p->stream));
    CU(launch_total_xs(p->V, G, p->d_mat, p->d_rho, p->d_sigt, p->d_sig, p->stream));
    CU(cudaStreamSynchronize(p->stream));
    p->nmat = n_mat;
    p->h_sigt.assign(sigma_t, sigma_t + (size_t)n_mat * G);
    p->h_sigs.assign(sigma_s, sigma_s + ss.size());
    p->have_mat = true;
    p->solved = false;
    p->adjoint_done = false;
    return DOCTORS_OK;
}

int doctors_set_source(doctors_problem* p, int n_src, const doctors_source* src) {
    int rc = check_problem(p);
    if (rc) return rc;
    CHECK_ARG(n_src >= 1 && n_src <= kMaxSrc, "n_src must be 1..4096");
    CHECK_ARG(src != nullptr, "null source array");
    std::vector<doctors_source> list(src, src + n_src);
    std::vector<std::vector<double>> spec(n_src);
    const double lo[3] = {p->mesh.origin[0], p->mesh.origin[1], p->mesh.origin[2]};
    const double hi[3] = {lo[0] + p->nx * p->mesh.dx, lo[1] + p->ny * p->mesh.dy, lo[2] + p->nz * p->mesh.dz};
    for (int s = 0; s < n_src; ++s) {
        doctors_source& q = list[s];
        CHECK_ARG(q.kind == DOCTORS_SRC_POINT || q.kind == DOCTORS_SRC_FAN_CONE || q.kind == DOCTORS_SRC_VOLUME,
                  "unknown source kind");
        CHECK_ARG(q.spectrum != nullptr, "null spectrum");
        CHECK_ARG(std::isfinite(q.weight) && q.weight >= 0, "source weight must be finite and >= 0");
        spec[s].assign(q.spectrum, q.spectrum + p->G);
        for (double x : spec[s]) CHECK_ARG(std::isfinite(x) && x >= 0, "spectrum must be finite and >= 0");
        q.spectrum = nullptr;
        if (q.kind == DOCTORS_SRC_VOLUME) continue;
        for (int d = 0; d < 3; ++d) CHECK_ARG(std::isfinite(q.pos[d]), "source position must be finite");
        const bool inside = q.pos[0] >= lo[0] && q.pos[0] <= hi[0] && q.pos[1] >= lo[1] && q.pos[1] <= hi[1] &&
                            q.pos[2] >= lo[2] && q.pos[2] <= hi[2];
        CHECK_ARG(!inside, "point sources must lie outside the mesh");
        if (q.kind == DOCTORS_SRC_FAN_CONE) {
            const double n = std::sqrt(q.axis[0] * q.axis[0] + q.axis[1] * q.axis[1] + q.axis[2] * q.axis[2]);
            CHECK_ARG(n > 0 && std::isfinite(n), "collimator axis must be non-zero");
            CHECK_ARG(std::fabs(n - 1.0) < 1e-9, "collimator axis must be a unit vector");
            CHECK_ARG(q.fan_deg > 0 && q.fan_deg < 180, "fan_deg must be in (0, 180)");
            CHECK_ARG(q.z_half_iso >= 0 && q.iso_dist > 0, "z_half_iso >= 0 and iso_dist > 0 required");
        }
    }
    p->srcs = list;
    p->spectra = spec;
    p->have_src = true;
    p->solved = false;
    p->adjoint_done = false;
    return DOCTORS_OK;
}

int doctors_solve(doctors_problem* p, doctors_result* info) {
    int rc = check_problem(p);
    if (rc) return rc;
    if (!p->have_mat || !p->have_src) {
        set_error("set materials and sources before solving");
        return DOCTORS_ERR_STATE;
    }
    doctors_result r{};
    p->solved = false;
    p->adjoint_done = false;
    p->launches = 0;
    CU(cudaEventRecord(p->ev[0], p->stream));
    rc = first_collision(p);
    if (rc) return rc;
    CU(cudaEventRecord(p->ev[1], p->stream));
    if (p->opt.device_loop) {
        doctors_problem* list[1] = {p};
        const float* Qs[1] = {p->d_Q};
        float* moms[1] = {p->d_mom};
        rc = graph_iterate(list, 1, 0, Qs, moms, &r);
    } else {
        rc = iterate(p, 0, p->d_Q, p->d_mom, &r);
    }
    if (rc && rc != DOCTORS_ERR_NOT_CONVERGED) return rc;
    CU(cudaEventRecord(p->ev[2], p->stream));
    CU(cudaEventSynchronize(p->ev[2]));
    float t01 = 0, t12 = 0, t02 = 0;
    cudaEventElapsedTime(&t01, p->ev[0], p->ev[1]);
    cudaEventElapsedTime(&t12, p->ev[1], p->ev[2]);
    cudaEventElapsedTime(&t02, p->ev[0], p->ev[2]);
    r.ms_raytrace = t01;
    r.ms_iterate = t12;
    r.ms_total = t02;
    r.launches = p->launches;
    if (info) *info = r;
    const int frc = check_flow(p);
    if (frc) return frc;
    p->solved = true;
    if (rc == DOCTORS_ERR_NOT_CONVERGED) set_error("iteration cap reached before convergence");
    return rc;
}

int doctors_get_fluence(doctors_problem* p, int which, float* out, int mem) {
    int rc = check_problem(p);
    if (rc) return rc;
    CHECK_ARG(out != nullptr, "null output");
    CHECK_ARG(which >= 0 && which <= 3, "which must be UNCOLLIDED, COLLIDED, TOTAL or ADJOINT");
    CHECK_ARG(mem == DOCTORS_MEM_HOST || mem == DOCTORS_MEM_DEVICE, "bad mem");
    if (!p->solved) {
        set_error("no solution: call doctors_solve first");
        return DOCTORS_ERR_STATE;
    }
    if (which == DOCTORS_FLUENCE_ADJOINT && !p->adjoint_done) {
        set_error("no adjoint solution: call doctors_adjoint_solve first");
        return DOCTORS_ERR_STATE;
    }
    const int mask = which == DOCTORS_FLUENCE_UNCOLLIDED ? 1 : which == DOCTORS_FLUENCE_TOTAL ? 3 : 2;
    const float* mom = which == DOCTORS_FLUENCE_ADJOINT ? p->d_Z : p->d_mom;
    const size_t GV = (size_t)p->G * p->V;
    if (mem == DOCTORS_MEM_DEVICE) {
        CU(launch_extract(p->V, p->G, p->M, mask, p->d_phiu, mom, out, p->stream));
        return DOCTORS_OK;
    }
    // stage through the (now free) source buffer
    CU(launch_extract(p->V, p->G, p->M, mask, p->d_phiu, mom, p->d_src, p->stream));
    CU(cudaMemcpyAsync(out, p->d_src, GV * sizeof(float), cudaMemcpyDeviceToHost, p->stream));
    CU(cudaStreamSynchronize(p->stream));
    return DOCTORS_OK;
}

int doctors_dose(doctors_problem* p, const double* k, double* dose, int mem) {
    int rc = check_problem(p);
    if (rc) return rc;
    CHECK_ARG(k && dose, "null argument");
    CHECK_ARG(mem == DOCTORS_MEM_HOST || mem == DOCTORS_MEM_DEVICE, "bad mem");
    if (!p->solved) {
        set_error("no solution: call doctors_solve first");
        return DOCTORS_ERR_STATE;
    }
    for (int q = 0; q < p->nmat * p->G; ++q) CHECK_ARG(std::isfinite(k[q]), "k must be finite");
    // the factor table and the host-output staging stay allocated between calls
    if (!p->d_k) rc = dalloc_t(&p->d_k, (size_t)kMaxMat * p->G, "dose factors");
    if (!rc && mem == DOCTORS_MEM_HOST && !p->d_dose_stage) rc = dalloc_t(&p->d_dose_stage, p->V, "dose staging");
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(p->d_k, k, (size_t)p->nmat * p->G * sizeof(double), cudaMemcpyHostToDevice,
                                    p->stream);
    double* dst = mem == DOCTORS_MEM_HOST ? p->d_dose_stage : dose;
    if (e == cudaSuccess)
        e = launch_dose(p->V, p->G, p->M, p->d_mat, p->d_rho, p->d_k, p->d_phiu, p->d_mom, dst, p->stream);
    if (e == cudaSuccess && mem == DOCTORS_MEM_HOST)
        e = cudaMemcpyAsync(dose, p->d_dose_stage, p->V * sizeof(double), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
        set_error(std::string("dose: ") + cudaGetErrorString(e));
        return DOCTORS_ERR_CUDA;
    }
    return DOCTORS_OK;
}

int doctors_debug_withhold_faces(doctors_problem* p, int task) {
    int rc = check_problem(p);
    if (rc) return rc;
    if (!(p->use_flow || p->use_split) || !p->d_flow) {
        set_error("the problem's sweep is not the dataflow kernel");
        return DOCTORS_ERR_STATE;
    }
    const int v = task < 0 ? 0 : task + 1;
    CU(cudaMemcpyAsync(p->d_flow + 3, &v, sizeof(int), cudaMemcpyHostToDevice, p->stream));
    CU(cudaStreamSynchronize(p->stream));
    return DOCTORS_OK;
}

int doctors_debug_ray_indices(doctors_problem* p, int src, int voxel, int32_t* idx, float* len, int cap, int* n) {
    int rc = check_problem(p);
    if (rc) return rc;
    CHECK_ARG(p->have_mat && p->have_src, "set materials and sources first");
    CHECK_ARG(src >= 0 && src < (int)p->srcs.size(), "source index out of range");
    CHECK_ARG(p->srcs[src].kind != DOCTORS_SRC_VOLUME, "not a point source");
    CHECK_ARG(voxel >= 0 && (size_t)voxel < p->V, "voxel index out of range");
    CHECK_ARG(idx && len && n && cap >= 0, "null output");
    const int dcap = p->nx + p->ny + p->nz + 4;
    int32_t* d_idx = nullptr;
    float* d_len = nullptr;
    int* d_cnt = nullptr;
    rc = dalloc_t(&d_idx, dcap, "debug ray");
    if (!rc) rc = dalloc_t(&d_len, dcap, "debug ray");
    if (!rc) rc = dalloc_t(&d_cnt, 1, "debug ray");
    if (rc) {
        cudaFree(d_idx); cudaFree(d_len); cudaFree(d_cnt);
        return rc;
    }
    RayArgs r = ray_args(p, p->srcs[src], nullptr);
    int cnt = 0;
    cudaError_t e = launch_debug_ray(r, voxel, d_idx, d_len, dcap, d_cnt, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, d_cnt, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e == cudaSuccess && cnt <= cap && cnt <= dcap) {
        e = cudaMemcpy(idx, d_idx, cnt * sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(len, d_len, cnt * sizeof(float), cudaMemcpyDeviceToHost);
    }
    cudaFree(d_idx); cudaFree(d_len); cudaFree(d_cnt);
    if (e != cudaSuccess) {
        set_error(std::string("debug ray: ") + cudaGetErrorString(e));
        return DOCTORS_ERR_CUDA;
    }
    *n = cnt;
    if (cnt > cap) {
        set_error("capacity too small for the ray's index list");
        return DOCTORS_ERR_INVALID_ARG;
    }
    return DOCTORS_OK;
}

int doctors_solve_batch(doctors_problem** problems, int n, doctors_result* results) {
    CHECK_ARG(problems && n >= 1, "empty batch");
    for (int q = 0; q < n; ++q) {
        CHECK_ARG(problems[q] != nullptr, "null problem in batch");
        CHECK_ARG(problems[q]->device == problems[0]->device, "batch problems must share one device");
        for (int r = 0; r < q; ++r) CHECK_ARG(problems[r] != problems[q], "a problem appears twice in the batch");
        if (!problems[q]->have_mat || !problems[q]->have_src) {
            set_error("set materials and sources of every batch problem before solving");
            return DOCTORS_ERR_STATE;
        }
    }
    doctors_problem* p0 = problems[0];
    int rc = check_problem(p0);
    if (rc) return rc;
    CU(cudaEventRecord(p0->ev[0], p0->stream));
    for (int q = 0; q < n; ++q) {
        problems[q]->solved = false;
        problems[q]->adjoint_done = false;
        problems[q]->launches = 0;
        CU(cudaStreamSynchronize(p0->stream));
        rc = first_collision(problems[q]);
        if (rc) return rc;
    }
    CU(cudaEventRecord(p0->ev[1], p0->stream));
    std::vector<const float*> Qs(n);
    std::vector<float*> moms(n);
    for (int q = 0; q < n; ++q) {
        Qs[q] = problems[q]->d_Q;
        moms[q] = problems[q]->d_mom;
    }
    std::vector<doctors_result> res(n);
    rc = graph_iterate(problems, n, 0, Qs.data(), moms.data(), res.data());
    if (rc && rc != DOCTORS_ERR_NOT_CONVERGED) return rc;
    CU(cudaEventRecord(p0->ev[2], p0->stream));
    CU(cudaEventSynchronize(p0->ev[2]));
    float t01 = 0, t12 = 0, t02 = 0;
    cudaEventElapsedTime(&t01, p0->ev[0], p0->ev[1]);
    cudaEventElapsedTime(&t12, p0->ev[1], p0->ev[2]);
    cudaEventElapsedTime(&t02, p0->ev[0], p0->ev[2]);
    for (int q = 0; q < n; ++q) {
        res[q].ms_raytrace = t01;
        res[q].ms_iterate = t12;
        res[q].ms_total = t02;
        res[q].launches = problems[q]->launches;
        if (results) results[q] = res[q];
    }
    for (int q = 0; q < n; ++q) {
        const int frc = check_flow(problems[q]);
        if (frc) return frc;
        problems[q]->solved = true;
    }
    if (rc == DOCTORS_ERR_NOT_CONVERGED) set_error("iteration cap reached before convergence");
    return rc;
}

int doctors_autotune(doctors_problem* p, doctors_tuning* out) {
    int rc = check_problem(p);
    if (rc) return rc;
    if (!p->have_mat || !p->have_src) {
        set_error("set materials and sources before autotuning");
        return DOCTORS_ERR_STATE;
    }
    const TuneKey key{p->nx, p->ny, p->nz, p->N, p->L, p->G, p->differencing};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            doctors_tuning t = it->second;
            rc = configure_sweep(p, t.tile_x, t.tile_y, t.angles_per_block, t.sweep_kernel);
            if (rc) return rc;
            t.candidates = 0;
            if (out) *out = t;
            p->solved = false;
            return DOCTORS_OK;
        }
    }
    p->solved = false;
    p->launches = 0;
    rc = first_collision(p);
    if (rc) return rc;
    const int tiles[][2] = {{16, 16}, {32, 8}, {16, 8}, {8, 16}, {8, 8}, {32, 4}, {16, 4}, {8, 4}, {4, 8}};
    const int abs_c[] = {36, 12, 10, 9, 7, 6, 5, 4, 3, 2, 1};
    std::vector<int> abs_ok;
    for (int ab : abs_c)
        if (p->A8 % ab == 0 && (int)abs_ok.size() < 3) abs_ok.push_back(ab);
    doctors_tuning best{};
    best.ms_per_sweep = 1e30;
    int count = 0;
    const int saved[4] = {p->tx, p->ty, p->ab,
                          p->use_split ? (p->split_tc ? 8 : 5) : p->use_flow ? (p->flow_hw ? 7 : 4)
                                                                          : (p->chain_slots > 0 ? 3 : 1)};
    for (const auto& t : tiles) {
        for (int ab : abs_ok) {
            for (int kernel = 1; kernel <= 8; ++kernel) {
                if (p->differencing == DOCTORS_DIFF_DIAMOND && kernel != 4) continue;
                if (kernel == 2 || kernel == 6) continue;
                if ((kernel == 1 || kernel == 3) && !sweep_supported(ab, p->M)) continue;
                if ((kernel == 5 || kernel == 8) && !(p->A8 == ab && chain_const_table_ab(ab))) continue;
                if ((kernel == 4 || kernel == 7) && !flow_block_ab(p->A8, ab)) continue;
                if (configure_sweep(p, t[0], t[1], ab, kernel) != DOCTORS_OK) continue;
                SweepArgs sw = sweep_args(p, 0, p->d_Q, p->d_mom);
                float total = 0.0f;
                cudaError_t e = cudaSuccess;
                for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
                    e = cudaMemsetAsync(p->d_mom, 0, (size_t)p->G * p->V * p->M * sizeof(float), p->stream);
                    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_red, 0, 5 * (size_t)p->G * sizeof(double), p->stream);
                    if (e == cudaSuccess) e = cudaEventRecord(p->ev[3], p->stream);
                    int nl = 0;
                    if (e == cudaSuccess) e = launch_sweep(p, sw, 0, p->stream, &nl);
                    if (e == cudaSuccess) e = cudaEventRecord(p->ev[4], p->stream);
                    if (e == cudaSuccess) e = cudaEventSynchronize(p->ev[4]);
                    float ms = 0.0f;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p->ev[3], p->ev[4]);
                    if (rep > 0) total += ms;   // first repetition is a warm-up
                }
                if (e != cudaSuccess) {
                    set_error(std::string("autotune: ") + cudaGetErrorString(e));
                    return DOCTORS_ERR_CUDA;
                }
                const int frc = check_flow(p);
                if (frc) return frc;
                ++count;
                const double ms = total / 2.0;
                if (ms < best.ms_per_sweep) {
                    best.tile_x = t[0]; best.tile_y = t[1]; best.angles_per_block = ab; best.sweep_kernel = kernel;
                    best.ms_per_sweep = ms;
                }
            }
        }
    }
    if (count == 0) {
        configure_sweep(p, saved[0], saved[1], saved[2], saved[3]);
        set_error("autotune: no valid schedule");
        return DOCTORS_ERR_INVALID_ARG;
    }
    rc = configure_sweep(p, best.tile_x, best.tile_y, best.angles_per_block, best.sweep_kernel);
    if (rc) return rc;
    best.candidates = count;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = best;
    }
    if (out) *out = best;
    return DOCTORS_OK;
}

void doctors_destroy(doctors_problem* p) {
    if (!p) return;
    cudaSetDevice(p->device);
    if (p->stream) cudaStreamSynchronize(p->stream);
    free_problem(p);
    delete p;
}

}  // extern "C"

namespace {

// one full sweep (all stages) of `src` into the zeroed accumulator `mom`
int sweep_once(doctors_problem* p, int reverse, int mode, const float* src, float* mom) {
    CU(cudaMemsetAsync(mom, 0, (size_t)p->G * p->V * p->M * sizeof(float), p->stream));
    CU(cudaMemsetAsync(p->d_red, 0, 5 * (size_t)p->G * sizeof(double), p->stream));
    SweepArgs sw = sweep_args(p, reverse, src, mom);
    sw.psi = p->d_psi;
    sw.prod = p->d_prod;
    int nl = 0;
    CU(launch_sweep(p, sw, mode, p->stream, &nl));
    p->launches += nl;
    return DOCTORS_OK;
}

int ensure_adjoint_buffers(doctors_problem* p, bool density) {
    const size_t GV = (size_t)p->G * p->V, GVM = GV * p->M;
    int rc = 0;
    if (!p->d_Z) rc = rc ? rc : dalloc_t(&p->d_Z, GVM, "adjoint moments");
    if (!p->d_Qa) rc = rc ? rc : dalloc_t(&p->d_Qa, GVM, "adjoint source");
    if (!p->d_T) rc = rc ? rc : dalloc_t(&p->d_T, GVM, "adjoint scattering");
    if (!p->d_rf) rc = rc ? rc : dalloc_t(&p->d_rf, GV, "response");
    if (!p->d_r) rc = rc ? rc : dalloc_t(&p->d_r, GV, "response");
    if (!p->d_acc) rc = rc ? rc : dalloc_t(&p->d_acc, 2 * (size_t)p->G, "gradient sums");
    if (!p->d_ones) rc = rc ? rc : dalloc_t(&p->d_ones, (size_t)p->G, "unit emission");
    if (!p->d_grad) rc = rc ? rc : dalloc_t(&p->d_grad, p->V, "density gradient");
    if (density) {
        if (!p->d_H) rc = rc ? rc : dalloc_t(&p->d_H, (size_t)kMaxMat * p->V, "ray importance");
        // [G][V][A] for the stage kernels, [G][V][8][A/8 padded to 4] for the dataflow kernel
        if (!p->d_psi)
            rc = rc ? rc : dalloc_t(&p->d_psi, GV * std::max((size_t)p->A, (size_t)8 * flow_abp_host(p->A8)),
                                    "stored angular fluence");
        if (!p->d_prod) rc = rc ? rc : dalloc_t(&p->d_prod, GV, "angular product");
    }
    if (rc) return rc;
    if (!p->h_acc) {
        cudaError_t e = cudaMallocHost(&p->h_acc, 2 * (size_t)p->G * sizeof(double));
        if (e != cudaSuccess) {
            set_error("pinned host allocation failed");
            return DOCTORS_ERR_OOM;
        }
    }
    // per-source sums of the view-weight and spectrum terms, read back once
    const size_t na = std::max<size_t>(1, p->srcs.size()) * p->G;
    if (p->acc_src_cap < na) {
        if (p->d_acc_src) {
            CU(cudaStreamSynchronize(p->stream));
            cudaFree(p->d_acc_src);
            p->d_acc_src = nullptr;
        }
        if (p->h_acc_src) cudaFreeHost(p->h_acc_src);
        p->h_acc_src = nullptr;
        p->acc_src_cap = 0;
        rc = dalloc_t(&p->d_acc_src, na, "per-source gradient sums");
        if (rc) return rc;
        if (cudaMallocHost(&p->h_acc_src, na * sizeof(double)) != cudaSuccess) {
            (void)cudaGetLastError();
            p->h_acc_src = nullptr;
            set_error("pinned host allocation failed");
            return DOCTORS_ERR_OOM;
        }
        p->acc_src_cap = na;
    }
    return DOCTORS_OK;
}

int copy_out(doctors_problem* p, double* dst, const double* src_host_or_dev, size_t n, int mem, bool src_is_dev) {
    cudaMemcpyKind kind;
    if (src_is_dev) kind = mem == DOCTORS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    else kind = mem == DOCTORS_MEM_DEVICE ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    CU(cudaMemcpyAsync(dst, src_host_or_dev, n * sizeof(double), kind, p->stream));
    return DOCTORS_OK;
}

}  // namespace

namespace {

// The ROI form of the adjoint: the response is formed on the device from the
// staged dose factors and ROI weights, and the explicit density term of the
// dose is added to the density gradient.
struct RoiTerms {
    const double* k;     // device [n_mat][G]
    const double* roi;   // device [V]
};

// The adjoint solve and gradients behind doctors_adjoint_solve (response
// given, roi null) and doctors_roi_gradients (response null, roi given).
// Arguments are checked by the callers.
int adjoint_impl(doctors_problem* p, const double* response, int mem, const RoiTerms* roi, double* d_weights,
                 double* d_spectrum, double* d_density, doctors_result* info) {
    const bool density = d_density != nullptr;
    int rc = ensure_adjoint_buffers(p, density);
    if (rc) return rc;
    const size_t GV = (size_t)p->G * p->V, GVM = GV * p->M;
    p->launches = 0;
    CU(cudaEventRecord(p->ev[0], p->stream));
    if (roi) {
        CU(launch_roi_response(p->V, p->G, p->d_mat, p->d_rho, roi->k, roi->roi, p->d_r, p->d_rf, p->stream));
    } else {
        CU(cudaMemcpyAsync(p->d_r, response, GV * sizeof(double),
                           mem == DOCTORS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           p->stream));
        CU(launch_to_float(GV, p->d_r, p->d_rf, p->stream));
    }
    ++p->launches;
    {
        std::vector<float> ones(p->G, 1.0f);
        CU(cudaMemcpyAsync(p->d_ones, ones.data(), p->G * sizeof(float), cudaMemcpyHostToDevice, p->stream));
        CU(cudaStreamSynchronize(p->stream));
    }
    ScatterArgs sa{};
    sa.V = p->V; sa.G = p->G; sa.M = p->M; sa.L = p->L; sa.nmat = p->nmat;
    sa.mat = p->d_mat; sa.rho = p->d_rho; sa.sigs = p->d_sigs;
    // 1. store the converged forward angular fluence (one extra forward sweep)
    if (density) {
        sa.transpose = 0; sa.base = p->d_Q; sa.iso = nullptr; sa.iso_field = nullptr; sa.phi = p->d_mom;
        sa.out = p->d_src;
        CU(launch_scatter(sa, p->stream));
        ++p->launches;
        rc = sweep_once(p, 0, 1, p->d_src, p->d_T);
        if (rc) return rc;
    }
    // 2. adjoint fixed source 4 pi r in the l = 0 moment
    sa.transpose = 1; sa.base = nullptr; sa.iso = nullptr; sa.iso_field = p->d_rf;
    sa.iso_field_scale = (float)(4.0 * M_PI); sa.phi = nullptr; sa.out = p->d_Qa;
    CU(launch_scatter(sa, p->stream));
    ++p->launches;
    CU(cudaEventRecord(p->ev[1], p->stream));
    // 3. adjoint source iteration
    doctors_result r{};
    const long long l0 = p->launches;
    int irc = iterate(p, 1, p->d_Qa, p->d_Z, &r);
    if (irc && irc != DOCTORS_ERR_NOT_CONVERGED) return irc;
    (void)l0;
    // 4. angular product against the stored forward fluence
    if (density) {
        sa.transpose = 1; sa.base = p->d_Qa; sa.iso_field = nullptr; sa.phi = p->d_Z; sa.out = p->d_src;
        CU(launch_scatter(sa, p->stream));
        ++p->launches;
        CU(cudaMemsetAsync(p->d_prod, 0, GV * sizeof(float), p->stream));
        rc = sweep_once(p, 1, 2, p->d_src, p->d_T);
        if (rc) return rc;
    }
    // 5. T = S^T Z
    sa.transpose = 1; sa.base = nullptr; sa.iso_field = nullptr; sa.phi = p->d_Z; sa.out = p->d_T;
    CU(launch_scatter(sa, p->stream));
    ++p->launches;
    // 6. per-source view-weight, spectrum and ray terms
    std::vector<double> gw(p->srcs.size(), 0.0), gs(p->G, 0.0);
    if (density) CU(cudaMemsetAsync(p->d_grad, 0, p->V * sizeof(double), p->stream));
    // the point sources' sums stay on the device until all are done (one
    // readback, no host round trip per source)
    CU(cudaMemsetAsync(p->d_acc_src, 0, p->srcs.size() * (size_t)p->G * sizeof(double), p->stream));
    bool have_z00 = false, any_point = false;
    for (size_t s = 0; s < p->srcs.size(); ++s) {
        const doctors_source& src = p->srcs[s];
        if (src.kind == DOCTORS_SRC_VOLUME) {
            CU(cudaMemsetAsync(p->d_acc, 0, 2 * (size_t)p->G * sizeof(double), p->stream));
            // J depends on a volume source through <q00 / (4 pi), Z00>
            if (!have_z00) {
                CU(launch_sum00(p->V, p->G, p->M, p->d_Z, p->d_acc + p->G, p->stream));
                ++p->launches;
                CU(cudaMemcpyAsync(p->h_acc, p->d_acc, 2 * (size_t)p->G * sizeof(double), cudaMemcpyDeviceToHost,
                                   p->stream));
                CU(cudaStreamSynchronize(p->stream));
                have_z00 = true;
            }
            for (int g = 0; g < p->G; ++g) {
                const double a = p->h_acc[p->G + g] / (4.0 * M_PI);
                gw[s] += p->spectra[s][g] * a;
                gs[g] += src.weight * a;
            }
            continue;
        }
        any_point = true;
        RayArgs ra = ray_args(p, src, p->d_ones);
        ra.phi_tot = nullptr;
        CU(launch_raytrace(ra, p->stream));
        ++p->launches;
        SourceGradArgs ga{};
        ga.nx = p->nx; ga.ny = p->ny; ga.nz = p->nz; ga.G = p->G; ga.M = p->M; ga.nmat = p->nmat;
        ga.ox = ra.ox; ga.oy = ra.oy; ga.oz = ra.oz; ga.dx = ra.dx; ga.dy = ra.dy; ga.dz = ra.dz;
        ga.sx = ra.sx; ga.sy = ra.sy; ga.sz = ra.sz;
        // emission w_s chi_g of this source: the forward solve's table
        ga.r = p->d_r; ga.T = p->d_T; ga.u = p->d_phiu_src; ga.emit = p->d_emit_all + s * p->G; ga.sigt = p->d_sigt;
        ga.acc = p->d_acc_src + s * p->G; ga.H = density ? p->d_H : nullptr;
        CU(launch_source_grad(ga, p->stream));
        ++p->launches;
        if (density) {
            CU(launch_backproject(ra, p->d_H, p->d_grad, p->stream));
            ++p->launches;
        }
    }
    if (any_point) {
        CU(cudaMemcpyAsync(p->h_acc_src, p->d_acc_src, p->srcs.size() * (size_t)p->G * sizeof(double),
                           cudaMemcpyDeviceToHost, p->stream));
        CU(cudaStreamSynchronize(p->stream));
        for (size_t s = 0; s < p->srcs.size(); ++s) {
            if (p->srcs[s].kind == DOCTORS_SRC_VOLUME) continue;
            const double* acc = p->h_acc_src + s * p->G;
            for (int g = 0; g < p->G; ++g) {
                gw[s] += p->spectra[s][g] * acc[g];
                gs[g] += p->srcs[s].weight * acc[g];
            }
        }
    }
    // 7. collision and scattering terms of the density gradient
    if (density) {
        DensityGradArgs da{};
        da.V = p->V; da.G = p->G; da.M = p->M; da.L = p->L; da.nmat = p->nmat;
        da.mat = p->d_mat; da.sigt = p->d_sigt; da.sigs = p->d_sigs;
        da.Z = p->d_Z; da.phic = p->d_mom; da.U = p->d_U; da.prod = p->d_prod; da.grad = p->d_grad;
        CU(launch_density_grad(da, p->stream));
        ++p->launches;
        if (roi) {
            // the dose's own density factor, at fixed fluence
            CU(launch_roi_explicit(p->V, p->G, p->M, p->d_mat, roi->k, roi->roi, p->d_phiu, p->d_mom, p->d_grad,
                                   p->stream));
            ++p->launches;
        }
    }
    // 8. outputs
    if (d_weights) {
        rc = copy_out(p, d_weights, gw.data(), gw.size(), mem, false);
        if (rc) return rc;
    }
    if (d_spectrum) {
        rc = copy_out(p, d_spectrum, gs.data(), gs.size(), mem, false);
        if (rc) return rc;
    }
    if (density) {
        rc = copy_out(p, d_density, p->d_grad, p->V, mem, true);
        if (rc) return rc;
    }
    CU(cudaEventRecord(p->ev[2], p->stream));
    CU(cudaStreamSynchronize(p->stream));
    float t01 = 0, t12 = 0, t02 = 0;
    cudaEventElapsedTime(&t01, p->ev[0], p->ev[1]);
    cudaEventElapsedTime(&t12, p->ev[1], p->ev[2]);
    cudaEventElapsedTime(&t02, p->ev[0], p->ev[2]);
    r.ms_raytrace = t01;
    r.ms_iterate = t12;
    r.ms_total = t02;
    r.launches = p->launches;
    if (info) *info = r;
    (void)GVM;
    const int frc = check_flow(p);
    if (frc) return frc;
    p->adjoint_done = true;
    if (irc == DOCTORS_ERR_NOT_CONVERGED) set_error("adjoint iteration cap reached before convergence");
    return irc;
}

}  // namespace

extern "C" int doctors_adjoint_solve(doctors_problem* p, const double* response, int mem, double* d_weights,
                                     double* d_spectrum, double* d_density, doctors_result* info) {
    int rc = check_problem(p);
    if (rc) return rc;
    CHECK_ARG(response != nullptr, "null response");
    CHECK_ARG(mem == DOCTORS_MEM_HOST || mem == DOCTORS_MEM_DEVICE, "bad mem");
    if (!p->solved) {
        set_error("no forward solution: call doctors_solve first");
        return DOCTORS_ERR_STATE;
    }
    return adjoint_impl(p, response, mem, nullptr, d_weights, d_spectrum, d_density, info);
}

namespace {

// Stages the dose factors (host, [n_mat][G]) and the ROI weights ([V] in
// `mem`) in the problem's ROI buffers, allocated on first use.
int stage_roi(doctors_problem* p, const double* k, const double* roi, int mem, RoiTerms* out) {
    int rc = 0;
    if (!p->d_k) rc = dalloc_t(&p->d_k, (size_t)kMaxMat * p->G, "dose factors");
    if (!rc && !p->d_part) rc = dalloc_t(&p->d_part, (size_t)kRoiPartials + 1, "ROI partial sums");
    if (!rc && mem == DOCTORS_MEM_HOST && !p->d_roi) rc = dalloc_t(&p->d_roi, p->V, "ROI weights");
    if (rc) return rc;
    // copies from pageable host memory are staged before the call returns, so
    // the caller may change k (and a host roi) as soon as this returns
    CU(cudaMemcpyAsync(p->d_k, k, (size_t)p->nmat * p->G * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    if (mem == DOCTORS_MEM_HOST) {
        CU(cudaMemcpyAsync(p->d_roi, roi, p->V * sizeof(double), cudaMemcpyHostToDevice, p->stream));
        out->roi = p->d_roi;
    } else {
        out->roi = roi;
    }
    out->k = p->d_k;
    return DOCTORS_OK;
}

int check_roi_args(doctors_problem* p, const double* k, const double* roi, int mem, const double* J) {
    int rc = check_problem(p);
    if (rc) return rc;
    CHECK_ARG(k && roi && J, "null argument");
    CHECK_ARG(mem == DOCTORS_MEM_HOST || mem == DOCTORS_MEM_DEVICE, "bad mem");
    if (!p->solved) {
        set_error("no forward solution: call doctors_solve first");
        return DOCTORS_ERR_STATE;
    }
    for (int q = 0; q < p->nmat * p->G; ++q) CHECK_ARG(std::isfinite(k[q]), "k must be finite");
    if (mem == DOCTORS_MEM_HOST)
        for (size_t v = 0; v < p->V; ++v) CHECK_ARG(std::isfinite(roi[v]), "roi must be finite");
    return DOCTORS_OK;
}

}  // namespace

extern "C" int doctors_roi_dose(doctors_problem* p, const double* k, const double* roi, int mem, double* J,
                                double* dose) {
    int rc = check_roi_args(p, k, roi, mem, J);
    if (rc) return rc;
    RoiTerms t{};
    rc = stage_roi(p, k, roi, mem, &t);
    if (rc) return rc;
    double* dose_dev = mem == DOCTORS_MEM_DEVICE ? dose : nullptr;
    // host output: the dose is staged through the FP64 response buffer
    if (dose && mem == DOCTORS_MEM_HOST) {
        rc = ensure_adjoint_buffers(p, false);
        if (rc) return rc;
        dose_dev = p->d_r;
    }
    CU(launch_roi_dose(p->V, p->G, p->M, p->d_mat, p->d_rho, t.k, t.roi, p->d_phiu, p->d_mom, dose_dev, p->d_part,
                       p->d_part + kRoiPartials, p->stream));
    if (dose && mem == DOCTORS_MEM_HOST)
        CU(cudaMemcpyAsync(dose, dose_dev, p->V * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    CU(cudaMemcpyAsync(J, p->d_part + kRoiPartials, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    CU(cudaStreamSynchronize(p->stream));
    return DOCTORS_OK;
}

extern "C" int doctors_roi_gradients(doctors_problem* p, const double* k, const double* roi, int mem, double* J,
                                     double* d_weights, double* d_spectrum, double* d_density,
                                     doctors_result* info) {
    int rc = check_roi_args(p, k, roi, mem, J);
    if (rc) return rc;
    RoiTerms t{};
    rc = stage_roi(p, k, roi, mem, &t);
    if (rc) return rc;
    CU(launch_roi_dose(p->V, p->G, p->M, p->d_mat, p->d_rho, t.k, t.roi, p->d_phiu, p->d_mom, nullptr, p->d_part,
                       p->d_part + kRoiPartials, p->stream));
    CU(cudaMemcpyAsync(J, p->d_part + kRoiPartials, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    CU(cudaStreamSynchronize(p->stream));
    return adjoint_impl(p, nullptr, mem, &t, d_weights, d_spectrum, d_density, info);
}
