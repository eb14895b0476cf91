// Internal declarations of libdoctors: problem state, kernel argument
// blocks and launchers.  Not part of the public C-ABI (include/doctors.h).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/doctors.h"

namespace doctors {

constexpr int kMaxMat = 8;      // materials per problem
constexpr int kMaxG = 64;       // energy groups
constexpr int kMaxSrc = 4096;   // sources per problem
constexpr double kTolFloor = 1e-6;   // FP32 sweep: relative-change floor

void set_error(const std::string& msg);

// Storage order of the flux moments of one cell.  For P3 (16 moments) the
// record is stored as the 4 x 4 transpose of the (l, m) order: position p
// holds moment lm = p / 4 + 4 (p % 4) (position 0 is still lm = 00).  Other
// orders are stored in (l, m) order.  Every kernel's moment tables and the
// host's staging go through lm_of_pos, so the order is a layout choice only.
__host__ __device__ constexpr int lm_of_pos(int p, int M) { return M == 16 ? (p >> 2) + 4 * (p & 3) : p; }
__host__ __device__ constexpr int degree_of_lm(int lm) { return lm >= 9 ? 3 : lm >= 4 ? 2 : lm >= 1 ? 1 : 0; }

bool build_quadrature(int N, std::vector<double>& dirs, std::vector<double>& w, std::string& err);
void real_harmonics(int L, double x, double y, double z, double* R);

// ---------------------------------------------------------------------------
// ray trace (uncollided fluence of one point source)
// ---------------------------------------------------------------------------
struct RayArgs {
    int nx, ny, nz, G, nmat, lit_all;
    float ox, oy, oz, dx, dy, dz;      // mesh origin and spacing
    float sx, sy, sz;                  // source position
    float ax, ay, az, px, py, pz, ux, uy, uz;   // collimator frame
    float tan_half, z_slope;
    const uint8_t* mat;
    const float* rho;
    const float* sigt;                 // [nmat][G]
    const float* emit;                 // [G] weight * spectrum
    float* phi_src;                    // [G][V] this source (overwritten)
    float* phi_tot;                    // [G][V] accumulated (+=), or null
};

cudaError_t launch_raytrace(const RayArgs& a, cudaStream_t s);
cudaError_t launch_debug_ray(const RayArgs& a, int voxel, int32_t* idx, float* len, int cap,
                             int* count, cudaStream_t s);
cudaError_t launch_backproject(const RayArgs& a, const float* H, double* grad, cudaStream_t s);

// ---------------------------------------------------------------------------
// adjoint gradients
// ---------------------------------------------------------------------------
// Per point source: imp[g](v) = r[g](v) + sum_lm (2l+1)/(4 pi) R_lm(Omega_sv) T[g][v][lm]
// (dJ/dphi_u of this source), acc[g] += sum_v u[g](v) imp[g](v) with u the unit
// uncollided fluence, and (if H) H[m][v] = sum_g sigma_t[m][g] imp emit[g] u.
struct SourceGradArgs {
    int nx, ny, nz, G, M, nmat;
    float ox, oy, oz, dx, dy, dz, sx, sy, sz;
    const double* r;                   // [G][V]
    const float* T;                    // [G][V][M]
    const float* u;                    // [G][V]
    const float* emit;                 // [G] weight * spectrum of this source
    const float* sigt;                 // [nmat][G]
    double* acc;                       // [G]
    float* H;                          // [nmat][V] or null
};
cudaError_t launch_source_grad(const SourceGradArgs& a, cudaStream_t s);

// grad[v] += sum_{g,lm} (2l+1)/(4 pi) Z[g][v][lm] rho-free sigma_s,l(g'->g) (phi_c + U)[g'][v][lm]
//            - sum_g sigma_t[mat][g] prod[g][v]     (prod may be null)
struct DensityGradArgs {
    size_t V;
    int G, M, L, nmat;
    const uint8_t* mat;
    const float* sigt;                 // [nmat][G]
    const float* sigs;                 // [nmat][L+1][G][G]
    const float* Z;                    // [G][V][M] adjoint moments
    const float* phic;                 // [G][V][M] forward collided moments
    const float* U;                    // [G][V][M] uncollided moments
    const float* prod;                 // [G][V] or null
    double* grad;                      // [V]
};
cudaError_t launch_density_grad(const DensityGradArgs& a, cudaStream_t s);
// out[g] += sum_v mom[g][v][0]
cudaError_t launch_sum00(size_t V, int G, int M, const float* mom, double* out, cudaStream_t s);
// out[i] = (float) in[i]
cudaError_t launch_to_float(size_t n, const double* in, float* out, cudaStream_t s);

// U[g][v][lm] += phi_src[g][v] * R_lm(unit(centre_v - source))
struct MomentArgs {
    int nx, ny, nz, G, M, L;
    float ox, oy, oz, dx, dy, dz, sx, sy, sz;
    const float* phi_src;              // [G][V]
    float* U;                          // [G][V][M]
    int accumulate;                    // 0: U = phi R (first source), 1: U += phi R
};
cudaError_t launch_uncollided_moments(const MomentArgs& a, cudaStream_t s);

// ---------------------------------------------------------------------------
// scattering source:  out[g][v][lm] = base[g][v][lm] + iso[g] * (lm == 0)
//                      + rho_v sum_g' sigma_s,l[mat v](g' -> g) phi[g'][v][lm]
// (transpose: sigma_s,l(g -> g') instead, i.e. the adjoint's upscatter)
// ---------------------------------------------------------------------------
struct ScatterArgs {
    size_t V;
    int G, M, L, nmat, transpose;
    const uint8_t* mat;
    const float* rho;
    const float* sigs;                 // [nmat][L+1][G][G] (from, to)
    const float* base;                 // [G][V][M] or null
    const float* iso;                  // [G] or null: added to lm = 0 of every voxel
    const float* iso_field;            // [G][V] or null: added to lm = 0 (per voxel)
    float iso_field_scale;
    const float* phi;                  // [G][V][M] or null (no scattering term)
    float* out;                        // [G][V][M]
    const int* skip;                   // if non-null and *skip != 0 the kernel does nothing
    int g0, g1;                        // destination groups updated: g0 .. g1 - 1 (g1 = 0: all)
    const int* win;                    // non-null: the window [win[0], win[1]) in device memory instead
};
cudaError_t launch_scatter(const ScatterArgs& a, cudaStream_t s);

// residual: res[g][0] += sum_v (phi00 - prev)^2, res[g][1] += sum_v phi00^2; prev = phi00
cudaError_t launch_residual(size_t V, int G, int M, const float* mom, float* prev, double* res,
                            cudaStream_t s, const int* skip = nullptr, int g0 = 0, int gcount = -1,
                            const int* win = nullptr);
// zero groups [win[0], win[1]) of a [G][per_group] float array unless *skip
cudaError_t launch_zero_window(float* p, size_t per_group, int G, const int* win, const int* skip, cudaStream_t s);
// out[g][v] = rho[v] * sigt[mat[v]][g] (FP32, the product the sweep forms)
cudaError_t launch_total_xs(size_t V, int G, const uint8_t* mat, const float* rho, const float* sigt, float* out,
                            cudaStream_t s);
cudaError_t launch_zero_window(double* p, size_t per_group, int G, const int* win, const int* skip, cudaStream_t s);
// zero n floats (or doubles) unless *skip
cudaError_t launch_zero(float* p, size_t n, const int* skip, cudaStream_t s);
cudaError_t launch_zero(double* p, size_t n, const int* skip, cudaStream_t s);

// One entry per instance of a device-side iteration loop.
struct LoopCtl {
    int done;                          // instance retired (converged or capped)
    int iters;                         // sweeps performed
    int max_iters;
    int G;
    double tol;
    double resid;                      // max over groups of the last relative change
    const double* res;                 // [G][2] residual sums of the instance
    int reverse;                       // adjoint: the window's trailing groups retire
    int use_window;                    // the instance's kernels follow win (else all groups, every sweep)
    int win[2];                        // active group window [win[0], win[1])
    long long group_sweeps;            // sum over iterations of the groups swept
};
// Retire converged instances; end the while loop when all are retired.
cudaError_t launch_decide(LoopCtl* ctl, int n, unsigned long long cond_handle, cudaStream_t s);

// balance: bal[g][0] += vol * sum s00, bal[g][1] += vol * sum sigma_t phi00
cudaError_t launch_balance(size_t V, int G, int M, const uint8_t* mat, const float* rho,
                           const float* sigt, const float* src, const float* mom, double vol,
                           double* bal, cudaStream_t s);

// dose[v] = sum_g k[mat][g] rho_v (phi_u + phi_c00)  (FP64)
cudaError_t launch_dose(size_t V, int G, int M, const uint8_t* mat, const float* rho,
                        const double* k, const float* phi_u, const float* mom, double* dose,
                        cudaStream_t s);

// out[g][v] = (which & 1 ? phi_u : 0) + (which & 2 ? mom00 : 0)
cudaError_t launch_extract(size_t V, int G, int M, int which, const float* phi_u, const float* mom,
                           float* out, cudaStream_t s);

// ---------------------------------------------------------------------------
// octant wavefront sweep
// ---------------------------------------------------------------------------
struct SweepArgs {
    int nx, ny, nz, G, A8, ab, nab, nmat;
    int tx, ty, ntx, nty, stage, reverse;
    int g0, gcount;                    // groups swept: g0 .. g0 + gcount - 1
    const uint8_t* mat;
    const float* rho;
    const float* sigt;                 // [nmat][G]
    const float* src;                  // [G][V][M] moment source
    float* mom;                        // [G][V][M] accumulated moments
    int table_base;                    // first row of this S_N set in the constant direction tables
    const float* coef;                 // [A][8] cx, cy, cz, cx+cy+cz, leak_x, leak_y, leak_z, w
    float* xface;                      // [8][A8][G][ntx-1][ny][nz]
    float* yface;                      // [8][A8][G][nty-1][nx][nz]
    double* leak;                      // [G]
    int A;                             // directions (psi indexing)
    float* psi;                        // written (mode 1) or read (mode 2): [G][V][A], dataflow kernel [G][V][8][ABP]
    float* prod;                       // [G][V]: mode 2 accumulator
    const int* skip;                   // if non-null and *skip != 0 the kernel does nothing
    int chain_slots;                   // > 0: chained kernel, at most this many CTAs per stage launch
    const int* win;                    // dataflow kernels: non-null: sweep the groups [win[0], win[1]) read from
                                       // device memory (g0, gcount then give only the buffer layout)
    int slot_share;                    // dataflow kernels: use chain_slots / slot_share CTAs (> 1 when
                                       // that many instances sweep concurrently; 0 or 1: all)
    const struct ChainDirTable* dir_table;   // host copy of the first-octant direction table (chained kernel)
    const float* qang;                 // split transforms: angular source [G][8][V][ABP] (direction octant)
    float* pang;                       // split transforms: angular fluence [G][8][V][ABP]
    int hw;                            // dataflow kernel: 1 = a face warp per CTA takes the incoming
                                       // face records (mode 0)
    const float* tc_b1;                // split transforms on the tensor cores (P3): moments -> directions
    const float* tc_b2;                // and directions -> moments operand tables, or null
    int dd;                            // dataflow kernel: 1 = diamond differencing (dir_table holds 2c), 0 = step
    int blk;                           // dataflow kernel: the direction block this launch sweeps (0 .. nab-1;
                                       // dir_table holds that block's rows)
    int* flow;                         // non-null: dataflow kernel; [0] task queue, [1] CTAs done, [2] wait timed out,
                                       // [3] test hook: task + 1 that writes no faces (0: none)
};

// Per-problem direction data of the first octant for the chained sweep,
// passed by value as a kernel parameter and read through the constant bank
// at compile-time offsets when a CTA sweeps whole octants.  Directions of
// octant o are the first octant's reflected by the signs of o (the quadrature
// builds them that way), and R_lm of a reflected direction is R_lm of the
// original times (-1) to the number of reflected axes in which R_lm is odd.
constexpr int kMaxA8 = 36;             // S16
constexpr int kFlowMaxAB = 36;         // whole octants of S2..S8, S12 and S16
struct ChainDirTable {
    float cx[kMaxA8], cy[kMaxA8], cz[kMaxA8], csum[kMaxA8];   // |Omega_q| / d_q and their sum
    float lx[kMaxA8], ly[kMaxA8], lz[kMaxA8];                  // boundary current per face (w |Omega_q| area)
    float w[kMaxA8];
    // the dataflow kernel's moment <-> direction tables of the first octant,
    // indexed by the moment's storage position m (lm = lm_of_pos(m, M)):
    // mop[q * 16 + m] = (2l+1)/(4 pi) R_lm(Omega_q) and, transposed,
    // dop[m * kFlowMaxAB + q] = w_q R_lm(Omega_q), so that the operands of a
    // packed two-lane FMA (two moments of one direction, two directions of one
    // moment) are adjacent kernel-parameter words
    float mop[kFlowMaxAB * 16], dop[16 * kFlowMaxAB];
    // the problem's [G][V] rho sigma_t of every cell and group (dataflow kernels);
    // last, so that the tables above keep their parameter offsets
    const float* sig;
};
// the dataflow and chained kernels take SweepArgs and the table by value: the
// parameter block (up to 32764 bytes on this architecture) must hold both
static_assert(sizeof(SweepArgs) + sizeof(ChainDirTable) < 32764, "kernel parameter block too large");
// R_lm odd in x, y, z (bit lm)
constexpr unsigned kOddX = (1u << 3) | (1u << 4) | (1u << 7) | (1u << 10) | (1u << 13) | (1u << 15);
constexpr unsigned kOddY = (1u << 1) | (1u << 4) | (1u << 5) | (1u << 9) | (1u << 10) | (1u << 11);
constexpr unsigned kOddZ = (1u << 2) | (1u << 5) | (1u << 7) | (1u << 10) | (1u << 12) | (1u << 14);
// chained kernels with the direction table in the constant bank exist for
// these directions per CTA (whole octants of S2, S4, S6, S8)
inline bool chain_const_table_ab(int ab) { return ab == 1 || ab == 3 || ab == 6 || ab == 10; }
// whole octants the dataflow kernels sweep with their table in the constant
// bank: S2, S4, S6, S8, S12 and S16
inline bool flow_octant_ab(int ab) { return chain_const_table_ab(ab) || ab == 21 || ab == 36; }
// direction blocks the dataflow kernels sweep (one launch per block, its
// table in the constant bank): whole octants, or blocks of 12 directions
// (S16: three per octant; a block's face and stored angular records are
// then exactly its 12 fluxes, no padding)
inline bool flow_block_ab(int A8, int ab) { return (A8 == ab && flow_octant_ab(ab)) || (ab == 12 && A8 % 12 == 0); }
// mode 0: plain; 1: store psi; 2: accumulate sum_n w_n psi_n psi_stored_n into prod
cudaError_t launch_sweep_stage(const SweepArgs& a, int M, int mode, cudaStream_t s);
bool sweep_supported(int ab, int M);
// CTAs of the chained sweep kernel resident per SM (0 if it cannot launch)
int sweep_chain_blocks_per_sm(int ab, bool ct, int M, int threads, size_t smem);
// Hyperplane plane of the chained sweep: a column's AB fluxes are one record
// of chain_rs(AB) floats (odd), columns are laid out with a row pitch of
// chain_px(tx) slots (even, halo column at 0) and a halo row at 0.  Threads
// on one diagonal of the tile are then an odd number of words apart, so
// their plane accesses fall in distinct shared-memory banks.
__host__ __device__ inline int chain_rs(int ab) { return ab | 1; }
__host__ __device__ inline int chain_px(int tx) { return (tx & 1) ? tx + 1 : tx + 2; }
// shared memory of one chained-sweep CTA: per chained task the direction rows
// (coef and R as float4, w), the per-group leakage (FP64), the two
// halo-padded hyperplanes and sigma_t of the swept groups
inline size_t sweep_chain_smem_bytes(int ab, int tx, int ty, int cmax, int gcount, int nmat) {
    return 16 * (size_t)cmax * ab * 5 + 8 * (size_t)gcount +
           4 * ((size_t)2 * chain_rs(ab) * chain_px(tx) * (ty + 1) + (size_t)cmax * ab + (size_t)gcount * nmat);
}
// shared memory of one dataflow-sweep CTA: the fetched face records of the
// tile's first row and column, per-group leakage, the two halo-padded
// hyperplanes, sigma_t of the swept groups and the task slot
inline int flow_abp_host(int ab) { return (ab + 3) & ~3; }
inline size_t sweep_flow_smem_bytes(int ab, int tx, int ty, int gcount, int nmat, bool dd = false) {
    // prefetched source moments (2 slots of 16 floats per thread), two landing
    // slots (pipeline depth 2) of one record per edge column, the leakage per
    // group, two planes of column records (diamond differencing: x-going and
    // y-going face fluxes in separate planes), the cross sections and the task slot
    return 2 * (size_t)16 * 4 * (size_t)tx * ty + 2 * (size_t)4 * (tx + ty) * flow_abp_host(ab) +
           8 * (size_t)gcount +
           4 * ((size_t)(dd ? 4 : 2) * chain_rs(ab) * chain_px(tx) * (ty + 1) + (size_t)gcount * nmat) + 16;
}
int sweep_flow_blocks_per_sm(int ab, int M, int threads, size_t smem, bool split = false, bool dd = false,
                             bool hw = false);
cudaError_t launch_sweep_flow(const SweepArgs& a, int M, int mode, cudaStream_t s);
// split transforms (whole octants of S2..S8): moments -> angular source for
// all 8 octants, the dataflow sweep on angular records (a.qang -> a.pang),
// angular fluence -> moments (plain stores into a.mom)
cudaError_t launch_split_sweep(const SweepArgs& a, int M, cudaStream_t s, int* count);
// Upload the shared direction tables (all S_N sets) to the current device,
// once per device; returns the first table row of order N in *base.
cudaError_t ensure_direction_tables(int device, int N, int* base);

// split transforms on the tensor cores (P3, whole octants of S2..S8):
// transform_tc.cu.  The operand tables (TF32 hi and lo parts in the kernels'
// shared-memory layout) are built on the host from the first-octant rows.
void build_tc_transform_tables(const ChainDirTable& dt, int AB, std::vector<float>& b1, std::vector<float>& b2);
cudaError_t launch_m2d_tc(const SweepArgs& a, cudaStream_t s);
cudaError_t launch_d2m_tc(const SweepArgs& a, cudaStream_t s);


// ---------------------------------------------------------------------------
// region-of-interest dose and its gradient terms (roi.cu)
// ---------------------------------------------------------------------------
constexpr int kRoiPartials = 1024;   // per-block partial sums of J (fixed grid)

// J = sum_v roi(v) D(v) into the device scalar *J (and dose [V], if non-null);
// partial holds kRoiPartials doubles.
cudaError_t launch_roi_dose(size_t V, int G, int M, const uint8_t* mat, const float* rho, const double* k,
                            const double* roi, const float* phi_u, const float* mom, double* dose,
                            double* partial, double* J, cudaStream_t s);
// r[g][v] = roi(v) k[mat v][g] rho(v) in FP64 (r) and FP32 (rf)
cudaError_t launch_roi_response(size_t V, int G, const uint8_t* mat, const float* rho, const double* k,
                                const double* roi, double* r, float* rf, cudaStream_t s);
// grad[v] += roi(v) sum_g k[mat v][g] (phi_u + phi_c)[g](v)
cudaError_t launch_roi_explicit(size_t V, int G, int M, const uint8_t* mat, const double* k, const double* roi,
                                const float* phi_u, const float* mom, double* grad, cudaStream_t s);

}  // namespace doctors

// ---------------------------------------------------------------------------
// the opaque handle
// ---------------------------------------------------------------------------
struct doctors_problem {
    int device = 0;
    cudaStream_t stream = nullptr;
    doctors_mesh mesh{};
    doctors_options opt{};
    int nx = 0, ny = 0, nz = 0;
    size_t V = 0;
    int G = 0, N = 0, L = 0, M = 0, A = 0, A8 = 0;
    // quadrature
    std::vector<double> dirs, w;
    // sweep tiling
    int tx = 16, ty = 16, ntx = 1, nty = 1, ab = 1, nab = 1;
    int chain_slots = 0;            // > 0: chained or dataflow sweep with this many CTA slots
    bool use_flow = false;          // dataflow sweep (one launch per sweep, task queue)
    bool use_split = false;         // dataflow sweep with the transforms in separate passes
    bool split_tc = false;          // ... those passes on the tensor cores (P3)
    bool flow_hw = false;           // dataflow sweep: a face warp per CTA
    int differencing = 0;           // DOCTORS_DIFF_STEP or DOCTORS_DIFF_DIAMOND
    int flow_slots = 0;             // CTA slots of the plain dataflow kernel (modes 1, 2 under split)
    float* d_qang = nullptr;        // [G][8][V][ABP] angular source (split)
    float* d_pang = nullptr;        // [G][8][V][ABP] angular fluence (split)
    float* d_tcb = nullptr;         // split transforms on the tensor cores: operand tables b1, b2
    size_t tcb1_floats = 0;         // floats of b1 (b2 follows)
    size_t ang_floats = 0;
    int* d_flow = nullptr;          // [4] dataflow queue, done count, timeout flag
    doctors::ChainDirTable dir_table{};   // first-octant direction table of the chained sweep
    std::vector<doctors::ChainDirTable> dir_blk;   // dataflow sweep: the table of each direction block
    // device tables
    float* d_coef = nullptr;
    int table_base = 0;
    // materials
    int nmat = 0;
    bool have_mat = false;
    uint8_t* d_mat = nullptr;
    float* d_rho = nullptr;
    float* d_sigt = nullptr;
    float* d_sigs = nullptr;
    std::vector<double> h_sigt, h_sigs;
    // sources
    std::vector<doctors_source> srcs;
    std::vector<std::vector<double>> spectra;
    bool have_src = false;
    // solver state
    float* d_phiu_src = nullptr;   // [G][V]
    float* d_phiu = nullptr;       // [G][V]
    float* d_U = nullptr;          // [G][V][M]
    float* d_Q = nullptr;          // [G][V][M]
    float* d_mom = nullptr;        // [G][V][M]
    float* d_src = nullptr;        // [G][V][M]
    float* d_src2 = nullptr;       // [G][V][M] the next iteration's source (formed ahead)
    float* d_prev = nullptr;       // [G][V]
    float* d_emit = nullptr;       // [G]
    float* d_emit_all = nullptr;   // [n_src][G] weight * spectrum of every source
    size_t emit_cap = 0;           // floats allocated in d_emit_all
    float* d_iso = nullptr;        // [G]
    float* d_xface = nullptr;
    float* d_yface = nullptr;
    size_t xface_bytes = 0, yface_bytes = 0;
    double* d_red = nullptr;       // reductions: leak [G], res [G][2], bal [G][2]
    double* h_red = nullptr;       // pinned mirror
    // adjoint state (allocated on the first adjoint solve)
    float* d_Z = nullptr;          // [G][V][M] adjoint moments
    float* d_Qa = nullptr;         // [G][V][M] adjoint fixed source
    float* d_T = nullptr;          // [G][V][M] S^T Z (also a throwaway accumulator)
    float* d_rf = nullptr;         // [G][V] response (FP32)
    double* d_r = nullptr;         // [G][V] response (FP64)
    double* d_acc = nullptr;       // [2G] per-group sums
    double* d_grad = nullptr;      // [V] density gradient
    float* d_H = nullptr;          // [kMaxMat][V]
    float* d_ones = nullptr;       // [G]
    float* d_psi = nullptr;        // stored forward angular fluence ([G][V][A], or the dataflow layout)
    float* d_prod = nullptr;       // [G][V] angular product
    double* h_acc = nullptr;       // pinned [2G]
    double* d_acc_src = nullptr;   // [S][G] per-source gradient sums (adjoint)
    double* h_acc_src = nullptr;   // pinned copy of it
    float* d_sig = nullptr;        // [G][V] rho * sigma_t per cell and group (the dataflow sweep's one load)
    size_t acc_src_cap = 0;        // doubles in both
    // region-of-interest dose (allocated on first use)
    double* d_k = nullptr;         // [kMaxMat][G] dose factors
    double* d_roi = nullptr;       // [V] ROI weights (staged from host memory)
    double* d_part = nullptr;      // [kRoiPartials + 1] partial sums of J, then J
    double* d_dose_stage = nullptr;  // [V] dose staging for host-memory output
    bool solved = false;
    bool adjoint_done = false;
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    long long launches = 0;        // kernels launched by the current call
};
