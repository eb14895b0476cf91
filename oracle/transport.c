/*
 * FP64 CPU oracle for the discrete-ordinates CT dose hot path: the loops
 * that are too slow in Python.  TEST INFRASTRUCTURE ONLY: the tests, the
 * smoke check and the CPU baseline of the benchmark load it; the product
 * library never does, and the two share no code.
 *
 * Compiled with -O2 -ffp-contract=off so that every float/double operation
 * is one IEEE-rounded operation in the order written.
 *
 * Mesh conventions: voxel (i,j,k) spans o + [i,i+1)*d on each axis, flat
 * index v = (k*ny + j)*nx + i (x fastest).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(i, j, k) (((size_t)(k) * (size_t)ny + (size_t)(j)) * (size_t)nx + (size_t)(i))

/* ------------------------------------------------------------------------ */
/* Siddon ray trace (Sec. II.A: the uncollided fluence is computed by ray    */
/* tracing).  Reading: a Siddon-style parametric walk along the segment      */
/* P(a) = S + a (T - S) from the source S to the centre T of the target      */
/* voxel, walked backward from a = 1 (inside the target voxel) toward the    */
/* source.  At each step the next plane crossed is the one with the largest  */
/* a below the current a; ties are crossed in x, y, z order and the          */
/* zero-length segments they leave are dropped.  The walk stops when it      */
/* leaves the mesh (space outside the mesh is void) or reaches a = 0.        */
/* Plane coordinates are o + p*d; the crossing parameter of plane p on axis  */
/* q is (o_q + p d_q - S_q) / (T_q - S_q).                                    */
/* ------------------------------------------------------------------------ */

/* FP32 walk: the index list is integer output decided by float compares;
 * the kernel takes the same decisions in FP32 with the same operations. */
int oracle_siddon_f32(const float *S, int vi, int vj, int vk, int nx, int ny, int nz,
                      const float *o, const float *d, int32_t *idx, float *len, int cap)
{
    int n[3] = {nx, ny, nz};
    int c[3] = {vi, vj, vk};
    float T[3], dir[3], an[3];
    int step[3];
    for (int q = 0; q < 3; ++q) {
        T[q] = o[q] + ((float)c[q] + 0.5f) * d[q];
        dir[q] = T[q] - S[q];
    }
    float norm = sqrtf(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    for (int q = 0; q < 3; ++q) {
        if (dir[q] > 0.0f) {          /* travelling +q: backward crosses the lower face */
            step[q] = -1;
            an[q] = ((o[q] + (float)c[q] * d[q]) - S[q]) / dir[q];
        } else if (dir[q] < 0.0f) {   /* travelling -q: backward crosses the upper face */
            step[q] = +1;
            an[q] = ((o[q] + (float)(c[q] + 1) * d[q]) - S[q]) / dir[q];
        } else {
            step[q] = 0;
            an[q] = -INFINITY;
        }
    }
    float a = 1.0f;
    int cnt = 0;
    for (;;) {
        int q = 0;
        if (an[1] > an[q]) q = 1;
        if (an[2] > an[q]) q = 2;
        float anext = an[q] > 0.0f ? an[q] : 0.0f;
        float seg = a - anext;
        if (seg > 0.0f) {
            if (cnt >= cap) return -1;
            idx[cnt] = (int32_t)IDX(c[0], c[1], c[2]);
            len[cnt] = seg * norm;
            ++cnt;
        }
        if (an[q] <= 0.0f) break;   /* reached the source */
        a = anext;
        c[q] += step[q];
        if (c[q] < 0 || c[q] >= n[q]) break;   /* left the mesh */
        if (step[q] < 0)
            an[q] = ((o[q] + (float)c[q] * d[q]) - S[q]) / dir[q];
        else
            an[q] = ((o[q] + (float)(c[q] + 1) * d[q]) - S[q]) / dir[q];
    }
    return cnt;
}

/* The same walk in FP64 (used for the fluence itself). */
int oracle_siddon_f64(const double *S, int vi, int vj, int vk, int nx, int ny, int nz,
                      const double *o, const double *d, int32_t *idx, double *len, int cap)
{
    int n[3] = {nx, ny, nz};
    int c[3] = {vi, vj, vk};
    double T[3], dir[3], an[3];
    int step[3];
    for (int q = 0; q < 3; ++q) {
        T[q] = o[q] + ((double)c[q] + 0.5) * d[q];
        dir[q] = T[q] - S[q];
    }
    double norm = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    for (int q = 0; q < 3; ++q) {
        if (dir[q] > 0.0) {
            step[q] = -1;
            an[q] = ((o[q] + (double)c[q] * d[q]) - S[q]) / dir[q];
        } else if (dir[q] < 0.0) {
            step[q] = +1;
            an[q] = ((o[q] + (double)(c[q] + 1) * d[q]) - S[q]) / dir[q];
        } else {
            step[q] = 0;
            an[q] = -INFINITY;
        }
    }
    double a = 1.0;
    int cnt = 0;
    for (;;) {
        int q = 0;
        if (an[1] > an[q]) q = 1;
        if (an[2] > an[q]) q = 2;
        double anext = an[q] > 0.0 ? an[q] : 0.0;
        double seg = a - anext;
        if (seg > 0.0) {
            if (cnt >= cap) return -1;
            idx[cnt] = (int32_t)IDX(c[0], c[1], c[2]);
            len[cnt] = seg * norm;
            ++cnt;
        }
        if (an[q] <= 0.0) break;
        a = anext;
        c[q] += step[q];
        if (c[q] < 0 || c[q] >= n[q]) break;
        if (step[q] < 0)
            an[q] = ((o[q] + (double)c[q] * d[q]) - S[q]) / dir[q];
        else
            an[q] = ((o[q] + (double)(c[q] + 1) * d[q]) - S[q]) / dir[q];
    }
    return cnt;
}

/* Optical depth per group and squared distance for every voxel centre:
 * tau[g][v] = sum over the ray's segments of rho * sigma_t[mat][g] * length
 * (FP64 walk), r2[v] = |T - S|^2.  Returns 0, or -1 if a ray overflows. */
int oracle_optical_depth(int nx, int ny, int nz, const double *o, const double *d,
                         const uint8_t *mat, const double *rho, int G,
                         const double *sigt /* [nmat][G] */, const double *S,
                         double *tau /* [G][V] */, double *r2 /* [V] */)
{
    size_t V = (size_t)nx * ny * nz;
    int cap = 4 * (nx + ny + nz) + 8;
    int rc = 0;
    /* every voxel's ray is independent: one z plane per OpenMP iteration */
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < nz; ++k) {
        int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * cap);
        double *len = (double *)malloc(sizeof(double) * cap);
        int err = !idx || !len;
        for (int j = 0; j < ny && !err; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t v = IDX(i, j, k);
                int cnt = oracle_siddon_f64(S, i, j, k, nx, ny, nz, o, d, idx, len, cap);
                if (cnt < 0) { err = 1; break; }
                for (int g = 0; g < G; ++g) tau[(size_t)g * V + v] = 0.0;
                for (int s = 0; s < cnt; ++s) {
                    size_t u = (size_t)idx[s];
                    for (int g = 0; g < G; ++g)
                        tau[(size_t)g * V + v] += rho[u] * sigt[(size_t)mat[u] * G + g] * len[s];
                }
                double t0 = o[0] + ((double)i + 0.5) * d[0] - S[0];
                double t1 = o[1] + ((double)j + 0.5) * d[1] - S[1];
                double t2 = o[2] + ((double)k + 0.5) * d[2] - S[2];
                r2[v] = t0 * t0 + t1 * t1 + t2 * t2;
            }
        free(idx);
        free(len);
        if (err) {
#pragma omp atomic write
            rc = -1;
        }
    }
    return rc;
}

/* Rectangular fan x cone collimator (Sec. II.B: a fan or cone beam is
 * described by its position and the azimuthal and polar angles it
 * subtends).  Reading: a voxel centre is lit when it lies in front of the
 * source (along > 0), within the fan half-angle in the source's transverse
 * plane (|across| <= tan_half * along) and within the cone's axial slope
 * (|up| <= z_slope * along).  The decision is taken in FP32 with the
 * operations in the order written; the kernel takes it the same way. */
void oracle_collimator_mask(int nx, int ny, int nz, const float *o, const float *d,
                            const float *S, const float *axis, const float *perp,
                            const float *up, float tan_half, float z_slope, uint8_t *W)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                float ux = (o[0] + ((float)i + 0.5f) * d[0]) - S[0];
                float uy = (o[1] + ((float)j + 0.5f) * d[1]) - S[1];
                float uz = (o[2] + ((float)k + 0.5f) * d[2]) - S[2];
                float along = (ux * axis[0] + uy * axis[1]) + uz * axis[2];
                float across = (ux * perp[0] + uy * perp[1]) + uz * perp[2];
                float vert = (ux * up[0] + uy * up[1]) + uz * up[2];
                int lit = along > 0.0f && fabsf(across) <= tan_half * along &&
                          fabsf(vert) <= z_slope * along;
                W[IDX(i, j, k)] = (uint8_t)lit;
            }
}

/* ------------------------------------------------------------------------ */
/* One transport sweep of one group (Eq. 2) for a given moment source.       */
/* For every direction n:                                                    */
/*   q_n(v) = sum_lm Mop[n][lm] src[lm][v]      (Legendre scattering source) */
/*   with c_q = |Omega_q| / d_q and psi_in,q the flux entering through the   */
/*   upwind face along q (0 on the mesh boundary: vacuum inflow):           */
/*   diamond = 0, step differencing: every outgoing face flux equals the     */
/*     cell flux,  psi(v) = (q_n(v) + sum_q c_q psi_in,q) / (sigt(v) + sum_q c_q);   */
/*   diamond = 1, diamond difference (no negative-flux fixup): the cell      */
/*     balance  sum_q c_q (psi_out,q - psi_in,q) + sigt(v) psi(v) = q_n(v)    */
/*     with the cell flux the mean of each face pair, psi(v) =                */
/*     (psi_in,q + psi_out,q) / 2, so                                         */
/*     psi(v) = (q_n(v) + 2 sum_q c_q psi_in,q) / (sigt(v) + 2 sum_q c_q),    */
/*     psi_out,q = 2 psi(v) - psi_in,q;                                       */
/*   phi[lm][v] += Dop[n][lm] psi(v)            (Eq. 3 for lm = 00)          */
/* The outgoing current through the mesh boundary is summed into *leak:     */
/*   w_n |Omega_q| psi_out,q(v) A_q over boundary faces (A_q the face area).  */
/* If psi_out is given, psi of every direction is stored there [A][V].      */
/* ------------------------------------------------------------------------ */
/* The directions are taken in ORACLE_DIRECTION_BLOCKS fixed contiguous     */
/* blocks; each block sums its directions' contributions to phi and to the   */
/* leakage in direction order, and the blocks are then added in block order  */
/* (Eq. 3's quadrature sum, in an order that does not depend on how many     */
/* host threads run the blocks: with OpenMP the blocks run in parallel).     */
#define ORACLE_DIRECTION_BLOCKS 8

static void sweep_direction(int nx, int ny, int nz, double dx, double dy, double dz, int n,
                            const double *dirs, const double *w, int M, const double *Mop,
                            const double *Dop, const double *sigt, const double *src,
                            double *phi, double *lk_out, double *psi_out, int diamond,
                            double *psi, double *fx, double *fy, double *fz)
{
    size_t V = (size_t)nx * ny * nz;
    double lk = 0.0;
    double ox = dirs[3 * n + 0], oy = dirs[3 * n + 1], oz = dirs[3 * n + 2];
    double cx = fabs(ox) / dx, cy = fabs(oy) / dy, cz = fabs(oz) / dz;
    int i0 = ox > 0 ? 0 : nx - 1, di = ox > 0 ? 1 : -1;
    int j0 = oy > 0 ? 0 : ny - 1, dj = oy > 0 ? 1 : -1;
    int k0 = oz > 0 ? 0 : nz - 1, dk = oz > 0 ? 1 : -1;
    for (int kk = 0; kk < nz; ++kk) {
        int k = k0 + dk * kk;
        for (int jj = 0; jj < ny; ++jj) {
            int j = j0 + dj * jj;
            for (int ii = 0; ii < nx; ++ii) {
                int i = i0 + di * ii;
                size_t v = IDX(i, j, k);
                double q = 0.0;
                for (int lm = 0; lm < M; ++lm) q += Mop[(size_t)n * M + lm] * src[(size_t)lm * V + v];
                double px = ii > 0 ? fx[IDX(i - di, j, k)] : 0.0;
                double py = jj > 0 ? fy[IDX(i, j - dj, k)] : 0.0;
                double pz = kk > 0 ? fz[IDX(i, j, k - dk)] : 0.0;
                double p;
                if (diamond) {
                    p = (q + 2.0 * (cx * px + cy * py + cz * pz)) / (sigt[v] + 2.0 * (cx + cy + cz));
                    fx[v] = 2.0 * p - px;
                    fy[v] = 2.0 * p - py;
                    fz[v] = 2.0 * p - pz;
                } else {
                    p = (q + cx * px + cy * py + cz * pz) / (sigt[v] + cx + cy + cz);
                    fx[v] = fy[v] = fz[v] = p;
                }
                psi[v] = p;
                if (ii == nx - 1) lk += w[n] * fabs(ox) * fx[v] * dy * dz;
                if (jj == ny - 1) lk += w[n] * fabs(oy) * fy[v] * dx * dz;
                if (kk == nz - 1) lk += w[n] * fabs(oz) * fz[v] * dx * dy;
            }
        }
    }
    for (int lm = 0; lm < M; ++lm) {
        double c = Dop[(size_t)n * M + lm];
        double *ph = phi + (size_t)lm * V;
        for (size_t v = 0; v < V; ++v) ph[v] += c * psi[v];
    }
    if (psi_out) memcpy(psi_out + (size_t)n * V, psi, sizeof(double) * V);
    *lk_out += lk;
}

/* Returns 0, or -1 if scratch memory could not be allocated. */
int oracle_sweep(int nx, int ny, int nz, double dx, double dy, double dz,
                 int A, const double *dirs /* [A][3] */, const double *w /* [A] */,
                 int M, const double *Mop /* [A][M] */, const double *Dop /* [A][M] */,
                 const double *sigt /* [V] */, const double *src /* [M][V] */,
                 double *phi /* [M][V] */, double *leak, double *psi_out /* [A][V] or NULL */,
                 int diamond)
{
    size_t V = (size_t)nx * ny * nz;
    const int NB = ORACLE_DIRECTION_BLOCKS;
    double lkb[ORACLE_DIRECTION_BLOCKS];
    /* block 0 accumulates into phi, blocks 1.. into their own arrays */
    double *part = (double *)calloc((size_t)(NB - 1) * M * V, sizeof(double));
    double *scratch = (double *)malloc(sizeof(double) * 4 * V * (size_t)NB);
    if (!part || !scratch) {
        free(part);
        free(scratch);
        return -1;
    }
    memset(phi, 0, sizeof(double) * V * (size_t)M);
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < NB; ++b) {
        double *acc = b == 0 ? phi : part + (size_t)(b - 1) * M * V;
        double *sc = scratch + (size_t)b * 4 * V;
        lkb[b] = 0.0;
        int n0 = (int)(((long)A * b) / NB), n1 = (int)(((long)A * (b + 1)) / NB);
        for (int n = n0; n < n1; ++n)
            sweep_direction(nx, ny, nz, dx, dy, dz, n, dirs, w, M, Mop, Dop, sigt, src, acc, &lkb[b],
                            psi_out, diamond, sc, sc + V, sc + 2 * V, sc + 3 * V);
    }
    double lk = lkb[0];
    for (int b = 1; b < NB; ++b) {
        const double *pb = part + (size_t)(b - 1) * M * V;
        for (size_t e = 0; e < (size_t)M * V; ++e) phi[e] += pb[e];
        lk += lkb[b];
    }
    *leak = lk;
    free(part);
    free(scratch);
    return 0;
}

/* Host threads used by the OpenMP loops (1 when built without OpenMP). */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Sets the number of host threads of the OpenMP loops; returns the number
 * in effect. */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
    return oracle_threads();
}

/* Back-projection along the rays for the density gradient of the
 * uncollided fluence: for every target voxel t, walk its ray (FP64) and add
 * -length * H[mat[u]][t] to grad[u] for each voxel u on the ray, where
 * H[m][t] = sum_g sigma_t[m][g] * dJ/dphi_u[g][t] * phi_u[g][t]
 * (d phi_u[g][t] / d rho_u = -sigma_t[mat u][g] * length * phi_u[g][t]). */
int oracle_backproject(int nx, int ny, int nz, const double *o, const double *d,
                       const uint8_t *mat, int nmat, const double *H /* [nmat][V] */,
                       const double *S, double *grad /* [V], accumulated */)
{
    size_t V = (size_t)nx * ny * nz;
    int cap = 4 * (nx + ny + nz) + 8;
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * cap);
    double *len = (double *)malloc(sizeof(double) * cap);
    int rc = 0;
    for (int k = 0; k < nz && rc == 0; ++k)
        for (int j = 0; j < ny && rc == 0; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t t = IDX(i, j, k);
                int cnt = oracle_siddon_f64(S, i, j, k, nx, ny, nz, o, d, idx, len, cap);
                if (cnt < 0) { rc = -1; break; }
                for (int s = 0; s < cnt; ++s) {
                    size_t u = (size_t)idx[s];
                    grad[u] -= len[s] * H[(size_t)mat[u] * V + t];
                }
            }
    (void)nmat;
    free(idx);
    free(len);
    return rc;
}
