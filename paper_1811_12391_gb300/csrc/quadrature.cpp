// Level-symmetric S_N quadrature and real spherical harmonics for the sweep
// tables (host code, FP64).
//
// Sec. II.D and Eq. 3: N(N+2) discrete directions with weights w_n whose
// weighted sum of the angular fluence is the scalar fluence.  The paper does
// not print its set; this is the level-symmetric LQ_N construction: the
// direction cosines of one octant come from N/2 levels with
// mu_i^2 = mu_1^2 + (i-1) * 2 (1 - 3 mu_1^2) / (N - 2), a direction is a level
// triple (a, b, c) with a + b + c = N/2 + 2, and all directions that are
// permutations of the same triple share one weight.  The weights are fixed
// by requiring exact integration of every even monomial x^2i y^2j z^2k of
// degree <= N-2 over the octant (solved here by Householder least squares;
// the system is consistent, which is checked).
//
// Eq. 2's scattering kernel is a Legendre expansion; the addition theorem
// turns it into sums over real spherical harmonics R_lm, here in the
// Schmidt semi-normalisation (sum_m R_lm(a) R_lm(b) = P_l(a.b)), written out
// as Cartesian polynomials for l <= 3.
#include "doctors_internal.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace doctors {

static double mu1_of(int N) {
    switch (N) {
        case 2: return std::sqrt(1.0 / 3.0);
        case 4: return 0.3500212;
        case 6: return 0.2666355;
        case 8: return 0.2182179;
        case 12: return 0.1672126;
        case 16: return 0.1389568;
        default: return -1.0;
    }
}

// integral of x^(2i) y^(2j) z^(2k) over one octant of the unit sphere:
// Gamma(i+1/2) Gamma(j+1/2) Gamma(k+1/2) / (4 Gamma(i+j+k+3/2))
static double octant_moment(int i, int j, int k) {
    return std::exp(std::lgamma(i + 0.5) + std::lgamma(j + 0.5) + std::lgamma(k + 0.5) -
                    std::lgamma(i + j + k + 1.5)) / 4.0;
}

// Least squares min ||A x - b|| for a tall, full-column-rank A (rows x cols,
// row-major) by Householder QR.  Returns the residual max norm.
static double householder_lsq(std::vector<double> A, std::vector<double> b, int rows, int cols,
                              std::vector<double>& x) {
    for (int c = 0; c < cols; ++c) {
        double nrm = 0.0;
        for (int r = c; r < rows; ++r) nrm += A[r * cols + c] * A[r * cols + c];
        nrm = std::sqrt(nrm);
        if (nrm == 0.0) continue;
        double alpha = A[c * cols + c] > 0 ? -nrm : nrm;
        std::vector<double> v(rows, 0.0);
        for (int r = c; r < rows; ++r) v[r] = A[r * cols + c];
        v[c] -= alpha;
        double vv = 0.0;
        for (int r = c; r < rows; ++r) vv += v[r] * v[r];
        if (vv == 0.0) continue;
        for (int cc = c; cc < cols; ++cc) {
            double dot = 0.0;
            for (int r = c; r < rows; ++r) dot += v[r] * A[r * cols + cc];
            double f = 2.0 * dot / vv;
            for (int r = c; r < rows; ++r) A[r * cols + cc] -= f * v[r];
        }
        double dot = 0.0;
        for (int r = c; r < rows; ++r) dot += v[r] * b[r];
        double f = 2.0 * dot / vv;
        for (int r = c; r < rows; ++r) b[r] -= f * v[r];
    }
    x.assign(cols, 0.0);
    for (int c = cols - 1; c >= 0; --c) {
        double s = b[c];
        for (int cc = c + 1; cc < cols; ++cc) s -= A[c * cols + cc] * x[cc];
        x[c] = s / A[c * cols + c];
    }
    double res = 0.0;
    for (int r = cols; r < rows; ++r) res = std::max(res, std::fabs(b[r]));
    return res;
}

bool build_quadrature(int N, std::vector<double>& dirs, std::vector<double>& w, std::string& err) {
    double mu1 = mu1_of(N);
    if (mu1 < 0) {
        err = "sn_order must be one of 2, 4, 6, 8, 12, 16";
        return false;
    }
    const int n = N / 2;
    std::vector<double> mu(n);
    if (N == 2) {
        mu[0] = mu1;
    } else {
        double step = 2.0 * (1.0 - 3.0 * mu1 * mu1) / (N - 2);
        for (int i = 0; i < n; ++i) mu[i] = std::sqrt(mu1 * mu1 + step * i);
    }
    // octant points (level indices, 0-based) and their permutation classes
    struct Pt { int a, b, c, cls; };
    std::vector<Pt> pts;
    std::vector<std::vector<int>> classes;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b)
            for (int c = 0; c < n; ++c)
                if (a + b + c + 3 == n + 2) {
                    std::vector<int> key = {a, b, c};
                    std::sort(key.begin(), key.end());
                    int cls = -1;
                    for (size_t q = 0; q < classes.size(); ++q)
                        if (classes[q] == key) cls = (int)q;
                    if (cls < 0) {
                        classes.push_back(key);
                        cls = (int)classes.size() - 1;
                    }
                    pts.push_back({a, b, c, cls});
                }
    const int ncls = (int)classes.size();
    std::vector<double> A, rhs;
    int rows = 0;
    for (int h = 0; 2 * h <= N - 2; ++h)
        for (int i = 0; i <= h; ++i)
            for (int j = 0; j <= h - i; ++j) {
                int k = h - i - j;
                std::vector<double> row(ncls, 0.0);
                for (const Pt& p : pts)
                    row[p.cls] += std::pow(mu[p.a], 2 * i) * std::pow(mu[p.b], 2 * j) *
                                  std::pow(mu[p.c], 2 * k);
                A.insert(A.end(), row.begin(), row.end());
                rhs.push_back(octant_moment(i, j, k));
                ++rows;
            }
    std::vector<double> cw;
    double res = householder_lsq(A, rhs, rows, ncls, cw);
    if (!(res < 1e-12)) {
        err = "level-symmetric moment system is inconsistent";
        return false;
    }
    for (double x : cw)
        if (!(x > 0)) {
            err = "level-symmetric set has a non-positive weight";
            return false;
        }
    dirs.clear();
    w.clear();
    for (int o = 0; o < 8; ++o) {
        double sx = (o & 1) ? -1.0 : 1.0, sy = (o & 2) ? -1.0 : 1.0, sz = (o & 4) ? -1.0 : 1.0;
        for (const Pt& p : pts) {
            dirs.push_back(sx * mu[p.a]);
            dirs.push_back(sy * mu[p.b]);
            dirs.push_back(sz * mu[p.c]);
            w.push_back(cw[p.cls]);
        }
    }
    return true;
}

// Schmidt semi-normalised real harmonics for l <= 3, flat index l*l + l + m.
void real_harmonics(int L, double x, double y, double z, double* R) {
    R[0] = 1.0;
    if (L < 1) return;
    R[1] = y;
    R[2] = z;
    R[3] = x;
    if (L < 2) return;
    const double s3 = std::sqrt(3.0);
    R[4] = s3 * x * y;
    R[5] = s3 * y * z;
    R[6] = 0.5 * (3.0 * z * z - 1.0);
    R[7] = s3 * x * z;
    R[8] = 0.5 * s3 * (x * x - y * y);
    if (L < 3) return;
    const double a = std::sqrt(5.0 / 8.0), b = std::sqrt(15.0), c = std::sqrt(3.0 / 8.0);
    R[9] = a * y * (3.0 * x * x - y * y);
    R[10] = b * x * y * z;
    R[11] = c * y * (5.0 * z * z - 1.0);
    R[12] = 0.5 * z * (5.0 * z * z - 3.0);
    R[13] = c * x * (5.0 * z * z - 1.0);
    R[14] = 0.5 * b * z * (x * x - y * y);
    R[15] = a * x * (x * x - 3.0 * y * y);
}

}  // namespace doctors

extern "C" int doctors_quadrature(int sn_order, int legendre, double* dirs, double* w, double* R,
                                  int* n_dirs) {
    std::vector<double> d, wt;
    std::string err;
    if (legendre < 0 || legendre > 3) {
        doctors::set_error("legendre must be 0..3");
        return DOCTORS_ERR_INVALID_ARG;
    }
    if (!doctors::build_quadrature(sn_order, d, wt, err)) {
        doctors::set_error(err);
        return DOCTORS_ERR_INVALID_ARG;
    }
    const int A = (int)wt.size();
    const int M = (legendre + 1) * (legendre + 1);
    if (n_dirs) *n_dirs = A;
    for (int n = 0; n < A; ++n) {
        if (dirs)
            for (int q = 0; q < 3; ++q) dirs[3 * n + q] = d[3 * n + q];
        if (w) w[n] = wt[n];
        if (R) {
            double r[16];
            doctors::real_harmonics(legendre, d[3 * n], d[3 * n + 1], d[3 * n + 2], r);
            for (int m = 0; m < M; ++m) R[(size_t)n * M + m] = r[m];
        }
    }
    return DOCTORS_OK;
}
