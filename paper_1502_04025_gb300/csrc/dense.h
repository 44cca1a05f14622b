// Small dense complex linear algebra on the host (matrices up to ~65 x 64)
// for the outer solver: least squares by Householder QR, the eigenproblem of
// the harmonic Ritz values (Hessenberg reduction, shifted QR iteration to
// Schur form, eigenvectors by back substitution), and a QR factorisation.
// Row-major storage, std::complex<double>.
#pragma once

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace qdd {
namespace dense {

typedef std::complex<double> zc;

struct Mat {
    int r = 0, c = 0;
    std::vector<zc> a;
    Mat() = default;
    Mat(int r_, int c_) : r(r_), c(c_), a((size_t)r_ * c_, zc(0, 0)) {}
    zc &operator()(int i, int j) { return a[(size_t)i * c + j]; }
    const zc &operator()(int i, int j) const { return a[(size_t)i * c + j]; }
};

inline double nrm(const std::vector<zc> &v)
{
    double s = 0;
    for (auto &x : v) s += std::norm(x);
    return std::sqrt(s);
}

// min |b - A y| over y (A: m x n, m >= n, full column rank).  Returns y and
// the residual vector b - A y.
inline bool lstsq(const Mat &A0, const std::vector<zc> &b0, std::vector<zc> &y, std::vector<zc> &res)
{
    const int m = A0.r, n = A0.c;
    Mat A = A0;
    std::vector<zc> b = b0;
    std::vector<std::vector<zc>> vs(n);
    for (int k = 0; k < n; k++) {
        // Householder reflector for column k, rows k..m-1
        double xn = 0;
        for (int i = k; i < m; i++) xn += std::norm(A(i, k));
        xn = std::sqrt(xn);
        std::vector<zc> v(m - k);
        for (int i = k; i < m; i++) v[i - k] = A(i, k);
        zc ph = std::abs(v[0]) > 0 ? v[0] / std::abs(v[0]) : zc(1, 0);
        v[0] += ph * xn;
        double vn = 0;
        for (auto &t : v) vn += std::norm(t);
        if (vn > 0) {
            // A <- (I - 2 v v^H / v^H v) A, b likewise
            for (int j = k; j < n; j++) {
                zc s = 0;
                for (int i = k; i < m; i++) s += std::conj(v[i - k]) * A(i, j);
                s *= 2.0 / vn;
                for (int i = k; i < m; i++) A(i, j) -= s * v[i - k];
            }
            zc s = 0;
            for (int i = k; i < m; i++) s += std::conj(v[i - k]) * b[i];
            s *= 2.0 / vn;
            for (int i = k; i < m; i++) b[i] -= s * v[i - k];
        }
        vs[k] = v;
    }
    y.assign(n, zc(0, 0));
    for (int i = n - 1; i >= 0; i--) {
        zc s = b[i];
        for (int j = i + 1; j < n; j++) s -= A(i, j) * y[j];
        if (std::abs(A(i, i)) == 0) return false;
        y[i] = s / A(i, i);
    }
    res.assign(m, zc(0, 0));
    for (int i = 0; i < m; i++) {
        zc s = b0[i];
        for (int j = 0; j < n; j++) s -= A0(i, j) * y[j];
        res[i] = s;
    }
    return true;
}

// Solve A X = B (A n x n) by Gaussian elimination with partial pivoting.
inline bool solve(Mat A, Mat &B)
{
    const int n = A.r;
    for (int k = 0; k < n; k++) {
        int p = k;
        for (int i = k + 1; i < n; i++)
            if (std::abs(A(i, k)) > std::abs(A(p, k))) p = i;
        if (std::abs(A(p, k)) == 0) return false;
        if (p != k) {
            for (int j = 0; j < n; j++) std::swap(A(k, j), A(p, j));
            for (int j = 0; j < B.c; j++) std::swap(B(k, j), B(p, j));
        }
        for (int i = k + 1; i < n; i++) {
            zc f = A(i, k) / A(k, k);
            if (f == zc(0, 0)) continue;
            for (int j = k; j < n; j++) A(i, j) -= f * A(k, j);
            for (int j = 0; j < B.c; j++) B(i, j) -= f * B(k, j);
        }
    }
    for (int j = 0; j < B.c; j++)
        for (int i = n - 1; i >= 0; i--) {
            zc s = B(i, j);
            for (int l = i + 1; l < n; l++) s -= A(i, l) * B(l, j);
            B(i, j) = s / A(i, i);
        }
    return true;
}

// Eigenvalues and eigenvectors of a general complex matrix F (n x n):
// Householder reduction to Hessenberg form, single-shift QR iteration with
// Wilkinson shifts and Givens rotations to the Schur form F = Q T Q^H, then
// eigenvectors of T by back substitution, mapped back with Q.  Columns of G
// are unit eigenvectors.  Returns false if the iteration does not converge.
inline bool eig(const Mat &F, std::vector<zc> &theta, Mat &G)
{
    const int n = F.r;
    Mat H = F, Q(n, n);
    for (int i = 0; i < n; i++) Q(i, i) = 1;
    // Hessenberg reduction
    for (int k = 0; k + 2 < n; k++) {
        std::vector<zc> v(n - k - 1);
        double xn = 0;
        for (int i = k + 1; i < n; i++) {
            v[i - k - 1] = H(i, k);
            xn += std::norm(H(i, k));
        }
        xn = std::sqrt(xn);
        if (xn == 0) continue;
        zc ph = std::abs(v[0]) > 0 ? v[0] / std::abs(v[0]) : zc(1, 0);
        v[0] += ph * xn;
        double vn = 0;
        for (auto &t : v) vn += std::norm(t);
        // H <- P H P, Q <- Q P with P = I - 2 v v^H / vn (on rows/cols k+1..n-1)
        for (int j = 0; j < n; j++) {
            zc s = 0;
            for (int i = k + 1; i < n; i++) s += std::conj(v[i - k - 1]) * H(i, j);
            s *= 2.0 / vn;
            for (int i = k + 1; i < n; i++) H(i, j) -= s * v[i - k - 1];
        }
        for (int i = 0; i < n; i++) {
            zc s = 0;
            for (int j = k + 1; j < n; j++) s += H(i, j) * v[j - k - 1];
            s *= 2.0 / vn;
            for (int j = k + 1; j < n; j++) H(i, j) -= s * std::conj(v[j - k - 1]);
        }
        for (int i = 0; i < n; i++) {
            zc s = 0;
            for (int j = k + 1; j < n; j++) s += Q(i, j) * v[j - k - 1];
            s *= 2.0 / vn;
            for (int j = k + 1; j < n; j++) Q(i, j) -= s * std::conj(v[j - k - 1]);
        }
        for (int i = k + 2; i < n; i++) H(i, k) = 0;
    }
    // shifted QR iteration
    const double eps = 2.2e-16;
    int hi = n - 1, iter = 0;
    while (hi > 0) {
        if (++iter > 60 * n) return false;
        int l = hi;
        while (l > 0) {
            double sc = std::abs(H(l - 1, l - 1)) + std::abs(H(l, l));
            if (std::abs(H(l, l - 1)) <= eps * (sc > 0 ? sc : 1.0)) {
                H(l, l - 1) = 0;
                break;
            }
            l--;
        }
        if (l == hi) {
            hi--;
            continue;
        }
        // Wilkinson shift from the trailing 2x2 block
        zc a = H(hi - 1, hi - 1), b = H(hi - 1, hi), c = H(hi, hi - 1), d = H(hi, hi);
        zc tr = a + d, det = a * d - b * c;
        zc disc = std::sqrt(tr * tr / 4.0 - det);
        zc e1 = tr / 2.0 + disc, e2 = tr / 2.0 - disc;
        zc mu = std::abs(e1 - d) < std::abs(e2 - d) ? e1 : e2;
        if (iter % 11 == 0) mu += zc(std::abs(H(hi, hi - 1)), 0);  // exceptional shift
        zc x = H(l, l) - mu, y = H(l + 1, l);
        for (int k = l; k < hi; k++) {
            double nu = std::sqrt(std::norm(x) + std::norm(y));
            double cs;
            zc sn;
            if (std::abs(x) == 0) {
                cs = 0;
                sn = 1;
            } else {
                cs = std::abs(x) / nu;
                sn = (x / std::abs(x)) * std::conj(y) / nu;
            }
            // rows k, k+1 by G = [[c, s], [-conj(s), c]]
            for (int j = std::max(k - 1, 0); j < n; j++) {
                zc p = H(k, j), q = H(k + 1, j);
                H(k, j) = cs * p + sn * q;
                H(k + 1, j) = -std::conj(sn) * p + cs * q;
            }
            // columns k, k+1 by G^H
            for (int i = 0; i <= std::min(k + 2, n - 1); i++) {
                zc p = H(i, k), q = H(i, k + 1);
                H(i, k) = cs * p + std::conj(sn) * q;
                H(i, k + 1) = -sn * p + cs * q;
            }
            for (int i = 0; i < n; i++) {
                zc p = Q(i, k), q = Q(i, k + 1);
                Q(i, k) = cs * p + std::conj(sn) * q;
                Q(i, k + 1) = -sn * p + cs * q;
            }
            if (k + 1 < hi) {
                x = H(k + 1, k);
                y = H(k + 2, k);
            }
        }
    }
    theta.resize(n);
    for (int i = 0; i < n; i++) theta[i] = H(i, i);
    // eigenvectors of the triangular T, then G = Q X
    G = Mat(n, n);
    double tn = 0;
    for (auto &t : H.a) tn = std::max(tn, std::abs(t));
    const double small = eps * (tn > 0 ? tn : 1.0);
    for (int i = 0; i < n; i++) {
        std::vector<zc> xv(n, zc(0, 0));
        xv[i] = 1;
        for (int j = i - 1; j >= 0; j--) {
            zc s = 0;
            for (int l2 = j + 1; l2 <= i; l2++) s += H(j, l2) * xv[l2];
            zc den = H(j, j) - H(i, i);
            if (std::abs(den) < small) den = small;
            xv[j] = -s / den;
        }
        double nn = 0;
        for (int r = 0; r < n; r++) {
            zc s = 0;
            for (int l2 = 0; l2 <= i; l2++) s += Q(r, l2) * xv[l2];
            G(r, i) = s;
            nn += std::norm(s);
        }
        nn = std::sqrt(nn);
        for (int r = 0; r < n; r++) G(r, i) /= nn;
    }
    return true;
}

// Orthonormal columns spanning the columns of A (m x k, m >= k): modified
// Gram-Schmidt, twice.
inline Mat orthonormal(const Mat &A)
{
    Mat Q = A;
    for (int j = 0; j < A.c; j++) {
        for (int pass = 0; pass < 2; pass++)
            for (int i = 0; i < j; i++) {
                zc s = 0;
                for (int r = 0; r < A.r; r++) s += std::conj(Q(r, i)) * Q(r, j);
                for (int r = 0; r < A.r; r++) Q(r, j) -= s * Q(r, i);
            }
        double nn = 0;
        for (int r = 0; r < A.r; r++) nn += std::norm(Q(r, j));
        nn = std::sqrt(nn);
        for (int r = 0; r < A.r; r++) Q(r, j) /= nn;
    }
    return Q;
}

}  // namespace dense
}  // namespace qdd
