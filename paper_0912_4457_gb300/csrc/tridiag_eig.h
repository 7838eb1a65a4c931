// Host routines for the eigenvalues and eigenvectors of a complex tridiagonal
// matrix H (the Ritz matrix H_k of the outer (two-sided) Lanczos recurrence),
// used by the eigensolver of the deflation (eigen.cu):
//
//  * tridiag_eigvals: all eigenvalues, by the QL algorithm with implicit
//    Wilkinson shifts applied to the complex symmetric tridiagonal matrix
//    similar to H (diagonal similarity: off-diagonal sqrt(H(j+1,j) H(j,j+1)),
//    so the eigenvalues are those of H).  For a Hermitian H this is the
//    classical symmetric QL; for a complex symmetric matrix the same
//    rotations are complex orthogonal (c^2 + s^2 = 1) and the iteration can in
//    principle break down (c^2 + s^2 = 0), which is reported.
//  * tridiag_eigvecs: right (or, with `left`, left) eigenvectors of H for an
//    eigenvalue, a basis of the invariant subspace of a cluster of nearly
//    equal eigenvalues, by block inverse iteration with a tridiagonal LU with
//    partial pivoting.
//
// Written from the algorithms' definitions (QL with implicit shifts; inverse
// iteration); no library.  Header-only, host C++.
#pragma once

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace nk {

typedef std::complex<double> cplx;

// Eigenvalues of the tridiagonal H with diagonal a[0..n-1], sub-diagonal
// b[0..n-2] (H(j+1, j)) and super-diagonal c[0..n-2] (H(j, j+1)) into w.
// Returns false if the iteration breaks down or does not converge.
inline bool tridiag_eigvals(int n, const cplx* a, const cplx* b, const cplx* c, std::vector<cplx>& w) {
    w.assign(a, a + n);
    std::vector<cplx> e(n, cplx(0.0));
    for (int j = 0; j + 1 < n; ++j) e[j] = std::sqrt(b[j] * c[j]);   // symmetrised off-diagonal
    std::vector<cplx>& d = w;
    for (int l = 0; l < n; ++l) {
        int iter = 0;
        int m;
        do {
            // the first negligible off-diagonal element at or after l
            for (m = l; m + 1 < n; ++m) {
                const double dd = std::abs(d[m]) + std::abs(d[m + 1]);
                if (std::abs(e[m]) <= 1e-16 * dd) break;
            }
            if (m != l) {
                if (++iter > 60) return false;
                // Wilkinson shift from the leading 2 x 2 block at l
                cplx g = (d[l + 1] - d[l]) / (2.0 * e[l]);
                cplx r = std::sqrt(g * g + 1.0);
                // the root of larger modulus in the denominator
                const cplx gp = g + r, gm = g - r;
                const cplx den = std::abs(gp) >= std::abs(gm) ? gp : gm;
                g = d[m] - d[l] + e[l] / den;
                cplx s(1.0), cc(1.0), p(0.0);
                int i;
                for (i = m - 1; i >= l; --i) {
                    cplx f = s * e[i];
                    const cplx bb = cc * e[i];
                    r = std::sqrt(f * f + g * g);
                    e[i + 1] = r;
                    if (std::abs(r) == 0.0) {   // deflation at i: restart from l
                        d[i + 1] -= p;
                        e[m] = 0.0;
                        break;
                    }
                    s = f / r;
                    cc = g / r;
                    g = d[i + 1] - p;
                    r = (d[i] - g) * s + 2.0 * cc * bb;
                    p = s * r;
                    d[i + 1] = g + p;
                    g = cc * r - bb;
                }
                if (std::abs(r) == 0.0 && i >= l) continue;
                d[l] -= p;
                e[l] = g;
                e[m] = 0.0;
            }
        } while (m != l);
    }
    for (const cplx& v : w)
        if (!std::isfinite(v.real()) || !std::isfinite(v.imag())) return false;
    return true;
}

// Inverse iteration for an eigenvalue theta of H that may be repeated (a
// cluster of nv nearly equal eigenvalues, as floating-point Lanczos produces
// for converged Ritz values): nv vectors spanning the invariant subspace of
// the cluster, (H - theta) Y ~ 0 (left: (H - theta)^dagger Y ~ 0), each of
// unit norm and orthogonal to the ones before.  Block inverse iteration from
// fixed start vectors: three solves of the shifted system by LU with partial
// pivoting (the shift perturbed by a relative 1e-13 so that the factorisation
// does not meet an exact zero pivot), modified Gram-Schmidt after each.
inline void tridiag_eigvecs(int n, const cplx* a, const cplx* b, const cplx* c, cplx theta, bool left, int nv,
                            std::vector<std::vector<cplx>>& Y) {
    const double scale = std::max(1.0, std::abs(theta));
    const cplx sh = theta + cplx(1e-13 * scale, 1e-13 * scale);
    // the matrix to factor: H - sh, or its conjugate transpose
    std::vector<cplx> dl(n > 1 ? n - 1 : 0), d(n), du(n > 1 ? n - 1 : 0), du2(n > 2 ? n - 2 : 0, cplx(0.0));
    for (int j = 0; j < n; ++j) d[j] = left ? std::conj(a[j] - sh) : a[j] - sh;
    for (int j = 0; j + 1 < n; ++j) {
        dl[j] = left ? std::conj(c[j]) : b[j];   // sub-diagonal
        du[j] = left ? std::conj(b[j]) : c[j];   // super-diagonal
    }
    std::vector<int> piv(n, 0);
    // LU with partial pivoting (rows j and j + 1 interchanged when |d_j| < |dl_j|)
    for (int j = 0; j + 1 < n; ++j) {
        if (std::abs(d[j]) >= std::abs(dl[j])) {
            const cplx f = std::abs(d[j]) > 0.0 ? dl[j] / d[j] : cplx(0.0);
            dl[j] = f;
            d[j + 1] -= f * du[j];
        } else {
            const cplx f = d[j] / dl[j];
            d[j] = dl[j];
            dl[j] = f;
            const cplx t = du[j];
            du[j] = d[j + 1];
            d[j + 1] = t - f * d[j + 1];
            if (j + 2 < n) {
                du2[j] = du[j + 1];
                du[j + 1] = -f * du[j + 1];
            }
            piv[j] = 1;
        }
    }
    for (int j = 0; j < n; ++j)
        if (std::abs(d[j]) == 0.0) d[j] = cplx(1e-300);
    auto solve = [&](std::vector<cplx>& y) {
        for (int j = 0; j + 1 < n; ++j) {   // L
            if (piv[j]) std::swap(y[j], y[j + 1]);
            y[j + 1] -= dl[j] * y[j];
        }
        for (int j = n - 1; j >= 0; --j) {   // U
            cplx t = y[j];
            if (j + 1 < n) t -= du[j] * y[j + 1];
            if (j + 2 < n) t -= du2[j] * y[j + 2];
            y[j] = t / d[j];
        }
    };
    auto orthonormalise = [&](int upto) {
        for (int i = 0; i < upto; ++i) {
            for (int q = 0; q < i; ++q) {
                cplx h(0.0);
                for (int j = 0; j < n; ++j) h += std::conj(Y[q][j]) * Y[i][j];
                for (int j = 0; j < n; ++j) Y[i][j] -= h * Y[q][j];
            }
            double nrm = 0.0;
            for (const cplx& v : Y[i]) nrm += std::norm(v);
            nrm = std::sqrt(nrm);
            if (nrm > 0.0)
                for (cplx& v : Y[i]) v /= nrm;
        }
    };
    Y.assign(nv, std::vector<cplx>(n));
    for (int i = 0; i < nv; ++i)
        for (int j = 0; j < n; ++j)
            Y[i][j] = cplx(1.0 + 0.5 * std::sin(1.7 * j + 1.1 * i), 0.3 * std::cos(0.9 * j + 2.3 * i));
    orthonormalise(nv);
    for (int rep = 0; rep < 3; ++rep) {
        for (int i = 0; i < nv; ++i) solve(Y[i]);
        orthonormalise(nv);
    }
}

// One eigenvector of H for a simple eigenvalue theta (tridiag_eigvecs with nv = 1).
inline void tridiag_eigvec(int n, const cplx* a, const cplx* b, const cplx* c, cplx theta, bool left,
                           std::vector<cplx>& y) {
    std::vector<std::vector<cplx>> Y;
    tridiag_eigvecs(n, a, b, c, theta, left, 1, Y);
    y.swap(Y[0]);
}

}  // namespace nk
