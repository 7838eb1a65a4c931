// Test harness for the host tridiagonal eigen-routines of the eigensolver
// (tridiag_eig.h).  Reads from stdin: n, then n diagonal, n - 1 sub-diagonal
// and n - 1 super-diagonal complex entries (re im), then the number of
// queries and, per query, theta (re im), left (0/1) and nv.  Writes: a line
// "ok" or "fail" for the QL iteration, the n eigenvalues, and per query the
// nv vectors (n entries each).
#include <cstdio>
#include <vector>

#include "tridiag_eig.h"

using nk::cplx;

static bool rd(cplx& v) {
    double x, y;
    if (std::scanf("%lf %lf", &x, &y) != 2) return false;
    v = cplx(x, y);
    return true;
}

int main() {
    int n;
    if (std::scanf("%d", &n) != 1 || n < 1) return 2;
    std::vector<cplx> a(n), b(n > 1 ? n - 1 : 0), c(n > 1 ? n - 1 : 0);
    for (auto& v : a)
        if (!rd(v)) return 2;
    for (auto& v : b)
        if (!rd(v)) return 2;
    for (auto& v : c)
        if (!rd(v)) return 2;
    std::vector<cplx> w;
    const bool ok = nk::tridiag_eigvals(n, a.data(), b.data(), c.data(), w);
    std::printf("%s\n", ok ? "ok" : "fail");
    for (const cplx& v : w) std::printf("%.17g %.17g\n", v.real(), v.imag());
    int nq;
    if (std::scanf("%d", &nq) != 1) return 2;
    for (int q = 0; q < nq; ++q) {
        cplx th;
        int left, nv;
        if (!rd(th) || std::scanf("%d %d", &left, &nv) != 2) return 2;
        std::vector<std::vector<cplx>> Y;
        nk::tridiag_eigvecs(n, a.data(), b.data(), c.data(), th, left != 0, nv, Y);
        for (const auto& y : Y)
            for (const cplx& v : y) std::printf("%.17g %.17g\n", v.real(), v.imag());
    }
    return 0;
}
