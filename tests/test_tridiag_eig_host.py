"""The host routines of the device eigensolver (tridiag_eig.h): eigenvalues of
the Ritz matrix H_k (QL on the diagonally symmetrised tridiagonal) and its
right/left eigenvectors by (block) inverse iteration, compiled with g++ into
a small harness and checked against numpy's dense eigensolvers on
tridiagonals shaped like those of App. A (real symmetric) and App. B
(complex, H(j+1,j) H(j,j+1) not real), on split matrices and on a matrix
with every eigenvalue doubled (the repeated Ritz values of floating-point
Lanczos).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("tridiag") / "tridiag_eig_harness")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_0912_4457_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "cpp", "tridiag_eig_harness.cpp"), "-o", exe], check=True)
    return exe


def run(exe, a, b, c, queries=()):
    n = len(a)
    lines = [str(n)]
    for arr in (a, b, c):
        lines += [f"{complex(v).real:.17g} {complex(v).imag:.17g}" for v in arr]
    lines.append(str(len(queries)))
    for th, left, nv in queries:
        lines.append(f"{complex(th).real:.17g} {complex(th).imag:.17g} {int(left)} {int(nv)}")
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True).stdout
    rows = out.split("\n")
    ok = rows[0] == "ok"
    vals = np.array([complex(*map(float, r.split())) for r in rows[1:1 + n]])
    rest = [complex(*map(float, r.split())) for r in rows[1 + n:] if r.strip()]
    vecs, i = [], 0
    for _, _, nv in queries:
        vecs.append(np.array(rest[i:i + nv * n]).reshape(nv, n))
        i += nv * n
    return ok, vals, vecs


def dense(a, b, c):
    return np.diag(a) + np.diag(b, -1) + np.diag(c, 1)


def match(got, want):
    """max over want of the distance to the nearest of got, and back"""
    return max(max(np.min(np.abs(got - x)) for x in want), max(np.min(np.abs(want - x)) for x in got))


def lanczos_like(n, seed, herm):
    rng = np.random.default_rng(seed)
    if herm:
        a = rng.normal(size=n).astype(complex)
        b = (0.2 + rng.random(n - 1)).astype(complex)
        return a, b, b.copy()
    a = rng.normal(size=n) + 0.3j * rng.normal(size=n)
    d = (0.2 + rng.random(n - 1)) * np.exp(0.4j * rng.normal(size=n - 1))   # delta = r^dagger l
    b = np.sqrt(d)
    return a, b, np.conj(d) / b                                              # gamma = delta^* / beta


def test_real_symmetric_eigenvalues_and_vectors(harness):
    a, b, c = lanczos_like(200, 1, True)
    h = dense(a, b, c)
    want = np.linalg.eigvalsh(h)
    q = [(want[i], 0, 1) for i in (0, 57, 199)]
    ok, got, vecs = run(harness, a, b, c, q)
    assert ok and np.abs(got.imag).max() == 0.0
    assert match(got, want) < 1e-12 * np.abs(want).max()
    for (th, _, _), y in zip(q, vecs):
        assert np.linalg.norm(y[0]) == pytest.approx(1.0, abs=1e-13)
        assert np.linalg.norm(h @ y[0] - th * y[0]) < 1e-12 * np.abs(want).max()


def test_complex_two_sided_eigenvalues_and_left_right_vectors(harness):
    a, b, c = lanczos_like(150, 2, False)
    h = dense(a, b, c)
    want = np.linalg.eigvals(h)
    sel = want[np.argsort(np.abs(want))[:3]]
    q = [(t, left, 1) for t in sel for left in (0, 1)]
    ok, got, vecs = run(harness, a, b, c, q)
    assert ok
    assert match(got, want) < 1e-9
    for (th, left, _), y in zip(q, vecs):
        m = h.conj().T if left else h
        t = np.conj(th) if left else th
        assert np.linalg.norm(m @ y[0] - t * y[0]) < 1e-9


def test_split_matrix_and_tiny_sizes(harness):
    a, b, c = lanczos_like(40, 3, False)
    b[17] = c[17] = 0.0                              # two independent blocks
    ok, got, _ = run(harness, a, b, c)
    assert ok and match(got, np.linalg.eigvals(dense(a, b, c))) < 1e-10
    ok, got, vecs = run(harness, [2.5 - 1j], [], [], [(2.5 - 1j, 0, 1)])
    assert ok and got[0] == 2.5 - 1j and abs(abs(vecs[0][0, 0]) - 1.0) < 1e-15
    a2, b2, c2 = [1.0, 3.0], [0.5 + 0.5j], [2.0 - 1.0j]
    ok, got, _ = run(harness, a2, b2, c2)
    assert ok and match(got, np.linalg.eigvals(dense(a2, b2, c2))) < 1e-13


def test_doubled_eigenvalues_give_an_orthonormal_basis_of_the_cluster(harness):
    # two copies of one tridiagonal joined by a coupling of 1e-15: every
    # eigenvalue appears twice, the two copies agreeing to rounding
    for herm in (True, False):
        a, b, c = lanczos_like(30, 4, herm)
        A = np.concatenate([a, a])
        B = np.concatenate([b, [1e-15], b])
        C = np.concatenate([c, [1e-15], c])
        h = dense(A, B, C)
        th = np.linalg.eigvals(dense(a, b, c))
        th = th[np.argsort(np.abs(th))[:2]]
        q = [(t, 0, 2) for t in th]
        ok, got, vecs = run(harness, A, B, C, q)
        assert ok and match(got, np.linalg.eigvals(h)) < 1e-10
        for t, Y in zip(th, vecs):
            assert np.allclose(Y.conj() @ Y.T, np.eye(2), atol=1e-12)      # orthonormal
            for y in Y:
                assert np.linalg.norm(h @ y - t * y) < 1e-10
            # the two span the invariant subspace {(u, 0), (0, u)} of the
            # doubled eigenvalue (u its eigenvector of one copy): the 2 x 2
            # matrix of their components along (u, 0) and (0, u) is unitary
            w, v = np.linalg.eig(dense(a, b, c))
            u = v[:, np.argmin(np.abs(w - t))]
            u = u / np.linalg.norm(u)
            M = np.array([[np.vdot(u, y[:30]), np.vdot(u, y[30:])] for y in Y])
            assert abs(np.linalg.det(M)) == pytest.approx(1.0, abs=1e-8)


def test_refined_combination_of_a_repeated_ritz_value(harness):
    """What the eigensolver's candidates rest on: the Hermitian Lanczos
    recurrence of App. A (the oracle's, no reorthogonalisation) on 3^3 x 4 at
    k = 1200 repeats its converged eigenvalues.  For each doubled eigenvalue
    among those of H_k nearest zero, the two-vector basis of its invariant
    subspace (block inverse iteration) combined so that the last component
    vanishes lifts, through V_k, to an eigenvector of the dense A: the
    residual of V_k y is |beta_k e_k^T y| |v_{k+1}| in the recurrence."""
    from oracle import dirac, krylov
    import inputs
    dims = (3, 3, 3, 4)
    U = inputs.su3_links(dims, 31)[0]
    a = dirac.dense_A(U, dims, 0.0, -2.0)
    r = krylov.lanczos(lambda v: a @ v, inputs.gaussian_sources(dims, 41)[0], 1200)
    al, be = r.alpha.astype(complex), r.beta.astype(complex)
    ok, w, _ = run(harness, al, be, be)
    assert ok
    w = w[np.argsort(np.abs(w))][:24]
    doubled = []
    for t in w:
        if any(abs(t - d) <= 1e-8 * max(1.0, abs(d)) for d in doubled):
            continue
        if sum(abs(t - u) <= 1e-8 * max(1.0, abs(t)) for u in w) >= 2:
            doubled.append(t)
    assert len(doubled) >= 4
    _, _, vecs = run(harness, al, be, be, [(t, 0, 2) for t in doubled])

    def res(t, y):
        x = r.V @ y
        return np.linalg.norm(a @ x - t * x) / np.linalg.norm(x)

    worst_single = 0.0
    for t, Y in zip(doubled, vecs):
        assert res(t, Y[1, -1] * Y[0] - Y[0, -1] * Y[1]) < 1e-12
        worst_single = max(worst_single, min(res(t, Y[0]), res(t, Y[1])))
    # without the combination some cluster has no good vector
    assert worst_single > 1e-9


def test_defective_matrix_is_reported_and_skew_matrix_solved(harness):
    """The complex orthogonal rotations of the symmetrised QL can break down:
    [[1, 1], [-1, -1]] (symmetrised [[1, i], [i, -1]], a double eigenvalue 0
    with one eigenvector) is reported as not converged, which the eigensolver
    returns as NK_ENOTCONV; a skew tridiagonal (eigenvalues +-i sqrt 2, 0,
    the spectrum on which the sign function is undefined) is solved."""
    ok, _, _ = run(harness, [1.0, -1.0], [-1.0], [1.0])
    assert not ok
    ok, got, _ = run(harness, [0.0, 0.0, 0.0], [-1.0, -1.0], [1.0, 1.0])
    assert ok and match(got, np.array([1j * np.sqrt(2.0), 0.0, -1j * np.sqrt(2.0)])) < 1e-14
