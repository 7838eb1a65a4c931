"""CPU oracle for the nested Krylov-Ritz sign function (Bloch & Heybrock 2009).

TEST INFRASTRUCTURE ONLY. This package is the plain, slow, FP64 reference that
the CUDA path is checked against. Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it. The product path
(``paper_0912_4457_gb300``) never imports it, and the oracle imports nothing
from the product path: the two share only the seeded input generators in
``inputs``, which hold none of the method's arithmetic.

Contents, each module citing the passage of the paper it follows:

* ``dirac``    -- gamma matrices (chiral basis), Wilson-Dirac operator D_w(mu)
                  of Sec. 2, A = gamma5 D_w(mu), dense matrix of A.
* ``signfun``  -- spectral matrix sign (Eqs. fAdef, sgnz) and the
                  Roberts-Higham iteration (Eq. Roberts).
* ``krylov``   -- Lanczos (App. A) and two-sided Lanczos (App. B).
* ``tridiag``  -- LU of pH_k and the application of H_k' (Eq. precond,
                  App. C steps 3-4) through LAPACK gttrf/gttrs, as the paper does.
* ``nested``   -- the non-nested Krylov-Ritz approximation (Eqs. non-nested,
                  non-nested-oblique), the nested method (Eq. nested, App. C
                  steps 2-6 without deflation), the p estimate (Eq. popt), the
                  sgn^2 error estimate of Sec. 3 and the overlap operator (Eq. Dovmu).
* ``precond``  -- closed forms for p_opt and the improvement factors
                  (Eqs. popt, condimp, condimpNH).
* ``deflation`` -- LR deflation of the eigenvalues of smallest modulus
                  (App. C steps 1 and 6, Sec. 3 and its footnote).
* ``nested.inner_sign_multilevel`` -- multi-level nesting (Sec. 4.5).

Pins (tests run with ``-m "not gpu"``) tie every function to something other
than itself: the free-field momentum-space closed form, gauge covariance,
gamma5-hermiticity, scipy's independent ``signm``, the paper's printed p/F
values, algebraic invariants (sgn^2 = 1, [sgn A, A] = 0, Ginsparg-Wilson) and
brute-force dense checks on tiny lattices.
"""
from . import dirac, signfun, krylov, tridiag, nested, precond, deflation  # noqa: F401
