"""The C-ABI library loads and exports every entry point declared in include/nksign.h.

No compute calls: this runs without a GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nksign.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nk_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_0912_4457_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = declared()
    for n in ("nk_create_lattice", "nk_load_links", "nk_set_mu_mw", "nk_sign_apply", "nk_overlap_apply",
              "nk_last_error", "nk_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_0912_4457_gb300 import nksign
    assert sorted(nksign.EXPORTED) == declared()


def test_null_and_invalid_arguments_without_gpu(lib):
    """Argument checks that fail before any CUDA call."""
    lib.nk_last_error.restype = ctypes.c_char_p
    lib.nk_last_error.argtypes = [ctypes.c_void_p]
    assert lib.nk_last_error(None) == b"null context"
    lib.nk_destroy.argtypes = [ctypes.c_void_p]
    lib.nk_destroy(None)
    out = ctypes.c_void_p()
    bad = (ctypes.c_int * 4)(4, 4, 1, 4)
    assert lib.nk_create_lattice(bad, 1, ctypes.byref(out)) == -1
    assert lib.nk_create_lattice(None, 1, ctypes.byref(out)) == -1


def test_null_context_is_rejected_by_every_setter_and_wait(lib):
    """The schedule setters, the launch-shape calls and nk_wait check their
    context before touching the device."""
    P, I = ctypes.c_void_p, ctypes.c_int
    for name in ("nk_set_precision", "nk_set_df_recurrence", "nk_set_adapt_start"):
        f = getattr(lib, name)
        f.argtypes, f.restype = [P, I], I
        assert f(None, 0) == -1, name
    lib.nk_set_mu_mw.argtypes, lib.nk_set_mu_mw.restype = [P, ctypes.c_double, ctypes.c_double], I
    assert lib.nk_set_mu_mw(None, 0.3, -2.0) == -1
    lib.nk_wait.argtypes, lib.nk_wait.restype = [P, P], I
    assert lib.nk_wait(None, None) == -1
    lib.nk_get_launch.argtypes, lib.nk_get_launch.restype = [P, I, ctypes.c_uint, P], I
    assert lib.nk_get_launch(None, 12, 0, None) == -1


def test_eigensolver_rejects_null_arguments_without_gpu(lib):
    """nk_eigs_smallest checks its context and output pointers before any
    device work."""
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    f = lib.nk_eigs_smallest
    f.argtypes, f.restype = [P, P, I, I, D, P, P, P, P, P], I
    buf = (ctypes.c_double * 64)()
    found = ctypes.c_int(5)
    assert f(None, buf, 32, 4, 1e-9, buf, buf, buf, buf, ctypes.byref(found)) == -1
    assert f(None, buf, 32, 4, 1e-9, buf, buf, buf, buf, None) == -1


def test_noalloc_binding_refuses_undersized_tensors_before_any_launch():
    """inner_sign_noalloc reads n_rhs * k complex entries of each input and
    writes as many to c; a smaller tensor is refused in the binding with
    ValueError before the library is called (here with CPU tensors: the
    size check comes before the device-pointer check)."""
    torch = pytest.importorskip("torch")
    from paper_0912_4457_gb300 import nksign
    k = 64
    ok = torch.zeros((2, k), dtype=torch.complex128)
    short = torch.zeros((1, k), dtype=torch.complex128)
    for args in ((short, ok, ok, ok), (ok, short, ok, ok), (ok, ok, short, ok), (ok, ok, ok, short)):
        with pytest.raises(ValueError):
            nksign.inner_sign_noalloc(*args, 2, k, 16, 0.0, True)
    # float64 with interleaved (re, im) counts two entries per complex
    f64 = torch.zeros((2, 2 * k - 1), dtype=torch.float64)
    with pytest.raises(ValueError):
        nksign.inner_sign_noalloc(ok, ok, ok, f64, 2, k, 16, 0.0, True)
    # the right sizes pass the check and then need a CUDA tensor
    with pytest.raises(TypeError):
        nksign.inner_sign_noalloc(ok, ok, ok, ok, 2, k, 16, 0.0, True)
