"""The C-ABI library builds, loads without a GPU, and exports every entry point include/lrfg.h declares;
the Python binding declares the same set.  No compute calls (those need a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lrfg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lrfg_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1902_07455_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["lrfg_create", "lrfg_destroy", "lrfg_problem_solve", "lrfg_problem_apply", "lrfg_tt_round",
                     "lrfg_tt_hadamard", "lrfg_fft_fibres", "lrfg_fibre_operator", "lrfg_solve"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_1902_07455_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == declared_functions()


def test_strerror_without_gpu(lib):
    lib.lrfg_strerror.restype = ctypes.c_char_p
    assert lib.lrfg_strerror(0) == b"ok"
    assert b"invalid" in lib.lrfg_strerror(1)


def test_create_rejects_null_out_pointer(lib):
    # argument checks that need no device
    assert lib.lrfg_create(None, 0, None, ctypes.c_size_t(0)) == 1


def test_product_package_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1902_07455_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f


def test_batch_entry_points_check_arguments_without_gpu(lib):
    # argument checks of the serving executor that need no device
    out = ctypes.c_void_p()
    assert lib.lrfg_batch_create(None, 0, 2, ctypes.c_size_t(0)) == 1          # null out pointer
    assert lib.lrfg_batch_create(ctypes.byref(out), 0, 0, ctypes.c_size_t(0)) == 1  # no workers
    assert lib.lrfg_batch_submit(None, None, None, None, None) == 1
    ready = ctypes.c_int()
    assert lib.lrfg_batch_poll(None, ctypes.c_ulonglong(1), 0, ctypes.byref(ready), None, None, None) == 1
    assert lib.lrfg_batch_destroy(None) == 1
    assert lib.lrfg_batch_set_group(None, 2) == 1


def test_batch_binding_without_gpu_raises():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1902_07455_gb300 as lrfg
    with pytest.raises(lrfg.LrfgError):
        lrfg.Batch(0, workers=2)


def test_host_coefficient_marshalling():
    """The executor's request structs (host buffers) for the three coefficient forms and the B array."""
    import numpy as np
    from paper_1902_07455_gb300 import _host_coeff, _set_b
    from paper_1902_07455_gb300 import _lib as L
    grid = np.ones((5, 7))
    c, keep = _host_coeff(grid)
    assert (c.d, c.fmt, c.N[0], c.N[1], c.on_device) == (2, L.LRFG_FULL, 5, 7, 0)
    _set_b(c, [[2.0, 1.0], [1.0, 3.0]])
    assert list(c.B)[:5] == [2.0, 1.0, 0.0, 1.0, 3.0]
    cores = [np.ones((1, 5, 3)), np.ones((3, 7, 2)), np.ones((2, 9, 1))]
    c, keep = _host_coeff(cores)
    assert (c.d, c.fmt, list(c.tt.r), list(c.tt.N)) == (3, L.LRFG_TT, [1, 3, 2, 1], [5, 7, 9])
    core, facs = np.ones((2, 3)), [np.ones((5, 2)), np.ones((7, 3))]
    c, keep = _host_coeff((core, facs))
    assert (c.d, c.fmt, list(c.tk.r)[:2], list(c.tk.N)[:2]) == (2, L.LRFG_TUCKER, [2, 3], [5, 7])
    with pytest.raises(ValueError):
        _set_b(c, np.ones((3, 3)))


def test_aeff_tensor_entry_point_rejects_a_null_problem(lib):
    """lrfg_problem_aeff_tensor, called directly through ctypes without a GPU: a null problem is an invalid
    argument, and nothing is written to the output array."""
    from paper_1902_07455_gb300 import _lib as L
    f = lib.lrfg_problem_aeff_tensor
    f.restype, f.argtypes = L.SIGNATURES["lrfg_problem_aeff_tensor"]
    A = (ctypes.c_double * 9)(*([7.0] * 9))
    assert f(None, A, None) == L.LRFG_EINVAL
    assert list(A) == [7.0] * 9


def test_problems_solve_rejects_bad_arguments(lib):
    """lrfg_problems_solve without a GPU: no problems, a null array or a null first problem are invalid arguments
    (checked before any device work)."""
    from paper_1902_07455_gb300 import _lib as L
    f = lib.lrfg_problems_solve
    f.restype, f.argtypes = L.SIGNATURES["lrfg_problems_solve"]
    E = (ctypes.c_double * 3)(1.0, 0.0, 0.0)
    res = (L.lrfg_result * 1)()
    hs = (ctypes.c_void_p * 1)(None)
    assert f(0, hs, E, res) == L.LRFG_EINVAL
    assert f(1, None, E, res) == L.LRFG_EINVAL
    assert f(1, hs, E, res) == L.LRFG_EINVAL
