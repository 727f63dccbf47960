"""CPU checks of the C-ABI boundary: the library loads without a GPU and
exports every function include/isort.h declares; the Python binding declares
the same set; argument errors are reported before any CUDA work."""
import ctypes
import os
import subprocess

import pytest

from tests._util import header_functions

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    import paper_1708_09495_gb300 as isort
    from paper_1708_09495_gb300 import _build

    _build.build()
    return isort.load()


def declared():
    names = []
    for h in HEADERS:
        names += header_functions(h)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared()
    for must in ("isort_radix", "isort_radix_u64", "isort_btn", "isort_oet", "isort_status_string"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_only_declared_symbols_are_exported(lib):
    import paper_1708_09495_gb300 as isort

    out = subprocess.run(["nm", "-D", "--defined-only", isort.LIB_PATH], capture_output=True, text=True).stdout
    exported = sorted({ln.split()[-1] for ln in out.splitlines() if " T " in ln})
    assert exported == declared()


def test_binding_covers_the_header():
    import paper_1708_09495_gb300 as isort

    assert sorted(n for n, _, _ in isort.SIGNATURES) == declared()


def test_status_strings(lib):
    for code, name in {0: "ISORT_OK", 2: "ISORT_ERR_KEY_RANGE", 5: "ISORT_ERR_TIMEOUT"}.items():
        assert lib.isort_status_string(code).decode() == name


def test_argument_errors_need_no_gpu(lib):
    # validated on the host before any CUDA call
    assert lib.isort_radix(None, None, 100, 33, 8, None) == 1
    assert lib.isort_radix(None, None, 100, 32, 0, None) == 1
    assert lib.isort_radix(None, None, 100, 32, 17, None) == 1
    assert lib.isort_radix_u64(None, None, 100, 65, 8, None) == 1
    assert lib.isort_radix(None, None, 0, 32, 8, None) == 0
    assert lib.isort_radix(None, None, 1 << 30, 32, 8, None) == 6
    assert lib.isort_btn_p(None, None, 10, 3, None, None) == 1
    assert lib.isort_oet_p(None, None, 10, 0, None, None) == 1
    assert lib.isort_btn_p(None, None, 1 << 20, 1024, None, None) == 6
    assert lib.isort_set_spin_limit(0) == 1
    assert lib.isort_count_round(None, None, None, None, 10, 30, 8, None) == 1
    # typed keys: key type, digit width and buffers are checked first
    assert lib.isort_radix_typed(None, 7, None, 100, 8, None) == 1
    assert lib.isort_radix_typed(None, 2, None, 100, 17, None) == 1
    assert lib.isort_radix_typed(None, 2, None, 100, 8, None) == 1
    assert lib.isort_radix_typed(None, 2, None, 1, 8, None) == 0
    # learned sort: bucket count and model are checked first
    assert lib.isort_learned(None, None, 100, 0, 1, 0, None, None) == 1
    assert lib.isort_learned(None, None, 100, 0, 65536, 0, None, None) == 1
    assert lib.isort_learned(None, None, 100, 0, 0, 3, None, None) == 1
    # the MLP model's entry points
    assert lib.isort_mlp_loss_grad(None, 10, None, None, None, None) == 1
    assert lib.isort_mlp_train(None, 1, 32, None, None, None, None, None) == 1


def test_graft_entry_build_is_importable():
    import __graft_entry__ as g

    assert callable(g.build) and callable(g.smoke)
