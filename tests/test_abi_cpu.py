"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point include/msgemm.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_2111_09947_gb300 import _build, _lib

HEADER = os.path.join(_build.INCLUDE_DIR, "msgemm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(msgemm_[a-z_]+)\s*\(", text)
    return sorted(set(n for n in names if not n.endswith("_fn")))


@pytest.fixture(scope="module")
def libpath():
    return _build.build_cuda()


def test_library_loads_and_exports_all_declared(libpath):
    lib = ctypes.CDLL(libpath)
    decl = declared_functions()
    assert len(decl) >= 14
    missing = [n for n in decl if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(decl) == sorted(_lib.EXPORTS)


def test_binding_loads(libpath):
    lib = _lib.load()
    assert lib.msgemm_num_kinds() == len(_lib.KIND_NAMES)


def test_sm103a_only_build_flags():
    assert _build.ARCH_FLAGS == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_handle_fails_loudly_without_a_gpu(libpath):
    """With no CUDA device the library refuses to make a handle and says so:
    the product path has no CPU fallback."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(Exception):
        _lib.Handle(torch.device("cuda", 0))
    lib = _lib.load()
    h = ctypes.c_void_p()
    status = lib.msgemm_create(ctypes.byref(h), None, _lib.ALLOC_FN(), _lib.FREE_FN(), None)
    assert status == 7 and not h.value   # MSGEMM_ERR_CUDA, no handle
