"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/nsg.h declares.  No compute call is made (no GPU needed); the argument
checks that run before any CUDA call are exercised."""
import ctypes as C
import os
import re
import shutil

import pytest

from paper_1707_00143_gb300 import build as nsg_build_mod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nsg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nsg_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libnsg():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    path = nsg_build_mod.build()
    from paper_1707_00143_gb300 import capi
    return capi.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("nsg_knn_init", "nsg_build", "nsg_search", "nsg_search_ex", "nsg_centroid",
                 "nsg_navigate", "nsg_collect", "nsg_prune", "nsg_connect", "nsg_recall",
                 "nsg_knn_query", "nsg_index_info", "nsg_save", "nsg_load", "nsg_free"):
        assert must in names


def test_every_declared_symbol_is_exported(libnsg):
    from paper_1707_00143_gb300 import capi
    bound = {name for name, _, _ in capi.SIGNATURES}
    for name in declared_functions():
        assert hasattr(libnsg, name), name
        assert name in bound, f"{name} has no binding"


def test_status_strings(libnsg):
    assert libnsg.nsg_status_str(0) == b"NSG_OK"
    for s in range(-1, -8, -1):
        assert libnsg.nsg_status_str(s).startswith(b"NSG_E")


def test_validation_rejects_before_any_launch(libnsg):
    from paper_1707_00143_gb300 import capi
    EINVAL = capi.NSG_EINVAL
    out = C.c_void_p()
    fake = C.c_void_p(16)  # never dereferenced: every call below fails validation first
    assert libnsg.nsg_build(None, 100, 8, 4, 10, 4, 8, 0, None, C.byref(out)) == EINVAL
    assert libnsg.nsg_build(fake, 100, 8, 100, 10, 4, 8, 0, None, C.byref(out)) == EINVAL  # K >= n
    assert libnsg.nsg_build(fake, 100, 8, 4, 10, 9, 8, 0, None, C.byref(out)) == EINVAL  # C < R
    assert libnsg.nsg_build(fake, 100, 8, 4, 10, 4, 8, 0, None, None) == EINVAL
    assert libnsg.nsg_knn_init(fake, 1, 8, 1, fake, None, None) == EINVAL  # n < 2
    assert libnsg.nsg_search(None, fake, 10, 5, 10, fake, None, None) == EINVAL
    assert libnsg.nsg_search_host(None, fake, 10, 5, 10, None, fake, None, None) == EINVAL
    assert libnsg.nsg_collect(fake, 100, 6, fake, 4, 0, 10, 8, 0, 10, fake, fake, fake, None, None) == EINVAL
    assert libnsg.nsg_recall(fake, 5, fake, 5, 3, 10, fake, None) == EINVAL  # k > ld
    info = capi.IndexInfo()
    assert libnsg.nsg_index_info(None, C.byref(info)) == EINVAL
    libnsg.nsg_free(None)  # ignored
