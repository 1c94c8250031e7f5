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


def _index_file(path, n, d, R, nav=0, magic=b"NSGGB300", ver=1, deg=None, adj=None, extra=b""):
    import numpy as np
    deg = np.ones(n, np.int32) if deg is None else np.asarray(deg, np.int32)
    adj = np.full((n, R), -1, np.int32) if adj is None else np.asarray(adj, np.int32)
    with open(path, "wb") as f:
        f.write(magic + np.int32(ver).tobytes() + np.int64(n).tobytes() + np.array([d, R, nav], np.int32).tobytes())
        f.write(deg.tobytes() + adj.tobytes() + np.zeros((n, d), np.float32).tobytes() + extra)


def test_load_rejects_bad_files_before_any_device_call(libnsg, tmp_path):
    # every case fails in the header or content checks, before memory of the
    # claimed size is allocated or the GPU is touched
    from paper_1707_00143_gb300 import capi
    out = C.c_void_p()
    p = tmp_path / "idx.nsg"
    assert libnsg.nsg_load(str(tmp_path / "missing").encode(), None, C.byref(out)) == capi.NSG_EIO
    p.write_bytes(b"NSGGB3")  # short header
    assert libnsg.nsg_load(str(p).encode(), None, C.byref(out)) == capi.NSG_EIO
    _index_file(p, 3, 4, 2, magic=b"NOTANIDX")
    assert libnsg.nsg_load(str(p).encode(), None, C.byref(out)) == capi.NSG_EFORMAT
    _index_file(p, 3, 4, 2, ver=2)
    assert libnsg.nsg_load(str(p).encode(), None, C.byref(out)) == capi.NSG_EFORMAT
    # a header claiming 2^30 rows over a file of a few bytes
    with open(p, "wb") as f:
        import numpy as np
        f.write(b"NSGGB300" + np.int32(1).tobytes() + np.int64(1 << 30).tobytes()
                + np.array([128, 50, 0], np.int32).tobytes() + b"\0" * 64)
    assert libnsg.nsg_load(str(p).encode(), None, C.byref(out)) == capi.NSG_EFORMAT
    _index_file(p, 3, 4, 2, extra=b"\0\0\0\0")  # trailing bytes
    assert libnsg.nsg_load(str(p).encode(), None, C.byref(out)) == capi.NSG_EFORMAT
    _index_file(p, 3, 4, 2, adj=[[1, -1], [7, -1], [0, -1]])  # id out of range
    assert libnsg.nsg_load(str(p).encode(), None, C.byref(out)) == capi.NSG_EFORMAT
    _index_file(p, 3, 4, 2, deg=[1, 3, 1])  # degree above R
    assert libnsg.nsg_load(str(p).encode(), None, C.byref(out)) == capi.NSG_EFORMAT
    _index_file(p, 3, 4, 2, nav=3)  # navigating node out of range
    assert libnsg.nsg_load(str(p).encode(), None, C.byref(out)) == capi.NSG_EFORMAT
    assert out.value is None
