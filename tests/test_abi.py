"""The C ABI without a GPU: the library builds, loads, exports every entry
point include/mcd.h declares, and rejects bad arguments on the host."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2507_21239_gb300 import build as B
from paper_2507_21239_gb300 import mcd, workloads as W

HEADER = os.path.join(B.ROOT, "include", "mcd.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return mcd.lib()


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:int|const char \*)\s*(mcd_\w+)\s*\(", text, re.M)))


def test_header_declares_the_path():
    names = declared()
    for n in ("mcd_init_disk", "mcd_collide", "mcd_transport", "mcd_regrid", "mcd_step"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(mcd_\w+)", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    for n in declared():
        getattr(lib, n)


def test_workspace_size_and_argument_checks(lib):
    P = W.benchmark_disk()
    b1 = mcd.mcd_workspace_size(P, (16, 4, 100), mcd.MCD_MIXED)
    b2 = mcd.mcd_workspace_size(P, (256, 16, 200), mcd.MCD_MIXED)
    assert 0 < b1 < b2
    # roughly linear in the particle count (about 0.1-0.2 kB per particle)
    assert 80 < b2 / (256 * 16 * 200) < 250
    two = mcd.mcd_workspace_size([P, P], [(16, 4, 100), (8, 2, 50)], mcd.MCD_FP64)
    assert two > b1
    for bad in ((0, 4, 100), (16, 0, 100), (16, 4, 0), (16, 4, 100000), (4, 100, 400)):
        with pytest.raises(mcd.McdError) as e:
            mcd.mcd_workspace_size(P, bad, mcd.MCD_MIXED)
        assert e.value.code == mcd.MCD_EINVAL
    with pytest.raises(mcd.McdError):
        mcd.mcd_workspace_size(P, (16, 4, 100), 7)
    with pytest.raises(mcd.McdError):
        mcd.mcd_workspace_size(W.benchmark_disk(r_out=0.5 * W.AU), (16, 4, 100), mcd.MCD_FP64)
    # init refuses a null workspace, a null context handle and a short workspace without touching a device
    Pa = (mcd.mcd_disk_params * 1)(mcd.mcd_disk_params.from_dict(P))
    G = (mcd.mcd_grid * 1)(mcd.mcd_grid(4, 2, 8, 0))
    h = C.c_void_p()
    assert lib.mcd_init_disk(C.byref(h), Pa, G, 1, 0, 0, None, 0, None) == mcd.MCD_EINVAL
    assert lib.mcd_init_disk(None, Pa, G, 1, 0, 0, C.c_void_p(256), 1 << 20, None) == mcd.MCD_EINVAL
    assert lib.mcd_init_disk(C.byref(h), Pa, G, 1, 0, 0, C.c_void_p(256), 64, None) == mcd.MCD_ENOMEM
    assert lib.mcd_init_disk(C.byref(h), Pa, G, 1, 0, 0, C.c_void_p(257), 1 << 30, None) == mcd.MCD_EINVAL
    for fn in ("mcd_collide", "mcd_transport", "mcd_step"):
        assert getattr(lib, fn)(None, 1.0) == mcd.MCD_EINVAL
    assert lib.mcd_regrid(None) == mcd.MCD_EINVAL
    assert lib.mcd_sync(None) == mcd.MCD_EINVAL
    assert lib.mcd_free(None) == mcd.MCD_EINVAL
    assert mcd.mcd_strerror(mcd.MCD_ETIMEOUT) == "a cell reached the event cap"


def test_binding_has_the_c_names():
    for n in declared():
        assert hasattr(mcd, n), n
