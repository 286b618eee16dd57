"""The C-ABI library loads without a GPU and exports every call declared in include/bhmc.h."""
import ctypes
import os
import re

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "bhmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bhmc_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_call():
    from paper_1305_1825_gb300 import _build
    lib_path = _build.build()
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert len(names) >= 17
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_validation_without_gpu():
    from paper_1305_1825_gb300 import bhmc, workloads
    assert bhmc.bhmc_status_string(bhmc.ECAPACITY).startswith("depth-Dmax")
    assert "non-finite" in bhmc.bhmc_status_string(bhmc.ENONFINITE)
    # invalid parameters are rejected on the host before any CUDA call
    wl = workloads.plain(n=16)
    for bad in (dict(p=11), dict(C=1), dict(theta=1.0), dict(root_side=30.0), dict(Dmax=21)):
        d = dict(wl["params"], **bad)
        P = bhmc.make_params(d)
        h = ctypes.c_void_p()
        rc = bhmc.lib().bhmc_create(ctypes.byref(P), 16, 0, wl["q"].ctypes.data_as(ctypes.c_void_p),
                                    wl["xyz"].ctypes.data_as(ctypes.c_void_p), 0, None, ctypes.byref(h))
        assert rc == bhmc.EINVAL, bad
