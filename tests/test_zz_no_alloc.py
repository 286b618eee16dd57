"""The allocation-free direct-sum energy entry point, called through the C-ABI.

bhmc_energy_direct_noalloc serves callers that cannot call cudaMalloc when they
need the energy: applications that reserve their device memory up front and
hand libraries only pre-allocated buffers, and loops that must not take the
device-wide synchronisation an allocation can cause.  It must agree with
bhmc_energy_direct, whose scratch comes from cudaMalloc, and with the FP64 CPU
oracle's direct sum, on two calls in a row (the second call reuses the fixed
scratch left by the first).  This file is named so that pytest collects it
last.
"""
import ctypes

import pytest

from paper_1305_1825_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_direct_energy_matches_allocating_call():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_1305_1825_gb300 import bhmc
    lib = bhmc.lib()
    lib.bhmc_energy_direct_noalloc.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    stream = torch.cuda.current_stream()
    for wl in (W.colloid(n=3000, seed=21), W.plain(n=1777, seed=22)):
        ctx = bhmc.Context(wl)
        ref = ctx.energy_direct()
        q, x = ctx.charges()
        # the oracle's O(N^2) sum of Eq. (1.1) over the same charges (FP64, CPU)
        ref_or = oracle.direct_energy_raw(q, x, wl["params"]["lB"])
        qd = torch.tensor(q, dtype=torch.float64, device="cuda")
        xd = torch.tensor(x.reshape(-1), dtype=torch.float64, device="cuda")
        for _ in range(2):
            E = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            rc = lib.bhmc_energy_direct_noalloc(len(q), qd.data_ptr(), xd.data_ptr(), wl["params"]["lB"],
                                                E.data_ptr(), stream.cuda_stream)
            assert rc == bhmc.OK, bhmc.bhmc_status_string(rc)
            torch.cuda.synchronize()
            # same FP64 pair sums, partials added in a different order
            assert E.item() == pytest.approx(ref, rel=1e-9)
            assert E.item() == pytest.approx(ref_or, rel=1e-9)
        ctx.close()
    # sizes beyond the fixed scratch are refused before any launch
    rc = lib.bhmc_energy_direct_noalloc(1048577, qd.data_ptr(), xd.data_ptr(), 1.0, E.data_ptr(),
                                        stream.cuda_stream)
    assert rc == bhmc.ESCRATCH
