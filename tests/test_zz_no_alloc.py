"""The allocation-free estimator entry point (ftq_estimators_noalloc).

It exists for callers that cannot let the library allocate device memory
(a framework pool owns the device memory under a fixed budget, or a
latency-sensitive loop must not trigger cudaMalloc's implicit
synchronisation).  Here it is called through the C ABI on Green's functions
produced by the context path and must reproduce the per-walker energies and
particle numbers of ftq_estimators to the parity tolerance, on two calls in
a row (the shared scratch array keeps the previous call's tables, so the
second call, on another basis size, checks that they are rewritten).

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from synthetic_inputs import WORKLOADS, gaussian_fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
RTOL = 1e-10


@pytest.fixture(scope="module")
def ftq():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2012_12228_gb300 as m
    return m


def context_estimates(ftq, wl, W, n):
    c = WORKLOADS[wl]
    p = ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W)
    f = torch.from_numpy(gaussian_fields(c["seed"], n, W, p.n_alpha)).cuda()
    p.propagate(f)
    G = p.green()
    ref = p.estimators()["per_walker"].cpu().numpy()
    torch.cuda.synchronize()
    p.close()
    return c, G, ref


def test_noalloc_estimators_match_context_path(ftq):
    lib = ftq.load_library()
    stream = torch.cuda.current_stream()
    for wl, W, n in (("ueg_n14_m57", 8, 12), ("ueg_n2_m7", 16, 22)):
        c, G, ref = context_estimates(ftq, wl, W, n)
        out = torch.full((W, 8), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.ftq_estimators_noalloc(c["N"], c["M"], c["rs"], ctypes.c_void_p(G.data_ptr()), W,
                                        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, lib.ftq_last_error(None)
        got = out.cpu().numpy()
        for col in (3, 4, 5, 6):
            scale = np.abs(ref[:, col]).max() + 1e-300
            assert np.abs(got[:, col] - ref[:, col]).max() <= RTOL * max(1.0, scale), (wl, col)


def test_noalloc_rejects_oversized_basis(ftq):
    lib = ftq.load_library()
    G = torch.zeros((1, 1), dtype=torch.complex128, device="cuda")
    out = torch.zeros((1, 8), dtype=torch.float64, device="cuda")
    st = lib.ftq_estimators_noalloc(2, 1021, 1.0, ctypes.c_void_p(G.data_ptr()), 1,
                                    ctypes.c_void_p(out.data_ptr()), None)
    assert st == -1 and b"scratch" in lib.ftq_last_error(None)
