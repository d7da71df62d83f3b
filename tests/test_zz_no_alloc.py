"""The allocation-free split-GEMM entry point (hotrg_gemm_split_noalloc).

It exists for callers that may not call cudaMalloc (device memory owned by
another allocator, or latency-bound loops where an allocation would
synchronise the device).  It must give the same result as the allocating
entry point hotrg_gemm_split_check, call after call, while keeping all of
its scratch in the library's static device array.  This file is collected
last so that a stop-at-first-failure run has already run every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_on_two_calls():
    torch = pytest.importorskip("torch")
    import paper_1912_02780_gb300 as hot
    L = hot.lib()
    rng = np.random.default_rng(11)
    M, N, K = 300, 200, 520
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    ref = hot.gemm_split_check(A, B, planes=3, kchunk=1)
    scale = np.abs(A) @ np.abs(B).T
    dev = torch.device("cuda", 0)
    dA = torch.tensor(A, dtype=torch.float64, device=dev)
    dB = torch.tensor(B, dtype=torch.float64, device=dev)
    dC = torch.empty((M, N), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for _ in range(2):
        dC.fill_(float("nan"))
        st = L.hotrg_gemm_split_noalloc(M, N, K, 3, 1, ctypes.c_void_p(dA.data_ptr()),
                                        ctypes.c_void_p(dB.data_ptr()),
                                        ctypes.c_void_p(dC.data_ptr()), ctypes.c_void_p(stream))
        assert st == 0
        C = dC.cpu().numpy()
        assert np.all(np.isfinite(C))
        assert np.max(np.abs(C - ref) / scale) < 4e-6
        assert np.max(np.abs(C - A @ B.T) / scale) < 4e-6


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    import paper_1912_02780_gb300 as hot
    L = hot.lib()
    dev = torch.device("cuda", 0)
    x = torch.zeros(8, dtype=torch.float64, device=dev)
    p = ctypes.c_void_p(x.data_ptr())
    # 3 planes x 2 B x (2 x 1024 x 1024) elements = 12 MiB > 8 MiB
    assert L.hotrg_gemm_split_noalloc(1024, 1024, 1024, 3, 1, p, p, p, None) == 1
