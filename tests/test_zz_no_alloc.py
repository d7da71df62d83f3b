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


def _noalloc(L, torch, A, B, planes, kchunk, calls=2):
    """C = A B^T through the allocation-free entry point, `calls` times in a
    row on the same device buffers; returns the result of every call."""
    M, K = A.shape
    N = B.shape[0]
    dev = torch.device("cuda", 0)
    dA = torch.tensor(A, dtype=torch.float64, device=dev)
    dB = torch.tensor(B, dtype=torch.float64, device=dev)
    dC = torch.empty((M, N), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    out = []
    for _ in range(calls):
        dC.fill_(float("nan"))
        st = L.hotrg_gemm_split_noalloc(M, N, K, planes, kchunk, ctypes.c_void_p(dA.data_ptr()),
                                        ctypes.c_void_p(dB.data_ptr()),
                                        ctypes.c_void_p(dC.data_ptr()), ctypes.c_void_p(stream))
        assert st == 0
        out.append(dC.cpu().numpy())
    return out


@pytest.mark.parametrize("planes,kchunk,M,N,K,bound", [
    (3, 1, 300, 200, 520, 4e-6),
    # accumulation chunks of 128 (the grid segment of the split): exact hi*hi sums
    (3, 2, 300, 200, 520, 5e-8),
    (3, 2, 256, 192, 1024, 5e-8),
    (2, 0, 130, 70, 264, 3e-5),
])
def test_noalloc_matches_allocating_entry_on_two_calls(planes, kchunk, M, N, K, bound):
    torch = pytest.importorskip("torch")
    import paper_1912_02780_gb300 as hot
    L = hot.lib()
    rng = np.random.default_rng(11 + M + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    ref = hot.gemm_split_check(A, B, planes=planes, kchunk=kchunk)
    scale = np.abs(A) @ np.abs(B).T
    for C in _noalloc(L, torch, A, B, planes, kchunk):
        assert np.all(np.isfinite(C))
        # same operand preparation and the same kernel as the allocating entry
        # point: the same C up to a few units in the last place
        assert np.max(np.abs(C - ref) / scale) < 1e-15
        assert np.max(np.abs(C - A @ B.T) / scale) < bound


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    import paper_1912_02780_gb300 as hot
    L = hot.lib()
    dev = torch.device("cuda", 0)
    x = torch.zeros(8, dtype=torch.float64, device=dev)
    p = ctypes.c_void_p(x.data_ptr())
    # 3 planes x 2 B x (2 x 1024 x 1024) elements = 12 MiB > 8 MiB
    assert L.hotrg_gemm_split_noalloc(1024, 1024, 1024, 3, 1, p, p, p, None) == 1
