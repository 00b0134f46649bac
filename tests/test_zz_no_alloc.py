"""vrs_sort_pairs_noalloc against vrs_sort_pairs, through the C ABI.

Some callers of this library cannot allocate GPU memory at the moment they sort: a
frame callback with a hard latency budget (cudaMalloc / cudaFree can synchronise the
device), an application whose own pool owns all GPU memory, code that must not fail
mid-frame on memory pressure.  They use the allocation-free entry point, which works
from a scratch array built into the library.  This file is collected last, so that a
run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

MAX_PAIRS = 1 << 20  # VRS_SORT_NOALLOC_MAX_PAIRS


@pytest.fixture(scope="module")
def lib():
    from paper_2505_10144_gb300 import build
    build.build()
    from paper_2505_10144_gb300 import _lib
    return _lib.load()


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _keys(rng, n):
    keys = rng.integers(0, 1 << 63, size=n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=n, dtype=np.uint64)
    keys[: n // 3] = keys[n // 2]  # repeated keys: the order must stay stable
    return torch.from_numpy(keys.view(np.int64)).cuda(), torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()


def test_noalloc_sort_matches_the_context_sort_on_two_calls(lib):
    from paper_2505_10144_gb300 import api
    R = api.Renderer()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (n, bits) in enumerate([(300_001, 46), (MAX_PAIRS, 64)]):
        k, v = _keys(np.random.default_rng(call), n)
        ref_k, ref_v = R.sort_pairs(k, v, bits)
        out_k, out_v = torch.empty_like(k), torch.empty_like(v)
        status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
        rc = lib.vrs_sort_pairs_noalloc(_p(k), _p(v), _p(out_k), _p(out_v), n, bits, _p(status), stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(out_k, ref_k) and torch.equal(out_v, ref_v)
    R.close()


def test_noalloc_sort_in_place_partial_digit_and_no_allocation(lib):
    """In place (out = in), with a last digit of fewer than 8 bits (bits = 5, 13), and
    without allocating: after a first call, which loads the library's module on this
    device, further calls leave the device's free memory and torch's allocator as they
    were."""
    from paper_2505_10144_gb300 import api
    R = api.Renderer()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = []
    for call, (n, bits) in enumerate([(4097, 5), (200_003, 13), (65_536, 64)]):
        k0, v0 = _keys(np.random.default_rng(100 + call), n)
        ref_k, ref_v = R.sort_pairs(k0, v0, bits)
        cases.append((k0, v0, ref_k, ref_v, n, bits))
    del k0, v0, ref_k, ref_v  # only the list holds the tensors: nothing is freed below
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    warm_k, warm_v = cases[0][0].clone(), cases[0][1].clone()
    assert lib.vrs_sort_pairs_noalloc(_p(warm_k), _p(warm_v), _p(warm_k), _p(warm_v), cases[0][4], cases[0][5],
                                      _p(status), stream) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for k, v, ref_k, ref_v, n, bits in cases:
        rc = lib.vrs_sort_pairs_noalloc(_p(k), _p(v), _p(k), _p(v), n, bits, _p(status), stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(k, ref_k) and torch.equal(v, ref_v), (n, bits)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == alloc0
    R.close()


def test_noalloc_sort_rejects_more_than_its_maximum(lib):
    k = torch.zeros(4, dtype=torch.int64, device="cuda")
    v = torch.zeros(4, dtype=torch.int32, device="cuda")
    rc = lib.vrs_sort_pairs_noalloc(_p(k), _p(v), _p(k), _p(v), MAX_PAIRS + 1, 32, None, None)
    assert rc == 1  # VRS_ERR_INVALID, nothing launched
