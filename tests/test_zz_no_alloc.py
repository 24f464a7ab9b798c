"""The allocation-free entry point heap_sort_noalloc, through the C ABI.

It serves callers that must not allocate device memory: it runs the heap's
insert and deleteMin kernels over a heap kept in a fixed scratch array inside
the library.  Its output must equal that of the allocating entry points
(heap_create + heap_insert + heap_delete_min) on the same keys -- keys are
integers, so equal means bit for bit -- on two calls in a row, which share
the one scratch array.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1906_06504_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GHEAP_ERR_TOO_LARGE = -7
MAX_KEYS = 1 << 20


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_06504_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    L = ctypes.CDLL(build.LIB)
    f = L.heap_sort_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
    return L


def existing_path(keys):
    from paper_1906_06504_gb300.heap import GHeap
    n = keys.size
    d_in = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    with GHeap(capacity=n, k=1024) as h:
        h.insert(d_in)
        out, cnt = h.delete_min(n)
        h.sync()
        assert int(cnt.item()) == n
        return out.cpu().numpy().view(np.uint32)


def test_noalloc_sort_matches_allocating_path_twice(lib):
    stream = torch.cuda.current_stream()
    for call, n in enumerate([MAX_KEYS - 12345, MAX_KEYS]):
        keys = inputs.keys_u32(inputs.config_seed(1) + 1000 + call, n)
        d_in = torch.from_numpy(keys.view(np.int32).copy()).cuda()
        d_out = torch.empty(n, dtype=torch.int32, device="cuda")
        rc = lib.heap_sort_noalloc(ctypes.c_void_p(d_in.data_ptr()),
                                   ctypes.c_void_p(d_out.data_ptr()), n,
                                   ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        got = d_out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, existing_path(keys))
        assert np.array_equal(got, np.sort(keys))


def test_noalloc_rejects_more_than_its_scratch_holds(lib):
    d = torch.empty(8, dtype=torch.int32, device="cuda")
    rc = lib.heap_sort_noalloc(ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                               MAX_KEYS + 1, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == GHEAP_ERR_TOO_LARGE
