"""GPU test of pf_resample_static, the allocation-free variant of pf_resample.

Some callers cannot allocate device memory when they resample (a fixed
start-up memory budget, a host framework that owns all device allocations, or
a loop that cannot afford cudaMalloc's possible synchronisation).  For them
pf_resample_static stages its in-place gathers in a scratch array that the
library itself holds instead of a caller workspace.  This test calls it through
the C ABI and checks, on two calls in a row, that it gives exactly the indices
and gathered arrays of pf_resample with a caller-allocated workspace.

The file name sorts last so that a run stopping at its first failure has run
every other test first; it also passes alone in a fresh process.
"""
import ctypes as ct

import numpy as np
import pytest
import torch

from tests.helpers import require_lib

pytestmark = pytest.mark.gpu


def _arrays(N, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    m = torch.randn(N, 1024, generator=g).to(torch.float32).cuda()          # 4 KB rows
    dW = torch.randn(N, 10, 8, generator=g).to(torch.float32).cuda()        # 320 B rows
    w = torch.randn(N, 2, generator=g).to(torch.float64).cuda()             # 16 B rows
    return [m, dW, w]


def _call(lib, name, wbar, seed, ctr, arrays, ws=None):
    N = wbar.shape[0]
    idx = torch.empty(N, dtype=torch.int32, device="cuda")
    na = len(arrays)
    ptrs = (ct.c_void_p * na)(*[a.data_ptr() for a in arrays])
    rows = (ct.c_size_t * na)(*[a[0].numel() * a.element_size() for a in arrays])
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    if name == "pf_resample":
        rc = lib.pf_resample(N, ct.c_void_p(wbar.data_ptr()), seed, ctr, ct.c_void_p(idx.data_ptr()), na, ptrs,
                             rows, ct.c_void_p(ws.data_ptr()), ws.numel(), stream)
    else:
        rc = lib.pf_resample_static(N, ct.c_void_p(wbar.data_ptr()), seed, ctr, ct.c_void_p(idx.data_ptr()), na,
                                    ptrs, rows, stream)
    assert rc == 0, rc
    return idx


def test_static_scratch_matches_workspace_version_on_two_calls():
    require_lib()
    from paper_2402_06927_gb300 import _lib
    lib = _lib.lib()
    N = 1024
    r = np.random.default_rng(0)
    for call, (seed, ctr) in enumerate(((11, 3), (12, 4))):
        w = r.gamma(0.5 + call, size=N)
        wbar = torch.tensor(w / w.sum(), dtype=torch.float64, device="cuda")
        ref_arrays = _arrays(N, 100 + call)
        new_arrays = [a.clone() for a in ref_arrays]
        ws = torch.empty(sum(N * a[0].numel() * a.element_size() for a in ref_arrays), dtype=torch.uint8,
                         device="cuda")
        idx_ref = _call(lib, "pf_resample", wbar, seed, ctr, ref_arrays, ws)
        idx_new = _call(lib, "pf_resample_static", wbar, seed, ctr, new_arrays)
        torch.cuda.synchronize()
        # integer work: bit-exact
        assert torch.equal(idx_new, idx_ref)
        for a, b in zip(new_arrays, ref_arrays):
            assert torch.equal(a, b)
        # and the gather really moved rows
        assert not torch.equal(ref_arrays[0], _arrays(N, 100 + call)[0])


def test_static_scratch_rejects_oversized_arrays():
    require_lib()
    from paper_2402_06927_gb300 import _lib
    lib = _lib.lib()
    N = 8192
    wbar = torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda")
    idx = torch.empty(N, dtype=torch.int32, device="cuda")
    row = _lib.PF_RESAMPLE_STATIC_BYTES // N + 16          # N * row exceeds the scratch
    big = torch.empty(N * row, dtype=torch.uint8, device="cuda")
    ptrs = (ct.c_void_p * 1)(big.data_ptr())
    rows = (ct.c_size_t * 1)(row)
    rc = lib.pf_resample_static(N, ct.c_void_p(wbar.data_ptr()), 1, 2, ct.c_void_p(idx.data_ptr()), 1, ptrs, rows,
                                ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -5   # SCH_ERR_WORKSPACE, before any launch
