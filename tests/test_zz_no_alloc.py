"""vgtb_split_cgemm_noalloc: the product C = A R^dagger for callers that cannot
allocate device memory (their device memory belongs to another allocator, or
cudaMalloc's implicit synchronisation is not acceptable in their loop).

Checked through the C-ABI against the existing entry point vgtb_diag_split_chain
(the same tcgen05 BF16x3 kernel, with its own allocations), within the product
tolerance of the other split-precision tests, on two calls in a row whose sizes
differ so that the second call must overwrite what the first one left in the
shared scratch array.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from tests._gpu_util import rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2308_09782_gb300 import vgtb
    return vgtb.load()


def _noalloc(lib, a, r):
    import torch
    n = a.shape[0]
    da = torch.from_numpy(a).cuda()
    dr = torch.from_numpy(r).cuda()
    dc = torch.zeros_like(da)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.vgtb_split_cgemm_noalloc(n, C.c_void_p(da.data_ptr()), C.c_void_p(dr.data_ptr()),
                                      C.c_void_p(dc.data_ptr()), C.c_void_p(stream))
    return rc, dc.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice(lib):
    from paper_2308_09782_gb300 import vgtb
    rng = np.random.default_rng(7)
    for n in (256, 150):                       # second call: smaller n, padding must be rewritten
        a = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
        r = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
        rc, c = _noalloc(lib, a, r)
        assert rc == 0
        w_ref, _ = vgtb.diag_split_chain(a, r, np.eye(n, dtype=complex))
        assert rel_fro([c], [w_ref]) < 3e-5
        assert rel_fro([c], [a @ r.conj().T]) < 3e-5


def test_noalloc_rejects_sizes_beyond_the_scratch(lib):
    import torch
    n = 257
    d = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    rc = lib.vgtb_split_cgemm_noalloc(n, C.c_void_p(d.data_ptr()), C.c_void_p(d.data_ptr()),
                                      C.c_void_p(d.data_ptr()), None)
    assert rc == -1
    rc = lib.vgtb_split_cgemm_noalloc(0, C.c_void_p(d.data_ptr()), C.c_void_p(d.data_ptr()),
                                      C.c_void_p(d.data_ptr()), None)
    assert rc == -1
