"""frnn_self_query_noalloc: the self-query that allocates nothing.

Some callers cannot allocate memory at query time (a fixed, pre-reserved
memory plan; code where an allocation is forbidden or would synchronise the
device).  This entry point keeps its grid in a fixed device array declared
by the library, so the caller passes only the points and the output rows.
Its results must equal the regular entry point's (frnn_build_grid +
frnn_query, the allocating path) bit for bit, on two calls in a row, since
every call reuses the same array.

Named to be collected last, so that a failure here comes after every other
test has run.
"""
import ctypes

import numpy as np
import pytest

from paper_2609_31980_gb300 import synth

pytestmark = pytest.mark.gpu


def _noalloc(frnn, t, r, K):
    import torch
    n = t.shape[0]
    c = torch.empty(n, dtype=torch.int32, device="cuda")
    i = torch.empty((n, K), dtype=torch.int32, device="cuda")
    d = torch.empty((n, K), dtype=torch.float32, device="cuda")
    rc = frnn.frnn_self_query_noalloc(ctypes.c_void_p(t.data_ptr()), n, t.shape[1],
                                      ctypes.c_float(r), K, ctypes.c_void_p(c.data_ptr()),
                                      ctypes.c_void_p(i.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, frnn.STATUS_NAMES.get(rc, rc)
    return c.cpu().numpy(), i.cpu().numpy(), d.cpu().numpy()


def test_noalloc_equals_regular_entry_point_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2609_31980_gb300 import frnn
    cases = [(synth.clustered(1500, 30, 12000, 8, 0.02, seed=700), 0.1, 64),   # 57,000 points
             (synth.uniform(4096, 3, seed=701), 0.05, 32)]                     # then a smaller one
    with frnn.Context() as ctx:
        for pts, r, K in cases:
            t = torch.from_numpy(pts).cuda()
            got = _noalloc(frnn, t, r, K)
            c, i, d = ctx.self_query(t, r, K, path="grid")
            ctx.sync()
            want = (c.cpu().numpy(), i.cpu().numpy(), d.cpu().numpy())
            np.testing.assert_array_equal(got[0], want[0])
            np.testing.assert_array_equal(got[1], want[1])
            np.testing.assert_array_equal(got[2].view(np.uint32), want[2].view(np.uint32))


def test_noalloc_rejects_more_points_than_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2609_31980_gb300 import frnn
    rc = frnn.frnn_self_query_noalloc(ctypes.c_void_p(16), 65537, 3, ctypes.c_float(0.1), 8,
                                      ctypes.c_void_p(16), ctypes.c_void_p(16),
                                      ctypes.c_void_p(16), None)
    assert rc == -1
