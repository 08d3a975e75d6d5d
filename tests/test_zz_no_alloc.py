"""frnn_self_query_noalloc: the self-query that allocates nothing.

Some callers cannot allocate memory at query time (a fixed, pre-reserved
memory plan; code where an allocation is forbidden or would synchronise the
device).  This entry point keeps its grid in a fixed device array declared
by the library, so the caller passes only the points and the output rows.
Its results must equal the regular entry point's (frnn_build_grid +
frnn_query, the allocating path) bit for bit, on two calls in a row, since
every call reuses the same array; every row is also compared with the CPU
oracle, so that a fault shared by both GPU paths cannot pass.

The cases cover the array's sizing point (65,536 points in 16 dimensions),
an odd point count (the pair padding slot), a smaller call after a larger
one (stale contents in the shared array) and sizes beyond the array, which
must be rejected.

Named to be collected last, so that a failure here comes after every other
test has run.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle
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


def _assert_equal(got, want, what):
    assert np.array_equal(got[0], want[0]), f"{what}: counts differ"
    assert np.array_equal(got[1], want[1]), f"{what}: indices differ"
    assert np.array_equal(np.ascontiguousarray(got[2]).view(np.uint32),
                          np.ascontiguousarray(want[2]).view(np.uint32)), f"{what}: distances differ"


def test_noalloc_equals_regular_entry_point_and_oracle_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2609_31980_gb300 import frnn
    cases = [
        # the array's sizing point: 65,536 points in 16 dimensions
        ("65536x16", synth.clustered(2048, 25, 14336, 16, 0.02, seed=702), 0.16, 48),
        # 57,000 points in 8 dimensions, the tracking-like mix
        ("57000x8", synth.clustered(1500, 30, 12000, 8, 0.02, seed=700), 0.1, 64),
        # odd N: the grid's pair padding slot
        ("4095x3", synth.uniform(4095, 3, seed=703), 0.05, 32),
        # a small call after the larger ones: nothing stale may leak
        ("301x5", synth.uniform(301, 5, seed=704), 0.3, 16),
    ]
    with frnn.Context() as ctx:
        for name, pts, r, K in cases:
            assert len(pts) <= 65536
            t = torch.from_numpy(pts).cuda()
            c, i, d = ctx.self_query(t, r, K, path="grid")
            ctx.sync()
            regular = (c.cpu().numpy(), i.cpu().numpy(), d.cpu().numpy())
            want = oracle.self_query(pts, r, K)
            _assert_equal(regular, want, f"{name}: allocating path vs oracle")
            for call in range(2):   # the second call reuses the array the first one left
                got = _noalloc(frnn, t, r, K)
                _assert_equal(got, regular, f"{name}, call {call}: no-alloc vs allocating path")
                _assert_equal(got, want, f"{name}, call {call}: no-alloc vs oracle")
            assert want[0].sum() > 0, f"{name}: no neighbour pairs at all"


def test_noalloc_rejects_more_points_than_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2609_31980_gb300 import frnn
    # rejected on the host before any pointer is used (the pointers are never read)
    for n in (65537, 1 << 20):
        rc = frnn.frnn_self_query_noalloc(ctypes.c_void_p(16), n, 3, ctypes.c_float(0.1), 8,
                                          ctypes.c_void_p(16), ctypes.c_void_p(16),
                                          ctypes.c_void_p(16), None)
        assert rc == -1
