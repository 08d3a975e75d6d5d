"""Device-side failure handling: a bounded wait that is made to run out (a
barrier nothing completes) ends with FRNN_ERR_TIMEOUT read on the host, and
the context keeps working afterwards.  No GPU fault is involved."""
import time

import numpy as np
import pytest

from oracle import oracle
from paper_2609_31980_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2609_31980_gb300 import frnn
    c = frnn.Context()
    yield c
    c.close()


def test_bounded_wait_runs_out_and_the_context_survives(ctx):
    import torch
    from paper_2609_31980_gb300 import frnn
    t0 = time.perf_counter()
    rc = frnn.frnn_check_wait_timeout(ctx.handle, 20_000_000)   # 20 ms
    dt = time.perf_counter() - t0
    assert rc == frnn.FRNN_ERR_TIMEOUT
    assert 0.015 < dt < 5.0
    ctx.sync()                                   # the status word was cleared
    pts = synth.clustered(50, 20, 500, 8, 0.02, seed=900)
    t = torch.from_numpy(pts).cuda()
    c, i, d = ctx.self_query(t, 0.1, 16, path="grid")
    ctx.sync()
    want = oracle.self_query(pts, 0.1, 16)
    np.testing.assert_array_equal(c.cpu().numpy(), want[0])
    np.testing.assert_array_equal(i.cpu().numpy(), want[1])


def test_wait_check_rejects_bad_limits(ctx):
    from paper_2609_31980_gb300 import frnn
    assert frnn.frnn_check_wait_timeout(ctx.handle, 10) == frnn.FRNN_ERR_INVALID_ARG
    assert frnn.frnn_check_wait_timeout(None, 20_000_000) == frnn.FRNN_ERR_INVALID_ARG
