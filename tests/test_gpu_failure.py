"""Failure detection on the GPU without a fault: a device wait on an mbarrier
that nothing arrives on must give up after its bound, report through the error
word (the host sees BCTS_ETIMEOUT) and leave the device usable for a search."""
import time

import numpy as np
import pytest

from paper_2107_01715_b300 import inputs

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_device_stays_usable():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_01715_b300 import bcts
    t0 = time.perf_counter()
    assert bcts.bcts_selftest_wait(2000) == bcts.BCTS_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert "expected" in bcts.bcts_last_error(None)
    ctx = bcts.bcts_create(inputs.qnet_weights(6), 6, 2, 0.99, 1.0, precision="bf16")
    act, val = bcts.bcts_search(ctx, inputs.root_states([0, 1]))
    assert np.isfinite(val).all() and ((act >= 0) & (act < 6)).all()
    ctx.close()
    assert bcts.bcts_selftest_wait(0) == bcts.BCTS_EINVAL
