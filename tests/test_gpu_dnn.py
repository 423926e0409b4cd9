"""GPU parity of the DNN forward-model workload (Batch-BFS over a randomly
initialised network standing in for a learned forward model, Sec. 4) against the
FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from paper_2107_01715_b300 import inputs
from tests._util import TOL, check_actions, value_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_01715_b300 import bcts
    return torch, bcts


@pytest.mark.parametrize("A,d,n,c,exact", [(2, 1, 3, 1.0, False), (2, 6, 4, 1.0, False), (2, 8, 2, 0.0, False),
                                           (10, 0, 5, 1.0, False), (10, 1, 3, 1.0, False), (10, 3, 4, 1.0, False),
                                           (10, 4, 2, 2.0, True), (3, 5, 3, 1.0, True), (1, 3, 2, 1.0, False),
                                           (32, 2, 2, 1.0, False)])
def test_dnn_search_matches_oracle(oracle_lib, dev, A, d, n, c, exact):
    torch, bcts = dev
    gamma = 0.97
    W = inputs.dnn_weights(A, seed=99)
    ctx = bcts.bcts_dnn_create(W, A, d, gamma, c, flags=bcts.BCTS_FLAG_EXACT_GEV if exact else 0)
    roots = inputs.dnn_root_states(range(1000, 1000 + n))
    act, val = bcts.bcts_dnn_search(ctx, roots)
    ref = oracle_lib.dnn_search(roots, W, A, d, float(np.float32(gamma)), c, exact_gev=exact)
    tol = TOL["fp32"]
    ok = value_close(val, ref["values"], tol)
    assert ok.all(), (np.abs(val - ref["values"]).max(), val, ref["values"])
    check_actions(act, ref["values"], tol)
    ctx.close()


def test_dnn_device_entry_and_chunked_levels(oracle_lib, dev):
    """Device pointers on a caller stream; a level of 2^21 + children crosses the
    forward model's pass limit (several chunks), sampled roots checked."""
    torch, bcts = dev
    A, d, n = 10, 5, 24  # 2.4 M leaves: the last expansion runs in two passes
    W = inputs.dnn_weights(A, seed=5)
    ctx = bcts.bcts_dnn_create(W, A, d, 0.99, 1.0)
    roots = inputs.dnn_root_states(range(n))
    d_roots = torch.from_numpy(roots).cuda()
    d_act = torch.empty(n, dtype=torch.int32, device="cuda")
    d_val = torch.empty(n * A, dtype=torch.float32, device="cuda")
    st = torch.cuda.Stream()
    bcts.bcts_dnn_search_device(ctx, d_roots, n, d_act, d_val, st)
    st.synchronize()
    act, val = d_act.cpu().numpy(), d_val.cpu().numpy().reshape(n, A)
    host_act, host_val = bcts.bcts_dnn_search(ctx, roots)
    np.testing.assert_array_equal(act, host_act)
    np.testing.assert_array_equal(val, host_val)
    sample = [0, 11, 23]
    ref = oracle_lib.dnn_search(roots[sample], W, A, d, float(np.float32(0.99)), 1.0)
    assert value_close(val[sample], ref["values"], TOL["fp32"]).all(), np.abs(val[sample] - ref["values"]).max()
    check_actions(act[sample], ref["values"], TOL["fp32"])
    ctx.close()


def test_dnn_bad_arguments(dev):
    torch, bcts = dev
    W = inputs.dnn_weights(2)
    for A, d in ((0, 2), (33, 2), (2, -1), (2, 17)):
        with pytest.raises((bcts.BctsError, ValueError)):
            bcts.bcts_dnn_create(inputs.dnn_weights(max(A, 1)) if 1 <= A <= 32 else W, A, d, 0.99, 1.0)
    ctx = bcts.bcts_dnn_create(W, 2, 16, 0.99, 1.0)
    with pytest.raises(bcts.BctsError):
        bcts.bcts_dnn_search(ctx, inputs.dnn_root_states(range(40000)))  # 40000 * 2^16 > 2^31 - 1
    act, val = bcts.bcts_dnn_search(ctx, np.zeros((0, 100), dtype=np.float32))
    assert act.size == 0
    ctx.close()


def test_dnn_misaligned_device_roots_rejected(dev):
    torch, bcts = dev
    W = inputs.dnn_weights(2)
    ctx = bcts.bcts_dnn_create(W, 2, 2, 0.99, 1.0)
    buf = torch.zeros(2 * 100 + 1, dtype=torch.float32, device="cuda")
    d_act = torch.empty(2, dtype=torch.int32, device="cuda")
    d_val = torch.empty(4, dtype=torch.float32, device="cuda")
    with pytest.raises(bcts.BctsError):
        bcts.bcts_dnn_search_device(ctx, buf.data_ptr() + 4, 2, d_act, d_val)
    ctx.close()
