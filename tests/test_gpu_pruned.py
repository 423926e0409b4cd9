"""GPU parity of the pruned search (index arrays of unpruned states, Sec. 4)
against the oracle's pruned search, through the C ABI.  Where two candidates'
scores are closer than the arithmetic can separate, FP32 and FP64 may keep
different nodes: values are compared on roots whose every selection is decided
by more than the tolerance, and checked for validity elsewhere."""
import os

import numpy as np
import pytest

from paper_2107_01715_b300 import inputs
from tests._util import TOL, check_actions, value_close

pytestmark = pytest.mark.gpu

PRECISIONS = [p for p in os.environ.get("BCTS_TEST_PRECISIONS", "fp32_simt,fp32,bf16,fp8").split(",")
              if p in ("fp32", "fp32_simt")]


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_01715_b300 import bcts
    return torch, bcts


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("A,d,n,keep", [(4, 4, 3, 2), (4, 4, 2, 3), (18, 3, 3, 8), (6, 5, 2, 4), (3, 3, 4, 1)])
def test_pruned_matches_oracle(oracle_lib, dev, precision, A, d, n, keep):
    torch, bcts = dev
    gamma = 0.99
    W = inputs.qnet_weights(A, seed=1234)
    ctx = bcts.bcts_create(W, A, d, gamma, 1.0, precision=precision)
    roots = inputs.root_states(range(700, 700 + n))
    act, val = bcts.bcts_search_pruned(ctx, roots, keep)
    ref = oracle_lib.search_pruned(roots, W, A, d, float(np.float32(gamma)), 1.0, keep)
    tol = TOL[precision]
    # FP32-class Q errors are below 1e-5 (measured); a kept/dropped margin of one
    # tolerance leaves the selection decided several times over
    decided = [i for i in range(n) if ref["gap"][i] > tol * max(1.0, np.abs(ref["values"][i]).max())]
    assert np.isfinite(val).all() and ((act >= 0) & (act < A)).all()
    assert decided, "every root of this case has an undecided selection: pick other seeds"
    ok = value_close(val[decided], ref["values"][decided], tol)
    assert ok.all(), (np.abs(val[decided] - ref["values"][decided]).max())
    check_actions(act[decided], ref["values"][decided], tol)
    ctx.close()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_pruned_without_pruning_is_the_search(dev, precision):
    """keep >= every level's candidate count: the full search's answer."""
    torch, bcts = dev
    A, d = 4, 3
    W = inputs.qnet_weights(A, seed=1234)
    ctx = bcts.bcts_create(W, A, d, 0.99, 1.0, precision=precision)
    roots = inputs.root_states(range(40, 45))
    act_f, val_f = bcts.bcts_search(ctx, roots)
    act_p, val_p = bcts.bcts_search_pruned(ctx, roots, A)
    assert value_close(val_p, val_f.astype(np.float64), TOL[precision] / 10).all()
    check_actions(act_p, val_f.astype(np.float64), TOL[precision] / 10)
    # d <= 2 has no level to prune: the same code path as bcts_search
    ctx2 = bcts.bcts_create(W, A, 2, 0.99, 1.0, precision=precision)
    a2, v2 = bcts.bcts_search(ctx2, roots)
    a3, v3 = bcts.bcts_search_pruned(ctx2, roots, 1)
    np.testing.assert_array_equal(a2, a3)
    np.testing.assert_array_equal(v2, v3)
    for bad in (0, 257):
        with pytest.raises(bcts.BctsError):
            bcts.bcts_search_pruned(ctx, roots, bad)
    ctx.close()
    ctx2.close()
