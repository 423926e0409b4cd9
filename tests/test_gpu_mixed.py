"""GPU parity of the batched form (bcts_search_mixed): roots of mixed depth and
action count in one call, against the FP64 oracle per root, identical across
the eager, captured and replayed passes, and identical to searching a root alone."""
import os

import numpy as np
import pytest

from paper_2107_01715_b300 import inputs
from tests._util import TOL, check_actions, pi_o_decided, value_close

pytestmark = pytest.mark.gpu

PRECISIONS = [p for p in os.environ.get("BCTS_TEST_PRECISIONS", "fp32_simt,fp32,bf16,fp8").split(",")
              if p in ("fp32", "bf16", "fp8", "fp32_simt")]

SHAPES = [(4, 0), (4, 1), (4, 2), (4, 3), (9, 1), (9, 2), (18, 0), (18, 1), (18, 2), (9, 2), (4, 2), (18, 2), (6, 1)]


def weights_for(W18, A):
    """The A-action network that uses FC2 rows 0..A-1 of the 18-action one."""
    p = inputs.split_weights(W18, 18)
    parts = [p[k].ravel() for k in ("conv1.w", "conv1.b", "conv2.w", "conv2.b", "conv3.w", "conv3.b", "fc1.w",
                                     "fc1.b")]
    parts += [p["fc2.w"][:A].ravel(), p["fc2.b"][:A]]
    return np.concatenate(parts).astype(np.float32)


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_01715_b300 import bcts
    return torch, bcts


@pytest.mark.parametrize("precision", PRECISIONS)
def test_mixed_matches_oracle_and_is_stable(oracle_lib, dev, precision):
    torch, bcts = dev
    gamma, c = 0.99, 1.0
    W = inputs.qnet_weights(18, seed=1234)
    try:
        ctx = bcts.bcts_create(W, 18, 3, gamma, c, precision=precision)
    except bcts.BctsError as e:
        if e.code == bcts.BCTS_ENOKERNEL:
            pytest.skip(str(e))
        raise
    roots = inputs.root_states(range(500, 500 + len(SHAPES)))
    acts = np.array([a for a, _ in SHAPES], dtype=np.int32)
    deps = np.array([d for _, d in SHAPES], dtype=np.int32)
    runs = [bcts.bcts_search_mixed(ctx, roots, deps, acts) for _ in range(3)]  # eager, capture, replay
    for r in runs[1:]:
        assert np.array_equal(r[0], runs[0][0]) and np.array_equal(r[1], runs[0][1])
    act, val = runs[0]
    tol = TOL[precision]
    for i, (A, d) in enumerate(SHAPES):
        ref = oracle_lib.search(roots[i:i + 1], weights_for(W, A), A, d, float(np.float32(gamma)), c)
        assert np.all(val[i, A:] == 0.0)
        if precision not in ("fp32", "fp32_simt") and d > 0 and not pi_o_decided(ref["q0"][0], tol):
            continue  # pi_o undecided at this precision (see pi_o_decided)
        assert value_close(val[i, :A], ref["values"][0], tol).all(), (i, A, d, val[i, :A], ref["values"][0])
        check_actions(act[i:i + 1], ref["values"], tol)
    # alone vs in the mix: bit-identical
    for i in (3, 8, 12):
        a1, v1 = bcts.bcts_search_mixed(ctx, roots[i:i + 1], deps[i:i + 1], acts[i:i + 1])
        assert a1[0] == act[i] and np.array_equal(v1[0], val[i])
    ctx.close()


def test_mixed_rejects_bad_shapes(dev):
    torch, bcts = dev
    W = inputs.qnet_weights(9)
    ctx = bcts.bcts_create(W, 9, 2, 0.99, 1.0, precision="bf16")
    roots = inputs.root_states(range(2))
    with pytest.raises(bcts.BctsError) as e:
        bcts.bcts_search_mixed(ctx, roots, [1, 7], [9, 9])
    assert e.value.code == bcts.BCTS_EINVAL
    with pytest.raises(bcts.BctsError):
        bcts.bcts_search_mixed(ctx, roots, [1, 1], [9, 10])
    ctx.close()
