"""GPU parity of every conv2 / conv3 kernel variant of the leaf Q-network (cp.async
gather, TMA im2col, shared-memory window, conv2 tap pairs), selected per context
with the BCTS_CONV_KERNELS mask, against the FP64 oracle and against each other.

The window kernels pad the output grid (conv2: 100 rows per node on the
space-to-depth view, conv3: 81) and read every filter tap as a row-shifted view
of one window: node counts below are chosen so that tiles straddle nodes and the
last tile is ragged (n * 100 and n * 81 not multiples of 128; the tap-pair
kernel's tiles advance by 127 rows)."""
import os

import numpy as np
import pytest

from paper_2107_01715_b300 import inputs
from tests._util import TOL, check_actions, pi_o_decided, value_close

pytestmark = pytest.mark.gpu

# bits 0 / 1: conv2 / conv3 through TMA im2col; bits 2 / 3: through windows;
# bit 4: conv2 through tap pairs (BF16, FP32-class; E4M3 ignores it)
MASKS = [0, 3, 4, 8, 12, 6, 9, 16, 18, 24]


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_01715_b300 import bcts
    return torch, bcts


def _ctx(bcts, monkeypatch, mask, A, d, precision, c=1.0, **kw):
    monkeypatch.setenv("BCTS_CONV_KERNELS", str(mask))
    W = inputs.qnet_weights(A, seed=1234)
    return bcts.bcts_create(W, A, d, 0.99, c, precision=precision, **kw), W


def _stacks(oracle_lib, n):
    states = inputs.root_states(range(300, 300 + n))
    for i in range(n):
        for a in (i % 18, (5 * i + 3) % 18, (7 * i) % 18):
            states[i], _ = oracle_lib.env_step(states[i], a)
    return np.stack([oracle_lib.render(s) for s in states])


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp8"])
@pytest.mark.parametrize("n", [1, 5, 77])
def test_qnet_variants_match_oracle(oracle_lib, dev, monkeypatch, precision, n):
    torch, bcts = dev
    A = 18
    frames = _stacks(oracle_lib, n)
    ref = oracle_lib.qnet(frames, inputs.qnet_weights(A, seed=1234), A)
    dfr = torch.from_numpy(frames.reshape(-1)).cuda()
    out = {}
    for mask in MASKS:
        ctx, _ = _ctx(bcts, monkeypatch, mask, A, 1, precision)
        dq = torch.empty(n * A, dtype=torch.float32, device="cuda")
        bcts.bcts_qnet(ctx, dfr, n, dq)
        torch.cuda.synchronize()
        ctx.close()
        q = dq.cpu().numpy().reshape(n, A)
        assert value_close(q, ref, TOL[precision]).all(), (mask, np.abs(q - ref).max())
        out[mask] = q
    # the variants sum the same products in different orders: FP32-class results
    # agree to FP32 rounding, bf16 / E4M3 ones to a rounding step of an activation
    agree = {"fp32": 1e-5, "bf16": 4e-3, "fp8": 2e-2}[precision]
    for mask in MASKS[1:]:
        d = np.abs(out[mask] - out[0]) / np.maximum(np.abs(out[0]), 1.0)
        assert d.max() <= agree, (mask, d.max())


@pytest.mark.parametrize("precision,mask", [("fp32", 12), ("fp32", 4), ("fp32", 18), ("bf16", 12), ("bf16", 3),
                                            ("bf16", 24), ("fp8", 12)])
def test_atari_scale_search_with_variant(dev, monkeypatch, precision, mask):
    """All 32 Atari-scale roots (A = 18, d = 3: 186,624 leaves in one Q-network pass,
    so each launch spans about 146,000 tiles) against the stored FP64 oracle values."""
    torch, bcts = dev
    import json
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_atari32_a18_d3.json")
    with open(path) as f:
        g = json.load(f)
    ref = np.array([r["values"] for r in g["roots"]])
    ctx, _ = _ctx(bcts, monkeypatch, mask, g["A"], g["d"], precision, c=g["correction"])
    act, val = bcts.bcts_search(ctx, inputs.root_states(g["seeds"]))
    ctx.close()
    tol = TOL[precision]
    assert value_close(val, ref, tol).all(), np.abs(val - ref).max()
    check_actions(act, ref, tol / 2 if precision != "fp32" else tol)


@pytest.mark.parametrize("mask", [4, 12, 16])
def test_ragged_chunks_with_windows(oracle_lib, dev, monkeypatch, mask):
    """Leaf chunks of 40 leaves (a window's tiles end inside a node at every chunk
    end) in every precision, against the oracle's search."""
    torch, bcts = dev
    A, d = 6, 2
    roots = inputs.root_states(range(50, 53))
    ref = oracle_lib.search(roots, inputs.qnet_weights(A, seed=1234), A, d, float(np.float32(0.99)), 1.0)
    keep = [i for i in range(3) if pi_o_decided(ref["q0"][i], TOL["fp32"])]
    for precision in ("fp32", "bf16", "fp8"):
        ctx, _ = _ctx(bcts, monkeypatch, mask, A, d, precision, leaf_chunk=40)
        act, val = bcts.bcts_search(ctx, roots)
        ctx.close()
        assert value_close(val[keep], ref["values"][keep], TOL[precision]).all(), (
            precision, np.abs(val[keep] - ref["values"][keep]).max())


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp8"])
def test_tuned_mix_bit_identical_alone(dev, monkeypatch, precision):
    """A batched call with 69,984 leaves (12 roots, A = 18, d = 3) runs the autotuner
    over leaf chunks and conv kernel variants; whatever it picks, a root's result is
    bit-identical to searching that root alone (5,832 leaves: no tuning, the
    precision's default kernels)."""
    torch, bcts = dev
    monkeypatch.delenv("BCTS_CONV_KERNELS", raising=False)
    monkeypatch.delenv("BCTS_TUNE_FILE", raising=False)
    W = inputs.qnet_weights(18, seed=1234)
    ctx = bcts.bcts_create(W, 18, 3, 0.99, 1.0, precision=precision)
    roots = inputs.root_states(range(700, 712))
    deps = np.full(12, 3, dtype=np.int32)
    acts = np.full(12, 18, dtype=np.int32)
    act, val = bcts.bcts_search_mixed(ctx, roots, deps, acts)
    for i in (0, 5, 11):
        a1, v1 = bcts.bcts_search_mixed(ctx, roots[i:i + 1], deps[i:i + 1], acts[i:i + 1])
        assert a1[0] == act[i] and np.array_equal(v1[0], val[i]), i
    ctx.close()
