"""The allocation-free entry point bcts_qnet_static, for callers that cannot
allocate device memory (allocator or memory-pool callbacks, engines that own
the whole device, hosts that forbid cudaMalloc after start-up).

After one n = 0 set-up call on the device (which loads the entry point's kernels
and places its static scratch), two calls in a row must give the same Q-values
as a context's bcts_qnet on the same plain FP32 kernels and as the FP64 oracle,
for A = 18 and A = 6, with the device's free memory unchanged across them; the
second call reuses the static scratch the first one left behind.  Batches above
BCTS_STATIC_MAX_NODES are rejected.  This file is named to be collected last."""
import numpy as np
import pytest

from paper_2107_01715_b300 import inputs
from tests._util import TOL, value_close

pytestmark = pytest.mark.gpu


def _frames(torch, bcts, seeds):
    st = inputs.root_states(seeds)
    d_st = torch.from_numpy(st.view(np.uint8).copy()).cuda()
    n = len(st)
    # advance one tick so the four history slots differ
    d_next = torch.empty(n * 18 * 80, dtype=torch.uint8, device="cuda")
    bcts.bcts_expand(d_st, None, n, 18, 1.0, d_next)
    fr = torch.empty(n * 18 * 28224, dtype=torch.uint8, device="cuda")
    bcts.bcts_render(d_next, n * 18, fr)
    return fr, n * 18


@pytest.mark.parametrize("A", [18, 6])
def test_static_qnet_matches_context_and_oracle_twice(oracle_lib, A):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_01715_b300 import bcts
    W = inputs.qnet_weights(A, seed=1234)
    d_w = torch.from_numpy(W).cuda()
    # set-up call: loads the kernels and places the static scratch on this device
    bcts.bcts_qnet_static(d_w, A, None, 0, None)
    ctx = bcts.bcts_create(W, A, 1, 0.99, 1.0, precision="fp32_simt")
    cases = [(range(0, 7), 126), (range(40, 48), 128)]  # two calls in a row, different inputs
    prepared = []
    for seeds, n in cases:  # every allocation and the context's reference first
        fr, total = _frames(torch, bcts, seeds)
        assert total >= n
        q_ref = torch.empty(n * A, dtype=torch.float32, device="cuda")
        q_static = torch.full((n * A,), float("nan"), dtype=torch.float32, device="cuda")
        bcts.bcts_qnet(ctx, fr, n, q_ref)
        prepared.append((fr, n, q_ref, q_static))
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for fr, n, _, q_static in prepared:
        bcts.bcts_qnet_static(d_w, A, fr, n, q_static)
        torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before, "the calls changed the device's free memory"
    for fr, n, q_ref, q_static in prepared:
        ref = q_ref.cpu().numpy().reshape(n, A)
        got = q_static.cpu().numpy().reshape(n, A)
        assert np.isfinite(got).all()
        assert value_close(got, ref, TOL["fp32_simt"]).all(), np.abs(got - ref).max()
        frames = fr[:n * 28224].cpu().numpy().reshape(n, 4, 84, 84)
        orq = oracle_lib.qnet(frames, W, A)
        assert value_close(got, orq, TOL["fp32_simt"]).all(), np.abs(got - orq).max()
    ctx.close()


def test_static_qnet_rejects_oversized_batch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_01715_b300 import bcts
    A = 6
    d_w = torch.from_numpy(inputs.qnet_weights(A)).cuda()
    n = bcts.BCTS_STATIC_MAX_NODES + 1
    fr = torch.zeros(n * 28224, dtype=torch.uint8, device="cuda")
    q = torch.zeros(n * A, dtype=torch.float32, device="cuda")
    with pytest.raises(bcts.BctsError) as e:
        bcts.bcts_qnet_static(d_w, A, fr, n, q)
    assert e.value.code == bcts.BCTS_EINVAL
    assert "BCTS_STATIC_MAX_NODES" in bcts.bcts_last_error(None)
