"""GPU tests of the serving form (bcts_submit / bcts_poll): continuous batching
returns for every request exactly what searching it alone returns, under
concurrent submitters and under an admission budget that forces requests to
run one by one; ticket bookkeeping errors are reported, not raised on the GPU."""
import threading

import numpy as np
import pytest

from paper_2107_01715_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_01715_b300 import bcts
    return torch, bcts


def _requests(k, seed=900):
    rng = np.random.default_rng(seed)
    roots = inputs.root_states(range(seed, seed + k))
    ds = rng.choice([0, 1, 2, 3], size=k, p=[0.1, 0.3, 0.4, 0.2]).astype(np.int32)
    As = rng.choice([4, 9, 18], size=k).astype(np.int32)
    return roots, ds, As


def _wait(bcts, ctx, ticket, A):
    rc, a, v = bcts.bcts_poll(ctx, ticket, A, timeout_us=-1)
    assert rc == bcts.BCTS_OK
    return a, v


@pytest.mark.parametrize("budget", [0, 2 << 20])
def test_served_results_equal_alone(dev, budget):
    torch, bcts = dev
    W = inputs.qnet_weights(18)
    ctx = bcts.bcts_create(W, 18, 2, 0.99, 1.0, precision="bf16", frame_budget_bytes=budget, max_roots=8)
    roots, ds, As = _requests(24)
    tickets = [bcts.bcts_submit(ctx, roots[i:i + 1], int(ds[i]), int(As[i])) for i in range(len(roots))]
    got = [_wait(bcts, ctx, t, int(As[i])) for i, t in enumerate(tickets)]
    ref_ctx = bcts.bcts_create(W, 18, 2, 0.99, 1.0, precision="bf16")
    for i in range(len(roots)):
        a, v = bcts.bcts_search_mixed(ref_ctx, roots[i:i + 1], ds[i:i + 1], As[i:i + 1])
        assert got[i][0] == a[0], i
        assert np.array_equal(got[i][1], v[0, :As[i]]), i
    ref_ctx.close()
    ctx.close()


def test_concurrent_submitters(dev):
    torch, bcts = dev
    W = inputs.qnet_weights(18)
    ctx = bcts.bcts_create(W, 18, 2, 0.99, 1.0, precision="bf16", max_roots=16)
    roots, ds, As = _requests(40, seed=1300)
    results = {}
    lock = threading.Lock()

    def client(idx):
        for i in idx:
            t = bcts.bcts_submit(ctx, roots[i:i + 1], int(ds[i]), int(As[i]))
            r = _wait(bcts, ctx, t, int(As[i]))
            with lock:
                results[i] = r

    th = [threading.Thread(target=client, args=(list(range(j, 40, 4)),)) for j in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert len(results) == 40
    a_all, v_all = bcts.bcts_search_mixed(ctx, roots, ds, As)
    for i in range(40):
        assert results[i][0] == a_all[i] and np.array_equal(results[i][1], v_all[i, :As[i]])
    ctx.close()


def test_ticket_errors(dev):
    torch, bcts = dev
    W = inputs.qnet_weights(6)
    ctx = bcts.bcts_create(W, 6, 1, 0.99, 1.0, precision="bf16")
    with pytest.raises(bcts.BctsError) as e:
        bcts.bcts_poll(ctx, 12345, 6)
    assert e.value.code == bcts.BCTS_ENOTICKET
    root = inputs.root_states([3])
    with pytest.raises(bcts.BctsError):
        bcts.bcts_submit(ctx, root, 1, 7)  # A above the context's
    t = bcts.bcts_submit(ctx, root, 1, 6)
    _wait(bcts, ctx, t, 6)
    with pytest.raises(bcts.BctsError) as e:  # already collected
        bcts.bcts_poll(ctx, t, 6)
    assert e.value.code == bcts.BCTS_ENOTICKET
    ctx.close()


def test_served_launches_are_counted(dev):
    """bcts_profile's total includes the serving workers' kernel launches."""
    torch, bcts = dev
    A = 6
    ctx = bcts.bcts_create(inputs.qnet_weights(A), A, 2, 0.99, 1.0, precision="bf16")
    bcts.bcts_profile(ctx, False)
    roots = inputs.root_states(range(4))
    tickets = [bcts.bcts_submit(ctx, roots[i:i + 1], 2, A) for i in range(4)]
    for t in tickets:
        assert bcts.bcts_poll(ctx, t, A, timeout_us=-1)[0] == bcts.BCTS_OK
    _, _, total = bcts.bcts_profile(ctx, False)
    assert total > 0
    _, _, again = bcts.bcts_profile(ctx, False)  # read and reset
    assert again == 0
    ctx.close()
