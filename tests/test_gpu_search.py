"""GPU parity of the leaf Q-network and of the full search (Alg. 1 + Eq. 3/4/7)
against the FP64 oracle, through the C ABI, per precision."""
import os

import numpy as np
import pytest

from paper_2107_01715_b300 import inputs
from tests._util import TOL, check_actions, pi_o_decided, value_close

pytestmark = pytest.mark.gpu

PRECISIONS = [p for p in os.environ.get("BCTS_TEST_PRECISIONS", "fp32_simt,fp32,bf16,fp8").split(",") if p]


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_01715_b300 import bcts
    return torch, bcts


def _ctx(bcts, A, d, gamma, c, precision, **kw):
    W = inputs.qnet_weights(A, seed=1234)
    try:
        return bcts.bcts_create(W, A, d, gamma, c, precision=precision, **kw), W
    except bcts.BctsError as e:
        if e.code == bcts.BCTS_ENOKERNEL:
            pytest.skip(f"{precision} path not available: {e}")
        raise


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("n", [1, 37, 300])
def test_qnet_matches_oracle(oracle_lib, dev, precision, n):
    torch, bcts = dev
    A = 18
    ctx, W = _ctx(bcts, A, 1, 0.99, 1.0, precision)
    states = inputs.root_states(range(n))
    for i in range(n):
        for a in (i % 18, (5 * i + 3) % 18, (7 * i) % 18):
            states[i], _ = oracle_lib.env_step(states[i], a)
    frames = np.stack([oracle_lib.render(s) for s in states])
    ref = oracle_lib.qnet(frames, W, A)
    dfr = torch.from_numpy(frames.reshape(-1)).cuda()
    dq = torch.empty(n * A, dtype=torch.float32, device="cuda")
    bcts.bcts_qnet(ctx, dfr, n, dq)
    torch.cuda.synchronize()
    q = dq.cpu().numpy().reshape(n, A)
    ok = value_close(q, ref, TOL[precision])
    assert ok.all(), (precision, np.abs(q - ref).max(), np.abs(ref).max())
    ctx.close()


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("A,d,n,c", [(6, 2, 1, 0.0), (6, 2, 1, 1.0), (6, 2, 5, 2.0), (4, 3, 3, 1.0),
                                     (9, 1, 4, 1.0), (18, 0, 6, 1.0), (1, 2, 2, 1.0), (18, 2, 2, 0.5)])
def test_search_matches_oracle(oracle_lib, dev, precision, A, d, n, c):
    torch, bcts = dev
    gamma = 0.99
    ctx, W = _ctx(bcts, A, d, gamma, c, precision)
    roots = inputs.root_states(range(n))
    act, val = bcts.bcts_search(ctx, roots)
    ref = oracle_lib.search(roots, W, A, d, float(np.float32(gamma)), c)
    tol = TOL[precision]
    # the roots' and depth-1 nodes' Q-values are FP32-class in every precision, so pi_o
    # can differ from the oracle's only where its top-2 root Q margin is within 1e-4
    keep = [i for i in range(n) if c == 0.0 or d == 0 or pi_o_decided(ref["q0"][i], TOL["fp32"])]
    ok = value_close(val[keep], ref["values"][keep], tol)
    assert ok.all(), (np.abs(val[keep] - ref["values"][keep]).max(), val, ref["values"])
    check_actions(act[keep], ref["values"][keep], tol)
    ctx.close()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_search_overlapping_sprites(oracle_lib, dev, precision):
    """Objects that share a cell in every frame (zero velocity), inside the grid
    and on its edges and corners: the later object paints over the earlier one's
    pixels (Sec. 5's renderer), which the leaves' conv1 must reproduce."""
    torch, bcts = dev
    A, d, gamma, c = 6, 2, 0.99, 1.0
    shared = [((3, 4), (2, 3)), ((0, 0), (1, 2)), ((20, 20), (1, 3)), ((10, 0), (1, 2, 3)), ((19, 7), (2, 3)),
              ((0, 20), (1, 2, 3)), ((11, 11), (1, 3))]
    roots = inputs.root_states(range(200, 200 + len(shared)))
    for i, ((x, y), objs) in enumerate(shared):
        for k in objs:
            roots["pos"][i, :, k, 0] = x
            roots["pos"][i, :, k, 1] = y
            roots["vel"][i, k] = 0
    ctx, W = _ctx(bcts, A, d, gamma, c, precision)
    act, val = bcts.bcts_search(ctx, roots)
    ref = oracle_lib.search(roots, W, A, d, float(np.float32(gamma)), c)
    tol = TOL[precision]
    keep = [i for i in range(len(shared)) if pi_o_decided(ref["q0"][i], TOL["fp32"])]
    assert value_close(val[keep], ref["values"][keep], tol).all(), np.abs(val[keep] - ref["values"][keep]).max()
    check_actions(act[keep], ref["values"][keep], tol)
    ctx.close()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_search_ragged_chunks(oracle_lib, dev, precision):
    """Leaf chunk smaller than the leaf count and not dividing it: 3 roots x 6^2
    leaves = 108 leaves in chunks of 40."""
    torch, bcts = dev
    A, d, gamma, c = 6, 2, 0.99, 1.0
    ctx, W = _ctx(bcts, A, d, gamma, c, precision, leaf_chunk=40)
    roots = inputs.root_states(range(50, 53))
    act, val = bcts.bcts_search(ctx, roots)
    ref = oracle_lib.search(roots, W, A, d, float(np.float32(gamma)), c)
    tol = TOL[precision]
    keep = [i for i in range(3) if pi_o_decided(ref["q0"][i], TOL["fp32"])]
    assert value_close(val[keep], ref["values"][keep], tol).all()
    check_actions(act[keep], ref["values"][keep], tol)
    ctx.close()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_search_empty_and_device_entry(oracle_lib, dev, precision):
    torch, bcts = dev
    A, d = 6, 2
    ctx, W = _ctx(bcts, A, d, 0.99, 1.0, precision)
    act, val = bcts.bcts_search(ctx, inputs.root_states([]))
    assert act.shape == (0,)
    roots = inputs.root_states(range(3))
    droots = torch.from_numpy(roots.view(np.uint8).copy()).cuda()
    dact = torch.full((3,), -1, dtype=torch.int32, device="cuda")
    dval = torch.zeros(3 * A, dtype=torch.float32, device="cuda")
    bcts.bcts_search_device(ctx, droots, 3, dact, dval)
    torch.cuda.synchronize()
    h_act, h_val = bcts.bcts_search(ctx, roots)
    assert np.array_equal(dact.cpu().numpy(), h_act)
    assert np.array_equal(dval.cpu().numpy().reshape(3, A), h_val)
    ctx.close()


def _stored(name):
    """Stored FP64 oracle values (tests/golden/make_oracle_values.py, oracle only)."""
    import json
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    with open(path) as f:
        g = json.load(f)
    return g, {k: np.array([r[k] for r in g["roots"]]) for k in ("values", "v_uncorrected", "action", "q0")}


@pytest.mark.parametrize("precision", [p for p in PRECISIONS if p in ("fp32", "fp32_simt")])
def test_atari_scale_all_roots(dev, precision):
    """The bench workload (32 roots, A = 18, d = 3, c = 1, FP32) in the bench's launch
    configuration: every root against the stored FP64 oracle values."""
    torch, bcts = dev
    g, ref = _stored("oracle_atari32_a18_d3.json")
    A, d, c = g["A"], g["d"], g["correction"]
    ctx, W = _ctx(bcts, A, d, 0.99, c, precision)
    roots = inputs.root_states(g["seeds"])
    act, val = bcts.bcts_search(ctx, roots)
    tol = TOL[precision]
    ok = value_close(val, ref["values"], tol)
    assert ok.all(), np.abs(val - ref["values"]).max()
    check_actions(act, ref["values"], tol)
    ctx.close()


@pytest.mark.parametrize("precision", [p for p in PRECISIONS if p in ("fp32", "bf16", "fp8")])
def test_precision_config_all_roots(dev, precision):
    """The precision form (8 roots, A = 18, d = 4, c = 1 and c = 0) in BF16 and FP8 leaf
    Q-networks, every root against the stored FP64 oracle values: values within the
    precision's tolerance, and the oracle's action wherever its top-2 margin exceeds
    that tolerance."""
    torch, bcts = dev
    g, ref = _stored("oracle_precision8_a18_d4.json")
    A, d, c = g["A"], g["d"], g["correction"]
    roots = inputs.root_states(g["seeds"])
    tol = TOL[precision]
    for cc, key in ((c, "values"), (0.0, "v_uncorrected")):
        ctx, W = _ctx(bcts, A, d, 0.99, cc, precision)
        act, val = bcts.bcts_search(ctx, roots)
        ctx.close()
        assert value_close(val, ref[key], tol).all(), (cc, np.abs(val - ref[key]).max())
        check_actions(act, ref[key], tol / 2)  # margins above the tolerance must agree


@pytest.mark.parametrize("precision", [p for p in PRECISIONS if p in ("fp32", "bf16", "fp8")])
@pytest.mark.parametrize("A,d,n,chunk", [(9, 1, 3, 0), (6, 2, 2, 0), (4, 3, 2, 0), (3, 4, 2, 0), (2, 6, 1, 0),
                                         (4, 3, 3, 50), (18, 2, 2, 100)])
def test_frame_path_matches_oracle(oracle_lib, dev, precision, A, d, n, chunk):
    """BCTS_FLAG_FRAMES: every node's newest frame rendered to device memory as its
    level is expanded, conv1 on the tensor cores over the stacks those frames form
    (roots and depth-1 nodes whole; the parents' partial maps over their slots 1-3;
    each leaf's newest slot plus its parent's map), against the oracle.  Depths 1-6
    reach every case of a slot coming from a root's stack or an inner level's
    frames; a leaf chunk below the leaf count makes ragged chunks."""
    torch, bcts = dev
    gamma, c = 0.99, 1.0
    kw = {"flags": bcts.BCTS_FLAG_FRAMES}
    if chunk:
        kw["leaf_chunk"] = chunk
    ctx, W = _ctx(bcts, A, d, gamma, c, precision, **kw)
    roots = inputs.root_states(range(600, 600 + n))
    act, val = bcts.bcts_search(ctx, roots)
    ref = oracle_lib.search(roots, W, A, d, float(np.float32(gamma)), c)
    tol = TOL[precision]
    keep = [i for i in range(n) if pi_o_decided(ref["q0"][i], TOL["fp32"])]
    assert value_close(val[keep], ref["values"][keep], tol).all(), np.abs(val[keep] - ref["values"][keep]).max()
    check_actions(act[keep], ref["values"][keep], tol)
    ctx.close()


@pytest.mark.parametrize("precision", [p for p in PRECISIONS if p in ("fp32", "bf16", "fp8")])
def test_frame_path_atari_scale_all_roots(dev, precision):
    """The frame path at the bench workload (32 roots, A = 18, d = 3): every root
    against the stored FP64 oracle values."""
    torch, bcts = dev
    g, ref = _stored("oracle_atari32_a18_d3.json")
    A, d, c = g["A"], g["d"], g["correction"]
    ctx, W = _ctx(bcts, A, d, 0.99, c, precision, flags=bcts.BCTS_FLAG_FRAMES)
    act, val = bcts.bcts_search(ctx, inputs.root_states(g["seeds"]))
    ctx.close()
    tol = TOL[precision]
    assert value_close(val, ref["values"], tol).all(), np.abs(val - ref["values"]).max()
    check_actions(act, ref["values"], tol)


@pytest.mark.parametrize("precision", [p for p in PRECISIONS if p in ("fp32", "bf16", "fp8")])
@pytest.mark.parametrize("d", [1, 2])
def test_fused_render_equals_materialised_frames(oracle_lib, dev, precision, d):
    """conv1 rendering its operand from node states must see exactly the pixels
    the frame renderer writes.  At d = 1 every node runs conv1 over its whole
    stack on both paths (same summation order): bit-identical.  At d = 2 the
    fused path takes the leaves' three older slots from per-parent partial maps
    (a different summation order), so the two agree within the tolerance."""
    torch, bcts = dev
    A = 9
    W = inputs.qnet_weights(A, seed=1234)
    roots = inputs.root_states(range(70, 76))
    out = []
    for flags in (0, bcts.BCTS_FLAG_FRAMES):
        try:
            ctx = bcts.bcts_create(W, A, d, 0.99, 1.0, precision=precision, flags=flags)
        except bcts.BctsError as e:
            if e.code == bcts.BCTS_ENOKERNEL:
                pytest.skip(str(e))
            raise
        out.append(bcts.bcts_search(ctx, roots))
        ctx.close()
    if d == 1:
        assert np.array_equal(out[0][0], out[1][0])
        assert np.array_equal(out[0][1], out[1][1])
    else:
        assert value_close(out[0][1], out[1][1], TOL[precision] / 10).all()
        check_actions(out[0][0], out[1][1].astype(np.float64), TOL[precision] / 10)


@pytest.mark.parametrize("precision", [p for p in PRECISIONS if p in ("fp32", "fp32_simt")])
@pytest.mark.parametrize("A,d,n,c", [(6, 2, 3, 1.0), (4, 3, 2, 2.0), (2, 1, 4, 1.0), (9, 1, 3, 1.0),
                                     (18, 2, 2, 1.0), (1, 2, 1, 1.0)])
def test_exact_gev_search_matches_oracle(oracle_lib, dev, precision, A, d, n, c):
    """BCTS_FLAG_EXACT_GEV: Lemma 2's exact bias gap in place of Eq. 7, against the
    oracle's exact mode (its own normal quantile, pinned to the library's)."""
    torch, bcts = dev
    gamma = 0.99
    ctx, W = _ctx(bcts, A, d, gamma, c, precision, flags=bcts.BCTS_FLAG_EXACT_GEV)
    roots = inputs.root_states(range(200, 200 + n))
    act, val = bcts.bcts_search(ctx, roots)
    ref = oracle_lib.search(roots, W, A, d, float(np.float32(gamma)), c, exact_gev=True)
    tol = TOL[precision]
    ok = value_close(val, ref["values"], tol)
    assert ok.all(), (np.abs(val - ref["values"]).max(), val, ref["values"])
    check_actions(act, ref["values"], tol)
    # the flag changes the answer wherever the two penalties differ
    if d >= 1 and A >= 3 and c > 0:
        eq7 = oracle_lib.search(roots, W, A, d, float(np.float32(gamma)), c)
        assert not np.allclose(eq7["values"], ref["values"], rtol=0, atol=1e-6)
    ctx.close()


def test_exact_gev_batched_and_served(oracle_lib, dev):
    """The flag reaches the batched form (mixed depths and action counts) and the
    serving workers."""
    torch, bcts = dev
    A = 9
    W = inputs.qnet_weights(A, seed=1234)
    ctx = bcts.bcts_create(W, A, 3, 0.99, 1.0, precision="fp32", flags=bcts.BCTS_FLAG_EXACT_GEV)
    roots = inputs.root_states(range(300, 306))
    depths = np.array([1, 2, 3, 2, 0, 3], dtype=np.int32)
    actions = np.array([9, 4, 9, 9, 9, 3], dtype=np.int32)
    act, val = bcts.bcts_search_mixed(ctx, roots, depths, actions)
    for i in range(len(roots)):
        Ai = int(actions[i])
        Wi = np.concatenate([W[:-(A * 512 + A)], W[-(A * 512 + A):-(A * 512 + A) + Ai * 512],
                             W[-A:][:Ai]]).astype(np.float32)
        ref = oracle_lib.search(roots[i:i + 1], Wi, Ai, int(depths[i]), float(np.float32(0.99)), 1.0,
                                exact_gev=True)
        assert value_close(val[i, :Ai], ref["values"][0], TOL["fp32"]).all(), (i, val[i, :Ai], ref["values"][0])
        check_actions(act[i:i + 1], ref["values"], TOL["fp32"])
        t = bcts.bcts_submit(ctx, roots[i:i + 1], int(depths[i]), Ai)
        rc, a_s, v_s = bcts.bcts_poll(ctx, t, A, timeout_us=-1)
        assert rc == bcts.BCTS_OK and a_s == act[i]
        np.testing.assert_array_equal(v_s[:Ai], val[i, :Ai])
    ctx.close()


@pytest.mark.parametrize("precision", [p for p in PRECISIONS if p in ("fp32", "fp32_simt")])
@pytest.mark.parametrize("A,d,n,sample", [(4, 3, 2, None), (6, 1, 3, None), (18, 3, 2, 60), (9, 2, 2, None)])
def test_tree_export_matches_oracle(oracle_lib, dev, precision, A, d, n, sample):
    """bcts_search_tree: every node's R and V (or a seeded sample per level) against
    the oracle's replay and recursive value; the search's own outputs unchanged."""
    torch, bcts = dev
    gamma = 0.99
    ctx, W = _ctx(bcts, A, d, gamma, 1.0, precision)
    roots = inputs.root_states(range(500, 500 + n))
    total = bcts.bcts_tree_nodes(n, A, d)
    assert total == sum(n * A ** i for i in range(1, d + 1))
    d_roots = torch.from_numpy(roots.view(np.uint8).copy()).cuda()
    d_act = torch.empty(n, dtype=torch.int32, device="cuda")
    d_val = torch.empty(n * A, dtype=torch.float32, device="cuda")
    d_R = torch.full((total,), float("nan"), dtype=torch.float32, device="cuda")
    d_V = torch.full((total,), float("nan"), dtype=torch.float32, device="cuda")
    bcts.bcts_search_tree(ctx, d_roots, n, d_act, d_val, d_R, d_V)
    torch.cuda.synchronize()
    R, V = d_R.cpu().numpy(), d_V.cpu().numpy()
    assert np.isfinite(R).all() and np.isfinite(V).all()
    act, val = bcts.bcts_search(ctx, roots)
    np.testing.assert_array_equal(d_act.cpu().numpy(), act)
    np.testing.assert_array_equal(d_val.cpu().numpy().reshape(n, A), val)
    g32 = float(np.float32(gamma))
    rng = np.random.default_rng(7)
    off = 0
    tol = TOL[precision]
    for level in range(1, d + 1):
        cnt = n * A ** level
        # the oracle's value of a depth-i node costs A^(d-i) Q-network evaluations:
        # fewer samples where the subtrees are large
        k_lvl = None if sample is None else max(2, sample // A ** (d - level))
        idx = np.arange(cnt) if k_lvl is None else rng.choice(cnt, size=min(k_lvl, cnt), replace=False)
        for k in idx:
            root, j = divmod(int(k), A ** level)
            r_ref, v_ref = oracle_lib.tree_node(roots[root], W, A, d, g32, level, j)
            assert abs(R[off + k] - r_ref) <= 1e-6 * max(abs(r_ref), 1.0), (level, k, R[off + k], r_ref)
            assert abs(V[off + k] - v_ref) <= tol * max(abs(v_ref), 1.0), (level, k, V[off + k], v_ref)
        off += cnt
    # depth-1 nodes: R + gamma V are the uncorrected root values
    ref = oracle_lib.search(roots, W, A, d, g32, 1.0)
    v1 = R[:n * A] + g32 * V[:n * A]
    assert value_close(v1.reshape(n, A), ref["v_uncorrected"], tol).all()
    ctx.close()


@pytest.mark.parametrize("precision", [p for p in PRECISIONS if p in ("fp32", "fp32_simt", "bf16")])
@pytest.mark.parametrize("A,n", [(2, 3), (3, 2)])
def test_maximum_depth_matches_oracle(oracle_lib, dev, precision, A, n):
    """d = 6, the deepest search the library accepts, on branching small enough for
    the oracle's exhaustive DFS (3^6 = 729 leaves)."""
    torch, bcts = dev
    d, gamma = 6, 0.99
    ctx, W = _ctx(bcts, A, d, gamma, 1.0, precision)
    roots = inputs.root_states(range(900, 900 + n))
    act, val = bcts.bcts_search(ctx, roots)
    ref = oracle_lib.search(roots, W, A, d, float(np.float32(gamma)), 1.0)
    tol = TOL[precision]
    keep = [i for i in range(n) if pi_o_decided(ref["q0"][i], TOL["fp32"])]
    assert value_close(val[keep], ref["values"][keep], tol).all(), np.abs(val[keep] - ref["values"][keep]).max()
    check_actions(act[keep], ref["values"][keep], tol)
    ctx.close()


def test_oversized_tree_rejected(dev):
    """n * A^d above 2^31 - 1 nodes in one level is refused before any allocation."""
    torch, bcts = dev
    A = 18
    ctx = bcts.bcts_create(inputs.qnet_weights(A), A, 6, 0.99, 1.0, precision="bf16")
    with pytest.raises(bcts.BctsError) as e:
        bcts.bcts_search(ctx, inputs.root_states(range(64)))  # 64 * 18^6 = 2.2e9 leaves
    assert e.value.code == bcts.BCTS_EINVAL
    act, val = bcts.bcts_search(ctx, inputs.root_states(range(0)))
    assert act.size == 0
    ctx.close()


@pytest.mark.parametrize("precision", [p for p in PRECISIONS if p in ("fp32", "bf16", "fp32_simt")])
def test_graph_replayed_searches_are_identical(dev, precision):
    """The host API captures a repeated root count into a CUDA graph on its second
    call and replays it afterwards: every call gives the same bits, other root
    counts in between still work, and replays count their launches."""
    torch, bcts = dev
    A, d = 9, 3
    ctx, W = _ctx(bcts, A, d, 0.99, 1.0, precision)
    roots = inputs.root_states(range(300, 305))
    other = inputs.root_states(range(310, 313))
    first = bcts.bcts_search(ctx, roots)
    ref_other = bcts.bcts_search(ctx, other)
    bcts.bcts_profile(ctx, False)
    for i in range(4):  # eager, capture, replay, replay
        act, val = bcts.bcts_search(ctx, roots)
        np.testing.assert_array_equal(act, first[0])
        np.testing.assert_array_equal(val, first[1])
        _, _, launches = bcts.bcts_profile(ctx, False)
        assert launches > 0
        a2, v2 = bcts.bcts_search(ctx, other)
        np.testing.assert_array_equal(v2, ref_other[1])
    # other roots of the same count replay the same graph with new inputs
    fresh = inputs.root_states(range(400, 405))
    act, val = bcts.bcts_search(ctx, fresh)
    ctx2, _ = _ctx(bcts, A, d, 0.99, 1.0, precision)
    act2, val2 = bcts.bcts_search(ctx2, fresh)  # a fresh context's eager answer
    np.testing.assert_array_equal(act, act2)
    np.testing.assert_array_equal(val, val2)
    ctx.close()
    ctx2.close()


@pytest.mark.parametrize("precision", [p for p in PRECISIONS if p in ("fp32", "bf16")])
def test_graph_replayed_device_searches(dev, precision):
    """The device API replays a captured graph for repeated (root count, pointers,
    stream): new inputs written into the same buffers give the eager answers, and
    other buffers or streams are separate graphs."""
    torch, bcts = dev
    A, d, n = 6, 3, 4
    ctx, W = _ctx(bcts, A, d, 0.99, 1.0, precision)
    ref_ctx, _ = _ctx(bcts, A, d, 0.99, 1.0, precision)
    d_roots = torch.empty(n * 80, dtype=torch.uint8, device="cuda")
    d_act = torch.empty(n, dtype=torch.int32, device="cuda")
    d_val = torch.empty(n * A, dtype=torch.float32, device="cuda")
    st = torch.cuda.Stream()
    for i in range(5):  # eager, capture, replays: new roots each time in the same buffers
        roots = inputs.root_states(range(100 * i, 100 * i + n))
        d_roots.copy_(torch.from_numpy(roots.view(np.uint8).copy()))
        torch.cuda.synchronize()
        bcts.bcts_search_device(ctx, d_roots, n, d_act, d_val, st)
        st.synchronize()
        act_ref, val_ref = bcts.bcts_search(ref_ctx, roots)
        np.testing.assert_array_equal(d_act.cpu().numpy(), act_ref)
        np.testing.assert_array_equal(d_val.cpu().numpy().reshape(n, A), val_ref)
    ctx.close()
    ref_ctx.close()
