"""Pin the oracle's search (Eq. 1, Prop. 1, Eq. 3, Eq. 4, Eq. 7, Alg. 1).

* Brute force: enumerate every action sequence of length d, replay it, score it
  with the flat sum of Eq. 1 (sum_t gamma^t r_t + gamma^d max_a Q(s_d, a)), take
  the max per first action -- must equal the oracle's recursive DFS.
* d = 0 is the base agent pi_o (Sec. 5.1); correction 0 is vanilla tree search.
* The correction moves only actions a != pi_o, each by exactly gamma^d c B (Eq. 3).
* Closed forms: with every Q-net weight zero, Q(s, .) = b_fc2 for every state,
  so V(a) = best discounted d-step return + gamma^d max(b_fc2); hand-built
  environments give those returns by counting steps.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2107_01715_b300 import inputs

FAR = [(0, 0), (20, 0), (0, 20)]


def brute_force(oracle_lib, root, W, A, d, gamma, c):
    q0 = oracle_lib.qnet(oracle_lib.render(root)[None], W, A)[0]
    pi_o = int(np.argmax(q0))  # numpy argmax returns the first maximum
    if d == 0:
        return q0, q0.copy(), pi_o, None
    best = np.full(A, -np.inf)
    for acts in itertools.product(range(A), repeat=d):
        s, ret = root, 0.0
        for t, a in enumerate(acts):
            s, r = oracle_lib.env_step(s, a)
            ret += gamma ** t * r
        leaf_q = oracle_lib.qnet(oracle_lib.render(s)[None], W, A)[0]
        ret += gamma ** d * leaf_q.max()
        best[acts[0]] = max(best[acts[0]], ret)
    # Prop. 1: Bellman error from depths 0 and 1
    delta = np.zeros(A)
    for a in range(A):
        s1, r = oracle_lib.env_step(root, a)
        q1 = oracle_lib.qnet(oracle_lib.render(s1)[None], W, A)[0]
        delta[a] = r + gamma * q1.max() - q0[a]
    d_o = abs(delta[pi_o])
    d_e = np.mean([abs(delta[a]) for a in range(A) if a != pi_o]) if A > 1 else 0.0
    # Eq. 7 through its Lemma 3 form at sigma = delta / sqrt(2)
    se, so = d_e / math.sqrt(2), d_o / math.sqrt(2)
    B = math.sqrt(2 * math.log(A)) * (se * math.sqrt(d) - so * math.sqrt(d - 1)) - (se - so) / 2
    corrected = np.array([best[a] - (0.0 if a == pi_o else gamma ** d * c * B) for a in range(A)])
    return q0, best, pi_o, corrected


@pytest.mark.parametrize("A,d,seed", [(3, 1, 0), (3, 2, 1), (4, 2, 2), (3, 3, 3), (2, 3, 4), (6, 1, 5)])
@pytest.mark.parametrize("c", [0.0, 1.0, 2.5])
def test_search_equals_brute_force(oracle_lib, A, d, seed, c):
    gamma = 0.97
    W = inputs.qnet_weights(A, seed=100 + seed)
    root = inputs.root_states([seed])
    res = oracle_lib.search(root, W, A, d, gamma, c)
    q0, best, pi_o, corrected = brute_force(oracle_lib, root[0], W, A, d, gamma, c)
    np.testing.assert_allclose(res["q0"][0], q0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(res["v_uncorrected"][0], best, rtol=0, atol=1e-13)
    assert res["pi_o"][0] == pi_o
    np.testing.assert_allclose(res["values"][0], corrected, rtol=1e-12, atol=1e-12)
    assert res["action"][0] == int(np.argmax(corrected))


@pytest.mark.parametrize("A", [4, 18])
def test_depth_zero_is_base_agent(oracle_lib, A):
    W = inputs.qnet_weights(A)
    roots = inputs.root_states(range(3))
    res = oracle_lib.search(roots, W, A, 0, 0.99, 1.0)
    q = oracle_lib.qnet(np.stack([oracle_lib.render(r) for r in roots]), W, A)
    np.testing.assert_array_equal(res["values"], q)
    np.testing.assert_array_equal(res["action"], np.argmax(q, axis=1))


def test_correction_moves_only_off_policy_actions(oracle_lib):
    A, d, gamma = 6, 2, 0.99
    W = inputs.qnet_weights(A)
    roots = inputs.root_states(range(4))
    v0 = oracle_lib.search(roots, W, A, d, gamma, 0.0)
    for c in (0.5, 1.0, 3.0):
        vc = oracle_lib.search(roots, W, A, d, gamma, c)
        for i in range(len(roots)):
            p = vc["pi_o"][i]
            shift = v0["values"][i] - vc["values"][i]
            assert shift[p] == 0.0
            others = np.delete(shift, p)
            np.testing.assert_allclose(others, gamma ** d * c * vc["B"][i], rtol=1e-12)
    np.testing.assert_array_equal(v0["values"], v0["v_uncorrected"])


def _bias_only_weights(A, b):
    W = np.zeros(inputs.qnet_numel(A), dtype=np.float32)
    W[-A:] = np.asarray(b, dtype=np.float32)
    return W


def test_closed_form_static_world(oracle_lib):
    """Objects far and static: no reward is reachable, every action is worth
    gamma^d max(b); all tie and the lowest index wins.  delta(a) = gamma max b - b_a."""
    A, d, gamma = 9, 3, 0.9
    b = np.linspace(-0.4, 0.4, A)
    W = _bias_only_weights(A, b)
    root = inputs.make_state((10, 10), FAR)
    res = oracle_lib.search(root.reshape(1), W, A, d, gamma, 0.0)
    bmax = float(np.float32(b).max())
    np.testing.assert_allclose(res["values"][0], gamma ** d * bmax, rtol=1e-15)
    assert res["action"][0] == 0
    np.testing.assert_allclose(res["delta"][0], gamma * bmax - np.float32(b).astype(np.float64), rtol=1e-14)


def test_closed_form_reward_two_cells_right(oracle_lib):
    """A = 9 (speed 1): the reward two cells right is reached at the second step
    by right, up-right or down-right first (2, 5, 7): V = gamma + gamma^2 max b;
    every other first action: gamma^2 max b."""
    A, d, gamma = 9, 2, 0.95
    b = np.array([0.3, -0.2, 0.1, 0.0, 0.05, -0.1, 0.2, 0.25, -0.3])
    W = _bias_only_weights(A, b)
    root = inputs.make_state((10, 10), [(12, 10), (0, 0), (0, 20)])
    res = oracle_lib.search(root.reshape(1), W, A, d, gamma, 0.0)
    bmax = float(np.float32(b).max())
    expect = np.full(A, gamma ** 2 * bmax)
    expect[[2, 5, 7]] += gamma
    np.testing.assert_allclose(res["values"][0], expect, rtol=1e-14)
    assert res["action"][0] == 2


def test_closed_form_hazard_avoidance(oracle_lib):
    """Hazard one cell right, reward two cells left, d = 1, A = 9:
    right is -1 + gamma max b, the rest gamma max b."""
    A, d, gamma = 9, 1, 0.99
    b = np.zeros(A)
    b[4] = 0.5
    W = _bias_only_weights(A, b)
    root = inputs.make_state((10, 10), [(8, 10), (11, 10), (0, 20)])
    res = oracle_lib.search(root.reshape(1), W, A, d, gamma, 0.0)
    expect = np.full(A, gamma * 0.5)
    expect[2] -= 1.0
    np.testing.assert_allclose(res["values"][0], expect, rtol=1e-14)
    np.testing.assert_array_equal(res["r0"][0], np.where(np.arange(A) == 2, -1.0, 0.0))


def test_closed_form_corrected(oracle_lib):
    """Static world, bias-only Q: delta(a) = gamma max b - b_a in closed form, so
    Eq. 3 with Eq. 7 gives the corrected values by hand."""
    A, d, gamma, c = 4, 2, 0.9, 1.0
    b = np.array([0.1, 0.4, -0.2, 0.0], dtype=np.float32).astype(np.float64)
    W = _bias_only_weights(A, b)
    root = inputs.make_state((10, 10), FAR)
    res = oracle_lib.search(root.reshape(1), W, A, d, gamma, c)
    pi_o = 1
    delta = gamma * b.max() - b
    d_o = abs(delta[pi_o])
    d_e = np.mean(np.abs(np.delete(delta, pi_o)))
    B = math.sqrt(math.log(A)) * (d_e * math.sqrt(2) - d_o * 1.0) - (d_e - d_o) / math.sqrt(8)
    expect = np.full(A, gamma ** 2 * b.max()) - gamma ** 2 * c * B
    expect[pi_o] = gamma ** 2 * b.max()
    assert res["pi_o"][0] == pi_o
    np.testing.assert_allclose(res["values"][0], expect, rtol=1e-13)
    assert res["action"][0] == (pi_o if B > 0 else 0)


@pytest.mark.parametrize("A,d", [(4, 3), (6, 2), (3, 1)])
def test_exact_gev_correction(oracle_lib, A, d):
    """Exact-GEV mode: the same uncorrected values, Bellman errors and pi_o, and the
    off-policy actions lowered by gamma^d c (B_e - B_o) with Lemma 2's biases at
    sigma = delta / sqrt(2), computed here from the normal quantile of Python's
    standard library."""
    from statistics import NormalDist
    ppf = NormalDist().inv_cdf
    em = 0.5772156649015329

    def shift(m):
        if m <= 1:
            return 0.0
        x1, xe = -ppf(1 / m), -ppf(1 / (math.e * m))
        return x1 + em * (xe - x1)

    W = inputs.qnet_weights(A, seed=5)
    roots = inputs.root_states(range(40, 43))
    gamma, c = 0.97, 1.5
    eq7 = oracle_lib.search(roots, W, A, d, gamma, c)
    ex = oracle_lib.search(roots, W, A, d, gamma, c, exact_gev=True)
    np.testing.assert_array_equal(ex["v_uncorrected"], eq7["v_uncorrected"])
    np.testing.assert_array_equal(ex["pi_o"], eq7["pi_o"])
    for i in range(len(roots)):
        de, do = ex["delta_e"][i], ex["delta_o"][i]
        gap = (de * shift(A ** d - A ** (d - 1)) - do * shift(A ** (d - 1))) / math.sqrt(2.0)
        assert ex["B"][i] == pytest.approx(gap, rel=1e-9, abs=1e-12)
        for a in range(A):
            want = ex["v_uncorrected"][i, a] - (0.0 if a == ex["pi_o"][i] else gamma ** d * c * gap)
            assert ex["values"][i, a] == pytest.approx(want, rel=1e-12, abs=1e-12)
        assert ex["action"][i] == int(np.argmax(ex["values"][i]))


def test_tree_node_export_brute_force(oracle_lib):
    """The per-node export: R is the replayed accumulated discounted reward, V the
    node's (d - level)-step value, checked by enumerating every remaining action
    sequence with the flat sum of Eq. 1's tail."""
    A, d, gamma = 3, 3, 0.9
    W = inputs.qnet_weights(A, seed=11)
    root = inputs.root_states([77])[0]
    for level in range(1, d + 1):
        for idx in range(A ** level):
            R, V = oracle_lib.tree_node(root, W, A, d, gamma, level, idx)
            s, Rr = oracle_lib.replay(root, A, level, idx, gamma)
            assert R == Rr
            best = -math.inf
            for acts in itertools.product(range(A), repeat=d - level):
                x, ret, g = s, 0.0, 1.0
                for a in acts:
                    x, r = oracle_lib.env_step(x, a)
                    ret += g * r
                    g *= gamma
                q = oracle_lib.qnet(oracle_lib.render(x)[None], W, A)[0]
                best = max(best, ret + g * q.max())
            assert V == pytest.approx(best, rel=1e-12, abs=1e-12)
    # the depth-1 nodes carry the uncorrected root values: R + gamma V
    ref = oracle_lib.search(root, W, A, d, gamma, 0.0)
    for a in range(A):
        R, V = oracle_lib.tree_node(root, W, A, d, gamma, 1, a)
        assert R + gamma * V == pytest.approx(ref["v_uncorrected"][0, a], rel=1e-12)
