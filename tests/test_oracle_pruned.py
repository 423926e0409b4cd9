"""Pin the oracle's pruned Batch-BFS (Sec. 4: an index array of unpruned states,
updated at each pruning step, traces the best root action).

* Nothing pruned (keep >= every level's candidate count): the full search.
* Pruning only removes leaves: V(a_0) never exceeds the full search's.
* The selection rule restated here in Python with explicit index arrays (on the
  oracle's environment, renderer and Q-network, themselves pinned elsewhere)
  gives the same root values.
"""
import numpy as np
import pytest

from paper_2107_01715_b300 import inputs


@pytest.mark.parametrize("A,d,keep", [(4, 3, 4), (3, 4, 9), (6, 2, 1), (2, 5, 8)])
def test_no_pruning_is_full_search(oracle_lib, A, d, keep):
    W = inputs.qnet_weights(A, seed=2)
    roots = inputs.root_states(range(3))
    full = oracle_lib.search(roots, W, A, d, 0.95, 1.0)
    pr = oracle_lib.search_pruned(roots, W, A, d, 0.95, 1.0, keep)
    np.testing.assert_allclose(pr["values"], full["values"], rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(pr["action"], full["action"])
    assert np.isinf(pr["gap"]).all()


@pytest.mark.parametrize("keep", [1, 2, 3])
def test_pruning_only_lowers_values(oracle_lib, keep):
    A, d = 3, 4
    W = inputs.qnet_weights(A, seed=2)
    roots = inputs.root_states(range(4))
    full = oracle_lib.search(roots, W, A, d, 0.95, 1.0)
    pr = oracle_lib.search_pruned(roots, W, A, d, 0.95, 1.0, keep)
    assert (pr["v_uncorrected"] <= full["v_uncorrected"] + 1e-12).all()
    np.testing.assert_allclose(pr["B"], full["B"], rtol=0, atol=0)  # the penalty is the full tree's


def restated(oracle_lib, root, W, A, d, gamma, keep):
    def maxq(s):
        return oracle_lib.qnet(oracle_lib.render(s)[None], W, A)[0].max()
    V = np.zeros(A)
    for a0 in range(A):
        s1, r = oracle_lib.env_step(root, a0)
        states, R = [s1], [float(r)]
        for i in range(2, d + 1):
            cand, candR = [], []
            for p, (s, rp) in enumerate(zip(states, R)):
                for a in range(A):
                    c, rc = oracle_lib.env_step(s, a)
                    cand.append(c)
                    candR.append(rp + gamma ** (i - 1) * rc)
            scores = [candR[j] + gamma ** i * maxq(cand[j]) for j in range(len(cand))]
            if i == d:
                V[a0] = max(scores)
                break
            order = sorted(range(len(cand)), key=lambda j: (-scores[j], j))
            idx = sorted(order[:keep])  # the index array of unpruned states
            states, R = [cand[j] for j in idx], [candR[j] for j in idx]
        if d == 1:
            V[a0] = R[0] + gamma * maxq(s1)
    return V


@pytest.mark.parametrize("A,d,keep", [(3, 4, 2), (2, 5, 3), (3, 3, 1)])
def test_pruned_values_match_restatement(oracle_lib, A, d, keep):
    W = inputs.qnet_weights(A, seed=6)
    roots = inputs.root_states(range(20, 22))
    pr = oracle_lib.search_pruned(roots, W, A, d, 0.9, 0.0, keep)
    for i, root in enumerate(roots):
        np.testing.assert_allclose(pr["v_uncorrected"][i], restated(oracle_lib, root, W, A, d, 0.9, keep),
                                   rtol=1e-12, atol=1e-12)
