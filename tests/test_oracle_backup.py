"""Pins of the oracle's stand-alone backup (Alg. 1's leaf max + the BCTS
correction on given leaf data): on real trees it must reproduce the recursive
depth-first search (Eq. 1 factorised level by level) from the leaves' flat
accumulated rewards, and its correction must move only the off-policy actions."""
import numpy as np
import pytest

from paper_2107_01715_b300 import inputs


def _tree_data(oracle_lib, roots, W, A, d, gamma):
    """Leaf R / max Q (Alg. 1 order), root Q, r(s_0, a) and depth-1 max Q from the
    oracle's own environment, renderer and Q-network."""
    leaf_R, leaf_q, q0, r1, m1 = [], [], [], [], []
    for root in roots:
        q0.append(oracle_lib.qnet(oracle_lib.render(root)[None], W, A)[0])
        s1, R1 = oracle_lib.level(root, A, 1, gamma)
        r1.append(R1)
        m1.append(oracle_lib.qnet(np.stack([oracle_lib.render(s) for s in s1]), W, A).max(axis=1))
        sd, Rd = oracle_lib.level(root, A, d, gamma)
        leaf_R.append(Rd)
        leaf_q.append(oracle_lib.qnet(np.stack([oracle_lib.render(s) for s in sd]), W, A).max(axis=1))
    return (np.concatenate(leaf_R), np.concatenate(leaf_q), np.stack(q0), np.stack(r1), np.stack(m1))


@pytest.mark.parametrize("A,d,c,exact", [(3, 1, 1.0, False), (4, 2, 1.0, False), (3, 3, 2.0, False),
                                         (4, 2, 1.0, True), (2, 3, 0.0, False)])
def test_backup_equals_recursive_search(oracle_lib, A, d, c, exact):
    gamma = 0.99
    W = inputs.qnet_weights(A, seed=1234)
    roots = inputs.root_states(range(60, 63))
    data = _tree_data(oracle_lib, roots, W, A, d, gamma)
    act, val = oracle_lib.backup(*data, len(roots), A, d, gamma, c, exact_gev=exact)
    ref = oracle_lib.search(roots, W, A, d, gamma, c, exact_gev=exact)
    np.testing.assert_allclose(val, ref["values"], rtol=0, atol=1e-12)
    assert np.array_equal(act, ref["action"])


def test_backup_depth0_and_correction_offsets(oracle_lib):
    """d = 0 returns Q_0 and its argmax; with c != 0 only a != pi_o move, each by the
    same gamma^d c B (Eq. 3)."""
    rng = np.random.default_rng(3)
    n, A, d, gamma = 4, 5, 2, 0.9
    leaf_R = rng.normal(size=n * A ** d)
    leaf_q = rng.normal(size=n * A ** d)
    q0, r1, m1 = rng.normal(size=(n, A)), rng.normal(size=(n, A)), rng.normal(size=(n, A))
    a0, v0 = oracle_lib.backup(leaf_R, leaf_q, q0, r1, m1, n, A, 0, gamma, 1.0)
    np.testing.assert_array_equal(v0, q0)
    assert np.array_equal(a0, q0.argmax(axis=1))
    _, vu = oracle_lib.backup(leaf_R, leaf_q, q0, r1, m1, n, A, d, gamma, 0.0)
    _, vc = oracle_lib.backup(leaf_R, leaf_q, q0, r1, m1, n, A, d, gamma, 2.0)
    for i in range(n):
        pi_o = int(np.argmax(q0[i]))
        diff = vu[i] - vc[i]
        assert diff[pi_o] == 0.0
        off = np.delete(diff, pi_o)
        np.testing.assert_allclose(off, off[0], rtol=0, atol=1e-12)
