"""Pin the oracle's DNN forward-model workload (Sec. 4's randomly initialised
network standing in for a learned forward model).

* The forward model and the Q head against torch.nn.functional.linear / relu /
  tanh in float64 (library pin), with the one-hot action as explicit input.
* The search against brute-force enumeration of every action sequence with the
  flat sum of Eq. 1, plus Prop. 1's Bellman errors and Eq. 3/7 evaluated here.
* A closed form: with only biases, every step returns the same state and reward.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2107_01715_b300 import inputs

torch = pytest.importorskip("torch")
F = torch.nn.functional


def torch_step(s, a, W, A):
    p = {k: torch.from_numpy(v.astype(np.float64)) for k, v in inputs.dnn_split(W, A).items()}
    x = torch.cat([torch.from_numpy(np.asarray(s, dtype=np.float64)), F.one_hot(torch.tensor(a), A).double()])
    h = F.relu(F.linear(x, p["fm1.w"], p["fm1.b"]))
    h = F.relu(F.linear(h, p["fm2.w"], p["fm2.b"]))
    h = F.relu(F.linear(h, p["fm3.w"], p["fm3.b"]))
    o = F.linear(h, p["fmo.w"], p["fmo.b"])
    return torch.tanh(o[:100]).numpy(), float(o[100])


def torch_q(s, W, A):
    p = inputs.dnn_split(W, A)
    return F.linear(torch.from_numpy(np.asarray(s, dtype=np.float64)), torch.from_numpy(p["q.w"].astype(np.float64)),
                    torch.from_numpy(p["q.b"].astype(np.float64))).numpy()


@pytest.mark.parametrize("A", [2, 10])
def test_dnn_step_and_q_match_torch(oracle_lib, A):
    W = inputs.dnn_weights(A, seed=3)
    for s in inputs.dnn_root_states(range(4)):
        for a in range(A):
            nxt, r = oracle_lib.dnn_step(s, a, W, A)
            tn, tr = torch_step(s, a, W, A)
            np.testing.assert_allclose(nxt, tn, rtol=0, atol=1e-13)
            assert r == pytest.approx(tr, abs=1e-13)
        np.testing.assert_allclose(oracle_lib.dnn_q(s, W, A), torch_q(s, W, A), rtol=0, atol=1e-13)


def brute(oracle_lib, s0, W, A, d, gamma, c):
    q0 = oracle_lib.dnn_q(s0, W, A)
    pi_o = int(np.argmax(q0))
    best = np.full(A, -np.inf)
    for acts in itertools.product(range(A), repeat=d):
        s, ret, g = np.asarray(s0, dtype=np.float64), 0.0, 1.0
        for a in acts:
            s, r = oracle_lib.dnn_step(s, a, W, A)
            ret += g * r
            g *= gamma
        best[acts[0]] = max(best[acts[0]], ret + g * oracle_lib.dnn_q(s, W, A).max())
    delta = np.zeros(A)
    for a in range(A):
        s1, r = oracle_lib.dnn_step(s0, a, W, A)
        delta[a] = r + gamma * oracle_lib.dnn_q(s1, W, A).max() - q0[a]
    do = abs(delta[pi_o])
    de = np.mean(np.abs(np.delete(delta, pi_o))) if A > 1 else 0.0
    B = math.sqrt(math.log(A)) * (de * math.sqrt(d) - do * math.sqrt(d - 1)) - (de - do) / math.sqrt(8)
    vals = best - np.where(np.arange(A) == pi_o, 0.0, gamma ** d * c * B)
    return vals, best


@pytest.mark.parametrize("A,d,c", [(2, 3, 1.0), (3, 2, 0.0), (2, 1, 2.0), (4, 2, 1.0)])
def test_dnn_search_equals_brute_force(oracle_lib, A, d, c):
    W = inputs.dnn_weights(A, seed=8)
    roots = inputs.dnn_root_states(range(10, 13))
    res = oracle_lib.dnn_search(roots, W, A, d, 0.95, c)
    for i, s0 in enumerate(roots):
        vals, unc = brute(oracle_lib, s0, W, A, d, 0.95, c)
        np.testing.assert_allclose(res["v_uncorrected"][i], unc, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(res["values"][i], vals, rtol=1e-12, atol=1e-12)
        assert res["action"][i] == int(np.argmax(vals))


def test_dnn_closed_form_bias_only(oracle_lib):
    A, d, gamma = 3, 3, 0.9
    W = np.zeros(inputs.dnn_numel(A), dtype=np.float32)
    p = inputs.dnn_split(W, A)
    p["fmo.b"][:] = np.linspace(-0.5, 0.5, 101, dtype=np.float32)
    p["fmo.b"][100] = np.float32(0.25)  # reward of every step
    p["q.b"][:] = np.array([0.1, -0.3, 0.4], dtype=np.float32)
    s0 = inputs.dnn_root_states([1])[0]
    nxt, r = oracle_lib.dnn_step(s0, 2, W, A)
    np.testing.assert_allclose(nxt, np.tanh(p["fmo.b"][:100].astype(np.float64)), rtol=0, atol=1e-15)
    assert r == pytest.approx(0.25, abs=1e-15)
    res = oracle_lib.dnn_search(s0[None], W, A, d, gamma, 0.0)
    expect = 0.25 * (1 + gamma + gamma ** 2) + gamma ** 3 * float(np.float32(0.4))
    np.testing.assert_allclose(res["v_uncorrected"][0], expect, rtol=0, atol=1e-12)
    assert res["action"][0] == 0  # all actions tie: lowest index
