"""GPU parity of Alg. 1's expansion and of the renderer: bit-exact states,
rewards and frames against the oracle (through the C ABI)."""
import numpy as np
import pytest

from paper_2107_01715_b300 import inputs
from tests._util import as_state_bytes, golden_expected_cells, golden_state, golden_transitions

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_01715_b300 import bcts
    return torch, bcts


def _to_dev(torch, arr):
    return torch.from_numpy(np.ascontiguousarray(arr).view(np.uint8).copy()).cuda()


def _expand_levels(torch, bcts, roots, A, depth, gamma):
    """Run `depth` expansions on the GPU; returns states/R of every level."""
    cur = _to_dev(torch, roots)
    curR = torch.zeros(len(roots), dtype=torch.float32, device="cuda")
    n = len(roots)
    out = [(cur, curR)]
    for i in range(depth):
        nxt = torch.empty(n * A * 80, dtype=torch.uint8, device="cuda")
        nxtR = torch.empty(n * A, dtype=torch.float32, device="cuda")
        rew = torch.empty(n * A, dtype=torch.int8, device="cuda")
        bcts.bcts_expand(cur, curR, n, A, float(np.float32(gamma ** i)), nxt, nxtR, rew)
        n *= A
        cur, curR = nxt, nxtR
        out.append((cur, curR))
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("A,depth,nroots", [(6, 2, 1), (18, 2, 3), (4, 4, 2), (1, 3, 5), (9, 3, 1)])
def test_expand_bit_exact(oracle_lib, dev, A, depth, nroots):
    torch, bcts = dev
    gamma = 0.99
    roots = inputs.root_states(range(10, 10 + nroots))
    levels = _expand_levels(torch, bcts, roots, A, depth, gamma)
    for lev in range(1, depth + 1):
        st = as_state_bytes(levels[lev][0], nroots * A ** lev)
        R = levels[lev][1].cpu().numpy()
        for r in range(nroots):
            ref_s, ref_R = oracle_lib.level(roots[r], A, lev, gamma)
            blk = slice(r * A ** lev, (r + 1) * A ** lev)
            assert st[blk].tobytes() == ref_s.tobytes(), (lev, r)
            np.testing.assert_allclose(R[blk], ref_R, rtol=0, atol=1e-6)


def test_expand_rewards_match_oracle_steps(oracle_lib, dev):
    torch, bcts = dev
    A = 18
    parents = inputs.root_states(range(200, 264))
    # move a few agents next to objects so that contacts happen
    pos = parents["pos"]
    for i in range(0, 64, 4):
        pos[i, 3, 0] = np.clip(pos[i, 3, 1] - np.array([1, 0], dtype=np.int16), 0, 20)
    parents["pos"] = pos
    dp = _to_dev(torch, parents)
    ch = torch.empty(64 * A * 80, dtype=torch.uint8, device="cuda")
    rew = torch.empty(64 * A, dtype=torch.int8, device="cuda")
    bcts.bcts_expand(dp, None, 64, A, 1.0, ch, None, rew)
    torch.cuda.synchronize()
    st = as_state_bytes(ch, 64 * A)
    rw = rew.cpu().numpy()
    nonzero = 0
    for p in range(64):
        for a in range(A):
            s, r = oracle_lib.env_step(parents[p], a)
            assert st[p * A + a].tobytes() == s.tobytes()
            assert rw[p * A + a] == r
            nonzero += r != 0
    assert nonzero > 0


@pytest.mark.parametrize("n", [1, 7, 300])
def test_render_bit_exact(oracle_lib, dev, n):
    torch, bcts = dev
    states = inputs.root_states(range(n))
    for i in range(n):  # vary the history slots
        for a in (i % 18, (3 * i) % 18):
            states[i], _ = oracle_lib.env_step(states[i], a)
    ds = _to_dev(torch, states)
    fr = torch.empty(n * 28224, dtype=torch.uint8, device="cuda")
    bcts.bcts_render(ds, n, fr)
    torch.cuda.synchronize()
    got = fr.cpu().numpy().reshape(n, 4, 84, 84)
    for i in range(n):
        assert np.array_equal(got[i], oracle_lib.render(states[i])), i


def test_render_large_batch_sampled(oracle_lib, dev):
    """A frontier as large as a d=3, A=18 leaf chunk; sampled stacks bit-exact."""
    torch, bcts = dev
    A = 18
    roots = inputs.root_states([1])
    levels = _expand_levels(torch, bcts, roots, A, 3, 0.99)
    leaves, _ = levels[3]
    n = A ** 3
    fr = torch.empty(n * 28224, dtype=torch.uint8, device="cuda")
    bcts.bcts_render(leaves, n, fr)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    for idx in list(rng.choice(n, 40, replace=False)) + [0, n - 1]:
        s, _ = oracle_lib.replay(roots[0], A, 3, int(idx), 0.99)
        got = fr[idx * 28224:(idx + 1) * 28224].cpu().numpy().reshape(4, 84, 84)
        assert np.array_equal(got, oracle_lib.render(s)), idx


def test_expand_matches_hand_derived_transitions(dev):
    """bcts_expand on the hand-derived transitions (tests/golden/env_transitions.txt):
    the child of each golden state under its action carries the listed agent cell,
    reward and respawn cells."""
    torch, bcts = dev
    A = 18
    rows = golden_transitions()
    parents = np.stack([golden_state(r)[0] for r in rows])
    ch = torch.empty(len(rows) * A * 80, dtype=torch.uint8, device="cuda")
    rew = torch.empty(len(rows) * A, dtype=torch.int8, device="cuda")
    bcts.bcts_expand(_to_dev(torch, parents), None, len(rows), A, 1.0, ch, None, rew)
    torch.cuda.synchronize()
    st = as_state_bytes(ch, len(rows) * A)
    rw = rew.cpu().numpy()
    for i, row in enumerate(rows):
        _, a = golden_state(row)
        agent, er, cells = golden_expected_cells(row)
        c = st[i * A + a]
        assert tuple(int(v) for v in c["pos"][3, 0]) == agent
        assert int(rw[i * A + a]) == er
        for k, cell in cells.items():
            assert tuple(int(v) for v in c["pos"][3, k]) == cell, (i, k)
