"""Pins of the oracle's environment, renderer and tree order.

The environment is the synthetic sprite world that stands in for the paper's
Atari forward model (Alg. 1's simulator G).  Its rules are fixed by the design
notes; these tests check the oracle against hand-derived transitions
(tests/golden/env_transitions.txt), closed-form movement, the render's pixel
invariants and a hand-painted frame, and Alg. 1's child = parent * A + a order.
"""
import itertools
import os

import numpy as np
import pytest

from paper_2107_01715_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "env_transitions.txt")

# Direction names of actions 0..8 (speed 2 for actions 9..17), as the design notes define them.
DIRS = {"noop": (0, 0), "up": (0, -1), "right": (1, 0), "left": (-1, 0), "down": (0, 1),
        "up-right": (1, -1), "up-left": (-1, -1), "down-right": (1, 1), "down-left": (-1, 1)}
ORDER = ["noop", "up", "right", "left", "down", "up-right", "up-left", "down-right", "down-left"]
FAR = [(0, 0), (20, 0), (0, 20)]


def _agent(s):
    return tuple(int(v) for v in s["pos"][3, 0])


@pytest.mark.parametrize("a", range(18))
def test_agent_moves_by_action_table(oracle_lib, a):
    s = inputs.make_state((10, 10), FAR)
    n, r = oracle_lib.env_step(s, a)
    dx, dy = DIRS[ORDER[a % 9]]
    speed = 1 + a // 9
    assert _agent(n) == (10 + speed * dx, 10 + speed * dy)
    assert r == 0


def test_agent_clamped_at_walls(oracle_lib):
    s = inputs.make_state((0, 0), [(20, 20), (20, 19), (19, 20)])
    for a in (3, 1, 6, 12, 10, 15):  # left, up, up-left and their speed-2 forms
        n, _ = oracle_lib.env_step(s, a)
        assert _agent(n) == (0, 0)
    s = inputs.make_state((20, 19), [(0, 0), (0, 1), (1, 0)])
    n, _ = oracle_lib.env_step(s, 16)  # speed-2 down-right from (20, 19)
    assert _agent(n) == (20, 20)


def test_objects_reflect_at_walls(oracle_lib):
    s = inputs.make_state((10, 10), [(20, 0), (0, 20), (5, 5)], vels=[(1, -1), (-1, 1), (1, 0)])
    n, _ = oracle_lib.env_step(s, 0)
    assert tuple(n["pos"][3, 1]) == (19, 1) and tuple(n["vel"][1]) == (-1, 1)
    assert tuple(n["pos"][3, 2]) == (1, 19) and tuple(n["vel"][2]) == (1, -1)
    assert tuple(n["pos"][3, 3]) == (6, 5) and tuple(n["vel"][3]) == (1, 0)


def test_history_shift_and_tick(oracle_lib):
    s = inputs.root_state(3)
    n1, _ = oracle_lib.env_step(s, 4)
    n2, _ = oracle_lib.env_step(n1, 2)
    assert np.array_equal(n2["pos"][0:3], n1["pos"][1:4])
    assert np.array_equal(n1["pos"][0:3], s["pos"][1:4])
    assert int(n2["tick"]) == int(s["tick"]) + 2
    assert int(n2["pad"]) == 0


def _parse_golden():
    cases = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            v = [int(t) for t in line.split()]
            cases.append(v)
    return cases


@pytest.mark.parametrize("case", _parse_golden())
def test_hand_derived_transitions(oracle_lib, case):
    # ax ay  o1x o1y o1vx o1vy  o2x o2y o2vx o2vy  o3x o3y o3vx o3vy  action tick | ax' ay' reward hit-mask
    # | respawn cell (x y) of each hit object, in object order
    (ax, ay, x1, y1, vx1, vy1, x2, y2, vx2, vy2, x3, y3, vx3, vy3, a, tick, eax, eay, er, hits) = case[:20]
    respawn = case[20:]
    hit_objs = [k for k in range(1, 4) if (hits >> k) & 1]
    assert len(respawn) == 2 * len(hit_objs), "one respawn cell per hit object"
    s = inputs.make_state((ax, ay), [(x1, y1), (x2, y2), (x3, y3)],
                          vels=[(vx1, vy1), (vx2, vy2), (vx3, vy3)], tick=tick)
    n, r = oracle_lib.env_step(s, a)
    assert _agent(n) == (eax, eay)
    assert r == er
    assert int(n["tick"]) == tick + 1
    moved = [(x1 + vx1, y1 + vy1), (x2 + vx2, y2 + vy2), (x3 + vx3, y3 + vy3)]
    cells = dict(zip(hit_objs, zip(respawn[0::2], respawn[1::2])))
    for k in range(1, 4):
        p = tuple(int(v) for v in n["pos"][3, k])
        if k in cells:
            assert p == cells[k], (k, p, cells[k])  # the hand-evaluated respawn hash
        else:
            assert p == moved[k - 1]  # an object that was not hit just moved


def test_respawn_is_deterministic_function_of_tick(oracle_lib):
    s = inputs.make_state((10, 10), [(11, 10), (0, 0), (20, 20)], tick=5)
    a1, _ = oracle_lib.env_step(s, 2)
    a2, _ = oracle_lib.env_step(s, 2)
    assert np.array_equal(a1["pos"], a2["pos"])
    seen = set()
    for t in range(40):
        s["tick"] = t
        n, r = oracle_lib.env_step(s, 2)
        assert r == 1
        seen.add(tuple(int(v) for v in n["pos"][3, 1]))
    assert len(seen) > 20  # the respawn position spreads over the grid


# ---- renderer ----------------------------------------------------------------
SPRITES = {  # rows top to bottom, as drawn in the design notes
    0: ["####", "####", "####", "####"],
    1: [".##.", "####", "####", ".##."],
    2: ["#..#", ".##.", ".##.", "#..#"],
    3: ["####", "#..#", "#..#", "####"],
}
PALETTE = {0: 240, 1: 192, 2: 128, 3: 64}


def _paint(state):
    """Hand painter: numpy slices, objects painted in index order."""
    out = np.zeros((4, 84, 84), dtype=np.uint8)
    for h in range(4):
        for k in range(4):
            x, y = (int(v) for v in state["pos"][h, k])
            mask = np.array([[c == "#" for c in row] for row in SPRITES[k]])
            block = out[h, 4 * y:4 * y + 4, 4 * x:4 * x + 4]
            block[mask] = PALETTE[k]
    return out


@pytest.mark.parametrize("seed", range(8))
def test_render_matches_hand_painter(oracle_lib, seed):
    s = inputs.root_state(seed)
    for a in (0, 5, 11):
        s, _ = oracle_lib.env_step(s, a)
    assert np.array_equal(oracle_lib.render(s), _paint(s))


def test_render_pixel_counts_without_overlap(oracle_lib):
    s = inputs.make_state((1, 1), [(5, 5), (9, 9), (13, 13)])
    fr = oracle_lib.render(s)
    assert set(np.unique(fr)) <= {0, 64, 128, 192, 240}
    per_frame = 16 + 12 + 8 + 12
    for h in range(4):
        assert int((fr[h] > 0).sum()) == per_frame
        assert int((fr[h] == 240).sum()) == 16
    # only the 4x4 blocks of occupied cells are painted
    assert fr[0, 4:8, 4:8].min() == 240 and fr[0, 0:4, :].max() == 0


def test_render_overlap_later_object_wins(oracle_lib):
    s = inputs.make_state((7, 7), [(7, 7), (7, 7), (7, 7)])
    fr = oracle_lib.render(s)
    blk = fr[3, 28:32, 28:32]
    # object 3 (ring) on top, object 2 (X) shows in the ring's hole, agent fills the rest
    assert blk[0].tolist() == [64, 64, 64, 64]
    assert blk[1].tolist() == [64, 128, 128, 64]
    assert blk[2].tolist() == [64, 128, 128, 64]


# ---- Alg. 1 tree order ---------------------------------------------------------
@pytest.mark.parametrize("A,depth", [(3, 2), (4, 3), (2, 4)])
def test_level_order_is_base_A_digits(oracle_lib, A, depth):
    """child = parent * A + a: node i of level `depth` has actions = base-A digits
    of i (most significant first); Alg. 1 returns floor(argmax / A^(d-1))."""
    gamma = 0.9
    root = inputs.root_state(5)
    states, R = oracle_lib.level(root, A, depth, gamma)
    for i, acts in enumerate(itertools.product(range(A), repeat=depth)):
        s, ret, g = root, 0.0, 1.0
        for a in acts:
            s, r = oracle_lib.env_step(s, a)
            ret += g * r
            g *= gamma
        assert states[i].tobytes() == s.tobytes()
        assert R[i] == pytest.approx(ret, abs=1e-15)
        assert i // A ** (depth - 1) == acts[0]
