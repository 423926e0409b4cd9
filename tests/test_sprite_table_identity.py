"""The identity the streaming conv1 passes rest on, checked on the CPU.

Every frame the renderer draws is four 4 x 4 sprites on the 4-pixel cell grid,
which is also conv1's stride (8 x 8 kernel, stride 4).  conv1 is linear in its
input, so its pre-activation at patch (ox, oy) is the bias plus, for every
history slot h and every object k whose cell (cx, cy) lies in the patch at
offset (dx, dy) = (cx - ox, cy - oy) in {0, 1}^2, the table entry

    T[h][k][dy][dx][c] = palette_k * sum over sprite k's set pixels (sy, sx) of
                         W[c][h][4 dy + sy][4 dx + sx] / 255,

except where two objects of one slot share a cell (the later one paints over
the earlier one): that cell's term is its rendered pixels times the weights.
Everywhere else the pre-activation is the bias alone.  The test builds the
tables from the weights, with the sprite masks and palette read off the
oracle's own renderer, and compares them with a direct float64 convolution of
the oracle-rendered frame stacks, on stepped states and on states with shared
cells at the grid's edges and corners.
"""
import numpy as np
import pytest

from paper_2107_01715_b300 import inputs


def _sprites(oracle):
    """Masks [4][4][4] and palette [4] of the four objects, from the renderer."""
    s = inputs.root_states([0])
    for h in range(4):
        for k in range(4):
            s["pos"][0, h, k] = (1 + 4 * k, 1)  # distinct cells, inside the grid
    fr = oracle.render(s[0])[0].astype(np.int64)
    masks, pal = np.zeros((4, 4, 4), dtype=bool), np.zeros(4, dtype=np.int64)
    for k in range(4):
        block = fr[4:8, 4 * (1 + 4 * k):4 * (1 + 4 * k) + 4]
        masks[k] = block != 0
        vals = np.unique(block[block != 0])
        assert vals.size == 1
        pal[k] = vals[0]
    return masks, pal


def _direct_conv1(frames, W1, b1):
    """float64 [n][32][20][20] pre-activations of conv1 over uint8 stacks [n][4][84][84]."""
    x = frames.astype(np.float64) / 255.0
    win = np.lib.stride_tricks.sliding_window_view(x, (8, 8), axis=(2, 3))[:, :, ::4, ::4]  # n,4,20,20,8,8
    return np.einsum("nhyxab,chab->ncyx", win, W1.astype(np.float64)) + b1.astype(np.float64)[None, :, None, None]


def _table_conv1(states, frames, W1, b1, masks, pal):
    W = W1.astype(np.float64) / 255.0  # [32][4][8][8]
    T = np.zeros((4, 4, 2, 2, 32))
    for h in range(4):
        for k in range(4):
            for dy in range(2):
                for dx in range(2):
                    sub = W[:, h, 4 * dy:4 * dy + 4, 4 * dx:4 * dx + 4]  # [32][4][4]
                    T[h, k, dy, dx] = pal[k] * sub[:, masks[k]].sum(axis=1)
    n = len(states)
    out = np.broadcast_to(b1.astype(np.float64)[None, :, None, None], (n, 32, 20, 20)).copy()
    for i in range(n):
        pos = states["pos"][i]  # [4 slots][4 objects][x, y]
        for h in range(4):
            cells = [(int(pos[h, k, 0]), int(pos[h, k, 1])) for k in range(4)]
            for oy in range(20):
                for ox in range(20):
                    for k, (cx, cy) in enumerate(cells):
                        dx, dy = cx - ox, cy - oy
                        if not (0 <= dx <= 1 and 0 <= dy <= 1):
                            continue
                        sharers = [j for j in range(4) if cells[j] == (cx, cy)]
                        if len(sharers) == 1:
                            out[i, :, oy, ox] += T[h, k, dy, dx]
                        elif k == sharers[0]:  # a shared cell, taken once: its rendered pixels
                            px = frames[i, h, 4 * cy:4 * cy + 4, 4 * cx:4 * cx + 4].astype(np.float64)
                            sub = W[:, h, 4 * dy:4 * dy + 4, 4 * dx:4 * dx + 4]
                            out[i, :, oy, ox] += np.einsum("ab,cab->c", px, sub)
    return out


def _states(oracle):
    st = list(inputs.root_states(range(40, 52)))
    for i, s in enumerate(list(st)):
        cur = s
        for t in range(3):
            cur, _ = oracle.env_step(cur, (5 * i + 7 * t) % 18)
            st.append(cur)
    shared = [((3, 4), (2, 3)), ((0, 0), (1, 2)), ((20, 20), (1, 3)), ((10, 0), (1, 2, 3)), ((19, 7), (0, 2)),
              ((0, 20), (0, 1, 2, 3)), ((11, 11), (1, 3))]
    base = inputs.root_states(range(300, 300 + len(shared)))
    for i, ((x, y), objs) in enumerate(shared):
        for k in objs:
            base["pos"][i, :, k] = (x, y)
        st.append(base[i])
    out = np.zeros(len(st), dtype=inputs.STATE_DTYPE)
    for i, s in enumerate(st):
        out[i] = s
    assert ((out["pos"] >= 0) & (out["pos"] <= 20)).all()
    return out


def test_conv1_is_bias_plus_sprite_table_terms(oracle_lib):
    W = inputs.split_weights(inputs.qnet_weights(6, seed=1234), 6)
    W1, b1 = W["conv1.w"], W["conv1.b"]
    masks, pal = _sprites(oracle_lib)
    states = _states(oracle_lib)
    frames = np.stack([oracle_lib.render(s) for s in states])
    direct = _direct_conv1(frames, W1, b1)
    table = _table_conv1(states, frames, W1, b1, masks, pal)
    scale = np.abs(direct).max()
    assert np.abs(table - direct).max() <= 1e-12 * scale


def test_rows_away_from_objects_are_the_bias(oracle_lib):
    """A patch whose 2 x 2 cells hold no object of any slot sees only background: its
    pre-activation is the bias exactly (the first of the two passes writes that)."""
    W = inputs.split_weights(inputs.qnet_weights(6, seed=77), 6)
    W1, b1 = W["conv1.w"], W["conv1.b"]
    states = _states(oracle_lib)
    frames = np.stack([oracle_lib.render(s) for s in states])
    direct = _direct_conv1(frames, W1, b1)
    for i in range(len(states)):
        near = np.zeros((20, 20), dtype=bool)
        for h in range(4):
            for k in range(4):
                cx, cy = states["pos"][i, h, k]
                for dy in range(2):
                    for dx in range(2):
                        if 0 <= cy - dy < 20 and 0 <= cx - dx < 20:
                            near[cy - dy, cx - dx] = True
        far = ~near
        assert far.any()
        assert np.array_equal(direct[i][:, far], np.broadcast_to(b1.astype(np.float64)[:, None], (32, far.sum())))


@pytest.mark.parametrize("k", range(4))
def test_sprite_masks_read_off_the_renderer_are_distinct(oracle_lib, k):
    masks, pal = _sprites(oracle_lib)
    assert masks[k].any() and pal[k] > 0
    assert len({m.tobytes() for m in masks}) == 4 and len(set(pal.tolist())) == 4
