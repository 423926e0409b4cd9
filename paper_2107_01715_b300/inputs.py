"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds no arithmetic of the method (no environment step, no renderer,
no Q-network, no backup).  It only draws numbers:

* root states of the synthetic sprite environment from a splitmix64 stream
  (published definition: Steele, Lea and Flood, "Fast splittable pseudorandom
  number generators", OOPSLA 2014), one stream per seed;
* Nature-DQN Q-network weights, He-normal initialised (std = sqrt(2 / fan_in)),
  biases 0.01, from numpy's PCG64 generator, flattened in PyTorch parameter order.

The paper evaluates pre-trained Rainbow agents on Atari (Sec. 5.1); neither the
games nor the weights are available, so these seeded inputs stand in for them.
"""
from __future__ import annotations

import numpy as np

# --- state layout (80 bytes, little endian), identical to `bcts_state` -------
#   int16 pos[4 history][4 objects][2]   (x, y), history slot 3 is the newest
#   int8  vel[4 objects][2]              object 0 (the agent) has velocity 0
#   uint32 tick
#   uint32 pad                           always 0
STATE_DTYPE = np.dtype(
    [("pos", "<i2", (4, 4, 2)), ("vel", "i1", (4, 2)), ("tick", "<u4"), ("pad", "<u4")]
)
assert STATE_DTYPE.itemsize == 80

GRID = 21          # cells per side
HIST = 4           # frames in a stack
NOBJ = 4           # objects: 0 agent, 1 reward, 2-3 hazards
FRAME = 84         # pixels per side
FRAME_BYTES = HIST * FRAME * FRAME   # 28,224

_MASK64 = (1 << 64) - 1


def splitmix64(seed: int):
    """Yield the splitmix64 sequence for `seed` (64-bit unsigned integers)."""
    x = seed & _MASK64
    while True:
        x = (x + 0x9E3779B97F4A7C15) & _MASK64
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        yield z ^ (z >> 31)


def root_state(seed: int) -> np.ndarray:
    """One root state: positions uniform on the 21x21 grid, velocities of objects
    1..3 in {-1, 0, 1} per axis, the same snapshot in all four history slots,
    tick in [0, 65535]."""
    g = splitmix64(seed)
    s = np.zeros((), dtype=STATE_DTYPE)
    snap = np.zeros((NOBJ, 2), dtype=np.int16)
    for k in range(NOBJ):
        snap[k, 0] = next(g) % GRID
        snap[k, 1] = next(g) % GRID
    vel = np.zeros((NOBJ, 2), dtype=np.int8)
    for k in range(1, NOBJ):
        vel[k, 0] = int(next(g) % 3) - 1
        vel[k, 1] = int(next(g) % 3) - 1
    s["pos"] = np.broadcast_to(snap, (HIST, NOBJ, 2))
    s["vel"] = vel
    s["tick"] = next(g) & 0xFFFF
    s["pad"] = 0
    return s


def root_states(seeds) -> np.ndarray:
    """Root states for a sequence of seeds, as a contiguous STATE_DTYPE array."""
    seeds = list(seeds)
    out = np.zeros(len(seeds), dtype=STATE_DTYPE)
    for i, sd in enumerate(seeds):
        out[i] = root_state(sd)
    return out


def make_state(agent, objects, vels=((0, 0), (0, 0), (0, 0)), tick=0) -> np.ndarray:
    """A hand-built state: `agent` = (x, y), `objects` = three (x, y) for objects
    1..3, `vels` their velocities; all history slots equal."""
    s = np.zeros((), dtype=STATE_DTYPE)
    snap = np.array([agent] + list(objects), dtype=np.int16)
    s["pos"] = np.broadcast_to(snap, (HIST, NOBJ, 2))
    v = np.zeros((NOBJ, 2), dtype=np.int8)
    v[1:] = np.array(vels, dtype=np.int8)
    s["vel"] = v
    s["tick"] = tick
    return s


# --- Nature-DQN parameters ----------------------------------------------------
def qnet_shapes(A: int):
    """(name, shape) in PyTorch parameter order: conv weight [Cout][Cin][kh][kw]
    then bias; linear weight [out][in] then bias; fc1's input is the conv3 map
    flattened as (C, H, W)."""
    return [
        ("conv1.w", (32, 4, 8, 8)), ("conv1.b", (32,)),
        ("conv2.w", (64, 32, 4, 4)), ("conv2.b", (64,)),
        ("conv3.w", (64, 64, 3, 3)), ("conv3.b", (64,)),
        ("fc1.w", (512, 3136)), ("fc1.b", (512,)),
        ("fc2.w", (A, 512)), ("fc2.b", (A,)),
    ]


def qnet_numel(A: int) -> int:
    return sum(int(np.prod(s)) for _, s in qnet_shapes(A))


def qnet_weights(A: int, seed: int = 1234, bias: float = 0.01) -> np.ndarray:
    """Flat float32 He-normal Nature-DQN weights for |A| = A actions."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in qnet_shapes(A):
        if name.endswith(".w"):
            fan_in = int(np.prod(shape[1:]))
            parts.append(rng.normal(0.0, np.sqrt(2.0 / fan_in), size=shape).astype(np.float32).ravel())
        else:
            parts.append(np.full(shape, bias, dtype=np.float32))
    return np.concatenate(parts)


def split_weights(flat: np.ndarray, A: int) -> dict:
    """View a flat weight vector as named arrays (no copy)."""
    out, off = {}, 0
    for name, shape in qnet_shapes(A):
        n = int(np.prod(shape))
        out[name] = flat[off:off + n].reshape(shape)
        off += n
    assert off == flat.size
    return out


def mixed_roots(n: int, seed: int = 7, depths=(1, 2, 3, 4), actions=(4, 9, 18)):
    """Batched-form workload: n roots, each with a depth and an action count drawn
    uniformly from `depths` and `actions` (splitmix64 stream of `seed`)."""
    g = splitmix64(seed)
    ds = np.array([depths[next(g) % len(depths)] for _ in range(n)], dtype=np.int32)
    As = np.array([actions[next(g) % len(actions)] for _ in range(n)], dtype=np.int32)
    return root_states(range(1000 + seed * 100000, 1000 + seed * 100000 + n)), ds, As


# ---- DNN forward-model workload (a learned forward model stand-in) -------------
DNN_D = 100  # state width
DNN_H = 100  # hidden width


def dnn_shapes(A: int):
    """Flat parameter order of the DNN forward model and its Q head, PyTorch [out][in]:
    three hidden layers of width 100 on [state (100); one-hot action (A)], an output
    layer giving the next state's 100 pre-activations and the reward, and a linear
    Q head on the state."""
    D, H = DNN_D, DNN_H
    return [("fm1.w", (H, D + A)), ("fm1.b", (H,)), ("fm2.w", (H, H)), ("fm2.b", (H,)),
            ("fm3.w", (H, H)), ("fm3.b", (H,)), ("fmo.w", (D + 1, H)), ("fmo.b", (D + 1,)),
            ("q.w", (A, D)), ("q.b", (A,))]


def dnn_numel(A: int) -> int:
    return int(sum(np.prod(s) for _, s in dnn_shapes(A)))


def dnn_weights(A: int, seed: int = 4321) -> np.ndarray:
    """Random initialisation: He-normal (std sqrt(2 / fan_in)) for the ReLU layers,
    std sqrt(1 / fan_in) for the output layer and the Q head, biases 0.01."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in dnn_shapes(A):
        if name.endswith(".w"):
            gain = 2.0 if name in ("fm1.w", "fm2.w", "fm3.w") else 1.0
            parts.append(rng.normal(0.0, np.sqrt(gain / shape[1]), size=shape).astype(np.float32).ravel())
        else:
            parts.append(np.full(shape, 0.01, dtype=np.float32))
    return np.concatenate(parts)


def dnn_split(flat: np.ndarray, A: int) -> dict:
    out, off = {}, 0
    for name, shape in dnn_shapes(A):
        n = int(np.prod(shape))
        out[name] = flat[off:off + n].reshape(shape)
        off += n
    assert off == flat.size
    return out


def dnn_root_states(seeds) -> np.ndarray:
    """float32 [n][100], uniform in [-1, 1), one splitmix64 stream per seed."""
    seeds = list(seeds)
    out = np.zeros((len(seeds), DNN_D), dtype=np.float32)
    for i, s in enumerate(seeds):
        g = splitmix64(0xD1B54A32D192ED03 ^ int(s))
        for j in range(DNN_D):
            out[i, j] = np.float32((next(g) >> 11) / float(1 << 53) * 2.0 - 1.0)
    return out
