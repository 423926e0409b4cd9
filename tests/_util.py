"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np

# Root values: |gpu - oracle| <= TOL * max(|oracle|, 1) per precision.
# FP32-class paths hold 1e-4; BF16 / FP8 leaf Q-networks carry their operand
# rounding (8 / 4 significant bits) through four layers.
TOL = {"fp32_simt": 1e-4, "fp32": 1e-4, "bf16": 2e-2, "fp8": 8e-2}


def value_close(gpu, ref, tol):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(gpu - ref) <= tol * np.maximum(np.abs(ref), 1.0)


def check_actions(gpu_actions, ref_values, tol):
    """Where the oracle's top-2 margin exceeds the tolerance the action is unique
    and must match; elsewhere the GPU's action must be within tolerance of the
    oracle's best value.  Returns the number of roots with a unique action."""
    ref_values = np.asarray(ref_values, dtype=np.float64)
    unique = 0
    for i, a in enumerate(np.asarray(gpu_actions)):
        v = ref_values[i]
        order = np.argsort(-v, kind="stable")
        best = v[order[0]]
        margin = best - v[order[1]] if v.size > 1 else np.inf
        thr = 2 * tol * max(abs(best), 1.0)
        if margin > thr:
            unique += 1
            assert a == order[0], (i, a, order[0], margin)
        else:
            assert best - v[a] <= thr, (i, a, best, v[a])
    return unique


def as_state_bytes(tensor_u8, n):
    from paper_2107_01715_b300.inputs import STATE_DTYPE
    return tensor_u8.cpu().numpy().view(STATE_DTYPE).reshape(n)


def pi_o_decided(q0_row, tol):
    """pi_o (argmax of the root Q-values, Sec. 3.3) is a discrete decision: where the
    oracle's top-2 root Q margin is within the precision's tolerance, a reduced-
    precision run may pick the other action and the Eq. 7 penalty then lands on
    different actions.  Values are compared only where pi_o is decided."""
    q = np.sort(np.asarray(q0_row, dtype=np.float64))
    if q.size < 2:
        return True
    return q[-1] - q[-2] > 2 * tol * max(abs(q[-1]), 1.0)


def golden_transitions():
    """Rows of tests/golden/env_transitions.txt as integer lists (hand-derived
    transitions: 16 inputs, 4 outputs, then the respawn cell of each hit object)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "env_transitions.txt")
    rows = []
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append([int(t) for t in line.split()])
    return rows


def golden_state(row):
    """The state and action of a golden transition row."""
    from paper_2107_01715_b300 import inputs
    (ax, ay, x1, y1, vx1, vy1, x2, y2, vx2, vy2, x3, y3, vx3, vy3, a, tick) = row[:16]
    s = inputs.make_state((ax, ay), [(x1, y1), (x2, y2), (x3, y3)],
                          vels=[(vx1, vy1), (vx2, vy2), (vx3, vy3)], tick=tick)
    return s, a


def golden_expected_cells(row):
    """{object k: (x, y)} after the step: the respawn cell of each hit object, the
    moved cell of the others (objects 1-3; every golden row keeps them off walls)."""
    (ax, ay, x1, y1, vx1, vy1, x2, y2, vx2, vy2, x3, y3, vx3, vy3, a, tick, eax, eay, er, hits) = row[:20]
    resp = row[20:]
    hit = [k for k in range(1, 4) if (hits >> k) & 1]
    cells = {k: (x + vx, y + vy) for k, (x, y, vx, vy) in
             zip(range(1, 4), ((x1, y1, vx1, vy1), (x2, y2, vx2, vy2), (x3, y3, vx3, vy3)))}
    for k, x, y in zip(hit, resp[0::2], resp[1::2]):
        cells[k] = (x, y)
    return (eax, eay), er, cells
