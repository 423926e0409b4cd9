"""Write the stored FP64 oracle values the GPU parity tests and the precision
report compare against, for workloads too large to search with the oracle inside
a test run.

    python tests/golden/make_oracle_values.py [atari|precision ...]

Calls only the oracle (oracle/) and the seeded input generators; nothing here
comes from the CUDA path.  Each output file holds, per root, the oracle's root
Q-values Q_0, the uncorrected d-step values V (Eq. 1), the Bellman errors
delta (Prop. 1), pi_o, delta_o, delta_e, the Eq. 7 penalty B, and the corrected
values and action (Eq. 3 / Eq. 4) at the stored correction c; the values at any
other c follow from V, pi_o and B.

  oracle_atari32_a18_d3.json    32 roots (seeds 0..31), A = 18, d = 3, c = 1
  oracle_precision8_a18_d4.json  8 roots (seeds 0..7),  A = 18, d = 4, c = 1
  oracle_precision256_a18_d2.json 256 roots (seeds 50000..50255), A = 18, d = 2, c = 1
Weights: He-normal Nature-DQN from seed 1234; gamma = float32(0.99).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2107_01715_b300 import inputs  # noqa: E402

CASES = {
    "atari": dict(file="oracle_atari32_a18_d3.json", seeds=list(range(32)), A=18, d=3, c=1.0),
    "precision": dict(file="oracle_precision8_a18_d4.json", seeds=list(range(8)), A=18, d=4, c=1.0),
    "precision_d2": dict(file="oracle_precision256_a18_d2.json", seeds=list(range(50000, 50256)), A=18, d=2,
                         c=1.0),
}


def make(name: str) -> str:
    cs = CASES[name]
    A, d, c = cs["A"], cs["d"], cs["c"]
    gamma = float(np.float32(0.99))
    W = inputs.qnet_weights(A, seed=1234)
    out = {"A": A, "d": d, "gamma": gamma, "correction": c, "weights_seed": 1234, "seeds": cs["seeds"],
           "oracle_threads": oracle.threads(), "roots": []}
    t0 = time.time()
    for s in cs["seeds"]:
        r = oracle.search(inputs.root_states([s]), W, A, d, gamma, c)
        out["roots"].append({
            "seed": s, "action": int(r["action"][0]), "values": r["values"][0].tolist(),
            "q0": r["q0"][0].tolist(), "v_uncorrected": r["v_uncorrected"][0].tolist(),
            "delta": r["delta"][0].tolist(), "r0": r["r0"][0].tolist(), "pi_o": int(r["pi_o"][0]),
            "delta_o": float(r["delta_o"][0]), "delta_e": float(r["delta_e"][0]), "B": float(r["B"][0])})
        print(f"{name}: seed {s} done, {time.time() - t0:.0f} s", flush=True)
    out["oracle_seconds"] = time.time() - t0
    path = os.path.join(HERE, cs["file"])
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    return path


if __name__ == "__main__":
    for name in (sys.argv[1:] or list(CASES)):
        print(make(name))
