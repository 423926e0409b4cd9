"""The ORACLE: a plain FP64 CPU reference of the BCTS / Batch-BFS search.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's CPU
baseline leg may import this package; the CUDA library never does, and the two
share no code (the oracle's C source restates the environment, the renderer,
the Q-network, Eq. 1, Eq. 3, Eq. 7 and Alg. 1's tree order on its own).

This module is the ctypes binding of `bcts_oracle.c` (built by `build()` into
`liboracle.so` beside it) plus thin numpy marshalling.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bcts_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

STATE_BYTES = 80
FRAME_BYTES = 4 * 84 * 84


def build(force: bool = False) -> str:
    """Compile bcts_oracle.c with gcc (-O2, OpenMP).  Returns the .so path."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-Wall", "-Wextra",
             "-o", _LIB_PATH, _SRC, "-lm"])
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        lib.or_env_step.argtypes = [P, ctypes.c_int, P]
        lib.or_env_step.restype = ctypes.c_int
        lib.or_render.argtypes = [P, P]
        lib.or_qnet.argtypes = [P, P, ctypes.c_int, P]
        lib.or_qnet_batch.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P]
        lib.or_qnet_numel.argtypes = [ctypes.c_int]
        lib.or_qnet_numel.restype = ctypes.c_size_t
        lib.or_bellman_penalty.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int]
        lib.or_bellman_penalty.restype = ctypes.c_double
        lib.or_search.argtypes = [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_double, P, P, P]
        lib.or_search.restype = ctypes.c_int
        lib.or_search_ex.argtypes = [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int, P, P, P]
        lib.or_search_ex.restype = ctypes.c_int
        lib.or_bellman_penalty_exact.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int]
        lib.or_bellman_penalty_exact.restype = ctypes.c_double
        lib.or_normal_upper_quantile.argtypes = [ctypes.c_double]
        lib.or_normal_upper_quantile.restype = ctypes.c_double
        lib.or_tree_node.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_longlong, P, P]
        lib.or_search_pruned.argtypes = [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_int, P, P, P]
        lib.or_search_pruned.restype = ctypes.c_int
        lib.or_dnn_numel.argtypes = [ctypes.c_int]
        lib.or_dnn_numel.restype = ctypes.c_size_t
        lib.or_dnn_step.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P]
        lib.or_dnn_step.restype = ctypes.c_double
        lib.or_dnn_q.argtypes = [P, P, ctypes.c_int, P]
        lib.or_dnn_search.argtypes = [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, P, P, P]
        lib.or_dnn_search.restype = ctypes.c_int
        lib.or_replay.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_longlong, ctypes.c_double, P, P]
        lib.or_backup.argtypes = [P, P, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_int, P, P]
        lib.or_backup.restype = ctypes.c_int
        lib.or_level.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong,
                                 ctypes.c_double, P, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _state_array(s) -> np.ndarray:
    a = np.ascontiguousarray(s)
    assert a.dtype.itemsize == STATE_BYTES
    return a


def env_step(state, a: int):
    """One environment tick: returns (next_state, reward)."""
    lib = _load()
    s = _state_array(state).reshape(1)
    out = np.zeros_like(s)
    r = lib.or_env_step(_ptr(s), int(a), _ptr(out))
    return out[0], int(r)


def render(state) -> np.ndarray:
    """The 4 x 84 x 84 uint8 frame stack of a state."""
    lib = _load()
    s = _state_array(state).reshape(1)
    fr = np.zeros((4, 84, 84), dtype=np.uint8)
    lib.or_render(_ptr(s), _ptr(fr))
    return fr


def qnet(frames: np.ndarray, weights: np.ndarray, A: int) -> np.ndarray:
    """FP64 Q-values for a batch of frame stacks [n][4][84][84] -> [n][A]."""
    lib = _load()
    fr = np.ascontiguousarray(frames, dtype=np.uint8).reshape(-1, FRAME_BYTES)
    w = np.ascontiguousarray(weights, dtype=np.float32)
    assert w.size == lib.or_qnet_numel(A)
    q = np.zeros((fr.shape[0], A), dtype=np.float64)
    lib.or_qnet_batch(_ptr(fr), fr.shape[0], _ptr(w), A, _ptr(q))
    return q


def bellman_penalty(delta_e: float, delta_o: float, A: int, d: int) -> float:
    """Eq. 7."""
    return float(_load().or_bellman_penalty(delta_e, delta_o, A, d))


def bellman_penalty_exact(delta_e: float, delta_o: float, A: int, d: int) -> float:
    """Lemma 2's exact bias gap B_e - B_o at sigma = delta / sqrt(2)."""
    return float(_load().or_bellman_penalty_exact(delta_e, delta_o, A, d))


def normal_upper_quantile(q: float) -> float:
    """x with 1 - Phi(x) = q (so Phi^-1(1 - q))."""
    return float(_load().or_normal_upper_quantile(q))


def search(roots, weights: np.ndarray, A: int, d: int, gamma: float, correction: float, exact_gev: bool = False):
    """Full BCTS search (Eq. 7's penalty, or Lemma 2's exact bias gap when
    exact_gev).  Returns dict(action [n], values [n][A], q0, v_uncorrected,
    delta, r0 [n][A], pi_o, delta_o, delta_e, B [n])."""
    lib = _load()
    r = _state_array(roots).reshape(-1)
    n = r.shape[0]
    w = np.ascontiguousarray(weights, dtype=np.float32)
    assert w.size == lib.or_qnet_numel(A)
    act = np.zeros(n, dtype=np.int32)
    val = np.zeros((n, A), dtype=np.float64)
    diag = np.zeros((n, 4 * A + 4), dtype=np.float64)
    rc = lib.or_search_ex(_ptr(r), n, _ptr(w), A, d, float(gamma), float(correction), int(bool(exact_gev)),
                          _ptr(act), _ptr(val), _ptr(diag))
    if rc != 0:
        raise ValueError("oracle search rejected its arguments")
    return {
        "action": act, "values": val,
        "q0": diag[:, 0:A], "v_uncorrected": diag[:, A:2 * A], "delta": diag[:, 2 * A:3 * A],
        "r0": diag[:, 3 * A:4 * A], "pi_o": diag[:, 4 * A].astype(np.int64),
        "delta_o": diag[:, 4 * A + 1], "delta_e": diag[:, 4 * A + 2], "B": diag[:, 4 * A + 3],
    }


def search_pruned(roots, weights: np.ndarray, A: int, d: int, gamma: float, correction: float, keep: int,
                  exact_gev: bool = False):
    """Pruned Batch-BFS: per root action, levels 2..d-1 keep the `keep` nodes with the
    highest R + gamma^i max Q.  Same dict as search() plus "gap" [n]: the smallest
    margin between a kept and a dropped score (inf when nothing was dropped)."""
    lib = _load()
    r = _state_array(roots).reshape(-1)
    n = r.shape[0]
    w = np.ascontiguousarray(weights, dtype=np.float32)
    act = np.zeros(n, dtype=np.int32)
    val = np.zeros((n, A), dtype=np.float64)
    diag = np.zeros((n, 4 * A + 5), dtype=np.float64)
    rc = lib.or_search_pruned(_ptr(r), n, _ptr(w), A, d, float(gamma), float(correction), int(bool(exact_gev)),
                              int(keep), _ptr(act), _ptr(val), _ptr(diag))
    if rc != 0:
        raise ValueError("oracle pruned search rejected its arguments")
    return {
        "action": act, "values": val, "q0": diag[:, 0:A], "v_uncorrected": diag[:, A:2 * A],
        "delta": diag[:, 2 * A:3 * A], "pi_o": diag[:, 4 * A].astype(np.int64), "B": diag[:, 4 * A + 3],
        "gap": diag[:, 4 * A + 4],
    }


def backup(leaf_R, leaf_maxq, q0, r1, maxq1, n: int, A: int, d: int, gamma: float, correction: float,
           exact_gev: bool = False):
    """Alg. 1's backup + the BCTS correction on given leaf data (FP64).  leaf_R and
    leaf_maxq hold n * A^d leaves in Alg. 1's order; q0, r1, maxq1 are [n][A].
    Returns (actions [n], values [n][A])."""
    lib = _load()
    f = [np.ascontiguousarray(x, dtype=np.float64).reshape(-1) for x in (leaf_R, leaf_maxq, q0, r1, maxq1)]
    act = np.zeros(n, dtype=np.int32)
    val = np.zeros((n, A), dtype=np.float64)
    rc = lib.or_backup(*[_ptr(x) for x in f], int(n), int(A), int(d), float(gamma), float(correction),
                       int(bool(exact_gev)), _ptr(act), _ptr(val))
    if rc != 0:
        raise ValueError("oracle backup rejected its arguments")
    return act, val


def tree_node(root, weights: np.ndarray, A: int, d: int, gamma: float, level: int, idx: int):
    """(R, V) of node idx at depth `level`: accumulated discounted reward from the
    root and the node's (d - level)-step value."""
    lib = _load()
    r = _state_array(root).reshape(1)
    w = np.ascontiguousarray(weights, dtype=np.float32)
    R = np.zeros(1, dtype=np.float64)
    V = np.zeros(1, dtype=np.float64)
    lib.or_tree_node(_ptr(r), _ptr(w), A, d, float(gamma), int(level), int(idx), _ptr(R), _ptr(V))
    return float(R[0]), float(V[0])


def replay(root, A: int, depth: int, idx: int, gamma: float):
    """State and accumulated discounted reward of node `idx` of level `depth`."""
    lib = _load()
    r = _state_array(root).reshape(1)
    out = np.zeros_like(r)
    R = np.zeros(1, dtype=np.float64)
    lib.or_replay(_ptr(r), A, depth, int(idx), float(gamma), _ptr(out), _ptr(R))
    return out[0], float(R[0])


def level(root, A: int, depth: int, gamma: float, first: int = 0, count: int | None = None):
    """States and rewards of nodes [first, first+count) of level `depth` (Alg. 1 order)."""
    lib = _load()
    r = _state_array(root).reshape(1)
    if count is None:
        count = A ** depth - first
    out = np.zeros(count, dtype=r.dtype)
    R = np.zeros(count, dtype=np.float64)
    lib.or_level(_ptr(r), A, depth, int(first), int(count), float(gamma), _ptr(out), _ptr(R))
    return out, R


def threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS or all cores)."""
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v else (os.cpu_count() or 1)


# ---- DNN forward-model workload ---------------------------------------------------
DNN_D = 100


def dnn_step(state: np.ndarray, a: int, weights: np.ndarray, A: int):
    """One forward-model step in FP64: (next_state [100] float64, reward)."""
    lib = _load()
    s = np.ascontiguousarray(state, dtype=np.float64).reshape(DNN_D)
    w = np.ascontiguousarray(weights, dtype=np.float32)
    assert w.size == lib.or_dnn_numel(A)
    out = np.zeros(DNN_D, dtype=np.float64)
    r = lib.or_dnn_step(_ptr(s), int(a), _ptr(w), A, _ptr(out))
    return out, float(r)


def dnn_q(state: np.ndarray, weights: np.ndarray, A: int) -> np.ndarray:
    lib = _load()
    s = np.ascontiguousarray(state, dtype=np.float64).reshape(DNN_D)
    w = np.ascontiguousarray(weights, dtype=np.float32)
    q = np.zeros(A, dtype=np.float64)
    lib.or_dnn_q(_ptr(s), _ptr(w), A, _ptr(q))
    return q


def dnn_search(roots: np.ndarray, weights: np.ndarray, A: int, d: int, gamma: float, correction: float,
               exact_gev: bool = False):
    """BCTS search over the DNN model; same result dict as search()."""
    lib = _load()
    r = np.ascontiguousarray(roots, dtype=np.float32).reshape(-1, DNN_D)
    n = r.shape[0]
    w = np.ascontiguousarray(weights, dtype=np.float32)
    assert w.size == lib.or_dnn_numel(A)
    act = np.zeros(n, dtype=np.int32)
    val = np.zeros((n, A), dtype=np.float64)
    diag = np.zeros((n, 4 * A + 4), dtype=np.float64)
    rc = lib.or_dnn_search(_ptr(r), n, _ptr(w), A, d, float(gamma), float(correction), int(bool(exact_gev)),
                           _ptr(act), _ptr(val), _ptr(diag))
    if rc != 0:
        raise ValueError("oracle DNN search rejected its arguments")
    return {
        "action": act, "values": val,
        "q0": diag[:, 0:A], "v_uncorrected": diag[:, A:2 * A], "delta": diag[:, 2 * A:3 * A],
        "r0": diag[:, 3 * A:4 * A], "pi_o": diag[:, 4 * A].astype(np.int64),
        "delta_o": diag[:, 4 * A + 1], "delta_e": diag[:, 4 * A + 2], "B": diag[:, 4 * A + 3],
    }
