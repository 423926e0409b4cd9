"""Python binding of libbcts.so (the C ABI declared in include/bcts.h).

Argument marshalling only: every step of the search runs in the library's CUDA
kernels.  Device-pointer entry points take anything with a `data_ptr()` method
(a torch CUDA tensor) or a plain integer address.  There is no CPU fallback: if
the library has not been built, importing this module raises ImportError.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .inputs import STATE_DTYPE

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbcts.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -m paper_2107_01715_b300.build` "
        "(the CUDA library is the only implementation; there is no CPU fallback)")
lib = ctypes.CDLL(LIB_PATH)

BCTS_OK, BCTS_PENDING = 0, 1
BCTS_EINVAL, BCTS_ENOMEM, BCTS_ECUDA, BCTS_ETIMEOUT = -1, -2, -3, -4
BCTS_EBUSY, BCTS_ENOTICKET, BCTS_EDEVICE, BCTS_ENOKERNEL = -5, -6, -7, -8
BCTS_PREC_FP32, BCTS_PREC_BF16, BCTS_PREC_FP8, BCTS_PREC_FP32_SIMT = 0, 1, 2, 3
PRECISIONS = {"fp32": BCTS_PREC_FP32, "bf16": BCTS_PREC_BF16, "fp8": BCTS_PREC_FP8,
              "fp32_simt": BCTS_PREC_FP32_SIMT}

EXPORTED = ["bcts_qnet_numel", "bcts_create", "bcts_destroy", "bcts_last_error", "bcts_search",
            "bcts_search_device", "bcts_search_mixed", "bcts_submit", "bcts_poll", "bcts_expand",
            "bcts_render", "bcts_qnet", "bcts_profile", "bcts_qnet_static", "bcts_env_step", "bcts_selftest_wait", "bcts_tree_nodes",
            "bcts_search_tree", "bcts_dnn_numel", "bcts_dnn_create", "bcts_dnn_destroy", "bcts_dnn_search",
            "bcts_dnn_search_device", "bcts_dnn_profile", "bcts_dnn_last_error", "bcts_search_pruned",
            "bcts_search_pruned_device", "bcts_backup"]
BCTS_STATIC_MAX_NODES = 128
BCTS_FLAG_FRAMES = 1
BCTS_FLAG_EXACT_GEV = 2
KERNEL_CLASSES = ["expand", "render", "conv1", "conv2", "conv3", "fc1", "fc2", "backup", "conv1_partial",
                  "conv1_leaf", "dnn_mlp", "dnn_q"]


class bcts_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("frame_budget_bytes", ctypes.c_size_t),
                ("max_roots", ctypes.c_int), ("flags", ctypes.c_int), ("leaf_chunk", ctypes.c_int)]


class bcts_env_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
lib.bcts_qnet_numel.argtypes = [_I]
lib.bcts_qnet_numel.restype = ctypes.c_size_t
lib.bcts_create.argtypes = [_P, _P, _I, _I, ctypes.c_float, ctypes.c_float, _P, ctypes.POINTER(_P)]
lib.bcts_create.restype = _I
lib.bcts_destroy.argtypes = [_P]
lib.bcts_destroy.restype = None
lib.bcts_last_error.argtypes = [_P]
lib.bcts_last_error.restype = ctypes.c_char_p
lib.bcts_search.argtypes = [_P, _P, _I, _P, _P]
lib.bcts_search_device.argtypes = [_P, _P, _I, _P, _P, _P]
lib.bcts_search_mixed.argtypes = [_P, _P, _P, _P, _I, _P, _P]
lib.bcts_submit.argtypes = [_P, _P, _I, _I, ctypes.POINTER(ctypes.c_uint64)]
lib.bcts_poll.argtypes = [_P, ctypes.c_uint64, _P, _P, _I]
lib.bcts_expand.argtypes = [_P, _P, _I64, _I, ctypes.c_float, _P, _P, _P, _P]
lib.bcts_render.argtypes = [_P, _I64, _P, _P]
lib.bcts_qnet.argtypes = [_P, _P, _I64, _P, _P]
lib.bcts_profile.argtypes = [_P, _I, _P, _P, _P]
lib.bcts_qnet_static.argtypes = [_P, _I, _P, _I64, _P, _P]
lib.bcts_env_step.argtypes = [_P, _I, _P, ctypes.POINTER(_I)]
lib.bcts_selftest_wait.argtypes = [_I]
lib.bcts_backup.argtypes = [_P, _P, _P, _P, _P, _I, _I, _I, ctypes.c_float, ctypes.c_float, _I, _P, _P, _P]
lib.bcts_backup.restype = _I
lib.bcts_tree_nodes.argtypes = [_I, _I, _I]
lib.bcts_tree_nodes.restype = ctypes.c_int64
lib.bcts_search_tree.argtypes = [_P, _P, _I, _P, _P, _P, _P, _P]
lib.bcts_search_pruned.argtypes = [_P, _P, _I, _I, _P, _P]
lib.bcts_search_pruned.restype = _I
lib.bcts_search_pruned_device.argtypes = [_P, _P, _I, _I, _P, _P, _P]
lib.bcts_search_pruned_device.restype = _I
lib.bcts_dnn_numel.argtypes = [_I]
lib.bcts_dnn_numel.restype = ctypes.c_size_t
lib.bcts_dnn_create.argtypes = [_P, _I, _I, ctypes.c_float, ctypes.c_float, _I, ctypes.POINTER(_P)]
lib.bcts_dnn_create.restype = _I
lib.bcts_dnn_destroy.argtypes = [_P]
lib.bcts_dnn_destroy.restype = None
lib.bcts_dnn_search.argtypes = [_P, _P, _I, _P, _P]
lib.bcts_dnn_search.restype = _I
lib.bcts_dnn_search_device.argtypes = [_P, _P, _I, _P, _P, _P]
lib.bcts_dnn_search_device.restype = _I
lib.bcts_dnn_profile.argtypes = [_P, _I, _P, _P, _P]
lib.bcts_dnn_profile.restype = _I
lib.bcts_dnn_last_error.argtypes = [_P]
lib.bcts_dnn_last_error.restype = ctypes.c_char_p
for _f in ("bcts_search", "bcts_search_device", "bcts_search_mixed", "bcts_submit", "bcts_poll",
           "bcts_expand", "bcts_render", "bcts_qnet", "bcts_profile", "bcts_qnet_static", "bcts_env_step", "bcts_selftest_wait", "bcts_search_tree"):
    getattr(lib, _f).restype = _I


class BctsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"bcts error {code}: {msg}")
        self.code = code


def _addr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take a device address of {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream  # torch.cuda.Stream


def _check(rc: int, ctx=None):
    if rc < 0:
        msg = lib.bcts_last_error(ctx.handle if ctx is not None else None)
        raise BctsError(rc, (msg or b"").decode())
    return rc


class Context:
    """Owns one `bcts_ctx`; destroyed by close() or garbage collection."""

    def __init__(self, handle, A, d, gamma, correction, precision):
        self.handle = handle
        self.A, self.d, self.gamma, self.correction, self.precision = A, d, gamma, correction, precision

    def close(self):
        if self.handle:
            lib.bcts_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def bcts_qnet_numel(A: int) -> int:
    return int(lib.bcts_qnet_numel(A))


def bcts_create(qnet_weights: np.ndarray, A: int, d: int, gamma: float, correction: float,
                precision="fp32", leaf_chunk: int = 0, frame_budget_bytes: int = 0, max_roots: int = 0,
                env_kind: int = 0, flags: int = 0) -> Context:
    w = np.ascontiguousarray(qnet_weights, dtype=np.float32)
    if w.size != bcts_qnet_numel(A):
        raise ValueError(f"expected {bcts_qnet_numel(A)} weights for A={A}, got {w.size}")
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    opt = bcts_options(prec, frame_budget_bytes, max_roots, flags, leaf_chunk)
    env = bcts_env_desc(env_kind)
    h = _P()
    rc = lib.bcts_create(ctypes.byref(env), w.ctypes.data, A, d, gamma, correction, ctypes.byref(opt),
                         ctypes.byref(h))
    _check(rc)
    return Context(h, A, d, gamma, correction, prec)


def bcts_destroy(ctx: Context) -> None:
    ctx.close()


def bcts_last_error(ctx: Context | None = None) -> str:
    return (lib.bcts_last_error(ctx.handle if ctx else None) or b"").decode()


def _roots(roots) -> np.ndarray:
    r = np.ascontiguousarray(roots)
    if r.dtype != STATE_DTYPE:
        raise TypeError("roots must be an array of STATE_DTYPE")
    return r.reshape(-1)


def bcts_search(ctx: Context, roots):
    """Host search: returns (actions int32 [n], root values float32 [n][A])."""
    r = _roots(roots)
    n = r.shape[0]
    act = np.zeros(n, dtype=np.int32)
    val = np.zeros((n, ctx.A), dtype=np.float32)
    _check(lib.bcts_search(ctx.handle, r.ctypes.data, n, act.ctypes.data, val.ctypes.data), ctx)
    return act, val


def bcts_search_device(ctx: Context, d_roots, n: int, d_action, d_values, stream=None) -> int:
    return _check(lib.bcts_search_device(ctx.handle, _addr(d_roots), n, _addr(d_action), _addr(d_values),
                                         _stream(stream)), ctx)


def bcts_search_mixed(ctx: Context, roots, depths, actions):
    r = _roots(roots)
    n = r.shape[0]
    ds = np.ascontiguousarray(depths, dtype=np.int32)
    As = np.ascontiguousarray(actions, dtype=np.int32)
    act = np.zeros(n, dtype=np.int32)
    val = np.zeros((n, ctx.A), dtype=np.float32)
    _check(lib.bcts_search_mixed(ctx.handle, r.ctypes.data, ds.ctypes.data, As.ctypes.data, n,
                                 act.ctypes.data, val.ctypes.data), ctx)
    return act, val


def bcts_submit(ctx: Context, root, d: int, A: int) -> int:
    r = _roots(root)
    t = ctypes.c_uint64()
    _check(lib.bcts_submit(ctx.handle, r.ctypes.data, d, A, ctypes.byref(t)), ctx)
    return t.value


def bcts_poll(ctx: Context, ticket: int, A: int, timeout_us: int = 0):
    """Returns (status, action, values): status BCTS_OK or BCTS_PENDING."""
    act = np.zeros(1, dtype=np.int32)
    val = np.zeros(A, dtype=np.float32)
    rc = _check(lib.bcts_poll(ctx.handle, ticket, act.ctypes.data, val.ctypes.data, timeout_us), ctx)
    return rc, int(act[0]), val


def bcts_expand(d_parents, d_parent_R, n_parents: int, A: int, gamma_pow: float, d_children, d_child_R=None,
                d_child_reward=None, stream=None) -> int:
    return _check(lib.bcts_expand(_addr(d_parents), _addr(d_parent_R), n_parents, A, gamma_pow,
                                  _addr(d_children), _addr(d_child_R), _addr(d_child_reward), _stream(stream)))


def bcts_backup(d_leaf_R, d_leaf_maxq, d_q0, d_r1, d_maxq1, n: int, A: int, d: int, gamma: float,
                correction: float, d_action, d_values, flags: int = 0, stream=None) -> int:
    """Alg. 1's backup + the BCTS correction on device leaf data (no context)."""
    return _check(lib.bcts_backup(_addr(d_leaf_R), _addr(d_leaf_maxq), _addr(d_q0), _addr(d_r1), _addr(d_maxq1),
                                  int(n), int(A), int(d), float(gamma), float(correction), int(flags),
                                  _addr(d_action), _addr(d_values), _stream(stream)))


def bcts_render(d_states, n: int, d_frames, stream=None) -> int:
    return _check(lib.bcts_render(_addr(d_states), n, _addr(d_frames), _stream(stream)))


def bcts_qnet(ctx: Context, d_frames, n: int, d_q, stream=None) -> int:
    return _check(lib.bcts_qnet(ctx.handle, _addr(d_frames), n, _addr(d_q), _stream(stream)), ctx)


def bcts_profile(ctx: Context, enable: bool):
    """Read and reset per-kernel-class device time; enable/disable recording.
    Returns (ms dict, launches dict, total launches)."""
    k = len(KERNEL_CLASSES)
    ms = np.zeros(k, dtype=np.float64)
    cnt = np.zeros(k, dtype=np.int64)
    tot = np.zeros(1, dtype=np.int64)
    _check(lib.bcts_profile(ctx.handle, 1 if enable else 0, ms.ctypes.data, cnt.ctypes.data, tot.ctypes.data), ctx)
    return dict(zip(KERNEL_CLASSES, ms.tolist())), dict(zip(KERNEL_CLASSES, cnt.tolist())), int(tot[0])


def bcts_qnet_static(d_qnet_weights, A: int, d_frames, n: int, d_q, stream=None) -> int:
    """Allocation-free Q-network on n <= BCTS_STATIC_MAX_NODES stacks (device pointers)."""
    return _check(lib.bcts_qnet_static(_addr(d_qnet_weights), A, _addr(d_frames), n, _addr(d_q), _stream(stream)))


def bcts_env_step(state, a: int):
    """Host environment tick: returns (next_state, reward)."""
    s = _roots(state)[:1]
    out = np.zeros(1, dtype=STATE_DTYPE)
    r = _I()
    _check(lib.bcts_env_step(s.ctypes.data, int(a), out.ctypes.data, ctypes.byref(r)))
    return out[0], int(r.value)


def bcts_selftest_wait(timeout_us: int) -> int:
    """Run the bounded-wait self-test; returns the raw status (BCTS_ETIMEOUT expected)."""
    return int(lib.bcts_selftest_wait(int(timeout_us)))


def bcts_tree_nodes(n: int, A: int, d: int) -> int:
    """Floats per array of the per-node export: n * (A + A^2 + ... + A^d)."""
    return int(lib.bcts_tree_nodes(int(n), int(A), int(d)))


def bcts_search_tree(ctx: Context, d_roots, n: int, d_action, d_values, d_node_R, d_node_V, stream=None) -> int:
    """Search plus the per-node export (accumulated reward R and propagated value V
    of every node at depths 1..d, level-major, Alg. 1 order); device pointers."""
    return _check(lib.bcts_search_tree(ctx.handle, _addr(d_roots), n, _addr(d_action), _addr(d_values),
                                       _addr(d_node_R), _addr(d_node_V), _stream(stream)), ctx)


# ---- DNN forward-model workload ---------------------------------------------------
DNN_STATE = 100


class DnnContext:
    """Owns one `bcts_dnn_ctx` (Batch-BFS over the DNN forward model)."""

    def __init__(self, handle, A, d):
        self.handle, self.A, self.d = handle, A, d

    def close(self):
        if self.handle:
            lib.bcts_dnn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _dnn_check(rc: int, ctx=None):
    if rc < 0:
        msg = lib.bcts_dnn_last_error(ctx.handle if ctx is not None else None)
        raise BctsError(rc, (msg or b"").decode())
    return rc


def bcts_dnn_numel(A: int) -> int:
    return int(lib.bcts_dnn_numel(A))


def bcts_dnn_create(weights: np.ndarray, A: int, d: int, gamma: float, correction: float,
                    flags: int = 0) -> DnnContext:
    w = np.ascontiguousarray(weights, dtype=np.float32)
    if w.size != bcts_dnn_numel(A):
        raise ValueError(f"expected {bcts_dnn_numel(A)} weights for A={A}, got {w.size}")
    h = _P()
    _dnn_check(lib.bcts_dnn_create(w.ctypes.data, A, d, gamma, correction, flags, ctypes.byref(h)))
    return DnnContext(h, A, d)


def bcts_dnn_search(ctx: DnnContext, roots: np.ndarray):
    """Host roots float32 [n][100] -> (actions [n] int32, values [n][A] float32)."""
    r = np.ascontiguousarray(roots, dtype=np.float32).reshape(-1, DNN_STATE)
    n = r.shape[0]
    act = np.zeros(n, dtype=np.int32)
    val = np.zeros((n, ctx.A), dtype=np.float32)
    _dnn_check(lib.bcts_dnn_search(ctx.handle, r.ctypes.data, n, act.ctypes.data, val.ctypes.data), ctx)
    return act, val


def bcts_dnn_search_device(ctx: DnnContext, d_roots, n: int, d_action, d_values, stream=None) -> int:
    return _dnn_check(lib.bcts_dnn_search_device(ctx.handle, _addr(d_roots), n, _addr(d_action), _addr(d_values),
                                                 _stream(stream)), ctx)


def bcts_dnn_profile(ctx: DnnContext, enable: bool):
    """As bcts_profile, for a DNN context: (ms dict, launches dict, total launches)."""
    k = len(KERNEL_CLASSES)
    ms = np.zeros(k, dtype=np.float64)
    cnt = np.zeros(k, dtype=np.int64)
    tot = np.zeros(1, dtype=np.int64)
    _dnn_check(lib.bcts_dnn_profile(ctx.handle, int(bool(enable)), ms.ctypes.data, cnt.ctypes.data, tot.ctypes.data),
               ctx)
    return ({c: float(ms[i]) for i, c in enumerate(KERNEL_CLASSES)},
            {c: int(cnt[i]) for i, c in enumerate(KERNEL_CLASSES)}, int(tot[0]))


def bcts_search_pruned(ctx: Context, roots, keep: int):
    """Pruned search (per root action, levels 2..d-1 keep the `keep` nodes with the
    highest R + gamma^i max Q): (actions [n], values [n][A]); host arrays."""
    r = _roots(roots)
    n = r.shape[0]
    act = np.zeros(n, dtype=np.int32)
    val = np.zeros((n, ctx.A), dtype=np.float32)
    _check(lib.bcts_search_pruned(ctx.handle, r.ctypes.data, n, int(keep), act.ctypes.data, val.ctypes.data), ctx)
    return act, val


def bcts_search_pruned_device(ctx: Context, d_roots, n: int, keep: int, d_action, d_values, stream=None) -> int:
    return _check(lib.bcts_search_pruned_device(ctx.handle, _addr(d_roots), n, int(keep), _addr(d_action),
                                                _addr(d_values), _stream(stream)), ctx)
