"""CPU checks of the C ABI: the library loads without a GPU, exports every
symbol include/bcts.h declares, and rejects bad arguments before touching CUDA."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bcts.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"BCTS_API\s+[\w\s\*]*?\b(bcts_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def binding():
    from paper_2107_01715_b300 import build
    build.build()
    from paper_2107_01715_b300 import bcts
    return bcts


def test_header_declares_entry_points():
    syms = declared_symbols()
    for s in ("bcts_create", "bcts_search", "bcts_submit", "bcts_poll", "bcts_destroy", "bcts_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol(binding):
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (bcts_\w+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    for s in declared_symbols():
        assert hasattr(binding.lib, s)
    assert set(binding.EXPORTED) <= exported


def test_library_does_not_need_a_driver_to_load(binding):
    out = subprocess.run(["ldd", binding.LIB_PATH], capture_output=True, text=True).stdout
    assert "libcuda.so" not in out  # driver API is reached through the runtime's entry-point query


def test_qnet_numel(binding):
    from paper_2107_01715_b300 import inputs
    for A in (1, 6, 18):
        assert binding.bcts_qnet_numel(A) == inputs.qnet_numel(A)
    assert binding.bcts_qnet_numel(18) == 1693362


def test_create_rejects_bad_arguments_without_cuda(binding):
    lib = binding.lib
    h = ctypes.c_void_p()
    w = np.zeros(binding.bcts_qnet_numel(6), dtype=np.float32)
    assert lib.bcts_create(None, None, 6, 2, 0.99, 1.0, None, ctypes.byref(h)) == binding.BCTS_EINVAL
    assert lib.bcts_create(None, w.ctypes.data, 0, 2, 0.99, 1.0, None, ctypes.byref(h)) == binding.BCTS_EINVAL
    assert lib.bcts_create(None, w.ctypes.data, 19, 2, 0.99, 1.0, None, ctypes.byref(h)) == binding.BCTS_EINVAL
    assert lib.bcts_create(None, w.ctypes.data, 6, 7, 0.99, 1.0, None, ctypes.byref(h)) == binding.BCTS_EINVAL
    assert lib.bcts_create(None, w.ctypes.data, 6, 2, 1.5, 1.0, None, ctypes.byref(h)) == binding.BCTS_EINVAL
    assert lib.bcts_create(None, w.ctypes.data, 6, 2, 0.0, 1.0, None, ctypes.byref(h)) == binding.BCTS_EINVAL
    assert b"invalid" in lib.bcts_last_error(None)
    assert lib.bcts_expand(None, None, 4, 6, 1.0, None, None, None, None) == binding.BCTS_EINVAL
    assert lib.bcts_render(None, 4, None, None) == binding.BCTS_EINVAL
    assert lib.bcts_search(None, None, 0, None, None) == binding.BCTS_EINVAL
    lib.bcts_destroy(None)  # no-op


def test_binding_refuses_wrong_weight_count(binding):
    with pytest.raises(ValueError):
        binding.bcts_create(np.zeros(10, dtype=np.float32), 6, 2, 0.99, 1.0)


def test_host_env_step_matches_oracle(binding, oracle_lib):
    """The library's host-side step (used to advance served episodes) equals the
    oracle's step bit for bit, rewards included."""
    from paper_2107_01715_b300 import inputs
    states = inputs.root_states(range(300, 340))
    pos = states["pos"]
    for i in range(0, 40, 3):  # put agents next to objects so that contacts happen
        pos[i, 3, 0] = np.clip(pos[i, 3, 1] - np.array([1, 0], dtype=np.int16), 0, 20)
    states["pos"] = pos
    hits = 0
    for s in states:
        for a in range(18):
            ours, r1 = binding.bcts_env_step(s, a)
            ref, r2 = oracle_lib.env_step(s, a)
            assert ours.tobytes() == ref.tobytes() and r1 == r2
            hits += r1 != 0
    assert hits > 0
    with pytest.raises(binding.BctsError):
        binding.bcts_env_step(states[0], 18)


def test_host_env_step_matches_hand_derived_transitions(binding):
    """bcts_env_step (the library's host copy of the simulator) against the hand-derived
    transitions, respawn cells included."""
    from tests._util import golden_expected_cells, golden_state, golden_transitions
    for row in golden_transitions():
        s, a = golden_state(row)
        n, r = binding.bcts_env_step(s, a)
        agent, er, cells = golden_expected_cells(row)
        assert tuple(int(v) for v in n["pos"][3, 0]) == agent
        assert r == er
        for k, cell in cells.items():
            assert tuple(int(v) for v in n["pos"][3, k]) == cell, (row, k)
