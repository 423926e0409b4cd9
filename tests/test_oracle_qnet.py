"""Pin the oracle's FP64 Nature-DQN against torch.nn.functional in float64.

The paper scores leaves with a pre-trained value network (Alg. 1, last step;
Sec. 5.1 uses Rainbow); the seeded Nature-DQN stands in for it.  The library
routines conv2d / linear are an independent implementation of the same
definition, so a transposed kernel, a wrong stride, a dropped bias or a wrong
flatten order in the oracle's direct loops fails here.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from paper_2107_01715_b300 import inputs


def torch_qnet(frames: np.ndarray, flat: np.ndarray, A: int) -> np.ndarray:
    p = {k: torch.from_numpy(v.astype(np.float64)) for k, v in inputs.split_weights(flat, A).items()}
    x = torch.from_numpy(frames.astype(np.float64)) / 255.0
    x = F.relu(F.conv2d(x, p["conv1.w"], p["conv1.b"], stride=4))
    x = F.relu(F.conv2d(x, p["conv2.w"], p["conv2.b"], stride=2))
    x = F.relu(F.conv2d(x, p["conv3.w"], p["conv3.b"], stride=1))
    x = x.reshape(x.shape[0], -1)
    x = F.relu(F.linear(x, p["fc1.w"], p["fc1.b"]))
    return F.linear(x, p["fc2.w"], p["fc2.b"]).numpy()


@pytest.mark.parametrize("A", [6, 18])
def test_qnet_matches_torch_on_rendered_frames(oracle_lib, A):
    W = inputs.qnet_weights(A, seed=1234)
    frames = np.stack([oracle_lib.render(inputs.root_state(s)) for s in range(4)])
    q = oracle_lib.qnet(frames, W, A)
    ref = torch_qnet(frames, W, A)
    np.testing.assert_allclose(q, ref, rtol=1e-12, atol=1e-13)


def test_qnet_matches_torch_on_dense_random_frames(oracle_lib):
    """Dense pixels exercise every weight (rendered frames are mostly zero)."""
    A = 9
    rng = np.random.default_rng(3)
    W = inputs.qnet_weights(A, seed=99, bias=-0.02)
    frames = rng.integers(0, 256, size=(3, 4, 84, 84), dtype=np.uint8)
    q = oracle_lib.qnet(frames, W, A)
    ref = torch_qnet(frames, W, A)
    np.testing.assert_allclose(q, ref, rtol=1e-12, atol=1e-12)


def test_zero_weights_give_fc2_bias(oracle_lib):
    A = 5
    W = np.zeros(inputs.qnet_numel(A), dtype=np.float32)
    W[-A:] = np.array([0.5, -1.0, 2.0, 0.0, 1.25], dtype=np.float32)
    frames = np.stack([oracle_lib.render(inputs.root_state(s)) for s in range(2)])
    q = oracle_lib.qnet(frames, W, A)
    assert np.array_equal(q, np.tile(W[-A:].astype(np.float64), (2, 1)))
