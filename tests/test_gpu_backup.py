"""GPU parity of the stand-alone backup (bcts_backup: Alg. 1's leaf max and the
BCTS correction, Eq. 1 / Prop. 1 / Eq. 7 / Eq. 3 / Eq. 4) against the oracle's
backup on the same seeded leaf data, from tiny trees to the bandwidth-bound size
the bench times (split segments with atomic maxima)."""
import numpy as np
import pytest

from tests._util import value_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_01715_b300 import bcts
    return torch, bcts


def _data(n, A, d, seed):
    """Seeded FP32 leaf data with the structure of a search: R a sum of discounted
    rewards in {-1, 0, 1}, max-Q values of a few tenths, ties between siblings."""
    rng = np.random.default_rng(seed)
    L = n * A ** d
    R = (rng.integers(-1, 2, size=L) * 0.99 + rng.integers(-1, 2, size=L) * 0.9801).astype(np.float32)
    mq = rng.normal(0.3, 0.1, size=L).astype(np.float32)
    mq[1::7] = mq[0::7][:mq[1::7].size]  # exact ties
    q0 = rng.normal(0.3, 0.1, size=(n, A)).astype(np.float32)
    r1 = rng.integers(-1, 2, size=(n, A)).astype(np.float32)
    m1 = rng.normal(0.3, 0.1, size=(n, A)).astype(np.float32)
    return R, mq, q0, r1, m1


@pytest.mark.parametrize("n,A,d,c,exact", [(3, 6, 0, 1.0, False), (5, 6, 1, 1.0, False), (7, 18, 2, 1.0, False),
                                           (4, 18, 3, 2.0, False), (2, 18, 4, 1.0, False), (3, 9, 4, 1.0, True),
                                           (1, 32, 2, 1.0, False), (2, 2, 14, 1.0, False), (1, 3, 10, 0.5, True)])
def test_backup_matches_oracle(oracle_lib, dev, n, A, d, c, exact):
    torch, bcts = dev
    gamma = float(np.float32(0.99))
    R, mq, q0, r1, m1 = _data(n, A, d, seed=n * 100 + A * 10 + d)
    if d == 1:
        R, mq = r1.reshape(-1).copy(), m1.reshape(-1).copy()
    t = [torch.from_numpy(x.reshape(-1)).cuda() for x in (R, mq, q0, r1, m1)]
    act = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    val = torch.full((n * A,), float("nan"), dtype=torch.float32, device="cuda")
    bcts.bcts_backup(*t, n, A, d, gamma, c, act, val, flags=bcts.BCTS_FLAG_EXACT_GEV if exact else 0)
    torch.cuda.synchronize()
    ra, rv = oracle_lib.backup(R, mq, q0, r1, m1, n, A, d, gamma, c, exact_gev=exact)
    v = val.cpu().numpy().reshape(n, A)
    assert value_close(v, rv, 1e-5).all(), np.abs(v - rv).max()
    a = act.cpu().numpy()
    for i in range(n):
        srt = np.sort(rv[i])
        if srt.size < 2 or srt[-1] - srt[-2] > 1e-5 * max(abs(srt[-1]), 1.0):
            assert a[i] == ra[i]
        else:
            assert rv[i].max() - rv[i][a[i]] <= 2e-5 * max(abs(rv[i].max()), 1.0)


def test_backup_bandwidth_size(oracle_lib, dev):
    """The bench's stand-alone backup size: 1,024 roots, A = 18, d = 4 (107.5 M
    leaves, 860 MB of leaf data; every root action's 5,832-leaf segment is split
    across blocks), every output against the oracle."""
    torch, bcts = dev
    n, A, d, gamma, c = 1024, 18, 4, float(np.float32(0.99)), 1.0
    R, mq, q0, r1, m1 = _data(n, A, d, seed=11)
    t = [torch.from_numpy(x.reshape(-1)).cuda() for x in (R, mq, q0, r1, m1)]
    act = torch.empty(n, dtype=torch.int32, device="cuda")
    val = torch.empty(n * A, dtype=torch.float32, device="cuda")
    bcts.bcts_backup(*t, n, A, d, gamma, c, act, val)
    torch.cuda.synchronize()
    ra, rv = oracle_lib.backup(R, mq, q0, r1, m1, n, A, d, gamma, c)
    v = val.cpu().numpy().reshape(n, A)
    assert value_close(v, rv, 1e-5).all(), np.abs(v - rv).max()
    srt = np.sort(rv, axis=1)
    sure = srt[:, -1] - srt[:, -2] > 1e-5 * np.maximum(np.abs(srt[:, -1]), 1.0)
    assert np.array_equal(act.cpu().numpy()[sure], ra[sure])


def test_backup_rejects_bad_arguments(dev):
    torch, bcts = dev
    z = torch.zeros(64, dtype=torch.float32, device="cuda")
    a = torch.zeros(4, dtype=torch.int32, device="cuda")
    for args in ((1, 33, 1), (1, 4, 17), (-1, 4, 1)):
        with pytest.raises(bcts.BctsError) as e:
            bcts.bcts_backup(z, z, z, z, z, *args, 0.99, 1.0, a, z)
        assert e.value.code == bcts.BCTS_EINVAL
