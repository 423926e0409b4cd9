"""Pin the oracle's Bellman penalty (Eq. 7).

Eq. 7 is Lemma 3's approximation of the bias gap B_e - B_o with the standard
deviations replaced by delta / sqrt(2) (Prop. 1).  Two independent checks:
  * the Lemma 3 form evaluated at sigma = delta / sqrt(2) (an algebraic identity);
  * the exact GEV biases of Lemma 2 (with the normal quantile from the standard
    library), which Eq. 7 approximates when A^(d-1) >> 1: within 5 % for
    A^(d-1) >= 18.  A dropped term, a wrong sign, sqrt(d) and sqrt(d-1) swapped or
    a log base other than e breaks one of the two.
"""
import math
from statistics import NormalDist

import pytest

EULER_GAMMA = 0.5772156649015329
_ppf = NormalDist().inv_cdf


def lemma3(sig_e, sig_o, A, d):
    return math.sqrt(2 * math.log(A)) * (sig_e * math.sqrt(d) - sig_o * math.sqrt(d - 1)) - (sig_e - sig_o) / 2


def bias_n(n):
    """B(n) of Lemma 2's proof: the GEV mean shift of the max of n unit normals."""
    if n == 1:
        return 0.0
    return EULER_GAMMA * _ppf(1 - 1 / (math.e * n)) + (1 - EULER_GAMMA) * _ppf(1 - 1 / n)


def lemma2_gap(sig_e, sig_o, A, d):
    return sig_e * bias_n(A ** d - A ** (d - 1)) - sig_o * bias_n(A ** (d - 1))


CASES = [(de, do, A, d) for de in (0.3, 1.7) for do in (0.05, 0.9) for A in (2, 6, 18) for d in (1, 2, 3, 4)]


@pytest.mark.parametrize("de,do,A,d", CASES)
def test_eq7_equals_lemma3_at_sigma_delta_over_sqrt2(oracle_lib, de, do, A, d):
    s2 = math.sqrt(2.0)
    assert oracle_lib.bellman_penalty(de, do, A, d) == pytest.approx(lemma3(de / s2, do / s2, A, d), rel=1e-13,
                                                                      abs=1e-14)


@pytest.mark.parametrize("A,d", [(18, 2), (18, 3), (18, 4), (6, 3), (6, 4), (9, 3)])
@pytest.mark.parametrize("de,do", [(4.0, 1.0), (1.0, 0.5), (2.0, 1.9)])
def test_eq7_approximates_exact_gev_gap(oracle_lib, A, d, de, do):
    assert A ** (d - 1) >= 6
    s2 = math.sqrt(2.0)
    exact = lemma2_gap(de / s2, do / s2, A, d)
    assert oracle_lib.bellman_penalty(de, do, A, d) == pytest.approx(exact, rel=0.05)


def test_eq7_hand_values(oracle_lib):
    # A = 4, d = 2, de = 2, do = 1:
    #   sqrt(ln 4) * (2*sqrt(2) - 1) - (2 - 1)/sqrt(8)
    #   = 1.1774100225 * 1.8284271247 - 0.3535533906 = 1.79927... (worked by hand)
    v = oracle_lib.bellman_penalty(2.0, 1.0, 4, 2)
    assert v == pytest.approx(1.1774100225154747 * 1.8284271247461903 - 0.3535533905932738, rel=1e-14)
    assert 1.7992 < v < 1.7993
    # d = 1: the delta_o * sqrt(d-1) term vanishes
    assert oracle_lib.bellman_penalty(1.0, 5.0, 18, 1) == pytest.approx(
        math.sqrt(math.log(18)) * 1.0 - (1.0 - 5.0) / math.sqrt(8), rel=1e-14)
    # equal errors at depth 1 with A = e^1 would cancel; with delta_e = delta_o = 0 it is 0
    assert oracle_lib.bellman_penalty(0.0, 0.0, 18, 3) == 0.0


def test_bias_ordering_lemma2():
    """0 <= B_o < B_e whenever sigma_e > sigma_o (Lemma 2) -- checks bias_n itself."""
    for A in (2, 3, 6, 18):
        for d in (1, 2, 3, 4):
            b_o, b_e = 1.0 * bias_n(A ** (d - 1)), 1.5 * bias_n(A ** d - A ** (d - 1))
            if A ** d - A ** (d - 1) == 1:  # d = 1, A = 2: both sub-trees hold one leaf
                assert b_o == b_e == 0.0
            else:
                assert 0.0 <= b_o < b_e


# ---- Lemma 2's exact bias gap (the exact-GEV correction) ------------------------

@pytest.mark.parametrize("q", [0.5, 0.3, 0.9, 1e-3, 1 / 18, 1 / 324, 1 / (math.e * 18 ** 5), 1e-9])
def test_normal_upper_quantile_matches_library(oracle_lib, q):
    # Phi^-1(1 - q) = -Phi^-1(q): the lower-tail library quantile keeps full precision
    assert oracle_lib.normal_upper_quantile(q) == pytest.approx(-_ppf(q), abs=1e-12)


@pytest.mark.parametrize("de,do,A,d", CASES)
def test_exact_penalty_equals_lemma2(oracle_lib, de, do, A, d):
    s2 = math.sqrt(2.0)
    assert oracle_lib.bellman_penalty_exact(de, do, A, d) == pytest.approx(
        lemma2_gap(de / s2, do / s2, A, d), rel=1e-9, abs=1e-12)


def test_exact_penalty_special_cases(oracle_lib):
    # d = 1, A = 2: both sub-trees hold one leaf, no maximisation bias at all
    assert oracle_lib.bellman_penalty_exact(3.0, 0.5, 2, 1) == 0.0
    # d = 1: B_o = 0 (one leaf under pi_o); B_e is the shift of a max of A - 1 normals
    assert oracle_lib.bellman_penalty_exact(2.0, 7.0, 18, 1) == pytest.approx(
        2.0 / math.sqrt(2.0) * bias_n(17), rel=1e-12)
    # A = 1: no other action, nothing to correct
    assert oracle_lib.bellman_penalty_exact(1.0, 1.0, 1, 3) == 0.0
    # linear in (delta_e, delta_o) and antisymmetric under swapping the leaf counts' roles
    a = oracle_lib.bellman_penalty_exact(1.0, 0.0, 6, 3)
    b = oracle_lib.bellman_penalty_exact(0.0, 1.0, 6, 3)
    assert oracle_lib.bellman_penalty_exact(2.5, 0.75, 6, 3) == pytest.approx(2.5 * a + 0.75 * b, rel=1e-12)
    assert a > 0.0 > b


# ---- Lemma 2 against simulation (Thm. 1's setting, Normal leaf noise) -------------

@pytest.mark.parametrize("m", [18, 324, 5832])
def test_gev_shift_approximates_expected_maximum(oracle_lib, m):
    """Lemma 2's shift of the maximum of m iid unit normals (its GEV mean) is close to
    the Monte Carlo mean of that maximum, and closer as m grows (an asymptotic
    statement): within 6 % at m = 18, 3 % beyond."""
    import numpy as np
    rng = np.random.default_rng(2021)
    trials = 4000 if m <= 324 else 1500
    mc = rng.standard_normal((trials, m)).max(axis=1).mean()
    # the oracle's exact gap at delta_o = 0, delta_e = sqrt 2 (sigma_e = 1) is this shift
    # for m = A^d - A^(d-1) leaves: 18 = 19 - 1 (A = 19, d = 1), 324 = 18^2 - 18 ... checked
    # directly where such (A, d) exist, through bias_n (the library quantile) otherwise
    shift = bias_n(m)
    if m == 18:
        assert oracle_lib.bellman_penalty_exact(math.sqrt(2.0), 0.0, 19, 1) == pytest.approx(shift, rel=1e-9)
    assert shift == pytest.approx(mc, rel=0.06 if m == 18 else 0.03)


def test_corrected_values_restore_the_ordering_in_expectation():
    """Thm. 1 in its Normal-noise model: with sigma_e > sigma_o the uncorrected maxima
    favour the noisier sub-trees even when pi_o is better, and subtracting the
    Lemma 2 gap (B_e - B_o) restores E[Q(pi_o)] > E[max other]."""
    import numpy as np
    rng = np.random.default_rng(7)
    A, d = 4, 3
    n_o, n_e = A ** (d - 1), A ** d - A ** (d - 1)
    mu_o, mu_e, s_o, s_e = 1.0, 0.8, 0.2, 1.0
    trials = 20000
    max_o = (mu_o + s_o * rng.standard_normal((trials, n_o))).max(axis=1)
    max_e = (mu_e + s_e * rng.standard_normal((trials, n_e))).max(axis=1)
    assert max_o.mean() < max_e.mean()  # the bias hands the noisier sub-tree the win
    gap = s_e * bias_n(n_e) - s_o * bias_n(n_o)
    assert max_o.mean() > (max_e - gap).mean()  # corrected: the true ordering returns
    # both sides then carry the same bias B_o: E[max_o] ~ mu_o + B_o, E[max_e - gap] ~ mu_e + B_o
    assert max_o.mean() == pytest.approx(mu_o + s_o * bias_n(n_o), abs=0.03)
    assert (max_e - gap).mean() == pytest.approx(mu_e + s_o * bias_n(n_o), abs=0.05)
