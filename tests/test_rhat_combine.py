"""The host half of R - 1 (Sec. 4.1), bst_r_minus_1_combine, from chain means and within-chain
cross products formed in numpy, against the oracle's R - 1 of the same draws (no GPU)."""
import numpy as np
import pytest

import oracle as O


def _parts(x):
    m = x.mean(axis=0)
    dev = x - m
    return m, np.einsum("tca,tcb->ab", dev, dev)


@pytest.mark.parametrize("n,M,d", [(2, 2, 1), (50, 7, 3), (300, 33, 6), (120, 64, 27)])
def test_combine_matches_the_oracle(n, M, d):
    from paper_2606_04895_gb300 import r_minus_1_combine
    rng = np.random.default_rng(n + M + d)
    A = rng.normal(size=(d, d)) / np.sqrt(d) + np.eye(d)
    x = rng.normal(size=(n, M, d)) @ A.T + 0.5 * rng.normal(size=(1, M, d))
    m, S = _parts(x)
    assert r_minus_1_combine(n, m, S) == pytest.approx(O.r_minus_1(x), rel=1e-10)


def test_combine_worked_example_and_undefined_cases():
    from paper_2606_04895_gb300 import BstError, r_minus_1_combine
    x = np.array([[[0.0], [4.0]], [[2.0], [6.0]]])  # chains (0, 2) and (4, 6): B / W = 8 / 2
    m, S = _parts(x)
    assert r_minus_1_combine(2, m, S) == pytest.approx(4.0, rel=1e-14)
    y = np.random.default_rng(1).normal(size=(20, 5, 2))
    y[:, :, 1] = 3.0  # no spread in one dimension
    assert np.isnan(r_minus_1_combine(20, *_parts(y)))
    with pytest.raises(BstError):
        r_minus_1_combine(1, m, S)  # one draw
    with pytest.raises(BstError):
        r_minus_1_combine(2, m[:1], S)  # one chain
    with pytest.raises(BstError):
        r_minus_1_combine(2, m, np.zeros((2, 2)))
