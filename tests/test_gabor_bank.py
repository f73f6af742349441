"""The library's Gabor bank (host code, no GPU) is the oracle's, bit for bit, and its arguments are
checked."""
import numpy as np
import pytest

import oracle


def test_bank_matches_the_oracle():
    import paper_2604_05794_b300 as hf
    for kw in (dict(), dict(sigma_along=3.0, sigma_across=1.0, lambda_=5.0)):
        got = hf.gabor_bank(**kw)
        want = oracle.gabor_bank(64, 7, kw.get("sigma_along", 2.5), kw.get("sigma_across", 1.5), kw.get("lambda_", 4.0))
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    with pytest.raises(Exception):
        hf.gabor_bank(n_theta=32)
