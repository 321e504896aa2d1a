"""The oracle against its own recorded output (tests/golden/, written by
tests/golden/make_golden.py): a regression guard, not an independent pin."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_golden  # noqa: E402


@pytest.mark.parametrize("name", sorted(make_golden.CASES))
def test_oracle_matches_recorded_output(name):
    ref = np.loadtxt(make_golden.path(name), comments="#")
    got = make_golden.run_case(name)
    assert got.shape == ref.shape
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-15)
