"""The oracle against its regression fixture (tests/golden/, written by
tests/golden/make_golden.py from the oracle alone): iteration counts and
level counts exactly, factor and solution summaries to 1e-10 (libm may round
the network's exp / log differently on another host)."""
import json
import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def test_oracle_matches_its_fixture():
    stored = json.load(open(os.path.join(HERE, "golden", "poisson2d_32_oracle.json")))
    now = make_golden.compute()
    for k in ("n", "nnz", "levels_fwd", "levels_bwd", "iters", "ic0_shift"):
        assert now[k] == stored[k], k
    for k in ("sum_L_learned", "sum_L_ic0", "norm_x_learned", "norm_x_ic0"):
        assert now[k] == pytest.approx(stored[k], rel=1e-10), k
