"""The oracle against its own stored outputs (tests/golden/oracle_regression.json).

A failure means the oracle's arithmetic changed: such a change must name, in its commit message,
the passage of the paper (or the reading of it) that justifies it, and regenerate the file with
tests/golden/make_oracle_regression.py.  The tolerance allows for a different libm on another host.
"""
import json
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_oracle_regression as gen  # noqa: E402


@pytest.mark.parametrize("case", sorted(gen.CASES))
def test_oracle_matches_stored_outputs(orc, case):
    with open(os.path.join(HERE, "golden", "oracle_regression.json")) as f:
        ref = json.load(f)[case]
    cfg, params, coord, typ, box = gen.system(case)
    E, Ei, F, W = orc.Model(cfg, params).compute(coord, typ, box)
    assert E == pytest.approx(ref["E"], rel=1e-12)
    scale = max(abs(v) for row in ref["F"].values() for v in row)
    for a, row in ref["F"].items():
        np.testing.assert_allclose(F[int(a)], row, rtol=0, atol=1e-11 * scale)
        assert Ei[int(a)] == pytest.approx(ref["Ei"][a], rel=1e-11, abs=1e-14)
    np.testing.assert_allclose(W.reshape(-1), ref["W"], rtol=0, atol=1e-11 * max(map(abs, ref["W"])))
