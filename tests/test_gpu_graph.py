"""dp_compute replayed from a captured graph (after one direct call per key) against direct calls:
the same results, and a new capture when the parameters, the precision or the routing change."""
import os

import numpy as np
import pytest

import dpsynth
from gpu_common import rms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    import paper_2005_00223_gb300 as pkg
    pkg.load()
    return pkg


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_compute_graph_replay(dp, prec):
    cfg = dpsynth.copper_config()
    coord, typ, box = dpsynth.copper_fcc(2, ncell=5)
    p1 = dpsynth.model_params(cfg, 1)
    p2 = dpsynth.model_params(cfg, 2)
    m = dp.Model(cfg, 0, params=p1)
    nl = dp.NeighborList(m, coord, typ, box, skin=1.0)
    rng = np.random.default_rng(3)
    shifted = coord + rng.normal(scale=0.05, size=coord.shape)
    tol = 1e-12 if prec == "fp64" else 1e-4   # MIX-16: run-to-run noise of its FP32 atomics
    # direct, then captured, then replayed; different coordinates each time through the same graph
    runs = [nl.compute(c, box, prec) for c in (coord, shifted, coord, shifted)]
    os.environ["DP_NO_GRAPH"] = "1"
    try:
        direct = [nl.compute(c, box, prec) for c in (coord, shifted)]
    finally:
        os.environ.pop("DP_NO_GRAPH", None)
    for got, ref in ((runs[2], runs[0]), (runs[3], runs[1]), (runs[2], direct[0]), (runs[3], direct[1])):
        assert abs(got[0] - ref[0]) <= tol * abs(ref[0])
        assert rms(got[2] - ref[2]) <= tol * rms(ref[2])
        np.testing.assert_allclose(got[3], ref[3], rtol=0, atol=tol * np.abs(ref[3]).max())
    assert abs(runs[1][0] - runs[0][0]) > 1e-9 * abs(runs[0][0])   # the coordinates did reach the graph
    # new parameters: the replay must not keep the old weights
    m.params = p2
    after = [nl.compute(coord, box, prec) for _ in range(3)]
    fresh = dp.Model(cfg, 0, params=p2)
    nf = dp.NeighborList(fresh, coord, typ, box, skin=1.0)
    ref = nf.compute(coord, box, prec)
    for got in after:
        assert abs(got[0] - ref[0]) <= tol * abs(ref[0])
        assert rms(got[2] - ref[2]) <= tol * rms(ref[2])
    nf.close()
    nl.close()
