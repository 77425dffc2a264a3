"""Deterministic force accumulation (dp_model_set_deterministic) on the FP64 and MIX-32 routes.

With the flag on, the pair terms g_ij (and the per-chunk virial terms of the FP64 split-product
route) are summed as exact fixed-point numbers in integer limbs, so an evaluation gives the same
bits every time; the result stays within FP64 rounding of the oracle and of the FP64-atomic path.
An MD run resumed from a checkpoint then follows the uninterrupted run bit for bit.
"""
import os

import numpy as np
import pytest

import dpsynth
from gpu_common import assert_close_fp64, rms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    import paper_2005_00223_gb300 as pkg
    pkg.load()
    return pkg


def _case(name):
    if name == "water192":
        return dpsynth.water_config(), *dpsynth.water_box(1)
    return dpsynth.copper_config(), *dpsynth.copper_fcc(1, ncell=5)


CASES = [("water192", "fp64", "simt"), ("water192", "fp64", "split"), ("cu500", "fp64", "split"),
         ("cu500", "mix32", "simt")]


@pytest.mark.parametrize("name,prec,route", CASES, ids=["-".join(c) for c in CASES])
def test_deterministic_evaluations_repeat_bit_for_bit(dp, orc, name, prec, route):
    cfg, coord, typ, box = _case(name)
    params = dpsynth.model_params(cfg, 3)
    if route == "split":
        os.environ["DP_OZ_MIN_ATOMS"] = "0"
    try:
        m = dp.Model(cfg, 1, params=params, deterministic=True)
        nl = dp.NeighborList(m, coord, typ, box)
        runs = [nl.compute(coord, box, prec) for _ in range(4)]   # direct calls, then graph replays
        nl2 = dp.NeighborList(m, coord, typ, box)                  # a second list and its own buffers
        runs.append(nl2.compute(coord, box, prec))
        free = dp.Model(cfg, 1, params=params)                    # FP64 atomics
        nlf = dp.NeighborList(free, coord, typ, box)
        ref_free = nlf.compute(coord, box, prec)
    finally:
        os.environ.pop("DP_OZ_MIN_ATOMS", None)
    E, Ei, F, W = runs[0]
    for r in runs[1:]:
        assert r[0] == E
        np.testing.assert_array_equal(r[1], Ei)
        np.testing.assert_array_equal(r[2], F)
        np.testing.assert_array_equal(r[3], W)
    if prec == "fp64":
        assert_close_fp64(runs[0], orc.Model(cfg, params).compute(coord, typ, box), rtol=1e-10)
    # the fixed-point sums differ from the FP64-atomic ones only by the atomics' rounding, which is
    # relative to pair terms many times larger than the net forces they cancel to
    assert np.sqrt(((F - ref_free[2]) ** 2).sum(1)).max() <= 1e-10 * rms(F)
    assert abs(E - ref_free[0]) <= 1e-13 * np.abs(Ei).sum()
    for x in (nl, nl2, nlf):
        x.close()
    m.close()
    free.close()


def test_flag_changes_captured_evaluations(dp):
    """Switching the flag re-captures: the first call after each switch runs the selected scatter."""
    cfg, coord, typ, box = _case("water192")
    m = dp.Model(cfg, 1)
    nl = dp.NeighborList(m, coord, typ, box)
    a = [nl.compute(coord, box, "fp64") for _ in range(3)]
    dp.dp_model_set_deterministic(m.h, True)
    b = [nl.compute(coord, box, "fp64") for _ in range(3)]
    np.testing.assert_array_equal(b[0][2], b[1][2])
    np.testing.assert_array_equal(b[0][2], b[2][2])
    assert np.abs(a[0][2] - b[0][2]).max() <= 1e-10 * rms(b[0][2])
    dp.dp_model_set_deterministic(m.h, False)
    c = nl.compute(coord, box, "fp64")
    assert np.abs(c[2] - b[0][2]).max() <= 1e-10 * rms(b[0][2])
    with pytest.raises(dp.DPError, match="DP_ERR_ARG"):
        dp._lib._check(dp._lib.load().dp_model_set_deterministic(m.h, 2), "dp_model_set_deterministic")
    nl.close()
    m.close()
