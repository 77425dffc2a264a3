"""GPU parity of the FP64 path against the FP64 oracle, through the C-ABI.

Neighbor lists must be bit-identical; E, E_i, F and W must agree within
1e-10 relative (norm-wise, against the oracle's scale).
"""
import os

import numpy as np
import pytest

import dpsynth
from gpu_common import assert_close_fp64, rms, sampled_oracle_force, systems

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    import paper_2005_00223_gb300 as pkg
    pkg.load()
    return pkg


def _model(dp, cfg, seed=1, params=None):
    m = dp.Model(cfg, seed)
    m.params = dpsynth.model_params(cfg, seed) if params is None else params
    return m


def test_seeded_weights_match_generator(dp):
    for cfg in (dpsynth.water_config(), dpsynth.copper_student_config()):
        m = dp.Model(cfg, 77)
        ref = dpsynth.model_params(cfg, 77)
        got = m.params
        assert got.shape == ref.shape
        np.testing.assert_allclose(got, ref, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("name,cfg,coord,typ,box", systems(), ids=[s[0] for s in systems()])
def test_nlist_bit_exact(dp, orc, name, cfg, coord, typ, box):
    m = _model(dp, cfg)
    ref, ntr_ref, _ = orc.Model(cfg, m.params).nlist(coord, typ, box)
    for skin in (0.0, 2.0):
        nl = dp.NeighborList(m, coord, typ, box, skin=skin)
        got, ntr = nl.get()
        np.testing.assert_array_equal(got, ref)
        assert ntr == ntr_ref


def test_nlist_truncation_and_update(dp, orc):
    cfg = dpsynth.ModelConfig(ntypes=1, rcut=8.0, rcut_smth=2.0, sel=(40,))
    m = _model(dp, cfg)
    om = orc.Model(cfg, m.params)
    coord, typ, box = dpsynth.copper_fcc(3, ncell=5)
    nl = dp.NeighborList(m, coord, typ, box, skin=1.0)
    got, ntr = nl.get()
    ref, ntr_ref, _ = om.nlist(coord, typ, box)
    np.testing.assert_array_equal(got, ref)
    assert ntr == ntr_ref > 0
    moved = coord + np.random.default_rng(0).normal(scale=0.3, size=coord.shape)
    nl.update(moved, box)
    got, ntr = nl.get()
    ref, ntr_ref, _ = om.nlist(moved, typ, box)
    np.testing.assert_array_equal(got, ref)


def test_nlist_exact_ties_and_cutoff(dp, orc):
    cfg = dpsynth.ModelConfig(ntypes=1, rcut=2.0, rcut_smth=0.5, sel=(8,), embed=(8, 16, 32), m2=4, fit=(16, 16, 16))
    m = _model(dp, cfg)
    c0 = np.array([5.0, 5.0, 5.0])
    coord = np.array([c0, c0 + [1.5, 0, 0], c0 - [1.5, 0, 0], c0 + [0, 1.5, 0], c0 + [2.0, 0, 0],
                      c0 + [0, 0, 1.25], c0 - [0, 0, 1.25]])
    typ = np.zeros(7, dtype=np.int32)
    box = np.diag([20.0, 20.0, 20.0])
    nl = dp.NeighborList(m, coord, typ, box)
    got, _ = nl.get()
    np.testing.assert_array_equal(got[0], [5, 6, 1, 2, 3, -1, -1, -1])
    ref, _, _ = orc.Model(cfg, m.params).nlist(coord, typ, box)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("route", ["auto", "split"])
@pytest.mark.parametrize("name,cfg,coord,typ,box", systems(), ids=[s[0] for s in systems()])
def test_fp64_matches_oracle(dp, orc, name, cfg, coord, typ, box, route):
    """route split: the tensor-core split products forced on (they are used from 1,024 atoms on)."""
    m = _model(dp, cfg)
    nl = dp.NeighborList(m, coord, typ, box)
    if route == "split":
        os.environ["DP_OZ_MIN_ATOMS"] = "0"
    try:
        got = nl.compute(coord, box, "fp64")
    finally:
        os.environ.pop("DP_OZ_MIN_ATOMS", None)
    ref = orc.Model(cfg, m.params).compute(coord, typ, box)
    assert_close_fp64(got, ref)
    assert rms(ref[2]) > 0


@pytest.mark.parametrize("name,cfg,coord,typ,box", systems()[:2], ids=[s[0] for s in systems()[:2]])
def test_fp64_cuda_core_route_matches_oracle(dp, orc, name, cfg, coord, typ, box):
    """The all-CUDA-core FP64 kernels (used for net shapes without a split-product route) still agree."""
    m = _model(dp, cfg)
    nl = dp.NeighborList(m, coord, typ, box)
    os.environ["DP_NO_OZAKI"] = "1"
    try:
        got = nl.compute(coord, box, "fp64")
    finally:
        os.environ.pop("DP_NO_OZAKI", None)
    assert_close_fp64(got, orc.Model(cfg, m.params).compute(coord, typ, box))


@pytest.mark.parametrize("route", ["cuda_cores", "split"])
def test_fp64_paper_net_shape(dp, orc, route):
    """The nets of the paper's production models (embedding 32-64-128, Sec. 5.1) on two neighbor types."""
    cfg = dpsynth.ModelConfig(ntypes=2, rcut=6.0, rcut_smth=0.5, sel=(46, 92), embed=(32, 64, 128), m2=16,
                              fit=(240, 240, 240))
    coord, typ, box = dpsynth.water_box(2)
    m = _model(dp, cfg, seed=4)
    nl = dp.NeighborList(m, coord, typ, box)
    os.environ["DP_OZ_MIN_ATOMS" if route == "split" else "DP_NO_OZAKI"] = "0" if route == "split" else "1"
    try:
        got = nl.compute(coord, box, "fp64")
    finally:
        os.environ.pop("DP_OZ_MIN_ATOMS", None)
        os.environ.pop("DP_NO_OZAKI", None)
    assert_close_fp64(got, orc.Model(cfg, m.params).compute(coord, typ, box))


def test_fp64_student_shape_and_batches(dp, orc):
    """Student-size nets (8, 16, 32), and the multi-batch path (batch of 97 atoms), on both routes."""
    cfg = dpsynth.copper_student_config()
    coord, typ, box = dpsynth.copper_fcc(2, ncell=5)
    ref = None
    for batch, route in (("0", "auto"), ("97", "auto"), ("0", "split"), ("97", "split")):
        os.environ["DP_BATCH_ATOMS"] = batch
        try:
            m = _model(dp, cfg, seed=3)
        finally:
            os.environ.pop("DP_BATCH_ATOMS", None)
        nl = dp.NeighborList(m, coord, typ, box, skin=1.0)
        if route == "split":
            os.environ["DP_OZ_MIN_ATOMS"] = "0"
        try:
            got = nl.compute(coord, box, "fp64")
        finally:
            os.environ.pop("DP_OZ_MIN_ATOMS", None)
        if ref is None:
            ref = orc.Model(cfg, m.params).compute(coord, typ, box)
        assert_close_fp64(got, ref)


def test_fp64_ragged_small_systems(dp, orc):
    """Two and three isolated atoms, and atoms with no neighbor of one type."""
    cfg = dpsynth.water_config()
    box = np.diag([20.0, 20.0, 20.0])
    m = _model(dp, cfg, seed=4)
    om = orc.Model(cfg, m.params)
    for coord, typ in [
        (np.array([[5.0, 5.0, 5.0], [6.2, 5.3, 4.9]]), np.array([0, 1])),
        (np.array([[5.0, 5.0, 5.0], [6.2, 5.3, 4.9], [15.0, 15.0, 15.0]]), np.array([0, 0, 1])),
        (np.array([[5.0, 5.0, 5.0], [5.9, 5.1, 5.2], [4.1, 5.3, 5.5], [9.5, 5.0, 5.0]]), np.array([0, 1, 1, 1])),
    ]:
        typ = typ.astype(np.int32)
        nl = dp.NeighborList(m, coord, typ, box)
        got = nl.compute(coord, box, "fp64")
        ref = om.compute(coord, typ, box)
        E, Ei, F, W = got
        assert abs(E - ref[0]) <= 1e-10 * abs(ref[0])
        np.testing.assert_allclose(Ei, ref[1], rtol=1e-10, atol=1e-14)
        np.testing.assert_allclose(F, ref[2], rtol=1e-9, atol=1e-12 * max(1e-300, np.abs(ref[2]).max()))


def test_empty_system(dp):
    cfg = dpsynth.water_config()
    m = _model(dp, cfg)
    box = np.diag([20.0, 20.0, 20.0])
    nl = dp.NeighborList(m, np.zeros((0, 3)), np.zeros(0, dtype=np.int32), box)
    E, Ei, F, W = nl.compute(np.zeros((0, 3)), box, "fp64")
    assert E == 0.0 and F.shape == (0, 3)


def test_bad_arguments_are_rejected(dp):
    cfg = dpsynth.water_config()
    m = _model(dp, cfg)
    coord, typ, box = dpsynth.water_box(1)
    with pytest.raises(dp.DPError, match="DP_ERR_BOX"):
        dp.NeighborList(m, coord, typ, np.diag([11.0, 12.42, 12.42]))
    bad = box.copy()
    bad[0, 1] = 0.5
    with pytest.raises(dp.DPError, match="DP_ERR_BOX"):
        dp.NeighborList(m, coord, typ, bad)
    t2 = typ.copy()
    t2[3] = 5
    with pytest.raises(dp.DPError, match="DP_ERR_ARG"):
        dp.NeighborList(m, coord, t2, box)
    with pytest.raises(dp.DPError, match="DP_ERR_CAPACITY"):
        dp.NeighborList(m, coord, typ, box, skin=2.0, cand_cap=32)
    with pytest.raises(dp.DPError, match="DP_ERR_ARG"):
        dp.dp_model_set_params(m.h, np.zeros(5))


def test_fp64_copper_4000_full_oracle(dp, orc):
    """The 4,000-atom copper workload: whole-system parity against the oracle."""
    cfg = dpsynth.copper_config()
    coord, typ, box = dpsynth.copper_fcc(1, ncell=10)
    m = _model(dp, cfg)
    nl = dp.NeighborList(m, coord, typ, box, skin=2.0)
    got = nl.compute(coord, box, "fp64")
    om = orc.Model(cfg, m.params)
    nref, _, _ = om.nlist(coord, typ, box)
    np.testing.assert_array_equal(nl.get()[0], nref)
    ref = om.compute(coord, typ, box, nref)
    assert_close_fp64(got, ref)


@pytest.mark.slow
def test_fp64_copper_108k_sampled(dp, orc):
    """The 108,000-atom copper box: sampled E_i and F_k against the oracle atom by atom."""
    cfg = dpsynth.copper_config()
    coord, typ, box = dpsynth.copper_fcc(1, ncell=30)
    m = _model(dp, cfg)
    nl = dp.NeighborList(m, coord, typ, box, skin=2.0)
    E, Ei, F, W = nl.compute(coord, box, "fp64")
    om = orc.Model(cfg, m.params)
    nref, _, _ = om.nlist(coord, typ, box)
    np.testing.assert_array_equal(nl.get()[0], nref)
    fs = rms(F)
    for k in (0, 4321, 107999):
        Ek, Fk = sampled_oracle_force(om, coord, typ, box, nref, k)
        assert abs(Ei[k] - Ek) <= 1e-10 * abs(Ek)
        assert np.linalg.norm(F[k] - Fk) <= 1e-10 * fs
    assert abs(E - Ei.sum()) <= 1e-12 * abs(E)
    np.testing.assert_allclose(F.sum(0), 0.0, atol=1e-9 * fs * np.sqrt(len(F)))
