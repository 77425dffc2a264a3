"""Mixed-precision schemes (Sec. 4.1.3) against the FP64 oracle: stated error budgets.

FP32 nets (MIX-32): budgets from FP32 rounding (unit roundoff 6e-8, sums of
up to 1600 terms, chains of six layers): relative energy error below 1e-6,
per-atom energy and force RMSE below 1e-5 of their scale.  MIX-16 (fp16 or
bf16 operands on the tensor cores, FP32 accumulation): budgets in units of
the operand's unit roundoff u.  The errors measured on the GPU are printed
for the record.
"""
import numpy as np
import pytest

import dpsynth
from gpu_common import rms, sampled_oracle_force, systems

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    import paper_2005_00223_gb300 as pkg
    pkg.load()
    return pkg


def _errors(got, ref):
    E, Ei, F, W = got
    Er, Eir, Fr, Wr = ref
    return {
        "dE_rel": abs(E - Er) / abs(Er),
        "dE_per_sum_abs_Ei": abs(E - Er) / float(np.abs(Eir).sum()),
        "dEi_max_rel": float(np.abs(Ei - Eir).max() / np.abs(Eir).max()),
        "F_rmse_rel": float(np.sqrt(((F - Fr) ** 2).sum(1).mean()) / rms(Fr)),
        "F_rmse": float(np.sqrt(((F - Fr) ** 2).sum(1).mean())),
        "W_rel": float(np.abs(W - Wr).max() / np.abs(Wr).max()),
    }


@pytest.mark.parametrize("name,cfg,coord,typ,box", systems(), ids=[s[0] for s in systems()])
def test_mix32_error_budget(dp, orc, name, cfg, coord, typ, box):
    m = dp.Model(cfg, 1, params=dpsynth.model_params(cfg, 1))
    nl = dp.NeighborList(m, coord, typ, box)
    got = nl.compute(coord, box, "mix32")
    ref = orc.Model(cfg, m.params).compute(coord, typ, box)
    err = _errors(got, ref)
    print(name, "mix32", err)
    assert err["dE_rel"] < 1e-6
    assert err["dEi_max_rel"] < 1e-5
    assert err["F_rmse_rel"] < 1e-5
    assert err["W_rel"] < 1e-5


def test_mix32_md_runs(dp):
    cfg = dpsynth.copper_config()
    coord, typ, box = dpsynth.copper_fcc(1, ncell=10)
    mass = np.array([dpsynth.MASS["Cu"]])
    vel = dpsynth.velocities(mass[typ], 300.0, 1)
    m = dp.Model(cfg, 1)
    st = dp.MDState(m, coord, vel, typ, mass, box, skin=2.0)
    th = st.step(20, 1.0, "mix32", thermo_every=10)
    assert np.isfinite(th).all()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("name,cfg,coord,typ,box", systems(), ids=[s[0] for s in systems()])
def test_mix16_tensor_core_error_budget(dp, orc, prec, name, cfg, coord, typ, box):
    """MIX-16 on tcgen05: embedding GEMMs with fp16/bf16 operands, FP32 accumulation and epilogues."""
    m = dp.Model(cfg, 1, params=dpsynth.model_params(cfg, 1))
    nl = dp.NeighborList(m, coord, typ, box)
    got = nl.compute(coord, box, prec)
    ref = orc.Model(cfg, m.params).compute(coord, typ, box)
    err = _errors(got, ref)
    print(name, prec, err)
    assert np.isfinite(got[2]).all()
    # budgets from the unit roundoff u of the operands (bf16 2^-9, fp16 2^-11) through
    # three embedding and three fitting layers: a few u per atom, ~10 u on forces
    u = 2.0 ** -9 if prec == "bf16" else 2.0 ** -11
    assert err["dE_per_sum_abs_Ei"] < 2 * u
    assert err["dEi_max_rel"] < 4 * u
    assert err["F_rmse_rel"] < 10 * u
    assert err["W_rel"] < 10 * u


@pytest.mark.parametrize("name,cfg,coord,typ,box", systems(), ids=[s[0] for s in systems()])
def test_split_bf16_tensor_core_error_budget(dp, orc, name, cfg, coord, typ, box):
    """bf16x3 on tcgen05: every embedding product as hi hi + hi lo + lo hi of split bf16 operands
    (16 significant bits, u = 2^-16), FP32 accumulation, tanhf; FP32 fitting net.  Budgets in units
    of that u as for MIX-16, and the force criterion 1e-3 of the RMS force."""
    m = dp.Model(cfg, 1, params=dpsynth.model_params(cfg, 1))
    nl = dp.NeighborList(m, coord, typ, box)
    got = nl.compute(coord, box, "bf16x3")
    ref = orc.Model(cfg, m.params).compute(coord, typ, box)
    err = _errors(got, ref)
    print(name, "bf16x3", err)
    assert np.isfinite(got[2]).all()
    u = 2.0 ** -16
    assert err["dE_per_sum_abs_Ei"] < 2 * u
    assert err["dEi_max_rel"] < 4 * u
    assert err["F_rmse_rel"] < 10 * u
    assert err["W_rel"] < 10 * u
    assert err["F_rmse_rel"] < 1e-3


def test_split_bf16_md_runs(dp):
    cfg = dpsynth.copper_config()
    coord, typ, box = dpsynth.copper_fcc(1, ncell=10)
    mass = np.array([dpsynth.MASS["Cu"]])
    vel = dpsynth.velocities(mass[typ], 300.0, 1)
    m = dp.Model(cfg, 1)
    st = dp.MDState(m, coord, vel, typ, mass, box, skin=2.0)
    th = st.step(20, 1.0, "bf16x3", thermo_every=10)
    assert np.isfinite(th).all()


@pytest.mark.parametrize("prec", ["mix32", "bf16", "fp16", "bf16x3"])
def test_paper_water_model_error_budget(dp, orc, prec):
    """The paper's production water model (embedding 32-64-128, 144 neighbors, Sec. 5.1) on the
    mixed schemes: the 32-64-128 tensor-core embedding and 2048-wide fitting kernels against the
    oracle, with the budgets above."""
    cfg = dpsynth.water_paper_config()
    coord, typ, box = dpsynth.water_box(4)
    m = dp.Model(cfg, 1, params=dpsynth.model_params(cfg, 3))
    nl = dp.NeighborList(m, coord, typ, box)
    got = nl.compute(coord, box, prec)
    ref = orc.Model(cfg, m.params).compute(coord, typ, box)
    err = _errors(got, ref)
    print("water192 paper model", prec, err)
    assert np.isfinite(got[2]).all()
    if prec == "mix32":
        assert err["dE_rel"] < 1e-6 and err["dEi_max_rel"] < 1e-5
        assert err["F_rmse_rel"] < 1e-5 and err["W_rel"] < 1e-5
    else:
        u = {"bf16": 2.0 ** -9, "fp16": 2.0 ** -11, "bf16x3": 2.0 ** -16}[prec]
        assert err["dE_per_sum_abs_Ei"] < 2 * u
        assert err["dEi_max_rel"] < 4 * u
        assert err["F_rmse_rel"] < 10 * u
        assert err["W_rel"] < 10 * u
    nl.close()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_mix16_student_shape_and_md(dp, prec):
    cfg = dpsynth.copper_student_config()
    coord, typ, box = dpsynth.copper_fcc(1, ncell=6)
    mass = np.array([dpsynth.MASS["Cu"]])
    vel = dpsynth.velocities(mass[typ], 300.0, 1)
    m = dp.Model(cfg, 2)
    st = dp.MDState(m, coord, vel, typ, mass, box, skin=2.0)
    th = st.step(10, 1.0, prec, thermo_every=5)
    assert np.isfinite(th).all()


@pytest.mark.parametrize("prec", ["bf16", "fp64"])
def test_far_unwrapped_coordinates(dp, prec):
    """Atoms shifted by random whole box vectors (up to 40 boxes away) give the same neighbor list and,
    up to the rounding of the larger coordinates, the same energy and forces: the minimum image works
    on raw coordinates, and the FP32 prefilter of the formatting uses coordinates wrapped in FP64."""
    cfg = dpsynth.water_config()
    coord, typ, box = dpsynth.water_box(3)
    L = np.diag(box)
    rng = np.random.default_rng(11)
    shifted = coord + rng.integers(-40, 41, size=coord.shape) * L
    m = dp.Model(cfg, 1)
    nl0 = dp.NeighborList(m, coord, typ, box)
    nl1 = dp.NeighborList(m, shifted, typ, box)
    E0, _, F0, W0 = nl0.compute(coord, box, prec)
    E1, _, F1, W1 = nl1.compute(shifted, box, prec)
    a, _ = nl0.get()
    b, _ = nl1.get()
    # the same neighbor set per atom (a key can move by one unit in its last place with the shifted rounding)
    nsel = sum(cfg.sel)
    for i in range(len(typ)):
        assert set(a.reshape(-1, nsel)[i]) == set(b.reshape(-1, nsel)[i])
    # MIX-16 sums T and the forces with FP32 / FP64 atomics in whatever order the blocks run, and a
    # last-bit change of an FP32 value can flip the rounding of a 16-bit operand (2^-8 for bf16): two
    # evaluations of the same coordinates already differ by up to about 1e-6 of the RMS force, with
    # rare flips near 1e-4; a wrong minimum image would move forces by O(1)
    tol = 1e-9 if prec == "fp64" else 1e-3
    assert abs(E1 - E0) <= tol * np.abs(E0)
    assert rms(F1 - F0) <= tol * rms(F0)
    assert np.abs(W1 - W0).max() <= tol * np.abs(W0).max()
    nl0.close()
    nl1.close()


@pytest.mark.slow
@pytest.mark.parametrize("prec,u", [("bf16", 2.0 ** -9), ("fp16", 2.0 ** -11)])
def test_mix16_copper_108k_sampled(dp, orc, prec, u):
    """The 108,000-atom copper workload on the tensor-core path: the neighbor list equals the oracle's, and
    sampled E_i and F_k are within the 16-bit error budget of the FP64 oracle (4u of E_k; 30u of the RMS
    force per atom, three times the 10u RMSE budget)."""
    cfg = dpsynth.copper_config()
    coord, typ, box = dpsynth.copper_fcc(1, ncell=30)
    p = dpsynth.model_params(cfg, 1)
    m = dp.Model(cfg, 0, params=p)
    nl = dp.NeighborList(m, coord, typ, box, skin=2.0)
    E, Ei, F, W = nl.compute(coord, box, prec)
    om = orc.Model(cfg, p)
    nref, _, _ = om.nlist(coord, typ, box)
    np.testing.assert_array_equal(nl.get()[0], nref)
    fs = rms(F)
    samples = [sampled_oracle_force(om, coord, typ, box, nref, k) for k in (0, 4321, 107999)]
    escale = max(abs(s[0]) for s in samples)
    for k, (Ek, Fk) in zip((0, 4321, 107999), samples):
        assert abs(Ei[k] - Ek) <= 4 * u * escale
        assert np.linalg.norm(F[k] - Fk) <= 30 * u * fs
    assert abs(E - Ei.sum()) <= 1e-12 * np.abs(Ei).sum()
    np.testing.assert_allclose(F.sum(0), 0.0, atol=1e-6 * fs * np.sqrt(len(F)))
    nl.close()
