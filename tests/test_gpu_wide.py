"""Wide embedding nets (Sec. 6, "Network size") on the tensor cores against the FP64 oracle.

Nets (w, 2w, 4w) up to the paper's largest last layer (1024 x 2048) run layer by layer (wide.cu) in
MIX-16 with bf16 operands; the budgets are those of the other MIX-16 kernels in units of the bf16 unit
roundoff u = 2^-9, except the force RMSE: 20 u instead of 10 u (every bf16 operand carries up to u, and
the wide nets pass each row through products of up to 2,048 terms and a contraction over 4 w channels,
where the MIX-16 nets of the configs have 50 and 100).  Small systems keep the oracle's evaluation of the
wide nets to seconds.
"""
import numpy as np
import pytest

import dpsynth
from gpu_common import rms

pytestmark = pytest.mark.gpu

U = 2.0 ** -9


@pytest.fixture(scope="module")
def dp():
    import paper_2005_00223_gb300 as pkg
    pkg.load()
    return pkg


def _disordered_copper():
    """108 copper atoms, FCC 3^3 cells with seeded 0.3 A displacements on top of the lattice's 0.1 A:
    near the perfect lattice the net forces nearly cancel (their RMS varies 10x from one seeded model
    to the next while the absolute error of the 16-bit products does not), so a disordered box gives
    relative force errors that measure the arithmetic rather than the cancellation."""
    coord, typ, box = dpsynth.copper_fcc(3, ncell=3)
    rng = np.random.default_rng(17)
    return coord + rng.normal(scale=0.3, size=coord.shape), typ, box


def _systems(w):
    emb = (w, 2 * w, 4 * w)
    cu = dpsynth.ModelConfig(ntypes=1, rcut=4.0, rcut_smth=1.0, sel=(48,), embed=emb)
    out = [("cu108", cu, *_disordered_copper())]
    if w == 64:
        wa = dpsynth.ModelConfig(ntypes=2, rcut=6.0, rcut_smth=0.5, sel=(46, 92), embed=emb)
        out.append(("water192", wa, *dpsynth.water_box(2)))
    return out


@pytest.mark.parametrize("w", [64, 128, 256, 512])
def test_wide_nets_match_oracle(dp, orc, w):
    for name, cfg, coord, typ, box in _systems(w):
        params = dpsynth.model_params(cfg, 4)
        m = dp.Model(cfg, 1, params=params)
        nl = dp.NeighborList(m, coord, typ, box)
        E, Ei, F, W = nl.compute(coord, box, "bf16")
        Er, Eir, Fr, Wr = orc.Model(cfg, params).compute(coord, typ, box)
        err = {"dE": abs(E - Er) / np.abs(Eir).sum(), "dEi": np.abs(Ei - Eir).max() / np.abs(Eir).max(),
               "F": np.sqrt(((F - Fr) ** 2).sum(1).mean()) / rms(Fr), "W": np.abs(W - Wr).max() / np.abs(Wr).max()}
        print(name, cfg.embed, err)
        assert np.isfinite(F).all()
        assert err["dE"] < 2 * U and err["dEi"] < 4 * U and err["F"] < 20 * U and err["W"] < 10 * U
        # a second call (graph replay of the evaluation) gives the same result up to the order of the
        # FP32 atomic additions into the descriptor sums: each E_i then moves by at most about
        # sum(sel) x 2^-24 of its size, so the total by that fraction of sum |E_i| (not of |E|, which
        # can be far smaller than the sum of its terms)
        E2, _, F2, _ = nl.compute(coord, box, "bf16")
        assert abs(E2 - E) <= sum(cfg.sel) * 2.0 ** -24 * np.abs(Eir).sum()
        assert np.abs(F2 - F).max() <= 1e-4 * rms(F)
        nl.close()
        m.close()


@pytest.mark.parametrize("w", [128, 256])
def test_wide_nets_fp8_against_oracle(dp, orc, w):
    """The same nets with e4m3 operands in the layer-2/3 products (DP_MIX_FP8).  e4m3 keeps 3 mantissa
    bits (u8 = 2^-4); the errors are stated in units of u8 and bounded at the level of one rounding of
    the operands (forces within 2 u8 of the RMS force, energy within u8 / 4 of sum |E_i|); the
    printout records them against bf16's."""
    u8 = 2.0 ** -4
    name, cfg, coord, typ, box = _systems(w)[0]
    params = dpsynth.model_params(cfg, 4)
    m = dp.Model(cfg, 1, params=params)
    nl = dp.NeighborList(m, coord, typ, box)
    E, Ei, F, W = nl.compute(coord, box, "fp8")
    Eb, _, Fb, _ = nl.compute(coord, box, "bf16")
    Er, Eir, Fr, Wr = orc.Model(cfg, params).compute(coord, typ, box)
    f8 = np.sqrt(((F - Fr) ** 2).sum(1).mean()) / rms(Fr)
    fb = np.sqrt(((Fb - Fr) ** 2).sum(1).mean()) / rms(Fr)
    e8 = abs(E - Er) / np.abs(Eir).sum()
    print(name, cfg.embed, "fp8 force", f8, "bf16 force", fb, "fp8 energy", e8)
    assert np.isfinite(F).all() and np.isfinite(E)
    assert f8 < 2 * u8 and e8 < u8 / 4
    assert np.abs(W - Wr).max() / np.abs(Wr).max() < 2 * u8


def test_wide_nets_other_precisions_are_rejected(dp):
    cfg = dpsynth.ModelConfig(ntypes=1, rcut=4.0, rcut_smth=1.0, sel=(32,), embed=(64, 128, 256))
    coord, typ, box = dpsynth.copper_fcc(3, ncell=3)
    m = dp.Model(cfg, 1)
    nl = dp.NeighborList(m, coord, typ, box)
    for prec in ("fp64", "mix32", "fp16", "bf16x3"):
        with pytest.raises(dp.DPError, match="DP_ERR_UNSUPPORTED"):
            nl.compute(coord, box, prec)
    with pytest.raises(dp.DPError, match="DP_ERR_UNSUPPORTED"):
        nl.compute(coord, box, "fp8")   # e4m3 K chunks of 128: w >= 128
    # and FP8 is for the wide nets only
    cfg2 = dpsynth.copper_config()
    c2, t2, b2 = dpsynth.copper_fcc(1, ncell=5)
    m2 = dp.Model(cfg2, 1)
    nl2 = dp.NeighborList(m2, c2, t2, b2)
    with pytest.raises(dp.DPError, match="DP_ERR_UNSUPPORTED"):
        nl2.compute(c2, b2, "fp8")


def test_wide_md_runs(dp):
    cfg = dpsynth.ModelConfig(ntypes=1, rcut=8.0, rcut_smth=2.0, sel=(512,), embed=(128, 256, 512))
    coord, typ, box = dpsynth.copper_fcc(1, ncell=5)
    mass = np.array([dpsynth.MASS["Cu"]])
    vel = dpsynth.velocities(mass[typ], 300.0, 1)
    m = dp.Model(cfg, 1)
    st = dp.MDState(m, coord, vel, typ, mass, box, skin=2.0)
    th = st.step(6, 1.0, "bf16", thermo_every=3)
    assert np.isfinite(th).all()
