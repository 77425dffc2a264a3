"""Small evaluations of every route through the bounds-checked debug build, each against the oracle.

Run as its own process with DP_LIBRARY=bounds (tests/test_gpu_bounds.py): it loads the library that
checks every neighbor, cell, work-list and type index its kernels read before using it, runs the
FP64 (CUDA cores and split products), MIX-32, BF16, FP16, split-bf16 and wide-net routes, the
force-loss gradient and a short NVE run with list rebuilds, checks each result against the oracle
with the budgets of the other GPU tests, and prints the bounds record, which must be all zeros.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import dpsynth  # noqa: E402
import oracle  # noqa: E402
import paper_2005_00223_gb300 as dp  # noqa: E402
from gpu_common import assert_close_fp64, rms  # noqa: E402


def check_mixed(got, ref, e_tol, f_tol, w_tol):
    """Energy within e_tol of sum |E_i|, force RMSE within f_tol of the RMS force, virial within w_tol."""
    E, Ei, F, W = got
    Er, Eir, Fr, Wr = ref
    assert abs(E - Er) <= e_tol * np.abs(Eir).sum(), (E, Er)
    assert np.sqrt(((F - Fr) ** 2).sum(1).mean()) <= f_tol * rms(Fr)
    assert np.abs(W - Wr).max() <= w_tol * np.abs(Wr).max()


def check_u(got, ref, u, fmult=10.0):
    """The MIX-16 budgets of the other GPU tests in units of the operands' unit roundoff u."""
    check_mixed(got, ref, 2 * u, fmult * u, 10 * u)


def main():
    assert os.environ.get("DP_LIBRARY") == "bounds"
    dp.load()
    assert dp.dp_bounds_checked(), "the bounds-checked build was not loaded"
    dp.dp_bounds_read(clear=True)
    oracle.build()
    done = []
    systems = [("water192", dpsynth.water_config(), *dpsynth.water_box(1)),
               ("cu500", dpsynth.copper_config(), *dpsynth.copper_fcc(1, ncell=5))]
    for name, cfg, c, t, b in systems:
        params = dpsynth.model_params(cfg, 1)
        ref = oracle.Model(cfg, params).compute(c, t, b)
        m = dp.Model(cfg, 1, params=params)
        nl = dp.NeighborList(m, c, t, b, skin=1.0)
        assert_close_fp64(nl.compute(c, b, "fp64"), ref)
        os.environ["DP_OZ_MIN_ATOMS"] = "0"     # the split-product FP64 route
        try:
            assert_close_fp64(nl.compute(c, b, "fp64"), ref)
        finally:
            del os.environ["DP_OZ_MIN_ATOMS"]
        check_mixed(nl.compute(c, b, "mix32"), ref, 1e-6, 1e-5, 1e-5)
        check_u(nl.compute(c, b, "bf16"), ref, 2.0 ** -9)
        check_u(nl.compute(c, b, "fp16"), ref, 2.0 ** -11)
        check_u(nl.compute(c, b, "bf16x3"), ref, 2.0 ** -16)
        nl.close()
        m.close()
        done.append(name)
    # wide embedding net (layer-wise tensor-core GEMMs)
    cfg = dpsynth.ModelConfig(ntypes=1, rcut=4.0, rcut_smth=1.0, sel=(48,), embed=(64, 128, 256))
    c, t, b = dpsynth.copper_fcc(3, ncell=3)
    c = c + np.random.default_rng(17).normal(scale=0.3, size=c.shape)
    params = dpsynth.model_params(cfg, 4)
    ref = oracle.Model(cfg, params).compute(c, t, b)
    m = dp.Model(cfg, 1, params=params)
    nl = dp.NeighborList(m, c, t, b)
    check_u(nl.compute(c, b, "bf16"), ref, 2.0 ** -9, fmult=20.0)
    nl.close()
    m.close()
    done.append("wide64")
    # force-loss parameter gradient (FP64) against the oracle's
    cfg = dpsynth.water_config()
    c, t, b = dpsynth.water_box(2)
    params = dpsynth.model_params(cfg, 3)
    rng = np.random.default_rng(5)
    Fref = rng.normal(scale=1e-3, size=c.shape)
    m = dp.Model(cfg, 1, params=params)
    nl = dp.NeighborList(m, c, t, b)
    loss, g = dp.dp_force_loss_grad(m.h, nl.h, c, b, Fref, 0.5, 1.0, 100.0, "fp64")
    lref, gref = oracle.Model(cfg, params).force_loss_grad([(c, t, b, 0.5, Fref)], p_e=1.0, p_f=100.0)
    assert abs(loss - lref) <= 1e-10 * abs(lref)
    assert np.linalg.norm(g - gref) <= 1e-9 * np.linalg.norm(gref)
    nl.close()
    m.close()
    done.append("grad")
    # NVE with device rebuilds of the skin list (cell grid, candidates, formatting)
    cfg = dpsynth.copper_config()
    c, t, b = dpsynth.copper_fcc(2, ncell=5)
    mass = np.array([dpsynth.MASS["Cu"]])
    v = dpsynth.velocities(mass[t], 3000.0, 2)
    m = dp.Model(cfg, 1, params=dpsynth.model_params(cfg, 1))
    st = dp.MDState(m, c, v, t, mass, b, skin=0.05)
    st.step(40, 1.0, "bf16")
    x, _, _, _ = st.get()
    st.close()
    m.close()
    assert np.isfinite(x).all()
    done.append("md")
    rec = dp.dp_bounds_read(clear=True)
    print(json.dumps({"cases": done, "bounds": list(rec)}))
    return 0 if rec[0] == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
