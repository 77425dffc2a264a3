"""Shared helpers of the GPU parity tests (inputs from dpsynth, expected values from the oracle)."""
import numpy as np

import dpsynth


def systems():
    """(name, cfg, coord, type, box) of the parity workloads, small enough for the oracle."""
    out = []
    cfg = dpsynth.water_config()
    c, t, b = dpsynth.water_box(1)
    out.append(("water192", cfg, c, t, b))
    cfg = dpsynth.copper_config()
    c, t, b = dpsynth.copper_fcc(1, ncell=5)
    out.append(("cu500", cfg, c, t, b))
    return out


def rms(F):
    return float(np.sqrt((F ** 2).sum(1).mean()))


def assert_close_fp64(gpu, ref, rtol=1e-10):
    """E, E_i, F, W within rtol relative (norm-wise for vectors, against the oracle's scale)."""
    E, Ei, F, W = gpu
    Er, Eir, Fr, Wr = ref
    assert abs(E - Er) <= rtol * abs(Er), (E, Er)
    escale = max(np.abs(Eir).max(), 1e-300)
    assert np.abs(Ei - Eir).max() <= rtol * escale, np.abs(Ei - Eir).max() / escale
    fs = rms(Fr)
    err = np.sqrt(((F - Fr) ** 2).sum(1)).max()
    assert err <= rtol * fs, err / fs
    assert np.abs(W - Wr).max() <= rtol * np.abs(Wr).max(), np.abs(W - Wr).max() / np.abs(Wr).max()


def sampled_oracle_force(om, coord, typ, box, nl_ref, k):
    """E_k and F_k = sum_s g_k,s - sum over atoms i with k in their list of g_i,slot(k), from the oracle."""
    Ek, gk, _ = om.atom(k, nl_ref[k], coord, typ, box)
    F = gk[nl_ref[k] >= 0].sum(0)
    for i in np.unique(np.where(nl_ref == k)[0]):
        _, gi, _ = om.atom(i, nl_ref[i], coord, typ, box)
        F -= gi[nl_ref[i] == k].sum(0)
    return Ek, F
