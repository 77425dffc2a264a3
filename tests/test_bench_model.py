"""The algorithmic work model and MD protocol of bench.py, against the closed forms they state."""
import os
import sys

import dpsynth

sys.path.insert(0, os.path.join(os.path.dirname(__file__), ".."))
import bench  # noqa: E402


def test_flop_per_neighbor_and_per_atom_closed_forms():
    cfg = dpsynth.copper_config()                      # nets 25-50-100, M2 16, fitting 240-240-240
    nn, n = 1000, 10
    g = bench.flops_per_group(cfg, nn, n)
    # embedding per real neighbor: forward 2 (25 + 25*50 + 50*100 + 4*100), backward
    # 2 (4*100 + 4*100 + 100*50 + 50*25 + 25): 13,350 + 14,150 = 27,500 FLOP
    assert g["embed_fwd"] == nn * 13350 + n * 2 * 4 * 100 * 16
    assert g["embed_bwd"] == nn * 14150 + n * 2 * 8 * 100 * 16
    # fitting per atom: forward and input gradient of 1600*240 + 2*240*240 + 240 multiply-adds
    assert g["fitting"] == n * 4 * (1600 * 240 + 2 * 240 * 240 + 240)
    # the split FP64 route only regroups the same work
    s = bench.flops_per_group(cfg, nn, n, split_route=True)
    assert sum(s.values()) == sum(g.values())
    assert s["embed_fwd_l2"] == nn * 2 * (50 * 100 + 4 * 100)


def test_student_flop_per_neighbor():
    cfg = dpsynth.copper_student_config()              # nets 8-16-32, M2 8, fitting 64-64-64
    g = bench.flops_per_group(cfg, 1, 0)
    assert g["embed_fwd"] + g["embed_bwd"] == 2 * (8 + 128 + 512 + 128) + 2 * (128 + 128 + 512 + 128 + 8)


def test_md_protocols():
    assert bench.md_protocol("cu4000", 50) == (300.0, 50)
    assert bench.md_protocol("water12k", 100) == (330.0, 20)      # the paper's thermo interval and 330 K
    assert bench.md_protocol("water12k", 10) == (330.0, 10)       # fewer steps than one interval


def test_workloads_match_their_descriptions():
    """Atom counts, composition, density and box shape of every bench workload."""
    import numpy as np
    amu_g = 1.66053906660e-24
    for name, n, dens in (("cu4000", 4000, 8.96), ("cu108k", 108000, 8.96), ("water192", 192, 1.0),
                          ("water12k", 12288, 1.0), ("water1p5m", 1572864, 1.0)):
        cfg, coord, typ, box, mass, dt, desc = bench.workload(name)
        assert coord.shape == (n, 3) and typ.shape == (n,)
        assert f"{n} atoms" in desc
        assert np.all(box == np.diag(np.diag(box)))                       # orthorhombic boxes
        frac = coord / np.diag(box)
        assert frac.min() >= 0.0 and frac.max() < 1.0                     # wrapped into the box
        counts = np.bincount(typ, minlength=cfg.ntypes)
        if cfg.ntypes == 2:
            assert counts[1] == 2 * counts[0]                             # H2O
        rho = (counts * mass).sum() * amu_g / (np.prod(np.diag(box)) * 1e-24)
        assert abs(rho - dens) < 0.05 * dens, (name, rho)
        assert dt == (1.0 if cfg.ntypes == 1 else 0.5)
    # the student is the copper model's
    cfg, *_ = bench.workload("cu4000", model="student")
    assert cfg.embed == (8, 16, 32)
