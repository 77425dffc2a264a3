"""Spatial decomposition (Sec. 4.3) on CPU: slab geometry, and decomposed evaluations against the oracle.

The decomposed evaluation (halo out, owned atoms as the only centers, ghost forces back to their owners,
energy and virial summed over ranks) must reproduce the single-domain evaluation of the periodic box:
DP's energy is a sum of atomic terms that each see only the atoms within r_c.  The evaluation engine here
is built from the oracle (tests/oracle_engine.py); the ranks run in one process (InProcessTransport) and
as two gloo processes under torch.distributed.run (TorchTransport).
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import dpsynth

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

from oracle_engine import OracleEngine, workload  # noqa: E402


def _domain():
    from paper_2005_00223_gb300 import domain
    return domain


@pytest.mark.parametrize("world", [2, 3, 4])
def test_slab_halos_cover_every_pair_across_faces(world):
    """Every atom within the halo width of a slab face is sent to the neighbor across that face, and
    lands in the neighbor's halo band of its extended frame at the distance it has from the neighbor's
    slab in the periodic box."""
    domain = _domain()
    L = 40.0
    box = np.diag([L, 21.0, 22.0])
    rng = np.random.default_rng(world)
    x = rng.uniform(0, L, size=(400, 3)) * [1.0, 21.0 / L, 22.0 / L]
    h = 6.0
    for r in range(world):
        s = domain.Slab(box, r, world, halo=h, rcut=h)
        for dest, side, lo, hi, shift in s.send_ranges():
            d = domain.Slab(box, dest, world, halo=h, rcut=h)
            sel = (x[:, 0] >= lo) & (x[:, 0] < hi)
            xe = x[sel, 0] + shift                       # in the destination's frame
            if side == "left":
                assert ((xe >= 0) & (xe < h + 1e-9)).all()
            else:
                assert ((xe >= h + d.width - 1e-9) & (xe < 2 * h + d.width + 1e-9)).all()
            # periodic distance to the destination slab equals the distance in its frame
            gap_frame = np.where(side == "left", h - xe, xe - (h + d.width))
            own_lo, own_hi = d.x0, d.x1
            gap_box = np.minimum(np.mod(own_lo - x[sel, 0], L), np.mod(x[sel, 0] - own_hi, L))
            np.testing.assert_allclose(np.maximum(gap_frame, 0), np.maximum(np.minimum(gap_box, h), 0), atol=1e-9)
    owned = [domain.owned_atoms(x, box, r, world) for r in range(world)]
    allidx = np.sort(np.concatenate(owned))
    np.testing.assert_array_equal(allidx, np.arange(len(x)))


def test_slab_rejects_narrow_slabs():
    domain = _domain()
    with pytest.raises(ValueError):
        domain.Slab(np.diag([20.0, 20.0, 20.0]), 0, 4, halo=6.0, rcut=6.0)
    with pytest.raises(ValueError):
        domain.Slab(np.diag([20.0, 20.0, 20.0]), 0, 1, halo=6.0, rcut=6.0)


def _in_process(name, world):
    import torch
    domain = _domain()
    cfg, coord, typ, box = workload(name)
    params = dpsynth.model_params(cfg, 1)
    ranks, owned = [], []
    for r in range(world):
        own = domain.owned_atoms(coord, box, r, world)
        slab = domain.Slab(box, r, world, halo=cfg.rcut, rcut=cfg.rcut)
        x = torch.tensor(np.mod(coord[own], np.diag(box)), dtype=torch.float64)
        t = torch.tensor(typ[own], dtype=torch.int32)
        ranks.append(domain.RankState(OracleEngine(cfg, params), slab, x, t))
        owned.append(own)
    E, W = domain.InProcessTransport(world).evaluate(ranks)
    F = np.zeros((len(typ), 3))
    for own, r in zip(owned, ranks):
        F[own] = r.F.numpy()
    return cfg, coord, typ, box, params, E, F, W


def _check_against_oracle(cfg, coord, typ, box, params, E, F, W):
    import oracle
    Er, _, Fr, Wr = oracle.Model(cfg, params).compute(coord, typ, box)
    frms = np.sqrt((Fr ** 2).sum(1).mean())
    assert abs(E - Er) <= 1e-10 * abs(Er), (E, Er)
    assert np.sqrt(((F - Fr) ** 2).sum(1)).max() <= 1e-10 * frms
    assert np.abs(np.asarray(W) - Wr).max() <= 1e-10 * np.abs(Wr).max()


@pytest.mark.parametrize("name", ["water192", "cu500"])
def test_in_process_decomposition_matches_oracle(name):
    _check_against_oracle(*_in_process(name, 2))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.timeout(600)
def test_gloo_two_ranks_match_oracle():
    pytest.importorskip("torch")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(HERE, "domain_ranks.py"), "cu500"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=os.path.dirname(HERE), env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    out = json.loads(lines[0])
    assert out["world"] == 2
    cfg, coord, typ, box = workload("cu500")
    _check_against_oracle(cfg, coord, typ, box, dpsynth.model_params(cfg, 1), out["E"], np.array(out["F"]),
                          np.array(out["W"]))
