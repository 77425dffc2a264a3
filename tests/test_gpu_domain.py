"""Spatial decomposition (Sec. 4.3) on the GPU: libdp's ghost atoms, halo kernels and decomposed evaluation.

One GPU stands in for the ranks (InProcessTransport: the phases of every rank in turn, exchanges as
array hand-overs; no collective kernels that wait on one another).  Expected values come from the
oracle's single-domain evaluation of the periodic box.
"""
import numpy as np
import pytest

import dpsynth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    import paper_2005_00223_gb300 as pkg
    pkg.load()
    return pkg


def test_halo_select_and_accumulate_kernels(dp):
    import torch
    rng = np.random.default_rng(3)
    n = 5000
    x = rng.uniform(0, 30.0, size=(n, 3))
    t = rng.integers(0, 2, size=n).astype(np.int32)
    dx, dt = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    xs = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    ts = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    dp.dp_halo_select_dev(dx, dt, 7.5, 13.25, -4.0, idx, xs, ts, cnt)
    torch.cuda.synchronize()
    k = int(cnt.item())
    ref = np.nonzero((x[:, 0] >= 7.5) & (x[:, 0] < 13.25))[0]
    assert k == len(ref)
    np.testing.assert_array_equal(idx[:k].cpu().numpy(), ref)          # index order
    np.testing.assert_array_equal(xs[:k].cpu().numpy(), x[ref] + [-4.0, 0.0, 0.0])
    np.testing.assert_array_equal(ts[:k].cpu().numpy(), t[ref])
    # a capacity below the count: the count is still reported, nothing beyond cap is written
    small = torch.full((8,), -7, dtype=torch.int32, device="cuda")
    dp.dp_halo_select_dev(dx, dt, 7.5, 13.25, 0.0, small[:5], xs, ts, cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) == len(ref) and (small[5:].cpu().numpy() == -7).all()
    F = torch.tensor(rng.normal(size=(n, 3)), device="cuda")
    F0 = F.cpu().numpy().copy()
    sel = torch.tensor(ref[::3].astype(np.int32), device="cuda")
    g = torch.tensor(rng.normal(size=(len(ref[::3]), 3)), device="cuda")
    dp.dp_halo_accumulate_dev(sel, g, F)
    torch.cuda.synchronize()
    F0[ref[::3]] += g.cpu().numpy()
    np.testing.assert_array_equal(F.cpu().numpy(), F0)


def test_ghost_atoms_are_not_centers(dp, orc):
    """With the second half of the atoms as ghosts: E is the sum of the first half's E_i, ghosts carry
    E_i = 0, and the forces are those of the first half's pair terms only."""
    cfg = dpsynth.water_config()
    coord, typ, box = dpsynth.water_box(2)
    params = dpsynth.model_params(cfg, 1)
    om = orc.Model(cfg, params)
    Er, Eir, _, _ = om.compute(coord, typ, box)
    n, nc = len(typ), len(typ) // 2
    nl_ref, _, _ = om.nlist(coord, typ, box)
    Fr = np.zeros((n, 3))
    for i in range(nc):
        _, g, _ = om.atom(i, nl_ref[i], coord, typ, box)
        ok = nl_ref[i] >= 0
        Fr[i] += g[ok].sum(0)
        np.subtract.at(Fr, nl_ref[i][ok], g[ok])
    m = dp.Model(cfg, 1, params=params)
    nl = dp.NeighborList(m, coord, typ, box)
    dp.dp_nlist_set_centers(nl.h, nc)
    for prec, tol in (("fp64", 1e-10), ("bf16x3", 1e-3)):
        E, Ei, F, W = nl.compute(coord, box, prec)
        assert abs(E - Eir[:nc].sum()) <= tol * np.abs(Eir[:nc]).sum()
        assert (Ei[nc:] == 0).all()
        frms = np.sqrt((Fr ** 2).sum(1).mean())
        assert np.sqrt(((F - Fr) ** 2).sum(1)).max() <= tol * frms * (1 if prec == "fp64" else 10)
    lst, _ = nl.get()
    assert (lst[nc:] == -1).all() and (lst[:nc] >= 0).any()
    dp.dp_nlist_set_centers(nl.h, n)
    E, _, _, _ = nl.compute(coord, box, "fp64")
    assert abs(E - Er) <= 1e-10 * abs(Er)
    with pytest.raises(dp.DPError):
        dp.dp_nlist_set_centers(nl.h, n + 1)


@pytest.mark.parametrize("world", [2, 3])
def test_decomposed_evaluation_matches_oracle(dp, orc, world):
    import torch

    from paper_2005_00223_gb300 import domain
    cfg = dpsynth.copper_config()
    coord, typ, box = dpsynth.copper_fcc(2, ncell=10)
    params = dpsynth.model_params(cfg, 1)
    Er, _, Fr, Wr = orc.Model(cfg, params).compute(coord, typ, box)
    m = dp.Model(cfg, 1, params=params)
    ranks, owned, engines = [], [], []
    for r in range(world):
        own = domain.owned_atoms(coord, box, r, world)
        slab = domain.Slab(box, r, world, halo=cfg.rcut, rcut=cfg.rcut)
        x = torch.tensor(np.mod(coord[own], np.diag(box)), dtype=torch.float64, device="cuda")
        t = torch.tensor(typ[own], dtype=torch.int32, device="cuda")
        eng = domain.LibdpEngine(m, "fp64")
        engines.append(eng)
        ranks.append(domain.RankState(eng, slab, x, t))
        owned.append(own)
    E, W = domain.InProcessTransport(world).evaluate(ranks)
    F = np.zeros_like(Fr)
    for own, r in zip(owned, ranks):
        F[own] = r.F.cpu().numpy()
    frms = np.sqrt((Fr ** 2).sum(1).mean())
    assert abs(E - Er) <= 1e-10 * abs(Er)
    assert np.sqrt(((F - Fr) ** 2).sum(1)).max() <= 1e-10 * frms
    assert np.abs(W - Wr).max() <= 1e-10 * np.abs(Wr).max()
    for e in engines:
        e.close()
