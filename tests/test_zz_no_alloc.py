"""The neighbor-list entry point that allocates no device memory.

Callers that cannot allocate device memory (their memory belongs to another
allocator, or a cudaMalloc / cudaFree must not synchronise the device in the
middle of their work) pass their own input and output buffers; the only
scratch is a static device array inside the library.  These tests call it
through the C-ABI, twice in a row on systems of different size, and check
each list against the list of the allocating path (dp_nlist_build +
dp_nlist_get) and against the oracle's canonical list: the lists are integer
data, so they must be identical.  Further cases cover the branches a caller
can reach: a grid coarsened to fit the static array, cells exactly r_c wide,
an out-of-range type, more neighbors than the per-atom key buffer holds, and
an empty system.
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


def _oracle_list(cfg, coord, typ, box, use_cells=True):
    import oracle
    om = oracle.Model(cfg, dpsynth.model_params(cfg, 1))
    out, ntr, _ = om.nlist(coord, typ, box, use_cells=use_cells)
    return out, ntr


def _noalloc_list(dp, cfg, coord, typ, box):
    import torch
    dev = torch.device("cuda")
    x = torch.tensor(coord, dtype=torch.float64, device=dev)
    t = torch.tensor(typ, dtype=torch.int32, device=dev)
    out = torch.full((len(typ), cfg.nsel), 7, dtype=torch.int32, device=dev)
    ntr = torch.full((1,), 5, dtype=torch.int64, device=dev)
    status = torch.ones(1, dtype=torch.int32, device=dev)
    dp.dp_nlist_format_noalloc(x, t, box, cfg.rcut, cfg.sel, out, ntr, status)
    torch.cuda.synchronize()
    return out.cpu().numpy(), int(ntr.item()), int(status.item())


def test_noalloc_list_matches_allocating_path_twice(dp):
    cases = [
        (dpsynth.copper_config(), *dpsynth.copper_fcc(3, ncell=10)),
        (dpsynth.ModelConfig(ntypes=2, rcut=6.0, rcut_smth=0.5, sel=(20, 40)), *dpsynth.water_box(4)),
    ]
    for cfg, coord, typ, box in cases:
        got, ntr, status = _noalloc_list(dp, cfg, coord, typ, box)
        m = dp.Model(cfg, 1)
        nl = dp.NeighborList(m, coord, typ, box)
        ref, ntr_ref = nl.get()
        assert status == 0
        np.testing.assert_array_equal(got, ref)
        assert ntr == ntr_ref
        orc, ntr_orc = _oracle_list(cfg, coord, typ, box)
        np.testing.assert_array_equal(got, orc)
        assert ntr == ntr_orc
    # the second case truncates (sel 20/40 is below the water box's counts)
    assert ntr > 0


def _lattice_block(nside, a, jitter, offset, L, seed):
    rng = np.random.default_rng(seed)
    g = np.arange(nside) * a
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    x = x + rng.normal(scale=jitter, size=x.shape) + offset
    return np.mod(x, L)


def test_noalloc_coarsened_grid_matches_oracle(dp):
    # 64 A box with r_c 1.5 A: 42^3 cells of r_c exceed the static grid, so the grid is coarsened;
    # the block straddles the periodic boundary in every direction
    L = 64.0
    cfg = dpsynth.ModelConfig(ntypes=1, rcut=1.5, rcut_smth=0.5, sel=(24,))
    coord = _lattice_block(12, 1.1, 0.05, np.array([58.0, 57.0, 59.5]), L, 11)
    typ = np.zeros(len(coord), dtype=np.int32)
    box = np.diag([L, L, L])
    got, ntr, status = _noalloc_list(dp, cfg, coord, typ, box)
    ref, ntr_ref = _oracle_list(cfg, coord, typ, box, use_cells=False)
    assert status == 0
    assert (got >= 0).sum() > 6 * len(coord)
    np.testing.assert_array_equal(got, ref)
    assert ntr == ntr_ref


def test_noalloc_cells_exactly_rcut_wide(dp):
    # L = 4 r_c exactly: pairs placed across every cell boundary of a 4-cell grid at r just below r_c
    rc, L = 3.0, 12.0
    cfg = dpsynth.ModelConfig(ntypes=1, rcut=rc, rcut_smth=0.5, sel=(64,))
    pts = []
    for k in range(1, 5):
        b = k * rc
        for eps in (0.0, 1e-15, 4e-15, 1e-12, 1e-9):
            xb = np.nextafter(b, -np.inf) - eps
            pts.append([np.mod(xb, L), 1.0 + 0.37 * k, 2.0 + 0.11 * k])
            pts.append([np.mod(xb - (rc - 1e-12), L), 1.0 + 0.37 * k, 2.0 + 0.11 * k])
            pts.append([6.5 + 0.21 * k, np.mod(xb, L), 8.0 - 0.13 * k])
            pts.append([6.5 + 0.21 * k, np.mod(xb - (rc - 1e-12), L), 8.0 - 0.13 * k])
    coord = np.array(pts)
    typ = np.zeros(len(coord), dtype=np.int32)
    box = np.diag([L, L, L])
    got, ntr, status = _noalloc_list(dp, cfg, coord, typ, box)
    ref, ntr_ref = _oracle_list(cfg, coord, typ, box, use_cells=False)
    assert status == 0
    np.testing.assert_array_equal(got, ref)
    assert ntr == ntr_ref


def test_noalloc_out_of_range_type_sets_status(dp):
    cfg = dpsynth.water_config()
    coord, typ, box = dpsynth.water_box(2)
    typ = typ.copy()
    typ[7] = cfg.ntypes    # not a type of the model
    got, _, status = _noalloc_list(dp, cfg, coord, typ, box)
    assert status == 1
    assert not (got == 7).any()


def test_noalloc_key_overflow_sets_status(dp):
    # 1 A lattice with r_c 6.9 A: about 1,370 neighbors per atom, above the 1,024 keys an atom may hold
    cfg = dpsynth.ModelConfig(ntypes=1, rcut=6.9, rcut_smth=0.5, sel=(64,))
    L = 14.0
    coord = _lattice_block(14, 1.0, 0.0, np.zeros(3), L, 0)
    typ = np.zeros(len(coord), dtype=np.int32)
    got, _, status = _noalloc_list(dp, cfg, coord, typ, np.diag([L, L, L]))
    assert status == 1
    assert ((got >= -1) & (got < len(coord))).all()


def test_noalloc_empty_system(dp):
    import torch
    cfg = dpsynth.water_config()
    x = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    t = torch.zeros(0, dtype=torch.int32, device="cuda")
    out = torch.zeros((0, cfg.nsel), dtype=torch.int32, device="cuda")
    ntr = torch.full((1,), 3, dtype=torch.int64, device="cuda")
    st = torch.ones(1, dtype=torch.int32, device="cuda")
    dp.dp_nlist_format_noalloc(x, t, np.diag([20.0, 20.0, 20.0]), cfg.rcut, cfg.sel, out, ntr, st)
    torch.cuda.synchronize()
    assert int(ntr.item()) == 0 and int(st.item()) == 0


def test_noalloc_rejects_too_many_atoms(dp):
    import torch
    n = 131073
    x = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    t = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    ntr = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(dp.DPError, match="static scratch limit"):
        dp.dp_nlist_format_noalloc(x, t, np.diag([50.0, 50.0, 50.0]), 4.0, [4], out, ntr, st)


def test_noalloc_binding_rejects_wrong_buffers(dp):
    import torch
    cfg = dpsynth.water_config()
    coord, typ, box = dpsynth.water_box(1)
    n = len(typ)
    x = torch.tensor(coord, dtype=torch.float64, device="cuda")
    t = torch.tensor(typ, dtype=torch.int32, device="cuda")
    out = torch.zeros((n, cfg.nsel), dtype=torch.int32, device="cuda")
    ntr = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    bad = [
        (x.float(), t, out),                      # float32 coordinates
        (x.cpu(), t, out),                        # host tensor
        (x, t, out[:, :-1].contiguous()),         # list too short
        (x, t, out[:, ::2]),                      # non-contiguous view
    ]
    for bx, bt, bo in bad:
        with pytest.raises(ValueError):
            dp.dp_nlist_format_noalloc(bx, bt, box, cfg.rcut, cfg.sel, bo, ntr, st)
