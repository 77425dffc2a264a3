"""The neighbor-list entry point that allocates no device memory.

Callers that cannot allocate device memory (their memory belongs to another
allocator, or a cudaMalloc / cudaFree must not synchronise the device in the
middle of their work) pass their own input and output buffers; the only
scratch is a static device array inside the library.  This test calls it
through the C-ABI twice in a row, on two systems of different size, and
checks each list against the list of the allocating path (dp_nlist_build +
dp_nlist_get): the lists are integer data, so they must be identical.
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


def _noalloc_list(dp, cfg, coord, typ, box):
    import torch
    dev = torch.device("cuda")
    x = torch.tensor(coord, dtype=torch.float64, device=dev)
    t = torch.tensor(typ, dtype=torch.int32, device=dev)
    out = torch.full((len(typ), cfg.nsel), 7, dtype=torch.int32, device=dev)
    ntr = torch.zeros(1, dtype=torch.int64, device=dev)
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
    # the second case truncates (sel 20/40 is below the water box's counts)
    assert ntr > 0


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
