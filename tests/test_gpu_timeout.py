"""Bounded device waits: a wait that runs out is reported, and the library stays usable.

dp_test_starve_wait makes the tensor-core embedding kernel skip the bulk copy
of its weights, so its wait on that copy expires (after a few polls) with
nothing in flight.  The evaluation must return DP_ERR_TIMEOUT; after
restoring normal mode the next evaluation of the same model, and one of a
second model (whose kernels allocate tensor memory again), must match the
oracle within the MIX-16 budget, which shows that the kernel that gave up
freed its tensor memory and left the context intact.
"""
import numpy as np
import pytest

import dpsynth

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -9


@pytest.fixture(scope="module")
def dp():
    import paper_2005_00223_gb300 as pkg
    pkg.load()
    return pkg


def _rel_force_err(F, Fr):
    return np.sqrt(((F - Fr) ** 2).sum(1).mean()) / np.sqrt((Fr ** 2).sum(1).mean())


def test_starved_wait_times_out_and_library_recovers(dp):
    import oracle
    cfg = dpsynth.water_config()
    coord, typ, box = dpsynth.water_box(1)
    params = dpsynth.model_params(cfg, 1)
    _, _, Fr, _ = oracle.Model(cfg, params).compute(coord, typ, box)
    m = dp.Model(cfg, 1, params=params)
    nl = dp.NeighborList(m, coord, typ, box)
    E0, _, F0, _ = nl.compute(coord, box, "bf16")
    assert _rel_force_err(F0, Fr) < 10 * U_BF16
    for polls in (1, 64):
        dp.dp_test_starve_wait(m.h, 1, polls)
        with pytest.raises(dp.DPError) as e:
            nl.compute(coord, box, "bf16")
        assert e.value.status == -6, str(e.value)   # DP_ERR_TIMEOUT
    dp.dp_test_starve_wait(m.h, 0)
    for _ in range(3):   # direct call, then graph capture and replay
        E1, _, F1, _ = nl.compute(coord, box, "bf16")
        assert _rel_force_err(F1, Fr) < 10 * U_BF16
        assert abs(E1 - E0) <= 1e-3 * abs(E0)
    m2 = dp.Model(cfg, 1, params=params)
    nl2 = dp.NeighborList(m2, coord, typ, box)
    _, _, F2, _ = nl2.compute(coord, box, "bf16")
    assert _rel_force_err(F2, Fr) < 10 * U_BF16
    nl2.close()
    m2.close()
    nl.close()
    m.close()


def test_starve_wait_rejects_bad_arguments(dp):
    cfg = dpsynth.water_config()
    m = dp.Model(cfg, 1)
    for which, polls in ((2, 10), (1, 0), (1, 1 << 21)):
        with pytest.raises(dp.DPError):
            dp.dp_test_starve_wait(m.h, which, polls)
    m.close()
