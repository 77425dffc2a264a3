"""DeepPot-SE energy / force / virial engine for one GB300 (sm_103a).

The computation lives in the CUDA library ``libdp`` (C-ABI in
``include/dp.h``); this package holds its build step and a thin ctypes
binding with the same entry-point names, plus small owning wrappers.
"""
from __future__ import annotations

import atexit
import weakref

import numpy as np

from . import _lib
from ._lib import (DP_FP64, DP_MIX32, DP_MIX_BF16, DP_MIX_FP16, DPError, EXPORTS, load,  # noqa: F401
                   dp_compute, dp_compute_dev, dp_md_state_create, dp_md_state_destroy, dp_md_state_get,
                   dp_md_step, dp_md_state_save, dp_md_state_load, dp_model_create, dp_model_destroy, dp_model_get_params, dp_model_n_params,
                   dp_model_set_params, dp_model_set_stream, dp_model_set_deterministic, dp_nlist_build, dp_nlist_destroy, dp_nlist_get,
                   dp_nlist_update, dp_profile_enable, dp_profile_group_name, dp_profile_read, dp_profile_select,
                   dp_nlist_update_dev, dp_param_grad, dp_force_loss_grad, dp_force_loss_grad_dev, dp_adam_step,
                   dp_model_sync_params, dp_md_step_judged, dp_nlist_format_noalloc, dp_tanh_f64_dev,
                   dp_nlist_build_frames, dp_ozaki_dgemm_dev, dp_test_starve_wait,
                   dp_md_set_rebuild_every, dp_nlist_set_centers, dp_halo_select_dev, dp_halo_accumulate_dev,
                   dp_bounds_checked, dp_bounds_read)


def build(force: bool = False, bounds_check: bool = False) -> str:
    from .builder import build as _build
    return _build(force=force, bounds_check=bounds_check)


# Live wrappers, released at interpreter exit in dependency order (MD states, then lists, then
# models) while the library and the CUDA runtime are still intact: the module teardown of the
# interpreter may otherwise destroy a model before the lists that refer to it.
_LIVE = {"state": weakref.WeakSet(), "nlist": weakref.WeakSet(), "model": weakref.WeakSet()}


@atexit.register
def _release_all():
    for kind in ("state", "nlist", "model"):
        for obj in list(_LIVE[kind]):
            try:
                obj.close()
            except Exception:
                pass


class Model:
    """Owning wrapper of a dp_model handle."""

    def __init__(self, cfg, seed: int = 0, params=None, deterministic: bool = False):
        self.cfg = cfg
        self.h = dp_model_create(cfg, seed)
        _LIVE["model"].add(self)
        if params is not None:
            dp_model_set_params(self.h, params)
        if deterministic:
            dp_model_set_deterministic(self.h, True)

    @property
    def params(self):
        return dp_model_get_params(self.h)

    @params.setter
    def params(self, flat):
        dp_model_set_params(self.h, flat)

    def close(self):
        if self.h:
            dp_model_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class NeighborList:
    """Owning wrapper of a dp_nlist handle (skin list + formatted list)."""

    def __init__(self, model: Model, coord, typ, box, skin: float = 0.0, cand_cap: int = 0, rcut=None):
        self.model = model
        self.n = len(typ)
        self.h = dp_nlist_build(model.h, coord, typ, box, model.cfg.rcut if rcut is None else rcut, skin, cand_cap)
        _LIVE["nlist"].add(self)

    @classmethod
    def frames(cls, model: Model, coords, typ, box, skin: float = 0.0, cand_cap: int = 0, rcut=None):
        """One list over independent frames coords [F][n][3] of the same atoms (see dp_nlist_build_frames)."""
        self = cls.__new__(cls)
        self.model = model
        coords = np.asarray(coords, dtype=np.float64)
        self.n = coords.shape[0] * len(typ)
        self.h = dp_nlist_build_frames(model.h, coords, typ, box, model.cfg.rcut if rcut is None else rcut, skin,
                                       cand_cap)
        _LIVE["nlist"].add(self)
        return self

    def update(self, coord, box):
        dp_nlist_update(self.h, coord, box)

    def get(self):
        return dp_nlist_get(self.h, self.n, int(sum(self.model.cfg.sel)))

    def compute(self, coord, box, prec="fp64"):
        return dp_compute(self.model.h, self.h, coord, box, prec)

    def close(self):
        if self.h:
            dp_nlist_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MDState:
    """Owning wrapper of a dp_md_state handle (velocity-Verlet NVE on the device)."""

    def __init__(self, model: Model, coord, vel, typ, mass_by_type, box, skin: float = 2.0, cand_cap: int = 0):
        self.model = model
        self.n = len(typ)
        self.h = dp_md_state_create(model.h, coord, vel, typ, mass_by_type, box, skin, cand_cap)
        _LIVE["state"].add(self)

    def step(self, nsteps: int, dt_fs: float, prec="fp64", thermo_every: int = 0):
        return dp_md_step(self.model.h, self.h, nsteps, dt_fs, prec, thermo_every)

    def get(self):
        return dp_md_state_get(self.h, self.n)

    def rebuild_every(self, every: int):
        """Also rebuild the skin list every `every` steps (0: only the displacement criterion)."""
        dp_md_set_rebuild_every(self.h, every)

    def save(self, path):
        """Checkpoint (coordinates, velocities, forces, step, box, types, masses) to a file."""
        dp_md_state_save(self.h, path)

    @classmethod
    def load(cls, model: Model, path):
        """Resume from a checkpoint written by save()."""
        self = cls.__new__(cls)
        self.model = model
        self.h, self.n = dp_md_state_load(model.h, path)
        _LIVE["state"].add(self)
        return self

    def close(self):
        if self.h:
            dp_md_state_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
