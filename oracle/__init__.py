"""FP64 CPU oracle for the DeepPot-SE energy/force/virial path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never calls it.

The arithmetic lives in ``dp_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module compiles it with gcc on first use and
marshals numpy arrays to it.  It imports nothing from the CUDA library.

Every function below states the section of the paper it follows.  Parity
of the absolute energy of a seeded model is unpinned (the paper prints no
values for it); the pins are the closed forms, invariants, finite
differences and brute-force checks in the tests.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile dp_oracle.c into _build/liboracle.so (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Model(C.Structure):
    _fields_ = [("ntypes", C.c_int32), ("rcut", C.c_double), ("rcut_smth", C.c_double),
                ("sel", C.POINTER(C.c_int32)), ("n_embed", C.c_int32),
                ("embed", C.POINTER(C.c_int32)), ("m2", C.c_int32), ("n_fit", C.c_int32),
                ("fit", C.POINTER(C.c_int32)), ("params", C.POINTER(C.c_double))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            lib.orc_n_params.argtypes = [P]
            lib.orc_n_params.restype = C.c_int64
            lib.orc_nlist.argtypes = [P, C.c_int64, P, P, P, C.c_int, P, P, P]
            lib.orc_nlist.restype = C.c_int
            lib.orc_switch.argtypes = [C.c_double, C.c_double, C.c_double, P]
            lib.orc_switch.restype = C.c_double
            lib.orc_env_row.argtypes = [P, C.c_double, C.c_double, P, P]
            lib.orc_env_row.restype = None
            lib.orc_atom.argtypes = [P, C.c_int64, P, P, P, P, P, P, P]
            lib.orc_atom.restype = C.c_int
            lib.orc_compute.argtypes = [P, C.c_int64, P, P, P, P, P, P, P, P, C.c_int]
            lib.orc_compute.restype = C.c_int
            lib.orc_md_nve.argtypes = [P, C.c_int64, P, P, P, P, P, C.c_int64, C.c_double, C.c_int32,
                                       P, C.c_int]
            lib.orc_md_nve.restype = C.c_int
            lib.orc_jvp_grad.argtypes = [P, C.c_int64, P, P, P, P, P, C.c_double, C.c_double, P, P, P, C.c_int]
            lib.orc_jvp_grad.restype = C.c_int
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class OracleError(RuntimeError):
    pass


def _check(st: int, what: str):
    if st != 0:
        raise OracleError(f"{what} failed with status {st}")


class Model:
    """Oracle view of a model: hyper-parameters plus a flat FP64 parameter vector."""

    def __init__(self, cfg, params: np.ndarray):
        self.cfg = cfg
        self.params = np.ascontiguousarray(params, dtype=np.float64)
        self._sel = np.ascontiguousarray(cfg.sel, dtype=np.int32)
        self._embed = np.ascontiguousarray(cfg.embed, dtype=np.int32)
        self._fit = np.ascontiguousarray(cfg.fit, dtype=np.int32)
        self._s = _Model(cfg.ntypes, float(cfg.rcut), float(cfg.rcut_smth),
                         self._sel.ctypes.data_as(C.POINTER(C.c_int32)), len(cfg.embed),
                         self._embed.ctypes.data_as(C.POINTER(C.c_int32)), int(cfg.m2), len(cfg.fit),
                         self._fit.ctypes.data_as(C.POINTER(C.c_int32)),
                         self.params.ctypes.data_as(C.POINTER(C.c_double)))
        lib = _load()
        n = lib.orc_n_params(C.byref(self._s))
        if n != self.params.size:
            raise OracleError(f"parameter vector has {self.params.size} entries, model needs {n}")

    @property
    def ref(self):
        return C.cast(C.byref(self._s), C.c_void_p)

    # -- neighbor list (Sec. 4.1.1, 4.1.2) ---------------------------------
    def nlist(self, coord, typ, box, use_cells: bool = True):
        """Canonical formatted list [n][sum(sel)] (-1 padded), n_truncated, counts[n][ntypes]."""
        coord = np.ascontiguousarray(coord, dtype=np.float64)
        typ = np.ascontiguousarray(typ, dtype=np.int32)
        box = np.ascontiguousarray(box, dtype=np.float64).reshape(3, 3)
        n = coord.shape[0]
        out = np.empty((n, self.cfg.nsel), dtype=np.int32)
        cnt = np.empty((n, self.cfg.ntypes), dtype=np.int32)
        ntr = np.zeros(1, dtype=np.int64)
        _check(_load().orc_nlist(self.ref, n, _p(coord), _p(typ), _p(box), int(use_cells), _p(out),
                                 _p(ntr), _p(cnt)), "orc_nlist")
        return out, int(ntr[0]), cnt

    # -- energy, forces, virial (Sec. 2, Fig. 1) ---------------------------
    def compute(self, coord, typ, box, nlist=None, nthreads: int = 0):
        """E, E_i[n], F[n,3], W[3,3] of the whole system (FP64)."""
        coord = np.ascontiguousarray(coord, dtype=np.float64)
        typ = np.ascontiguousarray(typ, dtype=np.int32)
        box = np.ascontiguousarray(box, dtype=np.float64).reshape(3, 3)
        if nlist is None:
            nlist = self.nlist(coord, typ, box)[0]
        nlist = np.ascontiguousarray(nlist, dtype=np.int32)
        n = coord.shape[0]
        E = np.zeros(1)
        Ei = np.empty(n)
        F = np.empty((n, 3))
        W = np.empty(9)
        _check(_load().orc_compute(self.ref, n, _p(coord), _p(typ), _p(box), _p(nlist), _p(E), _p(Ei),
                                   _p(F), _p(W), int(nthreads)), "orc_compute")
        return float(E[0]), Ei, F, W.reshape(3, 3)

    def energy(self, coord, typ, box, nthreads: int = 0) -> float:
        coord = np.ascontiguousarray(coord, dtype=np.float64)
        typ = np.ascontiguousarray(typ, dtype=np.int32)
        box = np.ascontiguousarray(box, dtype=np.float64).reshape(3, 3)
        nl = self.nlist(coord, typ, box)[0]
        E = np.zeros(1)
        _check(_load().orc_compute(self.ref, coord.shape[0], _p(coord), _p(typ), _p(box), _p(nl), _p(E),
                                   None, None, None, int(nthreads)), "orc_compute")
        return float(E[0])

    def atom(self, i: int, row, coord, typ, box):
        """E_i, g[sum(sel),3] = dE_i/dd_ij per slot, and D_i [M1*M2] of one atom."""
        row = np.ascontiguousarray(row, dtype=np.int32)
        coord = np.ascontiguousarray(coord, dtype=np.float64)
        typ = np.ascontiguousarray(typ, dtype=np.int32)
        box = np.ascontiguousarray(box, dtype=np.float64).reshape(3, 3)
        Ei = np.zeros(1)
        g = np.empty((self.cfg.nsel, 3))
        D = np.empty(self.cfg.m1 * self.cfg.m2)
        _check(_load().orc_atom(self.ref, int(i), _p(row), _p(coord), _p(typ), _p(box), _p(Ei), _p(g),
                                _p(D)), "orc_atom")
        return float(Ei[0]), g, D

    # -- parameter gradient of the force-matching loss ---------------------
    def jvp_grad(self, coord, typ, box, v, alpha: float, beta: float, nlist=None, nthreads: int = 0):
        """(E, Edot, grad) with Edot = sum_k v_k . dE/dr_k and grad = d(alpha E + beta Edot)/dtheta."""
        coord = np.ascontiguousarray(coord, dtype=np.float64)
        typ = np.ascontiguousarray(typ, dtype=np.int32)
        box = np.ascontiguousarray(box, dtype=np.float64).reshape(3, 3)
        v = np.ascontiguousarray(v, dtype=np.float64)
        if nlist is None:
            nlist = self.nlist(coord, typ, box)[0]
        nlist = np.ascontiguousarray(nlist, dtype=np.int32)
        E, Ed = np.zeros(1), np.zeros(1)
        grad = np.zeros(self.params.size)
        _check(_load().orc_jvp_grad(self.ref, coord.shape[0], _p(coord), _p(typ), _p(box), _p(nlist), _p(v),
                                    float(alpha), float(beta), _p(E), _p(Ed), _p(grad), int(nthreads)),
               "orc_jvp_grad")
        return float(E[0]), float(Ed[0]), grad

    def force_loss(self, frames, p_e: float = 0.0, p_f: float = 1.0):
        """L = sum over frames of p_e (dE/N)^2 + p_f/(3N) sum_k |F_k - F_ref,k|^2.

        frames: list of (coord, type, box, E_ref, F_ref)."""
        total = 0.0
        for coord, typ, box, E_ref, F_ref in frames:
            E, _, F, _ = self.compute(coord, typ, box)
            n = len(typ)
            total += p_e * ((E - E_ref) / n) ** 2 + p_f * float(((F - F_ref) ** 2).sum()) / (3 * n)
        return total

    def force_loss_grad(self, frames, p_e: float = 0.0, p_f: float = 1.0):
        """(L, dL/dtheta): dL/dtheta = 2 p_e dE/N^2 dE/dtheta - 2 p_f/(3N) dEdot/dtheta, v = F - F_ref."""
        total = 0.0
        grad = np.zeros(self.params.size)
        for coord, typ, box, E_ref, F_ref in frames:
            E, _, F, _ = self.compute(coord, typ, box)
            n = len(typ)
            v = F - F_ref
            total += p_e * ((E - E_ref) / n) ** 2 + p_f * float((v ** 2).sum()) / (3 * n)
            _, _, g = self.jvp_grad(coord, typ, box, v, alpha=2 * p_e * (E - E_ref) / n ** 2,
                                    beta=-2 * p_f / (3 * n))
            grad += g
        return total, grad

    # -- velocity-Verlet NVE (Sec. 5.1) ------------------------------------
    def md_nve(self, coord, vel, typ, mass_by_type, box, nsteps: int, dt: float, thermo_every: int,
               nthreads: int = 0):
        """Run NVE; returns (coord, vel, thermo[nsteps//thermo_every, 4] = KE, PE, T, P)."""
        coord = np.array(coord, dtype=np.float64, order="C", copy=True)
        vel = np.array(vel, dtype=np.float64, order="C", copy=True)
        typ = np.ascontiguousarray(typ, dtype=np.int32)
        mass = np.ascontiguousarray(mass_by_type, dtype=np.float64)
        box = np.ascontiguousarray(box, dtype=np.float64).reshape(3, 3)
        rows = nsteps // thermo_every if thermo_every > 0 else 0
        thermo = np.zeros((max(rows, 1), 4))
        _check(_load().orc_md_nve(self.ref, coord.shape[0], _p(coord), _p(vel), _p(typ), _p(mass), _p(box),
                                  int(nsteps), float(dt), int(thermo_every), _p(thermo), int(nthreads)),
               "orc_md_nve")
        return coord, vel, thermo[:rows]


def switch(r: float, rcs: float, rc: float):
    """s(r) and ds/dr of the smooth switching function (Sec. 2, C2 smoothness)."""
    ds = np.zeros(1)
    s = _load().orc_switch(float(r), float(rcs), float(rc), _p(ds))
    return s, float(ds[0])


def env_row(d, rcs: float, rc: float):
    """Environment-matrix row (s, s dx/r, s dy/r, s dz/r) and its 4x3 Jacobian."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    R = np.empty(4)
    J = np.empty(12)
    _load().orc_env_row(_p(d), float(rcs), float(rc), _p(R), _p(J))
    return R, J.reshape(4, 3)
