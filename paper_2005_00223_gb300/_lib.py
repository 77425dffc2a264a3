"""ctypes binding of libdp (include/dp.h): the same entry points, argument marshalling only.

Every function here converts Python / numpy / torch arguments to the
C-ABI's plain pointers and sizes, calls the entry point of the same name
and turns a non-OK status into a DPError.  No step of the computation runs
in Python.  The shared library must have been built (``build()``); loading
fails loudly otherwise — there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdp.so")
# The bounds-checked debug build (build(bounds_check=True)); a process selects it by setting
# DP_LIBRARY=bounds before its first load().
BOUNDS_LIB_PATH = os.path.join(_HERE, "_build_bounds", "libdp.so")

DP_OK = 0
STATUS = {0: "DP_OK", -1: "DP_ERR_ARG", -2: "DP_ERR_CUDA", -3: "DP_ERR_OOM", -4: "DP_ERR_BOX",
          -5: "DP_ERR_CAPACITY", -6: "DP_ERR_TIMEOUT", -7: "DP_ERR_NONFINITE", -8: "DP_ERR_UNSUPPORTED"}
DP_FP64, DP_MIX32, DP_MIX_BF16, DP_MIX_FP16, DP_MIX_BF16X3, DP_MIX_FP8 = 0, 1, 2, 3, 4, 5
PRECISION = {"fp64": DP_FP64, "mix32": DP_MIX32, "bf16": DP_MIX_BF16, "fp16": DP_MIX_FP16, "bf16x3": DP_MIX_BF16X3,
             "fp8": DP_MIX_FP8}

# Every entry point declared in include/dp.h.
EXPORTS = [
    "dp_status_string", "dp_last_error", "dp_model_create", "dp_model_n_params", "dp_model_get_params",
    "dp_model_set_params", "dp_model_destroy", "dp_model_set_stream", "dp_model_set_deterministic", "dp_profile_enable", "dp_profile_select", "dp_profile_read",
    "dp_profile_group_name", "dp_nlist_build", "dp_nlist_update", "dp_nlist_get",
    "dp_nlist_destroy", "dp_nlist_update_dev", "dp_compute", "dp_compute_dev", "dp_md_state_create",
    "dp_md_step", "dp_md_state_get", "dp_md_state_save", "dp_md_state_load", "dp_md_state_destroy", "dp_param_grad", "dp_force_loss_grad",
    "dp_force_loss_grad_dev", "dp_adam_step", "dp_model_sync_params", "dp_md_step_judged",
    "dp_nlist_format_noalloc", "dp_tanh_f64_dev", "dp_nlist_build_frames", "dp_ozaki_dgemm_dev",
    "dp_test_starve_wait", "dp_md_set_rebuild_every", "dp_nlist_set_centers", "dp_halo_select_dev",
    "dp_halo_accumulate_dev", "dp_bounds_checked", "dp_bounds_read",
]


class DPError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {message}")
        self.status = status


class _Config(C.Structure):
    _fields_ = [("ntypes", C.c_int32), ("rcut", C.c_double), ("rcut_smth", C.c_double),
                ("sel", C.POINTER(C.c_int32)), ("n_embed", C.c_int32), ("embed", C.POINTER(C.c_int32)),
                ("axis_neuron", C.c_int32), ("n_fit", C.c_int32), ("fit", C.POINTER(C.c_int32))]


_lock = threading.Lock()
_lib = None


def load(path: str = None):
    """Load libdp.so (the bounds-checked build when DP_LIBRARY=bounds); raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if path is None:
            path = BOUNDS_LIB_PATH if os.environ.get("DP_LIBRARY") == "bounds" else LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(f"libdp is not built ({path} missing): run paper_2005_00223_gb300.build()")
        lib = C.CDLL(path)
        P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        sig = {
            "dp_status_string": ([C.c_int], C.c_char_p),
            "dp_last_error": ([], C.c_char_p),
            "dp_model_create": ([P, C.c_uint64, P], C.c_int),
            "dp_model_n_params": ([P, P], C.c_int),
            "dp_model_get_params": ([P, P, I64], C.c_int),
            "dp_model_set_params": ([P, P, I64], C.c_int),
            "dp_model_destroy": ([P], None),
            "dp_model_set_stream": ([P, P], C.c_int),
            "dp_model_set_deterministic": ([P, I32], C.c_int),
            "dp_profile_enable": ([P, I32], C.c_int),
            "dp_profile_select": ([P, C.c_uint32], C.c_int),
            "dp_profile_read": ([P, I32, P, P], C.c_int),
            "dp_profile_group_name": ([I32], C.c_char_p),
            "dp_nlist_build": ([P, I64, P, P, P, D, D, I32, P], C.c_int),
            "dp_nlist_update": ([P, P, P], C.c_int),
            "dp_nlist_get": ([P, P, P], C.c_int),
            "dp_nlist_destroy": ([P], None),
            "dp_nlist_update_dev": ([P, P, P], C.c_int),
            "dp_nlist_format_noalloc": ([I64, P, P, P, D, I32, P, P, P, P, P], C.c_int),
            "dp_tanh_f64_dev": ([I64, P, P, P], C.c_int),
            "dp_nlist_build_frames": ([P, I32, I64, P, P, P, D, D, I32, P], C.c_int),
            "dp_ozaki_dgemm_dev": ([P, I64, I32, I32, P, P, P, P], C.c_int),
            "dp_test_starve_wait": ([P, I32, I64], C.c_int),
            "dp_bounds_checked": ([], C.c_int32),
            "dp_bounds_read": ([P, I32], C.c_int),
            "dp_md_set_rebuild_every": ([P, I32], C.c_int),
            "dp_nlist_set_centers": ([P, I64], C.c_int),
            "dp_halo_select_dev": ([I64, P, P, D, D, D, I64, P, P, P, P, P], C.c_int),
            "dp_halo_accumulate_dev": ([I64, P, P, P, P], C.c_int),
            "dp_param_grad": ([P, P, P, P, P, D, D, C.c_int, P, P, P], C.c_int),
            "dp_force_loss_grad": ([P, P, P, P, P, D, D, D, C.c_int, P, P], C.c_int),
            "dp_force_loss_grad_dev": ([P, P, P, P, P, P, D, D, C.c_int, P, P, P], C.c_int),
            "dp_adam_step": ([P, P, D, D, D, D, I64, P], C.c_int),
            "dp_model_sync_params": ([P], C.c_int),
            "dp_compute": ([P, P, P, P, C.c_int, P, P, P, P], C.c_int),
            "dp_compute_dev": ([P, P, P, P, C.c_int, P, P, P, P, P], C.c_int),
            "dp_md_state_create": ([P, I64, P, P, P, P, P, D, I32, P], C.c_int),
            "dp_md_step": ([P, P, I64, D, C.c_int, I32, P], C.c_int),
            "dp_md_state_get": ([P, P, P, P, P], C.c_int),
            "dp_md_state_save": ([P, C.c_char_p], C.c_int),
            "dp_md_state_load": ([P, C.c_char_p, P], C.c_int),
            "dp_md_step_judged": ([P, P, P, I64, D, C.c_int, C.c_int, I32, D, P, P], C.c_int),
            "dp_md_state_destroy": ([P], None),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def _check(st: int, where: str):
    if st != DP_OK:
        raise DPError(st, where, load().dp_last_error().decode())


def _ptr(a):
    """Address of a numpy array or a torch tensor (device or host); None -> NULL."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p)
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    raise TypeError(f"unsupported array type {type(a)}")


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(shape) if shape is not None else a


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _box(box):
    return _f64(box).reshape(9).copy()


def _prec(p):
    return PRECISION[p] if isinstance(p, str) else int(p)


# ------------------------------------------------------------------ model

def dp_model_create(cfg, seed: int):
    """cfg: any object with ntypes, rcut, rcut_smth, sel, embed, m2, fit."""
    lib = load()
    sel, emb, fit = _i32(cfg.sel), _i32(cfg.embed), _i32(cfg.fit)
    c = _Config(int(cfg.ntypes), float(cfg.rcut), float(cfg.rcut_smth), sel.ctypes.data_as(C.POINTER(C.c_int32)),
                len(emb), emb.ctypes.data_as(C.POINTER(C.c_int32)), int(cfg.m2), len(fit),
                fit.ctypes.data_as(C.POINTER(C.c_int32)))
    h = C.c_void_p()
    _check(lib.dp_model_create(C.byref(c), C.c_uint64(seed & ((1 << 64) - 1)), C.byref(h)), "dp_model_create")
    return h.value


def dp_model_n_params(m) -> int:
    n = C.c_int64()
    _check(load().dp_model_n_params(m, C.byref(n)), "dp_model_n_params")
    return n.value


def dp_model_get_params(m) -> np.ndarray:
    n = dp_model_n_params(m)
    out = np.empty(n)
    _check(load().dp_model_get_params(m, _ptr(out), n), "dp_model_get_params")
    return out


def dp_model_set_params(m, flat):
    flat = _f64(flat)
    _check(load().dp_model_set_params(m, _ptr(flat), flat.size), "dp_model_set_params")


def dp_model_destroy(m):
    if m:
        load().dp_model_destroy(m)


def dp_model_set_deterministic(m, on: bool = True):
    _check(load().dp_model_set_deterministic(m, 1 if on else 0), "dp_model_set_deterministic")


def dp_model_set_stream(m, stream=None):
    """Run the model's calls on `stream` (torch.cuda.Stream or raw handle); None = library stream."""
    sp = None if stream is None else C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)
    _check(load().dp_model_set_stream(m, sp), "dp_model_set_stream")


def dp_profile_enable(m, on: bool = True):
    _check(load().dp_profile_enable(m, int(bool(on))), "dp_profile_enable")


def dp_profile_select(m, groups=None):
    """Time only the named groups (None: all of them) while profiling is on."""
    if groups is None:
        mask = 0xFFFFFFFF
    else:
        names, g = {}, 0
        while (name := dp_profile_group_name(g)) is not None:
            names[name] = g
            g += 1
        mask = 0
        for name in groups:
            mask |= 1 << names[name]
    _check(load().dp_profile_select(m, mask), "dp_profile_select")


def dp_profile_group_name(g: int):
    r = load().dp_profile_group_name(int(g))
    return None if r is None else r.decode()


def dp_profile_read(m):
    """{group name: (launches, device ms)} since the last dp_profile_enable."""
    out = {}
    g = 0
    while True:
        name = dp_profile_group_name(g)
        if name is None:
            return out
        n, ms = C.c_int64(), C.c_double()
        _check(load().dp_profile_read(m, g, C.byref(n), C.byref(ms)), "dp_profile_read")
        out[name] = (n.value, ms.value)
        g += 1


# ---------------------------------------------------------- neighbor list

def dp_nlist_build(m, coord, typ, box, rcut: float, skin: float = 0.0, cand_cap: int = 0):
    coord, typ, box = _f64(coord), _i32(typ), _box(box)
    h = C.c_void_p()
    _check(load().dp_nlist_build(m, typ.size, _ptr(coord), _ptr(typ), _ptr(box), float(rcut), float(skin),
                                 int(cand_cap), C.byref(h)), "dp_nlist_build")
    return h.value


def dp_nlist_build_frames(m, coords, typ, box, rcut: float, skin: float = 0.0, cand_cap: int = 0):
    """One list over nframes configurations coords [F][n][3] of the same atoms typ [n] in the same box."""
    coords, typ, box = _f64(coords), _i32(typ), _box(box)
    nframes = coords.shape[0]
    h = C.c_void_p()
    _check(load().dp_nlist_build_frames(m, int(nframes), typ.size, _ptr(coords), _ptr(typ), _ptr(box), float(rcut),
                                        float(skin), int(cand_cap), C.byref(h)), "dp_nlist_build_frames")
    return h.value


def dp_nlist_update(nl, coord, box):
    coord, box = _f64(coord), _box(box)
    _check(load().dp_nlist_update(nl, _ptr(coord), _ptr(box)), "dp_nlist_update")


def dp_nlist_get(nl, n: int, nsel: int):
    out = np.empty((n, nsel), dtype=np.int32)
    ntr = C.c_int64()
    _check(load().dp_nlist_get(nl, _ptr(out), C.byref(ntr)), "dp_nlist_get")
    return out, ntr.value


def _stream(stream):
    if stream is None:
        return None
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)


def dp_nlist_update_dev(nl, d_coord, stream=None):
    _check(load().dp_nlist_update_dev(nl, _ptr(d_coord), _stream(stream)), "dp_nlist_update_dev")


def _check_dev_tensor(t, name: str, dtypes, numel: int):
    """Raise ValueError unless t is a contiguous CUDA tensor on the current device with the given
    dtype(s) and element count: the entry points behind this binding take raw device addresses."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: expected a torch CUDA tensor, got {type(t).__name__}")
    if t.device.type != "cuda" or t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: must live on the current CUDA device (cuda:{torch.cuda.current_device()}), "
                         f"not {t.device}")
    if t.dtype not in dtypes:
        raise ValueError(f"{name}: dtype {t.dtype}, expected {' or '.join(str(d) for d in dtypes)}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if t.numel() != numel:
        raise ValueError(f"{name}: {t.numel()} elements, expected {numel}")


def dp_nlist_format_noalloc(d_coord, d_type, box, rcut: float, sel, d_nlist, d_ntrunc, d_status, stream=None):
    """Formatted list into caller-owned device buffers; the library allocates nothing.

    d_coord float64 [n][3], d_type int32 [n], d_nlist int32 [n][sum(sel)], d_ntrunc one int64 / uint64,
    d_status one int32: contiguous CUDA tensors on the current device (checked here, ValueError
    otherwise).  stream: a torch stream or raw handle; None = torch's current stream."""
    import torch
    sel = _i32(sel)
    if not isinstance(d_type, torch.Tensor):
        raise ValueError("d_type: expected a torch CUDA tensor")
    n = int(d_type.numel())
    _check_dev_tensor(d_type, "d_type", (torch.int32,), n)
    _check_dev_tensor(d_coord, "d_coord", (torch.float64,), 3 * n)
    _check_dev_tensor(d_nlist, "d_nlist", (torch.int32,), n * int(sel.sum()))
    _check_dev_tensor(d_ntrunc, "d_ntrunc", (torch.int64, getattr(torch, "uint64", torch.int64)), 1)
    _check_dev_tensor(d_status, "d_status", (torch.int32,), 1)
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(load().dp_nlist_format_noalloc(n, _ptr(d_coord), _ptr(d_type), _ptr(_box(box)),
                                          float(rcut), int(sel.size), _ptr(sel), _ptr(d_nlist), _ptr(d_ntrunc),
                                          _ptr(d_status), _stream(stream)), "dp_nlist_format_noalloc")


def dp_tanh_f64_dev(d_x, d_y, stream=None):
    """y = tanh(x) by the FP64 kernels' own routine (device tensors of equal size)."""
    _check(load().dp_tanh_f64_dev(int(d_x.numel()), _ptr(d_x), _ptr(d_y), _stream(stream)), "dp_tanh_f64_dev")


def dp_ozaki_dgemm_dev(m, d_A, d_Bt, d_C, stream=None):
    """C = A Bt^T in FP64 on the tensor cores (device tensors A [M][K], Bt [N][K], C [M][N])."""
    M, K = d_A.shape
    N = d_Bt.shape[0]
    _check(load().dp_ozaki_dgemm_dev(m, int(M), int(N), int(K), _ptr(d_A), _ptr(d_Bt), _ptr(d_C), _stream(stream)),
           "dp_ozaki_dgemm_dev")


def dp_test_starve_wait(m, which: int, polls: int = 0):
    """Starve one bounded device wait of the model's later evaluations (1), or restore (0)."""
    _check(load().dp_test_starve_wait(m, int(which), int(polls)), "dp_test_starve_wait")


def dp_bounds_checked() -> bool:
    """True when the loaded library is the bounds-checked debug build."""
    return bool(load().dp_bounds_checked())


def dp_bounds_read(clear: bool = True):
    """(count, site, index, limit) of the bad indexes the bounds-checked build found (zeros otherwise)."""
    rec = np.zeros(4, dtype=np.int64)
    _check(load().dp_bounds_read(_ptr(rec), int(bool(clear))), "dp_bounds_read")
    return tuple(int(v) for v in rec)


def dp_nlist_set_centers(nl, n_centers: int):
    """Atoms [0, n_centers) are centers, the rest ghosts (neighbors only)."""
    _check(load().dp_nlist_set_centers(nl, int(n_centers)), "dp_nlist_set_centers")


def dp_halo_select_dev(d_coord, d_type, lo: float, hi: float, shift_x: float, d_idx, d_out_coord, d_out_type,
                       d_count, stream=None):
    """Atoms with lo <= x < hi, in index order, packed with x shifted (device tensors; cap = d_idx.numel())."""
    _check(load().dp_halo_select_dev(int(d_type.numel()), _ptr(d_coord), _ptr(d_type), float(lo), float(hi),
                                     float(shift_x), int(d_idx.numel()), _ptr(d_idx), _ptr(d_out_coord),
                                     _ptr(d_out_type), _ptr(d_count), _stream(stream)), "dp_halo_select_dev")


def dp_halo_accumulate_dev(d_idx, d_f_ghost, d_force, stream=None):
    """d_force[d_idx[k]] += d_f_ghost[k] (device tensors, distinct indices)."""
    _check(load().dp_halo_accumulate_dev(int(d_idx.numel()), _ptr(d_idx), _ptr(d_f_ghost), _ptr(d_force),
                                         _stream(stream)), "dp_halo_accumulate_dev")


def dp_nlist_destroy(nl):
    if nl:
        load().dp_nlist_destroy(nl)


# ----------------------------------------------------------------- compute

def dp_compute(m, nl, coord, box, prec="fp64"):
    """Host arrays in, (E, E_i[n], F[n,3], W[3,3]) out."""
    coord, box = _f64(coord), _box(box)
    n = coord.shape[0]
    e = np.zeros(1)
    ei = np.empty(n)
    f = np.empty((n, 3))
    w = np.empty(9)
    _check(load().dp_compute(m, nl, _ptr(coord), _ptr(box), _prec(prec), _ptr(e), _ptr(ei), _ptr(f), _ptr(w)),
           "dp_compute")
    return float(e[0]), ei, f, w.reshape(3, 3)


def dp_compute_dev(m, nl, d_coord, box, prec, d_energy, d_atom_energy, d_force, d_virial, stream=None):
    """Device pointers (torch CUDA tensors, float64) in and out; enqueued on `stream` (a torch stream or None)."""
    box = _box(box)
    sp = None if stream is None else C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)
    _check(load().dp_compute_dev(m, nl, _ptr(d_coord), _ptr(box), _prec(prec), _ptr(d_energy), _ptr(d_atom_energy),
                                 _ptr(d_force), _ptr(d_virial), sp), "dp_compute_dev")


# ---------------------------------------------------------------- training

def dp_param_grad(m, nl, coord, box, v, alpha: float, beta: float, prec="fp64", grad=None):
    """(E, Edot, grad) with grad += d(alpha E + beta Edot)/dtheta, Edot = sum_k v_k . dE/dr_k."""
    coord, box, v = _f64(coord), _box(box), _f64(v)
    if grad is None:
        grad = np.zeros(dp_model_n_params(m))
    e, ed = C.c_double(), C.c_double()
    _check(load().dp_param_grad(m, nl, _ptr(coord), _ptr(box), _ptr(v), float(alpha), float(beta), _prec(prec),
                                C.byref(e), C.byref(ed), _ptr(grad)), "dp_param_grad")
    return e.value, ed.value, grad


def dp_force_loss_grad(m, nl, coord, box, F_ref, E_ref: float, p_e: float, p_f: float, prec="fp64", grad=None):
    """(loss, grad): loss and grad ADDED for one configuration (host arrays)."""
    coord, box, F_ref = _f64(coord), _box(box), _f64(F_ref)
    if grad is None:
        grad = np.zeros(dp_model_n_params(m))
    loss = C.c_double(0.0)
    _check(load().dp_force_loss_grad(m, nl, _ptr(coord), _ptr(box), _ptr(F_ref), float(E_ref), float(p_e),
                                     float(p_f), _prec(prec), C.byref(loss), _ptr(grad)), "dp_force_loss_grad")
    return loss.value, grad


def dp_force_loss_grad_dev(m, nl, d_coord, box, d_F_ref, d_E_ref, p_e, p_f, prec, d_loss, d_grad, stream=None):
    _check(load().dp_force_loss_grad_dev(m, nl, _ptr(d_coord), _ptr(_box(box)), _ptr(d_F_ref), _ptr(d_E_ref),
                                         float(p_e), float(p_f), _prec(prec), _ptr(d_loss), _ptr(d_grad),
                                         _stream(stream)), "dp_force_loss_grad_dev")


def dp_adam_step(m, d_grad, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, t: int = 1,
                 stream=None):
    _check(load().dp_adam_step(m, _ptr(d_grad), float(lr), float(beta1), float(beta2), float(eps), int(t),
                               _stream(stream)), "dp_adam_step")


def dp_model_sync_params(m):
    _check(load().dp_model_sync_params(m), "dp_model_sync_params")


# ---------------------------------------------------------------------- MD

def dp_md_state_create(m, coord, vel, typ, mass_by_type, box, skin: float = 2.0, cand_cap: int = 0):
    coord, vel, typ, mass, box = _f64(coord), _f64(vel), _i32(typ), _f64(mass_by_type), _box(box)
    h = C.c_void_p()
    _check(load().dp_md_state_create(m, typ.size, _ptr(coord), _ptr(vel), _ptr(typ), _ptr(mass), _ptr(box),
                                     float(skin), int(cand_cap), C.byref(h)), "dp_md_state_create")
    return h.value


def dp_md_step(m, s, nsteps: int, dt_fs: float, prec="fp64", thermo_every: int = 0):
    rows = nsteps // thermo_every if thermo_every > 0 else 0
    th = np.zeros((max(rows, 1), 4))
    _check(load().dp_md_step(m, s, int(nsteps), float(dt_fs), _prec(prec), int(thermo_every),
                             _ptr(th) if rows else None), "dp_md_step")
    return th[:rows]


def dp_md_step_judged(student, teacher, s, nsteps: int, dt_fs: float, student_prec="mix32", teacher_prec="mix32",
                      judge_every: int = 10, rmse_max: float = 0.05):
    """(rmse per judgement, fallback flag per judgement)."""
    w = max(nsteps // judge_every, 1)
    rm = np.zeros(w)
    fb = np.zeros(w, dtype=np.int32)
    _check(load().dp_md_step_judged(student, teacher, s, int(nsteps), float(dt_fs), _prec(student_prec),
                                    _prec(teacher_prec), int(judge_every), float(rmse_max), _ptr(rm), _ptr(fb)),
           "dp_md_step_judged")
    k = nsteps // judge_every
    return rm[:k], fb[:k]


def dp_md_set_rebuild_every(s, every: int):
    """Also rebuild the skin list every `every` MD steps (0: only when an atom moved > skin/2)."""
    _check(load().dp_md_set_rebuild_every(s, int(every)), "dp_md_set_rebuild_every")


def dp_md_state_save(s, path: str):
    """Checkpoint of the state to `path` (flat FP64 file, see include/dp.h)."""
    _check(load().dp_md_state_save(s, os.fsencode(path)), "dp_md_state_save")


def dp_md_state_load(m, path: str):
    """A new MD state of model m from a checkpoint file; returns (handle, n)."""
    h = C.c_void_p()
    _check(load().dp_md_state_load(m, os.fsencode(path), C.byref(h)), "dp_md_state_load")
    n = int(np.fromfile(path, dtype=np.float64, count=3)[2])
    return h, n


def dp_md_state_get(s, n: int):
    x = np.empty((n, 3))
    v = np.empty((n, 3))
    step, nreb = C.c_int64(), C.c_int64()
    _check(load().dp_md_state_get(s, _ptr(x), _ptr(v), C.byref(step), C.byref(nreb)), "dp_md_state_get")
    return x, v, step.value, nreb.value


def dp_md_state_destroy(s):
    if s:
        load().dp_md_state_destroy(s)
