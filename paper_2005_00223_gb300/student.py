"""Distilled student: data from the full model's own MD, training with the library's kernels.

Orchestration only.  The teacher's trajectories (dp_md_step), the labels
(dp_compute), the loss and its parameter gradient (dp_force_loss_grad_dev),
the optimizer (dp_adam_step) and the judged student MD (dp_md_step_judged)
all run in libdp; Python picks frames, learning rates and loops.  PyTorch
only holds device buffers and the stream.
"""
from __future__ import annotations

import math

import numpy as np

from . import MDState, Model, NeighborList, _lib


def teacher_frames(teacher: Model, coord, typ, box, mass_by_type, velocities, nframes: int, stride: int,
                   dt_fs: float, md_prec="mix32", label_prec="mix32", skin: float = 2.0, return_temps: bool = False):
    """Frames sampled every `stride` NVE steps of the teacher, one run per initial velocity set.

    Returns (coords [F, n, 3], energies [F], forces [F, n, 3]) as numpy arrays, labelled by the
    teacher in `label_prec`; with return_temps also the instantaneous temperature (K) of each frame.
    """
    xs, es, fs, ts = [], [], [], []
    for vel in velocities:
        st = MDState(teacher, coord, vel, typ, mass_by_type, box, skin=skin)
        nl = NeighborList(teacher, coord, typ, box, skin=skin)
        for _ in range(nframes):
            th = st.step(stride, dt_fs, md_prec, thermo_every=stride)
            ts.append(float(np.asarray(th)[-1][2]))
            x, _, _, _ = st.get()
            nl.update(x, box)
            E, _, F, _ = nl.compute(x, box, label_prec)
            xs.append(x)
            es.append(E)
            fs.append(F)
        st.close()
        nl.close()
    if return_temps:
        return np.array(xs), np.array(es), np.array(fs), np.array(ts)
    return np.array(xs), np.array(es), np.array(fs)


def train(student: Model, typ, box, coords, energies, forces, steps: int, lr0: float = 1e-3, lr1: float = 1e-5,
          p_e: float = 1.0, p_f: float = 100.0, prec="mix32", seed: int = 0, log_every: int = 50):
    """Adam on the force-matching loss, one frame per step, lr decaying exponentially lr0 -> lr1.

    p_f: one force weight for every frame, or an array of one weight per frame (e.g. 1 / RMS(F_k)^2 for
    a relative force loss over frames whose force scales differ).  Returns the list of (step, mean loss
    over the last log_every steps).
    """
    import torch
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream(dev)
    _lib.dp_model_set_stream(student.h, stream)
    X = torch.tensor(coords, dtype=torch.float64, device=dev)
    Fr = torch.tensor(forces, dtype=torch.float64, device=dev)
    Er = torch.tensor(energies, dtype=torch.float64, device=dev)
    nparams = _lib.dp_model_n_params(student.h)
    grad = torch.zeros(nparams, dtype=torch.float64, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    pf = np.broadcast_to(np.asarray(p_f, dtype=np.float64), (len(coords),))
    nl = NeighborList(student, coords[0], typ, box, skin=0.0)
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(coords))
    log = []
    for s in range(steps):
        k = int(order[s % len(order)])
        if s % len(order) == len(order) - 1:
            order = rng.permutation(len(coords))
        _lib.dp_nlist_update_dev(nl.h, X[k], stream)
        grad.zero_()
        _lib.dp_force_loss_grad_dev(student.h, nl.h, X[k], box, Fr[k], Er[k:k + 1], p_e, float(pf[k]), prec, loss,
                                    grad, stream)
        lr = lr0 * math.exp(math.log(lr1 / lr0) * s / max(steps - 1, 1))
        _lib.dp_adam_step(student.h, grad, lr, 0.9, 0.999, 1e-8, s + 1, stream)
        if (s + 1) % log_every == 0:
            log.append((s + 1, float(loss.item()) / log_every))
            loss.zero_()
    torch.cuda.synchronize()
    nl.get()   # reports a capacity overflow of any rebuild
    nl.close()
    _lib.dp_model_sync_params(student.h)
    _lib.dp_model_set_stream(student.h, None)
    return log


def fit_to_reference(model: Model, coords, energies, forces, typ, box, steps: int, lr0: float = 2e-3,
                     lr1: float = 2e-5, p_e: float = 0.02, p_f: float = 100.0, segments: int = 4, prec="mix32"):
    """Fits a full model to labelled reference frames (e.g. a classical potential's) with the same
    kernels as the distillation: one-frame Adam steps on the force-matching loss, the learning rate
    decaying lr0 -> lr1 over `segments` restarts of train() (each reshuffles the frames).  A large
    force weight against a small energy weight (p_f / p_e = 5,000) fits the forces first, as
    DeePMD-kit's training schedule starts.  Returns the concatenated loss log."""
    log = []
    per = max(1, steps // segments)
    for k in range(segments):
        a = lr0 * (lr1 / lr0) ** (k / segments)
        z = lr0 * (lr1 / lr0) ** ((k + 1) / segments)
        log += train(model, typ, box, coords, energies, forces, steps=per, lr0=a, lr1=z, p_e=p_e, p_f=p_f,
                     prec=prec, seed=k, log_every=max(1, per // 5))
    return log


def force_rmse_vs_labels(model: Model, coords, forces, typ, box, prec="mix32"):
    """Force RMSE of a model against labelled frames, and the RMS of the labels."""
    nl = NeighborList(model, coords[0], typ, box)
    se, sf, cnt = 0.0, 0.0, 0
    for x, f in zip(coords, forces):
        nl.update(x, box)
        F = nl.compute(x, box, prec)[2]
        se += float(((F - f) ** 2).sum())
        sf += float((f ** 2).sum())
        cnt += len(typ)
    nl.close()
    return math.sqrt(se / cnt), math.sqrt(sf / cnt)


def force_rmse(a: Model, b: Model, coords, typ, box, prec_a="mix32", prec_b="mix32"):
    """Force RMSE sqrt(mean_i |F_a,i - F_b,i|^2) of two models over frames, and the RMS force of b."""
    nla = NeighborList(a, coords[0], typ, box)
    nlb = NeighborList(b, coords[0], typ, box)
    se, sf, cnt = 0.0, 0.0, 0
    for x in coords:
        nla.update(x, box)
        nlb.update(x, box)
        Fa = nla.compute(x, box, prec_a)[2]
        Fb = nlb.compute(x, box, prec_b)[2]
        se += float(((Fa - Fb) ** 2).sum())
        sf += float((Fb ** 2).sum())
        cnt += len(typ)
    nla.close()
    nlb.close()
    return math.sqrt(se / cnt), math.sqrt(sf / cnt)
