"""A decomposition engine built from the oracle, for the CPU tests of paper_2005_00223_gb300.domain.

It stands in for the GPU engine (libdp) where no GPU exists: the halo selection and the reverse halo as
plain numpy/torch operations, the evaluation of a rank's extended system as the oracle's per-center
energy and pair derivatives g_ij = dE_i/dd_ij (F_i += g_ij, F_j -= g_ij, W = -sum d_ij (x) g_ij) over
the owned centers only.  Arrays are torch CPU tensors, so that gloo can send them.
"""
import numpy as np
import torch

import dpsynth
import oracle


def workload(name):
    if name == "water192":
        cfg = dpsynth.water_config()
        return (cfg, *dpsynth.water_box(1))
    if name == "cu500":
        cfg = dpsynth.copper_config()
        return (cfg, *dpsynth.copper_fcc(1, ncell=5))
    raise ValueError(name)


class OracleEngine:
    def __init__(self, cfg, params):
        self.om = oracle.Model(cfg, params)

    @staticmethod
    def count(t):
        return int(t.numel())

    @staticmethod
    def cat(parts):
        return torch.cat(parts)

    @staticmethod
    def rows(a, b, e):
        return a[b:e]

    @staticmethod
    def host(t):
        return np.asarray(t, dtype=np.float64)

    def select(self, coord, typ, lo, hi, shift):
        x = coord[:, 0]
        idx = torch.nonzero((x >= lo) & (x < hi)).reshape(-1)
        xs = coord[idx].clone()
        xs[:, 0] += shift
        return idx.to(torch.int32), xs, typ[idx]

    def shift_all(self, coord, typ, shift):
        xs = coord.clone()
        xs[:, 0] += shift
        return xs, typ.clone()

    def evaluate(self, ext_x, ext_t, ext_box, n_centers):
        x, t = ext_x.numpy(), ext_t.numpy()
        box = np.asarray(ext_box, dtype=np.float64)
        L = np.diag(box)
        nl, _, _ = self.om.nlist(x, t, box)
        E, F, W = 0.0, np.zeros_like(x), np.zeros((3, 3))
        for i in range(n_centers):
            Ei, g, _ = self.om.atom(i, nl[i], x, t, box)
            row = nl[i]
            ok = row >= 0
            E += Ei
            F[i] += g[ok].sum(0)
            np.subtract.at(F, row[ok], g[ok])
            d = x[row[ok]] - x[i]
            d -= L * np.rint(d / L)
            W -= d.T @ g[ok]
        return E, torch.tensor(F), torch.tensor(W)

    def accumulate(self, F, idx, f):
        F[idx.long()] += f
