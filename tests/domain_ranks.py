"""One rank of the spatially decomposed evaluation on CPU, for tests/test_domain.py.

Run under torch.distributed.run with the gloo backend: every rank owns the atoms of its slab, exchanges
halos and ghost forces through paper_2005_00223_gb300.domain.TorchTransport, evaluates its extended
system with the oracle (tests/oracle_engine.py), and rank 0 gathers the forces and prints E, W and F as
one JSON line.  Arguments: workload name (water192 | cu500).
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402
import torch  # noqa: E402
import torch.distributed as dist  # noqa: E402

import dpsynth  # noqa: E402
from oracle_engine import OracleEngine, workload  # noqa: E402
from paper_2005_00223_gb300 import domain  # noqa: E402


def main():
    name = sys.argv[1]
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    cfg, coord, typ, box = workload(name)
    eng = OracleEngine(cfg, dpsynth.model_params(cfg, 1))
    own = domain.owned_atoms(coord, box, rank, world)
    slab = domain.Slab(box, rank, world, halo=cfg.rcut, rcut=cfg.rcut)
    x = torch.tensor(np.mod(coord[own], np.diag(box)), dtype=torch.float64)
    t = torch.tensor(typ[own], dtype=torch.int32)
    r = domain.RankState(eng, slab, x, t)
    E, W = domain.TorchTransport().evaluate_rank(r)
    n_own = torch.tensor([len(own)], dtype=torch.int64)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, n_own)
    mx = int(max(s.item() for s in sizes))
    pad_f = torch.zeros((mx, 3), dtype=torch.float64)
    pad_f[:len(own)] = r.F
    pad_i = torch.full((mx,), -1, dtype=torch.int64)
    pad_i[:len(own)] = torch.tensor(own, dtype=torch.int64)
    fs = [torch.zeros_like(pad_f) for _ in range(world)]
    ids = [torch.zeros_like(pad_i) for _ in range(world)]
    dist.all_gather(fs, pad_f)
    dist.all_gather(ids, pad_i)
    if rank == 0:
        F = np.zeros((len(typ), 3))
        for f, i in zip(fs, ids):
            k = i.numpy() >= 0
            F[i.numpy()[k]] = f.numpy()[k]
        print(json.dumps({"E": E, "W": W.tolist(), "F": F.tolist(), "world": world}))
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
