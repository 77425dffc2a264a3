"""Spatial decomposition of the energy / force / virial evaluation over ranks (Sec. 4.3).

The paper runs DP inside LAMMPS's spatial partitioning: every MPI rank holds
the atoms of its sub-domain, receives the ghost atoms of a halo around it
from its neighbors, evaluates the energies of its own atoms, returns the
forces that landed on ghosts (F_j -= g_ij for a ghost j) to their owners, and
all-reduces the energy and the virial.  DP's force decomposition makes this
exact: E_i depends only on the atoms within r_c of atom i.

Here the box is cut into `world` slabs along x.  Rank r owns the atoms with
x in [r L/P, (r+1) L/P) (wrapped coordinates) and evaluates them in its
extended frame: its slab plus a halo of width h (r_c, plus the list skin for
lists kept across steps) on both sides, shifted so that the frame starts at
x = 0, in a box whose x edge exceeds the extended region by r_c, so that no
periodic image of a ghost reaches an owned atom.  Each evaluation:

  1. pack: the atoms within h of each slab face, shifted into the receiving
     neighbor's frame (dp_halo_select_dev);
  2. exchange the ghosts with both neighbors;
  3. evaluate the extended system with the owned atoms as the only centers
     (dp_nlist_set_centers): E_i and the virial of the owned atoms, forces on
     owned atoms and ghosts;
  4. return each ghost's force to the rank that sent it;
  5. add the returned forces into the owned atoms' forces
     (dp_halo_accumulate_dev), one call per neighbor so that every sum has a
     fixed order;
  6. all-reduce E and W.

Communication goes through a transport: `TorchTransport` over
torch.distributed (NCCL between GPUs, gloo between CPU processes) or
`InProcessTransport`, which runs the phases of all ranks in turn in one
process (one GPU standing in for several, no collective kernels).  The
arithmetic of the evaluation runs in an engine: `LibdpEngine` calls libdp's
kernels on the GPU.  This module only moves data and calls them.
"""
from __future__ import annotations

import numpy as np


class Slab:
    """Geometry of rank `rank`'s slab of an orthorhombic box cut into `world` slabs along x."""

    def __init__(self, box, rank: int, world: int, halo: float, rcut: float):
        L = np.diag(np.asarray(box, dtype=np.float64).reshape(3, 3)).copy()
        if world < 2:
            raise ValueError("a decomposition needs at least two ranks")
        if not np.allclose(np.asarray(box, dtype=np.float64).reshape(3, 3), np.diag(L)):
            raise ValueError("orthorhombic boxes only")
        w = L[0] / world
        if halo > w:
            raise ValueError(f"slab width {w:.3f} A below the halo {halo:.3f} A: use fewer ranks")
        self.L, self.rank, self.world, self.halo, self.width = L, rank, world, float(halo), w
        self.x0, self.x1 = rank * w, (rank + 1) * w
        self.left, self.right = (rank - 1) % world, (rank + 1) % world
        self.origin = self.x0 - halo            # x of the extended frame's 0
        # the box of the extended frame: slab + two halos + r_c of empty space along x
        self.ext_box = np.diag([w + 2.0 * halo + rcut + 1e-6, L[1], L[2]])

    def frame_origin(self, r: int) -> float:
        return r * self.width - self.halo

    def send_ranges(self):
        """[(destination rank, side of the destination's halo, lo, hi, x shift)] of the two halos this rank
        sends: its lowest h of x to the left neighbor (that neighbor's right halo), its highest h to the
        right neighbor (its left halo); the shift maps x into the destination's extended frame, across
        the periodic boundary for the first and the last rank."""
        L = self.L[0]
        to_left = (self.left, "right", self.x0, self.x0 + self.halo,
                   (L if self.rank == 0 else 0.0) - self.frame_origin(self.left))
        to_right = (self.right, "left", self.x1 - self.halo, self.x1,
                    (-L if self.rank == self.world - 1 else 0.0) - self.frame_origin(self.right))
        return [to_left, to_right]


class RankState:
    """Phases of one rank's decomposed evaluation (see the module docstring)."""

    def __init__(self, engine, slab: Slab, coord, typ):
        self.engine, self.slab = engine, slab
        self.coord, self.typ = coord, typ          # owned atoms (engine arrays), wrapped coordinates
        self.sent = {}

    def pack(self):
        """{(destination, side): (coords in the destination's frame, types)}; remembers the indices sent."""
        out = {}
        for dest, side, lo, hi, shift in self.slab.send_ranges():
            idx, xs, ts = self.engine.select(self.coord, self.typ, lo, hi, shift)
            self.sent[side] = idx          # the destination's `side` halo holds these atoms
            out[(dest, side)] = (xs, ts)
        return out

    def evaluate(self, ghosts_left, ghosts_right):
        """Extended system [owned | left ghosts | right ghosts] with the owned atoms as centers."""
        own_x, own_t = self.engine.shift_all(self.coord, self.typ, -self.slab.origin)
        self.n_own = self.engine.count(own_t)
        self.n_left = self.engine.count(ghosts_left[1])
        ext_x = self.engine.cat([own_x, ghosts_left[0], ghosts_right[0]])
        ext_t = self.engine.cat([own_t, ghosts_left[1], ghosts_right[1]])
        E, F, W = self.engine.evaluate(ext_x, ext_t, self.slab.ext_box, self.n_own)
        self.E, self.W = E, W
        self.F = self.engine.rows(F, 0, self.n_own)
        return {"left": self.engine.rows(F, self.n_own, self.n_own + self.n_left),
                "right": self.engine.rows(F, self.n_own + self.n_left, self.engine.count(ext_t))}

    def accumulate(self, returned):
        """Forces of this rank's atoms that were ghosts elsewhere, returned by the ranks that held them:
        returned[side] are the forces of the atoms this rank sent as the destination's `side` halo."""
        for side in ("right", "left"):
            self.engine.accumulate(self.F, self.sent[side], returned[side])


class InProcessTransport:
    """All ranks' phases in turn in one process: exchanges are plain array hand-overs."""

    def __init__(self, world: int):
        self.world = world

    def evaluate(self, ranks):
        msgs = [r.pack() for r in ranks]
        ghosts = [dict() for _ in ranks]
        for src, m in enumerate(msgs):
            for (dest, side), payload in m.items():
                ghosts[dest][side] = payload
        back = [r.evaluate(ghosts[k]["left"], ghosts[k]["right"]) for k, r in enumerate(ranks)]
        # the forces of rank k's left halo go back to its left neighbor, which sent those atoms as the
        # destination's left halo; likewise for the right halo
        ret = [dict() for _ in ranks]
        for k, r in enumerate(ranks):
            ret[r.slab.left]["left"] = back[k]["left"]
            ret[r.slab.right]["right"] = back[k]["right"]
        for k, r in enumerate(ranks):
            r.accumulate(ret[k])
        E = sum(float(r.engine.host(r.E).reshape(-1)[0]) for r in ranks)
        W = sum(r.engine.host(r.W).reshape(3, 3) for r in ranks)
        return E, W


class TorchTransport:
    """Exchanges over torch.distributed: counts, then coordinates and types, then forces back.

    Tensors must live where the backend expects them (CUDA for NCCL, CPU for gloo).  With two ranks
    the left and the right neighbor are the same rank; the messages are told apart by their order."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group

    def _swap(self, sends, recv_like):
        """sends: [(peer, tensor)], recv_like: [(peer, shape, dtype, device)] -> received tensors (same order)."""
        import torch
        reqs, outs = [], []
        for (peer, shape, dtype, device) in recv_like:
            t = torch.empty(shape, dtype=dtype, device=device)
            outs.append(t)
            reqs.append(self.dist.irecv(t, src=peer, group=self.group))
        for peer, t in sends:
            reqs.append(self.dist.isend(t.contiguous(), dst=peer, group=self.group))
        for q in reqs:
            q.wait()
        return outs

    def evaluate_rank(self, r: RankState):
        import torch
        s = r.slab
        msgs = r.pack()
        (xl, tl), (xr, tr) = msgs[(s.left, "right")], msgs[(s.right, "left")]
        dev = xl.device
        cnt = self._swap([(s.left, torch.tensor([tl.numel()], dtype=torch.int64, device=dev)),
                          (s.right, torch.tensor([tr.numel()], dtype=torch.int64, device=dev))],
                         [(s.right, (1,), torch.int64, dev), (s.left, (1,), torch.int64, dev)])
        n_from_right, n_from_left = int(cnt[0].item()), int(cnt[1].item())
        # my right halo comes from my right neighbor, which sends its lowest slab; my left halo from the left
        gx = self._swap([(s.left, xl), (s.right, xr)],
                        [(s.right, (n_from_right, 3), xl.dtype, dev), (s.left, (n_from_left, 3), xl.dtype, dev)])
        gt = self._swap([(s.left, tl), (s.right, tr)],
                        [(s.right, (n_from_right,), tl.dtype, dev), (s.left, (n_from_left,), tl.dtype, dev)])
        back = r.evaluate((gx[1], gt[1]), (gx[0], gt[0]))
        # forces of my left halo go to my left neighbor (its atoms sent as its "right" halo), and so on
        fr = self._swap([(s.left, back["left"]), (s.right, back["right"])],
                        [(s.right, (tr.numel(), 3), back["left"].dtype, dev),
                         (s.left, (tl.numel(), 3), back["left"].dtype, dev)])
        r.accumulate({"left": fr[0], "right": fr[1]})
        ew = torch.cat([torch.as_tensor(r.E, dtype=torch.float64, device=dev).reshape(1),
                        torch.as_tensor(r.W, dtype=torch.float64, device=dev).reshape(9)])
        self.dist.all_reduce(ew, group=self.group)
        return float(ew[0].item()), ew[1:].reshape(3, 3).cpu().numpy()


class LibdpEngine:
    """Engine of one rank on the GPU: libdp's halo and evaluation kernels on CUDA tensors."""

    def __init__(self, model, precision: str = "fp64", skin: float = 0.0, stream=None):
        import torch
        self.model, self.precision, self.skin = model, precision, skin
        self.stream = stream or torch.cuda.current_stream()
        self.nl = None

    @staticmethod
    def count(t):
        return int(t.numel())

    @staticmethod
    def host(t):
        return t.detach().cpu().numpy().astype(np.float64)

    @staticmethod
    def cat(parts):
        import torch
        return torch.cat(parts)

    @staticmethod
    def rows(a, b, e):
        return a[b:e]

    def select(self, coord, typ, lo, hi, shift):
        import torch

        from . import _lib
        n = typ.numel()
        idx = torch.empty(n, dtype=torch.int32, device=coord.device)
        xs = torch.empty((n, 3), dtype=torch.float64, device=coord.device)
        ts = torch.empty(n, dtype=torch.int32, device=coord.device)
        cnt = torch.zeros(1, dtype=torch.int64, device=coord.device)
        _lib.dp_halo_select_dev(coord, typ, lo, hi, shift, idx, xs, ts, cnt, self.stream)
        k = int(cnt.item())
        return idx[:k], xs[:k], ts[:k]

    def shift_all(self, coord, typ, shift):
        _, xs, ts = self.select(coord, typ, -np.inf, np.inf, shift)
        return xs, ts

    def evaluate(self, ext_x, ext_t, ext_box, n_centers):
        import torch

        from . import NeighborList, _lib
        n = ext_t.numel()
        if self.nl is not None:
            self.nl.close()
        self.nl = NeighborList(self.model, ext_x.cpu().numpy(), ext_t.cpu().numpy(), ext_box, skin=self.skin)
        _lib.dp_nlist_set_centers(self.nl.h, n_centers)
        dev = ext_x.device
        e = torch.zeros(1, dtype=torch.float64, device=dev)
        ei = torch.empty(n, dtype=torch.float64, device=dev)
        f = torch.empty((n, 3), dtype=torch.float64, device=dev)
        w = torch.empty(9, dtype=torch.float64, device=dev)
        _lib.dp_compute_dev(self.model.h, self.nl.h, ext_x.contiguous(), ext_box, self.precision, e, ei, f, w,
                            self.stream)
        return e, f, w

    def accumulate(self, F, idx, f):
        from . import _lib
        _lib.dp_halo_accumulate_dev(idx, f.contiguous(), F, self.stream)

    def close(self):
        if self.nl is not None:
            self.nl.close()
            self.nl = None


def owned_atoms(coord, box, rank: int, world: int):
    """Indices of the atoms rank `rank` owns (x of the wrapped coordinates in its slab), in index order."""
    L = np.diag(np.asarray(box, dtype=np.float64).reshape(3, 3))
    x = np.mod(np.asarray(coord, dtype=np.float64)[:, 0], L[0])
    w = L[0] / world
    return np.nonzero((x >= rank * w) & (x < (rank + 1) * w))[0]
