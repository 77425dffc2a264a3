"""Seeded synthetic inputs for the DeepPot-SE energy/force engine.

This module holds only input generation: model hyper-parameters, seeded
weights, atomic geometries (water, FCC copper) and Maxwell-Boltzmann
velocities.  It contains none of the method's arithmetic (no neighbor
search, switching function, network evaluation or force), so both the CUDA
library and the CPU oracle can take their inputs from here without sharing
any of the computation they are compared on.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014) turned into
53-bit uniforms (top 53 bits times 2**-53) and into normals by the
Box-Muller transform, cosine branch first, then the sine branch of the
same pair.  The CUDA library's ``dp_model_create`` implements the same
published generator on its own side, so seeded weights agree without
either side calling the other.

Workloads follow the paper's benchmark systems (water and copper, Sec. 5.1
"Physical systems"): a 64-molecule water box and FCC copper supercells.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

__all__ = [
    "SplitMix64", "ModelConfig", "water_config", "copper_config",
    "copper_student_config", "param_shapes", "n_params", "model_params", "scale_output",
    "water_box", "replicate", "copper_fcc", "velocities", "MASS",
    "KB_EV", "MVV2E", "morse_copper", "MORSE_CU", "morse_frames",
]

# Boltzmann constant in eV/K and the factor that turns amu*A^2/fs^2 into eV
# (1 eV / (A amu) = 9.648533212e-3 A/fs^2).
KB_EV = 8.617333262e-5
MVV2E = 1.0 / 9.648533212e-3
# Atomic masses in amu: O, H (water types 0, 1) and Cu (copper type 0).
MASS = {"O": 15.9994, "H": 1.00794, "Cu": 63.546}

_M64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 stream: state += golden gamma; output is the mix64 finaliser."""

    GAMMA = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.state = seed & _M64
        self._spare = None

    def next_u64(self) -> int:
        self.state = (self.state + self.GAMMA) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1): the top 53 bits of one output."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def normal(self) -> float:
        """Standard normal by Box-Muller; cosine value first, sine value next."""
        if self._spare is not None:
            v, self._spare = self._spare, None
            return v
        u1 = self.uniform()
        u2 = self.uniform()
        rad = math.sqrt(-2.0 * math.log(1.0 - u1))
        ang = 2.0 * math.pi * u2
        self._spare = rad * math.sin(ang)
        return rad * math.cos(ang)

    def normals(self, count: int) -> np.ndarray:
        """`count` successive normals of this stream (vectorised `normal`).

        SplitMix64 is counter based: output k of the stream is the
        finaliser applied to seed + k * gamma, so a block of outputs is
        computed at once with wrapping uint64 arithmetic.
        """
        out = np.empty(count, dtype=np.float64)
        k = 0
        if self._spare is not None and count > 0:
            out[0], self._spare = self._spare, None
            k = 1
        rest = count - k
        npair = (rest + 1) // 2
        if npair:
            idx = np.arange(1, 2 * npair + 1, dtype=np.uint64)
            with np.errstate(over="ignore"):
                z = np.uint64(self.state) + idx * np.uint64(self.GAMMA)
                z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
                z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
                z = z ^ (z >> np.uint64(31))
            self.state = (self.state + 2 * npair * self.GAMMA) & _M64
            u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
            u1, u2 = u[0::2], u[1::2]
            rad = np.sqrt(-2.0 * np.log(1.0 - u1))
            ang = 2.0 * math.pi * u2
            pair = np.empty(2 * npair)
            pair[0::2] = rad * np.cos(ang)
            pair[1::2] = rad * np.sin(ang)
            out[k:] = pair[:rest]
            if rest % 2:
                self._spare = float(pair[-1])
        return out


@dataclasses.dataclass(frozen=True)
class ModelConfig:
    """DeepPot-SE (se_a) hyper-parameters.

    ntypes     number of atom types
    rcut       cut-off radius r_c in A
    rcut_smth  start of the smooth switching region r_cs in A
    sel        per-type maximal neighbor counts (padding size of each block)
    embed      embedding-net widths after the 1-wide input
    m2         axis neurons: number of leading embedding channels in D
    fit        fitting-net hidden widths (the output layer is width 1)
    """

    ntypes: int
    rcut: float
    rcut_smth: float
    sel: Tuple[int, ...]
    embed: Tuple[int, ...] = (25, 50, 100)
    m2: int = 16
    fit: Tuple[int, ...] = (240, 240, 240)

    @property
    def nsel(self) -> int:
        return int(sum(self.sel))

    @property
    def m1(self) -> int:
        return int(self.embed[-1])


def water_config() -> ModelConfig:
    """Water model: r_c 6 A, r_cs 0.5 A, sel O 46 / H 92, nets (25,50,100) and (240,240,240)."""
    return ModelConfig(ntypes=2, rcut=6.0, rcut_smth=0.5, sel=(46, 92))


def water_paper_config() -> ModelConfig:
    """The paper's production water model (Sec. 5.1): r_c 6 A, 144 neighbors in all (read as O 48 /
    H 96, the 1:2 split of the atom counts), embedding (32,64,128), fitting (240,240,240); r_cs 0.5 A
    as in the water config."""
    return ModelConfig(ntypes=2, rcut=6.0, rcut_smth=0.5, sel=(48, 96), embed=(32, 64, 128))


def copper_config() -> ModelConfig:
    """Copper model: r_c 8 A, r_cs 2 A, sel 512, same net shapes, one type."""
    return ModelConfig(ntypes=1, rcut=8.0, rcut_smth=2.0, sel=(512,))


def copper_student_config() -> ModelConfig:
    """Distilled copper student: embedding (8,16,32), M2 8, fitting (64,64,64)."""
    return ModelConfig(ntypes=1, rcut=8.0, rcut_smth=2.0, sel=(512,),
                       embed=(8, 16, 32), m2=8, fit=(64, 64, 64))


def param_shapes(cfg: ModelConfig) -> List[Tuple[str, Tuple[int, ...]]]:
    """Flat parameter order of a model.

    Embedding nets come first, one per (center type, neighbor type) pair in
    row-major pair order; then one fitting net per center type.  Inside a
    net the layers follow in order, each as W (fan_in x fan_out, row-major)
    followed by b (fan_out).
    """
    out = []
    widths_e = [1] + list(cfg.embed)
    for ti in range(cfg.ntypes):
        for tj in range(cfg.ntypes):
            for k in range(len(cfg.embed)):
                out.append((f"embed[{ti},{tj}].W{k}", (widths_e[k], widths_e[k + 1])))
                out.append((f"embed[{ti},{tj}].b{k}", (widths_e[k + 1],)))
    widths_f = [cfg.m1 * cfg.m2] + list(cfg.fit) + [1]
    for ti in range(cfg.ntypes):
        for k in range(len(widths_f) - 1):
            out.append((f"fit[{ti}].W{k}", (widths_f[k], widths_f[k + 1])))
            out.append((f"fit[{ti}].b{k}", (widths_f[k + 1],)))
    return out


def n_params(cfg: ModelConfig) -> int:
    return int(sum(int(np.prod(s)) for _, s in param_shapes(cfg)))


def model_params(cfg: ModelConfig, seed: int) -> np.ndarray:
    """Seeded weights: every W and b entry drawn N(0, 1/fan_in), in flat order."""
    rng = SplitMix64(seed)
    out = np.empty(n_params(cfg), dtype=np.float64)
    pos = 0
    for _name, shape, fan_in in _shapes_with_fan_in(cfg):
        cnt = int(np.prod(shape))
        out[pos:pos + cnt] = rng.normals(cnt) * math.sqrt(1.0 / fan_in)
        pos += cnt
    return out


def scale_output(cfg: ModelConfig, params: np.ndarray, lam: float) -> np.ndarray:
    """Copy of params with every fitting net's output layer (W and b) multiplied by lam.

    A documented global output scale: energies, forces and virials of the
    model scale by lam, so a random-weight model can be given forces of a
    chosen magnitude (e.g. an RMS force of 1 eV/A).
    """
    out = np.array(params, dtype=np.float64, copy=True)
    last = len(cfg.fit)
    pos = 0
    for name, shape in param_shapes(cfg):
        cnt = int(np.prod(shape))
        if name.startswith("fit[") and (name.endswith(f".W{last}") or name.endswith(f".b{last}")):
            out[pos:pos + cnt] *= lam
        pos += cnt
    return out


def _shapes_with_fan_in(cfg: ModelConfig):
    shapes = param_shapes(cfg)
    out = []
    for k in range(0, len(shapes), 2):
        (nw, sw), (nb, sb) = shapes[k], shapes[k + 1]
        out.append((nw, sw, sw[0]))
        out.append((nb, sb, sw[0]))
    return out


def _wrap(x: np.ndarray, box_len: np.ndarray) -> np.ndarray:
    return x - box_len * np.floor(x / box_len)


def _quat_uniform(rng: SplitMix64) -> np.ndarray:
    """Uniform random unit quaternion (Shoemake 1992) from three uniforms."""
    u1, u2, u3 = rng.uniform(), rng.uniform(), rng.uniform()
    a, b = math.sqrt(1.0 - u1), math.sqrt(u1)
    return np.array([a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2),
                     b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3)])


def _quat_rot(q: np.ndarray) -> np.ndarray:
    x, y, z, w = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def water_box(seed: int, nmol: int = 64, box_len: float = 12.42,
              min_oo: float = 2.5, r_oh: float = 0.96, hoh_deg: float = 104.5):
    """Water box: O uniform with min-image O-O >= min_oo, H at r_oh, angle HOH.

    All oxygens are placed first (rejection sampling, three uniforms per
    trial), then each molecule draws one uniform random orientation.  Atom
    order is (O, H, H) per molecule; types O = 0, H = 1; coordinates are
    wrapped into [0, L).  Returns (coord[n,3], type[n], box[3,3]).
    """
    rng = SplitMix64(seed + 1)
    L = float(box_len)
    oxy = []
    while len(oxy) < nmol:
        p = np.array([rng.uniform() * L, rng.uniform() * L, rng.uniform() * L])
        ok = True
        for q in oxy:
            d = p - q
            d -= L * np.round(d / L)
            if float(np.dot(d, d)) < min_oo * min_oo:
                ok = False
                break
        if ok:
            oxy.append(p)
    half = math.radians(hoh_deg) / 2.0
    h_local = np.array([[r_oh * math.sin(half), 0.0, r_oh * math.cos(half)],
                        [-r_oh * math.sin(half), 0.0, r_oh * math.cos(half)]])
    coord = np.empty((3 * nmol, 3))
    typ = np.empty(3 * nmol, dtype=np.int32)
    for m in range(nmol):
        rot = _quat_rot(_quat_uniform(rng))
        coord[3 * m] = oxy[m]
        coord[3 * m + 1] = oxy[m] + rot @ h_local[0]
        coord[3 * m + 2] = oxy[m] + rot @ h_local[1]
        typ[3 * m] = 0
        typ[3 * m + 1:3 * m + 3] = 1
    coord = _wrap(coord, np.full(3, L))
    return coord, typ, np.diag([L, L, L]).astype(np.float64)


def replicate(coord, typ, box, reps: Sequence[int]):
    """Periodic replication: atom index ((ix*ry + iy)*rz + iz)*n + local."""
    n = coord.shape[0]
    Lx, Ly, Lz = box[0, 0], box[1, 1], box[2, 2]
    rx, ry, rz = reps
    out = np.empty((rx * ry * rz * n, 3))
    tout = np.empty(rx * ry * rz * n, dtype=np.int32)
    for ix in range(rx):
        for iy in range(ry):
            for iz in range(rz):
                b = ((ix * ry + iy) * rz + iz) * n
                out[b:b + n] = coord + np.array([ix * Lx, iy * Ly, iz * Lz])
                tout[b:b + n] = typ
    return out, tout, np.diag([rx * Lx, ry * Ly, rz * Lz]).astype(np.float64)


def copper_fcc(seed: int, ncell: int = 10, a: float = 3.634, sigma: float = 0.1):
    """FCC copper: cells in (ix, iy, iz) order, 4 basis atoms each, N(0, sigma^2) noise.

    Returns (coord[n,3] wrapped into [0, L), type[n] (all 0), box[3,3]).
    """
    rng = SplitMix64(seed + 1)
    basis = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
    n = 4 * ncell ** 3
    coord = np.empty((n, 3))
    k = 0
    for ix in range(ncell):
        for iy in range(ncell):
            for iz in range(ncell):
                for b in range(4):
                    coord[k] = (np.array([ix, iy, iz]) + basis[b]) * a
                    k += 1
    noise = rng.normals(3 * n).reshape(n, 3) * sigma
    L = ncell * a
    coord = _wrap(coord + noise, np.full(3, L))
    return coord, np.zeros(n, dtype=np.int32), np.diag([L, L, L]).astype(np.float64)


def velocities(mass: np.ndarray, temperature: float, seed: int) -> np.ndarray:
    """Maxwell-Boltzmann velocities in A/fs at `temperature` K.

    Each component is N(0, k_B T / m); the centre-of-mass velocity is
    removed; the result is rescaled to exactly `temperature` with 3N-3
    degrees of freedom.
    """
    rng = SplitMix64(seed + 2)
    n = mass.shape[0]
    sig = np.sqrt(KB_EV * temperature / (mass * MVV2E))
    v = rng.normals(3 * n).reshape(n, 3) * sig[:, None]
    vcm = (mass[:, None] * v).sum(0) / mass.sum()
    v -= vcm
    ke = 0.5 * MVV2E * float((mass[:, None] * v * v).sum())
    t_now = 2.0 * ke / ((3 * n - 3) * KB_EV)
    if t_now > 0:
        v *= math.sqrt(temperature / t_now)
    return v


# Morse pair potential of copper, V(r) = D (exp(-2 a (r - r0)) - 2 exp(-a (r - r0))), with the
# parameters of Girifalco and Weizer, "Application of the Morse potential function to cubic metals",
# Phys. Rev. 114, 687 (1959): D in eV, a in 1/A, r0 in A.
MORSE_CU = {"D": 0.3429, "a": 1.3588, "r0": 2.866}


def morse_copper(coord: np.ndarray, box: np.ndarray, rcut: float = 8.0, chunk: int = 256):
    """Energy (eV) and forces (eV/A) of copper under the Morse pair potential, shifted-force at rcut.

    A classical reference for labels only: a stand-in for the first-principles data the paper's
    models are fitted to, used to fit the full copper model once so that its own MD stays a crystal
    (a seeded random-weight model has no stable lattice).  It is not part of the method.  Pairs under
    the minimum image of the orthorhombic box; V_sf(r) = V(r) - V(rc) - (r - rc) V'(rc) for r < rc,
    so energy and force both vanish at rc.  Rows of `chunk` atoms at a time (O(n^2) pairs).
    """
    D, a, r0 = MORSE_CU["D"], MORSE_CU["a"], MORSE_CU["r0"]
    x = np.asarray(coord, dtype=np.float64)
    n = x.shape[0]
    L = np.diag(np.asarray(box, dtype=np.float64))

    def v_dv(r):
        e1 = np.exp(-a * (r - r0))
        return D * (e1 * e1 - 2.0 * e1), -2.0 * a * D * (e1 * e1 - e1)

    vc, dvc = v_dv(np.float64(rcut))
    energy = 0.0
    force = np.zeros((n, 3))
    for i0 in range(0, n, chunk):
        i1 = min(n, i0 + chunk)
        d = x[None, :, :] - x[i0:i1, None, :]          # r_j - r_i
        d -= L * np.rint(d / L)
        r = np.sqrt((d * d).sum(-1))
        idx = np.arange(i0, i1)
        r[idx - i0, idx] = np.inf
        m = r < rcut
        rr = np.where(m, r, rcut)
        v, dv = v_dv(rr)
        vsf = np.where(m, v - vc - (rr - rcut) * dvc, 0.0)
        dvsf = np.where(m, dv - dvc, 0.0)
        energy += 0.5 * float(vsf.sum())
        # dE/dr_i = sum_j V'(r_ij) (r_i - r_j) / r_ij, F_i = -dE/dr_i
        force[i0:i1] = ((dvsf / rr)[:, :, None] * d).sum(1)
    return energy, force


def morse_frames(nframes: int, seed: int = 100, ncell: int = 5, sigma_min: float = 0.02, sigma_max: float = 0.18):
    """Labelled copper frames for fitting a model to the Morse reference (morse_copper).

    Frame k is the FCC supercell of `ncell`^3 cells (a = 3.634 A) with seeded N(0, sigma_k^2)
    displacements, sigma_k spread over [sigma_min, sigma_max] by the golden-ratio sequence (about
    the thermal displacements of a copper crystal from 50 K to 2,000 K).  Returns (coords [F, n, 3],
    energies [F], forces [F, n, 3], types [n], box [3, 3]).
    """
    xs, es, fs = [], [], []
    typ = box = None
    for k in range(nframes):
        sig = sigma_min + (sigma_max - sigma_min) * ((k * 0.6180339887498949) % 1.0)
        c, typ, box = copper_fcc(seed + k, ncell=ncell, sigma=sig)
        e, f = morse_copper(c, box)
        xs.append(c)
        es.append(e)
        fs.append(f)
    return np.array(xs), np.array(es), np.array(fs), typ, box
