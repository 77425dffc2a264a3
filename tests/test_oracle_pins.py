"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check is a closed form,
an invariant of the method (Sec. 2: translation, rotation and permutation
symmetry, smoothness of order 2, E = sum_i E_i with local E_i), a finite
difference, or an O(N^2) brute force written from the neighbor-list rules
of Sec. 4.1.1-4.1.2.  The absolute energy of a seeded random model has no
published value, so it stays unpinned beyond these checks.
"""
import math

import numpy as np
import pytest

import dpsynth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _offsets(cfg):
    out, pos = {}, 0
    for name, shape in dpsynth.param_shapes(cfg):
        cnt = int(np.prod(shape))
        out[name] = (pos, shape)
        pos += cnt
    return out


def _view(params, cfg, name):
    off, shape = _offsets(cfg)[name]
    return params[off:off + int(np.prod(shape))].reshape(shape)


def _cluster(n=6, seed=3, box=40.0, spread=3.2, ntypes=1):
    """Small isolated cluster in the middle of a large periodic box."""
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n:
        p = rng.uniform(-spread, spread, 3)
        if all(np.linalg.norm(p - q) > 1.0 for q in pts):
            pts.append(p)
    coord = np.array(pts) + box / 2
    typ = (np.arange(n) % ntypes).astype(np.int32)
    return coord, typ, np.diag([box, box, box])


def _small_cfg(ntypes=1, rcut=6.0, rcs=1.0, sel=None):
    sel = sel or tuple([24] * ntypes)
    return dpsynth.ModelConfig(ntypes=ntypes, rcut=rcut, rcut_smth=rcs, sel=sel,
                               embed=(4, 8, 16), m2=4, fit=(12, 12, 12))


# ----------------------------------------------------------- switching s(r)

def test_switch_closed_form(orc):
    rcs, rc = 2.0, 8.0
    for r in [0.3, 1.0, 1.999]:
        s, ds = orc.switch(r, rcs, rc)
        assert s == 1.0 / r
        assert ds == pytest.approx(-1.0 / r ** 2, rel=1e-15)
    s, _ = orc.switch(rcs, rcs, rc)
    assert s == pytest.approx(1.0 / rcs, rel=1e-15)
    # u = 1/2: u^3(-6u^2+15u-10)+1 = 1/8 * (-1.5 + 7.5 - 10) + 1 = 1/2
    rm = 0.5 * (rcs + rc)
    assert orc.switch(rm, rcs, rc)[0] == pytest.approx(0.5 / rm, rel=1e-15)
    assert orc.switch(rc, rcs, rc) == (0.0, 0.0)
    assert orc.switch(9.5, rcs, rc) == (0.0, 0.0)


def test_switch_is_c2(orc):
    """s, s' and s'' continuous at r_cs and r_c (Sec. 2: order-2 smoothness)."""
    rcs, rc = 0.5, 6.0
    h = 1e-4

    def d2(r):
        return (orc.switch(r + h, rcs, rc)[0] - 2 * orc.switch(r, rcs, rc)[0] + orc.switch(r - h, rcs, rc)[0]) / h ** 2

    for r0 in (rcs, rc):
        e = 1e-7
        sl, dl = orc.switch(r0 - e, rcs, rc)
        sr, dr = orc.switch(r0 + e, rcs, rc)
        assert abs(sl - sr) < 1e-6
        assert abs(dl - dr) < 1e-5
        assert abs(d2(r0 - 4 * h) - d2(r0 + 4 * h)) < 2e-2 * max(1.0, abs(d2(r0 - 4 * h)))
    for r in np.linspace(0.3, 6.2, 41):
        fd = (orc.switch(r + 1e-6, rcs, rc)[0] - orc.switch(r - 1e-6, rcs, rc)[0]) / 2e-6
        assert orc.switch(r, rcs, rc)[1] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_env_row_closed_form_and_jacobian(orc):
    rcs, rc = 1.0, 6.0
    r = 3.0
    s, _ = orc.switch(r, rcs, rc)
    R, _ = orc.env_row([r, 0.0, 0.0], rcs, rc)
    np.testing.assert_allclose(R, [s, s, 0.0, 0.0], rtol=1e-15)
    rng = np.random.default_rng(0)
    for _ in range(10):
        d = rng.normal(size=3)
        d *= rng.uniform(0.5, 5.9) / np.linalg.norm(d)
        R, J = orc.env_row(d, rcs, rc)
        s, _ = orc.switch(np.linalg.norm(d), rcs, rc)
        assert R @ R == pytest.approx(2 * s * s, rel=1e-13)      # |R|^2 = s^2 (1 + |d|^2/r^2)
        for k in range(3):
            e = np.zeros(3); e[k] = 1e-6
            fd = (orc.env_row(d + e, rcs, rc)[0] - orc.env_row(d - e, rcs, rc)[0]) / 2e-6
            np.testing.assert_allclose(J[:, k], fd, rtol=1e-6, atol=1e-9)


# ------------------------------------------------------------- neighbor list

def _brute_nlist(coord, typ, box, rc, sel):
    """O(N^2) list from the rules of Sec. 4.1.1-4.1.2, in plain Python floats."""
    L = [box[0][0], box[1][1], box[2][2]]
    inv = [1.0 / x for x in L]
    n = len(coord)
    out = np.full((n, sum(sel)), -1, dtype=np.int32)
    ntr = 0
    for i in range(n):
        items = []
        for j in range(n):
            if j == i:
                continue
            d = []
            for k in range(3):
                dk = float(coord[j][k]) - float(coord[i][k])
                d.append(dk - L[k] * float(np.rint(dk * inv[k])))
            r = math.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])
            if r < rc:
                items.append((int(typ[j]), math.floor(r * 1e8), j))
        items.sort()
        off = 0
        for t in range(len(sel)):
            blk = [it for it in items if it[0] == t]
            ntr += max(0, len(blk) - sel[t])
            for k, it in enumerate(blk[:sel[t]]):
                out[i, off + k] = it[2]
            off += sel[t]
    return out, ntr


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_nlist_matches_bruteforce(orc, seed):
    rng = np.random.default_rng(seed)
    n, Lb = 48, 11.0
    coord = rng.uniform(-2, Lb + 2, (n, 3))       # some outside [0, L): min image must wrap
    typ = rng.integers(0, 2, n).astype(np.int32)
    cfg = dpsynth.ModelConfig(ntypes=2, rcut=4.5, rcut_smth=1.0, sel=(6, 9), embed=(4, 8, 16), m2=4,
                              fit=(12, 12, 12))
    m = orc.Model(cfg, dpsynth.model_params(cfg, 1))
    box = np.diag([Lb, Lb + 1.0, Lb + 2.0])
    ref, ntr_ref = _brute_nlist(coord, typ, box, cfg.rcut, cfg.sel)
    for cells in (False, True):
        got, ntr, cnt = m.nlist(coord, typ, box, use_cells=cells)
        np.testing.assert_array_equal(got, ref)
        assert ntr == ntr_ref
    assert ntr_ref > 0   # the sel values are small enough that truncation occurs


def test_nlist_ties_and_exact_cutoff(orc):
    """Equal distances order by index; a neighbor exactly at r_c is excluded."""
    cfg = dpsynth.ModelConfig(ntypes=1, rcut=2.0, rcut_smth=0.5, sel=(8,), embed=(4, 8, 16), m2=4,
                              fit=(12, 12, 12))
    m = orc.Model(cfg, dpsynth.model_params(cfg, 1))
    c0 = np.array([5.0, 5.0, 5.0])
    coord = np.array([c0, c0 + [1.5, 0, 0], c0 - [1.5, 0, 0], c0 + [0, 1.5, 0], c0 + [2.0, 0, 0],
                      c0 + [0, 0, 1.25], c0 - [0, 0, 1.25]])
    typ = np.zeros(7, dtype=np.int32)
    box = np.diag([20.0, 20.0, 20.0])
    nl, ntr, cnt = m.nlist(coord, typ, box)
    # atom 0: 5 and 6 at 1.25 (tie -> index order), then 1, 2, 3 at 1.5; atom 4 at exactly 2.0 excluded
    np.testing.assert_array_equal(nl[0], [5, 6, 1, 2, 3, -1, -1, -1])
    assert cnt[0, 0] == 5 and ntr == 0
    ref, _ = _brute_nlist(coord, typ, box, cfg.rcut, cfg.sel)
    np.testing.assert_array_equal(nl, ref)


def test_nlist_truncation_keeps_nearest(orc):
    cfg = dpsynth.ModelConfig(ntypes=1, rcut=8.0, rcut_smth=2.0, sel=(40,), embed=(4, 8, 16), m2=4,
                              fit=(12, 12, 12))
    m = orc.Model(cfg, dpsynth.model_params(cfg, 1))
    coord, typ, box = dpsynth.copper_fcc(5, ncell=5, sigma=0.1)
    nl, ntr, cnt = m.nlist(coord, typ, box)
    L = box[0, 0]
    for i in (0, 17, 333):
        d = coord - coord[i]
        d -= L * np.rint(d / L)
        r = np.sqrt((d * d).sum(1))
        r[i] = np.inf
        order = np.lexsort((np.arange(len(r)), np.floor(r * 1e8)))
        np.testing.assert_array_equal(nl[i], order[:40])
    assert ntr == int((cnt[:, 0] - 40).clip(min=0).sum())


def test_copper_perfect_lattice_has_176_neighbors(orc):
    """FCC shells 12+6+24+12+24+8+48+6+36 = 176 inside 8 A at a = 3.634 A."""
    cfg = dpsynth.copper_config()
    m = orc.Model(cfg, dpsynth.model_params(cfg, 1))
    coord, typ, box = dpsynth.copper_fcc(1, ncell=5, sigma=0.0)
    nl, ntr, cnt = m.nlist(coord, typ, box)
    assert (cnt[:, 0] == 176).all() and ntr == 0
    assert ((nl >= 0).sum(1) == 176).all()


# ----------------------------------------------------- nets: closed forms

def _constant_embedding(cfg, params, ti, tj):
    """Embedding output when every W of net (ti, tj) is zero: propagate tanh(b)."""
    h = None
    win = 1
    for k, w in enumerate(cfg.embed):
        b = _view(params, cfg, f"embed[{ti},{tj}].b{k}")
        t = np.tanh(b)
        if h is None or (w != win and w != 2 * win):
            h = t
        elif w == win:
            h = h + t
        else:
            h = np.concatenate([h, h]) + t
        win = w
    return h


def _S(orc, cfg, coord, typ, box, row, i):
    """S = sum_j R_j over the real slots of atom i (closed form of the env rows)."""
    L = box[0, 0]
    S = np.zeros(4)
    for j in row:
        if j < 0:
            continue
        d = coord[j] - coord[i]
        d -= L * np.rint(d / L)
        r = np.linalg.norm(d)
        s, _ = orc.switch(r, cfg.rcut_smth, cfg.rcut)
        S += np.array([s, s * d[0] / r, s * d[1] / r, s * d[2] / r])
    return S


def test_descriptor_constant_embedding(orc):
    """Zero embedding weights: G_j = c for all j, so D = c c[:M2]^T |S|^2 / sum(sel)^2."""
    cfg = dpsynth.water_config()
    p = dpsynth.model_params(cfg, 11)
    for ti in range(2):
        for tj in range(2):
            for k in range(3):
                _view(p, cfg, f"embed[{ti},{tj}].W{k}")[:] = 0.0
    m = orc.Model(cfg, p)
    coord, typ, box = dpsynth.water_box(4)
    nl, _, _ = m.nlist(coord, typ, box)
    for i in (0, 1, 50):
        _, _, D = m.atom(i, nl[i], coord, typ, box)
        # one constant row per neighbor type; T = sum_t c_t (x) S_t / nsel
        T = np.zeros((cfg.m1, 4))
        off = 0
        for tj in range(2):
            c = _constant_embedding(cfg, p, typ[i], tj)
            blk = nl[i][off:off + cfg.sel[tj]]
            T += np.outer(c, _S(orc, cfg, coord, typ, box, blk, i))
            off += cfg.sel[tj]
        T /= cfg.nsel
        ref = (T @ T[:cfg.m2].T).reshape(-1)
        np.testing.assert_allclose(D, ref, rtol=1e-12, atol=1e-16)
    # one neighbor type only (copper): closed form in c and |S|^2
    cfg = dpsynth.copper_config()
    p = dpsynth.model_params(cfg, 12)
    for k in range(3):
        _view(p, cfg, f"embed[0,0].W{k}")[:] = 0.0
    m = orc.Model(cfg, p)
    coord, typ, box = dpsynth.copper_fcc(2, ncell=5)
    nl, _, _ = m.nlist(coord, typ, box)
    c = _constant_embedding(cfg, p, 0, 0)
    S = _S(orc, cfg, coord, typ, box, nl[7], 7)
    _, _, D = m.atom(7, nl[7], coord, typ, box)
    ref = np.outer(c, c[:cfg.m2]) * (S @ S) / cfg.nsel ** 2
    np.testing.assert_allclose(D, ref.reshape(-1), rtol=1e-12)


def test_fitting_zero_weights_gives_bias_chain(orc):
    """Zero fitting W: E_i = (y3 . w_out) + b_out with y propagated from tanh(b)."""
    cfg = dpsynth.water_config()
    p = dpsynth.model_params(cfg, 5)
    for ti in range(2):
        for k in range(3):
            _view(p, cfg, f"fit[{ti}].W{k}")[:] = 0.0
    m = orc.Model(cfg, p)
    coord, typ, box = dpsynth.water_box(2)
    E, Ei, F, W = m.compute(coord, typ, box)
    for ti in range(2):
        y1 = np.tanh(_view(p, cfg, f"fit[{ti}].b0"))
        y2 = y1 + np.tanh(_view(p, cfg, f"fit[{ti}].b1"))
        y3 = y2 + np.tanh(_view(p, cfg, f"fit[{ti}].b2"))
        ref = float(y3 @ _view(p, cfg, f"fit[{ti}].W3")[:, 0] + _view(p, cfg, f"fit[{ti}].b3")[0])
        np.testing.assert_allclose(Ei[typ == ti], ref, rtol=1e-13)
    np.testing.assert_allclose(F, 0.0, atol=1e-30)
    assert E == pytest.approx(float(Ei.sum()), rel=1e-14)


def test_one_hot_weights_pin_orientation_and_flattening(orc):
    """One-hot weights fix the W layout (fan_in x fan_out) and D's flat index a*M2 + b.

    Embedding: W1 = W2 = 0, W3 = w e_p e_q^T, so G = c except
    G[q] = h2[q mod 50] + tanh(w h2[p] + b3[q]).  Fitting: W1 has the single
    entry (a*M2 + b, q') = u, W2 = W3 = 0, w_out = e_q', so
    E_i = tanh(b1[q'] + u D[a][b]) + tanh(b2[q']) + tanh(b3[q']) + b_out,
    with D[a][b] = G_a G_b |S|^2 / nsel^2 (one neighbor type).
    """
    cfg = dpsynth.copper_config()
    p = dpsynth.model_params(cfg, 21)
    pe, qe, w = 7, 63, 1.7
    a, b, qf, u = 63, 5, 11, 300.0
    for k in range(3):
        _view(p, cfg, f"embed[0,0].W{k}")[:] = 0.0
    _view(p, cfg, "embed[0,0].W2")[pe, qe] = w
    for k in range(4):
        _view(p, cfg, f"fit[0].W{k}")[:] = 0.0
    _view(p, cfg, "fit[0].W0")[a * cfg.m2 + b, qf] = u
    _view(p, cfg, "fit[0].W3")[qf, 0] = 1.0
    m = orc.Model(cfg, p)
    coord, typ, box = dpsynth.copper_fcc(3, ncell=5)
    nl, _, _ = m.nlist(coord, typ, box)
    h1 = np.tanh(_view(p, cfg, "embed[0,0].b0"))
    h2 = np.concatenate([h1, h1]) + np.tanh(_view(p, cfg, "embed[0,0].b1"))
    b3 = _view(p, cfg, "embed[0,0].b2")
    G = np.concatenate([h2, h2]) + np.tanh(b3)
    G[qe] = h2[qe % 50] + np.tanh(w * h2[pe] + b3[qe])
    for i in (0, 99):
        S = _S(orc, cfg, coord, typ, box, nl[i], i)
        Dab = G[a] * G[b] * (S @ S) / cfg.nsel ** 2
        ref = (np.tanh(_view(p, cfg, "fit[0].b0")[qf] + u * Dab) + np.tanh(_view(p, cfg, "fit[0].b1")[qf])
               + np.tanh(_view(p, cfg, "fit[0].b2")[qf]) + _view(p, cfg, "fit[0].b3")[0])
        Ei, _, D = m.atom(i, nl[i], coord, typ, box)
        assert D[a * cfg.m2 + b] == pytest.approx(Dab, rel=1e-12)
        assert Ei == pytest.approx(ref, rel=1e-12)


def test_embedding_first_layer_two_atoms(orc):
    """Two atoms, one neighbor each: D = 2 s^2 G_a G_b / nsel^2 with the s-dependent first layer.

    Only W1[0][k0] = w is non-zero in the embedding net, so
    h1[k0] = tanh(w s + b1[k0]) and every other channel is a bias constant.
    """
    cfg = dpsynth.ModelConfig(ntypes=1, rcut=6.0, rcut_smth=1.0, sel=(8,))
    p = dpsynth.model_params(cfg, 4)
    for k in range(3):
        _view(p, cfg, f"embed[0,0].W{k}")[:] = 0.0
    k0, w = 9, 2.3
    _view(p, cfg, "embed[0,0].W0")[0, k0] = w
    m = orc.Model(cfg, p)
    box = np.diag([30.0, 30.0, 30.0])
    for r in (0.7, 2.5, 4.0, 5.9):
        coord = np.array([[10.0, 10.0, 10.0], [10.0 + r / math.sqrt(3)] * 3])
        typ = np.zeros(2, dtype=np.int32)
        nl, _, _ = m.nlist(coord, typ, box)
        s, _ = orc.switch(np.linalg.norm(coord[1] - coord[0]), cfg.rcut_smth, cfg.rcut)
        b1 = _view(p, cfg, "embed[0,0].b0").copy()
        h1 = np.tanh(b1)
        h1[k0] = np.tanh(w * s + b1[k0])
        h2 = np.concatenate([h1, h1]) + np.tanh(_view(p, cfg, "embed[0,0].b1"))
        G = np.concatenate([h2, h2]) + np.tanh(_view(p, cfg, "embed[0,0].b2"))
        _, _, D = m.atom(0, nl[0], coord, typ, box)
        ref = 2 * s * s * np.outer(G, G[:cfg.m2]) / cfg.nsel ** 2
        np.testing.assert_allclose(D, ref.reshape(-1), rtol=1e-12)


# ------------------------------------------------- forces, virial, invariants

def _fd_forces(m, coord, typ, box, atoms, h=1e-3):
    out = np.zeros((len(atoms), 3))
    for a, i in enumerate(atoms):
        for k in range(3):
            cp = coord.copy(); cp[i, k] += h
            cm = coord.copy(); cm[i, k] -= h
            cp2 = coord.copy(); cp2[i, k] += 2 * h
            cm2 = coord.copy(); cm2[i, k] -= 2 * h
            # 4th-order central difference
            out[a, k] = -(8 * (m.energy(cp, typ, box) - m.energy(cm, typ, box))
                          - (m.energy(cp2, typ, box) - m.energy(cm2, typ, box))) / (12 * h)
    return out


@pytest.mark.parametrize("system", ["water", "copper"])
def test_forces_are_minus_energy_gradient(orc, system):
    if system == "water":
        cfg = dpsynth.water_config()
        coord, typ, box = dpsynth.water_box(6)
        atoms = [0, 1, 2, 100]
    else:
        cfg = dpsynth.copper_config()
        coord, typ, box = dpsynth.copper_fcc(6, ncell=5)
        atoms = [0, 250]
    p = dpsynth.model_params(cfg, 8)
    for ti in range(cfg.ntypes):
        _view(p, cfg, f"fit[{ti}].W0")[:] *= 100.0     # larger forces relative to E
    m = orc.Model(cfg, p)
    E, Ei, F, W = m.compute(coord, typ, box)
    fd = _fd_forces(m, coord, typ, box, atoms)
    rms = np.sqrt((F ** 2).sum(1).mean())
    np.testing.assert_allclose(F[atoms], fd, atol=1e-6 * rms)
    np.testing.assert_allclose(F.sum(0), 0.0, atol=1e-12 * len(F) * rms)
    assert E == pytest.approx(Ei.sum(), rel=1e-14)


def test_virial_is_minus_strain_derivative(orc):
    """W = -dE/d(eps) under r -> (I + eps) r; symmetric (isolated cluster, all 9 entries)."""
    cfg = _small_cfg(ntypes=2, sel=(20, 20))
    m = orc.Model(cfg, dpsynth.model_params(cfg, 9))
    coord, typ, box = _cluster(n=10, ntypes=2)
    c0 = coord.mean(0)
    E, Ei, F, W = m.compute(coord, typ, box)
    h = 1e-5
    for a in range(3):
        for b in range(3):
            def e_at(eps):
                M = np.eye(3); M[a, b] += eps
                return m.energy((coord - c0) @ M.T + c0, typ, box)
            dEde = (8 * (e_at(h) - e_at(-h)) - (e_at(2 * h) - e_at(-2 * h))) / (12 * h)
            assert W[a, b] == pytest.approx(-dEde, rel=1e-6, abs=1e-9 * np.abs(W).max())
    np.testing.assert_allclose(W, W.T, rtol=1e-10, atol=1e-14)


def test_virial_periodic_diagonal_strain(orc):
    """Diagonal strain of a periodic box (positions and box scaled together)."""
    cfg = dpsynth.water_config()
    m = orc.Model(cfg, dpsynth.model_params(cfg, 10))
    coord, typ, box = dpsynth.water_box(7)
    E, Ei, F, W = m.compute(coord, typ, box)
    h = 1e-5
    for a in range(3):
        def e_at(eps):
            M = np.eye(3); M[a, a] += eps
            return m.energy(coord @ M.T, typ, box @ M.T)
        dEde = (e_at(h) - e_at(-h)) / (2 * h)
        assert W[a, a] == pytest.approx(-dEde, rel=1e-6)


def test_energy_and_force_vanish_smoothly_at_the_cutoff(orc):
    """A neighbor crossing r_c changes E by O(delta^3) and F by O(delta^2) (s is C^2 with
    s = s' = s'' = 0 at r_c, Sec. 2): a list cut-off or switch inconsistent with r_c breaks the scaling."""
    cfg = _small_cfg(ntypes=1, rcut=6.0, rcs=1.0)
    m = orc.Model(cfg, dpsynth.model_params(cfg, 21))
    box = np.diag([60.0, 60.0, 60.0])
    a = np.array([30.0, 30.0, 30.0])
    typ = np.zeros(3, dtype=np.int32)

    def at(r):
        coord = np.array([a, a + [2.0, 0.3, -0.2], a + [-r * 0.8, r * 0.6, 0.0]])
        E, _, F, _ = m.compute(coord, typ, box)
        return E, F

    E_out, F_out = at(cfg.rcut + 1e-3)
    E_out2, F_out2 = at(cfg.rcut + 0.3)
    assert E_out == E_out2 and np.array_equal(F_out, F_out2)      # outside: no interaction at all
    assert np.all(F_out[2] == 0.0)
    dE = {d: at(cfg.rcut - d)[0] - E_out for d in (1e-1, 1e-2)}   # 1e-3 would be near E's rounding
    dF = {d: np.abs(at(cfg.rcut - d)[1][2]).max() for d in (1e-1, 1e-2, 1e-3)}
    assert abs(dE[1e-1]) > 1e-12                                  # the neighbor does interact
    assert 900 < dE[1e-1] / dE[1e-2] < 1100                       # cubic
    for big, small in ((1e-1, 1e-2), (1e-2, 1e-3)):
        assert 90 < dF[big] / dF[small] < 110                     # quadratic


@pytest.mark.parametrize("reps", [(2, 1, 1), (1, 1, 3)])
def test_periodic_replica_is_extensive(orc, reps):
    """Box edges >= 2 r_c: every replica of an atom sees the same images, so in the replicated
    (non-cubic) box E and W scale by the replica count and F repeats; a minimum image taken along
    the wrong edge, or a missed image, breaks it."""
    cfg = dpsynth.copper_config()
    m = orc.Model(cfg, dpsynth.model_params(cfg, 22))
    coord, typ, box = dpsynth.copper_fcc(23, ncell=5)
    assert box[0, 0] >= 2 * cfg.rcut
    E, Ei, F, W = m.compute(coord, typ, box)
    c2, t2, b2 = dpsynth.replicate(coord, typ, box, reps)
    E2, Ei2, F2, W2 = m.compute(c2, t2, b2)
    k = int(np.prod(reps))
    assert E2 == pytest.approx(k * E, rel=1e-12)
    np.testing.assert_allclose(Ei2, np.tile(Ei, k), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(F2, np.tile(F, (k, 1)), rtol=0, atol=1e-12 * np.abs(F).max())
    np.testing.assert_allclose(W2, k * W, rtol=1e-11, atol=1e-12 * np.abs(W).max())


def test_translation_invariance(orc):
    cfg = dpsynth.water_config()
    m = orc.Model(cfg, dpsynth.model_params(cfg, 13))
    coord, typ, box = dpsynth.water_box(8)
    E0, _, F0, _ = m.compute(coord, typ, box)
    shifted = coord + np.array([3.3, -17.1, 5.55])
    shifted -= 12.42 * np.floor(shifted / 12.42)
    E1, _, F1, _ = m.compute(shifted, typ, box)
    assert E1 == pytest.approx(E0, rel=1e-12)
    np.testing.assert_allclose(F1, F0, atol=1e-10 * np.abs(F0).max())


def test_rotation_invariance(orc):
    cfg = _small_cfg(ntypes=2, sel=(20, 20))
    m = orc.Model(cfg, dpsynth.model_params(cfg, 14))
    coord, typ, box = _cluster(n=12, ntypes=2, seed=5)
    E0, _, F0, _ = m.compute(coord, typ, box)
    th = 0.7
    Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, math.cos(1.1), -math.sin(1.1)], [0, math.sin(1.1), math.cos(1.1)]])
    Q = Rz @ Rx
    c0 = coord.mean(0)
    E1, _, F1, _ = m.compute((coord - c0) @ Q.T + c0, typ, box)
    assert E1 == pytest.approx(E0, rel=1e-12)
    np.testing.assert_allclose(F1, F0 @ Q.T, atol=1e-10 * np.abs(F0).max())


def test_permutation_invariance(orc):
    cfg = dpsynth.water_config()
    m = orc.Model(cfg, dpsynth.model_params(cfg, 15))
    coord, typ, box = dpsynth.water_box(9)
    E0, Ei0, F0, _ = m.compute(coord, typ, box)
    rng = np.random.default_rng(1)
    perm = np.arange(len(typ))
    for t in (0, 1):
        idx = np.where(typ == t)[0]
        perm[idx] = rng.permutation(idx)
    E1, Ei1, F1, _ = m.compute(coord[perm], typ[perm], box)
    assert E1 == pytest.approx(E0, rel=1e-12)
    np.testing.assert_allclose(Ei1, Ei0[perm], rtol=1e-11)
    np.testing.assert_allclose(F1, F0[perm], atol=1e-10 * np.abs(F0).max())


def test_locality_and_decomposition(orc):
    """E_i depends only on atoms inside r_c of i (Sec. 2: local decomposition)."""
    cfg = dpsynth.copper_config()
    m = orc.Model(cfg, dpsynth.model_params(cfg, 16))
    coord, typ, box = dpsynth.copper_fcc(4, ncell=5)
    _, Ei0, _, _ = m.compute(coord, typ, box)
    L = box[0, 0]
    d = coord - coord[0]
    d -= L * np.rint(d / L)
    far = np.where(np.sqrt((d ** 2).sum(1)) > cfg.rcut + 0.5)[0][0]
    moved = coord.copy()
    moved[far] += [0.2, -0.1, 0.05]
    _, Ei1, _, _ = m.compute(moved, typ, box)
    assert Ei1[0] == Ei0[0]


# ---------------------------------------------------------------------- MD

def _md_cfg():
    return dpsynth.ModelConfig(ntypes=2, rcut=6.0, rcut_smth=0.5, sel=(46, 92), embed=(8, 16, 32), m2=8,
                               fit=(32, 32, 32))


def test_md_free_flight_closed_form(orc):
    """Zero fitting weights: F = 0, so x(t) = x0 + v t (wrapped), T and P stay at their ideal-gas values."""
    cfg = _md_cfg()
    p = dpsynth.model_params(cfg, 17)
    for ti in range(2):
        for k in range(4):
            _view(p, cfg, f"fit[{ti}].W{k}")[:] = 0.0
    m = orc.Model(cfg, p)
    coord, typ, box = dpsynth.water_box(10)
    mass = np.array([dpsynth.MASS["O"], dpsynth.MASS["H"]])
    vel = dpsynth.velocities(mass[typ], 300.0, 10)
    x, v, th = m.md_nve(coord, vel, typ, mass, box, nsteps=20, dt=0.5, thermo_every=10)
    L = box[0, 0]
    xr = coord + 20 * 0.5 * vel
    xr -= L * np.floor(xr / L)
    np.testing.assert_allclose(x, xr, atol=1e-11)
    np.testing.assert_array_equal(v, vel)
    n = len(typ)
    ke = 1.5 * (n - 1) * dpsynth.KB_EV * 300.0
    np.testing.assert_allclose(th[:, 0], ke, rtol=1e-12)
    np.testing.assert_allclose(th[:, 2], 300.0, rtol=1e-12)
    pressure = 2 * ke / (3 * L ** 3) * 1.602176634e6
    np.testing.assert_allclose(th[:, 3], pressure, rtol=1e-12)


def test_md_pressure_is_minus_volume_derivative(orc):
    """At rest the thermo pressure is -dE/dV (isotropic scaling of positions and box), in bar."""
    cfg = _md_cfg()
    p = dpsynth.model_params(cfg, 19)
    for ti in range(2):
        _view(p, cfg, f"fit[{ti}].W3")[:] *= 2000.0      # forces and virial well above rounding
    m = orc.Model(cfg, p)
    coord, typ, box = dpsynth.water_box(11)
    mass = np.array([dpsynth.MASS["O"], dpsynth.MASS["H"]])
    # one step of 1e-7 fs from rest: KE and the displacement are O(dt^2), far below the tolerance
    _, _, th = m.md_nve(coord, np.zeros_like(coord), typ, mass, box, nsteps=1, dt=1e-7, thermo_every=1)
    V = np.linalg.det(box)
    h = 1e-5

    def e_at(eps):
        return m.energy(coord * (1 + eps), typ, box * (1 + eps))

    dEdV = (8 * (e_at(h) - e_at(-h)) - (e_at(2 * h) - e_at(-2 * h))) / (12 * h) / (3 * V)
    assert abs(dEdV) * 1.602176634e6 > 1.0                        # a pressure of more than 1 bar
    assert th[0, 3] == pytest.approx(-dEdV * 1.602176634e6, rel=1e-6)


@pytest.mark.slow
def test_md_energy_error_scales_as_dt2(orc):
    """Velocity Verlet: the max total-energy deviation over a fixed time shrinks ~4x when dt halves."""
    cfg = _md_cfg()
    p = dpsynth.model_params(cfg, 18)
    for ti in range(2):
        _view(p, cfg, f"fit[{ti}].W3")[:] *= 2000.0      # strong forces: O(1) eV/A
        _view(p, cfg, f"fit[{ti}].b3")[:] *= 2000.0
    m = orc.Model(cfg, p)
    coord, typ, box = dpsynth.water_box(11)
    mass = np.array([dpsynth.MASS["O"], dpsynth.MASS["H"]])
    vel = dpsynth.velocities(mass[typ], 300.0, 11)
    E0, _, F0, _ = m.compute(coord, typ, box)
    ke0 = 0.5 * dpsynth.MVV2E * float((mass[typ][:, None] * vel ** 2).sum())
    assert np.sqrt((F0 ** 2).sum(1).mean()) > 0.3
    dev = []
    for dt in (0.4, 0.2, 0.1):
        steps = int(round(4.0 / dt))
        _, _, th = m.md_nve(coord, vel, typ, mass, box, nsteps=steps, dt=dt, thermo_every=1)
        etot = th[:, 0] + th[:, 1]
        dev.append(np.abs(etot - (E0 + ke0)).max())
    r1, r2 = dev[0] / dev[1], dev[1] / dev[2]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0, dev
