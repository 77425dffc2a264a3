"""Checks of the seeded input generators (dpsynth) against their definitions."""
import math

import numpy as np

import dpsynth


def test_splitmix64_published_vector():
    # first outputs of SplitMix64 seeded with 1234567 (Steele, Lea and Flood 2014 reference code)
    r = dpsynth.SplitMix64(1234567)
    assert [r.next_u64() for _ in range(5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_vectorised_normals_match_scalar_stream():
    a = dpsynth.SplitMix64(99)
    ref = np.array([a.normal() for _ in range(13)])
    b = dpsynth.SplitMix64(99)
    got = np.concatenate([b.normals(3), b.normals(4), b.normals(6)])
    np.testing.assert_allclose(got, ref, rtol=0, atol=4e-16 * np.abs(ref).max())


def test_param_counts():
    assert dpsynth.n_params(dpsynth.water_config()) == 4 * 6450 + 2 * 500161
    assert dpsynth.n_params(dpsynth.copper_config()) == 6450 + 500161
    # student: 8+8 + 8*16+16 + 16*32+32 = 704; 256*64+64 + 2*(64*64+64) + 64+1 = 24,833
    assert dpsynth.n_params(dpsynth.copper_student_config()) == 704 + 24833


def test_weight_variance_is_one_over_fan_in():
    cfg = dpsynth.copper_config()
    p = dpsynth.model_params(cfg, 3)
    off = 6450
    W0 = p[off:off + 1600 * 240]
    assert abs(W0.var() * 1600 - 1.0) < 0.02
    assert abs(W0.mean()) < 0.002


def test_water_geometry():
    coord, typ, box = dpsynth.water_box(5)
    L = box[0, 0]
    assert coord.shape == (192, 3) and (coord >= 0).all() and (coord < L).all()
    assert list(typ[:6]) == [0, 1, 1, 0, 1, 1]

    def mi(a, b):
        d = b - a
        return d - L * np.rint(d / L)

    for m in range(64):
        o, h1, h2 = coord[3 * m], coord[3 * m + 1], coord[3 * m + 2]
        v1, v2 = mi(o, h1), mi(o, h2)
        assert abs(np.linalg.norm(v1) - 0.96) < 1e-12 and abs(np.linalg.norm(v2) - 0.96) < 1e-12
        ang = math.degrees(math.acos(v1 @ v2 / (0.96 * 0.96)))
        assert abs(ang - 104.5) < 1e-9
    ox = coord[0::3]
    for a in range(64):
        for b in range(a + 1, 64):
            assert np.linalg.norm(mi(ox[a], ox[b])) >= 2.5


def test_replicate_order():
    coord, typ, box = dpsynth.water_box(1)
    c2, t2, b2 = dpsynth.replicate(coord, typ, box, (2, 3, 2))
    assert c2.shape == (12 * 192, 3)
    k = ((1 * 3 + 2) * 2 + 1) * 192 + 7
    np.testing.assert_allclose(c2[k], coord[7] + np.array([1, 2, 1]) * 12.42)
    np.testing.assert_allclose(np.diag(b2), [24.84, 37.26, 24.84])


def test_copper_lattice():
    coord, typ, box = dpsynth.copper_fcc(1, ncell=3, sigma=0.0)
    assert coord.shape == (108, 3)
    np.testing.assert_allclose(coord[5], [0.0, 0.5 * 3.634, 0.5 * 3.634 + 3.634], atol=1e-12)


def test_velocities_exact_temperature_and_zero_momentum():
    mass = np.array([15.9994, 1.00794, 1.00794] * 20)
    v = dpsynth.velocities(mass, 300.0, 4)
    np.testing.assert_allclose((mass[:, None] * v).sum(0), 0.0, atol=1e-14)
    ke = 0.5 * dpsynth.MVV2E * (mass[:, None] * v * v).sum()
    assert ke == np.float64(1.5 * (60 - 1) * dpsynth.KB_EV * 300.0) or \
        abs(ke / (1.5 * 59 * dpsynth.KB_EV * 300.0) - 1) < 1e-13


def test_paper_water_model_and_system():
    """The paper's production water model (Sec. 5.1: r_c 6 A, 144 neighbors, embedding 32-64-128,
    fitting 240-240-240) and its 4,096-molecule single-GPU system as the 64-molecule box replicated
    4 x 4 x 4; parameter count from the layer shapes."""
    cfg = dpsynth.water_paper_config()
    assert cfg.rcut == 6.0 and cfg.nsel == 144 and cfg.sel == (48, 96)
    assert cfg.embed == (32, 64, 128) and cfg.fit == (240, 240, 240) and cfg.m2 == 16
    emb = (1 * 32 + 32) + (32 * 64 + 64) + (64 * 128 + 128)
    fit = (128 * 16 * 240 + 240) + 2 * (240 * 240 + 240) + (240 + 1)
    assert dpsynth.n_params(cfg) == 4 * emb + 2 * fit
    c, t, b = dpsynth.water_box(1)
    coord, typ, box = dpsynth.replicate(c, t, b, (4, 4, 4))
    assert coord.shape == (12288, 3) and (typ == 0).sum() == 4096
    np.testing.assert_allclose(np.diag(box), 4 * 12.42)
    # replica k of atom i sits at coord[i] + the replica's box offset
    np.testing.assert_allclose(coord[5 * 192 + 7] - coord[7], [0.0, 12.42, 12.42])   # replica (0, 1, 1)


def test_morse_reference_forces_are_minus_energy_gradient():
    """The Morse copper reference used to fit config 4's teacher: forces are minus the central
    differences of its energy, they sum to zero, the perfect lattice is force free, and the
    shifted-force form takes energy and force of a pair to zero at the cut-off."""
    c, t, b = dpsynth.copper_fcc(3, ncell=5, sigma=0.1)
    E, F = dpsynth.morse_copper(c, b)
    assert np.abs(F.sum(0)).max() < 1e-10
    h = 1e-5
    for i, k in ((7, 0), (123, 1), (401, 2)):
        cp, cm = c.copy(), c.copy()
        cp[i, k] += h
        cm[i, k] -= h
        fd = -(dpsynth.morse_copper(cp, b)[0] - dpsynth.morse_copper(cm, b)[0]) / (2 * h)
        assert abs(fd - F[i, k]) < 1e-6 * max(1.0, abs(F[i, k]))
    c0, _, _ = dpsynth.copper_fcc(3, ncell=5, sigma=0.0)
    assert np.abs(dpsynth.morse_copper(c0, b)[1]).max() < 1e-10
    box = np.diag([30.0, 30.0, 30.0])
    for r in (8.0 - 1e-9, 8.0 + 1e-9):
        pair = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
        e2, f2 = dpsynth.morse_copper(pair, box)
        assert abs(e2) < 1e-12 and np.abs(f2).max() < 1e-9
    frames = dpsynth.morse_frames(4)
    assert frames[0].shape == (4, 500, 3) and frames[2].shape == (4, 500, 3)
