"""Pins of the oracle's parameter gradient (the force-matching loss of the training path).

Edot = sum_k v_k . dE/dr_k is pinned by a central finite difference of E
along v; d(alpha E + beta Edot)/dtheta and dL/dtheta of the loss
L = p_e (dE/N)^2 + p_f/(3N) sum |F - F_ref|^2 are pinned by central finite
differences over randomly chosen parameters (at least 50 entries).
"""
import numpy as np
import pytest

import dpsynth


def _small_water():
    cfg = dpsynth.ModelConfig(ntypes=2, rcut=6.0, rcut_smth=0.5, sel=(46, 92), embed=(8, 16, 32), m2=8,
                              fit=(32, 32, 32))
    return cfg, dpsynth.model_params(cfg, 3)


def _fd4(f, p, q, h):
    """Fourth-order central difference of f along parameter q."""
    vals = []
    for k in (2, 1, -1, -2):
        pp = p.copy()
        pp[q] += k * h
        vals.append(f(pp))
    return (-vals[0] + 8 * vals[1] - 8 * vals[2] + vals[3]) / (12 * h)


def test_edot_is_directional_derivative(orc):
    cfg, p = _small_water()
    m = orc.Model(cfg, p)
    c, t, b = dpsynth.water_box(2)
    v = np.random.default_rng(0).normal(size=c.shape)
    E, Ed, _ = m.jvp_grad(c, t, b, v, 0.0, 0.0)
    h = 1e-5
    fd = (m.energy(c + h * v, t, b) - m.energy(c - h * v, t, b)) / (2 * h)
    assert Ed == pytest.approx(fd, rel=1e-6)
    assert E == pytest.approx(m.energy(c, t, b), rel=1e-14)


def test_jvp_grad_matches_finite_differences(orc):
    cfg, p = _small_water()
    c, t, b = dpsynth.water_box(2)
    rng = np.random.default_rng(1)
    v = rng.normal(size=c.shape)
    alpha, beta = 0.3, -1.7
    _, _, g = orc.Model(cfg, p).jvp_grad(c, t, b, v, alpha, beta)
    nl = orc.Model(cfg, p).nlist(c, t, b)[0]

    def f(pp):
        E, Ed, _ = orc.Model(cfg, pp).jvp_grad(c, t, b, v, 0.0, 0.0, nlist=nl)
        return alpha * E + beta * Ed

    idx = rng.choice(len(p), 60, replace=False)
    for q in idx:
        fd = _fd4(f, p, q, 1e-4)
        assert g[q] == pytest.approx(fd, rel=1e-6, abs=1e-11)


def test_force_loss_gradient_matches_finite_differences(orc):
    cfg, p = _small_water()
    rng = np.random.default_rng(2)
    frames = []
    for s in range(2):
        c, t, b = dpsynth.water_box(10 + s)
        E_ref = rng.normal()
        F_ref = rng.normal(scale=1e-3, size=c.shape)
        frames.append((c, t, b, E_ref, F_ref))
    m = orc.Model(cfg, p)
    L, g = m.force_loss_grad(frames, p_e=0.5, p_f=100.0)
    assert L == pytest.approx(m.force_loss(frames, p_e=0.5, p_f=100.0), rel=1e-12)
    idx = rng.choice(len(p), 50, replace=False)
    for q in idx:
        fd = _fd4(lambda pp: orc.Model(cfg, pp).force_loss(frames, 0.5, 100.0), p, q, 1e-4)
        assert g[q] == pytest.approx(fd, rel=1e-6, abs=1e-11)
