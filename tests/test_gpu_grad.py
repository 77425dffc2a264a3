"""GPU parameter gradient, force-matching loss gradient, Adam, and the autograd.Function, against the oracle."""
import numpy as np
import pytest

import dpsynth
from gpu_common import rms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    import paper_2005_00223_gb300 as pkg
    pkg.load()
    return pkg


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


CASES = [
    ("water192", dpsynth.water_config, lambda: dpsynth.water_box(1)),
    ("cu500", dpsynth.copper_config, lambda: dpsynth.copper_fcc(1, ncell=5)),
    ("student_cu500", dpsynth.copper_student_config, lambda: dpsynth.copper_fcc(2, ncell=5)),
]


@pytest.mark.parametrize("name,cfgf,sysf", CASES, ids=[c[0] for c in CASES])
def test_param_grad_matches_oracle(dp, orc, name, cfgf, sysf):
    cfg = cfgf()
    coord, typ, box = sysf()
    p = dpsynth.model_params(cfg, 5)
    m = dp.Model(cfg, 0, params=p)
    nl = dp.NeighborList(m, coord, typ, box)
    v = np.random.default_rng(3).normal(size=coord.shape)
    E, Ed, g = dp.dp_param_grad(m.h, nl.h, coord, box, v, 0.3, -1.7, "fp64")
    Er, Edr, gr = orc.Model(cfg, p).jvp_grad(coord, typ, box, v, 0.3, -1.7)
    assert E == pytest.approx(Er, rel=1e-10)
    assert Ed == pytest.approx(Edr, rel=1e-9)
    assert _rel(g, gr) < 1e-9, _rel(g, gr)
    # the FP32 gradient (training precision) within FP32 rounding of the FP64 one
    E32, Ed32, g32 = dp.dp_param_grad(m.h, nl.h, coord, box, v, 0.3, -1.7, "mix32")
    print(name, "fp32 grad rel err", _rel(g32, gr))
    assert _rel(g32, gr) < 1e-3


def test_force_loss_grad_matches_oracle_and_fd(dp, orc):
    cfg = dpsynth.water_config()
    p = dpsynth.model_params(cfg, 6)
    rng = np.random.default_rng(4)
    frames = []
    for s in range(4):
        c, t, b = dpsynth.water_box(20 + s)
        frames.append((c, t, b, float(rng.normal()), rng.normal(scale=1e-3, size=c.shape)))
    m = dp.Model(cfg, 0, params=p)
    loss, grad = 0.0, np.zeros(len(p))
    for c, t, b, Eref, Fref in frames:
        nl = dp.NeighborList(m, c, t, b)
        l, _ = dp.dp_force_loss_grad(m.h, nl.h, c, b, Fref, Eref, 0.5, 100.0, "fp64", grad=grad)
        loss += l
    om = orc.Model(cfg, p)
    Lr, gr = om.force_loss_grad(frames, p_e=0.5, p_f=100.0)
    assert loss == pytest.approx(Lr, rel=1e-10)
    assert _rel(grad, gr) < 1e-9
    # central differences of the GPU loss along a few parameters
    idx = rng.choice(len(p), 8, replace=False)

    def gpu_loss(pp):
        mm = dp.Model(cfg, 0, params=pp)
        tot = 0.0
        for c, t, b, Eref, Fref in frames:
            nl = dp.NeighborList(mm, c, t, b)
            E, _, F, _ = nl.compute(c, b, "fp64")
            tot += 0.5 * ((E - Eref) / len(t)) ** 2 + 100.0 * float(((F - Fref) ** 2).sum()) / (3 * len(t))
        return tot

    h = 1e-4
    for q in idx:
        vals = []
        for k in (2, 1, -1, -2):
            pp = p.copy()
            pp[q] += k * h
            vals.append(gpu_loss(pp))
        fd = (-vals[0] + 8 * vals[1] - 8 * vals[2] + vals[3]) / (12 * h)
        assert grad[q] == pytest.approx(fd, rel=1e-5, abs=1e-10)


@pytest.mark.slow
def test_force_loss_grad_32_frames(dp, orc):
    """The 32 seeded 192-atom water frames: GPU FP64 gradient against the oracle."""
    cfg = dpsynth.water_config()
    p = dpsynth.model_params(cfg, 7)
    rng = np.random.default_rng(5)
    m = dp.Model(cfg, 0, params=p)
    frames, grad, loss = [], np.zeros(len(p)), 0.0
    for s in range(32):
        c, t, b = dpsynth.water_box(100 + s)
        fr = (c, t, b, float(rng.normal()), rng.normal(scale=1e-3, size=c.shape))
        frames.append(fr)
        nl = dp.NeighborList(m, c, t, b)
        l, _ = dp.dp_force_loss_grad(m.h, nl.h, c, b, fr[4], fr[3], 1.0, 100.0, "fp64", grad=grad)
        loss += l
    Lr, gr = orc.Model(cfg, p).force_loss_grad(frames, p_e=1.0, p_f=100.0)
    assert loss == pytest.approx(Lr, rel=1e-10)
    assert _rel(grad, gr) < 1e-9


def test_adam_step_matches_definition(dp):
    import torch
    cfg = dpsynth.copper_student_config()
    p = dpsynth.model_params(cfg, 8)
    m = dp.Model(cfg, 0, params=p)
    rng = np.random.default_rng(6)
    mo = np.zeros_like(p)
    ve = np.zeros_like(p)
    ref = p.copy()
    for t in range(1, 4):
        g = rng.normal(size=p.shape)
        dg = torch.tensor(g, dtype=torch.float64, device="cuda")
        dp.dp_adam_step(m.h, dg, 1e-3, 0.9, 0.999, 1e-8, t)
        torch.cuda.synchronize()
        mo = 0.9 * mo + 0.1 * g
        ve = 0.999 * ve + 0.001 * g * g
        ref -= 1e-3 * (mo / (1 - 0.9 ** t)) / (np.sqrt(ve / (1 - 0.999 ** t)) + 1e-8)
    np.testing.assert_allclose(m.params, ref, rtol=1e-12, atol=1e-15)
    dp.dp_model_sync_params(m.h)
    np.testing.assert_allclose(m.params, ref, rtol=1e-12, atol=1e-15)


def test_autograd_function_gives_forces(dp, orc):
    import torch
    from paper_2005_00223_gb300.torch_ops import dp_energy
    cfg = dpsynth.water_config()
    coord, typ, box = dpsynth.water_box(3)
    p = dpsynth.model_params(cfg, 9)
    m = dp.Model(cfg, 0, params=p)
    nl = dp.NeighborList(m, coord, typ, box, skin=1.0)
    x = torch.tensor(coord, dtype=torch.float64, device="cuda", requires_grad=True)
    E, Ei, F, W = dp_energy(m, nl, x, box, "fp64")
    (gx,) = torch.autograd.grad(E, x)
    Er, _, Fr, Wr = orc.Model(cfg, p).compute(coord, typ, box)
    assert float(E.detach()) == pytest.approx(Er, rel=1e-10)
    np.testing.assert_allclose(-gx.cpu().numpy(), Fr, atol=1e-10 * rms(Fr))
    np.testing.assert_allclose(W.detach().cpu().numpy(), Wr, atol=1e-10 * np.abs(Wr).max())
    # mixed precision through the same Function
    E16, _, F16, _ = dp_energy(m, nl, x.detach(), box, "bf16")
    Eir = orc.Model(cfg, p).compute(coord, typ, box)[1]
    assert abs(float(E16.detach()) - Er) < 2 * 2.0 ** -9 * float(np.abs(Eir).sum())


@pytest.mark.slow
def test_water_1p57m_bf16_autograd_sampled(dp, orc):
    """The 1,572,864-atom water box in MIX-16 through the autograd.Function; sampled E_i vs the oracle."""
    import torch
    from paper_2005_00223_gb300.torch_ops import dp_energy
    cfg = dpsynth.water_config()
    c0, t0, b0 = dpsynth.water_box(1)
    coord, typ, box = dpsynth.replicate(c0, t0, b0, (32, 16, 16))
    p = dpsynth.model_params(cfg, 1)
    m = dp.Model(cfg, 0, params=p)
    nl = dp.NeighborList(m, coord, typ, box)
    x = torch.tensor(coord, dtype=torch.float64, device="cuda", requires_grad=True)
    E, Ei, F, W = dp_energy(m, nl, x, box, "bf16")
    (gx,) = torch.autograd.grad(E, x)
    F = F.detach().cpu().numpy()
    Ei = Ei.detach().cpu().numpy()
    assert np.isfinite(F).all() and np.isfinite(Ei).all()
    np.testing.assert_array_equal(-gx.cpu().numpy(), F)
    om = orc.Model(cfg, p)
    nref, _, _ = om.nlist(coord, typ, box)
    np.testing.assert_array_equal(nl.get()[0], nref)
    # periodic replicas of the 192-atom box see identical environments
    Eb, Eib, Fb, _ = om.compute(c0, t0, b0)
    scale = float(np.abs(Eib).max())
    u = 2.0 ** -9                                   # bf16 unit roundoff
    for i in (0, 1, 777, 1572863):
        Ek, _, _ = om.atom(i, nref[i], coord, typ, box)
        assert abs(Ei[i] - Ek) < 4 * u * scale
        assert abs(Ek - Eib[i % 192]) < 1e-9 * abs(Ek)
    assert abs(float(E.detach()) - 8192 * Eb) < 2 * u * 8192 * float(np.abs(Eib).sum())


def test_frames_list_and_batched_loss_gradient(dp, orc):
    """32 water frames in one list: the list is the per-frame lists with offset indices (bit-exact), and one
    batched loss / gradient call equals the sum of the per-frame calls (FP64) and the oracle's."""
    import torch
    cfg = dpsynth.water_config()
    p = dpsynth.model_params(cfg, 7)
    rng = np.random.default_rng(5)
    m = dp.Model(cfg, 0, params=p)
    frames = []
    for s in range(32):
        c, t, b = dpsynth.water_box(100 + s)
        frames.append((c, t, b, float(rng.normal()), rng.normal(scale=1e-3, size=c.shape)))
    typ, box, n = frames[0][1], frames[0][2], len(frames[0][1])
    X = np.array([f[0] for f in frames])
    nlf = dp.NeighborList.frames(m, X, typ, box)
    big, ntr = nlf.get()
    assert ntr == 0
    nsel = sum(cfg.sel)
    for f in range(32):
        nl1 = dp.NeighborList(m, X[f], typ, box)
        one, _ = nl1.get()
        nl1.close()
        exp = np.where(one >= 0, one + f * n, -1)
        np.testing.assert_array_equal(big[f * n:(f + 1) * n].reshape(n, nsel), exp.reshape(n, nsel))
    # batched loss and gradient vs the per-frame host calls
    dev = torch.device("cuda")
    Xd = torch.tensor(X.reshape(-1, 3), device=dev)
    Fd = torch.tensor(np.array([f[4] for f in frames]).reshape(-1, 3), device=dev)
    Ed = torch.tensor([f[3] for f in frames], dtype=torch.float64, device=dev)
    grad = torch.zeros(len(p), dtype=torch.float64, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    dp.dp_model_set_stream(m.h, stream)
    dp.dp_force_loss_grad_dev(m.h, nlf.h, Xd, box, Fd, Ed, 1.0, 100.0, "fp64", loss, grad, stream)
    torch.cuda.synchronize()
    dp.dp_model_set_stream(m.h, None)
    gsum, lsum = np.zeros(len(p)), 0.0
    for f in frames:
        nl1 = dp.NeighborList(m, f[0], typ, box)
        l1, _ = dp.dp_force_loss_grad(m.h, nl1.h, f[0], box, f[4], f[3], 1.0, 100.0, "fp64", grad=gsum)
        lsum += l1
        nl1.close()
    nlf.close()
    assert float(loss.item()) == pytest.approx(lsum, rel=1e-12)
    assert _rel(grad.cpu().numpy(), gsum) < 1e-12
    Lr, gr = orc.Model(cfg, p).force_loss_grad(frames, p_e=1.0, p_f=100.0)
    assert float(loss.item()) == pytest.approx(Lr, rel=1e-10)
    assert _rel(grad.cpu().numpy(), gr) < 1e-9
