"""The learned part: a distilled student trained by the library's own kernels, judged by the full model.

The teacher is the seeded copper model as is: its trajectories stay near
the thermally displaced FCC lattice (scaling a random model's forces up to
~1 eV/A makes its MD unstable).  Its forces are ~1e-5 eV/A, so the force
term of the loss is weighted by 100/RMS(F)^2 (p_e = 1) and the judge threshold is
stated relative to the RMS force.  The test shows what training gains: the
trained student's force error against the teacher on held-out frames is
far below the untrained student's, and in judged MD the untrained student
is rejected at every judgement while the trained one is rejected less.
"""
import numpy as np
import pytest

import dpsynth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    import paper_2005_00223_gb300 as pkg
    pkg.load()
    return pkg


def _teacher(dp):
    cfg = dpsynth.copper_config()
    return dp.Model(cfg, 0, params=dpsynth.model_params(cfg, 1))


def test_student_distillation_and_judge(dp):
    from paper_2005_00223_gb300 import student as S
    coord, typ, box = dpsynth.copper_fcc(1, ncell=10)
    mass = np.array([dpsynth.MASS["Cu"]])
    teacher = _teacher(dp)
    vels = [dpsynth.velocities(mass[typ], T, 10 + k) for k, T in enumerate((300.0, 1200.0))]
    X, E, F = S.teacher_frames(teacher, coord, typ, box, mass, vels, nframes=24, stride=5, dt_fs=1.0)
    test_idx = np.r_[20:24, 44:48]
    train_idx = np.setdiff1d(np.arange(len(X)), test_idx)
    stu = dp.Model(dpsynth.copper_student_config(), seed=2)
    r0, frms = S.force_rmse(stu, teacher, X[test_idx], typ, box)
    log = S.train(stu, typ, box, X[train_idx], E[train_idx], F[train_idx], steps=800, lr0=3e-3, lr1=1e-4,
                  p_e=1.0, p_f=100.0 / frms ** 2)
    r1, _ = S.force_rmse(stu, teacher, X[test_idx], typ, box)
    print(f"RMS F {frms:.4g} eV/A; student force RMSE untrained {r0:.4g} ({r0 / frms:.3f} of RMS F), "
          f"trained {r1:.4g} ({r1 / frms:.3f}); loss log {log[:2]} ... {log[-2:]}")
    assert np.isfinite(r1) and r1 < 0.5 * r0
    # judged MD at 300 K: threshold 10% of the teacher's RMS force at the start;
    # the untrained student is rejected at every judgement
    nl0 = dp.NeighborList(teacher, coord, typ, box)
    F0 = nl0.compute(coord, box, "mix32")[2]
    rmse_max = 0.1 * float(np.sqrt((F0 ** 2).sum(1).mean()))
    fresh = dp.Model(dpsynth.copper_student_config(), seed=2)
    for model, expect_all in ((fresh, True), (stu, False)):
        st = dp.MDState(model, coord, vels[0], typ, mass, box, skin=2.0)
        rm, fb = dp.dp_md_step_judged(model.h, teacher.h, st.h, 60, 1.0, "mix32", "mix32", judge_every=10,
                                      rmse_max=rmse_max)
        print("judged", "untrained" if expect_all else "trained", rm, fb)
        assert len(rm) == 6 and np.isfinite(rm).all()
        if expect_all:
            assert fb.all()
        else:
            assert fb.sum() < len(fb)
