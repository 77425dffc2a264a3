"""GPU velocity-Verlet NVE (dp_md_step) against the oracle's integrator."""
import numpy as np
import pytest

import dpsynth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    import paper_2005_00223_gb300 as pkg
    pkg.load()
    return pkg


def _scaled_water_model(seed):
    """Water model with the output layer scaled so forces are O(1) eV/A (an input choice)."""
    cfg = dpsynth.water_config()
    p = dpsynth.model_params(cfg, seed)
    off = 0
    for name, shape in dpsynth.param_shapes(cfg):
        cnt = int(np.prod(shape))
        if name.startswith("fit[") and (name.endswith(".W3") or name.endswith(".b3")):
            p[off:off + cnt] *= 1000.0
        off += cnt
    return cfg, p


@pytest.mark.parametrize("skin,route", [(2.0, "auto"), (0.05, "auto"), (2.0, "split")])
def test_nve_matches_oracle(dp, orc, skin, route):
    """route split: the FP64 tensor-core split products forced on for this 192-atom box."""
    import os
    cfg, p = _scaled_water_model(5)
    coord, typ, box = dpsynth.water_box(5)
    mass = np.array([dpsynth.MASS["O"], dpsynth.MASS["H"]])
    vel = dpsynth.velocities(mass[typ], 600.0, 5)
    m = dp.Model(cfg, 0, params=p)
    st = dp.MDState(m, coord, vel, typ, mass, box, skin=skin)
    if route == "split":
        os.environ["DP_OZ_MIN_ATOMS"] = "0"
    try:
        th = st.step(20, 0.5, "fp64", thermo_every=5)
    finally:
        os.environ.pop("DP_OZ_MIN_ATOMS", None)
    x, v, step, nreb = st.get()
    xr, vr, thr = orc.Model(cfg, p).md_nve(coord, vel, typ, mass, box, nsteps=20, dt=0.5, thermo_every=5)
    assert step == 20
    if skin < 0.1:
        assert nreb > 1          # the list was rebuilt on the device during the run
    d = x - xr
    d -= box[0, 0] * np.rint(d / box[0, 0])
    assert np.abs(d).max() < 1e-9
    np.testing.assert_allclose(v, vr, rtol=0, atol=1e-9 * np.abs(vr).max())
    np.testing.assert_allclose(th, thr, rtol=1e-9)


def test_fixed_interval_rebuilds_match_oracle(dp, orc):
    """The paper's protocol (a list rebuild every N steps, Sec. 5.1) on top of the displacement
    criterion: copper at 300 K moves far less than skin/2 in 20 fs, so the extra rebuilds are exactly
    those of the interval, and the trajectory still matches the oracle's."""
    cfg = dpsynth.copper_config()
    coord, typ, box = dpsynth.copper_fcc(1, ncell=5)
    mass = np.array([dpsynth.MASS["Cu"]])
    vel = dpsynth.velocities(mass[typ], 300.0, 5)
    p = dpsynth.model_params(cfg, 1)
    m = dp.Model(cfg, 0, params=p)
    counts = []
    for every in (0, 5):
        st = dp.MDState(m, coord, vel, typ, mass, box, skin=2.0)
        st.rebuild_every(every)
        st.step(3, 1.0, "fp64")      # direct step, capture, replays
        st.step(17, 1.0, "fp64")
        x, v, step, nreb = st.get()
        counts.append(nreb)
        st.close()
    assert counts[1] - counts[0] == 4   # steps 5, 10, 15, 20
    xr, vr, _ = orc.Model(cfg, p).md_nve(coord, vel, typ, mass, box, nsteps=20, dt=1.0, thermo_every=20)
    d = x - xr
    d -= box[0, 0] * np.rint(d / box[0, 0])
    assert np.abs(d).max() < 1e-9
    np.testing.assert_allclose(v, vr, rtol=0, atol=1e-9 * np.abs(vr).max())
    with pytest.raises(dp.DPError):
        dp.dp_md_set_rebuild_every(None, 5)


def test_nve_energy_conservation_copper(dp):
    """Copper 4,000 atoms, 300 K: total energy drift small against KE fluctuations."""
    cfg = dpsynth.copper_config()
    coord, typ, box = dpsynth.copper_fcc(1, ncell=10)
    mass = np.array([dpsynth.MASS["Cu"]])
    vel = dpsynth.velocities(mass[typ], 300.0, 1)
    m = dp.Model(cfg, 1, params=dpsynth.model_params(cfg, 1))
    st = dp.MDState(m, coord, vel, typ, mass, box, skin=2.0)
    th = st.step(100, 1.0, "fp64", thermo_every=10)
    etot = th[:, 0] + th[:, 1]
    assert np.isfinite(th).all()
    assert np.abs(etot - etot[0]).max() < 1e-3 * np.abs(th[:, 0]).mean()


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_graph_replay_matches_direct_launches(dp, prec):
    """Steps replayed from one captured step (CUDA graph) against the same steps launched one by one
    (DP_NO_GRAPH): same trajectory, same rebuilds, same per-group launch counts under profiling;
    the second call reuses the capture and the profiling switch forces a new one."""
    import os
    cfg, p = _scaled_water_model(5)
    coord, typ, box = dpsynth.water_box(5)
    mass = np.array([dpsynth.MASS["O"], dpsynth.MASS["H"]])
    vel = dpsynth.velocities(mass[typ], 600.0, 5)
    m = dp.Model(cfg, 0, params=p)
    runs = []
    for direct in (True, False):
        if direct:
            os.environ["DP_NO_GRAPH"] = "1"
        try:
            st = dp.MDState(m, coord, vel, typ, mass, box, skin=0.05)
            dp.dp_profile_enable(m.h, True)
            th1 = st.step(7, 0.5, prec, thermo_every=1)
            prof = dp.dp_profile_read(m.h)
            dp.dp_profile_enable(m.h, False)
            th2 = st.step(6, 0.5, prec, thermo_every=3)
            th3 = st.step(4, 0.5, prec, thermo_every=2)
            x, v, step, nreb = st.get()
            st.close()
        finally:
            os.environ.pop("DP_NO_GRAPH", None)
        runs.append((th1, th2, th3, x, v, step, nreb, {g: c[0] for g, c in prof.items()}))
    a, b = runs
    if prec == "fp64":
        tol = 1e-9
        for k in range(3):
            np.testing.assert_allclose(b[k], a[k], rtol=tol, atol=tol * np.abs(a[k]).max())
        np.testing.assert_allclose(b[3], a[3], rtol=0, atol=tol * box[0, 0])
        np.testing.assert_allclose(b[4], a[4], rtol=0, atol=tol * np.abs(a[4]).max())
    else:
        # the force and virial sums take atomics in whatever order the blocks run, and a last-bit
        # change of an FP32 value can flip the rounding of a 16-bit operand; over 17 steps of this
        # hot, stiff system two direct runs drift apart by up to about 1e-3 of the velocities. That
        # run-to-run noise (not the replay) sets the bound; a replay of stale buffers or weights
        # moves everything by O(1)
        for k in (0, 1, 2, 4):
            assert np.linalg.norm(b[k] - a[k]) <= 2e-2 * np.linalg.norm(a[k]), k
        d = b[3] - a[3]
        d -= box[0, 0] * np.rint(d / box[0, 0])
        assert np.abs(d).max() < 1e-2   # A
    assert a[5] == b[5] == 17
    assert a[6] > 1 and b[6] > 1              # rebuilds inside the replayed steps
    if prec == "fp64":
        assert a[6] == b[6]
    assert a[7] == b[7]


@pytest.mark.parametrize("route", ["simt", "split"])
def test_checkpoint_resume_bit_for_bit_when_deterministic(dp, tmp_path, route):
    """With deterministic force accumulation the resumed run repeats the uninterrupted one exactly:
    coordinates, velocities and thermo rows, on the one-CTA-per-atom and the split-product FP64
    routes, across device list rebuilds (skin 0.3 A)."""
    cfg, p = _scaled_water_model(5)
    coord, typ, box = dpsynth.water_box(5)
    mass = np.array([dpsynth.MASS["O"], dpsynth.MASS["H"]])
    vel = dpsynth.velocities(mass[typ], 600.0, 5)
    import os
    if route == "split":
        os.environ["DP_OZ_MIN_ATOMS"] = "0"
    try:
        m = dp.Model(cfg, 0, params=p, deterministic=True)
        st = dp.MDState(m, coord, vel, typ, mass, box, skin=0.3)
        st.step(8, 0.5, "fp64")
        path = str(tmp_path / "md.ckpt")
        st.save(path)
        th_a = st.step(12, 0.5, "fp64", thermo_every=4)
        xa, va, stepa, nra = st.get()
        r = dp.MDState.load(m, path)
        th_b = r.step(12, 0.5, "fp64", thermo_every=4)
        xb, vb, stepb, _ = r.get()
        # and a second uninterrupted run from the start
        st2 = dp.MDState(m, coord, vel, typ, mass, box, skin=0.3)
        th_c = st2.step(20, 0.5, "fp64", thermo_every=4)
        xc, vc, _, _ = st2.get()
    finally:
        os.environ.pop("DP_OZ_MIN_ATOMS", None)
    assert stepb == stepa == 20 and nra > 1
    np.testing.assert_array_equal(xb, xa)
    np.testing.assert_array_equal(vb, va)
    np.testing.assert_array_equal(th_b, th_a)
    np.testing.assert_array_equal(xc, xa)
    np.testing.assert_array_equal(vc, va)
    np.testing.assert_array_equal(th_c[-len(th_a):], th_a)
    for x in (r, st, st2):
        x.close()
    m.close()


def test_checkpoint_resume(dp, tmp_path):
    """A state saved after 8 steps and resumed follows the uninterrupted run: the saved coordinates,
    velocities and step come back bit for bit, and the resumed steps match the uninterrupted ones
    within what the order of the force atomics leaves free; another model's types are refused."""
    cfg, p = _scaled_water_model(5)
    coord, typ, box = dpsynth.water_box(5)
    mass = np.array([dpsynth.MASS["O"], dpsynth.MASS["H"]])
    vel = dpsynth.velocities(mass[typ], 600.0, 5)
    m = dp.Model(cfg, 0, params=p)
    st = dp.MDState(m, coord, vel, typ, mass, box, skin=0.3)
    st.step(8, 0.5, "fp64")
    x8, v8, step8, _ = st.get()
    path = str(tmp_path / "md.ckpt")
    st.save(path)
    th_a = st.step(12, 0.5, "fp64", thermo_every=4)
    xa, va, stepa, _ = st.get()
    r = dp.MDState.load(m, path)
    x8r, v8r, step8r, _ = r.get()
    np.testing.assert_array_equal(x8r, x8)
    np.testing.assert_array_equal(v8r, v8)
    assert step8r == step8 == 8
    th_b = r.step(12, 0.5, "fp64", thermo_every=4)
    xb, vb, stepb, _ = r.get()
    assert stepb == stepa == 20
    np.testing.assert_allclose(xb, xa, rtol=0, atol=1e-10 * box[0, 0])
    np.testing.assert_allclose(vb, va, rtol=0, atol=1e-10 * np.abs(va).max())
    np.testing.assert_allclose(th_b, th_a, rtol=1e-9)
    r.close()
    st.close()
    cu = dp.Model(dpsynth.copper_config(), 0)
    with pytest.raises(dp.DPError, match="DP_ERR_ARG"):
        dp.MDState.load(cu, path)
