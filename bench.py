"""Benchmark: DeepPot-SE velocity-Verlet NVE on one GB300, in s/step/atom and ns/day.

Default workload: FCC copper, 10x10x10 cells = 4,000 atoms, seeded
N(0, 0.1^2) displacements, r_c 8 A, r_cs 2 A, sel 512, embedding
(25, 50, 100), M2 16, fitting (240, 240, 240), seeded N(0, 1/fan_in)
weights, Maxwell-Boltzmann velocities at 300 K, dt 1 fs, FP64, 2 A skin
list rebuilt on the device when needed.  One step = half kick, drift,
list check/rebuild, list formatting, energy/force/virial, half kick.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64]
                  [--impl mine|reference] [--workload cu4000|cu108k|water192|water12k|water1p5m]

Prints one JSON line.  value = s/step/atom over the whole job (lower is
better), timed with CUDA events on the library's stream, inputs resident
on the device.  e2e = the same metric through dp_compute with host
buffers (coordinates in from pinned memory, forces/energy/virial out) and
the velocity-Verlet update on the host.  --impl reference times the FP64
CPU oracle on the host cores on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import dpsynth  # noqa: E402

FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2 FLOP x 2070 MHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # 152 SMs x 128 FFMA/clk x 2 FLOP x 2070 MHz


# DRAM bytes per launch of the dominant kernel from one ncu capture of the same command
# (dram__bytes_read.sum + dram__bytes_write.sum), and the capture's summary file; valid while the
# kernel is unchanged since the capture.
NCU_TRAFFIC = {
    ("fp64", "cu4000", "embed_fwd_l2"): (2.068e9 + 1.266e9, "profiles/fp64_embed_fwd_l2_pipes_cu4000.md"),
    ("bf16", "cu4000", "embed_bwd"): (28.80e6 + 0.06e6, "profiles/bf16_cu4000_nve_step.md"),
}


# FP64-pipe work of the dominant FP64 kernel: thread instructions executed on the FP64 pipe per real
# neighbor (ncu sm__thread_inst_executed_pipe_fp64_pred_on.sum of one launch / the real neighbors of
# the list), its tensor-pipe busy fraction, and the capture's summary file.  The kernel's multiply-adds
# run on the tensor cores as exact split products; what bounds it is the FP64 pipe of its epilogue.
NCU_FP64_PIPE = {
    "embed_fwd_l2": (1.0752e9 / 718768, 0.0554, "profiles/fp64_embed_fwd_l2_pipes_cu4000.md"),
}


def tensor_peak():
    """Measured sustained dense bf16 TFLOP/s (fp16 runs at the same rate), else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["bf16_tflops_sustained"]), "measured: MEASURED_PEAKS.json bf16_tflops_sustained"
    except (OSError, KeyError, ValueError):
        return 1700.0, "fallback: 1.7 PFLOP/s bf16 sustained"


def workload(name: str, model: str = "full"):
    cfg, coord, typ, box, mass, dt, desc = _workload(name)
    if model == "student":
        if cfg.ntypes != 1:
            raise SystemExit("the student model is the copper one")
        cfg = dpsynth.copper_student_config()
        desc += "; student nets 8-16-32 / M2 8 / 64-64-64"
    return cfg, coord, typ, box, mass, dt, desc


# Initial temperature (K) and thermo interval (steps; None: one row at the end) of the timed MD.
# water12k follows the paper's production protocol: 330 K, a thermo row every 20 steps (Sec. 5.1).
MD_PROTOCOL = {"water12k": (330.0, 20)}
# Fixed-interval skin-list rebuilds (steps) on top of the displacement criterion; water12k follows the
# paper's production protocol: a 2 A skin list built every 50 steps (Sec. 5.1).
MD_REBUILD = {"water12k": 50}


def md_protocol(name: str, steps: int):
    T, every = MD_PROTOCOL.get(name, (300.0, None))
    return T, (every if every is not None and every <= steps else steps)


def _workload(name: str):
    if name == "cu4000":
        cfg = dpsynth.copper_config()
        coord, typ, box = dpsynth.copper_fcc(1, ncell=10)
        mass = np.array([dpsynth.MASS["Cu"]])
        return cfg, coord, typ, box, mass, 1.0, "Cu FCC 10^3 cells, 4000 atoms, rcut 8, sel 512, 300 K, dt 1 fs"
    if name == "cu108k":
        cfg = dpsynth.copper_config()
        coord, typ, box = dpsynth.copper_fcc(1, ncell=30)
        mass = np.array([dpsynth.MASS["Cu"]])
        return cfg, coord, typ, box, mass, 1.0, "Cu FCC 30^3 cells, 108000 atoms, rcut 8, sel 512, 300 K, dt 1 fs"
    if name == "water12k":
        cfg = dpsynth.water_paper_config()
        c, t, b = dpsynth.water_box(1)
        coord, typ, box = dpsynth.replicate(c, t, b, (4, 4, 4))
        mass = np.array([dpsynth.MASS["O"], dpsynth.MASS["H"]])
        return cfg, coord, typ, box, mass, 0.5, ("4096 H2O (64-molecule box replicated 4x4x4), 12288 atoms, rcut 6, "
                                                 "sel 48/96, nets 32-64-128 / 240-240-240 (the paper's water model "
                                                 "and single-GPU system), 330 K, dt 0.5 fs, thermo every 20 steps")
    if name == "water1p5m":
        cfg = dpsynth.water_config()
        c, t, b = dpsynth.water_box(1)
        coord, typ, box = dpsynth.replicate(c, t, b, (32, 16, 16))
        mass = np.array([dpsynth.MASS["O"], dpsynth.MASS["H"]])
        return cfg, coord, typ, box, mass, 0.5, ("64-molecule water box replicated 32x16x16, 1572864 atoms, rcut 6, "
                                                 "sel 46/92, 300 K, dt 0.5 fs")
    if name == "water192":
        cfg = dpsynth.water_config()
        coord, typ, box = dpsynth.water_box(1)
        mass = np.array([dpsynth.MASS["O"], dpsynth.MASS["H"]])
        return cfg, coord, typ, box, mass, 0.5, "64 H2O, 192 atoms, rcut 6, sel 46/92, 300 K, dt 0.5 fs"
    raise SystemExit(f"unknown workload {name}")


def flops_per_group(cfg, nnei_total: int, n: int, split_route: bool = False):
    """Algorithmic FLOP per evaluation (real neighbors only; padded rows are zero work).

    split_route: the FP64 route whose widest embedding layer (and its input gradient) are their own
    kernel groups (embed_fwd_l2, embed_bwd_l2), and D / dE/dT the descriptor group."""
    e0, e1, e2 = cfg.embed
    m1, m2 = e2, cfg.m2
    f = list(cfg.fit)
    fwd_n = 2 * (e0 + e0 * e1 + e1 * e2 + 4 * e2)
    bwd_n = 2 * (4 * e2 + 4 * e2 + e2 * e1 + e1 * e0 + e0)
    fit_a = 2 * 2 * (m1 * m2 * f[0] + sum(f[k] * f[k + 1] for k in range(len(f) - 1)) + f[-1])
    if split_route:
        return {
            "embed_fwd": nnei_total * 2 * (e0 + e0 * e1),
            "embed_fwd_l2": nnei_total * 2 * (e1 * e2 + 4 * e2),
            "descriptor": n * 2 * 12 * m1 * m2,
            "embed_bwd": nnei_total * 2 * (4 * e2 + 4 * e2 + e1 * e0 + e0),
            "embed_bwd_l2": nnei_total * 2 * e2 * e1,
            "fitting": n * fit_a,
        }
    return {
        "embed_fwd": nnei_total * fwd_n + n * 2 * 4 * m1 * m2,
        "embed_bwd": nnei_total * bwd_n + n * 2 * 8 * m1 * m2,
        "fitting": n * fit_a,
    }


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    def __init__(self):
        self.p = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "100", "-i", os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip() == "Active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def run_mine(args, rank, world):
    import torch

    import paper_2005_00223_gb300 as dp

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    cfg, coord, typ, box, mass, dt, desc = workload(args.workload, args.model)
    n = len(typ)
    T0, thermo_every = md_protocol(args.workload, args.steps)
    vel = dpsynth.velocities(mass[typ], T0, 1)
    model = dp.Model(cfg, seed=1)
    stream = torch.cuda.Stream(device=dev)
    dp.dp_model_set_stream(model.h, stream)
    nl0 = dp.NeighborList(model, coord, typ, box)
    nlist0, _ = nl0.get()
    nnei_total = int((nlist0 >= 0).sum())
    nl0.close()
    state = dp.MDState(model, coord, vel, typ, mass, box, skin=2.0)
    state.rebuild_every(MD_REBUILD.get(args.workload, 0))
    state.step(args.warmup, dt, args.precision)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # Untimed pass of the same length with every kernel group bracketed by events: the per-group
    # breakdown, the launch count and the dominant group.
    dp.dp_profile_select(model.h, None)
    dp.dp_profile_enable(model.h, True)
    ev0.record(stream)
    state.step(args.steps, dt, args.precision, thermo_every=thermo_every)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_all = ev0.elapsed_time(ev1)
    prof_all = dp.dp_profile_read(model.h)
    launches = int(sum(v[0] for v in prof_all.values()))
    split_route = prof_all.get("embed_fwd_l2", (0, 0.0))[0] > 0
    flops = flops_per_group(cfg, nnei_total, n, split_route)
    groups = {g: {"launches": v[0], "ms_total": round(v[1], 4), "share": round(v[1] / ms_all, 4)}
              for g, v in prof_all.items() if v[0] > 0}
    top = max((g for g in prof_all if prof_all[g][0] > 0), key=lambda g: prof_all[g][1])
    if top not in flops:   # dominant group outside the nets: report the heaviest net kernel
        top = max((g for g in flops if g in prof_all and prof_all[g][0] > 0), key=lambda g: prof_all[g][1],
                  default=None)
    # Timed pass: only the dominant group carries events (every other event pair costs the step a few us).
    dp.dp_profile_select(model.h, [top] if top is not None else [])
    dp.dp_profile_enable(model.h, True)
    state.step(2, dt, args.precision)   # the step is captured again with this set of events
    sampler = ClockSampler()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    dp.dp_profile_enable(model.h, True)
    ev0.record(stream)
    th = state.step(args.steps, dt, args.precision, thermo_every=thermo_every)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    clocks = sampler.stop()
    prof = dp.dp_profile_read(model.h)
    dp.dp_profile_enable(model.h, False)
    dp.dp_profile_select(model.h, None)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    roofline = None
    if top is not None:
        # one launch processes one batch; with one batch per step a launch covers the whole system
        batches = max(1, prof[top][0] // args.steps)
        per_launch_ms = prof[top][1] / prof[top][0]
        achieved = flops[top] / batches / (per_launch_ms * 1e-3) / 1e12
        if args.precision == "fp64":
            bound, peak, src = "alu", FP64_PEAK_TFLOPS, \
                "derived: 152 SMs x 2 FP64 FMA/clk x 2 FLOP x 2070 MHz (nominal 1.25 TFLOP/s)"
        elif args.precision == "mix32":
            bound, peak, src = "alu", FP32_PEAK_TFLOPS, "derived: 152 SMs x 128 FP32 FMA/clk x 2 FLOP x 2070 MHz"
        else:
            bound = "tensor"
            peak, src = tensor_peak()
        roofline = {"bound": bound, "kernel": top, "achieved": round(achieved, 4), "peak": round(peak, 4),
                    "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None, "peak_source": src}
        tr = NCU_TRAFFIC.get((args.precision, args.workload, top))
        if tr is not None and args.model == "full":
            roofline["traffic"] = tr[0]
            roofline["traffic_source"] = "ncu, " + tr[1]
        pipe = NCU_FP64_PIPE.get(top)
        if split_route and args.precision == "fp64" and pipe is not None and args.model == "full":
            # the FP64-pipe issue slots the kernel needs (ncu count per real neighbor, 2 FLOP each as for a
            # DFMA) per second of its measured launch time, against the FP64 pipe's peak
            fp64_equiv = dict(achieved=round(achieved, 4), frac_of_dfma_peak=round(achieved / peak, 4),
                              note="algorithmic FP64-accurate FLOP of the layer (10,800 per real neighbor) per "
                                   "second; above the FP64 peak because the multiply-adds run on the tensor "
                                   "cores as exact split products")
            work = 2.0 * pipe[0] * nnei_total / batches
            achieved = work / (per_launch_ms * 1e-3) / 1e12
            roofline.update({"achieved": round(achieved, 4), "frac": round(achieved / peak, 4),
                             "work": "FP64-pipe thread instructions of the kernel (ncu count, %.1f per real "
                                     "neighbor) x 2 FLOP, i.e. the FP64 pipe's busy time / the launch time" % pipe[0],
                             "work_source": "ncu, " + pipe[2], "tensor_pipe_frac_ncu": pipe[1],
                             "fp64_equivalent": fp64_equiv,
                             "note": "the layer's multiply-adds run on the tensor cores (tensor pipe %.1f%% busy); "
                                     "the FP64 work of the epilogue (tanh, skips, read-back of the split "
                                     "products, contraction) bounds the kernel" % (100 * pipe[1])})
    step_s = ms * 1e-3 / args.steps
    value = step_s / (n * world)
    total_flop = sum(flops.values())
    # end-to-end: host buffers through dp_compute + host velocity Verlet
    e2e = None
    if rank == 0 and args.e2e_steps > 0:
        e2e = run_e2e(dp, model, cfg, coord, vel, typ, box, mass, dt, args, stream)
    state.close()
    out = {
        "metric": "s/step/atom", "value": value, "unit": "s/step/atom", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "ns_per_day": 86400.0 * dt * 1e-6 / step_s,
        "dtype": "f64" if args.precision == "fp64" else args.precision,
        "precision": args.precision, "data": "synthetic (seeded FCC copper / water, seeded random-init weights)",
        "config": {"workload": desc, "atoms": n, "precision": args.precision, "real_neighbors": nnei_total,
                   "l2": "working set per step > L2 (stored activations, %.2f GB)" % (
                       nnei_total * (sum(cfg.embed) + cfg.embed[-1]) * 8 / 1e9),
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "launch": "each MD step replays one captured step (CUDA graph)",
                   "profiling": "timed pass: events around the dominant group only; kernel_groups and "
                                "gpu_launches from an untimed pass of the same length with every group timed"},
        "gflop_per_step": total_flop / 1e9, "tflops": total_flop / step_s / 1e12,
        "roofline": roofline, "kernel_groups": groups, "gpu_launches": launches,
        "thermo_last": [float(x) for x in th[-1]] if len(th) else None,
        "clocks": clocks, "e2e": e2e,
    }
    return out


PATHS = ("fp64", "mix32", "bf16", "fp16", "bf16x3", "student", "student_judged")
JUDGE_EVERY = 10


def _md_ms_per_step(dp, model, coord, vel, typ, mass, box, dt, prec, steps, warmup, stream, rebuild_every=0):
    """Device ms per NVE step of `steps` replayed steps after `warmup` (CUDA events on the model's stream)."""
    import torch
    state = dp.MDState(model, coord, vel, typ, mass, box, skin=2.0)
    state.rebuild_every(rebuild_every)
    state.step(warmup, dt, prec)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    state.step(steps, dt, prec)
    ev1.record(stream)
    torch.cuda.synchronize()
    state.close()
    return ev0.elapsed_time(ev1) / steps


def _errors(E, Ei, F, W, ref, n):
    """Deviation of one evaluation (E, E_i, F, W) from the reference (E, E_i, F, W) of the same coordinates."""
    Er, Eir, Fr, Wr = ref
    frms = float(np.sqrt((Fr ** 2).sum(1).mean()))
    rmse = float(np.sqrt(((F - Fr) ** 2).sum(1).mean()))
    return {"force_rmse_eV_per_A": rmse, "force_rmse_rel": rmse / frms,
            "force_rmse_at_1eV_per_A_scale": rmse / frms,
            "force_max_abs_err_eV_per_A": float(np.sqrt(((F - Fr) ** 2).sum(1)).max()),
            "energy_err_per_atom_eV": abs(E - Er) / n,
            "atom_energy_max_abs_err_eV": float(np.abs(Ei - Eir).max()),
            "virial_rel_err": float(np.abs(W - Wr).max() / np.abs(Wr).max()),
            "meets_1e-3_eV_per_A": rmse <= 1e-3, "meets_1e-3_at_1eV_per_A_scale": rmse / frms <= 1e-3}


def fitted_copper_teacher(dp, S, steps=20000, nframes=512):
    """The full copper model (seeded weights as the starting point) fitted to the Morse copper reference.

    A seeded random-weight model has no stable crystal: scaled to realistic forces its MD collapses,
    unscaled its forces are far below thermal energies and its atoms drift like a gas.  Fitting it
    first to a classical copper potential (dpsynth.morse_copper, a stand-in for the first-principles
    labels the paper's models are trained on) by the library's own training kernels gives a teacher
    whose NVE stays an FCC crystal from 300 to 1,300 K.  Frames: nframes 500-atom supercells with
    0.02-0.18 A displacements (plus 32 held out); Adam on the force-matching loss (fit_to_reference).
    Returns (parameters, info)."""
    cfg = dpsynth.copper_config()
    t0 = time.perf_counter()
    X, E, F, typ, box = dpsynth.morse_frames(nframes + 32)
    label_s = time.perf_counter() - t0
    m = dp.Model(cfg, 0, params=dpsynth.model_params(cfg, 1))
    r0, frms = S.force_rmse_vs_labels(m, X[nframes:], F[nframes:], typ, box)
    t1 = time.perf_counter()
    log = S.fit_to_reference(m, X[:nframes], E[:nframes], F[:nframes], typ, box, steps=steps)
    fit_s = time.perf_counter() - t1
    r1, _ = S.force_rmse_vs_labels(m, X[nframes:], F[nframes:], typ, box)
    params = m.params
    m.close()
    info = {"reference": "Morse copper (Girifalco and Weizer 1959), shifted-force at 8 A",
            "frames": f"{nframes} labelled 500-atom supercells, displacements 0.02-0.18 A; 32 held out",
            "adam_steps": steps, "labels_seconds": label_s, "fit_seconds": fit_s,
            "heldout_rms_force_eV_per_A": frms, "heldout_force_rmse_before_eV_per_A": r0,
            "heldout_force_rmse_eV_per_A": r1, "heldout_force_rmse_rel": r1 / frms, "loss_last": log[-1][1]}
    return params, info


def distil_student(dp, S, dev, temps=(300.0, 1200.0), frames_per_temp=24, adam_steps=800, md_prec="mix32",
                   label_prec="mix32", frames_per_run=None, relative=False, teacher_params=None):
    """Teacher (the seeded copper model) and a student distilled from its own MD, trained by libdp.

    Teacher frames every 5 NVE steps on 4,000 atoms, frames_per_temp at each temperature (default 24
    at 300 K and 1,200 K) from runs of frames_per_run frames (default: one run), each run starting at
    the lattice with its own Maxwell-Boltzmann velocities; Adam steps of one frame each with
    p_e = 1, p_f = 100 / RMS(F)^2, the learning rate decaying 3e-3 -> 1e-4 (the recipe of the
    distillation test).  Short runs keep the seeded teacher near the lattice: its long runs at
    900-1200 K leave it (a random-weight model has no physical minimum there).  relative: the force
    weight of each frame is 100 / RMS(F_k)^2 instead (a relative force loss), so that the frames of
    every temperature count alike although their force scales differ by orders.  teacher_params: a
    fitted teacher (fitted_copper_teacher) instead of the seeded model; its runs start at the perfect
    lattice with velocities drawn at twice the temperature, which equipartition in the crystal halves
    to about the target.  Returns (teacher, student, teacher RMS force of the frames, number of
    frames, RMS force per temperature, mean frame temperature per temperature)."""
    cfg = dpsynth.copper_config()
    fitted = teacher_params is not None
    teacher = dp.Model(cfg, 0, params=teacher_params if fitted else dpsynth.model_params(cfg, 1))
    c4, t4, b4 = dpsynth.copper_fcc(1, ncell=10, sigma=0.0 if fitted else 0.1)
    mass = np.array([dpsynth.MASS["Cu"]])
    # frames_per_run: one value for every temperature or a list, one per temperature
    per_runs = list(frames_per_run) if isinstance(frames_per_run, (list, tuple)) else [frames_per_run] * len(temps)
    Xs, Es, Fs, Ts = [], [], [], []
    for k, T in enumerate(temps):
        per_run = per_runs[k] or frames_per_temp
        runs = max(1, frames_per_temp // per_run)
        vels = [dpsynth.velocities(mass[t4], 2.0 * T if fitted else T, 10 + k * 100003 + r) for r in range(runs)]
        x, e, f, tt = S.teacher_frames(teacher, c4, t4, b4, mass, vels, nframes=per_run, stride=5, dt_fs=1.0,
                                       md_prec=md_prec, label_prec=label_prec, return_temps=True)
        Xs.append(x)
        Es.append(e)
        Fs.append(f)
        Ts.append(float(tt.mean()))
    X, E, F = np.concatenate(Xs), np.concatenate(Es), np.concatenate(Fs)
    frms = float(np.sqrt((F ** 2).sum(-1).mean()))
    frms_t = [float(np.sqrt((f ** 2).sum(-1).mean())) for f in Fs]
    stu = dp.Model(dpsynth.copper_student_config(), seed=2)
    pf = 100.0 / ((F ** 2).sum(-1).mean(-1) if relative else frms ** 2)
    S.train(stu, t4, b4, X, E, F, steps=adam_steps, lr0=3e-3, lr1=1e-4, p_e=1.0, p_f=pf)
    return teacher, stu, frms, len(X), frms_t, Ts


def run_paths(args, name, steps, warmup, ref, ref_kind, fp64_ms=None, student=None):
    """Every precision path and the student on one workload, in this process.

    Per path: device ms per NVE step (CUDA events, graph-replayed steps), s/step/atom, ns/day, the
    speed-up over the FP64 path, and the deviation of one evaluation at the initial coordinates
    from `ref` (the FP64 oracle's evaluation of the same coordinates, or the FP64 GPU path's when
    no oracle ran).  'student' is the distilled student's MD in BF16; 'student_judged' adds the
    full model (BF16) as judge every 10 steps, driving the MD while the student's force RMSE
    exceeds 0.1 x the full model's RMS force."""
    import torch

    import paper_2005_00223_gb300 as dp
    from paper_2005_00223_gb300 import student as S

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    cfg, coord, typ, box, mass, dt, desc = workload(name)
    n = len(typ)
    vel = dpsynth.velocities(mass[typ], md_protocol(name, 1)[0], 1)
    stream = torch.cuda.Stream(device=dev)
    full = dp.Model(cfg, seed=1)
    dp.dp_model_set_stream(full.h, stream)
    if ref is None:   # no oracle evaluation: the FP64 path's (equal to the oracle's within 1e-10 in the GPU tests)
        nl = dp.NeighborList(full, coord, typ, box)
        ref = nl.compute(coord, box, "fp64")
        nl.close()
    nl = dp.NeighborList(full, coord, typ, box)
    nnei_total = int((nl.get()[0] >= 0).sum())
    nl.close()
    work_real = sum(flops_per_group(cfg, nnei_total, n).values())
    work_pad = sum(flops_per_group(cfg, n * cfg.nsel, n).values())
    out = {"workload": desc, "atoms": n, "steps": steps, "warmup": warmup, "error_reference": ref_kind,
           "rms_force_eV_per_A": float(np.sqrt((ref[2] ** 2).sum(1).mean())),
           "rebuild_every": MD_REBUILD.get(name, 0),
           "work": {"real_neighbors_per_atom": nnei_total / n, "mflop_per_atom_eval": work_real / n / 1e6,
                    "mflop_per_atom_eval_if_padded_rows_counted": work_pad / n / 1e6,
                    "counted": "multiply-adds x 2 of the embedding net (forward, input gradient), contraction, "
                               "descriptor, fitting net (forward, input gradient) over real neighbors"},
           "paths": {}}
    for p in args.paths:
        if p.startswith("student") and (student is None or cfg.ntypes != 1):
            continue
        model, prec = (student[1], "bf16") if p.startswith("student") else (full, p)
        if p.startswith("student"):
            dp.dp_model_set_stream(model.h, stream)
            dp.dp_model_set_stream(student[0].h, stream)
        nl = dp.NeighborList(model, coord, typ, box)
        E, Ei, F, W = nl.compute(coord, box, prec)
        nl.close()
        rec = {"precision": prec, "model": "student 8-16-32 / M2 8 / 64-64-64" if p.startswith("student") else
               "full"}
        if p == "fp64" and fp64_ms is not None:
            ms = fp64_ms
        elif p == "student_judged":
            nlj = dp.NeighborList(student[0], coord, typ, box)
            Fj = nlj.compute(coord, box, "bf16")[2]
            nlj.close()
            rmse_max = 0.1 * float(np.sqrt((Fj ** 2).sum(1).mean()))
            st = dp.MDState(model, coord, vel, typ, mass, box, skin=2.0)
            nj = max(JUDGE_EVERY, warmup // JUDGE_EVERY * JUDGE_EVERY)
            dp.dp_md_step_judged(model.h, student[0].h, st.h, nj, dt, "bf16", "bf16", judge_every=JUDGE_EVERY,
                                 rmse_max=rmse_max)
            k = max(JUDGE_EVERY, steps // JUDGE_EVERY * JUDGE_EVERY)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(stream)
            rm, fb = dp.dp_md_step_judged(model.h, student[0].h, st.h, k, dt, "bf16", "bf16",
                                          judge_every=JUDGE_EVERY, rmse_max=rmse_max)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1) / k
            st.close()
            rec.update({"judge_every": JUDGE_EVERY, "judge_precision": "bf16", "rmse_max_eV_per_A": rmse_max,
                        "judgements": int(len(rm)), "fallback_windows": int(fb.sum()),
                        "judged_rmse_mean_eV_per_A": float(rm.mean()), "judged_rmse_max_eV_per_A": float(rm.max())})
        else:
            ms = _md_ms_per_step(dp, model, coord, vel, typ, mass, box, dt, prec, steps, warmup, stream,
                                 MD_REBUILD.get(name, 0))
        step_s = ms * 1e-3
        rec.update({"ms_per_step": ms, "s_per_step_atom": step_s / n, "ns_per_day": 86400.0 * dt * 1e-6 / step_s})
        rec.update(_errors(E, Ei, F, W, ref, n))
        out["paths"][p] = rec
    f64 = out["paths"].get("fp64", {}).get("ms_per_step")
    for rec in out["paths"].values():
        rec["speedup_vs_fp64"] = (f64 / rec["ms_per_step"]) if f64 else None
    full.close()
    return out


def grad_frames():
    """The training batch: 32 seeded 192-atom water frames with seeded reference labels."""
    cfg = dpsynth.water_config()
    params = dpsynth.model_params(cfg, 7)
    rng = np.random.default_rng(5)
    frames = []
    for s in range(32):
        c, t, b = dpsynth.water_box(100 + s)
        frames.append((c, t, b, float(rng.normal()), rng.normal(scale=1e-3, size=c.shape)))
    return cfg, params, frames


def grad_flops(cfg, nnei_total: int, n: int):
    """Algorithmic FLOP of one force-loss gradient of a frame: 3x an evaluation.

    Per layer with C multiply-adds per row, the evaluation does 2C (forward and
    input gradient); the gradient does the primal and the tangent forward (2C)
    and the reverse of both, input adjoints and weight gradients (4C).
    """
    f = flops_per_group(cfg, nnei_total, n)
    return 3 * sum(f.values())


def run_train(args, rank, world):
    """Device time per training step (one-frame force-loss gradient + Adam, MIX-32) of the two
    training runs of config 4: the full copper model on 500-atom Morse-labelled frames (the teacher
    fit) and the copper student on 4,000-atom frames (the distillation).  --warmup untimed steps,
    then --steps timed with CUDA events on the training stream; per-group times from the library's
    tracing (param_grad covers the gradient kernels)."""
    import torch

    import paper_2005_00223_gb300 as dp
    from paper_2005_00223_gb300 import _lib

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)

    def time_steps(model, typ, box, X, E, F, p_e, p_f):
        Xd = torch.tensor(X, dtype=torch.float64, device=dev)
        Fd = torch.tensor(F, dtype=torch.float64, device=dev)
        Ed = torch.tensor(E, dtype=torch.float64, device=dev)
        nparams = _lib.dp_model_n_params(model.h)
        grad = torch.zeros(nparams, dtype=torch.float64, device=dev)
        loss = torch.zeros(1, dtype=torch.float64, device=dev)
        _lib.dp_model_set_stream(model.h, stream)
        nl = dp.NeighborList(model, X[0], typ, box)

        def step(s):
            k = s % len(X)
            _lib.dp_nlist_update_dev(nl.h, Xd[k], stream)
            grad.zero_()
            _lib.dp_force_loss_grad_dev(model.h, nl.h, Xd[k], box, Fd[k], Ed[k:k + 1], p_e, p_f, "mix32", loss,
                                        grad, stream)
            _lib.dp_adam_step(model.h, grad, 1e-4, 0.9, 0.999, 1e-8, s + 1, stream)

        for s in range(args.warmup):
            step(s)
        dp.dp_profile_enable(model.h, True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for s in range(args.warmup, args.warmup + args.steps):
            step(s)
        ev1.record(stream)
        torch.cuda.synchronize()
        prof = dp.dp_profile_read(model.h)
        dp.dp_profile_enable(model.h, False)
        nl.close()
        _lib.dp_model_set_stream(model.h, None)
        return ev0.elapsed_time(ev1) / args.steps, {g: {"launches": v[0], "ms_total": round(v[1], 4)}
                                                    for g, v in prof.items() if v[0] > 0}

    sampler = ClockSampler()
    sampler.start()
    cfg = dpsynth.copper_config()
    X, E, F, t5, b5 = dpsynth.morse_frames(16)
    full = dp.Model(cfg, 0, params=dpsynth.model_params(cfg, 1))
    ms_full, g_full = time_steps(full, t5, b5, X, E, F, 0.02, 100.0)
    full.close()
    c4, t4, b4 = dpsynth.copper_fcc(1, ncell=10)
    F4 = np.zeros((4,) + c4.shape)
    X4 = np.array([dpsynth.copper_fcc(1 + k, ncell=10)[0] for k in range(4)])
    stu = dp.Model(dpsynth.copper_student_config(), seed=2)
    ms_stu, g_stu = time_steps(stu, t4, b4, X4, np.zeros(4), F4, 1.0, 100.0)
    stu.close()
    clocks = sampler.stop()
    return {"metric": "ms per training step (force-loss gradient + Adam, MIX-32)", "value": ms_full,
            "unit": "ms/step", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_full,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded FCC copper; Morse-labelled frames for the full model)",
            "config": {"workload": "full copper model on 500-atom frames (teacher fit) and copper student on "
                                   "4,000-atom frames (distillation)", "parallelism": "1 GPU"},
            "full_model_500_atoms": {"ms_per_step": ms_full, "kernel_groups": g_full},
            "student_4000_atoms": {"ms_per_step": ms_stu, "kernel_groups": g_stu},
            "gpu_launches": int(sum(v["launches"] for v in g_full.values()) + sum(v["launches"] for v in g_stu.values())),
            "clocks": clocks, "e2e": None}


def run_grad(args, rank, world):
    """Parameter gradient of the force-matching loss over 32 water frames of 192 atoms, one batched call."""
    import torch

    import paper_2005_00223_gb300 as dp

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    prec = args.precision if args.precision in ("fp64", "mix32") else "fp64"
    cfg, params, frames = grad_frames()
    typ, box = frames[0][1], frames[0][2]
    n = len(typ)
    model = dp.Model(cfg, 0, params=params)
    stream = torch.cuda.Stream(device=dev)
    dp.dp_model_set_stream(model.h, stream)
    coords = np.array([f[0] for f in frames])
    X = torch.tensor(coords.reshape(-1, 3), dtype=torch.float64, device=dev)
    Fr = torch.tensor(np.array([f[4] for f in frames]).reshape(-1, 3), dtype=torch.float64, device=dev)
    Er = torch.tensor([f[3] for f in frames], dtype=torch.float64, device=dev)
    grad = torch.zeros(dp.dp_model_n_params(model.h), dtype=torch.float64, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    # the 32 frames as one list (each frame its own cell grid): one call per gradient fills the GPU
    nl = dp.NeighborList.frames(model, coords, typ, box, skin=0.0)
    nnei_total = int((nl.get()[0] >= 0).sum())
    torch.cuda.synchronize()

    def one_gradient():
        grad.zero_()
        loss.zero_()
        dp.dp_nlist_update_dev(nl.h, X, stream)
        dp.dp_force_loss_grad_dev(model.h, nl.h, X, box, Fr, Er, 1.0, 100.0, prec, loss, grad, stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_gradient()
    sampler = ClockSampler()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    dp.dp_profile_enable(model.h, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            one_gradient()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    clocks = sampler.stop()
    prof = dp.dp_profile_read(model.h)
    dp.dp_profile_enable(model.h, False)
    groups = {g: {"launches": v[0], "ms_total": round(v[1], 4), "share": round(v[1] / ms, 4)}
              for g, v in prof.items() if v[0] > 0}
    per_grad_s = ms * 1e-3 / args.steps
    flop = grad_flops(cfg, nnei_total, n * len(frames))
    kg = prof.get("param_grad", (0, 0.0))
    peak = FP64_PEAK_TFLOPS if prec == "fp64" else FP32_PEAK_TFLOPS
    roofline = None
    if kg[0] > 0:
        achieved = flop * args.steps / (kg[1] * 1e-3) / 1e12
        roofline = {"bound": "alu", "kernel": "param_grad", "achieved": round(achieved, 4), "peak": round(peak, 4),
                    "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
                    "peak_source": "derived: 152 SMs x %s FMA/clk x 2 FLOP x 2070 MHz" % (
                        "2 FP64" if prec == "fp64" else "128 FP32"),
                    "flop_model": "3 x the evaluation's algorithmic FLOP per frame"}
    # end to end: frames and labels copied from pinned host memory each gradient, gradient and loss read back
    e2e = None
    if args.e2e_steps > 0:
        hX = torch.tensor(coords.reshape(-1, 3), dtype=torch.float64).pin_memory()
        hF = torch.tensor(np.array([f[4] for f in frames]).reshape(-1, 3), dtype=torch.float64).pin_memory()
        hE = torch.tensor([f[3] for f in frames], dtype=torch.float64).pin_memory()
        hg = torch.empty_like(grad, device="cpu").pin_memory()
        hl = torch.empty(1, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for _ in range(args.e2e_steps):
                X.copy_(hX, non_blocking=True)
                Fr.copy_(hF, non_blocking=True)
                Er.copy_(hE, non_blocking=True)
                one_gradient()
                hg.copy_(grad, non_blocking=True)
                hl.copy_(loss, non_blocking=True)
                stream.synchronize()
        t1 = time.perf_counter()
        e2e = {"value": (t1 - t0) / args.e2e_steps, "unit": "s/gradient",
               "h2d_bytes_per_step": int(hX.numel() + hF.numel() + hE.numel()) * 8,
               "d2h_bytes_per_step": int(hg.numel() + 1) * 8,
               "path": "pinned host frames -> dp_nlist_update_dev + dp_force_loss_grad_dev -> host gradient"}
    nl.close()
    out = {"metric": "s/gradient (32 water frames of 192 atoms)", "value": per_grad_s, "unit": "s/gradient",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if prec == "fp64" else "f32", "precision": prec,
           "data": "synthetic (seeded water frames and labels, seeded random-init weights)",
           "config": {"workload": "force-loss parameter gradient, 32 x 64 H2O (192 atoms), rcut 6, sel 46/92",
                      "frames": len(frames), "atoms_per_frame": n, "real_neighbors": nnei_total,
                      "parameters": int(grad.numel()), "l2": "working set below L2; frames differ each call",
                      "parallelism": "1 GPU"},
           "gflop_per_step": flop / 1e9, "roofline": roofline, "kernel_groups": groups,
           "gpu_launches": int(sum(v[0] for v in prof.values())), "clocks": clocks, "e2e": e2e}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        om = oracle.Model(cfg, params)
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        om.force_loss_grad(frames[:4], p_e=1.0, p_f=100.0)
        el = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": el * len(frames) / 4, "unit": "s/gradient", "cores": cores,
                               "kind": "oracle", "sample": "the FP64 oracle gradient of 4 of the 32 frames, x 8"}
    return out


def run_judged(args, rank, world):
    """Distilled student MD judged by the full model every 10 steps.

    Untimed: teacher frames every 5 steps of its own NVE at each of --temps on
    4,000 atoms (--frames-per-temp each) and --adam-steps one-frame Adam steps
    of the student on them.  Defaults: 300 K and 1,200 K, 24 frames each, 800
    steps (the distillation test's recipe); the copper student workload of
    the paper-scale run is 300/600/900/1200 K x 5,000 frames and 20,000 steps
    on 108,000 atoms for 1,000 steps.  Timed: judged MD of the trained student
    on the workload, the teacher evaluated at every judgement and taking over
    while the student's force RMSE exceeds the threshold.

    --teacher fitted (default): the full model is first fitted to the Morse copper reference
    (fitted_copper_teacher), its frame runs start at the lattice, the judge evaluates it in
    --judge-precision (default bf16x3, FP32-class) and the threshold is config 4's absolute
    0.05 eV/A.  --teacher seeded: the seeded random-weight model as is, judged in --precision, with
    the threshold 0.1 x its RMS force at the start (its forces are ~1e-4 eV/A).
    """
    import torch

    import paper_2005_00223_gb300 as dp
    from paper_2005_00223_gb300 import student as S

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    temps = tuple(float(t) for t in args.temps.split(","))
    fitted = args.teacher == "fitted"
    fit_info, tparams = None, None
    if fitted:
        tparams, fit_info = fitted_copper_teacher(dp, S, args.teacher_fit_steps, args.teacher_fit_frames)
    md_prec = args.teacher_md_precision or ("bf16x3" if fitted else "mix32")
    label_prec = args.label_precision or ("bf16x3" if fitted else "mix32")
    judge_prec = args.judge_precision or ("bf16x3" if fitted else args.precision)
    t0 = time.perf_counter()
    teacher, stu, frms_train, nframes, frms_t, temps_t = distil_student(
        dp, S, dev, temps, args.frames_per_temp, args.adam_steps, md_prec, label_prec,
        [int(v) for v in str(args.frames_per_run).split(",")] if "," in str(args.frames_per_run)
        else int(args.frames_per_run), args.relative_force_loss, teacher_params=tparams)
    distil_s = time.perf_counter() - t0
    _, coord, typ, box, mass, dt, desc = workload(args.workload)
    n = len(typ)
    vel = dpsynth.velocities(mass[typ], 300.0, 1)
    stream = torch.cuda.Stream(device=dev)
    dp.dp_model_set_stream(stu.h, stream)
    dp.dp_model_set_stream(teacher.h, stream)
    nl0 = dp.NeighborList(teacher, coord, typ, box)
    F0 = nl0.compute(coord, box, judge_prec)[2]
    nnei_total = int((nl0.get()[0] >= 0).sum())
    nl0.close()
    frms0 = float(np.sqrt((F0 ** 2).sum(1).mean()))
    rmse_max = 0.05 if fitted else 0.1 * frms0
    state = dp.MDState(stu, coord, vel, typ, mass, box, skin=2.0)
    every = 10
    steps = max(every, (args.steps // every) * every)
    warm = every * max(1, args.warmup // every)
    dp.dp_md_step_judged(stu.h, teacher.h, state.h, warm, dt, args.precision, judge_prec, judge_every=every,
                         rmse_max=rmse_max)
    sampler = ClockSampler()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    dp.dp_profile_enable(stu.h, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    rm, fb = dp.dp_md_step_judged(stu.h, teacher.h, state.h, steps, dt, args.precision, judge_prec,
                                  judge_every=every, rmse_max=rmse_max)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    clocks = sampler.stop()
    prof = dp.dp_profile_read(stu.h)
    dp.dp_profile_enable(stu.h, False)
    # the state after the judged run: temperature, and the teacher's RMS force there
    xe, ve, _, _ = state.get()
    state.close()
    t_end = float((mass[typ][:, None] * ve * ve).sum() * dpsynth.MVV2E / ((3 * n - 3) * dpsynth.KB_EV))
    nle = dp.NeighborList(teacher, xe, typ, box)
    Fe = nle.compute(xe, box, judge_prec)[2]
    nle.close()
    frms_end = float(np.sqrt((Fe ** 2).sum(1).mean()))
    step_s = ms * 1e-3 / steps
    scfg = dpsynth.copper_student_config()
    flops = flops_per_group(scfg, nnei_total, n)
    top = max((g for g in flops if prof.get(g, (0, 0.0))[0] > 0), key=lambda g: prof[g][1], default=None)
    roofline = None
    if top is not None:
        peak, src = tensor_peak()
        # one launch per student evaluation (the teacher keeps its own counters)
        achieved = flops[top] * prof[top][0] / (prof[top][1] * 1e-3) / 1e12
        roofline = {"bound": "tensor", "kernel": "student " + top, "achieved": round(achieved, 4),
                    "peak": round(peak, 4), "unit": "TFLOP/s", "frac": round(achieved / peak, 6), "traffic": None,
                    "peak_source": src}
    return {"metric": "s/step/atom (judged student MD)", "value": step_s / (n * world), "unit": "s/step/atom",
            "n_gpus": world, "steps": steps, "warmup": every * max(1, args.warmup // every),
            "ms_per_step": ms / steps, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "ns_per_day": 86400.0 * dt * 1e-6 / step_s, "dtype": args.precision, "precision": args.precision,
            "data": "synthetic (seeded FCC copper; student distilled from the %s teacher's own MD)" % (
                "Morse-fitted" if fitted else "seeded"),
            "teacher": {"kind": "fitted to the Morse copper reference" if fitted else "seeded random weights",
                        "fit": fit_info, "judge_precision": judge_prec},
            "distillation": {"temperatures_K": list(temps), "frames": nframes, "frame_stride_steps": 5,
                             "frame_atoms": 4000, "teacher_md_precision": md_prec,
                             "mean_frame_temperature_K": temps_t,
                             "runs_start": "perfect lattice, velocities at 2 T" if fitted
                             else "displaced lattice (0.1 A), velocities at T",
                             "label_precision": label_prec, "adam_steps": args.adam_steps,
                             "frames_per_run": args.frames_per_run,
                             "force_loss": "relative (100 / RMS(F_k)^2 per frame)" if args.relative_force_loss
                             else "100 / RMS(F)^2 over all frames",
                             "teacher_rms_force_of_frames_eV_per_A": frms_train,
                             "teacher_rms_force_per_temperature_eV_per_A": frms_t, "seconds": distil_s},
            "config": {"workload": desc, "atoms": n, "judge_every": every, "rmse_max_eV_per_A": rmse_max,
                       "threshold": "config 4's absolute 0.05 eV/A" if fitted else "0.1 x the teacher's RMS force",
                       "fallback_windows_at_0.05_eV_per_A": int((rm > 0.05).sum()),
                       "student_rmse_mean_over_rms_force": float(rm.mean()) / frms0,
                       "teacher_rms_force_eV_per_A": frms0, "teacher_rms_force_at_end_eV_per_A": frms_end,
                       "temperature_at_end_K": t_end, "judgements": int(len(rm)),
                       "fallback_windows": int(fb.sum()), "student_rmse_max": float(rm.max()),
                       "student_rmse_mean": float(rm.mean()), "parallelism": "1 GPU",
                       "l2": "working set per step > L2"},
            "roofline": roofline, "kernel_groups": {g: {"launches": v[0], "ms_total": round(v[1], 4)}
                                                 for g, v in prof.items() if v[0] > 0},
            "gpu_launches": int(sum(v[0] for v in prof.values())), "clocks": clocks, "e2e": None}


SWEEP = ((32, 64, 128), (64, 128, 256), (128, 256, 512), (256, 512, 1024), (512, 1024, 2048))


def run_sweep(args, rank, world):
    """Embedding-width sweep (Sec. 6, "Network size"): copper 4,000 atoms, r_c 8 A, sel 512, M2 16,
    fitting 240-240-240, MIX-16 bf16, nets (w, 2w, 4w) from the paper's 32-64-128 to its largest
    512-1024-2048 (last-layer matrices 64 x 128 .. 1024 x 2048).  Per net: device ms per NVE step
    (graph-replayed steps, CUDA events), the algorithmic work per atom and evaluation, and the
    achieved FLOP/s of the embedding kernels and of the whole step against the measured bf16 peak."""
    import torch

    import paper_2005_00223_gb300 as dp

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    coord, typ, box = dpsynth.copper_fcc(1, ncell=10)
    mass = np.array([dpsynth.MASS["Cu"]])
    vel = dpsynth.velocities(mass[typ], 300.0, 1)
    n = len(typ)
    peak, src = tensor_peak()
    points = []
    widths = [int(v) for v in args.sweep_widths.split(",")] if args.sweep_widths else [e[0] for e in SWEEP]
    precs = args.sweep_precisions.split(",")
    todo = [(e, "bf16") for e in SWEEP if e[0] in widths and "bf16" in precs]
    todo += [(e, "fp8") for e in SWEEP if e[0] >= 128 and e[0] in widths and "fp8" in precs]
    for emb, prec in todo:
        cfg = dpsynth.ModelConfig(ntypes=1, rcut=8.0, rcut_smth=2.0, sel=(512,), embed=emb)
        model = dp.Model(cfg, seed=1)
        stream = torch.cuda.Stream(device=dev)
        dp.dp_model_set_stream(model.h, stream)
        nl = dp.NeighborList(model, coord, typ, box)
        nnei = int((nl.get()[0] >= 0).sum())
        nl.close()
        fl = flops_per_group(cfg, nnei, n)
        steps = max(3, min(args.steps, 10 if emb[0] >= 256 else args.steps))
        state = dp.MDState(model, coord, vel, typ, mass, box, skin=2.0)
        state.step(max(3, min(args.warmup, 5)), 1.0, prec)
        dp.dp_profile_select(model.h, None)
        dp.dp_profile_enable(model.h, True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        state.step(steps, 1.0, prec)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        prof = dp.dp_profile_read(model.h)
        dp.dp_profile_enable(model.h, False)
        state.close()
        emb_ms = (prof.get("embed_fwd", (0, 0.0))[1] + prof.get("embed_bwd", (0, 0.0))[1]) / steps
        emb_fl = fl["embed_fwd"] + fl["embed_bwd"]
        total = sum(fl.values())
        # e4m3 products run at twice the dense bf16 rate (nominal 4.5 against 2.25 PFLOP/s)
        pk = peak * (2.0 if prec == "fp8" else 1.0)
        points.append({"embed": list(emb), "precision": prec, "last_layer": f"{emb[1]} x {emb[2]}",
                       "path": "fused per-tile kernels (tc.cu)" if emb[0] < 64 else "layer-wise GEMMs (wide.cu)",
                       "ms_per_step": ms, "s_per_step_atom": ms * 1e-3 / n, "mflop_per_atom_eval": total / n / 1e6,
                       "step_tflops": total / (ms * 1e-3) / 1e12, "step_frac_of_peak": total / (ms * 1e-3) / 1e12 / pk,
                       "embedding_ms": emb_ms, "embedding_tflops": emb_fl / (emb_ms * 1e-3) / 1e12 if emb_ms else None,
                       "embedding_frac_of_peak": emb_fl / (emb_ms * 1e-3) / 1e12 / pk if emb_ms else None,
                       "embedding_share_of_step": emb_ms / ms, "steps": steps})
        model.close()
    top = [p for p in points if p["precision"] == "bf16"][-1]
    return {"metric": "embedding-width sweep: s/step/atom and FLOP/s (MIX-16 bf16, and e4m3 for the wide nets)",
            "unit": "TFLOP/s", "value": top["step_tflops"], "higher_is_better": True, "n_gpus": world, "dtype": "bf16",
            "data": "synthetic (seeded FCC copper, seeded random-init weights)",
            "config": {"workload": "Cu FCC 10^3 cells, 4000 atoms, rcut 8, sel 512, M2 16, fitting 240-240-240, "
                                   "300 K, dt 1 fs", "atoms": n},
            "peak": {"tflops": peak, "source": src}, "points": points}


def run_e2e(dp, model, cfg, coord, vel, typ, box, mass, dt, args, stream):
    """dp_compute with host buffers every step; velocity Verlet on the host."""
    import torch
    n = len(typ)
    x = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    x[:] = coord
    v = vel.copy()
    minv = (9.648533212e-3 / mass[typ])[:, None]
    L = np.diag(box)
    nl = dp.NeighborList(model, x, typ, box, skin=2.0)
    for _ in range(2):   # untimed: the first call runs directly, the second captures the call's graph
        E, Ei, F, W = nl.compute(x, box, args.precision)
    steps = args.e2e_steps
    hdm = 0.5 * dt * minv                       # half kick per unit force
    disp = np.zeros_like(x)                     # displacement since the last list build
    tmp = np.empty_like(x)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        np.multiply(F, hdm, out=tmp)
        v += tmp
        np.multiply(v, dt, out=tmp)
        x += tmp
        disp += tmp
        np.floor(np.divide(x, L, out=tmp), out=tmp)
        tmp *= L
        x -= tmp                                # wrapped into [0, L)
        np.multiply(disp, disp, out=tmp)
        if tmp.sum(1).max() > 1.0:              # half the 2 A skin, squared
            nl.update(x, box)
            disp[:] = 0.0
        E, Ei, F, W = nl.compute(x, box, args.precision)
        np.multiply(F, hdm, out=tmp)
        v += tmp
    t1 = time.perf_counter()
    nl.close()
    step_s = (t1 - t0) / steps
    return {"value": step_s / n, "unit": "s/step/atom", "steps": steps, "ns_per_day": 86400.0 * dt * 1e-6 / step_s,
            "h2d_bytes_per_step": n * 3 * 8, "d2h_bytes_per_step": n * 3 * 8 + n * 8 + 10 * 8,
            "path": "dp_compute(host coord) -> host E, E_i, F, W; host velocity Verlet"}


def cpu_baseline(args, name=None, budget_s=15.0, md_steps=True):
    """The cpu_baseline leg: the FP64 oracle on the host cores, on the same workload.

    Times one oracle evaluation (energy, forces, virial) of the initial coordinates and, with
    md_steps, whole oracle NVE steps within about budget_s seconds.  Returns (baseline record,
    the oracle's evaluation (E, E_i, F, W) of the initial coordinates): that evaluation is the
    reference of the paths' error columns."""
    import oracle
    name = name or args.workload
    cfg, coord, typ, box, mass, dt, desc = workload(name, args.model)
    n = len(typ)
    params = dpsynth.model_params(cfg, 1)
    om = oracle.Model(cfg, params)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    E, Ei, F, W = om.compute(coord, typ, box, nthreads=cores)
    one_eval = time.perf_counter() - t0
    ref = (E, Ei, F, W)
    if not md_steps:
        return ({"value": one_eval / n, "unit": "s/step/atom", "cores": cores, "kind": "oracle",
                 "sample": f"one FP64 oracle evaluation (energy, forces, virial) of the {desc} workload; "
                           "an NVE step adds only the two half kicks and the drift"}, ref)
    vel = dpsynth.velocities(mass[typ], md_protocol(name, 1)[0], 1)
    steps = max(1, min(20, int(budget_s / max(one_eval, 1e-3))))
    t0 = time.perf_counter()
    om.md_nve(coord, vel, typ, mass, box, nsteps=steps, dt=dt, thermo_every=0, nthreads=cores)
    el = time.perf_counter() - t0
    return ({"value": el / steps / n, "unit": "s/step/atom", "cores": cores, "kind": "oracle",
             "sample": f"{steps} full NVE steps of the {desc} workload (FP64 oracle, OpenMP over atoms)"}, ref)


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle's NVE steps on the host cores, same workload and metric.

    args.warmup untimed oracle steps (at most 5), then args.steps timed ones.  The config carries
    the same keys as the GPU arm's line."""
    if rank != 0:
        return None
    import oracle
    cfg, coord, typ, box, mass, dt, desc = workload(args.workload, args.model)
    n = len(typ)
    om = oracle.Model(cfg, dpsynth.model_params(cfg, 1))
    nl, _, _ = om.nlist(coord, typ, box)
    nnei_total = int((nl >= 0).sum())
    vel = dpsynth.velocities(mass[typ], md_protocol(args.workload, 1)[0], 1)
    cores = os.cpu_count() or 1
    x, v = coord, vel
    warm = min(args.warmup, 5)
    if warm > 0:
        x, v, _ = om.md_nve(x, v, typ, mass, box, nsteps=warm, dt=dt, thermo_every=0, nthreads=cores)
    t0 = time.perf_counter()
    x, v, th = om.md_nve(x, v, typ, mass, box, nsteps=args.steps, dt=dt, thermo_every=args.steps, nthreads=cores)
    el = time.perf_counter() - t0
    value = el / args.steps / n
    base = {"value": value, "unit": "s/step/atom", "cores": cores, "kind": "oracle",
            "sample": f"{args.steps} full NVE steps of the {desc} workload after {warm} untimed ones"}
    return {"impl": "reference", "metric": "s/step/atom", "value": value, "unit": "s/step/atom", "n_gpus": world,
            "steps": args.steps, "warmup": warm, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "ns_per_day": 86400.0 * dt * 1e-6 / (el / args.steps), "dtype": "f64", "precision": "fp64",
            "data": "synthetic (seeded FCC copper / water, seeded random-init weights)",
            "config": {"workload": desc, "atoms": n, "precision": "fp64", "real_neighbors": nnei_total,
                       "l2": "host run (no GPU cache)", "parallelism": f"host, OpenMP over atoms on {cores} cores",
                       "launch": "oracle NVE steps (plain C, FP64)", "profiling": "wall clock around the timed steps"},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": "s/step/atom", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mix32", "bf16", "fp16", "bf16x3"])
    ap.add_argument("--workload", default="cu4000")
    ap.add_argument("--model", default="full", choices=["full", "student"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--paths", default=",".join(PATHS),
                    help="comma-separated paths timed beside the headline with their errors "
                         "(fp64, mix32, bf16, fp16, bf16x3, student, student_judged), or 'none'")
    ap.add_argument("--paths-workloads", default="cu4000,cu108k,water12k",
                    help="workloads of the paths blocks when the headline is the default FP64 copper 4,000 line")
    ap.add_argument("--temps", default="300,1200", help="judged task: teacher MD temperatures (K)")
    ap.add_argument("--frames-per-temp", type=int, default=24, help="judged task: teacher frames per temperature")
    ap.add_argument("--adam-steps", type=int, default=800, help="judged task: student training steps")
    ap.add_argument("--relative-force-loss", action="store_true",
                    help="judged task: weight each frame's force loss by 1 / its RMS force squared")
    ap.add_argument("--frames-per-run", default="0",
                    help="judged task: frames per teacher run (0: one run per temperature), one value or one "
                         "per temperature (comma-separated)")
    ap.add_argument("--teacher-md-precision", default="",
                    help="judged task: precision of the teacher's MD (default bf16x3 fitted, mix32 seeded)")
    ap.add_argument("--label-precision", default="",
                    help="judged task: precision of the teacher's labels (default bf16x3 fitted, mix32 seeded)")
    ap.add_argument("--teacher", default="fitted", choices=["fitted", "seeded"],
                    help="judged task: the full model fitted to the Morse copper reference, or the seeded model")
    ap.add_argument("--teacher-fit-steps", type=int, default=20000, help="judged task: Adam steps of the teacher fit")
    ap.add_argument("--teacher-fit-frames", type=int, default=512, help="judged task: Morse frames of the teacher fit")
    ap.add_argument("--judge-precision", default="",
                    help="judged task: precision of the judge (default bf16x3 fitted, --precision seeded)")
    ap.add_argument("--sweep-widths", default="", help="sweep task: first widths w of the nets (w, 2w, 4w) to run "
                    "(comma-separated; default all)")
    ap.add_argument("--sweep-precisions", default="bf16,fp8", help="sweep task: bf16 and/or fp8")
    ap.add_argument("--task", default="md", choices=["md", "grad", "judged", "sweep", "train"],
                    help="md: NVE steps (default); grad: force-loss parameter gradient over 32 water frames; "
                         "judged: distilled student MD judged by the full model; train: training steps of "
                         "config 4's teacher fit and distillation")
    args = ap.parse_args()
    args.paths = [] if args.paths in ("", "none") else [p for p in args.paths.split(",") if p]
    for p in args.paths:
        if p not in PATHS:
            raise SystemExit(f"unknown path {p}")
    if args.warmup < 3 and args.impl == "mine":
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl" if args.impl == "mine" else "gloo")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.task == "grad":
        out = run_grad(args, rank, world)
    elif args.task == "judged":
        out = run_judged(args, rank, world)
    elif args.task == "sweep":
        out = run_sweep(args, rank, world)
    elif args.task == "train":
        out = run_train(args, rank, world)
    else:
        out = run_mine(args, rank, world)
        ref = None
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"], ref = cpu_baseline(args)
        if rank == 0 and world == 1 and args.paths and args.model == "full":
            out["paths"] = paths_blocks(args, out, ref)
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


def paths_blocks(args, out, ref):
    """The paths blocks: the headline workload, then (for the default copper 4,000 headline) the
    other workloads of --paths-workloads, each with its own oracle reference when the cpu_baseline
    leg runs."""
    import torch

    import paper_2005_00223_gb300 as dp
    from paper_2005_00223_gb300 import student as S

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    student = None
    if any(p.startswith("student") for p in args.paths):
        t0 = time.perf_counter()
        teacher, stu, frms, _, _, _ = distil_student(dp, S, dev)
        student = (teacher, stu)
        distil_s = time.perf_counter() - t0
    kind = "FP64 oracle (cpu_baseline leg)" if ref is not None else "FP64 GPU path (oracle not run)"
    fp64_ms = out["ms_per_step"] if args.precision == "fp64" else None
    blocks = {args.workload: run_paths(args, args.workload, args.steps, args.warmup, ref, kind, fp64_ms, student)}
    if args.workload == "cu4000" and args.precision == "fp64":
        for name in args.paths_workloads.split(","):
            if not name or name == args.workload:
                continue
            ref2 = None
            if not args.no_cpu_baseline:
                base2, ref2 = cpu_baseline(args, name=name, md_steps=False)
            steps = max(JUDGE_EVERY, min(args.steps, 10), MD_REBUILD.get(name, 0))
            blocks[name] = run_paths(args, name, steps, min(args.warmup, 5), ref2,
                                     "FP64 oracle (cpu_baseline leg)" if ref2 is not None else
                                     "FP64 GPU path (oracle not run)", None, student)
            if ref2 is not None:
                blocks[name]["cpu_baseline"] = base2
    if student is not None:
        blocks["student_training"] = {
            "teacher": "the seeded full copper model", "frames": "48 (24 every 5 NVE steps at 300 K and 1200 K, "
            "4000 atoms)", "adam_steps": 800, "teacher_rms_force_eV_per_A": frms, "seconds": distil_s,
            "kernels": "dp_md_step, dp_compute (labels), dp_force_loss_grad_dev, dp_adam_step"}
        student[0].close()
        student[1].close()
    return blocks


if __name__ == "__main__":
    main()
