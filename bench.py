#!/usr/bin/env python
"""Benchmark: milliseconds per local-global iteration on the 57k-DoF star-pull scene.

Workload (synthetic stand-in for the paper's "crossing gingerbread man" teaser scene:
58.5k DoFs, 800 contacts, 5 local-global iterations per frame): an extruded five-point
star (19,926 vertices, 59,778 DoFs, 101,400 tetrahedra), stable Neo-Hookean E = 1e6 Pa,
nu = 0.45, rho = 1000, its leading cap pinned to a handle moving at 0.5 m/s through a
seeded 4 x 4 array of fixed cylinders (mu = 0.3); h = 1/60 s, 5 iterations and 10 CR
iterations per frame, FP32 device arithmetic (FP64 state and contact logic).

A step is one frame (collision, Delassus operator, 5 local-global iterations,
integration) from one fixed contact state: the rest-shape star translated along the pull
direction until its leading face is 9.4 cm beyond the axes of the first cylinder row,
moving at the pull speed (837 contacts at 837 contact vertices after the frame's
prediction step; the paper's scene peaks at 800); every timed step
replays that frame. The state is plain geometry of the scene, so both arms (and the CPU
baseline) start from exactly the same input. Each step's device time comes from
CUDA event nodes inside the frame's graph (launch stream); L2 is flushed (256 MB write)
before every timed step. value = mean frame time / iterations per frame, the paper's
own ms/iteration definition (frame time including the per-frame Delassus work, divided
by the iteration count).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms/local-global iter @58.5k DoFs; frame ms to 1e-4 residual, learned vs plain"
# DRAM bytes (read + write) per launch of the profile products in their register form
# (k_pass1 / k_pass2) on the placed star of this lattice, mean of both, from one ncu capture
# (dram__bytes.sum.per_second x gpu__time_duration.sum); keyed by (precision, n_side) and
# valid while those kernels are unchanged
PRODUCT_TRAFFIC_BYTES = {("fp32", 43): 112.25e6}
UNIT = "ms/iter"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--placement", type=float, default=0.094,
                    help="metres the star is moved past first touching the cylinders")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-side", type=int, default=43)
    ap.add_argument("--s-precision", choices=["fp32", "bf16"], default="fp32",
                    help="storage of the S~ values (bf16: FP32 accumulation)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the timing of the paper's variants on the star frame")
    ap.add_argument("--no-warmstart", action="store_true",
                    help="skip the learned-vs-plain frame time to residual 1e-4")
    ap.add_argument("--no-batch64", action="store_true",
                    help="skip the 64-scene BF16 batch sub-record")
    ap.add_argument("--no-trajectory", action="store_true",
                    help="skip the 300-frame pulls through the cylinders (seeds 0-4)")
    ap.add_argument("--workload", choices=["star", "batch64", "stack"], default="star",
                    help="star: the 57k-DoF pulled star (the headline); batch64: 64 uneven "
                         "cubes on tilted planes in one simulator; stack: the stress case, "
                         "8 x 32 stiff boxes of 12^3 vertices with box-box contacts")
    ap.add_argument("--autotune", type=int, default=1,
                    help="1: let the library time the products' launch configurations")
    ap.add_argument("--refine", type=int, default=1,
                    help="bf16 only: residual corrections, 0 none, 1 last iteration, 2 every")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value, device="cuda"):
    """The largest value over the ranks of the default process group (the job's time is
    its slowest rank's); the value itself without a group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6400.0), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """SM clocks and clock-event (throttle) reasons sampled every 10 ms during the timed
    region, through NVML (the same counters nvidia-smi reports); falls back to an
    nvidia-smi subprocess if NVML is unavailable."""

    BITS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown",
            0x4: "sw_power_cap", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index):
        self.cuda_index = cuda_index
        self.samples = []
        self.stop = False
        self.thread = None
        self.handle = None

    def _handle(self):
        import pynvml
        pynvml.nvmlInit()
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.cuda_index).uuid)
            if not uuid.startswith("GPU-"):
                uuid = "GPU-" + uuid
            return pynvml, pynvml.nvmlDeviceGetHandleByUUID(uuid)
        except Exception:
            return pynvml, pynvml.nvmlDeviceGetHandleByIndex(self.cuda_index)

    def _loop(self):
        nv, h = self.nv, self.handle
        get_reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            nv.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop:
            try:
                self.samples.append((nv.nvmlDeviceGetClockInfo(h, nv.NVML_CLOCK_SM),
                                     nv.nvmlDeviceGetMaxClockInfo(h, nv.NVML_CLOCK_SM),
                                     int(get_reasons(h))))
            except Exception:
                pass
            time.sleep(0.01)

    SMI = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
           "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
           "clocks_event_reasons.sw_power_cap")

    def _smi_loop(self):
        # nvidia-smi fallback: one query per 20 ms
        names = [0x8, 0x40, 0x20, 0x4]
        while not self.stop:
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.cuda_index}",
                                      f"--query-gpu={self.SMI}", "--format=csv,noheader,nounits"],
                                     capture_output=True, text=True, timeout=5).stdout
                parts = [x.strip() for x in out.strip().split(",")]
                bits = 0
                for b, val in zip(names, parts[2:6]):
                    if val.lower() == "active":
                        bits |= b
                self.samples.append((float(parts[0]), float(parts[1]), bits))
            except Exception as e:
                self.error = f"{type(e).__name__}: {e}"[:200]
            time.sleep(0.02)

    def __enter__(self):
        import threading
        self.error = None
        self.source = "nvml"
        try:
            self.nv, self.handle = self._handle()
            target = self._loop
        except Exception as e:          # no NVML binding: use nvidia-smi
            self.error = f"{type(e).__name__}: {e}"[:200]
            self.source = "nvidia-smi"
            target = self._smi_loop
        self.thread = threading.Thread(target=target, daemon=True)
        self.thread.start()
        time.sleep(0.05)
        return self

    def __exit__(self, *a):
        self.stop = True
        if self.thread is not None:
            self.thread.join(timeout=6)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0,
                    "error": self.error}
        reasons = set()
        for _, _, bits in self.samples:
            for b, name in self.BITS.items():
                if bits & b:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(x[0] for x in self.samples),
                "sm_max_mhz": max(x[1] for x in self.samples), "reasons": sorted(reasons),
                "samples": len(self.samples), "source": self.source}


# ----------------------------------------------------------------------------------------
# CPU oracle timing (bounded sample): shared by cpu_baseline and the reference arm
# ----------------------------------------------------------------------------------------
try:
    from threadpoolctl import threadpool_limits as _single_thread
    _HAVE_TPC = True
except ImportError:          # BLAS threads stay at their default; reported in "cores"
    import contextlib

    _HAVE_TPC = False

    def _single_thread(_n):
        return contextlib.nullcontext()


class OracleTimer:
    """Times the FP64 oracle on a benchmark state: the per-frame work (detection, and W
    from a subsample of its 3c direct solves scaled to all of them) once, then full
    local-global iterations (local step, RHS, FB evaluation, Schur right-hand side,
    conjugate residual on a 3c x 3c operator, final solve) one at a time. The one-time
    factorisation is not timed (it is the oracle's counterpart of the precompute)."""

    def __init__(self, scene, q, v, n_iters, w_cols=60):
        import numpy as np
        from oracle import Oracle
        from oracle import contact as C
        self.np, self.C, self.limits = np, C, _single_thread
        self.cores = 1 if _HAVE_TPC else (os.cpu_count() or 1)
        self.scene, self.q, self.v, self.n_iters = scene, q, v, n_iters
        with _single_thread(1):
            o = self.o = Oracle(scene)
            f = o.fem
            f.solve(np.zeros(len(f.free_dofs)))
            t0 = time.perf_counter()
            self.s_tilde = o.predict(q, v)
            self.contacts = C.detect(scene, self.s_tilde, f.free_verts)
            self.t_detect = time.perf_counter() - t0
            c = self.c = len(self.contacts)
            self.H = o.contact_jacobian(self.contacts)
            self.ncols = min(3 * c, w_cols)
            t0 = time.perf_counter()
            if self.ncols:
                f.solve(self.H[:self.ncols].T.copy())
            self.t_w = (time.perf_counter() - t0) * (3 * c / max(self.ncols, 1))
            rng = np.random.default_rng(0)
            B = rng.normal(size=(3 * c, 3 * c)) if c else np.zeros((0, 0))
            self.W = B @ B.T / max(3 * c, 1) + np.eye(3 * c) if c else np.zeros((0, 0))

    def iteration_seconds(self):
        np, C, o = self.np, self.C, self.o
        f = o.fem
        c = self.c
        with self.limits(1):
            q_it = self.s_tilde.copy()
            q_it[o.fem.pin_verts] = o.pinned_positions(self.q)
            lam = np.zeros((c, 3))
            r_n = np.full(c, 1e-6)
            r_f = np.full(c, 1e-4)
            t0 = time.perf_counter()
            p = o.local_step(q_it)
            b = f.assemble_rhs(self.s_tilde, p, o.pinned_positions(self.q))
            qf = q_it[f.free_verts].reshape(-1)
            if c:
                cs = o.contact_state(qf, self.q[f.free_verts].reshape(-1), lam, self.H,
                                     self.contacts, r_n, r_f)
                Om = cs["omega"].reshape(-1)
                J = Om[:, None] * self.H
                g = b + o.h ** 2 * (J.T @ lam.reshape(-1))
                rhs = J @ qf - J @ f.solve(g)
                K = Om[:, None] * self.W * Om[None, :] + np.diag((cs["E"] + 1e-9).reshape(-1))
                dl = C.conjugate_residual(lambda x: K @ x, rhs, 10)
                f.solve(b + o.h ** 2 * (J.T @ dl))
            else:
                f.solve(b)
            return time.perf_counter() - t0

    def ms_per_iteration(self, t_iter):
        return 1e3 * (t_iter + (self.t_detect + self.t_w) / self.n_iters)

    def description(self, n_timed):
        threads = "1 thread" if _HAVE_TPC else f"numpy/BLAS default threads (<= {self.cores})"
        return (f"FP64 oracle, {threads}, star_pull state with {self.c} contacts: detection "
                f"once, W from {self.ncols} of its {3 * self.c} direct solves scaled to all, "
                f"{n_timed} full local-global iteration(s); per-frame work divided by "
                f"{self.n_iters} iterations")


def contact_state(scene, placement):
    """The placed star: the rest shape moved `placement` metres past the first cylinder
    row's axes, moving at the pull speed (scenegen.star_placed; pure geometry)."""
    import scenegen as sg
    return sg.star_placed(scene, placement)


def batch_state(scenes):
    """Every cube moved along its plane's normal until its lowest vertex is a quarter of
    its lattice spacing inside the plane (pure geometry), at rest."""
    import numpy as np
    qs, vs = [], []
    for sc in scenes:
        pl = sc.obstacles[0]
        n = np.asarray(pl.axis, dtype=np.float64)
        n = n / np.linalg.norm(n)
        dist = (sc.q0 - np.asarray(pl.p)) @ n
        qs.append(sc.q0 - (dist.min() + 0.25 * sc.spacing) * n)
        vs.append(np.zeros_like(sc.q0))
    return np.concatenate(qs), np.concatenate(vs)


def warmstart_ab():
    """The second half of the metric: frame time to residual 1e-4, learned warm start vs the
    plain cold start, on the 6^3 cube drops (train on 16 seeds, 80 frames each, from frames
    the plain method solved; evaluate on 5 held-out seeds, every contact frame replayed from
    the same state with each start). Iterations and frame milliseconds are measured with
    frames that stop on the device when R <= 1e-4 (at least 1, at most 40 updates; the
    frame's device time from its first to its last event node); the residual after 5
    iterations comes from 40-iteration replays. "portfolio" runs the learned start beside
    the cold one as a two-copy batch and stops when either copy is done."""
    import numpy as np
    import scenegen as sg
    from paper_2503_15078_b300 import warmstart
    t0 = time.perf_counter()
    X, T = warmstart.collect(sg.warmstart_scenes(range(0, 16), frames=80), frames=80, n_iters=20)
    Xv, Tv = warmstart.collect(sg.warmstart_scenes(range(200, 204), frames=80), frames=80,
                               n_iters=20)
    net, losses = warmstart.train(X, T, epochs=60, batch=512, lr=1e-3, seed=0, X_val=Xv, T_val=Tv)
    # the blend of the network's outputs with the previous frame's start, chosen on the
    # validation seeds by frame time to the tolerance
    gains, table = warmstart.choose_gains(net, sg.warmstart_scenes(range(200, 204), frames=60),
                                          60)
    modes = ["cold", "previous", "learned", "portfolio"]
    held_out = sg.warmstart_scenes(range(100, 105), frames=60)
    traces = warmstart.evaluate_from_states(held_out, 60, modes, net=net, gains=gains)
    timed = warmstart.evaluate_to_tolerance(held_out, 60, modes, net=net, gains=gains)
    out = {"workload": "6^3 cube drops (config-1 scene, seeded height/rotation/tilt); 16 "
                       "training seeds x 80 frames, 4 validation seeds (output shrinkage), "
                       "5 held-out seeds x 60 frames",
           "training_samples": int(len(X)), "train_loss": [float(losses[0]), float(losses[-1])],
           "tolerance": 1e-4, "max_iters": 40,
           "gains": {"persist": gains[0], "fresh": gains[1], "move": gains[2],
                     "accept": gains[3],
                     "validation": {",".join(str(x) for x in g): [round(v[0], 2), round(v[1], 4)]
                                    for g, v in table.items()}}}
    for m in modes:
        R5 = traces[m]["residuals"][:, 5]
        r = timed[m]
        out[m] = {"frames": r["frames"], "mean_iters_to_tol": round(r["mean_iters"], 2),
                  "median_iters_to_tol": r["median_iters"], "at_max_iters": r["at_cap"],
                  "mean_frame_ms_to_tol": round(r["mean_ms"], 4),
                  "median_frame_ms_to_tol": round(r["median_ms"], 4),
                  "mean_log10_residual_after_5_iters":
                      round(float(np.nanmean(np.log10(np.maximum(R5, 1e-16)))), 3)}
    out["seconds"] = round(time.perf_counter() - t0, 1)
    net.close()
    return out


def variants_timing(scene, q0, v0, steps, flush):
    """The placed star frame with each of the paper's variants (and ADMM-PD and the anchored
    handle): device ms per local-global iteration of the production graph, mean over
    `steps` replays after 3 warm-ups, L2 flushed before each; the variant's final residual
    is reported with it."""
    import numpy as np
    import torch
    import scenegen as sg
    from paper_2503_15078_b300 import Simulator
    cases = {"minmap": dict(ncp="minmap"), "mass_precond": dict(precond="mass"),
             "admm_pd": dict(local_solver="admm"), "anchored_handle": {},
             "cr_cluster_barriers": dict(cr_sync=1), "cr_one_exchange": dict(cr_exchanges=1)}
    out = {}
    for name, kw in cases.items():
        sc, v = scene, v0.copy()
        if name == "anchored_handle":
            # the handle's vertices free, tied by hard anchors to targets that start where
            # the placed state has them and move with the handle
            sc = sg.anchored_handle(scene)
            sc.anchors = [sg.Anchor(a.vertex, tuple(q0[a.vertex]), a.vel, 0.0)
                          for a in sc.anchors]
            v[scene.pinned] = np.asarray(scene.handle_vel)
        sim = Simulator(sc, autotune=0, phase_marks=0, **kw)
        times, res = [], []
        for k in range(3 + steps):
            sim.set_state(q0, v)
            flush.zero_()
            torch.cuda.synchronize()
            sim.step()
            ph = sim.phase_times()
            if k >= 3:
                times.append(sum(ph.values()) / sc.n_iters)
                res.append(sim.stats()["residuals"][-1])
        out[name] = {"ms_per_iter": round(statistics.mean(times), 5),
                     "contacts": sim.stats()["n_contacts"],
                     "final_residual": float(f"{statistics.mean(res):.3e}")}
        sim.close()
    # a sheet of the paper's cloth size (20.2k vertices, 40k triangles) with Laplace-Beltrami
    # bending, lying across a cylinder (its middle rows in contact), from rest
    cyl = sg.Obstacle(sg.OBST_CYLINDER, (0.0, 0.0, -0.018), (1.0, 0.0, 0.0), radius=0.02,
                      mu=0.3)
    sheet = sg.cloth(n=142, size=1.0, model=sg.MODEL_COROT, bending=1e-4, pin="none",
                     height=0.0, obstacles=[cyl])
    sim = Simulator(sheet, autotune=0, phase_marks=0)
    times, res = [], []
    for k in range(3 + steps):
        sim.set_state(sheet.q0, sheet.v0)
        flush.zero_()
        torch.cuda.synchronize()
        sim.step()
        if k >= 3:
            times.append(sum(sim.phase_times().values()) / sheet.n_iters)
            res.append(sim.stats()["residuals"][-1])
    info = sim.plan_info()
    out["cloth_20k_bending"] = {"ms_per_iter": round(statistics.mean(times), 5),
                                "contacts": sim.stats()["n_contacts"],
                                "final_residual": float(f"{statistics.mean(res):.3e}"),
                                "verts": sheet.n_verts, "tris": int(len(sheet.tris)),
                                "nnz_S": info["nnz_S"]}
    sim.close()
    out["twisting_bar_20k"] = twisting_bar_timing(steps, flush)
    return out


def twisting_bar_timing(steps, flush):
    """The paper's largest twisting bar (its Tab. of timings: 20.8k vertices, ARAP, E = 1e9,
    nu = 0.45, rho = 1000) as a 12 x 12 x 145 lattice (20,880 vertices, 104.5k tets), the top
    turned 45 degrees: device ms per local-global iteration of the production graph with the
    complete global step (x = S^T S b) and with the single Jacobi sweep of Sec. 8's baseline,
    the instrumented graph's split of one iteration into local and global time, and how far
    the baseline's 60-iteration frame still is from the complete one (relative displacement)."""
    import numpy as np
    import torch
    import scenegen as sg
    from paper_2503_15078_b300 import Simulator
    bar = sg.twisting_bar(nxy=12, nz=145, spacing=0.01, E=1e9, nu=0.45, rho=1000.0)
    out = {"verts": bar.n_verts, "tets": int(len(bar.tets)), "iters": 10}
    q60 = {}
    for name, kw in (("complete", {}), ("jacobi1", dict(global_solver="jacobi",
                                                          jacobi_sweeps=1))):
        prod = Simulator(bar, autotune=0, phase_marks=0, **kw)
        inst = Simulator(bar, autotune=0, phase_marks=1, **kw)
        times, split = [], []
        for k in range(3 + steps):
            for sim, acc in ((prod, times), (inst, split)):
                sim.set_state(bar.q0, bar.v0)
                flush.zero_()
                torch.cuda.synchronize()
                sim.step(n_iters=10)
                if k >= 3:
                    acc.append(sim.phase_times())
        glob = ("spmv1", "reduce", "solve", "spmv2")
        out[name] = {
            "ms_per_iter": round(statistics.mean(sum(t.values()) for t in times) / 10, 5),
            "local_ms_per_iter": round(statistics.mean(t["local"] for t in split) / 10, 5),
            "global_ms_per_iter": round(statistics.mean(sum(t.get(g, 0.0) for g in glob)
                                                        for t in split) / 10, 5)}
        prod.set_state(bar.q0, bar.v0)
        prod.step(n_iters=60)
        q60[name] = prod.state()[0]
        prod.close()
        inst.close()
    out["jacobi1_gap_at_60_iters"] = float(f"{np.linalg.norm(q60['jacobi1'] - q60['complete']) / np.linalg.norm(q60['complete'] - bar.q0):.3e}")
    return out


def pull_trajectory(n_side, frames, seeds, steps, flush):
    """The config-2 scene as a trajectory: the star's pinned cap pulled at 0.5 m/s through the
    seeded 4 x 4 cylinder field for `frames` frames (5 local-global and 10 CR iterations each)
    for every seed, from rest, in the production graph. Per seed: contact counts (max, mean
    over frames with contact), the last iteration's residual R (max, median over contact
    frames), the largest penetration (as a fraction of the scene's residual length),
    finiteness, and the device time per frame. Then the frame with the most contacts of seed
    0 is replayed `steps` times from its start state (L2 flushed before each) and timed as
    ms per local-global iteration."""
    import numpy as np
    import torch
    import scenegen as sg
    from paper_2503_15078_b300 import SimError, Simulator
    out = {"frames": frames, "seeds": list(seeds), "per_seed": []}
    peak = None
    for seed in seeds:
        sc = sg.star_pull(n_side=n_side, seed=seed)
        sim = Simulator(sc, autotune=0, phase_marks=0)
        L = sc.bbox_diagonal
        cts, res, pen, ms, finite = [], [], [], [], True
        prev = sim.state()
        for f in range(frames):
            try:
                sim.step()
                st = sim.stats()
            except SimError:
                finite = False
                break
            ms.append(sum(sim.phase_times().values()))
            cts.append(st["n_contacts"])
            if st["n_contacts"]:
                res.append(st["residuals"][-1])
                pen.append(st["max_penetration"] / L)
            if seed == seeds[0] and (peak is None or st["n_contacts"] > peak[0]):
                peak = (st["n_contacts"], f, prev)
            if seed == seeds[0]:
                prev = sim.state()
        q, v = sim.state()
        finite = finite and bool(np.all(np.isfinite(q)) and np.all(np.isfinite(v)))
        cf = [c for c in cts if c]
        out["per_seed"].append({
            "seed": seed, "finite": finite, "frames_run": len(cts),
            "contact_frames": len(cf), "max_contacts": max(cts) if cts else 0,
            "mean_contacts": round(float(np.mean(cf)), 1) if cf else 0.0,
            "max_residual": float(f"{max(res):.3e}") if res else 0.0,
            "median_residual": float(f"{np.median(res):.3e}") if res else 0.0,
            "max_penetration_over_L": float(f"{max(pen):.3e}") if pen else 0.0,
            "mean_frame_ms": round(float(np.mean(ms)), 4) if ms else None,
            "max_frame_ms": round(float(np.max(ms)), 4) if ms else None})
        sim.close()
    if peak is not None and peak[0] > 0:
        sc = sg.star_pull(n_side=n_side, seed=seeds[0])
        sim = Simulator(sc, autotune=1, phase_marks=0)
        times = []
        for k in range(3 + steps):
            sim.set_state(*peak[2])
            flush.zero_()
            torch.cuda.synchronize()
            sim.step()
            if k >= 3:
                times.append(sum(sim.phase_times().values()) / sc.n_iters)
        out["peak_frame"] = {"seed": seeds[0], "frame": peak[1], "contacts": peak[0],
                             "ms_per_iter": round(statistics.mean(times), 5),
                             "final_residual": float(f"{sim.stats()['residuals'][-1]:.3e}")}
        sim.close()
    return out


def batch64_record(steps, flush):
    """The batch workload as a sub-record of the default run: 64 cubes of 8^3..20^3 vertices
    (seeded; mixed materials, tilted planes) in one simulator, S~ in BF16 with FP32
    accumulation and one FP32 residual correction per frame, each placed a quarter lattice
    spacing into its plane; every step replays one frame (L2 flushed before it). Reports ms
    per local-global iteration of the whole batch and the products' roofline on their BF16
    bytes (per launch, mean of both products, timed by the instrumented graph's event
    nodes)."""
    import torch
    import scenegen as sg
    from paper_2503_15078_b300 import Simulator
    scenes = sg.batch(n_scenes=64, seed=0)
    q0, v0 = batch_state(scenes)
    sim = Simulator(scenes, s_precision=1, refine=1, autotune=1, contact_capacity=16384)
    n_iters = scenes[0].n_iters
    prod, inst = [], []
    for marks, acc in ((False, prod), (True, inst)):
        sim.set_phase_marks(marks)
        for k in range(3 + steps):
            sim.set_state(q0, v0)
            flush.zero_()
            torch.cuda.synchronize()
            sim.step()
            if k >= 3:
                acc.append(sim.phase_times())
    info = sim.plan_info()
    ph = {k: statistics.mean(p[k] for p in inst) for k in inst[0]}
    t_pass = (ph["spmv1"] + ph["spmv2"]) / (2 * n_iters)
    bytes_pass = 2 * info["nnz_S"] + 2 * 12 * info["n_free"]
    peak, kind = measured_peaks()
    out = {"scenes": 64, "dofs": 3 * sim.n_verts, "nnz_S": info["nnz_S"],
           "contacts": sim.stats()["n_contacts"], "s_precision": "bf16", "refine": 1,
           "ms_per_iter": round(statistics.mean(sum(p.values()) for p in prod) / n_iters, 5),
           "roofline": {"kernel": "S~ profile products, BF16 values (mean of both, per launch)",
                        "bound": "hbm", "achieved": round(bytes_pass / (t_pass * 1e-3) / 1e9, 1),
                        "peak": peak, "peak_source": kind, "unit": "GB/s",
                        "frac": round(bytes_pass / (t_pass * 1e-3) / 1e9 / peak, 4),
                        "algorithmic_bytes_per_pass": bytes_pass}}
    sim.close()
    return out


def run_ours(args):
    import numpy as np
    import torch
    import scenegen as sg
    from paper_2503_15078_b300 import Simulator

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    batch = args.workload in ("batch64", "stack")
    stack = args.workload == "stack"
    n_batch = 0
    if batch:
        # one batch, split over the ranks by scene (nnz(S~)-balanced, no data-path exchange);
        # each rank simulates its own scenes in one simulator
        from paper_2503_15078_b300 import shard
        scenes = sg.stack_stress(seed=0) if stack else sg.batch(n_scenes=64, seed=0)
        n_batch = len(scenes)
        if world > 1:
            _, scenes = shard.shard(scenes, rank, world)
        scene = scenes[0]
    if stack:
        q0 = np.concatenate([sc.q0 for sc in scenes])
        v0 = np.zeros_like(q0)
    elif batch:
        if args.s_precision == "fp32" and "--s-precision" not in sys.argv:
            args.s_precision = "bf16"   # the batch workload stores S~ in BF16 by definition
        q0, v0 = batch_state(scenes)
    else:
        scene = sg.star_pull(n_side=args.n_side, seed=rank)
        q0, v0 = contact_state(scene, args.placement)
    bf16 = args.s_precision == "bf16"
    sim = Simulator(scenes if batch else scene, s_precision=1 if bf16 else 0,
                    refine=args.refine, autotune=args.autotune,
                    contact_capacity=65536 if stack else (16384 if batch else 4096))
    n_iters = scene.n_iters
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    # the one-time precompute: host ordering, symbolic analysis and FP64 Cholesky, then
    # S~ = L~^-1 P on the device in FP64; the host build of S~ for comparison
    pinfo = sim.plan_info()
    precompute = {"host_factor_seconds": round(pinfo["precompute_seconds"], 3),
                  "s_build_seconds": round(pinfo["s_build_seconds"], 4),
                  "s_built_on_device": pinfo["s_built_on_device"]}
    if not batch:
        from paper_2503_15078_b300 import Plan
        hp = Plan(scene).info()
        precompute["host_s_build_seconds"] = round(hp["s_build_seconds"], 3)
        precompute["host_total_seconds"] = round(hp["precompute_seconds"], 3)

    def one_step():
        # every step replays the same frame from the placed contact state;
        # the state upload and the L2 flush happen before the frame's graph starts, so the
        # device time (event nodes inside the graph) excludes them
        sim.set_state(q0, v0)
        flush.zero_()
        torch.cuda.synchronize()
        sim.step()
        return sim.phase_times()

    # two graphs of the same simulator (same launch configuration): the production frame,
    # with event nodes only around its once-per-frame phases, gives the value; the
    # instrumented frame, with event nodes around every phase of every iteration (each
    # costs a few microseconds), gives the per-phase times and the products' roofline
    sim.set_phase_marks(False)
    for _ in range(max(3, args.warmup)):
        one_step()
    sim.set_phase_marks(True)
    for _ in range(max(3, args.warmup)):
        one_step()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    frames, prod_frames, contacts = [], [], []
    with ClockSampler(local) as clk:
        sim.set_phase_marks(False)
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            prod_frames.append(one_step())
            contacts.append(sim.stats()["n_contacts"])
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        sim.set_phase_marks(True)
        for _ in range(args.steps):
            frames.append(one_step())
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.summary()
    frame_ms = sorted(sum(p.values()) for p in prod_frames)
    mean_frame = statistics.mean(frame_ms)
    mean_frame = max_over_ranks(mean_frame)
    spread = {"median_ms_per_iter": round(statistics.median(frame_ms) / n_iters, 5),
              "p10_ms_per_iter": round(frame_ms[len(frame_ms) // 10] / n_iters, 5),
              "p90_ms_per_iter": round(frame_ms[(9 * len(frame_ms)) // 10] / n_iters, 5),
              "timed_frames": len(frame_ms)}
    instrumented_frame = statistics.mean(sum(p.values()) for p in frames)
    phase_mean = {k: statistics.mean(p[k] for p in frames) for k in frames[0]}
    stats = sim.stats()
    # ---- roofline of the dominant kernels: the two S~ profile products -----------------
    info = sim.plan_info()
    nnz = info["nnz_S"]
    n_free = info["n_free"]
    # S~ values (4 or 2 bytes) + input and output vectors (FP32 triples)
    bytes_pass = (2 if bf16 else 4) * nnz + 2 * 12 * n_free
    # the spmv phases time the product kernels of every iteration (event nodes right before
    # and after each launch); their fixed-order reductions (and a BF16 frame's residual
    # correction) are the "reduce" phase
    t_pass = (phase_mean["spmv1"] + phase_mean["spmv2"]) / (2 * n_iters)   # ms per launch
    t_pass_red = t_pass + phase_mean["reduce"] / (2 * n_iters)
    peak, peak_kind = measured_peaks()
    achieved = bytes_pass / (t_pass * 1e-3) / 1e9
    achieved_red = bytes_pass / (t_pass_red * 1e-3) / 1e9
    # ---- end to end through the public API with host buffers ----------------------------
    e2e = []
    sim.set_phase_marks(False)             # the production frame, as the value
    for _ in range(3):                     # warm-up of the host path (pinned staging, caches)
        sim.set_state(q0, v0)
        sim.step()
        sim.state()
    for _ in range(max(args.steps, 10)):
        t0 = time.perf_counter()
        sim.set_state(q0, v0)
        sim.step()
        qh, vh = sim.state()
        e2e.append(time.perf_counter() - t0)
    e2e_ms = 1e3 * statistics.mean(e2e) / n_iters
    h2d = 2 * sim.n_verts * 3 * 8
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not batch:
        ot = OracleTimer(scene, q0, v0, n_iters)
        ts = [ot.iteration_seconds() for _ in range(2)]
        cpu = {"value": round(ot.ms_per_iteration(statistics.mean(ts)), 3), "unit": UNIT,
               "cores": ot.cores, "kind": "oracle", "sample": ot.description(len(ts))}
    tun = sim.tuning()
    # the recorded DRAM traffic belongs to the register form of both products
    register_form = tun["pass1_unroll"] != 3 and tun["pass2_unroll"] != 3
    out = {
        "metric": METRIC,
        "value": round(mean_frame / n_iters, 5),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": max(3, args.warmup),
        "ms_per_step": round(mean_frame, 5),
        "higher_is_better": False,
        "scaling": "strong" if batch else "weak",
        "vs_baseline": None,
        "dtype": "bf16/f32" if bf16 else "f32",
        "data": "synthetic",
        "config": {
            "workload": (
                "stack: the stress case, 8 copies x 32 stiff boxes of 12^3 vertices (SNH, "
                "E=1e8, nu=0.45), 16 columns of 2 boxes per copy, each column a scene "
                "(128 scenes), mu=0.8 on a 20 deg incline and between the boxes, boxes "
                "pressed 1/20 lattice spacing into each other and the plane (box-box "
                "contacts: vertex against the other box's surface triangles), FP32, "
                "cold start, 10 L-G + 10 CR iterations per frame"
                if stack else
                "batch64: 64 cubes of 8^3..20^3 vertices (seeded), ARAP/co-rot vs SNH, E "
                "log-uniform 1e4..1e7, nu 0.3..0.48, planes tilted 0..30 deg, mu 0.1..0.8, "
                "each placed a quarter lattice spacing into its plane; one simulator, "
                "S~ in BF16 + FP32 correction, 5 L-G + 10 CR iterations per frame"
                if batch else
                f"star_pull: extruded 5-point star {args.n_side}x{args.n_side}x27 lattice, "
                f"{sim.n_verts} verts / {3 * sim.n_verts} DoFs / {sim.n_tets} tets, SNH E=1e6 "
                "nu=0.45, pinned cap pulled at "
                "0.5 m/s through 4x4 seeded cylinders mu=0.3, h=1/60, 5 L-G + 10 CR "
                "iterations per frame; every step replays one frame from the star placed "
                f"{100 * args.placement:.2f} cm into the first cylinder row "
                f"({round(statistics.mean(contacts))} contacts)"),
            "dofs": 3 * sim.n_verts,
            "scenes": n_batch if batch else 1,
            "scenes_this_rank": sim.n_scenes,
            "free_dofs": 3 * n_free,
            "tets": sim.n_tets,
            "contacts_mean": round(statistics.mean(contacts), 1),
            "placement_m": args.placement,
            "n_iters": n_iters,
            "nnz_S": nnz,
            "s_precision": args.s_precision,
            "products_launch": {k: v for k, v in sim.tuning().items()
                                if k in ("tuned", "pass1_ctas", "pass2_ctas", "pass1_unroll",
                                         "pass2_unroll", "pass1_balance", "pass2_balance")},
            "refine": args.refine if bf16 else None,
            "precompute_s": precompute,
            "l2": "flushed (256 MB write) before every timed step",
            "parallelism": (f"scene shards x{world} of one {n_batch}-scene batch" if batch
                            else f"replicas x{world}") if world > 1 else "single GPU",
        },
        "spread": spread,
        "phases_ms_per_frame": {k: round(v, 5) for k, v in phase_mean.items()},
        "instrumented_ms_per_step": round(instrumented_frame, 5),
        "wall_ms_per_step": round(1e3 * t_wall / args.steps, 4),
        "roofline": {
            "kernel": "S~ profile products k_pass1 + k_pass2 (mean over both, per launch)",
            "bound": "hbm",
            "achieved": round(achieved, 1),
            "peak": peak,
            "peak_source": peak_kind,
            "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "algorithmic_bytes_per_pass": bytes_pass,
            "achieved_with_reduction": round(achieved_red, 1),
            "traffic": (PRODUCT_TRAFFIC_BYTES.get((args.s_precision, args.n_side))
                        if not batch and register_form else None),
        },
        "e2e": {"value": round(e2e_ms, 4), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": h2d},
        "gpu_launches": stats["kernels_per_frame"] * 2 * args.steps,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    if rank == 0 and not batch and not args.no_variants:
        out["variants"] = variants_timing(scene, q0, v0, min(args.steps, 10), flush)
    if rank == 0 and not batch:
        # the cost of one phase boundary: a kernel per phase in a graph with programmatic
        # dependent launch (the frame graph) against a grid barrier in one cooperative
        # kernel (a persistent kernel per iteration), at one and two CTAs per SM
        from paper_2503_15078_b300 import measure_phase_boundaries
        lb = {}
        for cps in (1, 2):
            g_us, b_us = measure_phase_boundaries(n_phases=128, ctas_per_sm=cps, device=local)
            lb[f"{cps}_cta_per_sm"] = {"graph_pdl_us": round(g_us, 3),
                                       "grid_barrier_us": round(b_us, 3)}
        out["phase_boundary"] = lb
    if rank == 0 and not batch and not args.no_batch64:
        out["batch64"] = batch64_record(min(args.steps, 20), flush)
    if rank == 0 and not batch and not args.no_trajectory:
        out["pull_trajectory"] = pull_trajectory(args.n_side, 300, range(5),
                                                 min(args.steps, 20), flush)
    if rank == 0 and not batch and not args.no_warmstart:
        out["warmstart"] = warmstart_ab()
    if rank == 0:
        print(json.dumps(out), flush=True)
    sim.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_reference(args):
    """The FP64 oracle timed on the host cores, each step a bounded sample of the same
    workload (rank 0 only)."""
    import numpy as np
    import scenegen as sg
    rank, world, _ = dist_env()
    if rank != 0:
        return
    scene = sg.star_pull(n_side=args.n_side, seed=0)
    q, v = contact_state(scene, args.placement)
    ot = OracleTimer(scene, q, v, scene.n_iters, w_cols=30)
    for _ in range(max(1, args.warmup)):
        ot.iteration_seconds()
    vals = [ot.ms_per_iteration(ot.iteration_seconds()) for _ in range(max(1, args.steps))]
    desc, cores = ot.description(len(vals)), ot.cores
    value = statistics.mean(vals)
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT,
           "n_gpus": world, "steps": len(vals), "warmup": max(1, args.warmup),
           "higher_is_better": False, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"star_pull {3 * scene.n_verts} DoFs (FP64 CPU oracle, "
                                  "bounded sample)"},
           "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": cores,
                            "kind": "oracle", "sample": desc},
           "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
