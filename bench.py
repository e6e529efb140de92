#!/usr/bin/env python
"""Benchmark: TV-regularised cone-beam CT reconstruction (Algorithm A1 with the
coarse-to-fine multigrid schedule) on GB300.

One step = one full reconstruction of the cubic workload (default): a 256^3
volume at 1 mm, 40 views over 360 degrees on a 512x384 detector at 0.78 mm
(SAD 1000 mm, SDD 1500 mm), a seeded head-and-neck-like ellipsoid phantom with
Poisson noise at 5e4 photons per ray, 3 multigrid levels (64 -> 128 -> 256
per axis), 40/30/30 FBS iterations, step 1/L from 20 power iterations on the
coarsest level and 4 per finer level started from the prolongated
eigenvector of the previous level, lambda 0.05. --workload paper takes the
paper-scale 256x256x128 volume instead. The metric is seconds per
reconstruction (lower is better); with N GPUs every rank reconstructs its own
scan (weak scaling, no data-path collective) and the value is the job's time
per scan. The same line carries the projector and transpose against HBM and
a serving block (latency percentiles and throughput of a stream of mixed
scans), measured after the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on this machine's host cores: per
step, a bounded sample of per-operation costs, multiplied by the operation
counts of one reconstruction.
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

FP32_LANES_PER_SM = 128
METRIC = "recon sec at 256^3x40 views; projector/backproj GB/s vs HBM; serve p50/p99"
PAPER_METRIC = "recon sec at 256x256x128 x 40 views (paper-scale workload)"
WORKLOAD = ("paper-scale: 256x256x128 voxels @1 mm, 40 views/360 deg, 512x384 detector @0.78 mm, "
            "SAD 1000 / SDD 1500 mm, head-and-neck-like ellipsoid phantom, Poisson 5e4 photons/ray, "
            "3-level multigrid, 40/30/30 FBS iterations, tau = 1/L (20 power iterations per level), "
            "lambda 0.05, eps_tv 1e-5, Armijo c 0.01 alpha 0.6 tol 0.1%")
PAPER_CONTEXT = {"seconds": 130.3, "hardware": "NVIDIA Tesla C1060",
                 "workload": "NCAT 512x512x70, 40 views, 512x384 imager, 4-level multigrid",
                 "source": "Table 1"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--validate-model", action="store_true",
                    help="reference arm: time one full oracle reconstruction of the workload and compare it with "
                         "the sampled per-operation model on that run's own schedule")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--power-fine", type=int, default=4,
                    help="power iterations on each level after the first, warm-started from the "
                         "prolongated eigenvector of the previous level (0: 20 from ones everywhere)")
    ap.add_argument("--gradient", default="matched", choices=["matched", "eq6"],
                    help="Step 1 gradient: matched transpose P^T or the paper's closed form (Eq. 6)")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "fp16"],
                    help="storage type of the sinograms and of the projector's volume copy "
                         "(FP32 arithmetic throughout)")
    ap.add_argument("--workload", default="cube40", choices=["paper", "lowdose", "cube40", "small"],
                    help="cube40: 256^3, 40 views (default); paper: 256x256x128, 40 views; "
                         "lowdose: 256^3, 360 views, 1e4 photons")
    ap.add_argument("--schedule", default=None,
                    help="reference arm: JSON schedule (accepted ROF steps and reductions per iteration) to "
                         "scale the oracle's unit costs by; default: the oracle's own, oracle/schedule_<workload>.json")
    ap.add_argument("--prof-steps", type=int, default=1,
                    help="untimed steps after the timed region with per-launch CUDA events (per-kernel figures)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving block of the default line")
    ap.add_argument("--level", type=int, default=0,
                    help="one-iteration mode: multigrid level (0 = finest)")
    ap.add_argument("--mode", default="recon", choices=["recon", "one-iteration", "serve"],
                    help="one-iteration: each step is one FBS iteration on the finest grid with a "
                         "given step (per-kernel timing and profiler captures); serve: a stream of "
                         "mixed scans through the serving runtime (latency percentiles, throughput)")
    ap.add_argument("--serve-scans", type=int, default=None,
                    help="scans in the serving stream (serve mode: 64; the default line's serve block: 32)")
    ap.add_argument("--no-serve-reuse", action="store_true",
                    help="serve without reusing each geometry's power-iteration step sizes")
    ap.add_argument("--serve-concurrency", type=int, default=4,
                    help="reconstructions the server runs at once (compute streams)")
    ap.add_argument("--serve-loads", default=None,
                    help="arrival rates as fractions of the sequential capacity (serve mode: 0.5,0.8,1.0; "
                         "the default line's serve block: 0.8,1.0)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"cbct_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and parts[0] != self.uuid:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_units(wl):
    """Per-operation seconds of the FP64 oracle on every multigrid level of a
    workload, from a bounded sample: P over 4 views spread over the first
    quarter turn (views differ in cost: an oblique view's rays cross more of
    a square grid), as the mean per view; P^T over 2 and 4 of those views (a
    per-call part -- the private per-thread volumes and their fixed-order sum
    -- plus a per-view part); and the ROF solve's per-call part, its cost per
    accepted step (gradient, trial, update) and per further trial (one
    energy evaluation and update)."""
    import numpy as np
    from oracle import oracle as orc
    g = orc.Geometry.from_workload(wl)
    levels = len(wl.iters)
    rng = np.random.default_rng(0)
    tv = orc.TVParams(eps_tv=1e-5)
    out = []
    nv = g.n_views
    spread = sorted({int(round(k * nv / 16.0)) % nv for k in range(4)})
    for lev in range(levels):
        gl = g.coarse(2 ** (levels - 1 - lev)) if lev < levels - 1 else g

        def sub(idx):
            return orc.Geometry(gl.nx, gl.ny, gl.nz, gl.dx, gl.dy, gl.dz, gl.nu, gl.nv, gl.du, gl.dv, gl.sad,
                                gl.sdd, gl.angles[idx].copy(), gl.step_ratio)

        f = rng.random(gl.vol_shape) * 0.02
        s4, s2 = sub(spread), sub(spread[::2])
        t0 = time.perf_counter()
        p4 = orc.forward_project(s4, f)
        t_p = (time.perf_counter() - t0) / len(spread)
        p2 = orc.forward_project(s2, f)
        t0 = time.perf_counter()
        orc.back_project(s2, p2)
        t_b2 = time.perf_counter() - t0
        t0 = time.perf_counter()
        orc.back_project(s4, p4)
        t_b4 = time.perf_counter() - t0
        bt_view = max(t_b4 - t_b2, 0.0) / (len(spread) - len(spread[::2]))
        gaux = f + 0.001 * rng.standard_normal(gl.vol_shape)
        t0 = time.perf_counter()
        orc.rof_solve(gl, gaux, wl.lam, 1e-5, tv, replay=[0])
        t_r1 = time.perf_counter() - t0
        t0 = time.perf_counter()
        orc.rof_solve(gl, gaux, wl.lam, 1e-5, tv, replay=[0, 0])
        t_r2 = time.perf_counter() - t0
        t0 = time.perf_counter()
        orc.rof_energy(gl, f, gaux, wl.lam, 1e-5, 1e-5)
        t_e = time.perf_counter() - t0
        step = max(t_r2 - t_r1, 0.0)
        out.append({"level": lev, "views": gl.n_views, "p_view": t_p,
                    "pt_call": max(t_b2 - bt_view * len(spread[::2]), 0.0),
                    "pt_view": bt_view, "rof_call": max(t_r1 - step, 0.0), "rof_step": step, "rof_trial": t_e})
    return out


def oracle_model_seconds(units, schedule):
    """One oracle reconstruction from the unit costs and a schedule: per level,
    its power iterations (P and P^T each) and its FBS iterations (P, P^T and
    one ROF solve with that iteration's accepted steps and step reductions)."""
    total = 0.0
    for u, lev in zip(units, schedule["levels"]):
        pp = u["p_view"] * u["views"] + u["pt_call"] + u["pt_view"] * u["views"]
        total += lev["power"] * pp
        for it in lev["fbs"]:
            total += pp + u["rof_call"] + it["n_inner"] * u["rof_step"] + it["backtracks"] * u["rof_trial"]
    return total


def schedule_from_stats(st, wl, power_fine: int):
    """The reconstruction's own schedule (accepted steps and reductions of every
    ROF solve) from the library's statistics."""
    levels = [{"power": 20 if lev == 0 or power_fine <= 0 else power_fine, "fbs": []} for lev in range(len(wl.iters))]
    for k in range(int(st.n_iters)):
        it = st.iters[k]
        levels[int(it.level)]["fbs"].append({"n_inner": int(it.n_inner), "backtracks": int(it.backtracks)})
    return {"levels": levels, "source": "this run's reconstruction statistics"}


def schedule_from_oracle(name: str, power_fine: int):
    """The oracle's own schedule for the workload (oracle/make_schedule.py)."""
    path = os.path.join(ROOT, "oracle", f"schedule_{name}.json")
    with open(path) as fh:
        d = json.load(fh)
    levels = [{"power": d["power_iters"] if lev == 0 or power_fine <= 0 else power_fine, "fbs": lv["fbs"]}
              for lev, lv in enumerate(d["levels"])]
    return {"levels": levels, "source": f"oracle/schedule_{name}.json (the oracle's full reconstruction)"}


def oracle_sample(wl, schedule):
    """Seconds per oracle reconstruction: unit costs timed now, multiplied by
    the schedule's operation counts."""
    units = oracle_units(wl)
    desc = ("per level: P on 4 views spread over a quarter turn, P^T on 2 and 4 of them (per-call and per-view "
            "parts), ROF per-call, "
            "per-step and per-trial costs; times the schedule's counts from " + schedule["source"])
    return oracle_model_seconds(units, schedule), desc, units


def rank_noise_seed(base_seed: int, rank: int) -> int:
    """Noise seed of the scan a rank reconstructs: rank 0 keeps the workload's
    seed, every other rank draws its own noise (independent scans)."""
    return base_seed if rank == 0 else base_seed + 1000 * rank


def job_seconds_per_scan(local_ms: float, scans_per_rank: int, world: int, dist=None, device="cpu") -> float:
    """Whole-job time per scan: the slowest rank's wall time over all scans of
    all ranks (max over ranks of the local timed region)."""
    t = local_ms
    if dist is not None and world > 1:
        import torch
        v = torch.tensor([local_ms], dtype=torch.float64, device=device)
        dist.all_reduce(v, op=dist.ReduceOp.MAX)
        t = float(v.item())
    return t / 1e3 / (scans_per_rank * world)


def oracle_sample_warm(wl):
    """One untimed single-view projection on the finest grid (thread pool and
    first-touch warm-up before the timed oracle sample)."""
    import numpy as np
    from oracle import oracle as orc
    g = orc.Geometry.from_workload(wl)
    sub = orc.Geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.nu, g.nv, g.du, g.dv, g.sad, g.sdd,
                       g.angles[:1].copy(), g.step_ratio)
    orc.back_project(sub, orc.forward_project(sub, np.ones(g.vol_shape)))


def workload_description(args):
    """(workload text, metric name) of a run's configuration."""
    workload = WORKLOAD if args.power_fine <= 0 else WORKLOAD.replace(
        "tau = 1/L (20 power iterations per level)",
        f"tau = 1/L (20 power iterations on the coarsest level, {args.power_fine} per finer level "
        f"warm-started from the prolongated eigenvector)")
    if args.gradient == "eq6":
        workload += "; Step 1 gradient from the paper's closed form (Eq. 6) instead of the matched transpose"
    metric = PAPER_METRIC
    if args.workload == "lowdose":
        workload = workload.replace("paper-scale: 256x256x128 voxels", "low-dose: 256x256x256 voxels").replace(
            "40 views/360 deg", "360 views/360 deg").replace("Poisson 5e4", "Poisson 1e4")
        metric = "recon sec at 256^3 x 360 views (low-dose workload)"
    if args.workload == "cube40":
        workload = workload.replace("paper-scale: 256x256x128 voxels", "cubic: 256x256x256 voxels")
        metric = METRIC
    if args.storage != "f32":
        workload += (f"; measured sinogram, residual and the projector's volume copy stored as {args.storage} "
                     "(FP32 arithmetic, FP64 sums)")
    return workload, metric


def cpu_baseline_subprocess(args, schedule):
    """The oracle sample timed in a fresh process (this one holds a CUDA context
    and PyTorch's thread pools), exactly as the reference arm times it, with
    this run's schedule."""
    import tempfile
    env = {k: v for k, v in os.environ.items()
           if k not in ("RANK", "LOCAL_RANK", "WORLD_SIZE", "MASTER_ADDR", "MASTER_PORT")}
    with tempfile.NamedTemporaryFile("w", suffix=".json", delete=False) as fh:
        json.dump(schedule, fh)
        path = fh.name
    try:
        res = subprocess.run([sys.executable, os.path.abspath(__file__), "--impl", "reference", "--steps", "1",
                              "--warmup", "0", "--workload", args.workload, "--power-fine", str(args.power_fine),
                              "--schedule", path], capture_output=True, text=True, env=env, cwd=ROOT)
    finally:
        os.unlink(path)
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    if res.returncode != 0 or not lines:
        return {"value": None, "unit": "s", "cores": cpu_cores(), "kind": "oracle",
                "sample": "failed: " + (res.stderr.strip().splitlines() or ["no output"])[-1]}
    ref = json.loads(lines[-1])["cpu_baseline"]
    ref["sample"] += " (timed in a separate process)"
    return ref


def cpu_cores():
    try:
        return int(os.environ.get("OMP_NUM_THREADS") or os.cpu_count())
    except ValueError:
        return os.cpu_count()


def validate_model(args, wl):
    """One full oracle reconstruction, timed, beside the sampled model of the
    reference arm evaluated on that reconstruction's own schedule (accepted
    steps and reductions per ROF solve): the model's error on this machine."""
    from oracle import oracle as orc
    from paper_1001_0599_gb300 import synthetic
    _, y = synthetic.make_problem(wl)
    g = orc.Geometry.from_workload(wl)
    power_fine = args.power_fine if len(wl.iters) > 1 else 0
    oracle_sample_warm(wl)
    t0 = time.perf_counter()
    res = orc.reconstruct(g, y, wl.lam, wl.iters, orc.TVParams(eps_tv=1e-5), power_iters=20, clamp=True,
                          power_iters_fine=power_fine)
    full = time.perf_counter() - t0
    levels = [{"power": 20 if lev == 0 or power_fine <= 0 else power_fine, "fbs": []} for lev in range(len(wl.iters))]
    for it in res.iters:
        levels[it.level]["fbs"].append({"n_inner": int(it.n_inner), "backtracks": int(sum(it.steps))})
    schedule = {"levels": levels, "source": "the timed full run"}
    model, _, units = oracle_sample(wl, schedule)
    print(json.dumps({"workload": wl.name, "oracle_full_s": full, "model_s": model, "model_over_full": model / full,
                      "cores": cpu_cores(), "units": units}), flush=True)
    return 0


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from oracle import oracle as orc
    from paper_1001_0599_gb300 import synthetic
    orc.build()
    wl = synthetic.workload(args.workload)
    if args.validate_model:
        return validate_model(args, wl)
    if args.schedule:
        with open(args.schedule) as fh:
            schedule = json.load(fh)
    else:
        schedule = schedule_from_oracle(args.workload, args.power_fine)
    oracle_sample_warm(wl)
    times = []
    sample, units = "", None
    for i in range(args.warmup + args.steps):
        t, sample, units = oracle_sample(wl, schedule)
        if i >= args.warmup:
            times.append(t)
    v = statistics.mean(times)
    workload, metric = workload_description(args)
    line = {"impl": "reference", "metric": metric, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": run_config(workload), "parallelism": "host cores (OpenMP)",
            "cpu_baseline": {"value": v, "unit": "s", "cores": cpu_cores(), "kind": "oracle", "sample": sample,
                             "units": units},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_config(workload: str):
    """The run's configuration, the same for both arms."""
    return {"workload": workload, "l2": "flushed (512 MB write) before every timed step",
            "reductions": "FP64 across blocks, compensated FP32 within"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.mode == "serve":
        return serve_bench(args, rank, world, local)

    import numpy as np
    import torch

    from paper_1001_0599_gb300 import build as lib_build
    lib_build.build()
    from paper_1001_0599_gb300 import cbct, synthetic

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    wl = synthetic.workload(args.workload)
    truth, y = synthetic.make_problem(wl)
    if world > 1:  # each rank reconstructs its own scan (different noise draw)
        y = synthetic.poisson_log_sinogram(synthetic.exact_sinogram(synthetic.make_phantom(wl), wl),
                                           wl.photons, rank_noise_seed(wl.noise_seed, rank))
    g = cbct.geometry_from_workload(wl)
    tv = cbct.TvParams.paper(eps_tv=1e-5)
    if args.mode == "one-iteration":
        iters = (1,) + (0,) * args.level   # coarsest level listed first
        params = cbct.make_recon_params(wl.lam, iters, tv, taus=[1.28e-5] * (args.level + 1), clamp=True,
                                        gradient=args.gradient, storage=args.storage)
    else:
        params = cbct.make_recon_params(wl.lam, wl.iters, tv, power_iters=20, clamp=True,
                                        power_iters_fine=args.power_fine, gradient=args.gradient,
                                        storage=args.storage)
    ws = cbct.workspace(cbct.cbct_workspace_size(g, params))
    stats = cbct.stats_buffer()
    d_y = torch.from_numpy(y.astype(np.float32)).cuda()
    vol = torch.zeros(g.vol_shape, device="cuda")
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        cbct.cbct_reconstruct(g, d_y, vol, params, ws, stats)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        if not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    cbct.cbct_profile_reset()
    # the reconstruction's timed steps run without the per-launch profiling
    # events; its per-kernel figures come from separate steps afterwards
    profile_timed = args.mode == "one-iteration"
    cbct.cbct_profile_enable(profile_timed)
    n0 = cbct.cbct_launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    step_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        if profile_timed:
            cbct.cbct_profile_collect()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    launches = cbct.cbct_launch_count() - n0
    prof_steps = args.steps
    if not profile_timed:
        # per-kernel figures (roofline, bandwidth, breakdown): untimed steps with
        # CUDA events around every launch, L2 flushed as in the timed steps
        prof_steps = max(args.prof_steps, 1)
        cbct.cbct_profile_enable(True)
        for _ in range(prof_steps):
            flush.zero_()
            step()
            cbct.cbct_profile_collect()
        torch.cuda.synchronize()
    cbct.cbct_profile_enable(False)
    prof = cbct.cbct_profile_query()
    prof_levels = {lev: cbct.cbct_profile_query_level(lev) for lev in range(len(wl.iters))}
    sec_per_scan = job_seconds_per_scan(sum(step_ms), args.steps, world, dist, "cuda")
    total_ms = sec_per_scan * 1e3 * args.steps * world
    st = cbct.read_stats(stats)
    recon = vol.cpu().numpy().astype(np.float64)
    rel_err = float(np.linalg.norm(recon - truth) / np.linalg.norm(truth))
    corr = float(np.corrcoef(recon.ravel(), truth.ravel())[0, 1])
    storage_error = None
    if args.storage != "f32" and args.mode == "recon":
        # the same reconstruction with FP32 storage, untimed: the reduced
        # storage's effect on the result
        p32 = cbct.make_recon_params(wl.lam, wl.iters, tv, power_iters=20, clamp=True,
                                     power_iters_fine=args.power_fine, gradient=args.gradient)
        ws32 = cbct.workspace(cbct.cbct_workspace_size(g, p32))
        vol32 = torch.zeros(g.vol_shape, device="cuda")
        cbct.cbct_reconstruct(g, d_y, vol32, p32, ws32)
        r32 = vol32.cpu().numpy().astype(np.float64)
        storage_error = {"rel_l2_vs_f32_storage": float(np.linalg.norm(recon - r32) / np.linalg.norm(r32)),
                         "f32_rel_error_vs_phantom": float(np.linalg.norm(r32 - truth) / np.linalg.norm(truth))}
        del ws32, vol32

    # end to end through the host-buffer entry point (pinned buffers)
    e2e = None
    if not args.no_e2e:
        h_y = torch.from_numpy(y.astype(np.float32)).pin_memory()
        h_vol = torch.empty(g.vol_shape, dtype=torch.float32).pin_memory()
        ws_h = cbct.workspace(cbct.cbct_workspace_size_host(g, params))
        for _ in range(max(1, args.warmup)):
            cbct.cbct_reconstruct_host(g, h_y.numpy(), h_vol.numpy(), params, ws_h)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()
            cbct.cbct_reconstruct_host(g, h_y.numpy(), h_vol.numpy(), params, ws_h)
        e2e_per_scan = job_seconds_per_scan((time.perf_counter() - t0) * 1e3, args.steps, world, dist, "cuda")
        e2e = {"value": e2e_per_scan, "unit": "s",
               "h2d_bytes_per_step": int(h_y.numel() * 4), "d2h_bytes_per_step": int(h_vol.numel() * 4)}
        del ws_h

    if args.mode == "one-iteration":
        nnz0 = None
        try:
            with open(os.path.join(ROOT, "tests", "golden", "nnz.json")) as fh:
                nnz0 = float(json.load(fh)["paper"][str(args.level)])
        except (OSError, KeyError, ValueError):
            pass
        out = {"mode": "one-iteration", "level": args.level, "steps": args.steps, "ms_per_step": total_ms / args.steps,
               "clocks": clocks, "kernels": {}}
        for k, (n, ms) in prof.items():
            if not n:
                continue
            ent = {"launches": n, "avg_ms": ms / n}
            if nnz0 and k in ("forward_residual", "back_project_step"):
                ent["tflops"] = 2.0 * nnz0 / (ms / n / 1e3) / 1e12
                ent["samples_per_s"] = nnz0 / 8.0 / (ms / n / 1e3)
            out["kernels"][k] = ent
        if rank == 0:
            print(json.dumps(out), flush=True)
        return 0

    # roofline of the dominant kernel
    roof = roofline(prof, prof_levels, wl)
    bandwidth = projector_bandwidth(prof_levels, wl)
    if bandwidth is not None:
        add_gather_peak(bandwidth, wl)
    peaks = measured_peaks()
    workload, metric = workload_description(args)
    line = {"metric": metric, "value": sec_per_scan, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.storage == "f32" else f"f32 ({args.storage} storage)",
            "data": "synthetic",
            "config": run_config(workload),
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "clocks": clocks, "gpu_launches": int(launches), "roofline": roof,
            "projector_bandwidth": bandwidth,
            "tv_sweeps": tv_sweep_bandwidth(st, prof_levels, wl) if args.mode == "recon" else None,
            "e2e": e2e,
            "kernels": {k: {"launches": n // prof_steps, "ms_per_step": ms / prof_steps}
                        for k, (n, ms) in prof.items() if n},
            "kernels_note": f"from {prof_steps} untimed step(s) after the timed region with CUDA events around "
                            "every launch; the timed steps ran without them",
            "storage_error": storage_error,
            "quality": {"rel_error_vs_phantom": rel_err, "correlation": corr, "flags": int(st.flags),
                        "status": int(st.status), "taus": [float(st.tau[i]) for i in range(3)]},
            "paper_context": PAPER_CONTEXT,
            "peaks_source": peaks.get("_source")}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_subprocess(args, schedule_from_stats(st, wl, args.power_fine))
    if rank == 0 and world == 1 and not args.no_serve and args.storage == "f32":
        del ws, d_y, vol, flush
        torch.cuda.empty_cache()
        line["serve"] = serve_summary(serve_measure(args.serve_scans or 32,
                                                    parse_loads(args.serve_loads or "0.8,1.0"), "f32", local,
                                                    args.serve_concurrency, not args.no_serve_reuse))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def parse_loads(text: str):
    return [float(x) for x in text.split(",") if x]


# ---------------------------------------------------------------------------
# serving: a stream of mixed scans
# ---------------------------------------------------------------------------
SERVE_GRIDS = [(128, 128, 128, 2.0, 2.0, 2.0), (192, 192, 128, 4.0 / 3.0, 4.0 / 3.0, 1.0),
               (256, 256, 128, 1.0, 1.0, 1.0), (256, 256, 256, 1.0, 1.0, 1.0)]
SERVE_DETECTORS = [(512, 384, 0.78, 0.78), (256, 192, 1.56, 1.56)]
SERVE_VIEWS = [20, 40, 60, 90]
SERVE_ITERS = (20, 15, 15)


def serve_stream(n_scans: int, seed: int = 10):
    """The scan mix: grid, detector and view count drawn uniformly per scan."""
    import numpy as np
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(len(SERVE_GRIDS))), int(rng.integers(len(SERVE_DETECTORS))),
             int(rng.integers(len(SERVE_VIEWS)))) for _ in range(n_scans)]


def fifo_latencies(arrivals, service):
    """Latencies of a one-at-a-time FIFO server with the given service times."""
    t, out = 0.0, []
    for a, s in zip(arrivals, service):
        t = max(t, a) + s
        out.append(t - a)
    return out


def serve_bench(args, rank, world, local):
    """Serving benchmark (--mode serve; no counterpart in the paper): the full
    table of serve_measure on --serve-scans scans (default 64) at loads
    0.5, 0.8 and 1.0 of the sequential capacity."""
    res = serve_measure(args.serve_scans or 64, parse_loads(args.serve_loads or "0.5,0.8,1.0"), args.storage,
                        local, args.serve_concurrency, not args.no_serve_reuse)
    if rank == 0:
        print(json.dumps(res), flush=True)
    return 0


def serve_summary(res):
    """The serving figures the default line carries."""
    keep = ("p50_s", "p99_s", "scans_per_min", "sequential_p50_s", "sequential_p99_s")
    return {"metric": "scan latency p50/p99 (s) and scans/min of a mixed stream, beside the sequential plain "
                      "FP32 path on the same GPU",
            "scans": res["scans"], "loads": [{"load": r["load"], **{k: r[k] for k in keep}} for r in res["loads"]],
            "sequential_scans_per_min": res["sequential"]["scans_per_min"],
            "server_burst_scans_per_min": res["server_burst"]["scans_per_min"],
            "server_burst_without_step_reuse_scans_per_min": (res["server_burst_without_step_reuse"] or {}).get(
                "scans_per_min"),
            "reuse_steps": res["reuse_steps"],
            "bit_identical_to_sequential": res["bit_identical_to_sequential"], "concurrency": res["concurrency"],
            "workload": res["config"]["workload"], "clocks": res["clocks"]}


def warm_up_server(srv, scans, geoms, sparams, lanes, passes=1):
    """Submit `lanes` scans of every shape at once and wait for them, so the
    slots that scans of a shape occupy side by side exist and hold their
    captured graphs before anything is timed. With step reuse a second pass
    captures the graphs that run with the taus the first pass found."""
    import torch
    first = {key: next(s for s in scans if s[0] == key) for key in geoms}
    for _ in range(passes):
        for key, (wl, g) in geoms.items():
            tickets = [srv.submit(g, sparams, first[key][2],
                                  torch.empty(g.vol_shape, dtype=torch.float32).pin_memory())
                       for _ in range(lanes)]
            for t in tickets:
                srv.wait(t)


def serve_measure(n_scans, loads, storage, local, lanes=4, reuse_steps=True):
    """A stream of n_scans scans drawn from 4 grids x 2 detectors x 4 view
    counts, each reconstructed with 50 FBS-TV iterations (3-level multigrid
    20/15/15), arriving as a Poisson stream at the given fractions of the
    sequential capacity. The sequential system processes one scan at a time
    through cbct_reconstruct_host (copy in, reconstruct, copy out, wait); the
    server overlaps copies with compute and replays captured graphs, and (with
    reuse_steps) runs every shape's scans after its first with the taus that
    scan's power iterations found. Outputs are checked bit-identical between
    the two, so the RMS error is equal by construction."""
    import hashlib

    import numpy as np
    import torch

    from paper_1001_0599_gb300 import build as lib_build
    lib_build.build()
    from paper_1001_0599_gb300 import cbct, synthetic

    torch.cuda.set_device(local)
    stream = serve_stream(n_scans)
    tv = cbct.TvParams.paper(eps_tv=1e-5)
    params = cbct.make_recon_params(0.05, SERVE_ITERS, tv, power_iters=20, clamp=True, power_iters_fine=4)
    # the service may store sinograms and the projector's volume copy at reduced
    # precision; the sequential baseline is plain FP32 storage
    sparams = cbct.make_recon_params(0.05, SERVE_ITERS, tv, power_iters=20, clamp=True, power_iters_fine=4,
                                     storage=storage)
    geoms, truths, scans = {}, {}, []
    for i, (gi, di, vi) in enumerate(stream):
        nx, ny, nz, dx, dy, dz = SERVE_GRIDS[gi]
        nu, nv, du, dv = SERVE_DETECTORS[di]
        key = (gi, di, vi)
        if key not in geoms:
            wl = synthetic.Workload(f"serve{gi}{di}{vi}", nx, ny, nz, dx, dy, dz, nu, nv, du, dv, SERVE_VIEWS[vi],
                                    photons=5e4, phantom="head_neck", phantom_seed=3, noise_seed=10,
                                    lam=0.05, iters=SERVE_ITERS)
            geoms[key] = (wl, cbct.geometry_from_workload(wl))
        wl, g = geoms[key]
        if gi not in truths:
            truths[gi] = synthetic.voxelise(synthetic.make_phantom(wl), nx, ny, nz, dx, dy, dz).astype(np.float32)
        # measured line integrals: projector of the voxelised phantom, Poisson counts
        p = torch.empty(g.sino_shape, device="cuda")
        cbct.cbct_forward_project(g, torch.from_numpy(truths[gi]).cuda(), p)
        gen = torch.Generator(device="cuda").manual_seed(10_000 + i)
        counts = torch.poisson(wl.photons * torch.exp(-p), generator=gen)
        y = torch.log(wl.photons / counts.clamp_min(1.0)).float()
        scans.append((key, g, y.cpu().contiguous().pin_memory(), gi))
    torch.cuda.synchronize()

    # sequential plain FP32: one scan at a time through the host-buffer entry point
    ws = {key: cbct.workspace(cbct.cbct_workspace_size_host(g, params)) for key, (wl, g) in geoms.items()}
    h_out = torch.empty(max(int(np.prod(g.vol_shape)) for _, g in geoms.values()), dtype=torch.float32).pin_memory()
    for key, (wl, g) in geoms.items():   # warm-up: one scan per shape
        first = next(s for s in scans if s[0] == key)
        cbct.cbct_reconstruct_host(g, first[2].numpy(), h_out[:int(np.prod(g.vol_shape))].numpy(), params, ws[key])
    service, digests, rms = [], [], []
    t_all = time.perf_counter()
    for key, g, y, gi in scans:
        n = int(np.prod(g.vol_shape))
        t0 = time.perf_counter()
        cbct.cbct_reconstruct_host(g, y.numpy(), h_out[:n].numpy(), params, ws[key])
        service.append(time.perf_counter() - t0)
        out = h_out[:n].numpy()
        digests.append(hashlib.sha1(out.tobytes()).hexdigest())
        rms.append(float(np.sqrt(np.mean((out.reshape(g.vol_shape) - truths[gi]) ** 2))))
    seq_total = time.perf_counter() - t_all
    del ws
    torch.cuda.empty_cache()
    capacity = len(scans) / sum(service)     # scans per second, one at a time

    results = []
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    passes = 2 if reuse_steps else 1
    srv = cbct.Server(use_graphs=True, concurrency=lanes, reuse_steps=reuse_steps)
    outs = [torch.empty(g.vol_shape, dtype=torch.float32).pin_memory() for _, g, _, _ in scans]
    # warm-up: `lanes` scans per shape at once capture the graphs of the slots
    # that scans of that shape occupy side by side
    warm_up_server(srv, scans, geoms, sparams, lanes, passes)
    identical = True
    sampler.start()
    for load in loads:
        rate = load * capacity
        arr = np.cumsum(np.random.default_rng(10).exponential(1.0 / rate, len(scans)))
        arr -= arr[0]
        tickets = []
        t0 = time.perf_counter()
        for (key, g, y, gi), a, o in zip(scans, arr, outs):
            delay = t0 + a - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(g, sparams, y, o))
        res = [srv.wait(t) for t in tickets]
        lat = [r.t_done - r.t_submit for r in res]
        span = max(r.t_done for r in res) - min(r.t_submit for r in res)
        for o, dgst in zip(outs, digests):
            identical &= hashlib.sha1(o.numpy().tobytes()).hexdigest() == dgst
        seq_lat = fifo_latencies(list(arr), service)
        results.append({"load": load, "arrivals_per_s": rate,
                        "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                        "scans_per_min": 60.0 * len(scans) / span,
                        "sequential_p50_s": float(np.percentile(seq_lat, 50)),
                        "sequential_p99_s": float(np.percentile(seq_lat, 99)),
                        "gpu_s_per_scan": float(np.mean([r.gpu_ms for r in res]) / 1e3),
                        "graph_replays": int(sum(r.graph_replay for r in res))})
    clocks = sampler.stop()
    info = srv.query()
    srv.close()
    # back-to-back stream (all scans submitted at once): the throughput ceiling,
    # with and without step reuse
    bursts = {}
    for reuse in ([True, False] if reuse_steps else [False]):
        srv = cbct.Server(use_graphs=True, concurrency=lanes, reuse_steps=reuse)
        warm_up_server(srv, scans, geoms, sparams, lanes, 2 if reuse else 1)
        t0 = time.perf_counter()
        tickets = [srv.submit(g, sparams, y, o) for (key, g, y, gi), o in zip(scans, outs)]
        res = [srv.wait(t) for t in tickets]
        bursts[reuse] = time.perf_counter() - t0
        srv.close()
        for o, dgst in zip(outs, digests):
            identical &= hashlib.sha1(o.numpy().tobytes()).hexdigest() == dgst
    burst = bursts[reuse_steps]
    rms_srv = [float(np.sqrt(np.mean((o.numpy().reshape(g.vol_shape) - truths[gi]) ** 2)))
               for (key, g, y, gi), o in zip(scans, outs)]
    line = {"metric": "serving: scan latency p50/p99 (s) and scans/min, mixed 64-scan stream",
            "mode": "serve", "value": results[-1]["p99_s"] if results else None, "unit": "s (p99 at the highest load)",
            "higher_is_better": False, "n_gpus": 1,
            "dtype": "f32" if storage == "f32" else f"f32 ({storage} storage)", "data": "synthetic",
            "config": {"workload": f"{len(scans)} scans; grids {SERVE_GRIDS}; detectors {SERVE_DETECTORS}; "
                                   f"views {SERVE_VIEWS}; 50 FBS-TV iterations (multigrid 20/15/15), "
                                   "lambda 0.05, Poisson 5e4 photons; stream seed 10",
                       "arrivals": "Poisson at the listed fractions of the sequential capacity"},
            "sequential": {"scans_per_min": 60.0 * capacity, "total_s": seq_total,
                           "mean_service_s": float(np.mean(service))},
            "server_burst": {"scans_per_min": 60.0 * len(scans) / burst, "total_s": burst},
            "server_burst_without_step_reuse": ({"scans_per_min": 60.0 * len(scans) / bursts[False],
                                                 "total_s": bursts[False]} if reuse_steps else None),
            "reuse_steps": bool(reuse_steps),
            "loads": results, "storage": storage, "scans": len(scans), "concurrency": lanes,
            "bit_identical_to_sequential": bool(identical) if storage == "f32" else None,
            "rms_error_vs_phantom": {"sequential_f32": float(np.mean(rms)), "server": float(np.mean(rms_srv)),
                                     "max_rel_diff_per_scan": float(max(abs(a - b) / b for a, b in
                                                                        zip(rms_srv, rms)))},
            "server": {"slots": int(info.slots), "graphs_captured": int(info.graphs_captured),
                       "graph_failures": int(info.graph_failures), "evictions": int(info.evictions),
                       "step_reuses": int(info.step_reuses),
                       "peak_arena_gb": info.peak_bytes_in_use / 1e9, "arena_gb": info.arena_bytes / 1e9},
            "clocks": clocks}
    return line


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        d["_source"] = "measured (MEASURED_PEAKS.json)"
        return d
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "_source": "fallback"}


KERNEL_SOURCES = {"back_project_step": ["bp.cu", "bps.cu", "bp_common.cuh"],
                  "back_project": ["bp.cu", "bps.cu", "bp_common.cuh"],
                  "forward_residual": ["fp.cu"], "forward_project": ["fp.cu"]}


def sources_sha1(names):
    import hashlib
    h = hashlib.sha1()
    for n in names + ["cbct_internal.cuh"]:
        with open(os.path.join(ROOT, "paper_1001_0599_gb300", "csrc", n), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(kernel, workload, level):
    """DRAM bytes per launch from the committed ncu capture (profiles/traffic.json),
    or None when there is none or the kernel's sources changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            ent = json.load(fh)[f"{kernel}/{workload}/L{level}"]
    except (OSError, KeyError, ValueError):
        return None
    if ent.get("sources_sha1") != sources_sha1(KERNEL_SOURCES.get(kernel, [])):
        return None
    return float(ent["dram_bytes_per_launch"])


def projector_bandwidth(prof_levels, wl):
    """Projector and transpose at the finest level against HBM: algorithmic
    bytes per call (forward + residual: f, y read, r written; transpose step:
    r, f read, g written) over the measured call time, as a fraction of the
    measured copy bandwidth; DRAM bytes from the ncu capture over the same
    time; and gathered bytes, 32 B (8 FP32 corner values) per trilinear sample,
    nnz / 8 samples per call."""
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    try:
        with open(os.path.join(ROOT, "tests", "golden", "nnz.json")) as fh:
            nnz0 = float(json.load(fh)[wl.name]["0"])
    except (OSError, KeyError, ValueError):
        return None
    nvox = wl.nx * wl.ny * wl.nz
    nray = wl.n_views * wl.nv * wl.nu
    out = {}
    for name, algo in (("forward_residual", 4 * (nvox + 2 * nray)), ("back_project_step", 4 * (nray + 2 * nvox))):
        n, ms = prof_levels.get(0, {}).get(name, (0, 0.0))
        if not n:
            continue
        t = ms / n / 1e3
        traffic = measured_traffic(name, wl.name, 0)
        out[name] = {"algorithmic_bytes": algo, "algorithmic_gbs": algo / t / 1e9, "hbm_peak_gbs": hbm,
                     "frac_of_hbm": algo / t / 1e9 / hbm,
                     "dram_gbs": (traffic / t / 1e9) if traffic else None,
                     "gathered_gbs": 32.0 * nnz0 / 8.0 / t / 1e9, "samples_per_s": nnz0 / 8.0 / t,
                     "avg_ms": t * 1e3}
    out["note"] = ("not HBM-bound: the per-call working set sits in L2 and both kernels are bound by "
                   "instruction issue; see roofline")
    return out


def tv_sweep_bandwidth(st, prof_levels, wl):
    """The ROF solves against HBM, per multigrid level: algorithmic bytes of
    a solve from its own step counts (every accepted step: a gradient sweep
    reading f and g and writing d, 12 B/voxel; its first trial and every
    reduction, reading f, d and g, 12 B/voxel; the update reading f and d and
    writing f, 12 B/voxel), over the solves' time measured by CUDA events."""
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    n_levels = len(wl.iters)
    sweeps = [0.0] * n_levels
    solves = [0] * n_levels
    for k in range(int(st.n_iters)):
        it = st.iters[k]
        gl = n_levels - 1 - int(it.level)   # geometry level, 0 = finest
        sweeps[gl] += 3 * int(it.n_inner) + int(it.backtracks)
        solves[gl] += 1
    out = {}
    for gl in range(n_levels):
        n, ms = prof_levels.get(gl, {}).get("rof_persistent", (0, 0.0))
        if not n or ms <= 0 or not solves[gl]:
            continue
        ms = ms / n * solves[gl]   # one reconstruction's solves on this level
        f = 2 ** gl
        nvox = (wl.nx // f) * (wl.ny // f) * (wl.nz // f)
        algo = 12.0 * nvox * sweeps[gl]
        out[str(gl)] = {"solves": solves[gl], "sweeps": int(sweeps[gl]), "algorithmic_bytes": algo,
                        "ms": ms, "algorithmic_gbs": algo / (ms / 1e3) / 1e9,
                        "frac_of_hbm": algo / (ms / 1e3) / 1e9 / hbm}
    return {"levels": out, "hbm_peak_gbs": hbm,
            "work": "12 B per voxel per sweep (gradient, trial, update), sweeps from this run's step counts"}


def gather_peak(wl, repeats: int = 5):
    """Peak trilinear gather rate on this GPU: the library's gather
    microbenchmark (cbct_gather_bench: warps walking ray lines, 32 lanes on
    32 neighbouring detector rows, 8 read-only loads per lane and sample) over
    an L2-resident volume of the workload's finest grid, timed with CUDA
    events on the launching stream after 3 warm-up launches; the best of
    ``repeats`` launches."""
    import torch
    from paper_1001_0599_gb300 import cbct
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    n_lines, n_samples = sms * 256, 256
    vol = torch.rand((wl.nx, wl.ny, wl.nz), device="cuda")
    out = torch.empty(n_lines * 32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(3):
        cbct.cbct_gather_bench(vol, n_lines, n_samples, out)
    best = float("inf")
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cbct.cbct_gather_bench(vol, n_lines, n_samples, out)
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    samples = n_lines * 32 * n_samples
    return {"samples_per_s": samples / best, "gbs": 32.0 * samples / best / 1e9, "ms": best * 1e3,
            "volume": [wl.nx, wl.ny, wl.nz],
            "how": (f"cbct_gather_bench: {n_lines} warps x 32 lanes x {n_samples} trilinear samples (8 read-only "
                    "loads each) from an L2-resident volume, best of 5 launches by CUDA events")}


def add_gather_peak(bandwidth, wl):
    """Gathered bytes of the projector pair as a fraction of the measured
    gather peak (the third roofline of the pair, beside HBM and FP32 issue)."""
    peak = gather_peak(wl)
    bandwidth["gather_peak"] = peak
    for name in ("forward_residual", "back_project_step"):
        if name in bandwidth:
            bandwidth[name]["frac_of_gather_peak"] = bandwidth[name]["samples_per_s"] / peak["samples_per_s"]


def roofline(prof, prof_levels, wl):
    """Dominant kernel by device time, reported for its finest-level launches
    (the bulk of its time). Projector kernels are bound by FP32 issue (no dense
    contraction, working set in L2): algorithmic work is 2 flops per non-zero
    weight of P, nnz per level from tests/golden/nnz.json; peak = SMs x 128
    FP32 lanes x 2 flops x max SM clock."""
    import torch
    name, (n, ms) = max(prof.items(), key=lambda kv: kv[1][1])
    if n == 0 or ms <= 0:
        return None
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count \
        if torch.cuda.is_available() else 152
    peaks = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    try:
        with open(os.path.join(ROOT, "tests", "golden", "nnz.json")) as fh:
            nnz = json.load(fh)[wl.name]
    except (OSError, KeyError, ValueError):
        nnz = None
    if name in KERNEL_SOURCES and nnz:
        levels = {}
        for lev, pl in prof_levels.items():
            nl, msl = pl.get(name, (0, 0.0))
            if nl and msl > 0 and str(lev) in nnz:
                avg = msl / nl
                levels[lev] = {"launches": nl, "avg_ms": avg,
                               "tflops": 2.0 * float(nnz[str(lev)]) / (avg / 1e3) / 1e12}
        if 0 not in levels:
            return None
        l0 = levels[0]
        return {"kernel": name, "level": 0, "bound": "alu", "achieved": l0["tflops"], "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": l0["tflops"] / fp32_peak,
                "traffic": measured_traffic(name, wl.name, 0),
                "work": "2 flops per non-zero sample-voxel weight of P at the finest level "
                        "(nnz from the oracle's count), per launch",
                "peak_source": "derived: SMs x 128 FP32 lanes x 2 x max SM clock (MEASURED_PEAKS.json)",
                "avg_launch_ms": l0["avg_ms"], "levels": levels}
    # TV sweeps: HBM-bound (report time only; bytes depend on the sweep count)
    return {"kernel": name, "bound": "hbm", "achieved": None, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
            "frac": None, "traffic": None, "avg_launch_ms": ms / n}


if __name__ == "__main__":
    sys.exit(main())
