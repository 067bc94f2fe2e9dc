"""Benchmark: Anderson-accelerated FWI on the batched workload (400 x 150 grid,
dx 20 m, 12 dipping layers cut by 2 normal faults, 32 shots with 60-400
receivers, Ricker 8 Hz, dt 1.5 ms, 2500 steps, AA(10)).

One step = one iteration of Alg. 2 on the GPU: the adjoint sweep with the
imaging condition (reusing the forward wavefield of the accepted trial), the
shot sum, the AA(10) step (FP64 Gram / solve), the line-search trial forward
sweep(s) with receiver gather and misfit, and the combine.  Metric: grid-point
updates per second, counting every forward and adjoint pass the step ran
(sum_s nt_s * NZ * NX per pass).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the checker of this library) on
the host cores, on a bounded sample of the same workload.  Under torchrun
(N > 1) every rank runs an independent replica (the path has no exchange step
on one problem: replicas only) and rank 0 prints the line.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "fwi-batched-400x150-32shots-2500steps-aa10"
METRIC = "grid-pt updates/s (fwd+adj)"
UNIT = "grid-pt updates/s"
# Algorithmic bytes per grid-point update (FP32 fields):
#   forward  k_fwd: read u^n, u^{n-1}, W; write u^{n+1}                       = 16 B
#   adjoint  k_adj: read z^{n+1}, z^{n+2}, W, u^n; write z^n; img read+write  = 28 B
BYTES_FWD = 16
BYTES_ADJ = 28


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_time_ms(ms_local, ws, device):
    """Whole-job time of N independent replicas: the maximum over ranks of the
    per-rank timed region (all-reduce MAX; no data-path collective)."""
    if ws <= 1:
        return ms_local
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(updates_per_rank, ws, ms_job):
    """Weak scaling: every rank processes the same workload, so the job's
    throughput is ws x the per-rank updates over the slowest rank's time."""
    return ws * updates_per_rank / (ms_job / 1e3)


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                               f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash():
    """Hash of the sources the wave-equation kernels are built from."""
    h = hashlib.sha256()
    for name in ("internal.cuh", "stencil_math.cuh", "wave_kernels.cu", "persist_kernels.cu"):
        with open(os.path.join(ROOT, "paper_2008_11778_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_record(kernel, shots_per_launch=None):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or
    None if absent or taken on a different kernel source.  Per-step kernels'
    records hold one launch of `shots_per_launch` shots; the bytes scale with
    the shots of the benchmark's launches (a lane of the batch)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    rec = d.get(kernel)
    if not rec or rec.get("source_hash") != kernel_source_hash():
        return None
    b = rec.get("bytes_per_launch_full")
    if b is not None and shots_per_launch and rec.get("shots_per_launch"):
        b = b * shots_per_launch / rec["shots_per_launch"]
    return b


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on the host cores
# ---------------------------------------------------------------------------

def oracle_sample(prob, shots, reps=1):
    """Time the oracle's FWI gradient (forward + adjoint) on `shots` shots at
    full record length; returns (updates/s, seconds, cores, sample text)."""
    import oracle
    g = prob.geom.subset(shots)
    d_obs = oracle.forward(g, prob.m_true)
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.fwi_gradient(g, prob.m_start, d_obs)
    dt = time.perf_counter() - t0
    upd = 2 * g.updates_per_pass() * reps
    return upd / dt, dt, oracle.num_threads(), "%d of %d shots at full nt=%d, %d gradient(s)" % (
        len(shots), prob.geom.S, int(g.nt.max()), reps)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2008_11778_gb300 import synth
    prob = synth.batched()
    import oracle
    cores = oracle.num_threads()
    nsh = min(prob.geom.S, max(1, cores))
    shots = list(range(nsh))
    times = []
    upd = 2 * prob.geom.subset(shots).updates_per_pass()
    for i in range(args.warmup + args.steps):
        v, dt, cores, sample = oracle_sample(prob, shots)
        if i >= args.warmup:
            times.append(dt)
    ms = 1e3 * float(np.mean(times))
    value = upd / (ms / 1e3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": sample, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample + " per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def active_points(geom, n):
    return int((geom.nt > n).sum()) * geom.NZ * geom.NX


ENGINES = {"auto": 0, "per_step": 1, "persistent": 2, "hybrid": 3}
ENGINE_NAMES = {v: k for k, v in ENGINES.items()}


def make_plan(aafwi, prob, g, m_tune, args):
    """The benchmark's plan: the library's autotuned launch configuration
    (timed on short sweeps of this geometry before the timed region), or the
    engine / tile height given on the command line."""
    kw = dict(pdl=not args.no_pdl, steps_per_launch=args.steps_per_launch, lanes=args.lanes)
    if args.engine == "tuned":
        return aafwi.Plan(g, c_max=prob.c_bounds[1], tune_model=m_tune, tune_cache=args.tune_cache, **kw)
    return aafwi.Plan(g, c_max=prob.c_bounds[1], engine=ENGINES[args.engine], tile_z=args.tile_z, **kw)


def run_ours(args):
    import torch
    from paper_2008_11778_gb300 import aafwi, solve, synth
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prob = synth.batched()
    g = prob.geom
    lo, hi = prob.m_bounds
    m_start = torch.as_tensor(prob.m_start.astype(np.float32), device=dev)
    plan = make_plan(aafwi, prob, g, m_start, args)
    tuning = getattr(plan, "tuning", None)
    # observed data from this library's own forward on the true model
    m_true = torch.as_tensor(prob.m_true.astype(np.float32), device=dev)
    d_obs = torch.empty(plan.trace_count, device=dev)
    plan.model_forward(m_true, d_obs)
    m0 = torch.as_tensor(prob.m_start.astype(np.float32), device=dev)
    run = solve.AAInversion(plan, d_obs, m0, M=prob.M, bounds=(lo, hi))
    upd_pass = g.updates_per_pass()
    # warm-up: the first iterations (input step and short histories)
    for _ in range(args.warmup):
        run.step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    nf0, na0 = run.n_forward, run.n_adjoint
    l0 = aafwi.launch_count()
    # per-step events around the gradient (adjoint sweep) and the rest
    evs = []
    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e_start.record(stream)
    t0 = time.perf_counter()
    adj_ms, fwd_ms = [], []
    for _ in range(args.steps):
        # Alg. 2 iteration, instrumented: time the pieces on the launching stream
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nf_before = run.n_forward
        a0.record(stream)
        run.step()
        a1.record(stream)
        evs.append((a0, a1, run.n_forward - nf_before))
    e_end.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = aafwi.launch_count() - l0
    clk = clocks.stop()
    ms_total = job_time_ms(e_start.elapsed_time(e_end), ws, dev)
    nf, na = run.n_forward - nf0, run.n_adjoint - na0
    upd = (nf + na) * upd_pass
    value = job_value(upd, ws, ms_total)

    # dominant kernel: the adjoint sweep timed alone (reusing a stored forward)
    kt = time_sweeps(plan, run, dev, args.kernel_reps)
    peak, peak_kind = read_peaks()
    nt = int(g.nt.max())
    pts_sweep = sum(active_points(g, n) for n in range(nt))
    eng = plan.info.engine
    spl = plan.info.steps_per_launch
    adj_per_sweep = 1 if eng in (aafwi.ENGINE_PERSISTENT, aafwi.ENGINE_HYBRID) else nt * plan.info.lanes
    lanes = plan.info.lanes
    # per-step sweeps: nt (or nt/2) launches per lane; lanes run concurrently,
    # so a launch's duration is the sweep's event time over all its launches
    fwd_per_sweep = 1 if eng == aafwi.ENGINE_PERSISTENT else lanes * ((nt + 1) // 2 if spl == 2 else nt)
    adj_name = "k_adj_persist" if adj_per_sweep == 1 else "k_adj"
    fwd_name = "k_fwd_persist" if fwd_per_sweep == 1 else "k_fwd2" if spl == 2 else "k_fwd"
    # the kernel with the larger share of the timed steps is the dominant one
    t_fwd, t_adj = nf * kt["fwd_ms"], na * kt["adj_ms"]

    def kernel_roof(name, what, bpu, per_sweep, sweep_ms, share):
        b = bpu * pts_sweep / per_sweep
        ms = sweep_ms / per_sweep
        gbs = b / (ms * 1e-3) / 1e9
        launch_shots = g.S / lanes if per_sweep > 1 else None
        return {"bound": "hbm", "kernel": name + " (" + what + ")", "achieved": gbs, "peak": peak,
                "unit": "GB/s", "frac": gbs / peak, "peak_kind": peak_kind,
                "traffic": traffic_record(name, launch_shots),
                "bytes_per_launch": b, "ms_per_launch": ms, "launches_per_sweep": per_sweep,
                "us_per_time_step": 1e3 * sweep_ms / nt, "share_of_step": share}

    fwd_roof = kernel_roof(fwd_name, "forward sweep, %d step(s) per launch" % (2 if spl == 2 else 1),
                           BYTES_FWD, fwd_per_sweep, kt["fwd_ms"], t_fwd / ms_total)
    adj_roof = kernel_roof(adj_name, "adjoint sweep + imaging", BYTES_ADJ, adj_per_sweep, kt["adj_ms"],
                           t_adj / ms_total)
    if t_fwd >= t_adj:
        roofline = dict(fwd_roof, other_kernel=adj_roof)
    else:
        roofline = dict(adj_roof, other_kernel=fwd_roof)

    e2e = run_e2e(plan, prob, dev, args.e2e_steps) if args.e2e_steps > 0 else None
    learned_cmp = None
    if args.learned_eval > 0:
        plan.close()
        learned_cmp = learned_vs_plain(args.learned_eval, args.learned_target, args.learned_max_iters)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(prob)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "grid": [g.nz, g.nx], "padded": [g.NZ, g.NX],
                           "shots": g.S, "nt": int(g.nt.max()), "M": prob.M,
                           "checkpoint_every": plan.info.checkpoint_every,
                           "engine": ENGINE_NAMES.get(plan.info.engine, plan.info.engine),
                           "tile_z": plan.info.tile_z, "pdl": not args.no_pdl,
                           "steps_per_launch": plan.info.steps_per_launch, "lanes": plan.info.lanes,
                           "autotune": None if tuning is None else {
                               "steps": tuning.get("steps"), "cached": tuning.get("cached"),
                               "lanes": tuning.get("lanes"),
                               "table_ms": [[ENGINE_NAMES.get(r[0], r[0])] + list(r[1:]) for r in tuning["table"]]},
                           "l2": "inputs larger than L2 (wavefield history %.1f GB)" % (
                               plan.info.workspace_bytes / 1e9),
                           "passes": {"forward": nf, "adjoint": na},
                           "fwi_iterations_per_s": args.steps / (ms_total / 1e3),
                           "J_over_J0": run.J / run.J0},
                "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "learned_vs_plain": learned_cmp,
                "clocks": clk, "host_wall_s": wall}
        print(json.dumps(line), flush=True)
    run.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def time_sweeps(plan, run, dev, reps):
    """CUDA-event time of the forward sweep (model_forward) and of the adjoint
    sweep (adjoint_gradient reusing it: adjoint, misfit and shot sum) on the
    launching stream; per-step engines include the gaps between launches."""
    import torch
    stream = torch.cuda.current_stream()
    nt = int(plan.geom.nt.max())
    grad = torch.empty_like(run.p)
    m = run.p
    f_ms, a_ms = [], []
    for _ in range(reps):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        plan.model_forward(m)
        e1.record(stream)
        plan.adjoint_gradient(0, m, None, run.d_obs, grad, sync=False, reuse_forward=True)
        e2.record(stream)
        torch.cuda.synchronize()
        f_ms.append(e0.elapsed_time(e1))
        a_ms.append(e1.elapsed_time(e2))
    return {"fwd_ms": statistics.median(f_ms), "adj_ms": statistics.median(a_ms)}


def run_e2e(plan, prob, dev, steps):
    """The FWI gradient through the C-ABI call with host buffers
    (aafwi_adjoint_gradient_host): each step copies m and d_obs from pinned
    host memory into the plan's device staging, runs forward + adjoint, and
    copies the gradient and J back, all inside the one call."""
    import torch
    g = prob.geom
    m_h = torch.as_tensor(prob.m_start.astype(np.float32)).pin_memory()
    d_dev = torch.empty(plan.trace_count, device=dev)
    plan.model_forward(torch.as_tensor(prob.m_true.astype(np.float32), device=dev), d_dev)
    d_h = d_dev.cpu().pin_memory()
    g_h = torch.empty_like(m_h).pin_memory()
    stream = torch.cuda.current_stream()

    def one():
        return plan.adjoint_gradient_host(0, m_h, None, d_h, g_h)   # synchronises

    one()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        one()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    upd = 2 * g.updates_per_pass()
    h2d = m_h.numel() * 4 + d_h.numel() * 4
    d2h = g_h.numel() * 4 + 8
    return {"value": upd / (ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": ms, "call": "aafwi_adjoint_gradient_host (FWI): host m and d_obs in, host gradient and J out"}


def learned_vs_plain(n_eval, target, max_iters):
    """Second half of the metric: wall seconds (same GPU) for plain AA(10) and
    for AA(10) with the trained learned preconditioner to reach J/J0 <= target
    on held-out 400 x 150 models (16 shots, 2500 steps)."""
    from paper_2008_11778_gb300 import learned
    params, meta = learned.load_weights()
    rows = learned.compare(params, n_eval, target, max_iters, log=lambda *a: None)
    sp = [r["plain"]["seconds"] / r["learned"]["seconds"] for r in rows]
    return {"metric": "wall-s to J/J0 <= %g, learned vs plain AA(10)" % target, "target": target,
            "max_iters": max_iters, "models": len(rows),
            "plain_s": [r["plain"]["seconds"] for r in rows],
            "learned_s": [r["learned"]["seconds"] for r in rows],
            "plain_reached": [bool(r["plain"]["reached"]) for r in rows],
            "learned_reached": [bool(r["learned"]["reached"]) for r in rows],
            "plain_iters": [r["plain"]["iterations"] for r in rows],
            "learned_iters": [r["learned"]["iterations"] for r in rows],
            "median_speedup": float(np.median(sp)),
            "training": {k: float(v) for k, v in meta.items()}}


def cpu_baseline(prob):
    import oracle
    cores = oracle.num_threads()
    nsh = min(prob.geom.S, max(1, cores))
    v, dt, cores, sample = oracle_sample(prob, list(range(nsh)))
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "seconds": dt}


def ncu_case(args):
    """A small case of the benchmark's kernels for ncu --set full captures: the
    batched geometry (all 32 shots, 400 x 150) cut to 64 time steps; one
    forward sweep and one adjoint sweep reusing it, with the engine and tile
    height given on the command line (the benchmark line's config)."""
    import torch
    from paper_2008_11778_gb300 import aafwi, synth
    prob = synth.batched()
    g = prob.geom.with_nt(64)
    plan = aafwi.Plan(g, c_max=prob.c_bounds[1], engine=ENGINES.get(args.engine, 0), tile_z=args.tile_z,
                      pdl=not args.no_pdl, steps_per_launch=args.steps_per_launch, lanes=args.lanes)
    m = torch.as_tensor(prob.m_start.astype(np.float32), device="cuda")
    d_obs = torch.zeros(plan.trace_count, device="cuda")
    grad = torch.empty_like(m)
    plan.model_forward(m)
    J = plan.adjoint_gradient(aafwi.MODE_FWI, m, None, d_obs, grad, reuse_forward=True)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": "batched-400x150-32shots-64steps", "J": J,
                      "engine": ENGINE_NAMES.get(plan.info.engine), "tile_z": plan.info.tile_z,
                      "steps_per_launch": plan.info.steps_per_launch,
                      "launches": aafwi.launch_count()}))


def ncu_lsrtm_case(args):
    """A small case of the LSRTM kernels for ncu: the LSRTM geometry (64 shots,
    737 x 240) cut to 64 time steps; one LSRTM gradient (Born pair forward
    storing the background history, adjoint with the Born imaging)."""
    import torch
    from paper_2008_11778_gb300 import aafwi, synth
    prob = synth.lsrtm()
    g = prob.geom.with_nt(64)
    plan = aafwi.Plan(g, c_max=4700.0, tile_z=args.tile_z, lanes=args.lanes)
    m0 = torch.as_tensor(prob.m_true.astype(np.float32), device="cuda")
    rho = torch.as_tensor(prob.extra["rho_true"].astype(np.float32), device="cuda")
    d = torch.empty(plan.trace_count, device="cuda")
    plan.born_forward(m0, rho, d)
    grad = torch.empty_like(m0)
    J = plan.adjoint_gradient(aafwi.MODE_LSRTM, m0, torch.zeros_like(rho), d, grad)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_lsrtm_case": "lsrtm-737x240-64shots-64steps", "J": J, "tile_z": plan.info.tile_z,
                      "lanes": plan.info.lanes, "launches": aafwi.launch_count()}))


def ncu_unet_case():
    """A small case of the learned preconditioner's kernels for ncu: the
    U-Net (C = 32) forward and one training step on a 16 x 96 x 256 batch."""
    import torch
    from paper_2008_11778_gb300 import aafwi
    net = aafwi.UNet(16, 96, 256, 32)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn((16, 2, 96, 256), device="cuda", generator=g)
    t = 0.1 * torch.randn((16, 96, 256), device="cuda", generator=g)
    y = torch.empty((16, 96, 256), device="cuda")
    net.forward(x, y)
    loss = net.train_step(x, t, 1e-4)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_unet_case": "unet-c32-16x96x256", "loss": loss, "launches": aafwi.launch_count()}))
    net.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--kernel-reps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ncu-case", action="store_true", help="small case for ncu captures")
    ap.add_argument("--ncu-unet-case", action="store_true", help="small U-Net case for ncu captures")
    ap.add_argument("--ncu-lsrtm-case", action="store_true", help="small LSRTM case for ncu captures")
    ap.add_argument("--engine", default="tuned", choices=["tuned"] + list(ENGINES),
                    help="sweep engine: the library's autotuner (default) or a fixed one")
    ap.add_argument("--tile-z", type=int, default=0, help="per-step tile rows with a fixed engine")
    ap.add_argument("--no-pdl", action="store_true", help="plain launches instead of programmatic dependents")
    ap.add_argument("--lanes", type=int, default=0, choices=range(9),
                    help="shot lanes of the per-step sweeps (0: the library's default)")
    ap.add_argument("--steps-per-launch", type=int, default=0, choices=(0, 1, 2),
                    help="forward time steps per launch (0: the library's default)")
    ap.add_argument("--tune-cache", default=None, help="autotuner cache file (default: the library's)")
    ap.add_argument("--learned-eval", type=int, default=3, help="held-out models for learned vs plain AA")
    ap.add_argument("--learned-target", type=float, default=1e-2)
    ap.add_argument("--learned-max-iters", type=int, default=120)
    args = ap.parse_args()
    if args.ncu_unet_case:
        ncu_unet_case()
    elif args.ncu_lsrtm_case:
        ncu_lsrtm_case(args)
    elif args.ncu_case:
        ncu_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
