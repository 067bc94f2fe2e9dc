"""Benchmark: Anderson-accelerated FWI on the large workload (2001 x 601 grid,
dx 10 m, layered-faulted 1500-5500 m/s with three high-velocity lenses, 200
shots with uneven apertures, Ricker 12 Hz, dt 0.8 ms, 6000 steps, AA(10));
the plan runs the shots in batches with the full wavefield history of a batch.

One step = one iteration of Alg. 2 on the GPU: the gradient at the accepted
iterate (per shot batch: forward sweep storing T^n = L u^n + s^n, adjoint
sweep with the imaging condition, misfit; shot sum and E^T), the AA(10) step
(FP64 Gram / solve), the line-search trial forward sweep(s) with receiver
gather and misfit, and the combine.  Metric: grid-point updates per second,
counting every forward and adjoint pass the step ran (sum_s nt_s * NZ * NX
per pass).  The batched workload (400 x 150, 32 shots, 2500 steps) is
reported beside it as a secondary line (its wavefields stay in L2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload large|batched]

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

WORKLOADS = {
    "large": "fwi-large-2001x601-200shots-6000steps-aa10",
    "batched": "fwi-batched-400x150-32shots-2500steps-aa10",
}
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


def traffic_record(workload, kernel, updates_per_launch):
    """DRAM bytes (read + write) per launch of `kernel` on `workload`, from
    the committed ncu record (bytes per grid-point update over the captured
    launches, scaled to the updates of the benchmark's launch), or None if
    absent or taken on different kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    rec = d.get(workload, {}).get(kernel)
    if not rec or rec.get("source_hash") != kernel_source_hash():
        return None
    return rec["dram_bytes_per_update"] * updates_per_launch


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def make_problem(name, shots=0, nt=0):
    """The workload's problem; shots > 0 keeps only its first `shots` shots
    and nt > 0 cuts the records to nt steps (profiling runs: the launch list
    of a smaller command with the same batches and kernels, whose per-step
    costs do not depend on the record length)."""
    from paper_2008_11778_gb300 import synth
    prob = synth.large() if name == "large" else synth.batched()
    if shots:
        prob.geom = prob.geom.subset(range(min(shots, prob.geom.S)))
    if nt:
        prob.geom = prob.geom.with_nt(nt)
    return prob


def workload_name(args):
    w = WORKLOADS[args.workload]
    if args.shots:
        w += "-first%dshots" % args.shots
    if args.nt:
        w += "-cut%dsteps" % args.nt
    return w


def host_mem_available():
    """MemAvailable of the host in bytes (Linux), or None."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return None


def oracle_sample_size(prob, cores, nt_cap):
    """A bounded sample of the workload for the FP64 oracle: one shot per host
    thread (the oracle parallelises over shots) and the record cut to at most
    nt_cap steps, fewer if the oracle's stored per-step fields (8 B x padded
    cells x steps per shot) would take more than a quarter of the free host
    memory."""
    g = prob.geom
    nsh = min(g.S, max(1, cores))
    nt = min(int(g.nt.max()), nt_cap)
    avail = host_mem_available()
    if avail:
        per_step = 8 * g.NZ * g.NX * nsh
        nt = max(16, min(nt, int(0.3 * avail / per_step)))
    return list(range(nsh)), nt


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on the host cores
# ---------------------------------------------------------------------------

def oracle_sample(prob, shots, nt, reps=1):
    """Time the oracle's FWI gradient (forward + adjoint) on `shots` shots with
    the record cut to nt steps; returns (updates/s, seconds, cores, sample text)."""
    import oracle
    g = prob.geom.subset(shots)
    g.nt = np.minimum(g.nt, nt).astype(np.int32)
    d_obs = oracle.forward(g, prob.m_true)
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.fwi_gradient(g, prob.m_start, d_obs)
    dt = time.perf_counter() - t0
    upd = 2 * g.updates_per_pass() * reps
    return upd / dt, dt, oracle.num_threads(), "%d of %d shots, record cut to %d of %d steps, %d gradient(s)" % (
        len(shots), prob.geom.S, int(g.nt.max()), int(prob.geom.nt.max()), reps)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    prob = make_problem(args.workload, args.shots, args.nt)
    import oracle
    cores = oracle.num_threads()
    # a few seconds per step on the host cores (the oracle stores every step
    # of a shot): the whole --steps K --warmup W run ends within minutes
    shots, nt = oracle_sample_size(prob, cores, 128 if args.workload == "large" else 2500)
    times = []
    g = prob.geom.subset(shots)
    upd = 2 * int(np.minimum(g.nt, nt).astype(np.int64).sum()) * g.NZ * g.NX
    sample = ""
    for i in range(args.warmup + args.steps):
        v, dt, cores, sample = oracle_sample(prob, shots, nt)
        if i >= args.warmup:
            times.append(dt)
    ms = 1e3 * float(np.mean(times))
    value = upd / (ms / 1e3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_name(args), "sample": sample, "l2": "inputs larger than L2"},
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


def make_plan(aafwi, prob, g, m_tune, args, lanes=None):
    """The benchmark's plan: the library's autotuned launch configuration
    (timed on short sweeps of this geometry before the timed region), or the
    engine / tile height given on the command line."""
    kw = dict(pdl=not args.no_pdl, steps_per_launch=args.steps_per_launch,
              lanes=args.lanes if lanes is None else lanes, shots_per_batch=args.shots_per_batch)
    if args.engine == "tuned":
        return aafwi.Plan(g, c_max=prob.c_bounds[1], tune_model=m_tune, tune_cache=args.tune_cache, **kw)
    return aafwi.Plan(g, c_max=prob.c_bounds[1], engine=ENGINES[args.engine], tile_z=args.tile_z, **kw)


class CallTimer:
    """CUDA events on the launching stream around every call of one plan
    method while `active` (the call itself is unchanged)."""

    def __init__(self, plan, name):
        import torch
        self.pairs, self.active = [], False
        orig = getattr(plan, name)

        def timed(*a, **k):
            if not self.active:
                return orig(*a, **k)
            st = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            r = orig(*a, **k)
            e1.record(st)
            self.pairs.append((e0, e1))
            return r

        setattr(plan, name, timed)

    def ms(self):
        return [e0.elapsed_time(e1) for e0, e1 in self.pairs]


def sweep_launches(plan, info, nt, forward=True):
    """Kernel launches of one sweep over every batch: per-step engines launch
    one kernel per time step and shot lane (two steps per launch for k_fwd2),
    persistent sweeps one per batch."""
    import paper_2008_11778_gb300.aafwi as aafwi
    eng, spl = info.engine, info.steps_per_launch
    if forward and eng == aafwi.ENGINE_PERSISTENT:
        return info.n_batches
    if not forward and eng in (aafwi.ENGINE_PERSISTENT, aafwi.ENGINE_HYBRID):
        return info.n_batches
    # lanes of the last batch may be fewer when it holds fewer shots
    S, Sb = plan.geom.S, info.shots_per_batch
    steps = (nt + 1) // 2 if (forward and spl == 2) else nt
    total = 0
    for b in range(info.n_batches):
        total += min(info.lanes, min(Sb, S - b * Sb)) * steps
    return total


def kernel_roof(name, what, bpu, points, launches, sweep_ms, share, peak, peak_kind, nt, traffic_key):
    """Algorithmic bytes of the sweep / launches over the sweep's CUDA-event
    time / launches (lanes overlap, so this is the time per launch of the
    launch chains together); beside it the DRAM bytes per launch of the
    committed ncu record (traffic_key = (workload, record name)) over the
    same time, as a fraction of the same peak."""
    b = bpu * points / launches
    ms = sweep_ms / launches
    gbs = b / (ms * 1e-3) / 1e9
    traffic = traffic_record(traffic_key[0], traffic_key[1], points / launches) if traffic_key else None
    out = {"bound": "hbm", "kernel": name + " (" + what + ")", "achieved": gbs, "peak": peak,
           "unit": "GB/s", "frac": gbs / peak, "peak_kind": peak_kind, "traffic": traffic,
           "bytes_per_launch": b, "ms_per_launch": ms, "launches_per_sweep": launches,
           "us_per_time_step": 1e3 * sweep_ms / nt, "share_of_step": share}
    if traffic:
        out["dram_achieved"] = traffic / (ms * 1e-3) / 1e9
        out["dram_frac"] = out["dram_achieved"] / peak
    return out


def alg2_run(aafwi, solve, prob, plan, dev, warmup, steps, ws, clocks=None):
    """Observed data from this library's forward on the true model, then
    `warmup` untimed and `steps` timed Alg. 2 iterations from the start model.
    Returns the run and the timed-region record."""
    import torch
    g = prob.geom
    lo, hi = prob.m_bounds
    m_true = torch.as_tensor(prob.m_true.astype(np.float32), device=dev)
    d_obs = torch.empty(plan.trace_count, device=dev)
    plan.model_forward(m_true, d_obs)
    del m_true
    m0 = torch.as_tensor(prob.m_start.astype(np.float32), device=dev)
    trial = CallTimer(plan, "model_forward")
    grad = CallTimer(plan, "adjoint_gradient")
    run = solve.AAInversion(plan, d_obs, m0, M=prob.M, bounds=(lo, hi))
    for _ in range(warmup):
        run.step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    stream = torch.cuda.current_stream()
    if clocks:
        clocks.start()
    nf0, na0 = run.n_forward, run.n_adjoint
    l0 = aafwi.launch_count()
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    trial.active = grad.active = True
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed_region")   # ncu --nvtx-include timed_region/ selects these launches
    e_start.record(stream)
    t0 = time.perf_counter()
    for _ in range(steps):
        run.step()
    e_end.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    trial.active = grad.active = False
    launches = aafwi.launch_count() - l0
    clk = clocks.stop() if clocks else None
    ms_total = job_time_ms(e_start.elapsed_time(e_end), ws, dev)
    nf, na = run.n_forward - nf0, run.n_adjoint - na0
    rec = {"ms_total": ms_total, "wall": wall, "launches": launches, "clocks": clk, "nf": nf, "na": na,
           "trial_ms": trial.ms(), "grad_ms": grad.ms(),
           "updates": (nf + na) * g.updates_per_pass()}
    return run, rec


def run_ours(args):
    import torch
    from paper_2008_11778_gb300 import aafwi, solve
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prob = make_problem(args.workload, args.shots, args.nt)
    g = prob.geom
    m_start = torch.as_tensor(prob.m_start.astype(np.float32), device=dev)
    plan = make_plan(aafwi, prob, g, m_start, args)
    tuning = getattr(plan, "tuning", None)
    info = plan.info
    peak, peak_kind = read_peaks()
    nt = int(g.nt.max())
    pts_sweep = sum(active_points(g, n) for n in range(nt))

    clocks = ClockSampler(local)
    run, rec = alg2_run(aafwi, solve, prob, plan, dev, args.warmup, args.steps, ws, clocks)
    ms_total = rec["ms_total"]
    value = job_value(rec["updates"], ws, ms_total)
    J_ratio = run.J / run.J0 if run.J0 > 0 else None
    run.close()

    # Dominant kernel, timed live over the timed region: the line search's
    # trial forward sweeps (k_fwd; with shot batches they store no history,
    # so their traffic is the algorithmic 16 B per update).
    fwd_launches = sweep_launches(plan, info, nt, forward=True)
    lanes = info.lanes
    spl = info.steps_per_launch
    fwd_name = ("k_fwd_persist" if info.engine == aafwi.ENGINE_PERSISTENT
                else "k_fwd2" if spl == 2 else "k_fwd")
    trial_ms = rec["trial_ms"]
    t_trials = float(np.sum(trial_ms)) if trial_ms else 0.0
    t_grads = float(np.sum(rec["grad_ms"])) if rec["grad_ms"] else 0.0
    # DRAM records: the line-search sweeps of a batched plan store no history
    trial_rec = (args.workload, "k_fwd_traces" if info.n_batches > 1 else "k_fwd_history")
    fwd_roof = None
    if trial_ms:
        fwd_roof = kernel_roof(fwd_name, "line-search forward sweeps, timed live over the timed region, "
                               "%d step(s) per launch" % (2 if spl == 2 else 1),
                               BYTES_FWD, pts_sweep, fwd_launches, float(np.median(trial_ms)),
                               t_trials / ms_total, peak, peak_kind, nt,
                               trial_rec if fwd_name == "k_fwd" else None)
        fwd_roof["sweeps_timed"] = len(trial_ms)

    e2e = run_e2e(plan, prob, dev, args.e2e_steps) if args.e2e_steps > 0 else None
    plan.close()
    del plan
    torch.cuda.empty_cache()

    # The other kernel (k_adj, the adjoint with imaging) and the forward that
    # stores the history, on one shot batch of the same geometry at the full
    # record length (a plan of its own, outside the timed region).
    roofline = dict(fwd_roof or {}, other_kernels=[])
    if args.kernel_reps > 0:
        roofline = batch_kernel_roofs(aafwi, prob, m_start, info, args, fwd_roof, fwd_name, t_grads, ms_total,
                                      peak, peak_kind, nt)

    secondary = None
    if args.workload == "large" and not args.no_secondary:
        secondary = run_secondary(aafwi, solve, dev, args, peak, peak_kind)

    learned_cmp = None
    if args.learned_eval > 0:
        learned_cmp = learned_vs_plain(args.learned_eval, args.learned_target, args.learned_max_iters)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(prob, args.workload)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": workload_name(args), "grid": [g.nz, g.nx], "padded": [g.NZ, g.NX],
                           "shots": g.S, "nt": nt, "M": prob.M,
                           "shots_per_batch": info.shots_per_batch, "batches": info.n_batches,
                           "checkpoint_every": info.checkpoint_every,
                           "engine": ENGINE_NAMES.get(info.engine, info.engine),
                           "tile_z": info.tile_z, "pdl": not args.no_pdl,
                           "steps_per_launch": info.steps_per_launch, "lanes": info.lanes,
                           "autotune": None if tuning is None else {
                               "steps": tuning.get("steps"), "cached": tuning.get("cached"),
                               "lanes": tuning.get("lanes"),
                               "table_ms": [[ENGINE_NAMES.get(r[0], r[0])] + list(r[1:]) for r in tuning["table"]]},
                           "l2": "inputs larger than L2 (wavefield history %.1f GB per batch)" % (
                               info.workspace_bytes / 1e9),
                           "passes": {"forward": rec["nf"], "adjoint": rec["na"]},
                           "fwi_iterations_per_s": args.steps / (ms_total / 1e3),
                           "J_over_J0": J_ratio},
                "gpu_launches": rec["launches"], "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "secondary": secondary, "learned_vs_plain": learned_cmp,
                "clocks": rec["clocks"], "host_wall_s": rec["wall"]}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def batch_kernel_roofs(aafwi, prob, m_start, info, args, fwd_roof, fwd_name, t_grads, ms_total, peak, peak_kind,
                       nt):
    """Roofline objects of the adjoint and of the history-storing forward,
    timed on one batch; the dominant kernel first, the others beside it."""
    kt = time_batch_sweeps(aafwi, prob, m_start, info, args)
    adj_roof = kernel_roof("k_adj_persist" if kt["adj_launches"] == 1 else "k_adj",
                           "adjoint sweep + imaging, one batch of %d shots, timed alone" % kt["shots"],
                           BYTES_ADJ, kt["points"], kt["adj_launches"], kt["adj_ms"],
                           None, peak, peak_kind, nt, (args.workload, "k_adj") if kt["adj_launches"] > 1 else None)
    adj_roof["share_of_step"] = (t_grads / ms_total) * kt["adj_ms"] / (kt["adj_ms"] + kt["fwd_ms"])
    fwdT_roof = kernel_roof(fwd_name, "forward sweep storing T^n for the adjoint, one batch of %d shots, "
                            "timed alone" % kt["shots"], BYTES_FWD, kt["points"], kt["fwd_launches"],
                            kt["fwd_ms"], None, peak, peak_kind, nt,
                            (args.workload, "k_fwd_history") if fwd_name == "k_fwd" else None)
    fwdT_roof["share_of_step"] = (t_grads / ms_total) * kt["fwd_ms"] / (kt["adj_ms"] + kt["fwd_ms"])
    # k_fwd runs both in the line-search sweeps and, storing T^n, in the
    # gradient: the kernel's share of the step is the sum of the two
    fwd_share = fwdT_roof["share_of_step"] + (fwd_roof["share_of_step"] if fwd_roof else 0.0)
    if fwd_roof is None or adj_roof["share_of_step"] > fwd_share:
        return dict(adj_roof, other_kernels=[k for k in (fwd_roof, fwdT_roof) if k])
    return dict(fwd_roof, kernel_share_of_step=fwd_share, other_kernels=[adj_roof, fwdT_roof])


def time_batch_sweeps(aafwi, prob, m_start, info, args):
    """CUDA-event time of the forward sweep storing the history (model_forward
    of a one-batch plan) and of the adjoint sweep reusing it (adjoint_gradient:
    adjoint, misfit, shot sum) for the first batch of shots at full record
    length, with the launch configuration of the benchmark's plan."""
    import torch
    g = prob.geom.subset(range(info.shots_per_batch))
    plan = aafwi.Plan(g, c_max=prob.c_bounds[1], engine=info.engine, tile_z=info.tile_z,
                      pdl=not args.no_pdl, steps_per_launch=info.steps_per_launch, lanes=info.lanes)
    pi = plan.info
    stream = torch.cuda.current_stream()
    nt = int(g.nt.max())
    grad = torch.empty_like(m_start)
    d_obs = torch.zeros(plan.trace_count, device=m_start.device)
    f_ms, a_ms = [], []
    for _ in range(args.kernel_reps + 1):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        plan.model_forward(m_start)
        e1.record(stream)
        plan.adjoint_gradient(0, m_start, None, d_obs, grad, sync=False, reuse_forward=True)
        e2.record(stream)
        torch.cuda.synchronize()
        f_ms.append(e0.elapsed_time(e1))
        a_ms.append(e1.elapsed_time(e2))
    out = {"fwd_ms": statistics.median(f_ms[1:]), "adj_ms": statistics.median(a_ms[1:]),
           "fwd_launches": sweep_launches(plan, pi, nt, True), "adj_launches": sweep_launches(plan, pi, nt, False),
           "points": sum(active_points(g, n) for n in range(nt)), "shots": g.S, "lanes": pi.lanes}
    plan.close()
    del d_obs
    torch.cuda.empty_cache()
    return out


def run_secondary(aafwi, solve, dev, args, peak, peak_kind):
    """The batched workload (400 x 150, 32 shots, 2500 steps, AA(10)) with
    the same protocol: its per-step wavefields fit in L2, so its algorithmic
    bytes do not reach DRAM."""
    import torch
    prob = make_problem("batched")
    g = prob.geom
    m_start = torch.as_tensor(prob.m_start.astype(np.float32), device=dev)
    plan = make_plan(aafwi, prob, g, m_start, args)
    info = plan.info
    run, rec = alg2_run(aafwi, solve, prob, plan, dev, 3, args.secondary_steps, 1)
    nt = int(g.nt.max())
    pts = sum(active_points(g, n) for n in range(nt))
    out = {"workload": WORKLOADS["batched"], "value": rec["updates"] / (rec["ms_total"] / 1e3), "unit": UNIT,
           "steps": args.secondary_steps, "warmup": 3, "ms_per_step": rec["ms_total"] / args.secondary_steps,
           "passes": {"forward": rec["nf"], "adjoint": rec["na"]},
           "fwi_iterations_per_s": args.secondary_steps / (rec["ms_total"] / 1e3),
           "J_over_J0": run.J / run.J0 if run.J0 > 0 else None,
           "engine": ENGINE_NAMES.get(info.engine, info.engine), "tile_z": info.tile_z, "lanes": info.lanes,
           "gpu_launches": rec["launches"]}
    if rec["trial_ms"]:
        out["k_fwd"] = kernel_roof("k_fwd", "line-search forward sweeps (L2-resident fields)", BYTES_FWD, pts,
                                   sweep_launches(plan, info, nt, True), float(np.median(rec["trial_ms"])),
                                   float(np.sum(rec["trial_ms"])) / rec["ms_total"], peak, peak_kind, nt,
                                   ("batched", "k_fwd_history"))
    run.close()
    plan.close()
    torch.cuda.empty_cache()
    return out


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
    del d_dev
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
            "ms_per_step": ms, "steps": steps,
            "call": "aafwi_adjoint_gradient_host (FWI): host m and d_obs in, host gradient and J out"}


def learned_vs_plain(n_eval, target, max_iters):
    """Second half of the metric: wall seconds (same GPU) for plain AA(10) and
    for AA(10) with the trained learned preconditioner to reach J/J0 <= target
    on held-out 400 x 150 models (16 shots, 2500 steps).  The committed
    evaluation record of the same weights on all held-out models (written by
    `python -m paper_2008_11778_gb300.learned --eval-only`) is attached."""
    from paper_2008_11778_gb300 import learned
    params, meta = learned.load_weights()
    rows = learned.compare(params, n_eval, target, max_iters, log=lambda *a: None)
    sp = [r["plain"]["seconds"] / r["learned"]["seconds"] for r in rows]
    out = {"metric": "wall-s to J/J0 <= %g, learned vs plain AA(10)" % target, "target": target,
           "max_iters": max_iters, "models": len(rows),
           "plain_s": [r["plain"]["seconds"] for r in rows],
           "learned_s": [r["learned"]["seconds"] for r in rows],
           "plain_reached": [bool(r["plain"]["reached"]) for r in rows],
           "learned_reached": [bool(r["learned"]["reached"]) for r in rows],
           "plain_iters": [r["plain"]["iterations"] for r in rows],
           "learned_iters": [r["learned"]["iterations"] for r in rows],
           "median_speedup": float(np.median(sp)),
           "training": {k: float(v) for k, v in meta.items()}}
    record = learned.load_eval_record()
    if record is not None:
        out["record"] = record
    return out


def cpu_baseline(prob, workload):
    """The FP64 oracle on the host cores, on a bounded sample of the workload
    (one shot per thread, the record cut to what host memory allows, and as
    many gradients as take 10-30 s)."""
    import oracle
    cores = oracle.num_threads()
    shots, nt = oracle_sample_size(prob, cores, 768 if workload == "large" else 2500)
    reps = 2 if workload == "large" else 1
    v, dt, cores, sample = oracle_sample(prob, shots, nt, reps)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "seconds": dt}


def ncu_case(args):
    """A small case of the benchmark's kernels for ncu captures: the
    workload's geometry cut to 64 time steps.  Large workload: two batches of
    the benchmark's batch size (the trial forward of a batched plan stores no
    history), one forward sweep, then one gradient (per batch: forward storing
    T^n, adjoint).  Batched workload: all 32 shots, one forward sweep and one
    adjoint sweep reusing it.  Engine, tile height and lanes from the command
    line (the benchmark line's config)."""
    import torch
    from paper_2008_11778_gb300 import aafwi
    prob = make_problem(args.workload)
    kw = dict(engine=ENGINES.get(args.engine, 0), tile_z=args.tile_z, pdl=not args.no_pdl,
              steps_per_launch=args.steps_per_launch, lanes=args.lanes)
    if args.workload == "large":
        Sb = args.ncu_batch
        g = prob.geom.subset(range(2 * Sb)).with_nt(64)
        plan = aafwi.Plan(g, c_max=prob.c_bounds[1], shots_per_batch=Sb, **kw)
        name = "large-2001x601-%dshots-in-2-batches-64steps" % (2 * Sb)
    else:
        g = prob.geom.with_nt(64)
        plan = aafwi.Plan(g, c_max=prob.c_bounds[1], **kw)
        name = "batched-400x150-32shots-64steps"
    m = torch.as_tensor(prob.m_start.astype(np.float32), device="cuda")
    d_obs = torch.zeros(plan.trace_count, device="cuda")
    grad = torch.empty_like(m)
    plan.model_forward(m)
    J = plan.adjoint_gradient(aafwi.MODE_FWI, m, None, d_obs, grad, reuse_forward=plan.keeps_forward)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": name, "J": J, "engine": ENGINE_NAMES.get(plan.info.engine),
                      "tile_z": plan.info.tile_z, "lanes": plan.info.lanes,
                      "shots_per_batch": plan.info.shots_per_batch, "batches": plan.info.n_batches,
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
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS))
    ap.add_argument("--shots", type=int, default=0, help="keep only the first N shots (profiling runs)")
    ap.add_argument("--nt", type=int, default=0, help="cut the records to N steps (profiling runs)")
    ap.add_argument("--shots-per-batch", type=int, default=0,
                    help="fix the plan's shot batch (profiling runs of a cut workload: the batches of the full one)")
    ap.add_argument("--kernel-reps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="end-to-end gradients through host buffers (default 1 large, 3 batched)")
    ap.add_argument("--secondary-steps", type=int, default=10)
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ncu-case", action="store_true", help="small case for ncu captures")
    ap.add_argument("--ncu-batch", type=int, default=3,
                    help="shots per batch of the large ncu case (the planner takes 3 on a GB300)")
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
    if args.e2e_steps is None:
        args.e2e_steps = 1 if args.workload == "large" else 3
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
