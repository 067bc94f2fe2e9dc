"""Learned preconditioner for Anderson-accelerated FWI (not part of the paper).

A U-Net (aafwi.UNet: BF16 tensor-core kernels of this library) maps the
normalised pair [grad J(m_k) / max|grad J|, (m_k - mean) / std] to a model
update in units of std(m_k).  Training pairs come from the method's own plain
AA runs on seeded layered-faulted models: for every recorded iterate m_k the
target is (m_final - m_k) / std(m_k), m_final the run's last iterate.

In the inversion (LearnedAAInversion) each iteration first proposes
p_L = clip(p_k + std(p_k) * NN(grad_k, p_k)); the proposal is accepted only if
J(p_L) < J(p_k) (one forward sweep); otherwise the plain Alg. 2 step of
solve.AAInversion is taken.  The AA history always holds accepted iterates
and their gradients.
"""
import time

import numpy as np
import torch

from . import aafwi, solve


def net_grid(nz, nx):
    """Network grid (multiples of 8) holding an nz x nx model in its top-left corner."""
    return -(-nz // 8) * 8, -(-nx // 8) * 8


class Proposer:
    """Applies the network to (grad, m): features -> U-Net -> clipped update."""

    def __init__(self, net, nz, nx, device="cuda"):
        self.net = net
        self.nz, self.nx = nz, nx
        self.H, self.W = net_grid(nz, nx)
        assert (self.H, self.W) == (net.H, net.W)
        self.x = torch.empty((1, 2, self.H, self.W), dtype=torch.float32, device=device)
        self.delta = torch.empty((1, self.H, self.W), dtype=torch.float32, device=device)
        self.stats = torch.empty(3, dtype=torch.float64, device=device)

    def features(self, grad, m, x=None, stats=None):
        aafwi.learned_features(grad, m, self.H, self.W, self.x if x is None else x,
                               self.stats if stats is None else stats)

    def propose(self, grad, m, out, lo=0.0, hi=0.0):
        self.features(grad, m)
        self.net.forward(self.x, self.delta)
        aafwi.learned_apply(m, self.delta[0], self.stats, out, lo, hi)
        return out


class LearnedAAInversion(solve.AAInversion):
    """Alg. 2 with a learned proposal tried first at every iteration."""

    def __init__(self, plan, d_obs, p0, M, proposer, **kw):
        super().__init__(plan, d_obs, p0, M, **kw)
        self.proposer = proposer
        self.p_learn = torch.empty_like(self.p)
        self.n_learned = 0
        self.history["learned"] = []

    def step(self):
        self.proposer.propose(self.grad, self.p, self.p_learn, self.lo, self.hi)
        Jl = self._misfit_only(self.p_learn)
        self.n_forward += 1
        if Jl < self.J:
            # accepted: the history receives the accepted iterate p_k and its
            # gradient (as a plain step would), then p_{k+1} = p_L, whose stored
            # forward wavefield the gradient reuses
            self.aa.step(self.p, self.grad, self.p_tilde, self.p_bar)
            self.p, self.p_learn = self.p_learn, self.p
            self.J = self._gradient(self.p, True)
            self.n_adjoint += 1
            self.n_learned += 1
            self.history["J"].append(self.J)
            self.history["lam"].append(-1.0)
            self.history["Mk"].append(-1)
            self.history["learned"].append(True)
            self.k += 1
            return self.J
        self.history["learned"].append(False)
        return super().step()


def aa_history_pairs(plan, prob, M=10, iters=20, keep=(0, 2, 5, 10, 15), eta_factor=1e-4):
    """Run plain AA on `prob` and return (features [K,2,H,W], targets [K,H,W])
    for the iterates listed in `keep` (device tensors)."""
    dev = "cuda"
    nz, nx = prob.geom.nz, prob.geom.nx
    H, W = net_grid(nz, nx)
    m_true = torch.as_tensor(prob.m_true.astype(np.float32), device=dev)
    d_obs = torch.empty(plan.trace_count, device=dev)
    plan.model_forward(m_true, d_obs)
    saved = []

    def cb(k, p, grad, J):
        if k + 1 in keep:
            saved.append((p.clone(), grad.clone()))

    m0 = torch.as_tensor(prob.m_start.astype(np.float32), device=dev)
    # iterate 0 too
    g0 = torch.empty_like(m0)
    plan.adjoint_gradient(aafwi.MODE_FWI, m0, None, d_obs, g0)
    if 0 in keep:
        saved.insert(0, (m0.clone(), g0.clone()))
    out = solve.aa_fwi(plan, d_obs, m0, M=M, iters=iters, eta_factor=eta_factor, bounds=prob.m_bounds,
                       callback=cb)
    m_fin = out["p"]
    X = torch.zeros((len(saved), 2, H, W), device=dev)
    T = torch.zeros((len(saved), H, W), device=dev)
    stats = torch.empty(3, dtype=torch.float64, device=dev)
    for i, (m, g) in enumerate(saved):
        aafwi.learned_features(g, m, H, W, X[i], stats)
        T[i, :nz, :nx] = (m_fin - m) / stats[2].float()
    return X, T, out


def train(net, X, T, steps, batch=16, lr=1e-3, seed=0, log_every=0):
    """Adam on minibatches drawn from (X, T); returns the loss history."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = X.shape[0]
    hist = []
    for s in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), generator=g).to(X.device)
        L = net.train_step(X[idx].contiguous(), T[idx].contiguous(), lr)
        hist.append(L)
        if log_every and s % log_every == 0:
            print("train step %d loss %.4e" % (s, L), flush=True)
    return hist


def time_to_target(run, target, max_iters):
    """Iterate `run` until J/J0 <= target or max_iters; wall seconds (GPU synchronised)."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it = 0
    while run.J > target * run.J0 and it < max_iters:
        run.step()
        it += 1
    torch.cuda.synchronize()
    return time.perf_counter() - t0, it, run.J / run.J0


# ---------------------------------------------------------------------------
# training / evaluation driver
# ---------------------------------------------------------------------------

TRAIN_SEED0 = 4 * 1000 + 2008          # training models: seeds TRAIN_SEED0 + i
EVAL_SEED0 = 4 * 1000 + 2008 + 100000  # held-out models: disjoint seeds
WEIGHTS = __file__.replace("learned.py", "weights/unet_c32.npz")
# evaluation record of the committed weights on the held-out models, written by
# `python -m paper_2008_11778_gb300.learned --eval-only --eval 50 --record`
EVAL_RECORD = __file__.replace("learned.py", "weights/unet_c32_eval.json")


def save_weights(path, params, meta):
    """Store the parameters as BF16 bits (the runtime's inference copy is BF16,
    so nothing the network computes with is lost) plus the training metadata."""
    import os
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    b = np.ascontiguousarray(params, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)
    np.savez_compressed(path, params_bf16=b, **meta)


def load_weights(path=WEIGHTS):
    d = np.load(path)
    p = (d["params_bf16"].astype(np.uint32) << 16).view(np.float32)
    return p, {k: d[k] for k in d.files if k != "params_bf16"}


def train_preconditioner(n_models, iters=20, steps=4000, batch=16, lr=1e-3, C=32, log=print):
    """Generate pairs from plain AA runs on n_models training models and train
    a fresh network (He-initialised from a seeded generator); returns
    (params, info)."""
    from . import synth as S
    rng = np.random.default_rng(TRAIN_SEED0)
    prob0 = S.learned_model(TRAIN_SEED0)
    plan = aafwi.Plan(prob0.geom, c_max=4500.0 * 1.2)
    t0 = time.perf_counter()
    Xs, Ts = [], []
    for i in range(n_models):
        X, T, _ = aa_history_pairs(plan, S.learned_model(TRAIN_SEED0 + i), iters=iters)
        Xs.append(X)
        Ts.append(T)
    X, T = torch.cat(Xs), torch.cat(Ts)
    t_data = time.perf_counter() - t0
    log("training pairs %s from %d models in %.1f s" % (tuple(X.shape), n_models, t_data))
    plan.close()
    H, W = net_grid(prob0.geom.nz, prob0.geom.nx)
    net = aafwi.UNet(batch, H, W, C)
    net.set_params(he_init(net.nparam, C, int(rng.integers(1 << 31))))
    t0 = time.perf_counter()
    hist = train(net, X, T, steps, batch, lr, log_every=max(1, steps // 8))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    log("trained %d steps in %.1f s, loss %.3e -> %.3e" % (steps, t_train, hist[0], np.mean(hist[-50:])))
    params = net.get_params()
    net.close()
    return params, {"n_models": n_models, "pairs": int(X.shape[0]), "steps": steps, "data_s": t_data,
                    "train_s": t_train, "loss0": hist[0], "loss_end": float(np.mean(hist[-50:]))}


def he_init(n, C, seed):
    """He-normal weights and zero biases in the runtime's parameter layout."""
    rng = np.random.default_rng(seed)
    out = np.zeros(n, dtype=np.float32)
    o = 0
    for up, ci, co in _layer_list(C):
        nw = (4 if up else 9) * ci * co
        fan = ci if up else 9 * ci
        out[o:o + nw] = rng.standard_normal(nw) * np.sqrt(2.0 / fan)
        o += nw + co
    out[o:o + C] = rng.standard_normal(C) * 0.1 / np.sqrt(C)
    assert o + C + 1 == n
    return out


def _layer_list(C):
    L = [(False, 2, C), (False, C, C), (False, C, 2 * C), (False, 2 * C, 2 * C), (False, 2 * C, 4 * C),
         (False, 4 * C, 4 * C), (False, 4 * C, 8 * C), (False, 8 * C, 8 * C)]
    for l in (2, 1, 0):
        L += [(True, C << (l + 1), C << l), (False, C << (l + 1), C << l), (False, C << l, C << l)]
    return L


def compare(params, n_eval, target, max_iters, C=32, log=print, plain_eta_factors=(1e-4,)):
    """Wall seconds (GPU synchronised) for plain AA(10) and learned AA(10) to
    reach J/J0 <= target on n_eval held-out 400 x 150 models.  Plain AA runs
    once per step factor in plain_eta_factors (eta = factor max|p_0| /
    max|grad J(p_0)|; the first is the default reading, which the learned run
    also uses); row["plain"] is the default, row["plain_eta"] holds them all."""
    from . import synth as S
    prob0 = S.learned_eval_model(EVAL_SEED0)
    g = prob0.geom
    plan = aafwi.Plan(g, c_max=4500.0 * 1.2)
    H, W = net_grid(g.nz, g.nx)
    net = aafwi.UNet(1, H, W, C)
    net.set_params(params)
    prop = Proposer(net, g.nz, g.nx)
    rows = []
    for i in range(n_eval):
        prob = S.learned_eval_model(EVAL_SEED0 + i)
        mt = torch.as_tensor(prob.m_true.astype(np.float32), device="cuda")
        d = torch.empty(plan.trace_count, device="cuda")
        plan.model_forward(mt, d)
        m0 = torch.as_tensor(prob.m_start.astype(np.float32), device="cuda")
        row = {"seed": EVAL_SEED0 + i, "plain_eta": {}}
        arms = [("plain", f) for f in plain_eta_factors] + [("learned", plain_eta_factors[0])]
        for name, f in arms:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if name == "plain":
                run = solve.AAInversion(plan, d, m0, 10, bounds=prob.m_bounds, eta_factor=f)
            else:
                run = LearnedAAInversion(plan, d, m0, 10, prop, bounds=prob.m_bounds, eta_factor=f)
            _, it, r = time_to_target(run, target, max_iters)
            torch.cuda.synchronize()
            total = time.perf_counter() - t0
            res = {"seconds": total, "iterations": it, "J_over_J0": r, "reached": bool(r <= target),
                   "forward_passes": run.n_forward, "adjoint_passes": run.n_adjoint,
                   "learned_steps": getattr(run, "n_learned", 0), "eta_factor": f}
            run.close()
            if name == "plain":
                row["plain_eta"]["%g" % f] = res
                if f == plain_eta_factors[0]:
                    row["plain"] = res
            else:
                row["learned"] = res
        log(row)
        rows.append(row)
    plan.close()
    net.close()
    return rows


def best_plain(row):
    """The fastest plain arm of a row among those that reached the target, else
    the one with the lowest final J/J0."""
    arms = list(row["plain_eta"].values())
    reached = [a for a in arms if a["reached"]]
    if reached:
        return min(reached, key=lambda a: a["seconds"])
    return min(arms, key=lambda a: a["J_over_J0"])


def summarize(rows, target, max_iters):
    """Per-model seconds and flags, and the median / minimum speed-up of the
    learned arm over the default plain arm and over the best plain arm."""
    sp = [r["plain"]["seconds"] / r["learned"]["seconds"] for r in rows]
    bp = [best_plain(r) for r in rows]
    spb = [b["seconds"] / r["learned"]["seconds"] for b, r in zip(bp, rows)]
    both = [r["plain"]["reached"] and r["learned"]["reached"] for r in rows]
    both_b = [b["reached"] and r["learned"]["reached"] for b, r in zip(bp, rows)]
    return {
        "target": target, "max_iters": max_iters, "models": len(rows),
        "plain_eta_factors": sorted({float(k) for r in rows for k in r["plain_eta"]}),
        "plain_reached": sum(r["plain"]["reached"] for r in rows),
        "best_plain_reached": sum(b["reached"] for b in bp),
        "learned_reached": sum(r["learned"]["reached"] for r in rows),
        "median_speedup": float(np.median(sp)), "min_speedup": float(np.min(sp)),
        "median_speedup_both_reached": float(np.median([x for x, k in zip(sp, both) if k])) if any(both) else None,
        "median_speedup_vs_best_plain": float(np.median(spb)), "min_speedup_vs_best_plain": float(np.min(spb)),
        "median_speedup_vs_best_plain_both_reached":
            float(np.median([x for x, k in zip(spb, both_b) if k])) if any(both_b) else None,
        "plain_s": [r["plain"]["seconds"] for r in rows],
        "plain_reached_flags": [r["plain"]["reached"] for r in rows],
        "best_plain_s": [b["seconds"] for b in bp],
        "best_plain_eta_factor": [b["eta_factor"] for b in bp],
        "best_plain_reached_flags": [b["reached"] for b in bp],
        "learned_s": [r["learned"]["seconds"] for r in rows],
        "learned_reached_flags": [r["learned"]["reached"] for r in rows],
    }


def load_eval_record(path=EVAL_RECORD):
    """The committed evaluation record's summary (None if absent)."""
    import json
    import os
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    out = dict(rec["summary"])
    out["source"] = os.path.basename(path)
    out["command"] = rec.get("command")
    out["gpu"] = rec.get("gpu")
    return out


def network_rate(C=32, reps=20):
    """CUDA-event times (best of `reps`) of the network (seeded He weights):
    forward and training step (forward, backward, Adam) on a 16 x 96 x 256
    training batch, and the forward on one 152 x 400 evaluation input."""
    out = {"C": C, "gpu": torch.cuda.get_device_name(0)}
    for key, (B, H, W), train_too in (("train_16x96x256", (16, 96, 256), True), ("eval_1x152x400", (1, 152, 400), False)):
        net = aafwi.UNet(B, H, W, C)
        net.set_params(he_init(net.nparam, C, 0))
        g = torch.Generator(device="cuda").manual_seed(0)
        x = torch.randn((B, 2, H, W), device="cuda", generator=g)
        t = 0.1 * torch.randn((B, H, W), device="cuda", generator=g)
        y = torch.empty((B, H, W), device="cuda")
        calls = [("forward_ms", lambda: net.forward(x, y))]
        if train_too:
            calls.append(("train_step_ms", lambda: net.train_step(x, t, 1e-6)))
        for name, f in calls:
            for _ in range(3):
                f()
            ms = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                f()
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            out.setdefault(key, {})[name] = min(ms)
        net.close()
    return out


if __name__ == "__main__":
    import argparse
    import json
    import sys
    ap = argparse.ArgumentParser(description="train / evaluate the learned preconditioner")
    ap.add_argument("--models", type=int, default=120)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--eval", type=int, default=4)
    ap.add_argument("--target", type=float, default=0.1)
    ap.add_argument("--max-iters", type=int, default=80)
    ap.add_argument("--eta-factors", default="1e-4", help="comma-separated step factors of the plain arms")
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--eval-only", action="store_true")
    ap.add_argument("--record", nargs="?", const=EVAL_RECORD, default=None,
                    help="write the evaluation record (default path: the committed record)")
    ap.add_argument("--rate", action="store_true", help="time the network's forward and training step and stop")
    a = ap.parse_args()
    if a.rate:
        print(json.dumps({"unet_rate": network_rate()}))
        raise SystemExit(0)
    if a.eval_only:
        params, meta = load_weights(a.out)
    else:
        params, meta = train_preconditioner(a.models, steps=a.steps)
        save_weights(a.out, params, {k: np.asarray(v) for k, v in meta.items()})
    factors = tuple(float(x) for x in a.eta_factors.split(","))
    rows = compare(params, a.eval, a.target, a.max_iters, plain_eta_factors=factors,
                   log=lambda r: print(json.dumps(r, default=float), flush=True))
    summary = summarize(rows, a.target, a.max_iters)
    if a.record:
        rec = {"what": "learned AA(10) vs plain AA(10) on held-out 400 x 150 models (seeds EVAL_SEED0 + i), "
                       "wall seconds to J/J0 <= target on one GPU",
               "command": "python -m paper_2008_11778_gb300.learned " + " ".join(sys.argv[1:]),
               "gpu": torch.cuda.get_device_name(0), "training": {k: float(v) for k, v in meta.items()},
               "summary": summary, "rows": rows}
        with open(a.record, "w") as f:
            json.dump(rec, f, indent=1, default=float)
    print(json.dumps({"train": {k: float(v) for k, v in meta.items()}, "summary": summary}, default=float))
