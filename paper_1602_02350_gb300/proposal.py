"""Training and evaluating the parameter-proposal network (rs_propose) on runs of the method itself.

Pipeline (every solve and every network step runs in librs.so; this module only draws problems,
measures, and keeps the records):

1. ``generate``: draw problems (n log-uniform, d from {256, 512, 1024, 2048} log-uniform,
   power-law spectrum j^-alpha with alpha ~ U[1, 2.5], lambda log-uniform), compute the network
   input (rank-64 sketch + tr(C)), then run a grid of settings for each problem in ONE batched
   call (rs_solve_batched: k in {16, 32, 64} x eta_mult x m / n, per-epoch snapshots).  Each
   setting's time to relative suboptimality 1e-6 is modelled from measured costs:
   t_pre(k) + epochs * (t_fg + m t_step), with t_pre, t_fg and t_step timed on this problem
   through the one-problem path, and epochs read off the snapshots against the closed-form
   minimiser (normal equations accumulated in double on the GPU, solved on the host).
   The label is the fastest setting.
2. ``train``: fit the network (rs_mlp_train_step, Adam) to (log2 k, ln eta_mult, log2(m/n)) of the
   labels, inputs and outputs normalised by the training set's mean and spread.
3. ``evaluate``: held-out problems; the proposal against the theory-set parameters (rs_propose
   without weights) and the fixed practice setting (k = 64, eta_mult = 1, m = 2n), each timed
   end to end through the one-problem path.

Run ``python -m paper_1602_02350_gb300.proposal all`` to regenerate the committed records.
"""

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import _lib as rs
from . import synth

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "proposal_weights.npz")
RUNS = os.path.join(HERE, "proposal_runs.npz")
EVAL = os.path.join(HERE, "proposal_eval.json")

K_GRID = (16, 32, 64)
ETA_GRID = (0.5, 1.0, 1.5, 2.0, 3.0)
M_GRID = (1 / 64, 1 / 32, 1 / 16, 1 / 8, 1 / 4, 1 / 2, 1.0)
TARGET = 1e-6


# ------------------------------------------------------------------ problems and reference solutions

def draw_problem(rng, n_range=(16384, 131072), d_choices=(256, 512, 1024, 2048), alpha=(1.0, 2.5),
                 lam=(1e-7, 1e-3), spike_prob=0.0):
    """A training or evaluation problem: n log-uniform, d from d_choices, spectrum j^-alpha; with
    probability spike_prob the leading r ~ U{5..40} eigenvalues are also multiplied by s, log-uniform
    in [10, 1000] (a few dominant directions over the power law)."""
    n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1]))) / 64) * 64)
    d = int(d_choices[int(rng.integers(len(d_choices)))])
    spec = dict(n=n, d=d, alpha=float(rng.uniform(*alpha)), lam=float(math.exp(rng.uniform(math.log(lam[0]),
                                                                                          math.log(lam[1])))),
                seed=int(rng.integers(1 << 30)), spike_r=0, spike_s=1.0)
    if spike_prob > 0.0 and rng.uniform() < spike_prob:
        spec["spike_r"] = int(rng.integers(5, 41))
        spec["spike_s"] = float(math.exp(rng.uniform(math.log(10.0), math.log(1000.0))))
    return spec


def make_data(spec, device="cuda"):
    spectrum = np.arange(1, spec["d"] + 1, dtype=np.float64) ** -spec["alpha"]
    spectrum[:spec.get("spike_r", 0)] *= spec.get("spike_s", 1.0)
    X, y, _ = synth.problem(spec["n"], spec["d"], spectrum, 0.05, spec["seed"], device=device, dtype=torch.float32)
    return X.contiguous(), y.float().contiguous()


class Reference:
    """w* of Eq. (1) from the normal equations (Gram matrix accumulated in double on the GPU,
    d x d solve on the host), and relative suboptimality of many iterates at once."""

    def __init__(self, X, y, lam):
        n, d = X.shape
        G = torch.zeros(d, d, dtype=torch.float64, device=X.device)
        b = torch.zeros(d, dtype=torch.float64, device=X.device)
        for r0 in range(0, n, 16384):
            Xb = X[r0:r0 + 16384].double()
            G += Xb.T @ Xb
            b += Xb.T @ y[r0:r0 + 16384].double()
        self.H = G / n + lam * torch.eye(d, dtype=torch.float64, device=X.device)
        ws = np.linalg.solve(self.H.cpu().numpy(), (b / n).cpu().numpy())
        self.w = torch.from_numpy(ws).to(X.device)
        r = torch.zeros((), dtype=torch.float64, device=X.device)
        for r0 in range(0, n, 16384):
            e = X[r0:r0 + 16384].double() @ self.w - y[r0:r0 + 16384].double()
            r += e @ e
        self.L = float(0.5 * r / n + 0.5 * lam * (self.w @ self.w))

    def rel(self, W):
        E = W.double().reshape(-1, self.w.shape[0]) - self.w
        return (0.5 * ((E @ self.H) * E).sum(1) / self.L).cpu().numpy()


def first_reached(rel, target=TARGET):
    hit = np.nonzero(rel <= target)[0]
    return int(hit[0]) if hit.size else -1


def _timed(fn):
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    out = fn()
    b.record()
    torch.cuda.synchronize()
    return out, a.elapsed_time(b)


def network_features(sigma2, lam, n, d):
    """The network's input as rs_propose forms it: 0.5 log(sigma2_i / sigma2_0) for the 64 leading
    sketched values, log(lam / sigma2_0), log n, log d (invariant to the scale of X)."""
    ls = 0.5 * np.log(np.maximum(np.asarray(sigma2, np.float64)[:64], 1e-60))
    return np.concatenate([ls - ls[0], [math.log(lam) - 2.0 * ls[0], math.log(n), math.log(d)]])


def features(ctx, X, lam, seed):
    V, s2 = rs.rs_sketch(ctx, X, 64, seed)
    trc = rs.rs_trace_c(ctx, X)
    return V, s2, trc


# ------------------------------------------------------------------ labelling runs

def label_problem(ctx, spec, epochs=64):
    X, y = make_data(spec)
    n, d, lam = spec["n"], spec["d"], spec["lam"]
    ref = Reference(X, y, lam)
    _, s2, trc = features(ctx, X, lam, spec["seed"] + 1)
    s2n = s2.cpu().numpy()
    feat = network_features(s2n, lam, n, d)
    # measured costs on this problem: preconditioning per k, full gradient, one inner step
    t_pre = {}
    rs.rs_precondition(ctx, X, *rs.rs_sketch(ctx, X, 32, 5), lam)          # warm-up
    for k in K_GRID:
        (V, s2k), ts = _timed(lambda: rs.rs_sketch(ctx, X, k, 5))
        (Z, beta, _), tp = _timed(lambda: rs.rs_precondition(ctx, X, V, s2k, lam))
        t_pre[k] = ts + tp
    ep = []
    for m in (n // 4, n):
        _, info = rs.rs_svrg_solve(ctx, Z, y, V, s2k, lam, 3, 1, beta=beta, m=m, eta_mult=1.0)
        ems = info["epoch_ms"]
        ep.append((m, min(ems[1] - ems[0], ems[2] - ems[1])))
    t_step = max(1e-7, (ep[1][1] - ep[0][1]) / (ep[1][0] - ep[0][0]))
    t_fg = max(0.0, ep[1][1] - t_step * ep[1][0])
    # the grid, all in one batched call
    problems = [(X, y, k) for k in K_GRID]
    chains, cfg = [], []
    for pi, k in enumerate(K_GRID):
        for eta in ETA_GRID:
            for r in M_GRID:
                m = max(64, int(round(r * n)))
                chains.append(dict(problem=pi, lam=lam, eta_mult=eta, m=m, seed=spec["seed"] + 2))
                cfg.append((k, eta, m))
    status = "ok"
    while True:
        try:
            _, snaps, _ = rs.rs_solve_batched(ctx, problems, chains, epochs, sketch_seed=spec["seed"] + 3,
                                              snapshots=True)
            break
        except rs.RsError as e:               # a setting diverged: drop the largest remaining step size
            if e.code != rs.RS_ENONFINITE or len({c[1] for c in cfg}) == 1:
                raise
            status = "dropped eta_mult >= %g" % max(c[1] for c in cfg)
            keep = [i for i, c in enumerate(cfg) if c[1] < max(c2[1] for c2 in cfg)]
            chains = [chains[i] for i in keep]
            cfg = [cfg[i] for i in keep]
    times = np.full(len(K_GRID) * len(ETA_GRID) * len(M_GRID), np.inf)
    full_cfg = [(k, eta, max(64, int(round(r * n)))) for k in K_GRID for eta in ETA_GRID for r in M_GRID]
    for c, sn in zip(cfg, snaps):
        rel = ref.rel(sn)
        rel[~np.isfinite(rel)] = np.inf
        e = first_reached(rel)
        if e >= 0:
            times[full_cfg.index(c)] = t_pre[c[0]] + (e + 1) * (t_fg + c[2] * t_step)
    best = int(np.argmin(times))
    k, eta, m = full_cfg[best]
    del X, y, ref
    torch.cuda.empty_cache()
    return dict(features=feat, target=np.array([math.log2(k), math.log(eta), math.log2(m / n)]),
                reached=bool(np.isfinite(times[best])), times=times, t_step=t_step, t_fg=t_fg,
                t_pre=[t_pre[k] for k in K_GRID], trace_c=trc, sigma2=s2n[:64], status=status, **spec)


def generate(ctx, count, seed=0, out=RUNS, log=print, n_range=(16384, 131072), d_choices=(256, 512, 1024, 2048),
             spike_prob=0.0):
    rng = np.random.default_rng(seed)
    recs = []
    t0 = time.time()
    for i in range(count):
        spec = draw_problem(rng, n_range=tuple(n_range), d_choices=tuple(d_choices), spike_prob=spike_prob)
        rec = label_problem(ctx, spec)
        recs.append(rec)
        log(f"[{i + 1}/{count}] n={spec['n']} d={spec['d']} alpha={spec['alpha']:.2f} lam={spec['lam']:.1e} "
            f"reached={rec['reached']} target={np.round(rec['target'], 2)} ({time.time() - t0:.0f} s)")
    keys = ["features", "target", "times", "sigma2"]
    arrs = {k: np.stack([r[k] for r in recs]) for k in keys}
    for k in ("reached", "t_step", "t_fg", "trace_c", "n", "d", "alpha", "lam", "seed", "spike_r", "spike_s"):
        arrs[k] = np.array([r[k] for r in recs])
    arrs["t_pre"] = np.array([r["t_pre"] for r in recs])
    np.savez_compressed(out, **arrs)
    return arrs


# ------------------------------------------------------------------ training

def grid_settings(n):
    return [(k, eta, max(64, int(round(r * n)))) for k in K_GRID for eta in ETA_GRID for r in M_GRID]


def soft_targets(times, n, tol=1.1):
    """Training target of one problem: the mean (log2 k, ln eta_mult, log2(m/n)) over every grid
    setting within `tol` of the fastest.  Neighbouring settings are often within a few percent
    of each other, so the plain argmin is a noisy label; the mean over the near-best set is not."""
    best = np.min(times)
    cfg = grid_settings(n)
    sel = [c for c, t in zip(cfg, times) if t <= tol * best]
    return np.mean([[math.log2(k), math.log(e), math.log2(m / n)] for k, e, m in sel], axis=0)


def merge_runs(paths, out):
    """Concatenate run records; records made before the spiked spectra count as spike_r = 0."""
    parts = [dict(np.load(p)) for p in paths]
    for q in parts:
        q.setdefault("spike_r", np.zeros(len(q["n"]), np.int64))
        q.setdefault("spike_s", np.ones(len(q["n"])))
    keys = [k for k in parts[0] if all(k in q for q in parts)]
    np.savez_compressed(out, **{k: np.concatenate([q[k] for q in parts]) for k in keys})


def train(ctx, runs=RUNS, out=WEIGHTS, steps=4000, lr=2e-3, seed=0, val_frac=0.15, log=print):
    """Adam on soft targets; the checkpoint with the lowest validation loss is kept."""
    D = np.load(runs)
    ok = D["reached"].astype(bool)
    # inputs recomputed from the stored spectra (records made before the inputs were taken relative
    # to the leading value hold the absolute form in "features")
    F = np.stack([network_features(s2, lam, n, d) for s2, lam, n, d in
                  zip(D["sigma2"][ok], D["lam"][ok], D["n"][ok], D["d"][ok])])
    T = np.stack([soft_targets(t, int(n)) for t, n in zip(D["times"][ok], D["n"][ok])])
    rng = np.random.default_rng(seed)
    perm = rng.permutation(len(F))
    nval = max(1, int(round(val_frac * len(F))))
    val, tr = perm[:nval], perm[nval:]
    in_mean, in_std = F[tr].mean(0), np.maximum(F[tr].std(0), 1e-3)
    out_mean, out_std = T[tr].mean(0), np.maximum(T[tr].std(0), 1e-3)
    Fn = torch.from_numpy((F - in_mean) / in_std).float().cuda()
    Tn = torch.from_numpy((T - out_mean) / out_std).float().cuda()
    theta = torch.from_numpy(synth.mlp_init(seed + 1)).float().cuda()
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    tr_t = torch.from_numpy(tr).cuda()
    B = min(64, len(tr))
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    hist = []
    val_t = torch.from_numpy(val).cuda()
    best = (math.inf, 0, theta.clone())
    for t in range(1, steps + 1):
        sel = tr_t[torch.randint(len(tr), (B,), generator=g, device="cuda")]
        lr_t = lr * (0.05 + 0.95 * 0.5 * (1 + math.cos(math.pi * t / steps)))
        _, loss = rs.rs_mlp_train_step(ctx, theta, m, v, Fn[sel].contiguous(), Tn[sel].contiguous(), t, lr=lr_t)
        if t % 50 == 0 or t == steps:
            pv = rs.rs_mlp_forward(ctx, theta, Fn[val_t].contiguous())
            vl = float(((pv - Tn[val_t]) ** 2).sum(1).mean())
            hist.append((t, float(loss.item()), vl))
            if vl < best[0]:
                best = (vl, t, theta.clone())
            if t % 500 == 0:
                log(f"step {t}: train loss {loss.item():.4f}, validation loss {vl:.4f}")
    # the validation loss of always predicting the training mean, for scale
    base = float((Tn[val_t] ** 2).sum(1).mean())
    log(f"kept step {best[1]}: validation loss {best[0]:.4f} (training-mean predictor: {base:.4f})")
    np.savez(out, theta=best[2].cpu().numpy(), in_mean=in_mean, in_std=in_std, out_mean=out_mean, out_std=out_std,
             history=np.array(hist), train_idx=tr, val_idx=val, kept_step=best[1], val_loss=best[0],
             val_loss_mean_predictor=base)
    return hist


def load_weights(path=WEIGHTS, device="cuda"):
    W = np.load(path)
    theta = torch.from_numpy(W["theta"]).float().to(device)
    norm = rs.mlp_norm(W["in_mean"], W["in_std"], W["out_mean"], W["out_std"])
    return theta, norm


# ------------------------------------------------------------------ evaluation

def propose(ctx, X, lam, theta=None, norm=None, seed=0):
    """Rank-64 sketch, tr(C) and rs_propose: ((k, eta_mult, m, fallback), V64, s2_64)."""
    V, s2, trc = features(ctx, X, lam, seed)
    n, d = X.shape
    prop = rs.rs_propose(ctx, s2.cpu().numpy(), lam, n, d, trc, theta=theta, norm=norm)
    return prop, V, s2


def solve_with(ctx, X, y, lam, k, eta_mult, m, V, s2, epochs, seed=1):
    """Precondition with the leading k Ritz pairs of the rank-64 sketch and run SVRG."""
    Vk = V[:, :k].contiguous()
    s2k = s2[:k].contiguous()
    Z, beta, _ = rs.rs_precondition(ctx, X, Vk, s2k, lam)
    _, info = rs.rs_svrg_solve(ctx, Z, y, Vk, s2k, lam, epochs, seed, beta=beta, m=m, eta_mult=eta_mult,
                               snapshots=True)
    return info


def time_to_target(ctx, X, y, lam, ref, mode, theta=None, norm=None, max_steps_mult=64, seed=0):
    """End-to-end time (ms) to relative suboptimality 1e-6 of one setting, or inf."""
    n, d = X.shape
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if mode == "practice":
        V, s2, _ = features(ctx, X, lam, seed)
        k, em, m, fb = 64, 1.0, 2 * n, False
    elif mode == "constant":                 # the training-set mean of the targets, without the network
        V, s2, _ = features(ctx, X, lam, seed)
        om = np.asarray(norm.out_mean, np.float64)
        k, em, m, fb = int(min(64, max(1, round(2.0 ** om[0])))), float(math.exp(om[1])), int(round(n * 2.0 ** om[2])), False
    else:
        (k, em, m, fb), V, s2 = propose(ctx, X, lam, theta if mode == "proposal" else None, norm, seed)
    torch.cuda.synchronize()
    t_setup = (time.perf_counter() - t0) * 1e3
    res = dict(mode=mode, k=k, eta_mult=em, m=m, fallback=fb)
    if m > max_steps_mult * n:                 # one epoch alone exceeds the step budget
        return dict(res, epochs=0, reached_epoch=-1, ms=math.inf, final_rel=math.inf)
    epochs = int(max(1, min(60, max_steps_mult * n // max(m, 1))))
    ta = time.perf_counter()
    info = solve_with(ctx, X, y, lam, k, em, m, V, s2, epochs)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - ta) * 1e3
    rel = ref.rel(info["snapshots"])
    e = first_reached(rel)
    ems = info["epoch_ms"]
    # the precondition step's share: wall time of the solve minus the SVRG epochs
    t_pre = max(0.0, wall - ems[-1])
    t = t_setup + t_pre + ems[e] if e >= 0 else math.inf
    return dict(res, epochs=epochs, reached_epoch=e, ms=t, final_rel=float(rel[-1]))


def evaluate(ctx, count=16, seed=12345, n=131072, d=2048, out=EVAL, weights=WEIGHTS, log=print):
    theta, norm = load_weights(weights)
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(count):
        spec = draw_problem(rng, n_range=(n, n), d_choices=(d,))
        X, y = make_data(spec)
        ref = Reference(X, y, spec["lam"])
        time_to_target(ctx, X, y, spec["lam"], ref, "practice")     # warm-up of this shape
        r = {m: time_to_target(ctx, X, y, spec["lam"], ref, m, theta, norm)
             for m in ("proposal", "theory", "practice", "constant")}
        rows.append(dict(spec=spec, **r))
        log(f"[{i + 1}/{count}] alpha={spec['alpha']:.2f} lam={spec['lam']:.1e}: " +
            ", ".join(f"{m} {r[m]['ms']:.1f} ms (k={r[m]['k']}, eta={r[m]['eta_mult']:.2f}, m={r[m]['m']})"
                      for m in r))
        del X, y, ref
        torch.cuda.empty_cache()
    summ = summarize(rows)
    with open(out, "w") as f:
        json.dump(dict(summary=summ, rows=rows), f, indent=1, default=float)
    return summ


def summarize(rows):
    out = {}
    for mode in ("proposal", "theory", "practice", "constant"):
        t = np.array([r[mode]["ms"] for r in rows])
        out[mode] = dict(reached=int(np.isfinite(t).sum()), median_ms=float(np.median(t[np.isfinite(t)]))
                         if np.isfinite(t).any() else None)
    for other in ("theory", "practice", "constant"):
        both = [(r["proposal"]["ms"], r[other]["ms"]) for r in rows
                if math.isfinite(r["proposal"]["ms"]) and math.isfinite(r[other]["ms"])]
        out[f"speedup_vs_{other}_median"] = float(np.median([b / a for a, b in both])) if both else None
        out[f"proposal_only_reached_vs_{other}"] = sum(1 for r in rows if math.isfinite(r["proposal"]["ms"]) and
                                                       not math.isfinite(r[other]["ms"]))
    out["count"] = len(rows)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["generate", "train", "evaluate", "all", "train+evaluate"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--merge", nargs="*", default=None, help="run files to merge into --runs before training")
    ap.add_argument("--count", type=int, default=160)
    ap.add_argument("--eval-count", type=int, default=16)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--eval-n", type=int, default=131072)
    ap.add_argument("--eval-d", type=int, default=2048)
    ap.add_argument("--runs", default=RUNS)
    ap.add_argument("--weights", default=WEIGHTS)
    ap.add_argument("--eval-out", default=EVAL)
    ap.add_argument("--n-range", type=int, nargs=2, default=[16384, 131072],
                    help="training problems: n log-uniform in this range")
    ap.add_argument("--d-choices", type=int, nargs="+", default=[256, 512, 1024, 2048],
                    help="training problems: d drawn log-uniformly from these")
    ap.add_argument("--spike-prob", type=float, default=0.0,
                    help="training problems: share with a few dominant directions over the power law")
    args = ap.parse_args()
    ctx = rs.Context(0)
    if args.what in ("generate", "all"):
        generate(ctx, args.count, seed=args.seed, out=args.runs, n_range=args.n_range, d_choices=args.d_choices,
                 spike_prob=args.spike_prob)
    if args.merge:
        merge_runs(args.merge, args.runs)
    if args.what in ("train", "all", "train+evaluate"):
        train(ctx, runs=args.runs, out=args.weights, steps=args.steps)
    if args.what in ("evaluate", "all", "train+evaluate"):
        print(json.dumps(evaluate(ctx, args.eval_count, n=args.eval_n, d=args.eval_d, out=args.eval_out,
                                  weights=args.weights), indent=1))


if __name__ == "__main__":
    main()
