"""Benchmark: time to 1e-6 relative suboptimality of sketched-preconditioned SVRG (Alg. 3) on one GB300.

Default workload (the largest single-GPU configuration): n = 2^20, d = 4096, spectrum j^-1.2 with
the leading 20 directions x100 in a random basis, y = X w_gen + 0.05 N(0,1), lambda = 1e-6,
Gaussian sketch of rank k = 256.  One step = one full solve from the device-resident (X, y) to w,
every epoch needed to reach 1e-6 (epochs calibrated once, untimed, against the FP64
normal-equation minimiser).

  chosen form (the reported value): X stored in BF16, BF16 components, snapshot gradients refined
    on the stored data (rs_solve with refine), k = 256, m = 2n, eta = 1/beta_hat;
  plain form (alongside): the same values stored in FP32, FP32 components, same k, m, eta.
  The proposal network's form (rs_solve_proposed) is reported alongside with its epochs to 1e-6.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {rs,reference}]
                  [--workload {bf16_n1048576_d4096,fp32_n65536_d1024,batched}]

Prints one JSON line.  `--impl reference` times the CPU oracle (the slow FP64 reference) on a
bounded sample of the same workload and extrapolates to one plain solve.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

TARGET = 1e-6
METRIC = "time-to-1e-6 rel. suboptimality & data-pass HBM GB/s, chosen vs plain, 1 GB300"
WORKLOAD = "bf16_n1048576_d4096"
SINGLE = ("bf16_n1048576_d4096", "fp32_n65536_d1024")
# epochs of the plain form to 1e-6 (measured by this bench on GB300); the CPU oracle's
# extrapolation to one plain solve uses them
PLAIN_EPOCHS = {"bf16_n1048576_d4096": 4, "fp32_n65536_d1024": 4}
# dram__bytes_read.sum + dram__bytes_write.sum that ncu measured for one launch of the data-pass
# kernel on each workload.  n = 2^20: captured at 262144 + 4096 rows (2.1857 GB, --profile-kernel
# fullgrad) and scaled by the rows to 2^20 + 4096 (the traffic is one read of every row).
DATA_PASS_TRAFFIC = {"bf16_n1048576_d4096": 2.185742e9 * (1048576 + 4096) / (262144 + 4096),
                     "fp32_n65536_d1024": 276.15e6}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _clock_sampler(out_path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(out_path, "w")
        dev = os.environ.get("LOCAL_RANK", "0")
        return subprocess.Popen(["nvidia-smi", "-i", dev, f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                 "-lms", "200"], stdout=f, stderr=subprocess.DEVNULL), f
    except Exception:
        return None, None


def _clock_summary(path):
    try:
        rows = [r.split(",") for r in open(path).read().strip().splitlines() if r.strip()]
    except Exception:
        return None
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
    reasons = set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows:
        if len(r) < 9:
            continue
        for nm, v in zip(names, r[5:9]):
            if "Active" in v and "Not" not in v:
                reasons.add(nm)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": sorted(reasons), "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        return dist, rank, ws
    return None, rank, ws


def max_over_ranks(dist, value):
    """Largest value over all ranks (the slowest replica sets the time)."""
    if dist is None:
        return value
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _load_proposal(rs):
    """Trained proposal weights (committed with the package), or (None, None) = theory setting."""
    path = os.path.join(ROOT, "paper_1602_02350_gb300", "proposal_weights.npz")
    if not os.path.exists(path):
        return None, None
    W = np.load(path)
    theta = torch.from_numpy(W["theta"]).float().cuda()
    return theta, rs.mlp_norm(W["in_mean"], W["in_std"], W["out_mean"], W["out_std"])


def _time_steps(step, steps, stream):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        out = step()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, out


def _workload_text(name):
    return {"bf16_n1048576_d4096": "bf16_n1048576_d4096: n=2^20 d=4096, spectrum j^-1.2 (x100 for j<=20), "
                                   "lambda=1e-6, Gaussian sketch k=256",
            "fp32_n65536_d1024": "fp32_n65536_d1024: n=65536 d=1024 fp32 data, spectrum j^-2, lambda=1e-5, "
                                 "CountSketch s=4096 -> Gaussian sketch k=64"}[name]


def run_rs(args):
    import paper_1602_02350_gb300 as rs
    from paper_1602_02350_gb300 import synth

    dist, rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    name = args.workload
    cfg = synth.CONFIGS[name]
    n, d, k, lam = cfg.n, cfg.d, cfg.k, cfg.lam
    big = name == "bf16_n1048576_d4096"
    if big:
        # one set of values, stored twice: BF16 for the chosen form, the same values in FP32 for the plain one
        Xc, y64, _ = synth.config_problem(cfg, device="cuda", dtype=torch.bfloat16)
        Xp = Xc.float()
    else:
        Xp, y64, _ = synth.config_problem(cfg, device="cuda", dtype=torch.float32)
        Xc = Xp
    y = y64.float().contiguous()
    del y64
    stream = torch.cuda.current_stream()
    ctx = rs.Context(local, stream)
    theta, norm = _load_proposal(rs)
    sk = dict(kind=cfg.kind, s=cfg.s)
    m_plain, em_plain = 2 * n, 1.0

    def plain(epochs, snapshots=False, X=Xp):
        return rs.rs_solve(ctx, X, y, k, lam, epochs, cfg.seed_sketch, cfg.seed_svrg, m=m_plain, eta_mult=em_plain,
                           snapshots=snapshots, **sk)

    def proposed(epochs, snapshots=False, X=Xc, yy=y, w_out=None):
        return rs.rs_solve_proposed(ctx, X, yy, lam, epochs, cfg.seed_sketch, cfg.seed_svrg, theta=theta, norm=norm,
                                    z_dtype=torch.bfloat16, snapshots=snapshots, w_out=w_out, **sk)

    if big:
        # the configured rank k; the network proposes eta and m from the first 64 Ritz values of the
        # rank-k sketch (rs_solve_proposed with a fixed rank), unless it falls back, when the chosen
        # form keeps the plain form's eta and m
        probe = rs.rs_solve_proposed(ctx, Xc, y, lam, 0, cfg.seed_sketch, cfg.seed_svrg, theta=theta, norm=norm,
                                     k_fixed=k, **sk)[1] if theta is not None else {"fallback": True}
        if not probe["fallback"]:
            def chosen(epochs, snapshots=False, X=Xc, yy=y, w_out=None):
                return rs.rs_solve_proposed(ctx, X, yy, lam, epochs, cfg.seed_sketch, cfg.seed_svrg, theta=theta,
                                            norm=norm, snapshots=snapshots, w_out=w_out, k_fixed=k, **sk)
            chosen_text = {"components": "bf16 from the bf16 data, snapshot gradients refined on the stored data",
                           "k": k, "eta_mult": probe["eta_mult"], "m": probe["m"],
                           "proposal": "network (eta, m) at the configured rank k"}
        else:
            def chosen(epochs, snapshots=False, X=Xc, yy=y, w_out=None):
                return rs.rs_solve(ctx, X, yy, k, lam, epochs, cfg.seed_sketch, cfg.seed_svrg, m=m_plain,
                                   eta_mult=em_plain, snapshots=snapshots, refine=True, w_out=w_out, **sk)
            chosen_text = {"components": "bf16 from the bf16 data, snapshot gradients refined on the stored data",
                           "k": k, "eta_mult": em_plain, "m": m_plain,
                           "proposal": "plain eta and m (the network falls back on this problem)"}
    else:
        chosen = proposed
        chosen_text = {"components": "bf16, snapshot gradients refined on the fp32 data",
                       "proposal": "network" if theta is not None else "theory setting (no weights)"}

    # launch layouts of the inner loop and the full-gradient pass for each storage type the two forms
    # use (cluster size, threads, ring stages), timed once by the library's autotuner on this
    # problem's components and kept in the context for every later call (untimed set-up)
    tuned = {}
    if not args.no_autotune:
        for X_, zt, label in ((Xc, torch.bfloat16, "bf16"), (Xp, torch.float32, "fp32")):
            V_, s2_ = rs.rs_sketch(ctx, X_, k, cfg.seed_sketch, **sk)
            Z_, _, _ = rs.rs_precondition(ctx, X_, V_, s2_, lam, z_dtype=zt)
            tuned[label] = rs.rs_autotune(ctx, Z_, n)
            del V_, s2_, Z_
        torch.cuda.empty_cache()

    if args.profile:
        # profiling run: each form twice (the first is the warm-up) with fixed epoch counts, nothing else
        for _ in range(2):
            plain(args.plain_epochs)
            chosen(args.chosen_epochs)
        torch.cuda.synchronize()
        ctx.close()
        return

    # reference minimiser for the accuracy target (normal equations in double; measurement only, untimed)
    ref = _Reference(Xc, y, lam)

    def first_epoch(snaps, cap):
        hist = ref.rel(snaps)
        reach = [i for i, r in enumerate(hist) if r <= TARGET]
        return ((reach[0] + 1) if reach else cap), [float(f"{h:.3e}") for h in hist]

    cap = args.cap_epochs
    _, info = plain(cap, snapshots=True)
    ep_plain, hist_plain = first_epoch(info["snapshots"], cap)
    del info
    _, cinfo = chosen(cap, snapshots=True)
    ep_chosen, hist_chosen = first_epoch(cinfo["snapshots"], cap)
    if not big:
        chosen_text.update(k=cinfo["k"], eta_mult=cinfo["eta_mult"], m=cinfo["m"], fallback=cinfo["fallback"])
    m_ch = cinfo.get("m", m_plain)
    ems = cinfo["epoch_ms"]
    del cinfo
    prop_text = None
    if big:
        # the proposal network's form alongside (epochs to 1e-6 from its snapshots, not timed)
        _, pinfo = proposed(cap, snapshots=True)
        ep_p, hist_p = first_epoch(pinfo["snapshots"], cap)
        prop_text = {"k": pinfo["k"], "eta_mult": pinfo["eta_mult"], "m": pinfo["m"], "fallback": pinfo["fallback"],
                     "epochs_to_1e-6": ep_p if min(hist_p) <= TARGET else None,
                     "epoch_ms_cumulative": [round(e, 2) for e in pinfo["epoch_ms"][:ep_p]]}
        del pinfo
    fp8_text = None
    if big:
        # the FP8-e4m3 variant of the precision configuration: components as FP8 codes with per-row
        # scales, snapshot gradients refined on the BF16 data, the chosen form's k, eta and m; its
        # time to 1e-6 is measured like the chosen form's (warm, events), outside the headline
        def fp8(epochs, snapshots=False):
            V8, s28 = rs.rs_sketch(ctx, Xc, k, cfg.seed_sketch, **sk)
            Z8, b8, _ = rs.rs_precondition(ctx, Xc, V8, s28, lam, z_dtype=torch.float8_e4m3fn)
            return rs.rs_svrg_solve(ctx, Z8, y, V8, s28, lam, epochs, cfg.seed_svrg, beta=b8, m=m_ch,
                                    eta_mult=chosen_text["eta_mult"], X=Xc, refine=True, snapshots=snapshots)
        try:
            _, finfo = fp8(cap, snapshots=True)
            ep8, hist8 = first_epoch(finfo["snapshots"], cap)
            del finfo
            if min(hist8) <= TARGET:
                ms8, _ = _event_ms(lambda: fp8(ep8), stream)
                fp8_text = {"components": "fp8-e4m3 codes with per-row scales from the bf16 data, refined",
                            "k": k, "eta_mult": chosen_text["eta_mult"], "m": m_ch, "epochs": ep8,
                            "seconds": ms8 / 1e3, "rel_subopt_per_epoch": hist8[:ep8]}
            else:
                fp8_text = {"epochs": None, "rel_subopt_per_epoch": hist8}
        except rs.RsError as e:
            fp8_text = {"unavailable": str(e)[:160]}
    torch.cuda.empty_cache()

    def plain_step():
        return plain(ep_plain)[0]

    def chosen_step():
        return chosen(ep_chosen)[0]

    for _ in range(args.warmup):
        plain_step()
        chosen_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # raw nvidia-smi samples of the timed region (summarised in the JSON line); RS_CLOCKS_DIR keeps them
    cdir = os.environ.get("RS_CLOCKS_DIR") or tempfile.gettempdir()
    cpath = os.path.join(cdir, f"clocks_rank{rank}.csv")
    os.makedirs(cdir, exist_ok=True)
    sampler, fh = _clock_sampler(cpath)
    time.sleep(0.3)
    ms_plain, w_plain = _time_steps(plain_step, args.steps, stream)
    l0 = ctx.launches
    ms, w = _time_steps(chosen_step, args.steps, stream)
    launches = (ctx.launches - l0) // max(1, args.steps)
    if sampler:
        sampler.terminate()
        sampler.wait()
        fh.close()
    final_rel, final_rel_plain = float(ref.rel(w)[0]), float(ref.rel(w_plain)[0])
    ms = max_over_ranks(dist, ms)
    ms_plain = max_over_ranks(dist, ms_plain)

    # end to end through the public call with host buffers (pinned), copies inside the timed region
    Xh = Xc.cpu().pin_memory()
    yh = y.cpu().pin_memory()
    wh = torch.empty(d, dtype=torch.float32).pin_memory()
    chosen(ep_chosen, X=Xh, yy=yh, w_out=wh)
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 5 if big else args.steps))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        chosen(ep_chosen, X=Xh, yy=yh, w_out=wh)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(dist, (time.perf_counter() - t0) / e2e_steps)
    e2e_ok = float(ref.rel(wh.cuda())[0])
    del Xh

    # dominant data pass: the full-gradient stream over the n + d component rows of the chosen form's
    # storage type, timed alone with events on the library's stream
    zt = torch.bfloat16 if big else torch.float32
    t_sk, (V, s2) = _event_ms(lambda: rs.rs_sketch(ctx, Xc, k, cfg.seed_sketch, **sk), stream)
    t_pc, (Z, beta, bh) = _event_ms(lambda: rs.rs_precondition(ctx, Xc, V, s2, lam, z_dtype=zt), stream)
    # speed-up diagnostic (ratio after Thm 1) from this sketch and tr(C)
    trc = rs.rs_trace_c(ctx, Xc)
    rat, rat_acc = rs.rs_speedup_ratio(ctx, s2, trc)
    rat, rat_acc = rat.cpu().numpy(), rat_acc.cpu().numpy()
    ratio = {"k": k, "ratio": float(rat[k - 1]), "accelerated": float(rat_acc[k - 1]), "trace_c": trc,
             "ratio_at_k": {str(kk): float(rat[kk - 1]) for kk in (1, 8, 16, 32, 64, 128, 256) if kk <= k}}
    wt = torch.zeros(d, dtype=torch.float32, device="cuda")
    for _ in range(3):
        rs.rs_full_gradient(ctx, Z, y, n, lam, wt)
    fg_ms, _ = _time_steps(lambda: rs.rs_full_gradient(ctx, Z, y, n, lam, wt), 10 if big else 20, stream)
    esz = Z.element_size()
    fg_bytes = (n + d) * d * esz + n * 4          # algorithmic: every component row and label read once
    peak, peak_kind = _peaks()
    achieved = fg_bytes / (fg_ms * 1e-3) / 1e9
    del Z, beta
    # tensor-core contractions of the chosen form's sketch and preconditioner (FLOP per call: the
    # range sketch X^T Pi and X Q of Rayleigh-Ritz, 2 n d k each; X V and (X V) V^T, 2 n d k each)
    tf_peak, tf_kind = _peak_tflops()
    tens = {"sketch": {"flop": 4.0 * n * d * k, "ms": t_sk}, "precondition": {"flop": 4.0 * n * d * k, "ms": t_pc}}
    for v in tens.values():
        v["tflops"] = v["flop"] / (v["ms"] * 1e-3) / 1e12
        v["frac_of_bf16_peak"] = v["tflops"] / tf_peak
    tens["peak_tflops"], tens["peak_kind"] = tf_peak, tf_kind

    per_epoch = (ems[-1] - ems[0]) / max(1, len(ems) - 1) if len(ems) > 1 else (ems[0] if ems else None)
    xb = Xc.element_size() * n * d
    out = {
        "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16+f32", "data": "synthetic",
        "config": {"workload": _workload_text(name),
                   "chosen": dict(chosen_text, epochs=ep_chosen, rel_subopt_per_epoch=hist_chosen[:ep_chosen],
                                  final_rel_subopt=final_rel),
                   "plain": {"components": "fp32", "k": k, "eta_mult": em_plain, "m": m_plain, "epochs": ep_plain,
                             "seconds": ms_plain / 1e3, "final_rel_subopt": final_rel_plain,
                             "rel_subopt_per_epoch": hist_plain[:ep_plain]},
                   "speedup_chosen_vs_plain": ms_plain / ms,
                   "n": n, "d": d, "k": k, "lambda": lam, "parallelism": f"replicas x{ws}",
                   "autotune": {lab: {key: (round(v, 4) if isinstance(v, float) else v) for key, v in r.items()}
                                for lab, r in tuned.items()},
                   "l2": f"inputs exceed L2 (X {xb / 1e9:.2f} GB vs 129 MB L2); no flush"},
        "roofline": {"kernel": f"full-gradient data pass over the n+d component rows ({'bf16' if big else 'fp32'})",
                     "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "traffic": DATA_PASS_TRAFFIC.get(name), "traffic_unit": "B per launch",
                     "algorithmic_bytes": fg_bytes, "ms_per_launch": fg_ms},
        "tensor": tens,
        "speedup_ratio": ratio,
        "inner_loop": {"ms_per_epoch": per_epoch, "m": m_ch,
                       "ns_per_step": per_epoch * 1e6 / m_ch if per_epoch else None,
                       "steps_per_s": m_ch / (per_epoch * 1e-3) if per_epoch else None},
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": xb + n * 4, "d2h_bytes_per_step": d * 4,
                "final_rel_subopt": e2e_ok},
        "gpu_launches": launches,
        "clocks": _clock_summary(cpath),
    }
    if prop_text is not None:
        out["config"]["proposal_form"] = prop_text
    if fp8_text is not None:
        out["config"]["fp8_form"] = fp8_text
    if rank == 0:
        out["cpu_baseline"] = (cpu_baseline_sample(name, budget_s=args.cpu_budget, epochs=ep_plain)
                               if args.cpu_budget > 0 else None)
        print(json.dumps(out))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    ctx.close()


def _event_ms(fn, stream):
    """(ms, result) of one call timed with events on ``stream`` (after one untimed call)."""
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    out = fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b), out


def _peak_tflops():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (bf16 burst)"
    return 1900.0, "fallback"


def _normal_equations(X, y):
    """X^T X and X^T y accumulated in double on the device in row chunks (measurement only)."""
    n, d = X.shape
    G = torch.zeros(d, d, dtype=torch.float64, device=X.device)
    b = torch.zeros(d, dtype=torch.float64, device=X.device)
    for r0 in range(0, n, 16384):
        Xb = X[r0:r0 + 16384].double()
        G += Xb.T @ Xb
        b += Xb.T @ y[r0:r0 + 16384].double()
        del Xb
    return G, b


class _Reference:
    """w* of Eq. (1) from the normal equations accumulated in double on the device in row chunks
    (measurement only, untimed), and relative suboptimality of iterates through e^T H e / 2."""

    def __init__(self, X, y, lam, normal=None):
        n, d = X.shape
        G, b = normal if normal is not None else _normal_equations(X, y)
        self.H = G / n + lam * torch.eye(d, dtype=torch.float64, device=X.device)
        self.w = torch.from_numpy(np.linalg.solve(self.H.cpu().numpy(), (b / n).cpu().numpy())).to(X.device)
        r = torch.zeros((), dtype=torch.float64, device=X.device)
        for r0 in range(0, n, 16384):
            e = X[r0:r0 + 16384].double() @ self.w - y[r0:r0 + 16384].double()
            r += e @ e
        self.L = float(0.5 * r / n + 0.5 * lam * (self.w @ self.w))

    def rel(self, W):
        E = W.double().reshape(-1, self.w.shape[0]) - self.w
        return (0.5 * ((E @ self.H) * E).sum(1) / self.L).cpu().numpy()


def run_batched(args):
    """Batching workload (one GPU): 64 BF16 problems (n uniform in [8192, 262144], d in {256, 512,
    1024, 2048}, spectrum j^-alpha with alpha ~ U[1, 2.5]), each at the 8 lambda 10^(-3-4j/7) with
    one sketch of rank d/16 per problem, solved in one rs_solve_batched call (epochs 2..S in one
    CUDA graph), eta = 1.5 / beta^, m = n / 4.  Reports the batch's time, aggregate inner steps/s
    and how many of the 512 chains reached 1e-6 (against FP64 normal-equation solutions)."""
    import paper_1602_02350_gb300 as rs
    from paper_1602_02350_gb300 import synth
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = rs.Context(local, stream)
    rng = np.random.default_rng(4004)
    nprob = args.batch_problems
    lams = [10.0 ** (-3 - 4 * j / 7) for j in range(8)]
    probs, specs = [], []
    for p in range(nprob):
        n = int(rng.integers(8192 // 64, 262144 // 64 + 1)) * 64
        d = int(rng.choice([256, 512, 1024, 2048]))
        alpha = float(rng.uniform(1.0, 2.5))
        X, y, _ = synth.problem(n, d, np.arange(1, d + 1, dtype=np.float64) ** -alpha, 0.05, 5000 + p,
                                device="cuda", dtype=torch.bfloat16)
        probs.append((X, y.float().contiguous(), 0))
        specs.append((n, d, alpha))
    chains = [dict(problem=p, lam=lam, eta_mult=1.5, m=specs[p][0] // 4, seed=p) for p in range(nprob) for lam in lams]
    S = args.batch_epochs
    steps = sum(c["m"] for c in chains) * S
    rs.rs_solve_batched(ctx, probs, chains[:8], 2, sketch_seed=7)          # warm-up of the code paths
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ws, snaps, ems = rs.rs_solve_batched(ctx, probs, chains, S, sketch_seed=7, snapshots=True)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    reached, first, missed = 0, [], []
    for p in range(nprob):
        X, y, _ = probs[p]
        ne = _normal_equations(X, y)
        ref_p = [_Reference(X, y, lam, ne) for lam in lams]
        for j in range(8):
            rel = ref_p[j].rel(snaps[p * 8 + j])
            hit = [i for i, r in enumerate(rel) if r <= TARGET]
            if hit:
                reached += 1
                first.append(hit[0] + 1)
            else:
                # kappa^ = tr(H) / lambda_min(H) of the unpreconditioned problem (Eq. (3)), for context
                H = ref_p[j].H.cpu().numpy()   # host eigensolve (measurement only)
                kap = float(np.trace(H) / np.linalg.eigvalsh(H)[0])
                n_, d_, a_ = specs[p]
                missed.append({"problem": p, "n": n_, "d": d_, "alpha": round(a_, 3), "lambda": lams[j],
                               "m": chains[p * 8 + j]["m"], "final_rel_subopt": float(f"{rel[-1]:.3e}"),
                               "kappa_hat": float(f"{kap:.3e}")})
        del ref_p
    out = {"metric": "batched solve time (64 problems x 8 lambda, one graph)", "value": secs, "unit": "s",
           "n_gpus": 1, "steps": 1, "warmup": 1, "higher_is_better": False, "dtype": "bf16+f32",
           "data": "synthetic",
           "config": {"workload": f"{nprob} bf16 problems x 8 lambda, k=d/16, eta=1.5/beta^, m=n/4, {S} epochs",
                      "chains": len(chains), "inner_steps": steps, "inner_steps_per_s": steps / secs,
                      "epoch_ms_cumulative": ems, "chains_reaching_1e-6": reached, "chains_not_reaching": missed,
                      "median_epochs_to_1e-6": float(np.median(first)) if first else None,
                      "data_bytes": int(sum(X.numel() * 2 for X, _, _ in probs))}}
    print(json.dumps(out))
    ctx.close()


def run_fig2(args):
    """Sec. 6's synthetic comparison (Fig. 2 a, b): singular values q^-1 and q^-2, unit-norm examples,
    lambda = 1e-8, SVRG (k = 1, i.e. M = I) against sketched-preconditioned SVRG with k = 30, m = n, the
    step size tuned per method over a grid (lowest suboptimality after the last epoch), 30 epochs; in
    FP32 at n = 16384, d = 4096 (the paper's 4:1 shape at the widest d the inner loop takes) and in
    FP64 at n = 4096, d = 1024 (FP32 rounding of the components sets a floor near 1e-5 relative at
    lambda = 1e-8).  Prints one JSON line with the suboptimality L(w_t) - L* per epoch of each method
    next to the paper's values."""
    import paper_1602_02350_gb300 as rs
    from paper_1602_02350_gb300 import synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ctx = rs.Context(int(os.environ.get("LOCAL_RANK", "0")), torch.cuda.current_stream())
    lam, E = 1e-8, 30
    grid = (0.25, 0.5, 1.0, 2.0, 4.0, 8.0)
    # the paper's curves (Fig. 2 a, b: 5000 x 20000), epochs 1, 5, 10, 15, 20 where printed
    paper = {1: {"SVRG": {1: 5.38e-2, 5: 2.63e-3, 10: 1.99e-3, 15: 1.74e-3, 20: 1.59e-3},
                 "SCSVRG-k=30": {1: 7.32e-2, 5: 1.87e-3, 10: 9.48e-4, 15: 6.50e-4, 20: 4.86e-4}},
             2: {"SVRG": {1: 6.13e-2, 5: 7.43e-5, 10: 4.74e-5, 15: 4.00e-5, 20: 3.61e-5},
                 "SCSVRG-k=30": {1: 7.03e-2, 5: 4.69e-5, 10: 5.46e-6, 15: 1.08e-6, 20: 3.29e-7}}}
    out = {}
    cases = [(args.fig2_n, args.fig2_d, torch.float32, decay) for decay in (1, 2)] + \
            [(4096, 1024, torch.float64, decay) for decay in (1, 2)]
    for n, d, dt, decay in cases:
        X, y64, _ = synth.spectrum_problem(n, d, decay, 0.1, 6000 + decay, dtype=dt)
        y = y64.to(dt).contiguous()
        ref = _Reference(X, y, lam)
        res = {}
        for name, k in (("SVRG", 1), ("SCSVRG-k=30", 30)):
            V, s2 = rs.rs_sketch(ctx, X, k, 7000 + decay)
            Z, beta, _ = rs.rs_precondition(ctx, X, V, s2, lam)
            best = None
            for em in grid:
                try:
                    _, info = rs.rs_svrg_solve(ctx, Z, y, V, s2, lam, E, 8000 + decay, beta=beta, m=n, eta_mult=em,
                                               snapshots=True)
                except rs.RsError:
                    continue                           # this step size diverged
                sub = ref.rel(info["snapshots"]) * ref.L
                if np.all(np.isfinite(sub)) and (best is None or sub[-1] < best[1][-1]):
                    best = (em, sub, info["epoch_ms"][-1])
            em, sub, ms = best
            res[name] = {"eta_mult": em, "ms_30_epochs": ms,
                         "suboptimality": [float(f"{v:.3e}") for v in sub]}
            del Z, beta
        r = {e: res["SVRG"]["suboptimality"][e - 1] / res["SCSVRG-k=30"]["suboptimality"][e - 1] for e in (5, 10, 20, 30)}
        pr = {e: paper[decay]["SVRG"][e] / paper[decay]["SCSVRG-k=30"][e] for e in (5, 10, 20)}
        out[f"{'fp64' if dt == torch.float64 else 'fp32'}_n{n}_d{d}_decay_{decay}"] = dict(
            res, svrg_over_scsvrg=r, paper_svrg_over_scsvrg=pr, paper=paper[decay], L_star=ref.L)
        del X, y, ref
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "suboptimality per epoch, SVRG vs sketched-preconditioned SVRG (Sec. 6, Fig. 2 a, b)",
                      "unit": "L(w_t) - L*", "n_gpus": 1, "data": "synthetic",
                      "config": {"workload": "singular values q^-1 / q^-2, unit-norm rows, lambda=1e-8, k=30, m=n, "
                                             f"eta tuned over {list(grid)} / beta^, {E} epochs; fp32 n={args.fig2_n} "
                                             f"d={args.fig2_d} and fp64 n=4096 d=1024"},
                      "results": out}))
    ctx.close()


def run_krylov(args):
    """Alg. 2 with q = 1, 2, 3 Krylov blocks (k = 64) on the n = 65536, d = 1024 FP32 workload and the
    n = 2^20, d = 4096 BF16 workload: the average condition number kappa^ = tr(H) / lambda_min(H) of the
    preconditioned Hessian H = M (C + lambda I) M (Eq. (3); measured from the double normal equations),
    the sketch time, and the time to relative suboptimality 1e-6 of the solve (m = 2n, eta = 1/beta^)."""
    import paper_1602_02350_gb300 as rs
    from paper_1602_02350_gb300 import synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    ctx = rs.Context(int(os.environ.get("LOCAL_RANK", "0")), stream)
    out = {}
    for name in ("fp32_n65536_d1024", "bf16_n1048576_d4096"):
        cfg = synth.CONFIGS[name]
        dt = torch.bfloat16 if name.startswith("bf16") else torch.float32
        X, y64, _ = synth.config_problem(cfg, device="cuda", dtype=dt)
        y = y64.float().contiguous()
        del y64
        n, d, lam, k = cfg.n, cfg.d, cfg.lam, 64
        ref = _Reference(X, y, lam)
        rows = {}
        for q in (1, 2, 3):
            sk = dict(kind=cfg.kind, s=cfg.s) if q == 1 else dict(kind="gaussian")
            t_sk, (V, s2) = _event_ms(lambda: rs.rs_sketch(ctx, X, k, cfg.seed_sketch, q=q, **sk), stream)
            Vd = V.double()
            a = 1.0 - torch.sqrt((s2[-1] + lam) / (s2 + lam))
            M = torch.eye(d, dtype=torch.float64, device="cuda") - (Vd * a[None, :]) @ Vd.T
            H = M @ ref.H @ M
            ev = torch.linalg.eigvalsh(H)
            kappa_hat = float(torch.trace(H) / ev[0])
            cap = 20
            _, info = rs.rs_solve(ctx, X, y, k, lam, cap, cfg.seed_sketch, cfg.seed_svrg, q=q, m=2 * n, eta_mult=1.0,
                                  snapshots=True, refine=dt == torch.bfloat16, **sk)
            rel = ref.rel(info["snapshots"])
            hit = [i for i, r in enumerate(rel) if r <= TARGET]
            e = hit[0] + 1 if hit else None
            secs = None
            if e:
                ms, _ = _event_ms(lambda: rs.rs_solve(ctx, X, y, k, lam, e, cfg.seed_sketch, cfg.seed_svrg, q=q,
                                                      m=2 * n, eta_mult=1.0, refine=dt == torch.bfloat16, **sk),
                                  stream)
                secs = ms / 1e3
            rows[f"q={q}"] = {"kappa_hat": kappa_hat, "sketch_ms": t_sk, "epochs_to_1e-6": e, "seconds_to_1e-6": secs,
                              "sigma2_k": float(s2[-1]), "rel_subopt_per_epoch": [float(f"{r:.3e}") for r in rel[:e or cap]]}
            del M, H
        kap_exact = None
        ev_c = torch.linalg.eigvalsh(ref.H)
        kap_exact = float(torch.trace(ref.H) / ev_c[0])
        out[name] = {"k": k, "kappa_hat_unpreconditioned": kap_exact, "by_q": rows}
        del X, y, ref
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "kappa^ of the preconditioned problem and time to 1e-6 vs Krylov blocks q (Alg. 2)",
                      "n_gpus": 1, "data": "synthetic", "results": out}))
    ctx.close()


def run_profile_kernel(args):
    """Small cases of the top kernels for ncu captures (inputs above L2, a few GB at most): each call
    below is made two or three times, so `ncu -k <kernel> -s <warm-up launches> -c 1` captures a warm
    launch.  chain: one inner-loop epoch, bf16 components, n = 16384, d = 4096, m = 16384;
    fullgrad: the full-gradient pass over bf16 components, n = 262144, d = 4096; sketch: the range
    sketch X^T Pi, bf16 X 262144 x 4096, k = 256; resid: the components Z = X - P V^T, same X, k = 256."""
    import paper_1602_02350_gb300 as rs
    from paper_1602_02350_gb300 import synth
    ctx = rs.Context(0)
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    which = args.profile_kernel
    if which == "chain":
        n, d, m = 16384, 4096, 16384
        Z = (torch.randn(n + d, d, device="cuda", generator=g) / 64).to(torch.bfloat16)
        idx = torch.randint(0, n + d, (m,), device="cuda", dtype=torch.int32, generator=g)
        inq = torch.rand(m, device="cuda", generator=g) + 0.5
        w = torch.zeros(d, device="cuda")
        mu = torch.randn(d, device="cuda", generator=g) * 1e-3
        if not args.no_autotune:
            rs.rs_autotune(ctx, Z, n)   # the layout the benchmark's solves use for bf16 rows at this d
        for _ in range(2):
            rs.rs_svrg_epoch(ctx, Z, n, 1e-3, idx, inq, 0.1, w, mu, True)
    elif which == "fullgrad":
        n, d = 262144, 4096
        Z = (torch.randn(n + d, d, device="cuda", generator=g) / 64).to(torch.bfloat16)
        y = torch.randn(n, device="cuda", generator=g)
        w = torch.randn(d, device="cuda", generator=g) * 0.01
        for _ in range(3):
            rs.rs_full_gradient(ctx, Z, y, n, 1e-3, w)
    elif which in ("sketch", "resid"):
        n, d, k = 262144, 4096, 256
        X = torch.randn(n, d, device="cuda", generator=g).to(torch.bfloat16)
        if which == "sketch":
            for _ in range(2):
                rs.rs_range_sketch(ctx, X, k, 7)
        else:
            V = torch.from_numpy(synth.random_orthonormal(d, k, 3)).float().cuda()
            s2 = torch.from_numpy(synth.random_sigma2(k, 4)).cuda()
            for _ in range(2):
                rs.rs_precondition(ctx, X, V, s2, 1e-4)
    torch.cuda.synchronize()
    ctx.close()
    print(json.dumps({"profile_kernel": which, "ok": True}))


def cpu_baseline_sample(name=WORKLOAD, budget_s=20.0, epochs=None, _cache={}):
    """Time the FP64 oracle on host cores on a bounded sample of the workload and extrapolate to one
    plain solve: (sketch + precondition) once, plus epochs x (full gradient + m steps).

    At n = 65536 the oracle runs the passes on the whole data; at n = 2^20 it runs them on the first
    n_s = 16384 rows of the same distribution (d, k, lambda and spectrum unchanged) and the pass times
    are scaled by n / n_s (they are linear in n).  The sequential inner loop is timed for a bounded
    number of steps at the full d and scaled to m = 2n steps per epoch."""
    from oracle import precond, sketch, streams, svrg
    from paper_1602_02350_gb300 import synth
    cfg = synth.CONFIGS[name]
    n, d, lam = cfg.n, cfg.d, cfg.lam
    ns = min(n, 16384) if n > 65536 else n
    if name not in _cache:
        X, y, _ = synth.problem(ns, d, cfg.spectrum(), cfg.noise, cfg.seed_data, dtype=torch.float64)
        _cache[name] = (X.numpy(), y.numpy())
    Xn, yn = _cache[name]
    m = 2 * n
    epochs = epochs or PLAIN_EPOCHS[name]
    scale = n / ns
    t0 = time.perf_counter()
    V, s2 = sketch.block_lanczos(Xn, cfg.k, cfg.seed_sketch, kind=cfg.kind, s=cfg.s)
    M = precond.m_matrix(V, s2, lam)
    Z, yz, g = precond.components(*precond.transform(Xn, M), yn, lam)
    beta = precond.smoothness(Z, g)
    t_prep = time.perf_counter() - t0
    t1 = time.perf_counter()
    wbar = np.zeros(d)
    mu = svrg.full_gradient_fast(Z, yz, g, wbar)
    t_fg = time.perf_counter() - t1
    W, cum, q = svrg.sampling_table(beta)
    per_step_guess = 10e-6 * max(1.0, d / 1024)
    steps = int(min(m, max(2000, (budget_s - t_prep - t_fg) / per_step_guess)))
    idx = streams.sample_indices(cum, cfg.seed_svrg, 0, steps)
    t2 = time.perf_counter()
    svrg.epoch(Z, yz, g, wbar, idx, q, 1.0 / precond.beta_hat(beta), v_bar=mu)
    t_step = (time.perf_counter() - t2) / steps
    total = scale * t_prep + epochs * (scale * t_fg + m * t_step)
    rows = f"the first {ns} rows (pass times x{scale:g})" if ns < n else f"all {n} rows"
    return {"value": total, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"sketch+precondition once ({t_prep:.1f} s) and one full-gradient pass ({t_fg:.2f} s) on {rows}, "
                      f"{steps} inner steps at d={d} ({t_step * 1e6:.1f} us/step) of the {name} workload, "
                      f"extrapolated to {epochs} epochs of m={m}; numpy BLAS threads for the dense steps, "
                      f"one thread for the sequential inner loop"}


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, on host cores, same workload, metric and unit."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    name = args.workload if args.workload in SINGLE else WORKLOAD
    vals = []
    cb = None
    # a bounded sample per step, sized so that the whole run stays within a few minutes
    per_step = args.cpu_budget if args.cpu_budget > 0 else 15.0
    per_step = min(per_step, max(3.0, 150.0 / max(1, args.steps)))
    for _ in range(args.steps):
        cb = cpu_baseline_sample(name, budget_s=per_step)
        vals.append(cb["value"])
    v = statistics.mean(vals)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s",
           "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": _workload_text(name) + " (oracle on a bounded sample, extrapolated to one "
                                                       "plain solve: see cpu_baseline.sample)",
                      "parallelism": "cpu"},
           "cpu_baseline": cb, "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="rs", choices=["rs", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=15.0,
                    help="seconds of oracle work for the cpu_baseline sample (0 = skip)")
    ap.add_argument("--profile", action="store_true",
                    help="run two solves of each form with the given epoch counts and exit (for ncu launch lists)")
    ap.add_argument("--plain-epochs", type=int, default=4)
    ap.add_argument("--chosen-epochs", type=int, default=4)
    ap.add_argument("--cap-epochs", type=int, default=30, help="epoch cap of the untimed calibration runs")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the autotuner step before timing (the library's default launch layouts)")
    ap.add_argument("--profile-kernel", choices=["chain", "fullgrad", "sketch", "resid"], default=None,
                    help="run a small case of one kernel (for an ncu capture) and exit")
    ap.add_argument("--fig2-n", type=int, default=16384)
    ap.add_argument("--fig2-d", type=int, default=4096)
    ap.add_argument("--workload", default=WORKLOAD, choices=list(SINGLE) + ["batched", "fig2", "krylov"],
                    help="bf16_n1048576_d4096 (default): n=2^20, d=4096; fp32_n65536_d1024: n=65536, d=1024; "
                         "batched: 64 problems x 8 lambda (each its own JSON line)")
    ap.add_argument("--batch-problems", type=int, default=64)
    ap.add_argument("--batch-epochs", type=int, default=20)
    args = ap.parse_args()
    if args.profile_kernel:
        run_profile_kernel(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "fig2":
        run_fig2(args)
    elif args.workload == "krylov":
        run_krylov(args)
    else:
        run_rs(args)


if __name__ == "__main__":
    main()
