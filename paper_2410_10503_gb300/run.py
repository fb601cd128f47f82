"""Command-line runs of the motion-compensated reconstruction with a per-epoch
JSONL log.

    python -m paper_2410_10503_gb300.run paper_2410_10503_gb300/configs/config2_rigid512.json \\
        --out trace.jsonl

A config names a synthetic workload of ``mc_synth`` (seeded phantom, motion
and noise: d_i = A_i x + eps_i, eps_i ~ N(0, sigma^2 / N), sigma = 1% of the
largest clean value, Sec. II-A), the solvers (SPDHG of Algorithm 1 and/or
PDHG), the number of epochs, the storage type of d and y, and the run index
that selects the gate-draw seed.  The run computes the data with the GPU
operators, the squared operator norms by power iteration (Theorem, Sec. II-B)
and x* by conjugate gradients, then writes one JSON line per epoch:
{"config", "solver", "storage", "epoch", "rel_err" (||x - x*|| / ||x*||),
"saddle_dist2" (||x - x*||^2 + sum_i ||y_i - y_i*||^2, the distance of Fig. 1),
"objective" (O(x), when the config asks for it), "seconds" (device time since
the start of the solver)}.  A config with "batch" runs that many slices of
``mc_synth.slice_batch`` through the merged batched path and writes one line
per slice and one summary line.
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time


def _problem(W, mc, torch, run):
    import mc_synth as S
    sd = S.seeds(W.cid, run=run)
    if W.motion == "rigid":
        kw = dict(rigid=S.rigid_motion(W.n_gates, W.max_rot_deg, W.max_shift, sd["motion"]))
    else:
        kw = dict(fields=S.rbf_fields(W.n, W.n_gates, sd["motion"], W.rbf_count, W.rbf_width, W.rbf_max_disp))
    ctx = mc.Context(W.n, W.n_angles, W.n_bins, W.n_gates, **kw)
    xt = torch.as_tensor(S.phantom(W.n, W.n_ellipses, sd["phantom"], W.axis_lo, W.axis_hi),
                         dtype=torch.float32, device="cuda")
    d = torch.stack([ctx.forward(i, xt) for i in range(W.n_gates)])
    torch.cuda.synchronize()
    sigma = W.noise_level * float(d.max())
    eps = S.noise(W.n_gates, W.n_angles, W.n_bins, sd["noise"])
    d += torch.as_tensor(eps * (sigma / math.sqrt(W.n_gates)), dtype=torch.float32, device="cuda")
    return ctx, d, sd


def run_single(cfg, out, mc, torch):
    import mc_synth as S
    W = S.WORKLOADS[cfg["workload"]]
    ctx, d, sd = _problem(W, mc, torch, int(cfg.get("run", 0)))
    ctx.set_data(d, W.alpha)
    norms = ctx.norms(max_iter=int(cfg.get("norm_iters", 40)), tol=1e-7)
    x_star = torch.empty((W.n, W.n), dtype=torch.float32, device="cuda")
    _, iters, res = ctx.solve_normal(max_iter=int(cfg.get("cg_iters", 2000)), tol=float(cfg.get("cg_tol", 1e-9)),
                                     x_out=x_star)
    out.write(json.dumps({"config": cfg["name"], "x_star_cg_iterations": iters, "x_star_cg_rel_residual": res,
                          "norms2": [float(v) for v in norms], "kappa_spdhg": ctx.steps()["kappa"],
                          "kappa_pdhg": ctx.steps(pdhg=True)["kappa"]}) + "\n")
    ctx.set_option(3, 1 if cfg.get("trace_objective") else 0)
    chunk = int(cfg.get("chunk", 10))
    for store in cfg.get("storages", [cfg.get("storage", "f32")]):
        ctx.set_storage(store)
        ctx.set_reference(x_star)
        for solver in cfg["solvers"]:
            ctx.reset()
            t = 0.0
            done = 0
            while done < int(cfg["epochs"]):
                m = min(chunk, int(cfg["epochs"]) - done)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(ctx.stream)
                if solver == "spdhg":
                    _, tr = ctx.spdhg_run(m, seed=sd["gates"], x_out=False, trace=True)
                else:
                    _, tr = ctx.pdhg_run(m, x_out=False, trace=True)
                b.record(ctx.stream)
                b.synchronize()
                dt = a.elapsed_time(b) / 1e3
                for e in range(m):
                    row = {"config": cfg["name"], "solver": solver, "storage": store, "epoch": done + e + 1,
                           "rel_err": float(tr[e, 0]), "saddle_dist2": float(tr[e, 1]),
                           "seconds": round(t + dt * (e + 1) / m, 6)}
                    if cfg.get("trace_objective"):
                        row["objective"] = float(tr[e, 2])
                    out.write(json.dumps(row) + "\n")
                t += dt
                done += m
            out.flush()
    ctx.close()


def run_batch(cfg, out, mc, torch):
    import mc_synth as S
    ws = S.slice_batch(int(cfg["batch"]["count"]), seed=int(cfg["batch"].get("seed", 5000)))
    ctxs, seeds = [], []
    for W in ws:
        ctx, d, sd = _problem(W, mc, torch, int(cfg.get("run", 0)))
        ctx.set_data(d, W.alpha)
        ctx.set_norms(ctx.norms(max_iter=12, tol=1e-4) * 1.05)
        ctxs.append(ctx)
        seeds.append(sd["gates"])
    with mc.Batch(ctxs) as b:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.run(int(cfg["epochs"]), seeds)
        dt = time.perf_counter() - t0
    for W, ctx in zip(ws, ctxs):
        out.write(json.dumps({"config": cfg["name"], "slice": W.name, "n": W.n, "n_angles": W.n_angles,
                              "n_bins": W.n_bins, "gates": W.n_gates, "motion": W.motion,
                              "iterations": ctx.iteration()}) + "\n")
        ctx.close()
    pairs = int(cfg["epochs"]) * sum(W.n_gates for W in ws)
    out.write(json.dumps({"config": cfg["name"], "slices": len(ws), "epochs": int(cfg["epochs"]), "pairs": pairs,
                          "seconds": round(dt, 3), "pairs_per_s": round(pairs / dt, 1)}) + "\n")


def main(argv=None):
    ap = argparse.ArgumentParser(description="run one config, per-epoch JSONL log")
    ap.add_argument("config", help="JSON config (see paper_2410_10503_gb300/configs)")
    ap.add_argument("--out", default="-", help="JSONL output file ('-': standard output)")
    args = ap.parse_args(argv)
    with open(args.config) as f:
        cfg = json.load(f)
    import torch

    import paper_2410_10503_gb300 as mc
    if not torch.cuda.is_available():
        raise SystemExit("a CUDA device (sm_103a) is required")
    out = sys.stdout if args.out == "-" else open(args.out, "w")
    try:
        if "batch" in cfg:
            run_batch(cfg, out, mc, torch)
        else:
            run_single(cfg, out, mc, torch)
    finally:
        if out is not sys.stdout:
            out.close()


if __name__ == "__main__":
    main()
