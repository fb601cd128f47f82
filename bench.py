"""Benchmark: A_i + A_i^* pairs per second of GPU SPDHG at 512^2.

Workload (synthetic, seeded; stands in for the paper's walnut/chest slices):
512 x 512 phantom of 40 random ellipses, 720 angles x 729 bins, N = 10 rigid
gates (rotation U[-8, 8] deg, shift U[-6, 6] px), data d_i = A_i x + noise at
1% of the largest clean value, alpha = 1e-3.

One step = one SPDHG epoch = N iterations of Algorithm 1, i.e. N gate draws,
N warps, N forward projections with the fused dual update, N backprojections
and N transpose warps with the fused z / zbar / prox update: N pairs.  The
epoch is replayed as a CUDA graph.  Inputs stay resident in HBM; L2 (129 MB)
is flushed between steps by writing a 256 MB buffer outside the timed events.

--impl reference times the FP64 CPU oracle (a deliberately slow checker) on a
bounded sample per step: one pair on every s-th angle of the workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

import mc_synth as S

WORKLOAD = "rigid512"
METRIC = "A_i+A_i^* pairs/s at 512^2"
UNIT = "pairs/s"


def workload_config(W):
    return {
        "workload": f"{W.name}: {W.n}x{W.n} image ({W.n_ellipses} ellipses), {W.n_angles} angles x "
                    f"{W.n_bins} bins, N={W.n_gates} " + (
                        f"rigid gates (+-{W.max_rot_deg:g} deg, +-{W.max_shift:g} px)" if W.motion == "rigid"
                        else f"dense-field gates ({W.rbf_count} Gaussian bumps of sigma {W.rbf_width:g} px, "
                             f"max |u| = {W.rbf_max_disp:g} px)") + f", alpha={W.alpha:g}, SPDHG",
        "step": f"one SPDHG epoch = {W.n_gates} iterations = {W.n_gates} A_i+A_i^* pairs",
        "l2": "flushed between steps (256 MB write outside the timed events)",
    }


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampled every 100 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.start = 0

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi takes a moment to start: wait (at most 3 s) for its first
            # sample so that the timed region is covered from its start
            t_end = time.perf_counter() + 3.0
            while not self.lines and self.proc.poll() is None and time.perf_counter() < t_end:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        self.start = len(self.lines)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        # samples taken inside the timed region; the one before it only when the
        # region was shorter than the sampling interval
        inside = self.lines[self.start:]
        for ln in inside or self.lines:
            p = [t.strip() for t in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ setup
def make_problem(W, torch, mc, rank=0):
    sd = S.seeds(W.cid, run=rank)
    rig = S.rigid_motion(W.n_gates, W.max_rot_deg, W.max_shift, sd["motion"])
    xt = S.phantom(W.n, W.n_ellipses, sd["phantom"], W.axis_lo, W.axis_hi)
    eps = S.noise(W.n_gates, W.n_angles, W.n_bins, sd["noise"])
    stream = torch.cuda.Stream()
    ctx = mc.Context(W.n, W.n_angles, W.n_bins, W.n_gates, rigid=rig, stream=stream.cuda_stream)
    # data model d_i = A_i x + eps_i, eps_i ~ N(0, sigma^2/N), computed with the GPU operators
    x_t = torch.as_tensor(xt, dtype=torch.float32, device="cuda")
    d = torch.empty((W.n_gates, W.n_angles, W.n_bins), dtype=torch.float32, device="cuda")
    for i in range(W.n_gates):
        ctx.forward(i, x_t, out=d[i])
    torch.cuda.synchronize()
    sigma = W.noise_level * float(d.max())
    d += torch.as_tensor(eps * (sigma / math.sqrt(W.n_gates)), dtype=torch.float32, device="cuda")
    ctx.set_data(d, W.alpha)
    norms = ctx.norms(max_iter=40, tol=1e-7)
    return ctx, stream, d, norms, sd


def algorithmic_units(W):
    """Joseph samples S per projection (in-image line crossings) and the
    adjoint's (pixel, angle) pairs, counted from the geometry exactly."""
    n, na, nb = W.n, W.n_angles, W.n_bins
    h, hb = 0.5 * (n - 1), 0.5 * (nb - 1)
    S_cnt = 0
    for k in range(na):
        phi = k * math.pi / na
        c, s = math.cos(phi), math.sin(phi)
        xd = na <= 4 * k <= 3 * na
        inv, t = (1 / s, c / s) if xd else (1 / c, s / c)
        b = np.arange(nb) - hb
        l = np.arange(n) - h
        u = b[:, None] * inv - l[None, :] * t + h       # position on each line
        S_cnt += int(np.count_nonzero((u > -1.0) & (u < n)))
    return S_cnt


def reduce_over_ranks(tot_ms: float, units: float, dist, device):
    """Whole-job timing over ranks: the slowest rank's time and the sum of
    the units every rank processed (replicas, no data-path collective)."""
    if dist is None:
        return tot_ms, units
    import torch
    t = torch.tensor([tot_ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def profiled_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from profiles/ncu_traffic.json, or
    None when the kernel's source changed since that capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            rec = json.load(f)[kernel]
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()[:16]
        return rec["dram_bytes_per_launch"] if digest == rec["source_sha256_16"] else None
    except Exception:
        return None


def run_ours(args, W):
    import torch

    import paper_2410_10503_gb300 as mc
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2410_10503_gb300 import build
    build.build()

    ctx, stream, d, norms, sd = make_problem(W, torch, mc, rank)
    N = W.n_gates
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        ctx.spdhg_run(1, seed=sd["gates"], x_out=False)

    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 0)):
            step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        with ClockSampler(local) as clk:
            t0 = time.perf_counter()
            for a, b in evs:
                flush.zero_()
                a.record(stream)
                step()
                b.record(stream)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        step_ms = [a.elapsed_time(b) for a, b in evs]
        tot_ms, pairs = reduce_over_ranks(float(sum(step_ms)), float(args.steps * N), dist, "cuda")
        if dist:
            dist.barrier()
    value = pairs / (tot_ms / 1e3)

    # ---- per-kernel durations: same steps, per-launch CUDA events on the
    # context's stream (plain launches instead of the graph replay)
    ctx.set_option(2, 1)
    ctx.profile_reset()
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.zero_()
            step()
    prof = ctx.profile()
    ctx.set_option(2, 0)
    kernels = {k: {"launches": c, "avg_us": (ms * 1e3 / c) if c else None} for k, (c, ms) in prof.items()}

    # ---- end to end through the C ABI with host buffers: every step uploads
    # its gated data from pinned memory, runs one epoch and reads x back to
    # pinned memory.  Steps are pipelined as a streaming caller would: the
    # upload of step k + 1 is staged while step k runs (mc_stage_data) and
    # committed (mc_commit_data) right after step k is enqueued, and x_k is
    # copied to the host asynchronously and waited for one step later; the
    # first upload and the last read-back are inside the timed region.
    d_host = d.cpu().pin_memory()
    x_host = [torch.empty((W.n, W.n), dtype=torch.float32).pin_memory() for _ in range(2)]
    x_dev = [torch.empty((W.n, W.n), dtype=torch.float32, device="cuda") for _ in range(2)]
    cs = ctx.stream
    side = torch.cuda.Stream()          # the read-back runs beside the next epoch

    def e2e_steps(steps, sync_each):
        ctx.stage_data(d_host)
        ctx.commit_data(W.alpha)
        evs = []
        for k in range(steps):
            if sync_each:
                if k + 1 < steps:
                    ctx.stage_data(d_host)
                ctx.spdhg_run(1, seed=sd["gates"], x_out=x_host[0])
                if k + 1 < steps:
                    ctx.commit_data(W.alpha)
                continue
            if k + 1 < steps:
                ctx.stage_data(d_host)
            ctx.spdhg_run(1, seed=sd["gates"], x_out=x_dev[k % 2])
            side.wait_stream(cs)
            with torch.cuda.stream(side):
                x_host[k % 2].copy_(x_dev[k % 2], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(side)
            evs.append(ev)
            if k + 1 < steps:
                ctx.commit_data(W.alpha)
            if k >= 1:
                evs[k - 1].synchronize()
        if evs:
            evs[-1].synchronize()

    e2e_steps(2, False)
    e2e_steps(2, True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps(args.steps, False)
    e2e_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps(args.steps, True)
    e2e_sync_s = time.perf_counter() - t0
    e2e = {"value": args.steps * N * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(d_host.numel() * 4), "d2h_bytes_per_step": int(x_dev[0].numel() * 4),
           "pipeline": "step k+1's data uploaded (mc_stage_data) while step k runs and committed right after "
                       "step k is enqueued; x_k copied to pinned host memory on a side stream while step k+1 "
                       "runs and waited for during step k+1",
           "value_one_step_at_a_time": round(args.steps * N * world / e2e_sync_s, 2)}

    # ---- roofline of the dominant kernel (on-chip gather bytes per unit of work)
    S_cnt = algorithmic_units(W)
    smem_peak = mc.shared_load_peak(reps=20)
    if smem_peak is not None:
        peak = smem_peak["bytes_per_s"] / 1e9
        peak_source = (f"measured in this run by mc_measure_shared_load_peak: conflict-free 64-bit shared "
                       f"loads, {smem_peak['bytes_per_clk_per_sm']:.1f} B/clk/SM at "
                       f"{smem_peak['sm_ghz']:.3f} GHz over {smem_peak['sms']} SMs")
    else:
        peak = float(args.l1_peak_gbs)
        peak_source = "152 SMs x 128 B/clk shared/L1 load x 2.07 GHz (derived; measurement failed)"

    def roofline(kern):
        # both projectors: 8 B per unit of work (forward: two texel reads per
        # in-image sample; backprojection: 2 S (pixel, bin) pairs x 4 B)
        alg_bytes = 8.0 * S_cnt
        avg_s = kernels[kern]["avg_us"] * 1e-6
        achieved = alg_bytes / avg_s / 1e9
        return {"bound": "l1", "kernel": kern, "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": profiled_traffic(kern),
                "alg_bytes_per_launch": alg_bytes, "avg_launch_us": round(avg_s * 1e6, 2),
                "peak_source": peak_source, "peak_nominal_gbs": 152 * 128 * 2.07,
                "frac_of_nominal": round(achieved / (152 * 128 * 2.07), 4)}

    dom = max(("project", "backproject"), key=lambda k: kernels[k]["avg_us"] or 0)
    roof = roofline(dom)
    roof_other = roofline("backproject" if dom == "project" else "project")
    hbm_peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm_peak = json.load(f).get("hbm_gbs")
    except Exception:
        pass

    out = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot_ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": workload_config(W) | {"parallelism": f"replicas x{world}"},
        "roofline": roof, "roofline_other_projector": roof_other, "e2e": e2e,
        "gpu_launches": args.steps * (1 + 4 * N),
        "clocks": clk.summary(), "kernels": kernels,
        "norms2_max": float(np.max(norms[:N])), "kappa_spdhg": ctx.steps()["kappa"],
        "hbm_peak_gbs_measured": hbm_peak, "wall_s": round(wall, 3),
    }
    if args.convergence_epochs > 0:
        out["time_to_1e-3"] = convergence_legs(ctx, stream, d, W, norms, sd, args.convergence_epochs,
                                               args.alpha_epochs,
                                               tuple(int(v) for v in args.alpha_subsets.split(",") if v))
    if args.storage_epochs > 0:
        out["storage_rbf512"] = storage_legs(args.storage_epochs)
    if args.batch_slices > 0:
        out["batch_mixed_slices"] = batch_legs(args.batch_slices, args.batch_epochs, args.batch_seq_epochs,
                                               not args.batch_no_autotune)
        # the same recipe with every slice at the smallest side, where one
        # slice's launches leave most of the GPU idle
        out["batch_small_slices"] = batch_legs(args.batch_slices, args.batch_epochs, args.batch_seq_epochs,
                                               not args.batch_no_autotune, sides=(256,))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(W, samples=args.cpu_pairs)
        out["cpu_baseline_more"] = cpu_baseline_more(W)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def run_ncu_batch_case(args):
    """Kernel-profiling driver of the merged batched path: --ncu-batch slices
    of the mixed recipe (one of each side first), data A_i x, a fixed squared
    norm, then warm-up + timed batched epochs (mc_batch_run)."""
    import torch

    import paper_2410_10503_gb300 as mc
    from paper_2410_10503_gb300 import build
    build.build()
    ctxs, seeds = [], []
    for W in S.slice_batch(args.ncu_batch):
        sd = S.seeds(W.cid)
        if W.motion == "rigid":
            kw = dict(rigid=S.rigid_motion(W.n_gates, W.max_rot_deg, W.max_shift, sd["motion"]))
        else:
            kw = dict(fields=S.rbf_fields(W.n, W.n_gates, sd["motion"], W.rbf_count, W.rbf_width,
                                          W.rbf_max_disp))
        ctx = mc.Context(W.n, W.n_angles, W.n_bins, W.n_gates, **kw)
        xt = torch.as_tensor(S.phantom(W.n, W.n_ellipses, sd["phantom"], W.axis_lo, W.axis_hi),
                             dtype=torch.float32, device="cuda")
        d = torch.stack([ctx.forward(i, xt) for i in range(W.n_gates)])
        ctx.set_data(d, W.alpha)
        ctx.set_norms(np.full(W.n_gates + 1, 1.4 * W.n_angles * W.n))
        ctxs.append(ctx)
        seeds.append(sd["gates"])
    b = mc.Batch(ctxs)
    for _ in range(args.warmup + args.steps):
        b.run(1, seeds)
    torch.cuda.synchronize()
    b.close()
    for c in ctxs:
        c.close()
    print(json.dumps({"ncu_batch_case": args.ncu_batch, "epochs": args.warmup + args.steps}))


def run_ncu_case(args, W):
    """Kernel-profiling driver: warm-up + timed SPDHG epochs of the workload as
    plain launches (41 per epoch at N = 10), nothing else on the GPU after the
    data setup.  Step sizes come from a fixed squared norm, which changes no
    kernel's work."""
    import torch

    import paper_2410_10503_gb300 as mc
    from paper_2410_10503_gb300 import build
    build.build()
    sd = S.seeds(W.cid)
    rig = S.rigid_motion(W.n_gates, W.max_rot_deg, W.max_shift, sd["motion"])
    ctx = mc.Context(W.n, W.n_angles, W.n_bins, W.n_gates, rigid=rig)
    x_t = torch.as_tensor(S.phantom(W.n, W.n_ellipses, sd["phantom"], W.axis_lo, W.axis_hi),
                          dtype=torch.float32, device="cuda")
    d = torch.empty((W.n_gates, W.n_angles, W.n_bins), dtype=torch.float32, device="cuda")
    for i in range(W.n_gates):
        ctx.forward(i, x_t, out=d[i])
    ctx.set_data(d, W.alpha)
    if args.subsets > 1:
        ctx.set_subsets(args.subsets)
    ctx.set_norms(np.full(ctx.n_blocks + 1, 3.5e5 / args.subsets))
    ctx.set_option(1, 0)
    for _ in range(args.warmup + args.steps):
        ctx.spdhg_run(1, seed=sd["gates"], x_out=False)
    torch.cuda.synchronize()
    ctx.close()
    print(json.dumps({"ncu_case": W.name, "subsets": args.subsets, "epochs": args.warmup + args.steps}))


def time_to_tol(ctx, stream, which, tol, max_epochs, seed, graph=True, chunk=1):
    """Epochs (SPDHG: N iterations; PDHG: 1 iteration) from a zero start until
    ||x - x*|| / ||x*|| <= tol, timed with CUDA events (trace reductions
    included); returns a dict with epochs (None if not reached), seconds to the
    crossing (or to max_epochs) and the last relative error.  Epochs run in
    calls of `chunk` epochs, each timed by its own events; the crossing's time
    is the chunks before it plus the crossing chunk's time prorated to the
    crossing epoch (epochs of one run cost the same), exact for chunk = 1."""
    import torch
    ctx.reset()
    ctx.set_option(1, 1 if graph else 0)
    tot = 0.0
    rel = float("nan")
    done = 0
    with torch.cuda.stream(stream):
        while done < max_epochs:
            m = min(chunk, max_epochs - done)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if which == "spdhg":
                _, tr = ctx.spdhg_run(m, seed=seed, x_out=False, trace=True)
            else:
                _, tr = ctx.pdhg_run(m, x_out=False, trace=True)
            b.record(stream)
            b.synchronize()
            t = a.elapsed_time(b) / 1e3
            hit = np.nonzero(tr[:, 0] <= tol)[0]
            if len(hit):
                e = int(hit[0]) + 1
                ctx.set_option(1, 1)
                return {"epochs": done + e, "seconds": round(tot + t * e / m, 6), "rel_err": float(tr[e - 1, 0])}
            tot += t
            done += m
            rel = float(tr[-1, 0])
    ctx.set_option(1, 1)
    return {"epochs": None, "seconds_for_max_epochs": round(tot, 6), "max_epochs": max_epochs,
            "rel_err": rel}


def convergence_legs(ctx, stream, d, W, norms, sd, max_epochs, alpha_epochs, alpha_subsets=(8,)):
    """Time to 1e-3 relative distance to x* for graph-replayed SPDHG, SPDHG
    with plain launches and PDHG, in the paper's regime (alpha such that
    ||A||^2 / alpha = 70, Sec. III; at most max_epochs, timed epoch by epoch)
    and at the workload's own alpha (at most alpha_epochs, timed in chunks of
    100 epochs); also SPDHG over gates x S angle subsets, S = 2, 4, 8 in the
    paper's regime and S in alpha_subsets at the workload's alpha.  x* by float32 CG to a relative residual of 1e-6
    (paper regime) or 1e-9 (the workload's alpha, where the normal operator's
    condition number is ~3.5e7)."""
    import torch
    out = {}
    nA = float(np.max(norms[:W.n_gates]))
    for label, alpha, cg_iters, cg_tol, cap, chunk in [
            ("paper_regime_kappa70", nA / 70.0, 400, 1e-6, max_epochs, 1),
            ("workload_alpha", W.alpha, 2000, 1e-9, alpha_epochs, 100)]:
        if cap <= 0:
            continue
        ctx.set_data(d, alpha)
        ctx.set_norms(norms)
        x_star = torch.empty((W.n, W.n), dtype=torch.float32, device="cuda")
        _, iters, rel = ctx.solve_normal(max_iter=cg_iters, tol=cg_tol, x_out=x_star)
        ctx.set_reference(x_star)
        leg = {"alpha": alpha, "kappa": nA / alpha,
               "kappa_spdhg": ctx.steps()["kappa"], "kappa_pdhg": ctx.steps(pdhg=True)["kappa"],
               "x_star_cg": {"iterations": iters, "rel_residual": rel},
               "rate_bound_per_epoch": {"spdhg": _rate(ctx.steps()["kappa"], W.n_gates),
                                        "pdhg": _rate(ctx.steps(pdhg=True)["kappa"], 1)}}
        leg["spdhg_graph"] = time_to_tol(ctx, stream, "spdhg", 1e-3, cap, sd["gates"], True, chunk)
        if chunk == 1:
            leg["spdhg_plain"] = time_to_tol(ctx, stream, "spdhg", 1e-3, cap, sd["gates"], False, chunk)
        # the same SPDHG iterates through the three launch paths (plain launches,
        # graph-replayed epochs, merged batched iterations: bit-identical), timed
        # per epoch without the trace on a 1000-epoch sample, times the epochs
        leg["spdhg_same_iterates_no_trace"] = {
            how: projected_time(ctx, stream, how, leg["spdhg_graph"], sd["gates"], 1000)
            for how in ("graph", "plain", "batched")}
        leg["pdhg_graph"] = time_to_tol(ctx, stream, "pdhg", 1e-3, cap, sd["gates"], True, chunk)
        # sampling over gates x angle subsets (Sec. IV): same objective and x*,
        # blocks of 1/S of the angles, N S iterations per epoch; per epoch the
        # bound improves from l(kappa, N) to l(kappa / S, N S) (block norms^2 ~1/S)
        subs = {}
        for n_sub in ((2, 4, 8) if label == "paper_regime_kappa70" else alpha_subsets):
            ctx.set_subsets(n_sub)
            ctx.norms(max_iter=100, tol=1e-7)
            r = time_to_tol(ctx, stream, "spdhg", 1e-3, cap, sd["gates"], True, chunk)
            r["kappa_spdhg"] = ctx.steps()["kappa"]
            r["rate_bound_per_epoch"] = _rate(ctx.steps()["kappa"], W.n_gates * n_sub)
            subs[f"S={n_sub}"] = r
        ctx.set_subsets(1)
        ctx.set_norms(norms)
        if subs:
            leg["spdhg_angle_subsets_graph"] = subs
        out[label] = leg
    ctx.set_data(d, W.alpha)
    ctx.set_norms(norms)
    return out


def projected_time(ctx, stream, how, graph_leg, seed, sample_epochs):
    """Time to the tolerance of an SPDHG path whose iterates equal the graph
    run's bit for bit (graph replay, plain launches, or the merged batched path
    with this one slice): the graph run's epochs times this path's time per
    epoch, measured on `sample_epochs` epochs without the trace, so that the
    three paths compare on one basis."""
    import torch

    import paper_2410_10503_gb300 as mc
    ctx.reset()
    out = {"sample_epochs": sample_epochs}
    if how in ("plain", "graph"):
        ctx.set_option(1, 1 if how == "graph" else 0)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            ctx.spdhg_run(2, seed=seed, x_out=False)
            stream.synchronize()
            t0 = time.perf_counter()
            ctx.spdhg_run(sample_epochs, seed=seed, x_out=False)
            stream.synchronize()
            per_epoch = (time.perf_counter() - t0) / sample_epochs
        ctx.set_option(1, 1)
        out["timing"] = "host clock around mc_spdhg_run of the sample and a stream synchronisation (no trace)"
    else:
        batch = mc.Batch([ctx])
        batch.run(2, [seed])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        batch.run(sample_epochs, [seed])
        per_epoch = (time.perf_counter() - t0) / sample_epochs
        batch.close()
        out["timing"] = "host clock around mc_batch_run (returns after the batch finished; no trace)"
    out["seconds_per_epoch"] = round(per_epoch, 7)
    ctx.reset()
    e = graph_leg.get("epochs")
    out["epochs"] = e
    if e is not None:
        out["seconds"] = round(e * per_epoch, 6)
    else:
        out["seconds_for_max_epochs"] = round(graph_leg["max_epochs"] * per_epoch, 6)
    return out


def _rate(kappa, n):
    """l(kappa, n) = (1 - 2 n^-1 (1 + sqrt(1 + kappa))^-1)^n, the Theorem's
    per-epoch contraction (Sec. II-B)."""
    return (1.0 - 2.0 / (n * (1.0 + math.sqrt(1.0 + kappa)))) ** n


def storage_legs(max_epochs, steps=20):
    """The non-rigid workload rbf512 (512^2, 720 x 729, N = 20 Gaussian-bump
    fields) with d and y stored as float32, binary16 and bfloat16 (float32
    arithmetic): time to 1e-3 relative distance to the float32 problem's x*
    in the paper's regime (||A_i||^2 / alpha = 70), the distance reached
    after max_epochs (the storage floor), and pairs/s of graph-replayed
    epochs without trace."""
    import torch

    import paper_2410_10503_gb300 as mc
    W = S.WORKLOADS["rbf512"]
    sd = S.seeds(W.cid)
    fields = S.rbf_fields(W.n, W.n_gates, sd["motion"], W.rbf_count, W.rbf_width, W.rbf_max_disp)
    xt = S.phantom(W.n, W.n_ellipses, sd["phantom"], W.axis_lo, W.axis_hi)
    eps = S.noise(W.n_gates, W.n_angles, W.n_bins, sd["noise"])
    stream = torch.cuda.Stream()
    ctx = mc.Context(W.n, W.n_angles, W.n_bins, W.n_gates, fields=fields, stream=stream.cuda_stream)
    x_t = torch.as_tensor(xt, dtype=torch.float32, device="cuda")
    d = torch.empty((W.n_gates, W.n_angles, W.n_bins), dtype=torch.float32, device="cuda")
    for i in range(W.n_gates):
        ctx.forward(i, x_t, out=d[i])
    torch.cuda.synchronize()
    sigma = W.noise_level * float(d.max())
    d += torch.as_tensor(eps * (sigma / math.sqrt(W.n_gates)), dtype=torch.float32, device="cuda")
    ctx.set_data(d, W.alpha)
    norms = ctx.norms(max_iter=40, tol=1e-7)
    alpha = float(np.max(norms[:W.n_gates])) / 70.0
    ctx.set_data(d, alpha)
    ctx.set_norms(norms)
    x_star = torch.empty((W.n, W.n), dtype=torch.float32, device="cuda")
    _, iters, rel = ctx.solve_normal(max_iter=400, tol=1e-6, x_out=x_star)
    ctx.set_reference(x_star)
    out = {"workload": workload_config(W)["workload"], "alpha": alpha,
           "kappa_spdhg": ctx.steps()["kappa"], "x_star_cg": {"iterations": iters, "rel_residual": rel}}
    for store in ("f32", "f16", "bf16"):
        ctx.set_storage(store)
        leg = time_to_tol(ctx, stream, "spdhg", 1e-3, max_epochs, sd["gates"], True)
        ctx.reset()
        with torch.cuda.stream(stream):
            _, tr = ctx.spdhg_run(max_epochs, seed=sd["gates"], x_out=False, trace=True)
        leg["rel_err_after_max_epochs"] = float(tr[-1, 0])
        leg["max_epochs"] = max_epochs
        with torch.cuda.stream(stream):
            ctx.spdhg_run(2, seed=sd["gates"], x_out=False)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.spdhg_run(steps, seed=sd["gates"], x_out=False)
            b.record(stream)
            b.synchronize()
        leg["pairs_per_s"] = round(steps * W.n_gates / (a.elapsed_time(b) / 1e3), 1)
        out[store] = leg
    ctx.close()
    return out


def batch_legs(count, epochs, seq_epochs, autotune=True, sides=None):
    """The batched-slices workload: `count` independent slices of mixed size
    (mc_synth.slice_batch: sides 256-1024, angles round(1.4 side), bins
    side + 17, gates U{4..32}, rigid and dense-field motion alternating;
    data A_i x + 1% noise), each in its own context with autotuned launch
    shapes.  Timed: `epochs` SPDHG epochs of every slice as merged batched
    iterations (mc_batch_run: one launch per stage over all slices in flight,
    graph-replayed), and the same slices one after another through their own
    epoch graphs (mc_spdhg_run, `seq_epochs` epochs each: the same
    iterations, so pairs/s compare directly); throughput in A_i + A_i^* pairs
    per second of the whole batch."""
    import torch

    import paper_2410_10503_gb300 as mc
    t_setup = time.perf_counter()
    ws = S.slice_batch(count) if sides is None else S.slice_batch(count, sides=sides)
    ctxs, seeds, tunes = [], [], []
    for W in ws:
        sd = S.seeds(W.cid)
        if W.motion == "rigid":
            kw = dict(rigid=S.rigid_motion(W.n_gates, W.max_rot_deg, W.max_shift, sd["motion"]))
        else:
            kw = dict(fields=S.rbf_fields(W.n, W.n_gates, sd["motion"], W.rbf_count, W.rbf_width,
                                          W.rbf_max_disp))
        ctx = mc.Context(W.n, W.n_angles, W.n_bins, W.n_gates, **kw)
        xt = torch.as_tensor(S.phantom(W.n, W.n_ellipses, sd["phantom"], W.axis_lo, W.axis_hi),
                             dtype=torch.float32, device="cuda")
        d = torch.empty((W.n_gates, W.n_angles, W.n_bins), dtype=torch.float32, device="cuda")
        for i in range(W.n_gates):
            ctx.forward(i, xt, out=d[i])
        torch.cuda.synchronize()
        sigma = W.noise_level * float(d.max())
        g = torch.Generator(device="cuda").manual_seed(sd["noise"])
        d += torch.randn(d.shape, generator=g, device="cuda") * (sigma / math.sqrt(W.n_gates))
        ctx.set_data(d, W.alpha)
        ctx.set_norms(ctx.norms(max_iter=12, tol=1e-4) * 1.05)
        if autotune:
            tunes.append(ctx.autotune(reps=2))
        ctxs.append(ctx)
        seeds.append(sd["gates"])
        del d, xt
    setup_s = time.perf_counter() - t_setup
    pairs = epochs * sum(W.n_gates for W in ws)
    batch = mc.Batch(ctxs)
    batch.run(1, seeds)                              # captures every phase's graphs
    for c, sdg in zip(ctxs, seeds):                  # and every slice's own epoch graph
        c.spdhg_run(1, seed=sdg, x_out=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch.run(epochs, seeds)
    bat_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    for c, sdg in zip(ctxs, seeds):
        c.spdhg_run(seq_epochs, seed=sdg, x_out=False)
        c.stream.synchronize()
    seq_s = time.perf_counter() - t0
    seq_pairs = seq_epochs * sum(W.n_gates for W in ws)
    sizes = sorted({W.n for W in ws})
    out = {"workload": f"{count} slices, sides {sizes} (angles round(1.4 side), bins side + 17), gates U{{4..32}} "
                       f"(total {sum(W.n_gates for W in ws)}), rigid and dense-field motion alternating, "
                       f"alpha 1e-3, 1% noise",
           "epochs_per_slice": epochs, "pairs": pairs,
           "batched_merged": {"seconds": round(bat_s, 3), "pairs_per_s": round(pairs / bat_s, 1),
                              "launches_per_batched_iteration": "4: warp, forward, backprojection, transpose warp "
                                                                "(+ gate draw), each over all slices in flight"},
           "one_after_another": {"epochs_per_slice": seq_epochs, "seconds": round(seq_s, 3),
                                 "pairs_per_s": round(seq_pairs / seq_s, 1)},
           "setup_s": round(setup_s, 1), "autotuned": bool(autotune)}
    out["speedup_merged_over_one_after_another"] = round((pairs / bat_s) / (seq_pairs / seq_s), 3)
    batch.close()
    for c in ctxs:
        c.close()
    return out


def _oracle_pair_setup(W, stride: int = 1):
    """The oracle's problem for workload W.  With stride s > 1 the geometry
    keeps every s-th angle (n_angles / s angles: angle k' of it is angle k' s
    of the workload, same rays), so one pair on it is 1/s of a workload pair."""
    import oracle as O
    if W.n_angles % stride:
        raise ValueError("stride must divide the angle count")
    na = W.n_angles // stride
    sd = S.seeds(W.cid)
    g = O.Geometry(W.n, na, W.n_bins)
    rig = S.rigid_motion(W.n_gates, W.max_rot_deg, W.max_shift, sd["motion"])
    P = O.Problem(g, O.Motion(rigid=rig), np.zeros((W.n_gates, na, W.n_bins)), W.alpha)
    x = S.phantom(W.n, W.n_ellipses, sd["phantom"], W.axis_lo, W.axis_hi)
    y = S.random_sinogram(na, W.n_bins, 5)
    return O, P, x, y


def reference_stride(n_angles: int, steps_total: int, pair_s: float = 1.3, budget_s: float = 90.0) -> int:
    """Smallest divisor s of n_angles such that steps_total oracle steps of
    1/s of a pair each (pair_s seconds per whole pair) fit in budget_s."""
    need = steps_total * pair_s / budget_s
    return next(s for s in range(1, n_angles + 1) if n_angles % s == 0 and s >= need)


def cpu_baseline(W, samples=3):
    """The FP64 oracle, as it stands (one thread), on a bounded sample:
    `samples` A_i + A_i^* pairs of the same workload."""
    O, P, x, y = _oracle_pair_setup(W)
    t0 = time.perf_counter()
    for i in range(samples):
        O.Ai(x, P, i % W.n_gates)
        O.Ait(y, P, i % W.n_gates)
    dt = time.perf_counter() - t0
    return {"value": round(samples / dt, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{samples} A_i+A_i^* pairs of {W.name} (FP64, single thread)"}


_START = None


def _oracle_pool_init(barrier):
    global _START
    _START = barrier


def _oracle_pairs_worker(job):
    """Spawned process: set up, wait until every worker is ready (the pool's
    shared barrier), then time `count` A_i + A_i^* pairs of workload `wl` on
    the oracle (one thread); returns (count, start, end) on the host's
    monotonic clock, which all processes share."""
    wl, count, first, wait_s = job
    W = S.WORKLOADS[wl]
    O, P, x, y = _oracle_pair_setup(W)
    _START.wait(timeout=wait_s)
    t0 = time.perf_counter()
    for i in range(first, first + count):
        O.Ai(x, P, i % W.n_gates)
        O.Ait(y, P, i % W.n_gates)
    return count, t0, time.perf_counter()


def cpu_baseline_more(W, cores=None, small="rigid128", small_pairs=20, epochs=50, timeout_s=300.0):
    """Further timings of the oracle as it stands, baselines only; each leg is
    fenced, so that a failure is reported in its entry instead of ending the run:
    - all_cores: one pair of W per core, in that many spawned processes (the
      oracle itself stays single-threaded) that start together on a barrier;
      pairs / the wall span from the first start to the last end;
    - pairs_<small>: pairs/s on the 128^2 workload, one thread;
    - solvers_<small>: a whole `epochs`-epoch SPDHG and PDHG run of it, one
      thread (norms and data set up outside the timing)."""
    from concurrent.futures import ProcessPoolExecutor
    import multiprocessing as mp
    out = {}
    try:
        if cores is None:
            cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        spawn = mp.get_context("spawn")
        barrier = spawn.Barrier(cores)
        ex = ProcessPoolExecutor(max_workers=cores, mp_context=spawn, initializer=_oracle_pool_init,
                                 initargs=(barrier,))
        try:
            futs = [ex.submit(_oracle_pairs_worker, (W.name, 1, c, timeout_s)) for c in range(cores)]
            res = [f.result(timeout=timeout_s) for f in futs]
        finally:
            # stragglers of a timed-out leg must not run on into the next legs
            procs = list(getattr(ex, "_processes", {}).values())
            ex.shutdown(wait=False, cancel_futures=True)
            for pr in procs:
                if pr.is_alive():
                    pr.terminate()
            for pr in procs:
                pr.join(timeout=5)
        n = sum(r[0] for r in res)
        span = max(r[2] for r in res) - min(r[1] for r in res)
        out["all_cores"] = {"value": round(n / span, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"one A_i+A_i^* pair of {W.name} in each of {cores} spawned processes "
                                      f"(one thread each, started together on a barrier); pairs / the wall "
                                      f"span from the first start to the last end"}
    except Exception as e:
        out["all_cores"] = {"error": f"{type(e).__name__}: {e}"[:300]}
    W1 = S.WORKLOADS[small]
    try:
        O, P1, x1, y1 = _oracle_pair_setup(W1)
        t0 = time.perf_counter()
        for i in range(small_pairs):
            O.Ai(x1, P1, i % W1.n_gates)
            O.Ait(y1, P1, i % W1.n_gates)
        dt = time.perf_counter() - t0
        out[f"pairs_{small}"] = {"value": round(small_pairs / dt, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": f"{small_pairs} A_i+A_i^* pairs of {small}"}
    except Exception as e:
        out[f"pairs_{small}"] = {"error": f"{type(e).__name__}: {e}"[:300]}
    try:
        import oracle as O
        sd = S.seeds(W1.cid)
        g = O.Geometry(W1.n, W1.n_angles, W1.n_bins)
        m = O.Motion(rigid=S.rigid_motion(W1.n_gates, W1.max_rot_deg, W1.max_shift, sd["motion"]))
        xt = S.phantom(W1.n, W1.n_ellipses, sd["phantom"], W1.axis_lo, W1.axis_hi)
        P = O.make_problem(g, m, xt, S.noise(W1.n_gates, W1.n_angles, W1.n_bins, sd["noise"]),
                           W1.alpha, W1.noise_level)
        norms = O.gate_norms2(P, iters=30, tol=1e-13)
        t0 = time.perf_counter()
        O.spdhg(P, epochs, O.step_sizes(norms[:P.N].max(), P.alpha, P.N, P.N), seed=sd["gates"])
        t_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        O.pdhg(P, epochs, O.step_sizes(norms[P.N], P.alpha, P.N, 1))
        t_p = time.perf_counter() - t0
        out[f"solvers_{small}"] = {"epochs": epochs, "spdhg_s": round(t_s, 3), "pdhg_s": round(t_p, 3),
                                   "cores": 1, "kind": "oracle"}
    except Exception as e:
        out[f"solvers_{small}"] = {"error": f"{type(e).__name__}: {e}"[:300]}
    return out


def run_reference(args, W):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # each step: A_i + A_i^* on every s-th angle of the workload (1/s of a
    # pair), s chosen so that the whole run stays within about a minute and a half
    stride = reference_stride(W.n_angles, max(args.warmup, 0) + args.steps,
                              budget_s=args.reference_budget_s)
    O, P, x, y = _oracle_pair_setup(W, stride)
    for i in range(max(args.warmup, 0)):
        O.Ai(x, P, i % W.n_gates); O.Ait(y, P, i % W.n_gates)
    t0 = time.perf_counter()
    for i in range(args.steps):
        O.Ai(x, P, i % W.n_gates); O.Ait(y, P, i % W.n_gates)
    dt = time.perf_counter() - t0
    v = args.steps / stride / dt
    sample = (f"one A_i+A_i^* pair of {W.name} per step" if stride == 1 else
              f"per step one A_i+A_i^* pair of {W.name} on the {W.n_angles // stride} angles "
              f"k = 0, {stride}, {2 * stride}, ... of {W.n_angles} (1/{stride} of a pair)")
    out = {"metric": METRIC, "value": round(v, 4), "unit": UNIT, "impl": "reference",
           "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(dt / args.steps * 1e3, 2), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(W) | {"step": f"1/{stride} of an A_i+A_i^* pair (FP64 oracle, host)",
                                           "l2": "not applicable (host oracle)"},
           "cpu_baseline": {"value": round(v, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(v, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(S.WORKLOADS))
    ap.add_argument("--cpu-pairs", type=int, default=3)
    ap.add_argument("--reference-budget-s", type=float, default=90.0,
                    help="--impl reference: seconds the warm-up and timed oracle steps may take "
                         "together; each step is then 1/s of a pair (every s-th angle)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--convergence-epochs", type=int, default=100,
                    help="epoch cap of the time-to-1e-3 legs (0 skips them)")
    ap.add_argument("--alpha-epochs", type=int, default=60000,
                    help="epoch cap of the time-to-1e-3 legs at the workload's own alpha (0: skip)")
    ap.add_argument("--alpha-subsets", default="8",
                    help="comma-separated angle-subset counts S of the gates x subsets SPDHG legs at "
                         "the workload's own alpha ('' skips them)")
    ap.add_argument("--storage-epochs", type=int, default=100,
                    help="epoch cap of the rbf512 float32/binary16/bfloat16 storage legs (0 skips)")
    ap.add_argument("--batch-slices", type=int, default=64,
                    help="independent mixed-size slices of the batched leg (0 skips)")
    ap.add_argument("--batch-epochs", type=int, default=100)
    ap.add_argument("--batch-seq-epochs", type=int, default=10,
                    help="epochs per slice of the one-after-another comparison (a bounded sample)")
    ap.add_argument("--batch-no-autotune", action="store_true")
    ap.add_argument("--l1-peak-gbs", type=float, default=152 * 128 * 2.07)
    ap.add_argument("--ncu-case", action="store_true",
                    help="profiling driver: set up the workload, then only warm-up + timed "
                         "epochs as plain launches (no norms, e2e, profile or CPU legs)")
    ap.add_argument("--ncu-batch", type=int, default=0,
                    help="with --ncu-case: profile the merged batched path on this many mixed slices")
    ap.add_argument("--subsets", type=int, default=1,
                    help="--ncu-case only: sample gates x this many angle subsets")
    args = ap.parse_args()
    W = S.WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, W)
    elif args.ncu_case and args.ncu_batch > 0:
        run_ncu_batch_case(args)
    elif args.ncu_case:
        run_ncu_case(args, W)
    else:
        run_ours(args, W)


if __name__ == "__main__":
    main()
