"""Benchmark: FIRLS reconstructions per second at 256x256 (TV + Daubechies-4).

Workload (one GPU): a batch of ``--batch`` independent 256x256 complex
slices, each the TV + 4-level D4 problem (20 % variable-density mask,
sigma 0.01, lambda_TV 1e-3, lambda_W 5e-4) with its own seed, solved with
a FIRLS schedule of at most ``--outer`` reweighting steps x ``--inner`` PCG
steps with a per-slice stop on the relative change (defaults reach the FP64
oracle's converged solution to 1e-4).  ``--learned`` adds the learned warm
start: a CNN trained (untimed) on pairs the solver itself generates, then
timed as CNN + data consistency + guard + the same solve.  One bench step = reconstructing a queue of ``--queue`` slices through
``--batch`` concurrent slots (continuous batching: a slot is refilled as
soon as its slice has converged); the value is reconstructions per second
over all ranks.  Inputs are synthetic
(seeded phantoms standing in for the paper's MR images).

``--impl reference`` times the FP64 CPU oracle instead, on a bounded sample
of the same workload (one slice, ``--ref-outer`` outer steps per bench
step), and reports the same metric.

Under torchrun every rank solves its own batch (independent slices, no data
exchange: weak scaling); only the step timing is reduced (max over ranks).
"""
from __future__ import annotations

import argparse
import json
import os
import math
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "recons/sec at 256^2 to 1e-4 of FP64 oracle (TV+D4 FIRLS)"
UNIT = "recons/s"
N = 256
RATIO, SIGMA, LAM_TV, LAM_W, LEVELS = 0.20, 0.01, 1e-3, 5e-4, 4
# Schedule that brings every TV + D4 256^2 slice within 1e-4 of the FP64
# oracle's converged minimiser x*.  Inner solves: 60 PCG steps per outer step
# (an oracle study of 40..120 found 60 needs the fewest PCG steps to 1e-4 on
# a typical slice), and 240 from a slice's 60th outer step on: the slices
# still running then have ill-conditioned subproblems whose outer rate is set
# by the inexact inner solve (with 60 steps they crawl to 1e-4 in 400-560
# outer steps; with 240 from the 60th step the slowest stored slice needs
# 18k PCG steps instead of 34k, and slices done by then are unaffected).
# Every slice advances on its own, so slices in either phase never wait for
# each other.  Outer stop per slice: the estimated distance to the limit,
# relchg * mu / (1 - mu) with mu the mean contraction over the last 24 outer
# steps, below OUTER_TOL, or the relative change at the FP32 floor of the
# outer iteration (<= STALL_TOL four steps in a row); at most OUTER outer
# steps.  Per-step GPU trajectories of the 20 stored-x* seeds (the slowest
# slices of the queue among them) picked these values (worst 5.6e-5 at the
# stop).  Slices are served by continuous batching: a converged slice leaves
# its slot, the next enters.  Checked against stored oracle x* by
# tests/test_gpu_parity.py::test_bench_workload_reaches_converged_oracle and
# reported per result in the bench line ("accuracy").
OUTER, INNER, INNER_LATE, OUTER_LATE, OUTER_TOL, STALL_TOL = 800, 60, 240, 60, 3e-5, 6e-7
# the ILU(0) variant's late inner schedule (its subproblems are solved in fewer
# PCG steps, and a shorter late schedule is the faster one for it)
ILU0_INNER_LATE = 160
SERVE_CHUNK = 64   # macro steps between polls of the slots
BOUNDARY_PERIOD = 8  # outer-step transitions (and their weight updates) every 8th macro step
REF_OUTER_PER_RECON = 43   # FP64 oracle outer steps (x 60 PCG) to 1e-4 of x* on seed 2

# Algorithmic bytes per pixel per launch of each kernel class: every distinct
# input read once and every output written once (complex64 8 B, float 4 B,
# mask 1 B).  Wavelet passes move the full pyramid (4/3 of the image).
ALG_BYTES_PER_PX = {
    "row_fft": 32.0,            # read z, d; write d, t
    "col_fft_mask": 17.0,       # read t, mask; write t
    "wavelet_S": 8.0 + 4.0 + 8.0,     # read d and w, write u = Phi^T (w o Phi d)
    "row_ifft_combine": 36.0,   # read t, d, u, W_tv; write q
    "ilu": 64.0,                # read x, d, r, q, W_tv, 1/a; write x, r, z
    "axpy": 32.0,
}

# DRAM bytes per pixel per launch (dram__bytes_read.sum + dram__bytes_write.sum)
# of the dominant kernel at the bench's 304 slots of 256^2, by the ILU ring
# shape the autotuner picks, from one-pass ncu captures of those two counters
# (profiles/kernels_tv_db4_256_b96.md gives the commands), for the kernel as
# it is now: 1.634 GB per launch with ring 22, 1.618 GB with ring 42.  Other
# shapes: not measured (traffic null).
MEASURED_TRAFFIC_PER_PX = {("ilu", 22): 82.0, ("ilu", 42): 81.2}


def problem(seed):
    import firls_synth as fs
    return fs.make_problem(N, RATIO, SIGMA, seed, real=False, psi=fs.PSI_TV | fs.PSI_DB4, levels=LEVELS,
                           lam=LAM_W, lam_tv=LAM_TV)


def make_batch(batch, first_seed):
    probs = [problem(first_seed + i) for i in range(batch)]
    masks = np.stack([p.mask for p in probs])
    b = np.stack([p.b for p in probs]).astype(np.complex64)
    return masks, b


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def rank_first_seed(rank, queue):
    """First seed of a rank's queue: ranks serve disjoint, consecutive seed
    ranges (replicas; no data is exchanged)."""
    return 2 + rank * queue


def max_over_ranks(value, dist, device):
    """The largest value over the ranks (the step time every rank reports)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_ours(args):
    import torch
    import paper_1411_5057_gb300 as F

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    B, S = args.batch, args.queue
    masks_h, b_h = make_batch(S, rank_first_seed(rank, S))
    stream = torch.cuda.Stream()
    params = F.make_params(args.outer, args.inner, lam=LAM_W, lam_tv=LAM_TV, outer_tol=args.outer_tol,
                           stop_on_distance=True, stall_tol=args.stall_tol, pcg_late=args.inner_late,
                           outer_late=args.outer_late, boundary_period=args.boundary_period,
                           precond=args.precond)
    lams, lam_tvs = [LAM_W] * S, [LAM_TV] * S
    with torch.cuda.stream(stream):
        masks = torch.from_numpy(masks_h).cuda()
        b = torch.from_numpy(b_h).cuda()
        ctx = F.Context(N, batch=B, stream=stream)
        ctx.set_operator(masks[:B], F.PSI_TV | F.PSI_DB4, LEVELS)
        # tile shapes (wavelet rows per CTA, on-chip wavelet block, ILU ring)
        # timed on this context's own buffers before anything is measured
        tuning = ctx.autotune() if args.autotune else ctx.tuning()
        x = torch.empty_like(b)
    stream.synchronize()
    print(f"[bench] tuning {tuning}", file=sys.stderr, flush=True)
    mlist, blist, xlist = list(masks), list(b), list(x)

    def barrier():
        if dist is not None:
            dist.barrier()

    done_per_step = S - B if args.steady else S
    pcg_counts = [0] * S

    def step(x0s=None, counters=None):
        with torch.cuda.stream(stream):
            return F.serve(ctx, mlist, blist, lams, lam_tvs, params, xlist, x0s=x0s, max_outer=args.outer,
                           chunk=SERVE_CHUNK, pcg_steps=pcg_counts,
                           stop_after=S - B if args.steady else None, counters=counters)

    def serve_queue(ml, bl, xl, pcg, x0s=None, stop_after=None):
        """Another queue through the same slots and schedule (drained, or
        stopped after `stop_after` completions)."""
        with torch.cuda.stream(stream):
            return F.serve(ctx, ml, bl, [LAM_W] * len(ml), [LAM_TV] * len(ml), params, xl, x0s=x0s,
                           max_outer=args.outer, chunk=SERVE_CHUNK, pcg_steps=pcg, stop_after=stop_after)

    # ---- device-resident throughput: continuous batching over S slices ----
    for _ in range(args.warmup):
        steps = step()
    stream.synchronize()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    served = {}
    e0.record(stream)
    for _ in range(args.steps):
        steps = step(counters=served)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    barrier()
    ms = max_over_ranks(ms, dist, "cuda")
    value = world * done_per_step / (ms / 1e3)
    acc = accuracy(xlist, rank_first_seed(rank, S), steps)
    if acc is not None:
        print(f"[bench] accuracy vs stored oracle x*: {acc['n_checked']} slices, max rel err {acc['max_rel_err']:.2e} "
              f"(seed {acc['worst_seed']}), median {acc['median_rel_err']:.2e}", file=sys.stderr, flush=True)
    steps = np.asarray(steps)
    steps = steps[steps > 0]
    print(f"[bench] {S} slices through {B} slots, <= {args.outer}x{args.inner}, stop {args.outer_tol}: "
          f"{ms:.1f} ms/step for {done_per_step} completions; outer steps mean {steps.mean():.1f} "
          f"max {steps.max()} capped {(steps >= args.outer).sum()}; PCG steps mean {np.mean(pcg_counts):.0f} "
          f"max {np.max(pcg_counts)}", file=sys.stderr, flush=True)

    # ---- per-kernel timing of one outer step over all B slots ----
    ctx.set_timing(True)
    one = F.make_params(1, args.inner, lam=LAM_W, lam_tv=LAM_TV, precond=args.precond)
    with torch.cuda.stream(stream):
        ctx.solve(b[:B], one, out=x[:B])
        ctx.solve(b[:B], one, out=x[:B])
    kt = ctx.get_timing()
    ctx.set_timing(False)
    print("[bench] per outer step: " + ", ".join(f"{k} {v[0]:.2f} ms/{v[1]}" for k, v in kt.items()),
          file=sys.stderr, flush=True)
    launches_per_outer = sum(v[1] for v in kt.values())
    kern = {k: {"ms_per_outer": round(v[0], 4), "launches": v[1], "applications": v[2]} for k, v in kt.items()}
    # operator applications per outer step (inner + 1 macro steps): the S
    # operator (three FFT passes and the wavelet term, one cluster launch) and
    # the ILU (first residual, then inner PCG steps) inner + 1 times each
    apps = {k: v[2] for k, v in kt.items()}
    dom = max((k for k in ALG_BYTES_PER_PX if kt[k][1] > 0), key=lambda k: kt[k][0])
    per_app_s = kt[dom][0] / apps[dom] / 1e3
    alg = ALG_BYTES_PER_PX[dom] * N * N * B
    achieved = alg / per_app_s / 1e9
    tkey = (dom, tuning.get("ilu_depth"))
    traffic = MEASURED_TRAFFIC_PER_PX[tkey] * N * N * B if tkey in MEASURED_TRAFFIC_PER_PX and N == 256 and B == 304 \
        else None
    for k in ALG_BYTES_PER_PX:  # op-apply bandwidth of every operator class, on algorithmic bytes
        if kt[k][0] > 0 and k in apps:
            kern[k]["alg_gbs"] = round(ALG_BYTES_PER_PX[k] * N * N * B / (kt[k][0] / apps[k] / 1e3) / 1e9, 1)
    peak, peak_source = hbm_peak()
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": peak_source,
                "alg_bytes_per_launch": alg, "launches_per_application": kt[dom][1] / apps[dom]}

    # ---- end to end through the public API with host buffers ----
    e2e = None
    if args.e2e_steps > 0:
        bh = torch.from_numpy(b_h).pin_memory()
        mh = torch.from_numpy(masks_h).pin_memory()
        xh = torch.empty(b_h.shape, dtype=torch.complex64).pin_memory()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            with torch.cuda.stream(stream):
                masks.copy_(mh, non_blocking=True)
                b.copy_(bh, non_blocking=True)
            step()
            with torch.cuda.stream(stream):
                xh.copy_(x, non_blocking=True)
            stream.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        e2e_s = max_over_ranks(e2e_s, dist, "cuda")
        e2e = {"value": world * done_per_step / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(bh.numel() * 8 + mh.numel()),
               "d2h_bytes_per_step": int(xh.numel() * 8)}

    # ---- the same queue with the ILU(0) variant of the TV preconditioner ----
    ilu0 = None
    # the measurements beside the main line run at N = 1 (the scaling runs time
    # the main line only)
    aux = world == 1
    if aux and args.ilu0_variant and args.precond == "paper":
        p_ilu = F.make_params(args.outer, args.inner, lam=LAM_W, lam_tv=LAM_TV, outer_tol=args.outer_tol,
                              stop_on_distance=True, stall_tol=args.stall_tol, pcg_late=ILU0_INNER_LATE,
                              outer_late=args.outer_late, boundary_period=args.boundary_period, precond="ilu0")
        pcg_ilu = [0] * S

        def ilu_step():
            with torch.cuda.stream(stream):
                return F.serve(ctx, mlist, blist, lams, lam_tvs, p_ilu, xlist, max_outer=args.outer,
                               chunk=SERVE_CHUNK, pcg_steps=pcg_ilu)

        ilu_step()
        stream.synchronize()
        e0.record(stream)
        for _ in range(args.ilu0_variant):
            ist = ilu_step()
        e1.record(stream)
        e1.synchronize()
        ims = max_over_ranks(e0.elapsed_time(e1) / args.ilu0_variant, dist, "cuda")
        iacc = accuracy(xlist, rank_first_seed(rank, S), ist)
        ist = np.asarray(ist)
        ilu0 = {"value": round(world * done_per_step / (ims / 1e3), 3), "unit": UNIT, "ms_per_step": round(ims, 3),
                "vs_paper": round(ms / ims, 4), "timed_steps": args.ilu0_variant, "warmup": 1,
                "precond": "ilu0 (Sec. 4.2's incomplete LU with updated pivots)", "inner": args.inner,
                "inner_late": ILU0_INNER_LATE, "outer_late": args.outer_late,
                "mean_outer_steps": round(float(ist.mean()), 2), "max_outer_steps": int(ist.max()),
                "mean_pcg_steps": round(float(np.mean(pcg_ilu)), 1), "max_pcg_steps": int(np.max(pcg_ilu)),
                "accuracy": iacc}
        print(f"[bench] ILU(0) variant: {ilu0['value']} recons/s ({ilu0['vs_paper']}x), PCG steps mean "
              f"{ilu0['mean_pcg_steps']}, accuracy max {iacc['max_rel_err'] if iacc else None}", file=sys.stderr,
              flush=True)

    # ---- preconditioner comparison (PCG iteration counts, untimed) ----
    pcg_iters = _aux(precond_comparison, F, torch, stream) if aux and args.precond_cmp else None
    if _ok(pcg_iters):
        print("[bench] PCG steps to 1e-6: " + json.dumps({k: v for k, v in pcg_iters.items()
                                                           if isinstance(v, dict)}), file=sys.stderr, flush=True)

    # ---- the uneven batch (four sizes in one graph), untimed w.r.t. the main line ----
    c4 = _aux(uneven_batch_run, F, torch, args) if aux and args.uneven else None
    if _ok(c4):
        print(f"[bench] uneven batch: {c4['value']} recons/s ({c4['s_per_batch']} s per 64 slices), "
              f"accuracy {json.dumps(c4['accuracy'])}", file=sys.stderr, flush=True)

    # ---- multi-contrast cross sections (joint sparsity), untimed w.r.t. the main line ----
    mt = _aux(multi_contrast_run, F, torch, args) if aux and args.mt_sets > 0 else None
    if _ok(mt):
        print(f"[bench] multi-contrast: {mt['value']} cross sections/s ({mt['s_per_batch']} s per "
              f"{args.mt_sets}), accuracy {json.dumps(mt['accuracy_vs_oracle_same_schedule'])}, "
              f"SNR {mt['snr_db_mean']} dB", file=sys.stderr, flush=True)

    # ---- overlapping tree groups at 512^2, untimed w.r.t. the main line ----
    tree = _aux(tree_run, F, torch, args) if aux and args.tree_slices > 0 else None
    if _ok(tree):
        print(f"[bench] tree groups 512^2: {tree['value']} recons/s ({tree['s_per_batch']} s per "
              f"{args.tree_slices}), accuracy {json.dumps(tree['accuracy_vs_oracle_same_schedule'])}, "
              f"SNR {tree['snr_db_mean']} dB", file=sys.stderr, flush=True)

    # ---- dense random projections (Sec. 5.3), untimed w.r.t. the main line ----
    dense = _aux(dense_run, F, torch, args) if aux and args.dense_problems > 0 else None
    if _ok(dense):
        print(f"[bench] dense A: {dense['value']} problems/s ({dense['us_per_pcg_step']} us per PCG step), rows "
              f"{dense['roofline_rows']['achieved']} GB/s ({dense['roofline_rows']['frac']} of peak), accuracy "
              f"{json.dumps(dense['accuracy_vs_oracle_same_schedule'])}", file=sys.stderr, flush=True)

    # ---- learned warm start (CNN trained on solver-generated pairs) ----
    learned = None
    if aux and args.learned:
        learned = _aux(run_learned, args, F, torch, stream, B, rank, world, dist, serve_queue)
    if _ok(learned):
        print(f"[bench] learned vs plain on {learned['heldout_slices']} held-out slices: "
              f"{learned['value']} vs {learned['plain_value']} recons/s ({learned['vs_plain']}x), "
              f"PCG steps {learned['mean_pcg_steps']} vs {learned['plain_mean_pcg_steps']}; steady state "
              f"{learned['steady']['value']} vs {learned['steady']['plain_value']} ({learned['steady']['vs_plain']}x)",
              file=sys.stderr, flush=True)

    out = None
    if rank == 0:
        cpu = cpu_baseline(args) if (world == 1 and not args.no_cpu_baseline) else None
        out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32 (FP64 PCG scalars)", "data": "synthetic",
               "config": workload_config(args, world, done_per_step),
               "roofline": roofline, "kernels_per_outer_step": kern,
               # kernels per macro step x macro steps run, plus 4 kernels per slot load and 1 per
               # retire or slot move
               "gpu_launches": int(launches_per_outer / (args.inner + 1) * served["runs"] * SERVE_CHUNK
                                   + 4 * served["loads"] + served["retires"] + served.get("moves", 0)),
               "clocks": clk, "e2e": e2e, "cpu_baseline": cpu,
               "solve_stats": {"mean_outer_steps": round(float(steps.mean()), 2), "max_outer_steps": int(steps.max()),
                               "capped": int((steps >= args.outer).sum()),
                               "mean_pcg_steps": round(float(np.mean(pcg_counts)), 1),
                               "max_pcg_steps": int(np.max(pcg_counts))},
               "accuracy": acc, "learned": learned, "pcg_iterations": pcg_iters, "uneven_batch": c4,
               "multi_contrast": mt, "dense_l1": dense, "tree_512": tree, "ilu0_variant": ilu0}
        print(json.dumps(out), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return out


HELDOUT_FIRST = 20000


def run_learned(args, F, torch, stream, B, rank, world, dist, serve_queue):
    """The learned warm start against the plain start (A^H b) on held-out
    slices: the CNN is trained (untimed) on pairs the solver generates (seeds
    10000..), then both starts serve the same `args.heldout` held-out 256^2
    TV + D4 slices (seeds 20000.., never trained on) through the same slots
    and stop rule.  Per start: wall time (the learned one including the CNN,
    data consistency and F_eps guard), PCG and outer steps per slice, and the
    error of the slices that have a stored oracle x*."""
    from paper_1411_5057_gb300 import learned as Lr
    import firls_synth as fs
    H = args.heldout
    first = HELDOUT_FIRST + rank * H
    masks_h, b_h = make_batch(H, first)
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        masks = torch.from_numpy(masks_h).cuda()
        b = torch.from_numpy(b_h).cuda()
        x = torch.empty_like(b)
        seeds = list(range(10000 + rank * args.learned_train, 10000 + (rank + 1) * args.learned_train))
        atb_t, masks_t, xt = Lr.generate_pairs(N, seeds, 50, args.inner)
        net = F.Cnn(N, 16, stream=stream)
        net.set_params(fs.cnn_init_weights(0))
        Lr.train(net, atb_t, masks_t, xt, epochs=args.learned_epochs, lr=1e-3, batch=16)
        prm = net.get_params()
        net.close()
        del atb_t, masks_t, xt
        # the CNN start runs in chunks of the largest divisor of H up to B slices
        Bc = max(k for k in range(1, B + 1) if H % k == 0)
        inf = F.Cnn(N, Bc, stream=stream)
        inf.set_params(prm)
        prep = F.Context(N, batch=Bc, stream=stream)
        x0 = torch.empty_like(b)
        one = F.make_params(1, 1, lam=LAM_W, lam_tv=LAM_TV)
    stream.synchronize()
    train_s = time.perf_counter() - t0
    ml, bl, xl = list(masks), list(b), list(x)
    kept = [0]
    pcg_plain, pcg_learned = [0] * H, [0] * H

    def plain_step(stop_after=None):
        return serve_queue(ml, bl, xl, pcg_plain, stop_after=stop_after)

    def learned_step(stop_after=None):
        kept[0] = 0
        with torch.cuda.stream(stream):
            for i in range(0, H, Bc):
                prep.set_operator(masks[i:i + Bc], F.PSI_TV | F.PSI_DB4, LEVELS)
                atb = prep.adjoint(b[i:i + Bc])
                xs, chosen = Lr.warm_start(prep, inf, b[i:i + Bc], atb, masks[i:i + Bc], one)
                x0[i:i + Bc].copy_(xs)
                kept[0] += int(sum(chosen))
        return serve_queue(ml, bl, xl, pcg_learned, x0s=list(x0), stop_after=stop_after)

    def timed(fn):
        fn()  # warm-up
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.learned_steps):
            st = fn()
        e1.record(stream)
        e1.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1) / args.learned_steps, dist, "cuda")
        acc = accuracy(xl, first, st)
        st = np.asarray(st)
        return ms, st, acc

    ms_p, st_p, acc_p = timed(plain_step)
    ms_l, st_l, acc_l = timed(learned_step)

    # steady state: the completions while the queue still refills every slot
    # (the learned pass includes the CNN start of all H slices)
    def steady(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        e0.record(stream)
        fn(stop_after=H - B)
        e1.record(stream)
        e1.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), dist, "cuda")

    sms_p, sms_l = steady(plain_step), steady(learned_step)
    inf.close()
    prep.close()
    v_p, v_l = world * H / (ms_p / 1e3), world * H / (ms_l / 1e3)
    return {"value": round(v_l, 3), "plain_value": round(v_p, 3), "unit": UNIT, "vs_plain": round(v_l / v_p, 4),
            "heldout_slices": H, "heldout_seeds": f"{first}..{first + H - 1}",
            "ms_per_step": round(ms_l, 3), "plain_ms_per_step": round(ms_p, 3),
            "mean_pcg_steps": round(float(np.mean(pcg_learned)), 1),
            "plain_mean_pcg_steps": round(float(np.mean(pcg_plain)), 1),
            "pcg_ratio": round(float(np.mean(pcg_learned)) / float(np.mean(pcg_plain)), 4),
            "max_pcg_steps": int(np.max(pcg_learned)), "plain_max_pcg_steps": int(np.max(pcg_plain)),
            "mean_outer_steps": round(float(st_l.mean()), 2), "plain_mean_outer_steps": round(float(st_p.mean()), 2),
            "max_outer_steps": int(st_l.max()), "plain_max_outer_steps": int(st_p.max()),
            "kept_cnn_start": kept[0], "train_instances": args.learned_train, "train_epochs": args.learned_epochs,
            "setup_s": round(train_s, 1), "accuracy": acc_l, "plain_accuracy": acc_p,
            "steady": {"completions": H - B, "value": round(world * (H - B) / (sms_l / 1e3), 3),
                       "plain_value": round(world * (H - B) / (sms_p / 1e3), 3), "vs_plain": round(sms_p / sms_l, 4),
                       "counted": "slices completed while the queue refills every slot (one pass each)"}}


XSTAR_DIR = os.path.join(ROOT, "tests", "golden", "xstar_tv_db4_256")


def stored_xstar():
    """{seed: (x*, estimated distance of x* to the limit)} written by
    tests/golden/make_xstar.py (FP64 oracle run to its limit)."""
    out = {}
    if os.path.isdir(XSTAR_DIR):
        for f in sorted(os.listdir(XSTAR_DIR)):
            if f.startswith("seed") and f.endswith(".npz"):
                z = np.load(os.path.join(XSTAR_DIR, f))
                out[int(f[4:-4])] = (z["x"].astype(np.complex128), float(z["dist_est"]))
    return out


def accuracy(xs, first_seed, steps=None):
    """Relative l2 error of each served result that has a stored oracle x*
    (untimed, after the timed steps)."""
    ref = stored_xstar()
    errs, seeds = [], []
    for seed, (xstar, _) in ref.items():
        i = seed - first_seed
        if 0 <= i < len(xs):
            x = xs[i].cpu().numpy().astype(np.complex128)
            errs.append(float(np.linalg.norm(x - xstar) / np.linalg.norm(xstar)))
            seeds.append(seed)
    if not errs:
        return None
    worst = int(np.argmax(errs))
    out = {"n_checked": len(errs), "max_rel_err": max(errs), "median_rel_err": float(np.median(errs)),
           "worst_seed": seeds[worst], "seeds": seeds, "rel_err": [round(e, 8) for e in errs],
           "reference": "FP64 oracle x* (tests/golden/xstar_tv_db4_256), estimated distance to its limit <= "
                        f"{max(ref[s][1] for s in seeds):.1e}"}
    if steps is not None:
        out["outer_steps"] = [int(steps[s - first_seed]) for s in seeds]
    return out


XSTAR_UNEVEN_DIR = os.path.join(ROOT, "tests", "golden", "xstar_uneven")
XMT_DIR = os.path.join(ROOT, "tests", "golden", "xmt_db4_256")


def uneven_batch_run(F, torch, args, reps=2):
    """The uneven batch: 64 slices, 16 each at 128^2, 192^2, 256^2 and 320^2
    (TV + D4, per-slice lambdas and mask ratios, seeds 1000..1063), solved
    together by firls_solve_multi (one context and stream per size, one
    graph) with the bench schedule.  Reconstructions per second over the 64,
    device-resident inputs, and the error of the slices that have a stored
    oracle x*.  Untimed set-up; `reps` timed solves after one warm-up."""
    import firls_synth as fs
    groups = {}
    for seed, p in zip(range(1000, 1064), fs.uneven_batch()):
        groups.setdefault(p.n, []).append((seed, p))
    sizes = sorted(groups)
    streams = [torch.cuda.Stream() for _ in sizes]
    ctxs, bs, ps, outs = [], [], [], []
    for n, st in zip(sizes, streams):
        probs = [p for _, p in groups[n]]
        with torch.cuda.stream(st):
            ctx = F.Context(n, batch=len(probs), stream=st)
            ctx.set_operator(torch.from_numpy(np.stack([p.mask for p in probs])).cuda(), probs[0].psi, probs[0].levels)
            b = torch.from_numpy(np.stack([p.b for p in probs]).astype(np.complex64)).cuda()
        ctxs.append(ctx)
        bs.append(b)
        outs.append(torch.empty_like(b))
        ps.append(F.make_params(args.outer, args.inner, lam_per_slice=[p.lam for p in probs],
                                lam_tv_per_slice=[p.lam_tv for p in probs], outer_tol=args.outer_tol,
                                stop_on_distance=True, stall_tol=args.stall_tol, pcg_late=args.inner_late,
                                outer_late=args.outer_late, boundary_period=args.boundary_period))
    torch.cuda.synchronize()
    F.solve_multi(ctxs, bs, ps, outs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        stats = F.solve_multi(ctxs, bs, ps, outs, stats=True)
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / reps
    outer = [s["outer_done"] for s in stats]
    errs = {}
    if os.path.isdir(XSTAR_UNEVEN_DIR):
        for n, out in zip(sizes, outs):
            for i, (seed, _) in enumerate(groups[n]):
                f = os.path.join(XSTAR_UNEVEN_DIR, f"seed{seed}.npz")
                if os.path.exists(f):
                    xs = np.load(f)["x"].astype(np.complex128)
                    x = out[i].cpu().numpy().astype(np.complex128)
                    errs[seed] = float(np.linalg.norm(x - xs) / np.linalg.norm(xs))
    for c in ctxs:
        c.close()
    return {"value": round(64 / sec, 3), "unit": UNIT, "s_per_batch": round(sec, 4),
            "workload": "64 slices, 16 each at 128^2/192^2/256^2/320^2, TV + D4, per-slice lambda and mask",
            "method": "firls_solve_multi: one graph over four contexts (one per size), bench schedule",
            "max_outer_steps_per_size": dict(zip([str(n) for n in sizes], outer)),
            "accuracy": {"n_checked": len(errs), "max_rel_err": max(errs.values()) if errs else None,
                         "rel_err_by_seed": errs}}


MT_OUTER, MT_INNER = 100, 20


def multi_contrast_run(F, torch, args, reps=2):
    """Multi-contrast reconstruction with joint wavelet sparsity (FIRLS_MT,
    Sec. 5.6): `args.mt_sets` cross sections of 3 contrasts at 256^2 (25 %
    masks, one per contrast, joint 4-level D4, lambda 1e-3, seeds 1..), all
    in one context with channels = 3, for the paper's budget of 100
    iterations (20 PCG steps each).  Cross sections per second with
    device-resident inputs; error against the FP64 oracle's result of the same
    schedule for the seeds stored, and the SNR against the phantoms.  Untimed
    set-up; `reps` timed solves after one warm-up."""
    import firls_synth as fs
    sets = args.mt_sets
    probs = [p for seed in range(1, sets + 1) for p in fs.mt_db4_256(seed)]
    p0 = probs[0]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = F.Context(p0.n, batch=len(probs), stream=stream)
        ctx.set_channels(3)
        ctx.set_operator(torch.from_numpy(np.stack([p.mask for p in probs])).cuda(), p0.psi, p0.levels)
        b = torch.from_numpy(np.stack([p.b for p in probs]).astype(np.complex64)).cuda()
        out = torch.empty_like(b)
        prm = F.make_params(MT_OUTER, MT_INNER, lam=p0.lam)
        ctx.solve(b, prm, out=out)
    stream.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for _ in range(reps):
            ctx.solve(b, prm, out=out)
    stream.synchronize()
    sec = (time.perf_counter() - t0) / reps
    x = out.cpu().numpy().astype(np.complex128)
    snr = [20 * np.log10(np.linalg.norm(p.x0) / np.linalg.norm(x[i] - p.x0)) for i, p in enumerate(probs)]
    errs = {}
    for seed in range(1, sets + 1):
        f = os.path.join(XMT_DIR, f"seed{seed}.npz")
        if os.path.exists(f):
            ref = np.load(f)["x"].astype(np.complex128)
            got = x[3 * (seed - 1):3 * seed]
            errs[seed] = max(float(np.linalg.norm(got[t] - ref[t]) / np.linalg.norm(ref[t])) for t in range(3))
    ctx.close()
    return {"value": round(sets / sec, 3), "unit": "cross sections/s (3 contrasts each)",
            "images_per_s": round(3 * sets / sec, 3), "s_per_batch": round(sec, 4),
            "workload": f"{sets} cross sections x 3 contrasts, 256^2, 25% masks, joint 4-level D4, lambda 1e-3",
            "method": "one context, channels = 3: joint weights, PCG on the stacked contrasts",
            "schedule": f"{MT_OUTER} outer x {MT_INNER} PCG (the paper's 100-iteration budget)",
            "accuracy_vs_oracle_same_schedule": {"n_checked": len(errs),
                                                 "max_rel_err": max(errs.values()) if errs else None},
            "snr_db_mean": round(float(np.mean(snr)), 2), "paper_s_per_cross_section": 4.6}


def _aux(fn, *a):
    """Run one measurement beside the main line; an exception in it is
    reported in its JSON key (and its traceback on stderr) instead of ending
    the run before the main line prints."""
    try:
        return fn(*a)
    except Exception as e:  # noqa: BLE001 - reported, not hidden
        import traceback
        traceback.print_exc(file=sys.stderr)
        return {"error": f"{type(e).__name__}: {e}"}


def _ok(r):
    return r is not None and "error" not in r


def hbm_peak():
    """The measured HBM copy bandwidth (GB/s) of the GB300s, else the fallback."""
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(peaks["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


TREE_OUTER, TREE_INNER = 100, 20
XTREE_DIR = os.path.join(ROOT, "tests", "golden", "xtree_db4_512")


def tree_run(F, torch, args, reps=2):
    """Overlapping group sparsity at 512^2 (5-level D4, parent-child tree
    groups of size 2, 15 % mask, sigma 0.005, lambda 2e-4; FIRLS_OG):
    `args.tree_slices` slices (seeds 3..) in one context for the paper's
    budget of 100 iterations (20 PCG steps each).  Reconstructions per second
    with device-resident inputs, the error against the FP64 oracle's stored
    result of the same schedule (seeds 3-4, tests/golden/make_xtree.py) and
    the mean SNR against the phantoms.  Untimed set-up; `reps` timed solves
    after one warm-up."""
    import firls_synth as fs
    S = args.tree_slices
    probs = [fs.tree_db4_512(seed=3 + i) for i in range(S)]
    p0 = probs[0]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = F.Context(p0.n, batch=S, stream=stream)
        ctx.set_operator(torch.from_numpy(np.stack([p.mask for p in probs])).cuda(), p0.psi, p0.levels,
                         torch.from_numpy(p0.groups).cuda())
        b = torch.from_numpy(np.stack([p.b for p in probs]).astype(np.complex64)).cuda()
        out = torch.empty_like(b)
        prm = F.make_params(TREE_OUTER, TREE_INNER, lam=p0.lam)
        ctx.solve(b, prm, out=out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(reps):
            ctx.solve(b, prm, out=out)
    e1.record(stream)
    e1.synchronize()
    sec = e0.elapsed_time(e1) / 1e3 / reps
    x = out.cpu().numpy().astype(np.complex128)
    snr = [20 * np.log10(np.linalg.norm(p.x0) / np.linalg.norm(x[i] - p.x0)) for i, p in enumerate(probs)]
    errs = {}
    for i in range(min(S, 2)):
        f = os.path.join(XTREE_DIR, f"seed{3 + i}.npz")
        if os.path.exists(f):
            ref = np.load(f)["x"].astype(np.complex128)
            errs[3 + i] = float(np.linalg.norm(x[i] - ref) / np.linalg.norm(ref))
    ctx.close()
    return {"value": round(S / sec, 3), "unit": UNIT, "s_per_batch": round(sec, 4),
            "workload": f"{S} slices 512^2, 5-level D4, parent-child tree groups (overlapping), lambda 2e-4",
            "schedule": f"{TREE_OUTER} outer x {TREE_INNER} PCG (the paper's 100-iteration budget)",
            "accuracy_vs_oracle_same_schedule": {"n_checked": len(errs),
                                                 "max_rel_err": max(errs.values()) if errs else None},
            "snr_db_mean": round(float(np.mean(snr)), 2)}


DENSE_OUTER, DENSE_INNER = 200, 30
XDENSE_DIR = os.path.join(ROOT, "tests", "golden", "xdense_l1")


def dense_run(F, torch, args, reps=2):
    """The dense random-projection workload (Sec. 5.3: signals of length
    4000 with 10 % non-zeros, 800 Gaussian measurements each, FIRLS_L1 with
    30 PCG steps per outer step for 200 outer steps): `args.dense_problems`
    problems, each with its own A (seeds 1..), in one context.  Problems per
    second with device-resident inputs; the HBM roofline of the row kernel
    (one pass over A per S d, timed through firls_dense_apply_AtA with CUDA
    events); the error against the FP64 oracle's stored result of the same
    schedule (seeds 1-2) and the MSE against the sparse truth.  Untimed
    set-up; `reps` timed solves after one warm-up."""
    import firls_synth as fs
    P = args.dense_problems
    M, Nd = 800, 4000
    A = np.empty((P, M, Nd), np.float32)
    bh = np.empty((P, M), np.float32)
    x0 = []
    for i in range(P):
        p = fs.dense_l1(i + 1)
        A[i], bh[i] = p.A, p.b
        x0.append(p.x0)
    lam = p.lam
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = F.DenseContext(M, Nd, P, stream=stream)
        At = torch.from_numpy(A).cuda()
        ctx.set_matrix(At)
        del At
        b = torch.from_numpy(bh).cuda()
        out = torch.empty(P, Nd, dtype=torch.float32, device="cuda")
        prm = F.make_params(DENSE_OUTER, DENSE_INNER, lam=lam)
        ctx.solve(b, prm, out=out)
    del A
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(reps):
            ctx.solve(b, prm, out=out)
    e1.record(stream)
    e1.synchronize()
    sec = e0.elapsed_time(e1) / 1e3 / reps
    # the row kernel alone: q = A^T A d over all problems (A is 12.8 MB per problem)
    with torch.cuda.stream(stream):
        d = torch.randn(P, Nd, device="cuda")
        q = torch.empty_like(d)
        for _ in range(3):
            ctx.apply_AtA(d, q)
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(20):
            ctx.apply_AtA(d, q)
    e1.record(stream)
    e1.synchronize()
    t_apply = e0.elapsed_time(e1) / 1e3 / 20
    abytes = P * M * Nd * 4
    x = out.cpu().numpy().astype(np.float64)
    errs = {}
    for seed in (1, 2):
        f = os.path.join(XDENSE_DIR, f"seed{seed}.npz")
        if seed <= P and os.path.exists(f):
            ref = np.load(f)["x"]
            errs[seed] = float(np.linalg.norm(x[seed - 1] - ref) / np.linalg.norm(ref))
    mse = float(np.mean([np.mean((x[i] - x0[i]) ** 2) for i in range(P)]))
    ctx.close()
    steps = DENSE_OUTER * (DENSE_INNER + 1)
    return {"value": round(P / sec, 3), "unit": "problems/s", "s_per_batch": round(sec, 4),
            "workload": f"{P} problems, A 800 x 4000 Gaussian (own A each), 10% non-zeros, lambda {lam}",
            "schedule": f"{DENSE_OUTER} outer x {DENSE_INNER} PCG (the paper's 30 PCG steps, converged in 200)",
            "us_per_pcg_step": round(sec / steps * 1e6, 1),
            "roofline_rows": {"bound": "hbm", "kernel": "k_dense_rows (+ k_dense_reduce)",
                              "achieved": round(abytes / t_apply / 1e9, 1), "peak": hbm_peak()[0], "unit": "GB/s",
                              "frac": round(abytes / t_apply / 1e9 / hbm_peak()[0], 3),
                              "algorithmic_bytes": abytes, "us_per_apply": round(t_apply * 1e6, 1)},
            "accuracy_vs_oracle_same_schedule": {"n_checked": len(errs),
                                                 "max_rel_err": max(errs.values()) if errs else None},
            "mse_vs_truth_mean": round(mse, 4), "paper_mse": "0.0427-0.0481 (FIRLS_L1, Table 1)",
            "shared_matrix": dense_shared_run(F, torch, args) if args.dense_shared_problems > 0 else None}


def dense_shared_run(F, torch, args, reps=2):
    """The same workload with one A shared by `args.dense_shared_problems`
    signals (firls_synth.dense_l1_shared(1, P): problem 0 is dense_l1(1)),
    where S d for all problems is two FP32 GEMMs (T = D A^T, Q = T A).
    Problems per second for the 200 x 30 schedule with device-resident
    inputs; the GEMM pair's FLOP rate against the FP32 FMA peak of the SMs
    (SMs x 128 lanes x 2 flops x 2.07 GHz), timed through
    firls_dense_apply_AtA with CUDA events; problem 0 against the FP64
    oracle's stored result of dense_l1(1); the MSE against the truth."""
    import firls_synth as fs
    P = args.dense_shared_problems
    M, Nd = 800, 4000
    A, B, X0, lam = fs.dense_l1_shared(1, P)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = F.DenseContext(M, Nd, P, shared=True, stream=stream)
        ctx.set_matrix(torch.from_numpy(A.astype(np.float32)).cuda())
        b = torch.from_numpy(B.astype(np.float32)).cuda()
        out = torch.empty(P, Nd, dtype=torch.float32, device="cuda")
        prm = F.make_params(DENSE_OUTER, DENSE_INNER, lam=lam)
        ctx.solve(b, prm, out=out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(reps):
            ctx.solve(b, prm, out=out)
    e1.record(stream)
    e1.synchronize()
    sec = e0.elapsed_time(e1) / 1e3 / reps
    with torch.cuda.stream(stream):
        d = torch.randn(P, Nd, device="cuda")
        q = torch.empty_like(d)
        for _ in range(3):
            ctx.apply_AtA(d, q)
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(20):
            ctx.apply_AtA(d, q)
    e1.record(stream)
    e1.synchronize()
    t_apply = e0.elapsed_time(e1) / 1e3 / 20
    flops = 4.0 * P * M * Nd
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sms * 128 * 2 * 2.07e9 / 1e12
    x = out.cpu().numpy().astype(np.float64)
    ctx.close()
    f = os.path.join(XDENSE_DIR, "seed1.npz")
    err = None
    if os.path.exists(f):
        ref = np.load(f)["x"]
        err = float(np.linalg.norm(x[0] - ref) / np.linalg.norm(ref))
    return {"value": round(P / sec, 3), "unit": "problems/s", "s_per_batch": round(sec, 4),
            "workload": f"{P} signals, one A 800 x 4000 Gaussian, 10% non-zeros each, lambda {lam}",
            "roofline_gemm": {"bound": "alu", "kernel": "k_dense_gemm (x2) + k_dense_sum_splits",
                              "achieved": round(flops / t_apply / 1e12, 2), "peak": round(peak, 1),
                              "unit": "TFLOP/s", "frac": round(flops / t_apply / 1e12 / peak, 3),
                              "peak_derivation": f"{sms} SMs x 128 FP32 lanes x 2 flops x 2.07 GHz",
                              "us_per_apply": round(t_apply * 1e6, 1)},
            "accuracy_vs_oracle_same_schedule": {"n_checked": 0 if err is None else 1, "max_rel_err": err},
            "mse_vs_truth_mean": round(float(np.mean((x - X0) ** 2)), 4)}


def precond_comparison(F, torch, stream, outer_steps=(1, 5, 20), tol=1e-6, cap=5000):
    """PCG steps to ||r|| <= tol ||A^H b|| with the proposed P, Jacobi and no
    preconditioner (Sec. 5.2, Fig. 2 and the TV figure), and with TV also the
    ILU(0) factors with updated pivots (Sec. 4.2's incomplete LU), from the iterates of
    the proposed PCG's own FIRLS trajectory (20 PCG steps per outer step) at
    the given outer steps; workload 1 (64^2 Haar l1, real) and one 256^2
    TV + D4 slice (seed 2).  Untimed."""
    import firls_synth as fs
    out = {"tol_rel_residual": tol, "cap": cap, "trajectory_inner": 20}
    for name, p in (("haar_l1_64", fs.haar_l1_64()), ("tv_db4_256", problem(2))):
        with torch.cuda.stream(stream):
            ctx = F.Context(p.n, batch=1, real=p.real, stream=stream)
            ctx.set_operator(torch.from_numpy(p.mask).cuda()[None], p.psi, p.levels)
            b = torch.from_numpy(p.b.astype(np.complex64)).cuda()[None]
            rows = {}
            for k in outer_steps:
                x0 = None
                if k > 1:
                    x0 = ctx.solve(b, F.make_params(k - 1, 20, lam=p.lam, lam_tv=p.lam_tv)).clone()
                row = {}
                for pre in ("paper", "jacobi", "none") + (("ilu0",) if p.psi & fs.PSI_TV else ()):
                    _, st = ctx.solve(b, F.make_params(1, cap, lam=p.lam, lam_tv=p.lam_tv, pcg_tol=tol,
                                                       precond=pre), x0=x0, stats=True)
                    row[pre] = int(st["pcg_steps"])
                rows[f"outer_step_{k}"] = row
            ctx.close()
        out[name] = rows
    return out


def workload_config(args, world, done_per_step=None):
    """The workload both arms report: the served 256^2 TV + D4 queue."""
    return {"workload": f"firls_tv_db4_{N}", "n": N, "slices_per_step_per_gpu": args.queue, "slots": args.batch,
            "outer_max": args.outer, "inner": args.inner, "inner_late": args.inner_late,
            "outer_late": args.outer_late, "outer_tol": args.outer_tol, "stall_tol": args.stall_tol,
            "boundary_period": args.boundary_period, "precond": args.precond,
            "mask_ratio": RATIO, "sigma": SIGMA, "lambda_tv": LAM_TV, "lambda_w": LAM_W,
            "wavelet": "db4", "levels": LEVELS, "batching": "continuous (slots refilled on convergence)",
            "completions_per_step": args.queue if done_per_step is None else done_per_step,
            "counted": ("steady state: slices completed while the queue refills every slot; "
                        "slices still in flight at the end are retired uncounted") if args.steady
            else "every slice of the queue, including the drain",
            "l2": "working set > L2 (no flush needed)", "parallelism": f"replicas{world}"}


def oracle_sample(outer_steps, seed=2):
    """Time ``outer_steps`` FIRLS outer steps of the FP64 oracle on one slice."""
    from oracle import firls_oracle as O
    p = problem(seed)
    t0 = time.perf_counter()
    O.firls_problem(p, outer=outer_steps, inner=ARGS_INNER[0])
    return time.perf_counter() - t0


ORACLE_INNER = 60   # the oracle's schedule: 60 PCG steps per outer step
ARGS_INNER = [ORACLE_INNER]


def cpu_baseline(args):
    """The FP64 oracle as it stands (its own schedule: 60 PCG steps per outer
    step) on one host core: one outer step of one slice, scaled by the
    oracle's own mean outer steps to 1e-4 of x* on the stored seeds."""
    env_threads = 1
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = str(env_threads)
    ARGS_INNER[0] = ORACLE_INNER
    sec = oracle_sample(args.ref_outer)
    outer, covered = oracle_outer_per_recon(range(2, 18))
    recon_s = sec / args.ref_outer * outer
    return {"value": round(1.0 / recon_s, 6), "unit": UNIT, "cores": env_threads, "kind": "oracle",
            "sample": f"FP64 oracle, one {N}^2 slice, {args.ref_outer} outer step(s) x {ORACLE_INNER} PCG "
                      f"({sec:.1f} s), scaled to {outer:.1f} outer steps per reconstruction (the oracle's own mean "
                      f"to 1e-4 of its x* on seeds {covered or [2]})"}


def _oracle_worker(a):
    """One oracle sample in a worker process: (outer steps, PCG steps, seed)."""
    outer, inner, seed = a
    ARGS_INNER[0] = inner
    return oracle_sample(outer, seed)


def oracle_outer_per_recon(seeds):
    """Mean of the FP64 oracle's own outer steps (60 PCG each) to 1e-4 of x*
    on the given seeds, as stored by tests/golden/make_xstar.py (--steps-to),
    and the seeds it covers; REF_OUTER_PER_RECON where none is stored."""
    got = []
    for s in seeds:
        f = os.path.join(XSTAR_DIR, f"seed{s}.npz")
        if os.path.exists(f):
            z = np.load(f)
            if "outer_to_1e4" in z.files:
                got.append((s, int(z["outer_to_1e4"])))
    if not got:
        return float(REF_OUTER_PER_RECON), []
    return float(np.mean([v for _, v in got])), [s for s, _ in got]


def host_cores():
    """Cores this process may run on (affinity / cgroup), not the host's count."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return None
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"  # one thread per oracle instance (inherited by the workers)
    ARGS_INNER[0] = args.ref_inner
    procs = args.ref_procs if args.ref_procs > 0 else host_cores()
    seeds = [2 + i for i in range(procs)]
    if procs == 1:
        oracle_sample(1)  # warm-up: imports and first-touch costs
        for _ in range(args.warmup):
            oracle_sample(1)
        t = [oracle_sample(args.ref_outer) for _ in range(args.steps)]
    else:
        # one independent slice per host core (seeds 2, 3, ...), all at once;
        # a step takes as long as its slowest worker
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(procs) as pool:
            for _ in range(max(1, args.warmup)):
                pool.map(_oracle_worker, [(1, args.ref_inner, s) for s in seeds])
            t = [max(pool.map(_oracle_worker, [(args.ref_outer, args.ref_inner, s) for s in seeds]))
                 for _ in range(args.steps)]
    sec = float(np.mean(t))
    outer, covered = oracle_outer_per_recon(seeds)
    value = procs * (args.ref_outer / outer) / sec
    how = (f"the mean of the oracle's own outer steps to 1e-4 of its x* on seeds {covered}" if covered else
           f"{REF_OUTER_PER_RECON} outer steps (the oracle's own outer steps to 1e-4 of x* on seed 2)")
    cpu = {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
           "sample": f"FP64 oracle, {procs} independent {N}^2 slice(s) at once, one per host core, each "
                     f"{args.ref_outer} outer step(s) x {args.ref_inner} PCG per bench step, scaled to {outer:.1f} "
                     f"outer steps per reconstruction ({how})"}
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(args, world),
           "cpu_baseline": cpu, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return out


def profile_step(args):
    """Profiling target (no timing, no JSON line): one outer step of 60 PCG
    steps (61 macro steps) of the 256^2 TV + D4 workload on --profile-step
    slices, run twice, with the given ILU ring shape (0: the default)."""
    import torch
    import paper_1411_5057_gb300 as F
    B = args.profile_step
    masks_h, b_h = make_batch(B, 2)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        masks = torch.from_numpy(masks_h).cuda()
        b = torch.from_numpy(b_h).cuda()
        ctx = F.Context(N, batch=B, stream=stream)
        ctx.set_operator(masks, F.PSI_TV | F.PSI_DB4, LEVELS)
        ctx.set_tuning(rows_per_cta=1, coarse_max=64, ilu_depth=args.profile_ilu_shape)
        one = F.make_params(1, INNER, lam=LAM_W, lam_tv=LAM_TV)
        for _ in range(2):
            ctx.solve(b, one)
    stream.synchronize()
    ctx.close()
    print(f"[bench] profile step: {B} slices, one outer step x2", file=sys.stderr)


def profile_dense(args):
    """Profiling target (no timing, no JSON line): q = A^T A d on
    --profile-dense problems of the dense workload's shape (800 x 4000, own A
    each, or one shared A with --profile-dense-shared; seeded device draws),
    five applications."""
    import torch
    import paper_1411_5057_gb300 as F
    P, M, Nd = args.profile_dense, 800, 4000
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        shared = bool(args.profile_dense_shared)
        A = torch.randn(1 if shared else P, M, Nd, device="cuda", generator=g) / math.sqrt(M)
        ctx = F.DenseContext(M, Nd, P, shared=shared, stream=stream)
        ctx.set_matrix(A)
        del A
        d = torch.randn(P, Nd, device="cuda", generator=g)
        q = torch.empty_like(d)
        for _ in range(5):
            ctx.apply_AtA(d, q)
    stream.synchronize()
    ctx.close()
    print(f"[bench] profile dense: {P} problems ({'shared' if shared else 'own'} A), five applications",
          file=sys.stderr)


def build_parser():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=304, help="slots solved concurrently")
    ap.add_argument("--queue", type=int, default=608, help="slices entering the slots per step")
    ap.add_argument("--steady", type=int, default=0,
                    help="1: count the queue minus one batch of completions (slots full); 0: drain everything")
    ap.add_argument("--outer", type=int, default=OUTER)
    ap.add_argument("--inner", type=int, default=INNER)
    ap.add_argument("--outer-tol", type=float, default=OUTER_TOL)
    ap.add_argument("--inner-late", type=int, default=INNER_LATE, help="PCG steps per outer step from --outer-late on")
    ap.add_argument("--outer-late", type=int, default=OUTER_LATE)
    ap.add_argument("--boundary-period", type=int, default=BOUNDARY_PERIOD,
                    help="macro steps between outer-step transitions of the served slots")
    ap.add_argument("--stall-tol", type=float, default=STALL_TOL)
    ap.add_argument("--precond", default="paper", choices=["paper", "ilu0", "jacobi", "none"],
                    help="PCG preconditioner of the served queue (paper: the printed L U factors of Sec. 4.2)")
    ap.add_argument("--autotune", type=int, default=1, help="autotune tile shapes before timing (1/0)")
    ap.add_argument("--learned", type=int, default=1, help="also time the learned warm start (1/0)")
    ap.add_argument("--learned-train", type=int, default=4000, help="training instances solved by the method")
    ap.add_argument("--learned-epochs", type=int, default=10)
    ap.add_argument("--heldout", type=int, default=512, help="held-out slices of the learned comparison")
    ap.add_argument("--learned-steps", type=int, default=2, help="timed passes per start over the held-out slices")
    ap.add_argument("--ref-outer", type=int, default=1, help="oracle outer steps per sample")
    ap.add_argument("--ref-inner", type=int, default=ORACLE_INNER, help="oracle PCG steps per outer step")
    ap.add_argument("--ref-procs", type=int, default=0,
                    help="reference arm: oracle instances run at once, one per host core (0: all cores)")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--uneven", type=int, default=1, help="also time the 64-slice uneven batch (1/0)")
    ap.add_argument("--ilu0-variant", type=int, default=1,
                    help="timed passes of the queue with the ILU(0) preconditioner after one warm-up (0: none)")
    ap.add_argument("--tree-slices", type=int, default=32,
                    help="512^2 tree-group slices timed beside the main line (0: none)")
    ap.add_argument("--dense-shared-problems", type=int, default=256,
                    help="signals sharing one A in the dense measurement (0: skip)")
    ap.add_argument("--dense-problems", type=int, default=152,
                    help="dense random-projection problems timed beside the main line (0: none)")
    ap.add_argument("--mt-sets", type=int, default=100,
                    help="multi-contrast cross sections timed beside the main line (0: none)")
    ap.add_argument("--precond-cmp", type=int, default=1,
                    help="report PCG steps to 1e-6 for the proposed, Jacobi and no preconditioner (1/0)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-step", type=int, default=0,
                    help="profiling target only: one outer step on this many slices, twice")
    ap.add_argument("--profile-ilu-shape", type=int, default=0)
    ap.add_argument("--profile-dense", type=int, default=0,
                    help="profiling target: q = A^T A d on this many dense problems, no timing")
    ap.add_argument("--profile-dense-shared", type=int, default=0, help="1: one A shared by the profiled problems")
    return ap


def main(argv=None):
    args = build_parser().parse_args(argv)
    if args.profile_step > 0:
        return profile_step(args)
    if args.profile_dense > 0:
        return profile_dense(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    main()
