"""Benchmark: batched plain pressure projection on GB300.

Workload (one step): 16 independent 512 x 512 MAC grids, initial velocity a sum
of 32 seeded Gaussian vortices, 1-6 solid rectangles/discs per grid, each grid
projected by masked Jacobi until mean|div u| <= 1e-4 (cap 5000 sweeps), then
corrected.  Metric: projections per second (one projection = one grid taken
from u* to the corrected u).  Inputs are synthetic and seeded; they are
resident in HBM when the timed region starts (device-to-device restore of u*
is inside the step, L2 is flushed between steps).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank projects its own 16 grids (weak scaling, no
collective on the data path); the max time over ranks is reported.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "projections/s at fixed mean|div|: CNN-hybrid vs plain Jacobi; % HBM roofline"
UNIT = "projections/s"
B, N, THR, CAP = 16, 512, 1e-4, 5000
# cap under which every grid of the workload converges with a zero guess
# (the slowest needs 26,199 sweeps in the FP64 oracle)
CAP_UNCAPPED, UNCAPPED_STEPS = 40000, 3
# fixed Jacobi sweeps behind each 128^2 training target (about 0.5 % relative
# L2 error against the exact solve)
TRAIN_SWEEPS = 40000
# multiply-adds per full-resolution pixel of each network: the scale-1 branch,
# a quarter of the scale-1/2 branch, a sixteenth of the scale-1/4 branch
# (MultiScale 148,608 + 148,608 / 4 + 74,592 / 16; SmallScale 47,232 +
# 47,232 / 4 + 28,512 / 16); the MonoScale's one branch 222,048; the Unet's
# levels n .. n/16 weighted by 1, 1/4, .., 1/256
CNN_MACS_PER_PIXEL = {"multiscale": 190422, "smallscale": 60822, "monoscale": 222048,
                      "unet": 68000}
NETWORKS = ("multiscale", "smallscale", "monoscale", "unet")  # trained in the hybrid arm
FORWARD_NETWORKS = NETWORKS
# held-out grids of the training distribution for the in-distribution comparison
IN_DIST_GRIDS, IN_DIST_SEED = 256, 100000
T_BLOCK = 8
BYTES_PER_CELL_SWEEP = 13  # read phi 4, div 4, mask 1; write phi 4
# FP32 operations of one masked Jacobi cell update in increment form: the two
# neighbour differences it owns (each difference serves two cells), 3 adds,
# the closed-face, residual and update FMAs, the |r| add
OPS_PER_CELL_UPDATE = 9
WORKLOAD = ("16 x 512^2 MAC grids, 32 Gaussian vortices + 1-6 obstacles each, plain Jacobi "
            "to mean|div| <= 1e-4 (cap 5000), FP32 sweeps, FP64 stop test")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(value: float, device) -> float:
    """The largest value over all ranks (the step time of the slowest GPU);
    timing only, nothing on the data path is exchanged."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_inputs(rank: int):
    from paper_2109_09363_gb300 import workloads as W
    u, v, fl = W.batched_vortex_case(B, N, seed0=rank * B)
    return u.astype(np.float32), v.astype(np.float32), fl


def cpu_oracle_sample(u, v, fl, budget_s=20.0, gpu=None):
    """Time the FP64 oracle projection on whole grids until ~budget_s of work.
    With the GPU's results of the same grids (gpu = (iters, u, v) on the host)
    the oracle's results also give the parity of the benchmark run itself."""
    import oracle
    oracle.build()
    cores = oracle.set_threads(0)
    done, t0 = 0, time.perf_counter()
    refs = []
    while True:
        b = done % B
        refs.append(oracle.project(u[b].astype(np.float64), v[b].astype(np.float64), fl[b],
                                   THR, CAP, hist_len=CAP + 2))
        done += 1
        el = time.perf_counter() - t0
        if el >= budget_s or done >= B:
            break
    res = {"value": done / el, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{done} of the {B} grids (512^2, full projection each), FP64 C oracle, "
                     f"{el:.1f} s"}
    # the same oracle on one host core: the first grid's full projection
    oracle.set_threads(1)
    t1 = time.perf_counter()
    oracle.project(u[0].astype(np.float64), v[0].astype(np.float64), fl[0], THR, CAP)
    e1 = time.perf_counter() - t1
    oracle.set_threads(cores)
    res["single_thread"] = {"value": 1.0 / e1, "unit": UNIT, "cores": 1,
                            "sample": f"grid 0 (512^2, full projection), {e1:.1f} s"}
    # the oracle network (FP64 numpy): one MultiScale forward of one 128^2 grid
    from oracle import cnn as OC
    g = np.random.default_rng(0)
    params = OC.init_params(seed=0)
    t2 = time.perf_counter()
    OC.forward(params, g.standard_normal((128, 128)), (g.random((128, 128)) < 0.1).astype(np.uint8))
    res["cnn_forward_128"] = {"ms": (time.perf_counter() - t2) * 1e3,
                              "sample": "one MultiScale forward of one 128^2 grid, FP64 numpy oracle"}
    if gpu is not None:
        it_g, u_g, v_g = gpu
        equal, near_tie, err = 0, 0, 0.0
        for b, ref in enumerate(refs[:B]):
            ko, kg = int(ref["iters"][0]), int(it_g[b])
            if ko == kg:
                equal += 1
                umax = max(np.abs(ref["u"]).max(), np.abs(ref["v"]).max())
                err = max(err, np.abs(u_g[b] - ref["u"][0]).max() / umax,
                          np.abs(v_g[b] - ref["v"][0]).max() / umax)
            else:
                lo, hi = sorted((ko, kg))
                eh = ref["e_hist"][0, lo:hi + 1]
                eh = eh[np.isfinite(eh)]  # the oracle's history ends at its own stop
                near_tie += int(eh.size > 0 and np.all(np.abs(eh - THR) / THR <= 5e-5))
        res["parity"] = {"grids": min(done, B), "iters_equal": equal,
                         "iters_differ_at_a_near_tie": near_tie,
                         "max_velocity_error_rel": err,
                         "note": "the benchmark's own last step against the FP64 oracle: "
                                 "iteration counts, and max |u - u_oracle| / max |u_oracle| "
                                 "where the counts agree"}
    return res


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    u, v, fl = make_inputs(0)
    import oracle
    oracle.build()
    cores = oracle.set_threads(0)
    # each step: one grid (a bounded sample of the 16-grid workload)
    for s in range(args.warmup):
        b = s % B
        oracle.project(u[b].astype(np.float64), v[b].astype(np.float64), fl[b], THR, CAP)
    t0 = time.perf_counter()
    for s in range(args.steps):
        b = s % B
        oracle.project(u[b].astype(np.float64), v[b].astype(np.float64), fl[b], THR, CAP)
    el = time.perf_counter() - t0
    val = args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "method": "plain Jacobi (FP64 CPU oracle)",
                       "step": "one 512^2 grid of the 16-grid batch"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "one 512^2 grid per step, full projection"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def streaming_chosen(kernel: int, cells: int) -> bool:
    """The library's sweep-kernel choice (hp_project with sweep_kernel = 0)."""
    return kernel == 1


def profile_sweep(batch: int, n: int, sweeps: int, host_loop: bool = False,
                  kernel: int = 0) -> int:
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2109_09363_gb300 as hp
    from paper_2109_09363_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    us, vs, fs = [], [], []
    for b in range(batch):
        u, v = W.vortex_velocity(n, n, 1000 + b, n_vortices=32)
        us.append(u); vs.append(v)
        fs.append(W.random_obstacles(n, n, 2000 + b))
    u = torch.from_numpy(np.stack(us).astype(np.float32)).to(dev)
    v = torch.from_numpy(np.stack(vs).astype(np.float32)).to(dev)
    fl = torch.from_numpy(np.stack(fs)).to(dev)
    ctx = hp.Context(batch, n, n)
    times = []
    if host_loop:
        prm = hp.ProjectParams(fixed_iters=sweeps, temporal_block=T_BLOCK, use_graph=0,
                               sweep_kernel=kernel)
        uw, vw = torch.empty_like(u), torch.empty_like(v)
        for _ in range(3):
            uw.copy_(u)
            vw.copy_(v)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            hp.hp_project(ctx, uw, vw, fl, prm)
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
    else:
        div = hp.hp_divergence(u, v, fl)
        phi = torch.zeros_like(div)
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            hp.hp_jacobi_sweeps(ctx, phi, div, fl, sweeps)
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
    torch.cuda.synchronize()
    # the last call, whole projection (host loop) or sweeps only; effective
    # bandwidth = 13 B per cell-sweep
    ms = times[-1]
    print(json.dumps({"profile_sweep": [batch, n, sweeps], "ok": True, "ms_last_call": ms,
                      "effective_gbs": BYTES_PER_CELL_SWEEP * batch * n * n * sweeps /
                      (ms * 1e-3) / 1e9}))
    ctx.close()
    return 0


def run_hybrid_arm(args, hp, u0, v0, fl, u, v, ctx, prm, flush, stream, ms_plain, ws):
    """CNN-hybrid projection of the same grids to the same threshold, with the
    MultiScale, the SmallScale and the MonoScale network (Sec. 3.1).

    Untimed set-up (10,000 pairs, 20 epochs, batch 64): training pairs from the plain solver
    (128^2, vortex field + divergence sources + 0-4 obstacles), Adam training
    of each network on the GPU with the same pairs and schedule (batch 64,
    lr 1e-3).  Timed: the same per-step protocol as the plain arm (device
    restore of u*, L2 flush between steps, CUDA events).  Then, with the same
    networks, the 1024^2 plume with a cylinder and the 2048^2 plume with eight
    cylinders (large_plumes)."""
    import torch
    from paper_2109_09363_gb300 import training as T
    from paper_2109_09363_gb300 import workloads as W
    t0 = time.perf_counter()
    n_tr = 128
    data = T.generate_pairs(args.train_pairs, n_tr, seed0=0, sweeps=TRAIN_SWEEPS,
                            device=u0.device)
    torch.cuda.synchronize()
    t_pairs = time.perf_counter() - t0
    batch = 64
    epochs = args.train_epochs
    trained, train_info = {}, {}
    for arch in NETWORKS:
        t1 = time.perf_counter()
        cnn = hp.CNN(batch, n_tr, n_tr, params=T.init_params(seed=1, arch=arch), arch=arch)
        losses = T.train(cnn, data, epochs=epochs, batch=batch, lr=1e-3, lambda_div=1.0)
        trained[arch] = cnn.get_params()
        cnn.close()
        train_info[arch] = {"steps": len(losses), "final_loss": float(np.mean(losses[-20:])),
                            "seconds": time.perf_counter() - t1}
    del data

    def time_capped(net):
        res = None

        def step():
            nonlocal res
            u.copy_(u0)
            v.copy_(v0)
            res = hp.hp_project_hybrid(ctx, net, u, v, fl, prm, out=res)

        for _ in range(max(args.warmup, 3)):
            step()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for s_ in range(args.steps):
            flush.fill_(float(s_))
            ev[s_][0].record(stream)
            step()
            ev[s_][1].record(stream)
        torch.cuda.synchronize()
        return sum(a_.elapsed_time(b2) for a_, b2 in ev) / args.steps, res

    def time_inference(net):
        # inference alone (t_inf of the paper)
        div = hp.hp_divergence(u0, v0, fl)
        a_, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        hp.hp_cnn_forward(net, div, fl)
        a_.record(stream)
        for _ in range(5):
            hp.hp_cnn_forward(net, div, fl)
        b2.record(stream)
        torch.cuda.synchronize()
        return a_.elapsed_time(b2) / 5

    # the same grids and threshold with the cap lifted far enough that every
    # grid converges in both arms: projections/s at equal mean|div|
    prm_u = hp.ProjectParams(threshold=THR, max_iters=CAP_UNCAPPED, temporal_block=T_BLOCK,
                             use_graph=prm.use_graph, sweep_kernel=prm.sweep_kernel)

    def time_uncapped(net):
        res = None

        def ustep():
            nonlocal res
            u.copy_(u0)
            v.copy_(v0)
            if net is None:
                res = hp.hp_project(ctx, u, v, fl, prm_u, out=res)
            else:
                res = hp.hp_project_hybrid(ctx, net, u, v, fl, prm_u, out=res)

        ustep()
        torch.cuda.synchronize()
        ev_u = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(UNCAPPED_STEPS)]
        for s_, (e0, e1) in enumerate(ev_u):
            flush.fill_(float(s_))
            e0.record(stream)
            ustep()
            e1.record(stream)
        torch.cuda.synchronize()
        ms_u = sum(a_.elapsed_time(b2) for a_, b2 in ev_u) / UNCAPPED_STEPS
        return {"value": ws * B / (ms_u * 1e-3), "ms_per_step": ms_u,
                "iters_per_grid": res["iters"].cpu().numpy().tolist(),
                "converged": int(res["converged"].sum().item()),
                "e1_max": float(res["e1"].max().item())}

    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    tpk = float(peaks.get("bf16_tflops", 1900.0))
    uncapped_plain = time_uncapped(None)
    arms = {}
    for arch in NETWORKS:
        net = hp.CNN(B, N, N, params=trained[arch], arch=arch)
        ms, out = time_capped(net)
        t_inf = time_inference(net)
        unc = time_uncapped(net)
        # MACs per full-resolution pixel: the scale-1 branch, a quarter of the
        # scale-1/2 branch and a sixteenth of the scale-1/4 branch
        flop = 2.0 * CNN_MACS_PER_PIXEL[arch] * B * N * N
        tf = flop / (t_inf * 1e-3) / 1e12
        t_roof = cnn_layer_roofline(arch, B * N * N, float(peaks.get("hbm_gbs", 6800.0)), tpk)
        arms[arch] = {
            "params": net.n_params, "value": ws * B / (ms * 1e-3), "unit": UNIT,
            "ms_per_step": ms, "speedup_vs_plain": ms_plain / ms,
            "iters_per_grid": out["iters"].cpu().numpy().tolist(),
            "converged": int(out["converged"].sum().item()),
            "t_inf_ms_16_grids": t_inf,
            "cnn_roofline": {"bound": "tensor", "achieved": tf, "peak": tpk, "unit": "TFLOP/s",
                             "frac": tf / tpk,
                             "peak_kind": "measured" if peaks else "fallback",
                             "note": "whole network forward (BF16, FP32 accumulate), "
                                     f"{2 * CNN_MACS_PER_PIXEL[arch] / 1e3:.1f} kFLOP per "
                                     "full-resolution pixel",
                             "layer_roofline_ms": t_roof, "frac_of_layer_roofline": t_roof / t_inf,
                             "layer_roofline_note": "every kernel at its own bound (HBM bytes "
                                                    "or tensor FLOPs, measured peaks), summed: "
                                                    "most layers sit at or below the ridge"},
            "equal_threshold_uncapped": {"hybrid": unc, "plain": uncapped_plain,
                                         "cap": CAP_UNCAPPED, "steps": UNCAPPED_STEPS,
                                         "speedup": uncapped_plain["ms_per_step"] /
                                         unc["ms_per_step"]},
            "training": dict(train_info[arch], pairs=args.train_pairs, grid=[n_tr, n_tr],
                             target_sweeps=TRAIN_SWEEPS, batch=batch, epochs=epochs,
                             pair_generation_seconds=t_pairs)}
        net.close()
    ms_arm = arms.pop("multiscale")
    in_dist = compare_in_distribution(hp, trained, flush, stream, u0.device, ws)
    heads128 = {}
    plume = compare_plume_same_threshold(hp, trained, u0.device, heads_out=heads128)
    # the paper's size (Sec. 2.1, 512^2), networks trained at 128^2 as in Sec. 3.2
    plume512 = compare_plume_same_threshold(hp, trained, u0.device, n=512, steps=300)
    plume_min = compare_plume_min_threshold(hp, trained, u0.device,
                                            reference=heads128.get("plain"))
    ms_arm["in_distribution_128"] = in_dist
    ms_arm["plume_same_threshold"] = plume
    ms_arm["plume_same_threshold_512"] = plume512
    ms_arm["plume_min_threshold"] = plume_min
    for arch in NETWORKS[1:]:
        ms_arm[arch] = arms[arch]
        ms_arm[arch]["t_inf_over_multiscale"] = (arms[arch]["t_inf_ms_16_grids"] /
                                                 ms_arm["t_inf_ms_16_grids"])
    if not args.no_large_plumes:
        torch.cuda.empty_cache()
        ms_arm["large_plumes"] = large_plumes(hp, trained, u0.device)
    return ms_arm


def compare_plume_same_threshold(hp, nets, dev, n=128, steps=300, thr=1e-5, cap=20000,
                                 heads_out=None):
    """The paper's plume with the cylinder (Sec. 2.1 geometry) at 128^2,
    MacCormack advection, buoyancy g = -0.5 (the plume rises about 20 cells in
    300 steps of dt = 0.5), every projection stopped by the same mean |div|
    threshold: plain Jacobi from zero against the hybrid with each trained
    network (nets: architecture -> parameters).  Reports the sweeps and time
    of each run and how far each hybrid's plume-head trajectory is from the
    plain solver's (Sec. 4.2: the same E_1 should give the same plume, whatever
    the network)."""
    import torch
    from paper_2109_09363_gb300 import workloads as W
    from paper_2109_09363_gb300.plume import Plume, PlumeConfig
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    fl, (x0, x1) = W.paper_plume_geometry(n)
    fl = t(fl[None])
    u0, v0, rho0 = W.plume_initial_state(n, seed=2)
    cfg = PlumeConfig(ny=n, nx=n, dt=0.5, gravity=-0.5, inlet=(x0, x1), threshold=thr,
                      max_iters=cap, scheme=1)
    res = {"workload": f"{n}^2 plume, inlet 0.29 n, cylinder 0.312 n at 0.625 n, MacCormack, "
                       f"g = -0.5, dt = 0.5, {steps} steps, E_t = {thr}, cap {cap}"}
    heads = {}
    # the MultiScale run keeps the key "hybrid"
    modes = {"plain": None}
    modes.update({("hybrid" if a == "multiscale" else "hybrid_" + a): a for a in nets})
    for mode, arch in modes.items():
        cnn = hp.CNN(1, n, n, params=nets[arch], arch=arch) if arch else None
        sim = Plume(cfg, t(u0[None].astype(np.float32)), t(v0[None].astype(np.float32)),
                    t(rho0[None].astype(np.float32)), fl, cnn=cnn)
        it = torch.zeros(steps, dtype=torch.int32, device=dev)
        cv = torch.zeros(steps, dtype=torch.uint8, device=dev)
        hd = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(steps):
            out = sim.step()
            it[k:k + 1].copy_(out["iters"])
            cv[k:k + 1].copy_(out["converged"])
            hd.append(torch.stack(sim.head()).view(-1))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        heads[mode] = torch.stack(hd).cpu().numpy() * n
        res[mode] = {"sweeps": int(it.sum().item()), "converged_steps": int(cv.sum().item()),
                     "seconds": wall, "final_head_cells": heads[mode][-1].tolist()}
        if cnn is not None:
            cnn.check()
            cnn.close()
    for mode in modes:
        if mode == "plain":
            continue
        d = np.abs(heads["plain"] - heads[mode]).max(axis=0)
        res[mode]["max_head_difference_cells"] = {"h_y": float(d[0]), "left": float(d[1]),
                                                  "right": float(d[2])}
        res[mode]["sweep_ratio"] = res["plain"]["sweeps"] / max(res[mode]["sweeps"], 1)
        # the paper's eta (Sec. 5) on whole solver steps: wall time of the plain
        # run over the hybrid's, advection and head diagnostic included in both
        # (the projections alone give a larger ratio)
        res[mode]["eta"] = res["plain"]["seconds"] / res[mode]["seconds"]
    res["max_head_difference_cells"] = res["hybrid"]["max_head_difference_cells"]
    res["sweep_ratio"] = res["hybrid"]["sweep_ratio"]
    if heads_out is not None:
        heads_out.update(heads)
    return res


def compare_plume_min_threshold(hp, nets, dev, n=128, steps=300, cap=20000, reference=None):
    """The paper's threshold rule (Sec. 4.2): first every network runs the
    plume alone (its guess is the projection, no Jacobi sweep) and records E_1
    per step; the threshold of step k is the smallest of those E_1.  Then
    plain Jacobi and the hybrid with each network run the same plume with that
    per-step threshold.  Reports the threshold's range, and per run the sweeps,
    time, eta against plain Jacobi and the plume-head distance to the plain
    solver's trajectory (for the networks alone too) and, with reference (the
    head trajectory [steps][3] of an accurate run of the same plume), to that."""
    import torch
    from paper_2109_09363_gb300 import workloads as W
    from paper_2109_09363_gb300.plume import Plume, PlumeConfig
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    fl, (x0, x1) = W.paper_plume_geometry(n)
    fl = t(fl[None])
    u0, v0, rho0 = W.plume_initial_state(n, seed=2)

    def run(arch, thresholds, max_iters):
        cfg = PlumeConfig(ny=n, nx=n, dt=0.5, gravity=-0.5, inlet=(x0, x1),
                          threshold=float(thresholds[0]), max_iters=max_iters, scheme=1)
        cnn = hp.CNN(1, n, n, params=nets[arch], arch=arch) if arch else None
        sim = Plume(cfg, t(u0[None].astype(np.float32)), t(v0[None].astype(np.float32)),
                    t(rho0[None].astype(np.float32)), fl, cnn=cnn)
        it = torch.zeros(steps, dtype=torch.int32, device=dev)
        cv = torch.zeros(steps, dtype=torch.uint8, device=dev)
        e1 = torch.zeros(steps, dtype=torch.float64, device=dev)
        hd = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(steps):
            sim.prm.threshold = float(thresholds[k])
            out = sim.step()
            it[k:k + 1].copy_(out["iters"])
            cv[k:k + 1].copy_(out["converged"])
            e1[k:k + 1].copy_(out["e1"])
            hd.append(torch.stack(sim.head()).view(-1))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if cnn is not None:
            cnn.check()
            cnn.close()
        return {"sweeps": int(it.sum().item()), "converged_steps": int(cv.sum().item()),
                "seconds": wall, "e1": e1.cpu().numpy(),
                "heads": torch.stack(hd).cpu().numpy() * n}

    alone = {a: run(a, np.zeros(steps), 0) for a in nets}
    e_t = np.min(np.stack([r["e1"] for r in alone.values()]), axis=0)
    res = {"workload": f"{n}^2 plume, inlet 0.29 n, cylinder 0.312 n at 0.625 n, MacCormack, "
                       f"g = -0.5, dt = 0.5, {steps} steps, E_t(step) = min over the networks "
                       f"alone, cap {cap}",
           "threshold": {"min": float(e_t.min()), "median": float(np.median(e_t)),
                         "max": float(e_t.max()),
                         "set_by": {a: int(np.sum(r["e1"] == e_t)) for a, r in alone.items()}}}
    runs = {"plain": run(None, e_t, cap)}
    runs.update({"hybrid_" + a: run(a, e_t, cap) for a in nets})
    runs.update({"alone_" + a: r for a, r in alone.items()})
    ref = runs["plain"]["heads"]
    for mode, r in runs.items():
        out = {"sweeps": r["sweeps"], "converged_steps": r["converged_steps"],
               "seconds": r["seconds"], "final_head_cells": r["heads"][-1].tolist()}
        if mode != "plain":
            d = np.abs(r["heads"] - ref).max(axis=0)
            out["max_head_difference_cells"] = {"h_y": float(d[0]), "left": float(d[1]),
                                                "right": float(d[2])}
        if mode.startswith("hybrid_"):
            out["eta"] = runs["plain"]["seconds"] / r["seconds"]
        if reference is not None:
            d = np.abs(r["heads"] - reference).max(axis=0)
            out["max_head_difference_to_reference_cells"] = {
                "h_y": float(d[0]), "left": float(d[1]), "right": float(d[2])}
        res[mode] = out
    if reference is not None:
        res["reference"] = "plain Jacobi with every projection stopped at E_t = 1e-5 (cap 20,000)"
    return res


# scales (down-sampling factors) of the layers of each network, in order
LAYER_SCALES = {"multiscale": [4] * 5 + [2] * 7 + [1] * 7, "smallscale": [4] * 5 + [2] * 7 + [1] * 7,
                "monoscale": [1] * 9,
                "unet": [1, 1, 2, 2, 4, 4, 8, 8, 16, 16, 16, 8, 8, 4, 4, 2, 2, 1, 1, 1]}


def cnn_layer_roofline(arch, pixels, hbm_gbs, tflops):
    """Roofline time of one network forward on `pixels` full-resolution
    pixels: every kernel at its own bound, max(algorithmic bytes / HBM
    bandwidth, FLOPs / tensor rate), summed over the kernels (no overlap
    between kernels).  Bytes per pixel at a kernel's resolution: a 32/64-
    channel convolution reads and writes its BF16 activations (2 B per
    channel); a branch's first layer reads the 16-channel BF16 input (32 B),
    its last writes FP32 (4 B); a branch input reads div and flags (5 B) of
    the pixels it pools and writes 32 B; the scale s reads 5 B per pixel; the
    Unet's pooling reads four 64 B pixels and writes one, its up-sampling
    concatenation writes 128 B and reads the 64 B skip and a quarter of a
    coarse pixel.  FLOPs: 2 x 9 x cin x cout per output pixel (1 x 1: 2 x cin)."""
    from paper_2109_09363_gb300 import training as T
    layers, scales = T.ARCH_LAYERS[arch], LAYER_SCALES[arch]
    hbm, tc = hbm_gbs * 1e9, tflops * 1e12
    t = 5.0 * pixels / hbm                          # the scale s
    prev_cout = None
    for (lay, sc) in zip(layers, scales):
        cin, cout = lay[0], lay[1]
        ks = lay[2] if len(lay) > 2 else 3
        px = pixels / (sc * sc)
        flops = 2.0 * ks * ks * cin * cout * px
        if cin <= 3:                                 # branch input + first layer
            t += (5.0 * sc * sc + 32.0) * px / hbm
            rd = 32.0
        elif arch == "unet" and prev_cout is not None and (sc != prev_sc):
            if sc > prev_sc:                         # max pooling before the layer
                t += (4 * 64.0 + 64.0) * px / hbm
            else:                                    # up-sampling concatenation
                t += (128.0 + 64.0 + 16.0) * px / hbm
            rd = 2.0 * cin
        else:
            rd = 2.0 * cin
        wr = 4.0 if cout == 1 else 2.0 * cout
        t += max((rd + wr) * px / hbm, flops / tc)
        prev_cout, prev_sc = cout, sc
    return t * 1e3


def plume_eval(hp, nets, dev, n, steps, flags_np, inlet, literal_thr=1e-3, literal_cap=2000,
               rule_cap=5000, scheme=0, dt=0.1, gravity=-0.002, seed=3):
    """One large plume (first-order semi-Lagrangian by
    default, g = -0.002, dt = 0.1, inlet rho = 1.1, rho = 1 + N(0, 1e-4^2)),
    run `steps` steps per arm; each arm's projections are timed alone (CUDA
    events around the projection of every step).  Arms:
    - literal: plain Jacobi and the MultiScale hybrid at E_t = literal_thr;
    - the paper's rule (Sec. 4.2): every network first runs the plume alone
      (its guess is the projection, no sweep) and E_t of step k is the
      smallest E_1 any of them reaches; then plain Jacobi and the hybrid with
      each network at that per-step E_t (cap rule_cap).
    Per arm: projections/s over the projection time, sweeps (mean, max),
    converged steps, and the largest plume-head distance to plain Jacobi's
    trajectory (cells)."""
    import torch
    from paper_2109_09363_gb300 import workloads as W
    from paper_2109_09363_gb300.plume import Plume, PlumeConfig
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    fl = t(flags_np[None])
    u0, v0, rho0 = W.plume_initial_state(n, seed=seed)
    stream = torch.cuda.current_stream()

    def run(arch, thresholds, cap):
        cfg = PlumeConfig(ny=n, nx=n, dt=dt, gravity=gravity, inlet=tuple(inlet),
                          threshold=float(thresholds[0]), max_iters=cap, scheme=scheme)
        cnn = hp.CNN(1, n, n, params=nets[arch], arch=arch) if arch else None
        sim = Plume(cfg, t(u0[None].astype(np.float32)), t(v0[None].astype(np.float32)),
                    t(rho0[None].astype(np.float32)), fl, cnn=cnn)
        it = torch.zeros(steps, dtype=torch.int32, device=dev)
        cv = torch.zeros(steps, dtype=torch.uint8, device=dev)
        e1 = torch.zeros(steps, dtype=torch.float64, device=dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        hd = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(steps):
            sim.prm.threshold = float(thresholds[k])
            sim.advect()
            ev[k][0].record(stream)
            out = sim.project()
            ev[k][1].record(stream)
            it[k:k + 1].copy_(out["iters"])
            cv[k:k + 1].copy_(out["converged"])
            e1[k:k + 1].copy_(out["e1"])
            hd.append(torch.stack(sim.head()).view(-1))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        proj_ms = sum(a.elapsed_time(b) for a, b in ev)
        if cnn is not None:
            cnn.check()
            cnn.close()
        sim.ctx.close()
        its = it.cpu().numpy()
        return {"projections_per_s": steps / (proj_ms * 1e-3), "projection_ms_total": proj_ms,
                "solver_seconds": wall, "sweeps_mean": float(its.mean()),
                "sweeps_max": int(its.max()), "converged_steps": int(cv.sum().item()),
                "e1": e1.cpu().numpy(), "heads": torch.stack(hd).cpu().numpy() * n}

    def summary(runs):
        ref = runs["plain"]["heads"]
        out = {}
        for mode, r in runs.items():
            o = {k: v for k, v in r.items() if k not in ("e1", "heads")}
            if mode != "plain":
                d = np.abs(r["heads"] - ref).max(axis=0)
                o["max_head_difference_cells"] = {"h_y": float(d[0]), "left": float(d[1]),
                                                  "right": float(d[2])}
                if mode.startswith("hybrid"):
                    o["speedup_vs_plain"] = (runs["plain"]["projection_ms_total"] /
                                             r["projection_ms_total"])
            out[mode] = o
        return out

    lit = np.full(steps, literal_thr)
    res = {"literal": summary({"plain": run(None, lit, literal_cap),
                               "hybrid_multiscale": run("multiscale", lit, literal_cap)})}
    res["literal"]["threshold"] = literal_thr
    res["literal"]["cap"] = literal_cap
    alone = {a: run(a, np.zeros(steps), 0) for a in nets}
    e_t = np.min(np.stack([r["e1"] for r in alone.values()]), axis=0)
    runs = {"plain": run(None, e_t, rule_cap)}
    runs.update({"hybrid_" + a: run(a, e_t, rule_cap) for a in nets})
    runs.update({"alone_" + a: r for a, r in alone.items()})
    res["paper_rule"] = summary(runs)
    res["paper_rule"]["threshold"] = {
        "min": float(e_t.min()), "median": float(np.median(e_t)), "max": float(e_t.max()),
        "set_by": {a: int(np.sum(r["e1"] == e_t)) for a, r in alone.items()}, "cap": rule_cap}
    return res


def large_plumes(hp, nets, dev):
    """Two large plumes with the trained networks (nets: architecture ->
    parameters): the 1024^2 plume (inlet 128 cells) with a solid disc of
    radius 64 centred 256 cells above the inlet, 200 steps; the 2048^2 plume
    (inlet 256 cells) with 8 non-overlapping discs of radius U(32, 128), 500
    steps (plume_eval: the literal E_t = 1e-3 and the paper's per-step rule)."""
    from paper_2109_09363_gb300 import workloads as W
    res = {}
    n3 = 1024
    fl3 = W.plume_flags(n3, cylinder_radius=64, cylinder_height=256)
    res["plume_1024_cylinder"] = plume_eval(hp, nets, dev, n3, 200, fl3, W.inlet_columns(n3))
    res["plume_1024_cylinder"]["workload"] = ("1024^2 plume, inlet cols [448, 576) of the bottom row, solid "
                                  "disc r = 64 centred 256 cells above it, first-order "
                                  "semi-Lagrangian, g = -0.002, dt = 0.1, 200 steps")
    n5 = 2048
    fl5 = W.random_cylinders(n5, 8, 5, radius=(32, 128), inlet=W.inlet_columns(n5))
    res["plume_2048_cylinders"] = plume_eval(hp, nets, dev, n5, 500, fl5, W.inlet_columns(n5))
    res["plume_2048_cylinders"]["workload"] = ("2048^2 plume, inlet cols [896, 1152) of the bottom row, 8 "
                                  "non-overlapping solid discs r ~ U(32, 128) (seed 5), "
                                  "first-order semi-Lagrangian, g = -0.002, dt = 0.1, "
                                  "500 steps")
    return res


def compare_in_distribution(hp, nets, flush, stream, dev, ws):
    """Plain vs hybrid with each trained network (nets: architecture ->
    parameters; the MultiScale's run keeps the key "hybrid") on held-out grids
    of the training distribution at the training resolution (256 x 128^2,
    vortex field + divergence sources + 0-4 obstacles, seeds disjoint from the
    training pairs), E_t = 1e-3, cap 5000: the regime where the network sees
    most of the domain.  Same protocol as the plain arm: device restore of u*,
    L2 flush between steps, CUDA events."""
    import torch
    from paper_2109_09363_gb300 import workloads as W
    nb, n, thr, cap = IN_DIST_GRIDS, 128, 1e-3, 5000
    u_np, v_np, f_np = W.training_case(nb, n, seed0=IN_DIST_SEED)
    uh = torch.from_numpy(u_np.astype(np.float32)).to(dev)
    vh = torch.from_numpy(v_np.astype(np.float32)).to(dev)
    fd = torch.from_numpy(f_np).to(dev)
    ud, vd = torch.empty_like(uh), torch.empty_like(vh)
    ctx = hp.Context(nb, n, n, device=dev.index)
    prm = hp.ProjectParams(threshold=thr, max_iters=cap, temporal_block=T_BLOCK)
    res = {}
    arms = {"plain": None}
    arms.update({("hybrid" if a == "multiscale" else "hybrid_" + a): a for a in nets})
    for arm, arch in arms.items():
        out = None
        cnn = hp.CNN(nb, n, n, params=nets[arch], arch=arch) if arch else None

        def step():
            nonlocal out
            ud.copy_(uh)
            vd.copy_(vh)
            if cnn is None:
                out = hp.hp_project(ctx, ud, vd, fd, prm, out=out)
            else:
                out = hp.hp_project_hybrid(ctx, cnn, ud, vd, fd, prm, out=out)

        for _ in range(3):
            step()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(5)]
        for k, (e0, e1) in enumerate(ev):
            flush.fill_(float(k))
            e0.record(stream)
            step()
            e1.record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
        it = out["iters"].cpu().numpy()
        res[arm] = {"value": ws * nb / (ms * 1e-3), "ms_per_step": ms,
                    "iters_mean": float(it.mean()), "iters_max": int(it.max()),
                    "converged": int(out["converged"].sum().item())}
        if cnn is not None:
            res[arm]["speedup"] = res["plain"]["ms_per_step"] / ms
            cnn.close()
    ctx.close()
    res["speedup"] = res["hybrid"]["speedup"]
    res["workload"] = (f"{nb} x {n}^2 held-out training-distribution grids (seeds "
                       f"{IN_DIST_SEED}..), E_t = {thr}, cap {cap}")
    return res


def run_pdnn_arm(hp, dev, steps: int = 10, warmup: int = 3, batch: int = 64, n: int = 128):
    """Physics-driven training (Sec. 3.2, Eq. 4) at the paper's training
    resolution: one Adam step = the rollout of the training solver over
    n_roll - 1 steps (network-only projection + advection) from a batch of
    velocity states, then the loss gradient on 2 x batch grids (t and
    t + n_roll - 1) and the update.  Timed with CUDA events per step for
    n_roll = 4 and 16 (the paper draws 4 nine times in ten); inputs resident,
    a fixed random network."""
    import torch
    from paper_2109_09363_gb300 import training as T
    from paper_2109_09363_gb300 import workloads as W
    u_np, v_np, f_np = W.training_case(batch, n, seed0=IN_DIST_SEED + 4096)
    u = torch.from_numpy(u_np.astype(np.float32)).to(dev)
    v = torch.from_numpy(v_np.astype(np.float32)).to(dev)
    fl = torch.from_numpy(f_np).to(dev)
    cnn = hp.CNN(2 * batch, n, n, params=T.init_params(seed=5))
    ctx = hp.Context(batch, n, n, device=dev.index)
    tr = hp.Trainer(cnn, 2 * batch, n, n)
    stream = torch.cuda.current_stream()
    res = {"workload": f"{batch} x {n}^2 training-distribution grids (vortex field + divergence "
                       "sources + 0-4 obstacles), random network, norm 1, alpha = beta = 1",
           "batch": batch, "grid": [n, n]}
    for n_roll in (4, 16):
        def one():
            div, f2, w = T.pdnn_batch(cnn, ctx, u, v, fl, n_roll)
            tr.pdnn_step(div, f2, w, norm=1, lr=1e-5)
        for _ in range(warmup):
            one()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for k in range(steps):
            ev[k][0].record(stream)
            one()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        res[f"ms_per_step_n{n_roll}"] = ms
    ms_mean = 0.9 * res["ms_per_step_n4"] + 0.1 * res["ms_per_step_n16"]
    res["ms_per_step_mean"] = ms_mean
    res["samples_per_s"] = batch / (ms_mean * 1e-3)
    tr.close()
    ctx.close()
    cnn.close()
    return res


def run_driver_timing(hp, u0, v0, fl, reps: int = 10):
    """Driver step (a8 and the f3 MacCormack scheme) on the bench grids: one
    hp_advect_step with first-order semi-Lagrangian and with MacCormack
    advection, and the plume-head reduction, CUDA events over `reps` calls
    each (inputs resident)."""
    import torch
    B_, ny, nx = fl.shape
    g = torch.Generator(device="cpu").manual_seed(7)
    rho = (1.0 + 1e-4 * torch.randn((B_, ny, nx), generator=g)).to(u0.device)
    outs = (torch.empty_like(u0), torch.empty_like(v0), torch.empty_like(rho))
    res = {"workload": f"{B_} x {ny}x{nx} bench grids, rho = 1 + N(0, 1e-4^2), dt = 0.1"}
    for name, scheme in (("sl", 0), ("maccormack", 1)):
        pp = hp.PlumeParams(dt=0.1, inlet_x0=nx // 2 - nx // 16, inlet_x1=nx // 2 + nx // 16,
                            scheme=scheme)
        for _ in range(3):
            hp.hp_advect_step(u0, v0, rho, fl, pp, *outs)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            hp.hp_advect_step(u0, v0, rho, fl, pp, *outs)
        b.record()
        torch.cuda.synchronize()
        res[f"{name}_ms"] = a.elapsed_time(b) / reps
    # algorithmic bytes of one step: u, v, rho and the flags read once, u*,
    # v* and the new rho written once
    floats = ny * (nx + 1) + (ny + 1) * nx + ny * nx
    step_bytes = B_ * (2 * 4 * floats + ny * nx)
    peak, kind = load_peaks()
    for name in ("sl", "maccormack"):
        gbs = step_bytes / res[f"{name}_ms"] / 1e6
        res[f"{name}_hbm"] = {"gbs": gbs, "frac": gbs / peak, "peak_kind": kind,
                              "bytes_per_step": step_bytes}
    head = torch.empty((B_, 3), dtype=torch.int32, device=u0.device)
    for _ in range(3):
        hp.hp_plume_head(outs[2], 1.0, 0.01, out=head)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        hp.hp_plume_head(outs[2], 1.0, 0.01, out=head)
    b.record()
    torch.cuda.synchronize()
    res["plume_head_ms"] = a.elapsed_time(b) / reps
    return res


def profile_conv(batch, h, w, cin, cout) -> int:
    """Time and run one tensor-core convolution layer (FLOP/s printed)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2109_09363_gb300 as hp
    dev = torch.device("cuda", 0)
    g = torch.Generator(device="cpu").manual_seed(0)
    x = torch.randn((batch, h, w, cin), generator=g).to(torch.bfloat16).to(dev)
    wt = (torch.randn((3, 3, cout, cin), generator=g) / (3 * cin ** 0.5)).to(torch.bfloat16).to(dev)
    bias = torch.zeros(cout, dtype=torch.float32, device=dev)
    y = torch.empty((batch, h, w, cout), dtype=torch.bfloat16, device=dev)
    for _ in range(3):
        hp.hp_conv3x3_bf16(x, wt, bias, True, y=y)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(10):
        hp.hp_conv3x3_bf16(x, wt, bias, True, y=y)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / 10
    flop = 2.0 * batch * h * w * 9 * cin * cout
    print(json.dumps({"profile_conv": [batch, h, w, cin, cout], "ms": ms,
                      "tflops": flop / ms / 1e9}))
    return 0


def stencil_timing(hp, dev, batch, n):
    """The HBM-streaming stencil calls on batch grids of n x n with obstacles
    and random velocities (CUDA events around 20 back-to-back calls after 3,
    so that the host's launch overhead stays behind the device's work): the
    divergence, the face mask and the divergence norms; GB/s from each call's
    algorithmic bytes per cell (divergence: u 4 + v 4 + flags 1 read, div 4
    written; mask: 1 + 1; norms: 9) and the fraction of the measured HBM
    bandwidth.  (The correction runs only inside a projection; its kernel is
    measured with ncu.)"""
    import torch
    from paper_2109_09363_gb300 import workloads as W
    hbm, kind = load_peaks()
    g = torch.Generator(device=dev).manual_seed(0)
    u0 = torch.randn((batch, n, n + 1), generator=g, device=dev)
    v0 = torch.randn((batch, n + 1, n), generator=g, device=dev)
    fl = torch.from_numpy(np.stack([W.random_obstacles(n, n, 100 + b) for b in range(batch)])).to(dev)
    ctx = hp.Context(batch, n, n)
    div = torch.empty((batch, n, n), dtype=torch.float32, device=dev)
    mask = torch.empty_like(fl)
    calls = {
        "divergence": (lambda: hp.hp_divergence(u0, v0, fl, div_out=div), 13),
        "face_mask": (lambda: hp.hp_face_mask(fl, mask_out=mask), 2),
        "div_norms": (lambda: hp.hp_div_norms(ctx, u0, v0, fl), 9),
    }
    cells = batch * n * n
    out = {"workload": f"{batch} x {n}^2, random obstacles and velocities",
           "peak_gbs": hbm, "peak_kind": kind}
    for name, (fn, bpc) in calls.items():
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(20):
            fn()
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / 20
        gbs = bpc * cells / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "bytes_per_cell": bpc, "gbs": gbs, "frac": gbs / hbm}
    out["note"] = "whole calls (the norms with their FP64 finishing kernel)"
    ctx.close()
    del u0, v0, div, mask, fl
    torch.cuda.empty_cache()
    return out


def profile_stencil(batch, n) -> int:
    """Print stencil_timing for batch grids of n x n."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2109_09363_gb300 as hp
    out = {"profile_stencil": [batch, n]}
    out.update(stencil_timing(hp, torch.device("cuda", 0), batch, n))
    print(json.dumps(out))
    return 0


def profile_advect(batch, n) -> int:
    """Print run_driver_timing for batch vortex grids of n x n."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2109_09363_gb300 as hp
    from paper_2109_09363_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    u, v, fl = W.batched_vortex_case(batch, n)
    ud = torch.from_numpy(u.astype(np.float32)).to(dev)
    vd = torch.from_numpy(v.astype(np.float32)).to(dev)
    fd = torch.from_numpy(fl).to(dev)
    out = {"profile_advect": [batch, n]}
    out.update(run_driver_timing(hp, ud, vd, fd))
    print(json.dumps(out))
    return 0


def profile_cnn(batch, n, arch="multiscale") -> int:
    """Time the CNN forward (t_inf) on BATCH vortex grids of N x N."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2109_09363_gb300 as hp
    from paper_2109_09363_gb300 import training as T
    from paper_2109_09363_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    u, v, fl = W.batched_vortex_case(batch, n)
    ud = torch.from_numpy(u.astype(np.float32)).to(dev)
    vd = torch.from_numpy(v.astype(np.float32)).to(dev)
    fd = torch.from_numpy(fl).to(dev)
    cnn = hp.CNN(batch, n, n, params=T.init_params(seed=1, arch=arch), arch=arch)
    div = hp.hp_divergence(ud, vd, fd)
    for _ in range(3):
        hp.hp_cnn_forward(cnn, div, fd)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(5):
        hp.hp_cnn_forward(cnn, div, fd)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / 5
    flop = 2.0 * CNN_MACS_PER_PIXEL[arch] * batch * n * n
    print(json.dumps({"profile_cnn": [batch, n], "arch": arch, "ms": ms,
                      "tflops": flop / ms / 1e9}))
    return 0


def profile_cnn_scaling(sizes=(32, 64, 128, 256, 512, 1024, 2048)) -> int:
    """t_inf of one grid against its size for every network (the paper's
    Fig. 15): CUDA events over 20 forwards after 5 untimed ones, one JSON line
    per network and size."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2109_09363_gb300 as hp
    from paper_2109_09363_gb300 import training as T
    from paper_2109_09363_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    for n in sizes:
        u, v, fl = W.batched_vortex_case(1, n)
        ud = torch.from_numpy(u.astype(np.float32)).to(dev)
        vd = torch.from_numpy(v.astype(np.float32)).to(dev)
        fd = torch.from_numpy(fl).to(dev)
        div = hp.hp_divergence(ud, vd, fd)
        for arch in FORWARD_NETWORKS:
            cnn = hp.CNN(1, n, n, params=T.init_params(seed=1, arch=arch), arch=arch)
            for _ in range(5):
                hp.hp_cnn_forward(cnn, div, fd)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(20):
                hp.hp_cnn_forward(cnn, div, fd)
            b.record()
            torch.cuda.synchronize()
            cnn.check()
            ms = a.elapsed_time(b) / 20
            flop = 2.0 * CNN_MACS_PER_PIXEL[arch] * n * n
            print(json.dumps({"profile_cnn_scaling": arch, "n": n, "ms": ms,
                              "tflops": flop / ms / 1e9}), flush=True)
            cnn.close()
    return 0


def profile_train(batch, n, norm=1, arch="multiscale") -> int:
    """Time the physics-driven loss gradient (network forward, loss, backward)
    of the network `arch` on BATCH training-distribution grids of N x N,
    after 3 untimed calls."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2109_09363_gb300 as hp
    from paper_2109_09363_gb300 import training as T
    from paper_2109_09363_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    u, v, fl = W.training_case(batch, n, seed0=IN_DIST_SEED + 8192)
    ud = torch.from_numpy(u.astype(np.float32)).to(dev)
    vd = torch.from_numpy(v.astype(np.float32)).to(dev)
    fd = torch.from_numpy(fl).to(dev)
    cnn = hp.CNN(batch, n, n, params=T.init_params(seed=1, arch=arch), arch=arch)
    tr = hp.Trainer(cnn, batch, n, n)
    div = hp.hp_divergence(ud, vd, fd)
    w = torch.full((batch,), 1.0 / batch, dtype=torch.float32, device=dev)
    for _ in range(3):
        tr.pdnn_gradient(div, fd, w, norm=norm)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(5):
        tr.pdnn_gradient(div, fd, w, norm=norm)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / 5
    tr.check()
    # forward + two backward contractions (data and weight gradients)
    flop = 3 * 2.0 * CNN_MACS_PER_PIXEL[arch] * batch * n * n
    print(json.dumps({"profile_train": [batch, n], "arch": arch, "ms": ms,
                      "tflops": flop / ms / 1e9}))
    return 0


def main():
    global T_BLOCK
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-sweep", nargs=3, type=int, metavar=("BATCH", "N", "SWEEPS"),
                    help="only run the sweep kernel: SWEEPS Jacobi sweeps on BATCH vortex grids "
                         "of N x N, three times (a small case for ncu)")
    ap.add_argument("--temporal-block", type=int, default=T_BLOCK,
                    help="sweeps per launch of the temporally blocked kernel (1..8)")
    ap.add_argument("--sweep-kernel", type=int, default=0, choices=[0, 1, 2, 3, 4],
                    help="0 = library choice, 1 = streaming, 2 = temporally blocked "
                         "(4 rows per thread), 3 = temporally blocked (2 rows per thread), "
                         "4 = grid-resident")
    ap.add_argument("--profile-conv", nargs=5, type=int,
                    metavar=("BATCH", "H", "W", "CIN", "COUT"),
                    help="only run the tensor-core 3x3 convolution, 3 times (a small case for ncu)")
    ap.add_argument("--profile-stencil", nargs=2, type=int, metavar=("BATCH", "N"),
                    help="only time the divergence, mask, norms and a projection without "
                         "sweeps on BATCH grids of N x N")
    ap.add_argument("--profile-advect", nargs=2, type=int, metavar=("BATCH", "N"),
                    help="time the driver step (first-order and MacCormack advection) on "
                         "BATCH vortex grids of N x N and exit")
    ap.add_argument("--profile-cnn", nargs=2, type=int, metavar=("BATCH", "N"),
                    help="only run the CNN forward on BATCH grids of N x N, 3 times")
    ap.add_argument("--profile-cnn-scaling", action="store_true",
                    help="only time one forward of every network on one grid of 32^2 .. 2048^2")
    ap.add_argument("--arch", default="multiscale", choices=list(FORWARD_NETWORKS),
                    help="network of --profile-cnn and --profile-train")
    ap.add_argument("--profile-train", nargs=2, type=int, metavar=("BATCH", "N"),
                    help="only run the physics-driven loss gradient on BATCH grids of N x N, "
                         "8 times (a small case for ncu)")
    ap.add_argument("--no-hybrid", action="store_true",
                    help="skip the CNN-hybrid arm (training + timing)")
    ap.add_argument("--no-pdnn", action="store_true",
                    help="skip the timing of physics-driven training steps")
    ap.add_argument("--train-pairs", type=int, default=10000,
                    help="training pairs (128^2) of the networks of the hybrid arm")
    ap.add_argument("--train-epochs", type=int, default=20,
                    help="epochs (batch 64) of the networks of the hybrid arm")
    ap.add_argument("--no-large-plumes", action="store_true",
                    help="skip the 1024^2 and 2048^2 plumes with cylinders in the "
                         "hybrid arm")
    ap.add_argument("--host-loop", action="store_true",
                    help="launch the sweep blocks from a host-polled loop instead of the "
                         "CUDA-graph conditional loop (same kernels; ncu cannot profile kernel "
                         "nodes of graphs with conditional nodes)")
    args = ap.parse_args()
    T_BLOCK = args.temporal_block
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_sweep:
        return profile_sweep(*args.profile_sweep, host_loop=args.host_loop,
                             kernel=args.sweep_kernel)
    if args.profile_conv:
        return profile_conv(*args.profile_conv)
    if args.profile_stencil:
        return profile_stencil(*args.profile_stencil)
    if args.profile_advect:
        return profile_advect(*args.profile_advect)
    if args.profile_cnn:
        return profile_cnn(*args.profile_cnn, arch=args.arch)
    if args.profile_cnn_scaling:
        return profile_cnn_scaling()
    if args.profile_train:
        return profile_train(*args.profile_train, arch=args.arch)

    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)

    import __graft_entry__
    __graft_entry__.build()
    import paper_2109_09363_gb300 as hp

    u_np, v_np, fl_np = make_inputs(rank)
    u0 = torch.from_numpy(u_np).to(dev)
    v0 = torch.from_numpy(v_np).to(dev)
    fl = torch.from_numpy(fl_np).to(dev)
    u = torch.empty_like(u0)
    v = torch.empty_like(v0)
    ctx = hp.Context(B, N, N, device=local)
    prm = hp.ProjectParams(threshold=THR, max_iters=CAP, temporal_block=T_BLOCK,
                           use_graph=0 if args.host_loop else 1,
                           sweep_kernel=args.sweep_kernel)
    # the grid-resident kernel runs when the library picks it (0) or it is
    # asked for (4) and one cluster per grid fits on this device
    resident = args.sweep_kernel in (0, 4) and hp.hp_resident_clusters(ctx, B, N, N) > 0
    streaming = not resident and streaming_chosen(args.sweep_kernel, B * N * N)
    per_launch = 1 if streaming else T_BLOCK
    stream = torch.cuda.current_stream()
    out = None
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        nonlocal out
        u.copy_(u0)
        v.copy_(v0)
        out = hp.hp_project(ctx, u, v, fl, prm, out=out)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    iters = out["iters"].cpu().numpy()
    if resident:
        # mask/div, init, reset, the resident sweep loop, correction, norms (2)
        launches_per_step = 7
    elif streaming:
        # 8 sweep launches per graph-loop iteration, plus mask/div, init,
        # reset, correction, norms, finish
        launches_per_step = 6 + 8 * ((int(iters.max()) + 1 + 7) // 8)
    else:
        launches_per_step = 7 + int(iters.max()) // T_BLOCK + 1

    # timed region: per-step CUDA events, L2 flushed (untimed) between steps
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for s in range(args.steps):
        flush.fill_(float(s))
        ev[s][0].record(stream)
        step()
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    # the last timed step's results, kept for the parity check of the CPU leg
    gpu_result = (out["iters"].cpu().numpy(), u.cpu().numpy(), v.cpu().numpy())
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    if ws > 1:
        ms = max_over_ranks(ms, dev)
    value = ws * B / (ms * 1e-3)

    # dominant kernel: the sweep kernel; its time per sweep of the batch from
    # the difference of two fixed-length sweep runs (same shape, all 16 grids
    # active), CUDA events on the launching stream
    n1, n2 = 8 * 20, 8 * 220
    fprm = [hp.ProjectParams(fixed_iters=n, temporal_block=T_BLOCK, use_graph=1,
                             sweep_kernel=args.sweep_kernel) for n in (n1, n2)]
    for _ in range(2):
        for fp in fprm:
            u.copy_(u0)
            v.copy_(v0)
            hp.hp_project(ctx, u, v, fl, fp)
    tl = []
    for fp in fprm:
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        u.copy_(u0)
        v.copy_(v0)
        flush.fill_(1.0)
        a.record(stream)
        hp.hp_project(ctx, u, v, fl, fp)
        b_.record(stream)
        torch.cuda.synchronize()
        tl.append(a.elapsed_time(b_))
    t_launch_ms = (tl[1] - tl[0]) / ((n2 - n1) / per_launch)
    t_sweep_ms = (tl[1] - tl[0]) / (n2 - n1)
    cells = B * N * N
    alg_bytes = BYTES_PER_CELL_SWEEP * cells * per_launch
    peak, peak_kind = load_peaks()
    achieved = alg_bytes / (t_launch_ms * 1e-3) / 1e9
    # DRAM bytes per launch from an ncu capture of the same kernel and
    # workload (committed summary); null when the kernel changed since
    traffic = None
    tp = os.path.join(ROOT, "profiles", "dram_traffic_16x512.json")
    kname = ("sweep_resident_kernel" if resident else "sweep1_kernel" if streaming
             else f"sweep_tb_kernel<{8 if T_BLOCK > 4 else 4}>")
    if os.path.exists(tp):
        traffic = json.load(open(tp)).get(kname)
    if resident:
        # on-chip for all sweeps: bound by FP32 issue, not by HBM.
        # OPS_PER_CELL_UPDATE FP32 operations per cell update against the FP32
        # lane rate (SMs x 128 lanes x maximum SM clock)
        sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
        max_mhz = clk.get("sm_max_mhz") or 2070.0
        alu_peak = sm_count * 128 * max_mhz * 1e6 / 1e12
        alu_achieved = OPS_PER_CELL_UPDATE * cells / (t_sweep_ms * 1e-3) / 1e12
        hbm_eff = BYTES_PER_CELL_SWEEP * cells / (t_sweep_ms * 1e-3) / 1e9
        roofline = {"bound": "alu", "kernel": kname, "achieved": alu_achieved,
                    "peak": alu_peak, "unit": "TOP/s", "frac": alu_achieved / alu_peak,
                    "traffic": traffic, "peak_kind": "derived: SMs x 128 FP32 lanes x max clock",
                    "ops_per_cell_update": OPS_PER_CELL_UPDATE, "sweep_ms_batch": t_sweep_ms,
                    "clusters_resident": hp.hp_resident_clusters(ctx, B, N, N),
                    "hbm_effective": {"achieved": hbm_eff, "peak": peak, "unit": "GB/s",
                                      "frac": hbm_eff / peak, "peak_kind": peak_kind,
                                      "note": "13 B per cell-sweep of a sweep that streams "
                                              "from HBM; the resident kernel reads the grid "
                                              "once per projection"},
                    "note": "one cluster of 16 CTAs per 512^2 grid keeps phi on chip for all "
                            "sweeps; per-sweep time of the 16-grid batch from two fixed-length "
                            "runs"}
    else:
        roofline = {"bound": "hbm",
                    "kernel": kname,
                    "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": traffic,
                    "peak_kind": peak_kind,
                    "algorithmic_bytes_per_launch": alg_bytes,
                    "launch_ms": t_launch_ms,
                    "note": ("13 B per cell-sweep x 4.19 M cells, one sweep per launch; "
                             "the 54.5 MB working set is L2-resident between launches"
                             if streaming else
                             "13 B per cell-sweep x 4.19 M cells x 8 sweeps per launch; "
                             "temporal blocking keeps 8 sweeps on chip, so frac is an "
                             "effective HBM fraction")}

    # end to end through the public API with host buffers: every step copies its
    # inputs u*, v*, flags from pinned memory to the device, projects, and
    # copies u, v, p and the iteration counts back.  Uploads and downloads run
    # on two more streams with two sets of device inputs, so that step i + 1's
    # inputs and step i - 1's results move while step i computes (an input set
    # is refilled only after its previous results have been read back); the
    # timed region spans the first upload to the last download.
    hu, hv, hf = (torch.from_numpy(x).pin_memory() for x in (u_np, v_np, fl_np))
    ou, ov = torch.empty_like(hu).pin_memory(), torch.empty_like(hv).pin_memory()
    op = torch.empty((B, N, N), dtype=torch.float32).pin_memory()
    oi = torch.empty(B, dtype=torch.int32).pin_memory()
    dev_in = [(torch.empty_like(u), torch.empty_like(v), torch.empty_like(fl)) for _ in range(2)]
    e2e_outs = [None, None]
    s_up, s_down = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

    def e2e_run(nsteps):
        read_back = [None, None]  # per input set: its last download
        for i in range(nsteps):
            k = i % 2
            du, dv, df = dev_in[k]
            h2d_done = torch.cuda.Event()
            with torch.cuda.stream(s_up):
                if read_back[k] is not None:
                    s_up.wait_event(read_back[k])
                du.copy_(hu, non_blocking=True)
                dv.copy_(hv, non_blocking=True)
                df.copy_(hf, non_blocking=True)
                h2d_done.record(s_up)
            stream.wait_event(h2d_done)
            e2e_outs[k] = hp.hp_project(ctx, du, dv, df, prm, out=e2e_outs[k], stream=stream)
            comp_done = torch.cuda.Event()
            comp_done.record(stream)
            with torch.cuda.stream(s_down):
                s_down.wait_event(comp_done)
                ou.copy_(du, non_blocking=True)
                ov.copy_(dv, non_blocking=True)
                op.copy_(e2e_outs[k]["p"], non_blocking=True)
                oi.copy_(e2e_outs[k]["iters"], non_blocking=True)
                read_back[k] = torch.cuda.Event()
                read_back[k].record(s_down)
        torch.cuda.synchronize()

    e2e_steps = max(3, args.steps)
    e2e_run(2)  # untimed warm-up of both input sets
    t0 = time.perf_counter()
    e2e_run(e2e_steps)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    h2d = hu.nbytes + hv.nbytes + hf.nbytes
    d2h = ou.nbytes + ov.nbytes + op.nbytes + oi.nbytes

    hybrid = None
    if not args.no_hybrid:
        hybrid = run_hybrid_arm(args, hp, u0, v0, fl, u, v, ctx, prm, flush, stream, ms, ws)
    pdnn = None if args.no_pdnn else run_pdnn_arm(hp, dev)
    driver = run_driver_timing(hp, u0, v0, fl)
    # the streaming stencil calls on a DRAM-sized batch (16 x 2048^2)
    stencil = stencil_timing(hp, dev, 16, 2048) if rank == 0 else None

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "method": "plain Jacobi", "grids_per_gpu": B,
                       "grid": [N, N], "threshold": THR, "cap": CAP,
                       "sweep_kernel": ("grid-resident (one cluster per grid)" if resident
                                        else "streaming" if streaming else "temporally blocked"),
                       "temporal_block": None if (streaming or resident) else T_BLOCK,
                       "loop": ("one launch per projection" if resident else "host-polled"
                                if args.host_loop else "CUDA-graph conditional while"),
                       "l2": "flushed between steps (256 MB write, untimed)",
                       "iters_per_grid": iters.tolist()},
            "roofline": roofline,
            "paper_times": {"t_p_ms": ms / B, "t_it_us": roofline.get("sweep_ms_batch",
                                                                      t_sweep_ms) * 1e3 / B,
                            "note": "Sec. 5's t_p (one projection) and t_it (one Jacobi "
                                    "iteration of one grid), amortised over the 16 grids "
                                    "that run at once"},
            "e2e": {"value": ws * B / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk,
        }
        # how many grids of the last timed step reached E_t before the cap
        line["converged"] = {"grids": int(out["converged"].sum().item()), "of": B}
        if hybrid is not None:
            line["hybrid"] = hybrid
            # the headline comparison: CNN-hybrid against plain Jacobi on the
            # same grids, both at the same E_t; under the cap of 5000, and with
            # the cap lifted so that every grid of both arms converges (the
            # paper's comparison at equal mean|div|)
            unc = hybrid["equal_threshold_uncapped"]
            eq = {"multiscale": unc["speedup"]}
            eq.update({a: hybrid[a]["equal_threshold_uncapped"]["speedup"]
                       for a in NETWORKS[1:] if a in hybrid})
            best = max(eq, key=eq.get)
            line["hybrid_vs_plain"] = {
                "best_network_equal_threshold": {"network": best, "speedup": eq[best]},
                "network": "multiscale",
                "equal_threshold": {
                    "speedup": unc["speedup"], "threshold": THR, "cap": unc["cap"],
                    "converged_hybrid": unc["hybrid"]["converged"],
                    "converged_plain": unc["plain"]["converged"], "of": B,
                    "all_converged": unc["hybrid"]["converged"] == B and
                    unc["plain"]["converged"] == B},
                "capped": {"speedup": hybrid["speedup_vs_plain"], "threshold": THR, "cap": CAP,
                           "converged_hybrid": hybrid["converged"],
                           "converged_plain": int(out["converged"].sum().item()), "of": B},
                "others": {a: {"equal_threshold": hybrid[a]["equal_threshold_uncapped"]["speedup"],
                               "capped": hybrid[a]["speedup_vs_plain"]}
                           for a in NETWORKS[1:] if a in hybrid}}
            bc = hybrid.get("large_plumes")
            if bc:
                # projection time of the hybrid against plain Jacobi on the
                # two large plumes (literal E_t, and the paper's rule)
                line["hybrid_vs_plain"]["plumes"] = {
                    c: {"literal_multiscale": bc[c]["literal"]["hybrid_multiscale"][
                            "speedup_vs_plain"],
                        "paper_rule": {a: bc[c]["paper_rule"]["hybrid_" + a]["speedup_vs_plain"]
                                       for a in NETWORKS},
                        "plain_sweeps_mean_paper_rule": bc[c]["paper_rule"]["plain"][
                            "sweeps_mean"]}
                    for c in ("plume_1024_cylinder", "plume_2048_cylinders")}
        if pdnn is not None:
            line["pdnn_training"] = pdnn
        line["driver_step"] = driver
        line["stencil_roofline"] = stencil
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_oracle_sample(u_np, v_np, fl_np, gpu=gpu_result)
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
