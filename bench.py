"""Benchmark: Phi^dagger Phi applies/s on the 4096^2 / 50M-visibility workload.

One step = one application of Phi^dagger Phi (Eq. 7, Eq. 8) over the whole w-stack
(all 32 w-bins, all 50M visibilities) with the stored de-gridding matrix, on seeded
synthetic MeerKAT-like data.  Inputs (G taps: tens of GB; grids: 0.5 GB each) are far
larger than the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl rimo|reference]

Prints one JSON line.  Under torchrun (N > 1) every rank runs an independent replica
(the operator has no exchange step on one GPU per w-stack) and rank 0 reports the
aggregate over ranks with the slowest rank's time.  --impl reference times the FP64
CPU oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Phi^dagger Phi applies/s at 4096^2, 50M vis (Mvis/s and rel. l2 err vs FP64 oracle alongside)"
UNIT = "applies/s"
WORKLOAD = "surrogate-4096 config, exact stored-G path: 4096x4096 image, FoV 3 deg, 8192x8192 grid, " \
           "50M visibilities, 32 w-bins, KB 7x7 (*) w-kernels <= 9x9"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="rimo", choices=["rimo", "reference"])
    ap.add_argument("--m", type=int, default=50_000_000, help="visibilities (default: the full workload)")
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--bins", type=int, default=32)
    ap.add_argument("--no-oracle", action="store_true", help="skip the oracle error sample and CPU baseline")
    ap.add_argument("--cpu-sample-vis", type=int, default=20000)
    ap.add_argument("--tile", type=int, default=0, help="uv-tile size (0: library default)")
    ap.add_argument("--config", default="c5", choices=["c5", "wideband", "holo", "holo-dense"],
                    help="c5: the 4096^2 / 50M workload (default); wideband: 32 channels of 1024^2 "
                         "batched into one graph launch; holo: 2048^2 / 20M / 16 bins with H_p = G_p^dagger G_p; "
                         "holo-dense: 256^2 / 20M / 4 bins, where visibilities per grid cell are many")
    ap.add_argument("--channels", type=int, default=32, help="wideband: channels")
    ap.add_argument("--autotune", default="", help="wideband: JSON cache path; tile sizes by the autotuner")
    ap.add_argument("--wideband-bins", default="linear", choices=["linear", "auto"],
                    help="wideband: w-bins per channel, linear 4 -> 32 with frequency (default) or the planner's")
    return ap.parse_args()


# ----------------------------------------------------------------------------- distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index: int):
        self.path = os.path.join(tempfile.gettempdir(), f"rimo_clocks_{os.getpid()}.csv")
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.remove(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- workload
def workload(args):
    import synth
    t = time.time()
    uvw = synth.make_uvw(args.m, 28_800, 1.28e9, seed=1005)
    sky = synth.make_sky(args.n, seed=2005)
    return uvw, sky, time.time() - t


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def stage_bytes(info: dict, n: int, P: int, M: int, tiles: int, PW: int):
    """Algorithmic bytes of each stage (complex64 = 8 B; n = image side, PW = patch side).

    Per launch for the transform passes; per step (all bins) for the gridding stage and
    for the whole apply.
    """
    n2 = float(n) * n
    K = float(info["K"])
    patches = 8.0 * tiles * PW * PW        # one (TS + H)^2 patch per active uv-tile
    return {
        "fwd_rows": 24 * n2,               # read x (n^2), write A^T (2 n^2)
        "fwd_cols": 48 * n2,               # read A^T (2 n^2), write X (4 n^2)
        "inv_cols_per_step": patches + P * 16 * n2,   # read the patches, write B (2 n^2)
        "inv_rows": 32 * n2,               # read B (2 n^2), read + write the output (n^2 each)
        # taps (8 B each) and 16 B metadata per visibility, plus the X patch read and the
        # accumulator patch written for every active uv-tile
        "gtg_per_step": 8 * K + 16 * M + 2 * patches,
        "apply_per_step": 8 * K + 16 * M + 3 * patches + P * (24 + 48 + 16 + 32) * n2,
    }


def oracle_error_sample(uvw, sky, plan, args, n_vis=24):
    """Relative l2 error of GPU Phi against the FP64 oracle on sampled visibilities."""
    import torch
    from oracle import operator as oop
    from oracle import plan as opl
    fov = math.radians(3.0)
    ws, bins, sw = plan.bins()
    pp = opl.PlanParams(nx=args.n, ny=args.n, fov_x=fov, fov_y=fov, n_wbins=args.bins)
    # the oracle's own plan (centroids by its k-means), checked equal to the library's
    oplan = opl.make_plan(uvw, pp)
    same_bins = bool(np.array_equal(oplan.bins, bins) and np.array_equal(oplan.s_w, sw))
    op = oop.Operator(uvw, oplan, build_g=False)
    rng = np.random.default_rng(7)
    cand_bins = rng.choice(np.unique(bins), 2, replace=False)
    ks = np.concatenate([rng.choice(np.nonzero(bins == b)[0], n_vis // 2, replace=False) for b in cand_bins])
    ks = ks[np.argsort(bins[ks], kind="stable")]
    x = torch.from_numpy(sky).cuda()
    y = plan.phi(x)
    torch.cuda.synchronize()
    yg = y.cpu().numpy()[ks].astype(np.complex128)
    yo = op.phi_sampled(sky.astype(np.complex128), ks)
    err = float(np.linalg.norm(yg - yo) / np.linalg.norm(yo))
    _, _, S, taps = plan.tiles(ks[:8])
    ref = op.tiles(ks[:8])
    terr = max(float(np.linalg.norm(taps[q] - ref[q]) / np.linalg.norm(ref[q])) for q in range(8))
    return {"phi_sampled_rel_l2": err, "taps_max_rel_l2": terr, "n_sampled": int(ks.size),
            "plan_matches_oracle": same_bins}


def cpu_oracle_sample(uvw, args):
    """Time the FP64 oracle on a bounded sample and extrapolate to one full apply.

    Dense part: one w-bin's Z_p, oversampled FFT, adjoint FFT and crop at full image size.
    Sparse part: the oracle's G_p and G_p^dagger products for a sample of visibilities.
    t_apply = P * t_dense + M * t_sparse_per_visibility.
    """
    from oracle import operator as oop
    from oracle import plan as opl
    fov = math.radians(3.0)
    n = args.n
    rng = np.random.default_rng(11)
    ms = min(args.cpu_sample_vis, uvw.shape[0])
    sel = np.sort(rng.choice(uvw.shape[0], ms, replace=False))
    sub = uvw[sel]
    pp = opl.PlanParams(nx=n, ny=n, fov_x=fov, fov_y=fov, n_wbins=1)
    op = oop.Operator(sub, opl.make_plan(sub, pp))
    x = np.zeros((n, n), dtype=np.complex128)
    x.real = rng.random((n, n))
    t0 = time.perf_counter()
    Z = op.z_layer(0)
    X = op.fwd_grid(Z * x)
    t1 = time.perf_counter()
    y = op.G[0] @ X.ravel()
    Xh = (op.G[0].conj().T @ y).reshape(op.gx, op.gy)
    t2 = time.perf_counter()
    _ = np.conj(Z) * op.adj_grid(Xh)
    t3 = time.perf_counter()
    t_dense = (t1 - t0) + (t3 - t2)
    t_vis = (t2 - t1) / ms
    t_apply = args.bins * t_dense + uvw.shape[0] * t_vis
    return {"value": 1.0 / t_apply, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"one w-bin's dense part (Z_p, {2*n}^2 FP64 FFT pair, crop) and the sparse "
                      f"G/G^dagger products of {ms} sampled visibilities, extrapolated to "
                      f"{args.bins} bins and {uvw.shape[0]} visibilities",
            "t_dense_s": t_dense, "t_sparse_per_vis_s": t_vis, "t_apply_s": t_apply,
            "sample_wall_s": t3 - t0}


# ----------------------------------------------------------------------------- arms
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    uvw, _, _ = workload(args)
    vals = []
    for s in range(args.warmup + args.steps):
        r = cpu_oracle_sample(uvw, args)
        if s >= args.warmup:
            vals.append(r)
    v = float(np.mean([r["value"] for r in vals]))
    cb = dict(vals[-1])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": WORKLOAD, "M": uvw.shape[0], "n": args.n,
                                            "bins": args.bins},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_rimo(args):
    import torch
    import paper_2605_26347_gb300 as pkg

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    uvw, sky, t_synth = workload(args)
    fov = math.radians(3.0)
    params = pkg.default_params(args.n, args.n, fov, fov, n_wbins=args.bins, mode=pkg.MODE_STORED_G,
                                tile_size=args.tile)
    t0 = time.time()
    plan = pkg.Plan(uvw, params)
    t_plan = time.time() - t0
    info = plan.info()
    x = torch.from_numpy(sky).cuda()
    out = torch.empty_like(x)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        plan.phi_adj_phi(x, out)
    barrier()
    plan.profile(True)
    plan.profile_read(reset=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.phi_adj_phi(x, out)
    e1.record(stream)
    barrier()
    ms_total = e0.elapsed_time(e1)
    clk = clocks.stop()
    prof = plan.profile_read(reset=True)
    plan.profile(False)
    ms_step = ms_total / args.steps
    if dist is not None:
        t = torch.tensor([ms_step], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())

    # end to end through the public API: pinned host image in, host image out
    xh = torch.from_numpy(sky).pin_memory()
    oh = torch.empty_like(xh).pin_memory()
    xd = torch.empty_like(x)
    barrier()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        xd.copy_(xh, non_blocking=True)
        plan.phi_adj_phi(xd, out)
        oh.copy_(out, non_blocking=True)
    e3.record(stream)
    barrier()
    ms_e2e = e2.elapsed_time(e3) / args.steps
    if dist is not None:
        t = torch.tensor([ms_e2e], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_e2e = float(t.item())

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    M = uvw.shape[0]
    value = ws * 1000.0 / ms_step
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    sb = stage_bytes(info, args.n, info["P"], M, info["n_tiles"], info["tile_size"] + info["max_tile"] - 1)
    stage_ms = {k: v[0] for k, v in prof.items() if v[1] > 0 or v[0] > 0}
    launches = {k: v[1] for k, v in prof.items() if v[1] > 0}
    dom = max((k for k in stage_ms if k != "grid_clear"), key=lambda k: stage_ms[k])
    if dom in ("gtg", "inv_cols"):
        per_launch_bytes = sb[dom + "_per_step"] * args.steps / max(1, launches[dom])
    else:
        per_launch_bytes = sb[dom]
    per_launch_ms = stage_ms[dom] / max(1, launches[dom])
    achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        try:
            traffic = json.load(open(tfile)).get(dom)
        except Exception:
            traffic = None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": args.n, "grid": 2 * args.n, "M": M, "P": info["P"],
                   "fov_deg": 3.0, "kb_support": 7, "max_wsupport": 9, "mode": "stored_G",
                   "l2": "inputs larger than L2 (G taps %.1f GB, grids 2 x %.2f GB): no flush"
                         % (info["g_bytes"] / 1e9, (2 * args.n) ** 2 * 8 / 1e9),
                   "parallelism": f"replicas x{ws}"},
        "mvis_per_s": value * M / 1e6,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic,
                     "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks
                     else "fallback 6800 GB/s",
                     "bytes_per_launch": per_launch_bytes, "ms_per_launch": per_launch_ms},
        "apply_bytes": sb["apply_per_step"],
        "apply_gbs": sb["apply_per_step"] / (ms_step * 1e-3) / 1e9,
        "stages_ms_per_step": {k: v / args.steps for k, v in stage_ms.items()},
        "gpu_launches": int(sum(launches.values())),
        "clocks": clk,
        "e2e": {"value": ws * 1000.0 / ms_e2e, "unit": UNIT, "h2d_bytes_per_step": int(sky.nbytes),
                "d2h_bytes_per_step": int(sky.nbytes)},
        "plan": {"t_synth_s": t_synth, "t_plan_s": t_plan, "K": info["K"], "g_bytes": info["g_bytes"],
                 "n_blocks": info["n_blocks"], "n_tiles": info["n_tiles"], "max_tile": info["max_tile"],
                 "wr_max": info["wr_max"]},
    }
    if not args.no_oracle and ws == 1:
        line["rel_l2_err"] = oracle_error_sample(uvw, sky, plan, args)
        line["cpu_baseline"] = cpu_oracle_sample(uvw, args)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def run_wideband(args):
    """32 channels x 1024^2 (0.9-1.7 GHz, 0.5M-4M visibilities each, automatic w-bins per
    channel): every channel's Phi^dagger Phi in one graph launch per step."""
    import torch
    import synth
    import paper_2605_26347_gb300 as pkg

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    n, fov = 1024, math.radians(2.5)
    t0 = time.time()
    chans = synth.wideband_channels(n_chan=args.channels)
    t_synth = time.time() - t0
    plans, tiles, t_tune = [], [], 0.0
    t0 = time.time()
    for c, (f, uvw) in enumerate(chans):
        # higher frequencies see larger w (in wavelengths): 4 bins at 0.9 GHz up to 32 at 1.7 GHz
        nb = 0 if args.wideband_bins == "auto" else int(round(4 + 28 * c / max(1, len(chans) - 1)))
        params = pkg.default_params(n, n, fov, fov, n_wbins=nb)
        if args.autotune:
            t1 = time.time()
            tile, _ = pkg.autotune_tile(uvw, params, args.autotune)
            t_tune += time.time() - t1
            params.tile_size = tile
        plans.append(pkg.Plan(uvw, params))
        tiles.append(plans[-1].info()["tile_size"])
    t_plan = time.time() - t0 - t_tune
    infos = [p.info() for p in plans]
    M = sum(i["M"] for i in infos)
    batch = pkg.Batch(plans)
    sky = np.stack([synth.make_sky(n, 2004 + c) for c in range(len(plans))])
    x = torch.from_numpy(sky).cuda()
    out = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        batch.phi_adj_phi(x, out)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        batch.phi_adj_phi(x, out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_step = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    xh = torch.from_numpy(sky).pin_memory()
    oh = torch.empty_like(xh).pin_memory()
    xd = torch.empty_like(x)
    od = torch.empty_like(x)
    batch.phi_adj_phi(xd, od)  # record the graph for these buffers outside the timed region
    torch.cuda.synchronize()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        xd.copy_(xh, non_blocking=True)
        batch.phi_adj_phi(xd, od)
        oh.copy_(od, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e2.elapsed_time(e3) / args.steps
    if rank != 0:
        return
    Ps = [i["P"] for i in infos]
    line = {
        "metric": "batched wideband Phi^dagger Phi: all-channel applies/s (Mvis/s alongside)",
        "value": ws * 1000.0 / ms_step, "unit": "batch applies/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": {"workload": "wideband: %d channels 0.9-1.7 GHz, 1024^2 images, FoV 2.5 deg, "
                               "0.5M-4M visibilities per channel, %s w-bins per channel"
                               % (len(plans), "4-32 (linear in frequency)" if args.wideband_bins == "linear"
                                  else "automatic"),
                   "channels": len(plans), "M_total": M, "P_per_channel": Ps,
                   "tile_per_channel": tiles, "launch": "one CUDA graph per step",
                   "kernels_truncated_channels": sum(int(i["truncated"]) for i in infos),
                   "l2": "inputs larger than L2 (G taps %.1f GB): no flush" % (sum(i["g_bytes"] for i in infos) / 1e9),
                   "parallelism": f"replicas x{ws}"},
        "mvis_per_s": ws * M / (ms_step * 1e-3) / 1e6,
        "clocks": clk,
        "e2e": {"value": ws * 1000.0 / ms_e2e, "unit": "batch applies/s", "h2d_bytes_per_step": int(sky.nbytes),
                "d2h_bytes_per_step": int(sky.nbytes)},
        "plan": {"t_synth_s": t_synth, "t_plan_s": t_plan, "t_autotune_s": t_tune},
    }
    print(json.dumps(line), flush=True)


def run_holo(args):
    """Phi^dagger Phi through the holographic matrices H_p against the G^dagger G path on the
    same plan: build time, bytes, applies/s of both, and their relative l2 difference."""
    import torch
    import synth
    import paper_2605_26347_gb300 as pkg

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dense = args.config == "holo-dense"
    n, fov, bins, m = (256, 1.0, 4, 20_000_000) if dense else (2048, 2.5, 16, 20_000_000)
    if args.m != 50_000_000:
        m = args.m
    uvw = synth.make_uvw(m, 28_800, 1.28e9, seed=1003)
    sky = synth.make_sky(n, seed=2003)
    fovr = math.radians(fov)
    t0 = time.time()
    plan = pkg.Plan(uvw, pkg.default_params(n, n, fovr, fovr, n_wbins=bins, mode=pkg.MODE_STORED_G))
    t_plan = time.time() - t0
    x = torch.from_numpy(sky).cuda()
    out = torch.empty_like(x)
    stream = torch.cuda.current_stream()

    def timed(k):
        for _ in range(args.warmup):
            plan.phi_adj_phi(x, out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        plan.profile(True)
        plan.profile_read(reset=True)
        e0.record(stream)
        for _ in range(k):
            plan.phi_adj_phi(x, out)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = plan.profile_read(reset=True)
        plan.profile(False)
        return e0.elapsed_time(e1) / k, {kk: v[0] / k for kk, v in prof.items() if v[1] > 0}

    ms_g, st_g = timed(args.steps)
    ref = out.clone()
    torch.cuda.synchronize()
    t0 = time.time()
    plan.build_holographic()
    t_build = time.time() - t0
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms_h, st_h = timed(args.steps)
    clk = clocks.stop()
    diff = float(torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref))
    info = plan.info()
    if rank != 0:
        return
    line = {
        "metric": "Phi^dagger Phi applies/s through H_p (G^dagger G path alongside)",
        "value": ws * 1000.0 / ms_h, "unit": "applies/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_h, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": {"workload": ("holographic dense: 256^2 image, FoV 1 deg, 20M visibilities, 4 w-bins" if dense
                                else "holographic: 2048^2 image, 4096^2 grid, FoV 2.5 deg, 20M visibilities, 16 w-bins"),
                   "n": n, "M": m, "P": info["P"], "parallelism": f"replicas x{ws}"},
        "g_path_ms_per_apply": ms_g, "h_path_ms_per_apply": ms_h, "speedup_h_over_g": ms_g / ms_h,
        "h_vs_g_rel_l2": diff, "g_bytes": info["g_bytes"], "h_bytes": info["h_bytes"],
        "t_plan_s": t_plan, "t_h_build_s": t_build,
        "stages_ms_g": st_g, "stages_ms_h": st_h, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "wideband":
        run_wideband(args)
    elif args.config in ("holo", "holo-dense"):
        run_holo(args)
    else:
        run_rimo(args)


if __name__ == "__main__":
    main()
