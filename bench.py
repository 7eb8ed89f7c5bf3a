"""Benchmark: masked forward+backward of MaskGaussian's rasteriser on GB300.

One step = the whole hot path over one view of the 1.2M-Gaussian clustered
scene at 1557x1038: mask sampling + preprocess, binning, radix sort, tile
ranges, masked render, L1 loss gradient, render backward, preprocess
backward.  Inputs are resident in HBM; they (293 MB of parameters) are larger
than the 129 MB L2, so no separate flush is done.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  ``--impl reference`` times the CPU oracle (FP64,
host cores) on a bounded crop of the same workload.  Under torchrun (N > 1)
every rank renders its own replica (no data-path collective: the views are
independent); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "masked fwd+bwd ms & Mpix/s per view (1.2M Gaussians, 1557x1038) vs plain FP32 form"
WORKLOAD = "scene-scale single view, FP32: 1.2M clustered Gaussians, 1557x1038, f=1150"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _init_ranks(ws, local):
    """One process per GPU (NCCL); gloo when no GPU is present (host tests)."""
    import torch
    import torch.distributed as dist
    if ws > 1 and not dist.is_initialized():
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")


def _max_over_ranks(ms, ws, device):
    """The slowest rank's time: every rank renders its own replica, so the job
    ends when the last one does."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _whole_job_value(mpix_per_rank, ws, ms):
    """Mpix/s of the whole job: the pixels all ranks rendered (weak scaling,
    a fixed view per rank) over the slowest rank's step time."""
    return ws * mpix_per_rank / (ms * 1e-3)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        import tempfile
        self.index = index
        self.proc = None
        self.dir = tempfile.mkdtemp(prefix="maskgs_clocks_")
        self.path = os.path.join(self.dir, f"clocks_rank{index}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        try:
            os.remove(self.path)
            os.rmdir(self.dir)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


PROFILE_KERNEL = {"render_bwd": ("render_backward", "render.cu"),
                  "render": ("render_forward", "render.cu"),
                  "sort": ("onesweep", "binsort.cu"),
                  "preprocess": ("preprocess", "preprocess.cu"),
                  "preprocess_bwd": ("preprocess_backward", "preprocess.cu")}


def _profile_text(stage):
    """The committed ncu summary of the stage's kernel, if it was taken on the
    current source (else None)."""
    import hashlib
    import re
    if stage not in PROFILE_KERNEL:
        return None
    label, src = PROFILE_KERNEL[stage]
    path = os.path.join(ROOT, "profiles", f"{label}_scene_1p2M_1557x1038.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"sha256\[:16\] at capture: `([0-9a-f]+)`", text)
    cur = hashlib.sha256(open(os.path.join(ROOT, "paper_2412_20522_gb300", "csrc", src), "rb")
                         .read()).hexdigest()[:16]
    return text if m and m.group(1) == cur else None


def _profiled_traffic(stage):
    """DRAM bytes per launch from the committed ncu summary (None if stale)."""
    import re
    text = _profile_text(stage)
    t = re.search(r"traffic_bytes_per_launch \| (\d+)", text) if text else None
    return int(t.group(1)) if t else None


def _profiled_issue(stage, sms):
    """Warp instructions issued per cycle over all SMs, from the committed ncu
    summary, as a fraction of the SMs' issue capacity (one per SM sub-partition
    per cycle, four per SM); None if the summary is stale."""
    import re
    text = _profile_text(stage)
    t = re.search(r"sm__inst_executed\.sum\.per_cycle_active`\) \| ([0-9.]+)", text) if text else None
    if not t:
        return None
    ipc = float(t.group(1))
    return {"warp_inst_per_cycle": ipc, "capacity": 4 * sms, "frac": ipc / (4 * sms),
            "source": "ncu summary in profiles/ (same source)"}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# Algorithmic FP32 flops of the render kernels (FMA = 2; ex2, div = 1), from
# the arithmetic of the method per (pixel, splat) pair:
#   alpha evaluation (offset, eigen-form quadratic, exp, opacity)       15
#   forward blend of an unmasked splat (test T, weight, 3 colours)        9
#   backward of a masked splat (T_i, g.(c - b), dL/dM)                  12
#   backward of an unmasked splat (T_i, g.(c - b), dL/dM, dL/dc, b,
#     dL/dalpha, dL/do, dL/dconic, dL/dmean2d)                           48
FLOPS_ALPHA, FLOPS_FWD_BLEND, FLOPS_BWD_MASKED, FLOPS_BWD_UNMASKED = 15, 9, 12, 48


def render_flops(counts):
    walked, walked_on, blend_on, contrib_off = (int(x) for x in counts)
    fwd = walked_on * FLOPS_ALPHA + blend_on * FLOPS_FWD_BLEND
    bwd = walked * FLOPS_ALPHA + contrib_off * FLOPS_BWD_MASKED + blend_on * FLOPS_BWD_UNMASKED
    return fwd, bwd


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2412_20522_gb300 import abi, scenes
    from paper_2412_20522_gb300.rasterize import PARAM_NAMES, RasterConfig, Rasterizer

    ws, rank, local = _dist()
    _init_ranks(ws, local)
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    w2 = scenes.workload("c2_scene")
    g, cams, target = w2.gaussians, w2.cams, w2.targets[0]
    W, H = cams[0].width, cams[0].height
    params = {k: torch.as_tensor(np.ascontiguousarray(getattr(g, k))).to(dev)
              for k in PARAM_NAMES}
    tgt = torch.as_tensor(target).to(dev).reshape(-1)
    cfg = RasterConfig()
    rast = Rasterizer(dev)
    grads = {k: torch.empty_like(v) for k, v in params.items()}
    stream = torch.cuda.current_stream(dev)

    # size the instance buffers once (one synchronising step), then run the
    # whole sequence asynchronously
    rast.forward(params, cams, cfg, check=True)
    torch.cuda.synchronize()

    stage_names = ["preprocess", "bin", "sort", "render", "loss", "render_bwd", "preprocess_bwd"]

    def step(ev=None, count=False):
        # the render kernel takes the L1 loss in its epilogue ("loss" holds
        # only the mask loss, none here: lambda_m = 0)
        img, loss, dimg = rast.forward_l1(params, cams, cfg, tgt, check=False,
                                          count_fragments=count, stage_events=ev)
        rast.backward(dimg, grads, stage_events=ev, count_iterations=count)
        return loss

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    st = abi.mg_read_status(rast.status, rast._stream())
    if st.status != abi.MG_OK:
        raise RuntimeError(f"device status {st.status} after warm-up")

    # per-stage CUDA events over the timed steps (same stream as the kernels)
    evs = [{k: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for k in stage_names} for _ in range(args.steps)]
    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    clocks.start()
    time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        step(evs[i])
    t1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    eager_ms = _max_over_ranks(t0.elapsed_time(t1) / args.steps, ws, dev)

    # the headline: the same step (every kernel of a1-a12, the loss included)
    # replayed as one CUDA graph -- the production form, without the launch
    # gaps of eager issue -- timed the same way, right after
    from paper_2412_20522_gb300.autotune import GraphStep
    gs = GraphStep(params, cams, cfg, tgt)
    for _ in range(max(args.warmup, 3)):
        gs.replay()
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)

    def timed_block():
        # exactly K steps, a barrier and a synchronisation on both sides
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        g0.record(stream)
        for _ in range(args.steps):
            gs.replay()
        g1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        return g0.elapsed_time(g1)

    # blocks of K steps until at least 0.5 s is timed (the same number of
    # blocks on every rank); the headline is the median block
    blocks = [timed_block()]
    n_blocks = int(_max_over_ranks(max(3.0, math.ceil(500.0 / max(blocks[0], 1e-3))), ws, dev))
    n_blocks = min(n_blocks, 400)
    while len(blocks) < n_blocks:
        blocks.append(timed_block())
    clk = clocks.stop()
    ms = _max_over_ranks(statistics.median(blocks) / args.steps, ws, dev)
    timed_blocks = {"blocks": len(blocks), "steps_per_block": args.steps,
                    "block_ms_min": min(blocks), "block_ms_median": statistics.median(blocks),
                    "block_ms_max": max(blocks), "timed_s": sum(blocks) / 1e3}
    if gs.status() != abi.MG_OK:
        raise RuntimeError(f"device status {gs.status()} after the graph steps")
    # the timed step's launches (the graph step's rasteriser: fused L1 render)
    gpu_launches_per_step = gs.rast.launches_per_step() + gs.rast.backward_launches()
    del gs
    stage_ms = {k: statistics.mean(e[k][0].elapsed_time(e[k][1]) for e in evs) for k in stage_names}
    # per-step distribution: first stage's start to last stage's end of each step
    per_step = sorted(e["preprocess"][0].elapsed_time(e["preprocess_bwd"][1]) for e in evs)
    q = lambda f: per_step[min(len(per_step) - 1, int(f * len(per_step)))]
    step_dist = {"p10": q(0.10), "median": q(0.50), "p90": q(0.90), "n": len(per_step)}

    # counts of this workload (extra counted steps, outside the timed region):
    # the method's fragments over its own tile lists (whole 3-sigma
    # rectangles, as the 3DGS rasteriser bins), and what our kernels execute
    # over the filtered lists
    step(count=True)
    torch.cuda.synchronize()
    counts_exec = rast.frag_count.cpu().tolist()
    bwd_counts = rast.bwd_count.cpu().tolist()
    K_kept = int(rast.num_sorted.item())
    rect = Rasterizer(dev)
    rect.forward(params, cams, RasterConfig(bin_mode=abi.MG_BIN_RECT), check=True,
                 count_fragments=True)
    torch.cuda.synchronize()
    counts = rect.frag_count.cpu().tolist()
    del rect
    # algorithmic flops on the lists the timed kernels walk (filtered tile
    # lists, every pair up to each pixel's stop); the same on the whole
    # 3-sigma rectangles of the 3DGS binning (method-equivalent, secondary)
    flops_fwd, flops_bwd = render_flops(counts_exec)
    flops_fwd_rect, flops_bwd_rect = render_flops(counts)
    # executed by the backward: every (warp, splat) iteration evaluates 64 alphas
    flops_bwd_exec = (bwd_counts[0] * 64 * FLOPS_ALPHA + counts_exec[3] * FLOPS_BWD_MASKED +
                      counts_exec[2] * FLOPS_BWD_UNMASKED)
    K = int(rast.num_instances.item())
    so = rast.splat_outputs()
    visible = int((so["radius"] > 0).sum().item())
    mask_on = float(so["mask"].float().mean().item())

    # end to end through the C ABI with host buffers: every step copies the
    # parameters and the target from pinned host memory and the image, loss
    # and all gradients back, pipelined over copy and compute streams
    # (HostPipeline); the same steps with the copies in series are reported too
    from paper_2412_20522_gb300.hoststep import HostPipeline
    host_params = {k: v.cpu().pin_memory() for k, v in params.items()}
    host_tgt = tgt.cpu().pin_memory()
    hp = HostPipeline(host_params, host_tgt, cams, cfg, device=dev)      # graph replays
    h2d, d2h = hp.h2d_bytes(), hp.d2h_bytes()
    e2e_n = max(50, args.steps)
    for _ in range(3):
        hp.step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if ws > 1:
        dist.barrier()
    e0.record(hp.h2d)
    for _ in range(e2e_n):
        b = hp.step()
    e1.record(hp.d2h)
    torch.cuda.synchronize()
    e2e_ms = _max_over_ranks(e0.elapsed_time(e1) / e2e_n, ws, dev)
    _, host_loss, _ = hp.results(b)
    e2e_loss = float(host_loss[0])
    link = host_link_times(hp)
    del hp

    host_img = torch.empty(3 * W * H, dtype=torch.float32).pin_memory()
    host_grads = {k: torch.empty(v.shape, dtype=torch.float32).pin_memory() for k, v in params.items()}
    host_loss1 = torch.empty(1, dtype=torch.float32).pin_memory()

    def serial_step():
        for k in PARAM_NAMES:
            params[k].copy_(host_params[k], non_blocking=True)
        tgt.copy_(host_tgt, non_blocking=True)
        img, loss, dimg = rast.forward_l1(params, cams, cfg, tgt, check=False)
        rast.backward(dimg, grads)
        host_img.copy_(img, non_blocking=True)
        host_loss1.copy_(loss, non_blocking=True)
        for k in PARAM_NAMES:
            host_grads[k].copy_(grads[k], non_blocking=True)

    for _ in range(2):
        serial_step()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(max(3, e2e_n // 2)):
        serial_step()
    e1.record(stream)
    torch.cuda.synchronize()
    serial_ms = _max_over_ranks(e0.elapsed_time(e1) / max(3, e2e_n // 2), ws, dev)

    peaks, peak_src = _peaks()
    mpix = W * H / 1e6
    # dominant kernel: the stage with the largest share
    dom = max(("render_bwd", "render", "sort", "preprocess", "preprocess_bwd"),
              key=lambda k: stage_ms[k])
    smmax = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak_tflops = sms * 128 * 2 * smmax * 1e6 / 1e12
    if dom in ("render", "render_bwd"):
        achieved = (flops_fwd if dom == "render" else flops_bwd) / (stage_ms[dom] * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": fp32_peak_tflops,
                "unit": "TFLOP/s", "frac": achieved / fp32_peak_tflops,
                "traffic": _profiled_traffic(dom),
                "peak_source": f"FP32 FMA lanes x 2 x max SM clock ({sms} SMs, {smmax:.0f} MHz)",
                "flops_basis": "the filtered tile lists the kernels walk: every (pixel, splat) "
                               "pair up to each pixel's stop, 15 flops of alpha; masked splats "
                               "above the floor 12, blended splats 48 (backward)",
                "flops_per_launch": flops_fwd if dom == "render" else flops_bwd,
                "pairs": {"walked": counts_exec[0], "walked_unmasked": counts_exec[1],
                          "blended": counts_exec[2], "masked_above_floor": counts_exec[3]}}
        rect_f = (flops_fwd_rect if dom == "render" else flops_bwd_rect)
        roof["method_equivalent"] = {
            "achieved": rect_f / (stage_ms[dom] * 1e-3) / 1e12,
            "frac": rect_f / (stage_ms[dom] * 1e-3) / 1e12 / fp32_peak_tflops,
            "basis": "the same flops counted on the whole 3-sigma rectangle lists of the 3DGS "
                     "binning (work the tile filter removes is counted as done)"}
        # the kernels are bound by instruction issue: its utilisation
        issue = _profiled_issue(dom, sms)
        if issue is not None:
            roof["issue"] = issue
        if dom == "render_bwd":
            ex = flops_bwd_exec / (stage_ms[dom] * 1e-3) / 1e12
            roof["executed"] = {"achieved": ex, "frac": ex / fp32_peak_tflops,
                                "basis": "alphas our kernel evaluates (warp iterations x 64) "
                                         "+ masked and blended fragment work"}
    else:
        bytes_per = {"sort": K * 152, "preprocess": g.n * 244 + visible * 60,
                     "preprocess_bwd": g.n * (244 + 244) + visible * 48}[dom]
        achieved = bytes_per / (stage_ms[dom] * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved,
                "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                "frac": achieved / float(peaks["hbm_gbs"]), "traffic": _profiled_traffic(dom),
                "peak_source": peak_src}

    # algorithmic bytes of the memory-bound stages (FP32 storage; per-unit
    # figures of the design notes): achieved GB/s against the measured copy peak
    n_g, R_ = g.n, g.n
    tiles_total = int(rast._state["tiles"])
    sh_b = 3 * 16 * 4
    stage_bytes = {
        # read means, scales, quats, opacity, mask scores (all) + SH (visible);
        # write tiles, radius, clamp, mask, soft mask, depth key (all) +
        # render and bin records (visible)
        "preprocess": n_g * (12 + 12 + 16 + 4 + 8) + visible * sh_b +
                      n_g * (4 + 4 + 1 + 1 + 4 + 4) + visible * (48 + 48),
        # depth order (histogram and first pass read the keys, the first pass
        # writes key + index, 3 passes of key + index), scan (tiles, order in;
        # offsets out), duplicate (order, offset, tiles, binning record per
        # visible record; key + value per candidate)
        "bin": R_ * 4 + R_ * (4 + 8) + 3 * R_ * 16 + R_ * 12 + visible * (4 + 4 + 4 + 48) +
               K * 8,
        # histogram (keys), first pass (all candidates in, kept out), second
        # pass (kept in and out), ranges (kept keys in, tile ranges out)
        "sort": K * 4 + K * 8 + K_kept * 8 + K_kept * 16 + K_kept * 4 + tiles_total * 8,
        # read parameters (all) + 2D gradients, SH (visible); write every gradient
        "preprocess_bwd": n_g * (12 + 12 + 16 + 4 + 4) + visible * (48 + sh_b + 4 + 1) +
                          n_g * (12 + 12 + 16 + 4 + 8 + sh_b),
    }
    hbm = float(_peaks()[0]["hbm_gbs"])
    stage_roof = {k: {"bytes": int(b), "achieved_gbs": b / (stage_ms[k] * 1e-3) / 1e9,
                      "frac_of_measured_hbm": b / (stage_ms[k] * 1e-3) / 1e9 / hbm}
                  for k, b in stage_bytes.items()}

    line = {
        "metric": METRIC, "value": _whole_job_value(mpix, ws, ms), "unit": "Mpix/s", "n_gpus": ws,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
        "execution": "the whole step replayed as one CUDA graph (autotune.GraphStep); "
                     "eager issue of the same kernels in eager_ms_per_step, which the stage "
                     "split and the per-step distribution come from",
        "eager_ms_per_step": eager_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded cluster-mixture scene standing in for Mip-NeRF360-scale captures)",
        "config": {"workload": WORKLOAD, "gaussians": g.n, "width": W, "height": H, "views": 1,
                   "tile": "16x16", "sh_degree": 3, "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"replicas x{ws}", "instances_K": K,
                   "instances_kept": K_kept,
                   "fragments": {"walked": counts[0], "walked_unmasked": counts[1],
                                 "blended": counts[2], "masked_above_floor": counts[3],
                                 "walked_filtered_lists": counts_exec[0]},
                   "render_gflop": {"fwd": flops_fwd / 1e9, "bwd": flops_bwd / 1e9,
                                    "fwd_rect_lists": flops_fwd_rect / 1e9,
                                    "bwd_rect_lists": flops_bwd_rect / 1e9},
                   "bwd_iterations": dict(zip(("list", "masked", "contrib_unmasked",
                                               "contrib_masked", "contrib_lanes", "batches"),
                                              bwd_counts)),
                   "visible": visible, "mask_on_fraction": mask_on},
        "stage_ms": stage_ms,
        "timed_blocks": timed_blocks,
        "step_ms_distribution": step_dist,
        "roofline": roof,
        "stage_roofline_hbm": stage_roof,
        "e2e": {"value": _whole_job_value(mpix, ws, e2e_ms), "unit": "Mpix/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "copies": "pinned host <-> device every step, overlapped with the neighbouring "
                          "steps' compute (two copy streams, double-buffered; each slot "
                          "replays its captured graph of the step)",
                "steps_timed": e2e_n,
                "achieved_h2d_gbs": h2d / (e2e_ms * 1e-3) / 1e9,
                "achieved_d2h_gbs": d2h / (e2e_ms * 1e-3) / 1e9,
                "host_link": link,
                "serial_ms_per_step": serial_ms, "loss": e2e_loss},
        "gpu_launches": gpu_launches_per_step * args.steps,
        "clocks": clk,
    }
    if not args.no_forms and ws == 1:
        # the single-GPU forms (multi-view graph, storage, scene batch, next
        # rows); a multi-rank run times the replicated step only
        line["forms"] = run_forms(dev, g, cams, target, eager_ms, W * H)
        line["forms"]["next_rows"] = run_next_rows(dev, g, cams, target, ms, peaks)
        line["forms"]["tiny_c1"] = tiny_workload_times(dev)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # the oracle runs only here: timed as the CPU baseline, and compared
        # with the GPU output by output (parity, and the precision forms'
        # error per output)
        cb, parity = oracle_step_and_parity(dev, params, g, cams[0], target)
        line["cpu_baseline"] = cb
        line["cpu_baseline"]["tiny_workload"] = tiny_workload_oracle_seconds()
        line["parity"] = parity
        line["precision_c4_error"] = precision_c4_error(dev)
    if clk is not None and clk["samples"] < 3:
        line["clocks"]["note"] = "timed region shorter than three 100 ms samples"
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def host_link_times(hp, n=20):
    """The host link alone, with the step's own buffers: every input copied
    host -> device, every output device -> host, each direction by itself and
    both at once on their two streams (no compute), ms per step and GB/s."""
    import torch
    from paper_2412_20522_gb300.rasterize import PARAM_NAMES

    def h2d():
        with torch.cuda.stream(hp.h2d):
            for k in PARAM_NAMES:
                hp.params[0][k].copy_(hp.host_params[k], non_blocking=True)
            hp.target[0].copy_(hp.host_target, non_blocking=True)

    def d2h():
        with torch.cuda.stream(hp.d2h):
            hp.host_image[0].copy_(hp.image[0], non_blocking=True)
            hp.host_loss[0].copy_(hp.loss[0], non_blocking=True)
            for k in PARAM_NAMES:
                hp.host_grads[0][k].copy_(hp.grads[0][k], non_blocking=True)

    out = {}
    for name, fns in (("h2d_alone", (h2d,)), ("d2h_alone", (d2h,)), ("both", (h2d, d2h))):
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(n):
            for f in fns:
                f()
        torch.cuda.synchronize()
        out[name + "_ms"] = (time.perf_counter() - t) * 1e3 / n
    out["h2d_alone_gbs"] = hp.h2d_bytes() / (out["h2d_alone_ms"] * 1e-3) / 1e9
    out["d2h_alone_gbs"] = hp.d2h_bytes() / (out["d2h_alone_ms"] * 1e-3) / 1e9
    return out


def _device_params(g, dev, storage=None):
    import torch
    from paper_2412_20522_gb300.rasterize import PARAM_NAMES, STORED
    p = {k: torch.as_tensor(np.ascontiguousarray(getattr(g, k))).to(dev) for k in PARAM_NAMES}
    if storage is not None:
        for k in STORED:
            p[k] = p[k].to(storage)
    return p


def run_forms(dev, g, cams, target, plain_ms, plain_pix, steps=10):
    """The batched and reduced-storage forms, each against the plain FP32
    single-view form measured above (same GPU, same run)."""
    import torch
    from paper_2412_20522_gb300 import scenes
    from paper_2412_20522_gb300.autotune import GraphStep, autotune, time_step
    from paper_2412_20522_gb300.rasterize import RasterConfig

    forms = {"plain_fp32_single_view": {"ms_per_step": plain_ms,
                                        "mpix_per_s": plain_pix / 1e6 / (plain_ms * 1e-3)}}

    # multi-view batch: 8 ring cameras, one shared mask sample, summed
    # gradients, one captured launch sequence, autotuned tile shape
    w3 = scenes.workload("c3_multiview")         # the same scene as g, 8 ring cameras
    cams8 = w3.cams
    p = _device_params(w3.gaussians, dev)
    tgt8 = torch.as_tensor(np.concatenate([t.reshape(-1) for t in w3.targets])).to(dev)
    tuned = autotune(p, cams8, tgt8, steps=3)
    gs = GraphStep(p, cams8, tuned, tgt8)
    ms = time_step(gs.replay, steps=steps)
    pix = sum(c.width * c.height for c in cams8)
    forms["multiview_graph"] = {"views": len(cams8), "tile": f"{tuned.tile_w}x{tuned.tile_h}",
                                "sort": tuned.sort,
                                "staging": [tuned.render_batch, tuned.render_batch_bwd],
                                "ms_per_step": ms, "mpix_per_s": pix / 1e6 / (ms * 1e-3),
                                "status": gs.status()}
    del gs, p, w3
    torch.cuda.empty_cache()

    # precision variant: 3M Gaussians, 4 views at 1957x1297, BF16 / FP16 storage
    w4 = scenes.workload("c4_precision")
    g3, cams4 = w4.gaussians, w4.cams
    tgt4 = torch.as_tensor(np.concatenate([t.reshape(-1) for t in w4.targets])).to(dev)
    pix4 = sum(c.width * c.height for c in cams4)
    for name, dt in (("precision_bf16", torch.bfloat16), ("precision_fp16", torch.float16),
                     ("precision_fp32", None)):
        p = _device_params(g3, dev, dt)
        gs = GraphStep(p, cams4, RasterConfig(), tgt4)
        ms = time_step(gs.replay, steps=max(3, steps // 2))
        forms[name] = {"gaussians": g3.n, "views": len(cams4), "ms_per_step": ms,
                       "mpix_per_s": pix4 / 1e6 / (ms * 1e-3), "status": gs.status()}
        del gs, p
        torch.cuda.empty_cache()
    del g3, w4

    # uneven batch: 6 scenes, one camera each, BF16 storage, one launch sequence
    w5 = scenes.workload("c5_uneven")
    scs = [part[0] for part in w5.parts]
    sizes = [sc.n for sc in scs]
    camsu = w5.cams
    res = [(c.width, c.height) for c in camsu]
    tgtu = torch.as_tensor(np.concatenate([t.reshape(-1) for t in w5.targets])).to(dev)
    ranges = w5.view_ranges
    p = _device_params(w5.gaussians, dev, torch.bfloat16)
    gs = GraphStep(p, camsu, RasterConfig(), tgtu, view_ranges=ranges)
    ms = time_step(gs.replay, steps=max(3, steps // 2))
    pix = sum(w * h for w, h in res)
    per_scene = []
    del gs, p
    torch.cuda.empty_cache()
    for k, sc in enumerate(scs):
        pk = _device_params(sc, dev, torch.bfloat16)
        w, h = res[k]
        tk = torch.as_tensor(w5.targets[k]).to(dev).reshape(-1)
        gk = GraphStep(pk, [camsu[k]], RasterConfig(), tk)
        mk = time_step(gk.replay, steps=max(3, steps // 2))
        per_scene.append({"gaussians": sizes[k], "resolution": f"{w}x{h}", "ms_per_step": mk,
                          "mpix_per_s": w * h / 1e6 / (mk * 1e-3)})
        del gk, pk
        torch.cuda.empty_cache()
    forms["uneven_batch_bf16"] = {"scenes": len(sizes), "ms_per_step": ms,
                                  "mpix_per_s": pix / 1e6 / (ms * 1e-3), "per_scene": per_scene}
    return forms


PRUNE_OPS_PER_DRAW = 98 + 10 + 4 * 29 + 3


def run_next_rows(dev, g, cams, target, plain_ms, peaks, steps=10):
    """The rows after the hot path, on the same 1.2M-Gaussian view: the mask
    loss (Eq. 7-8) and the ablations of Sec. 4.3 in the training step; the
    pruning of Sec. 3.5 (the sampler ALU-bound, the compaction HBM-bound); the inference
    renderer of the pruned model (rendering speed, Sec. 4.2)."""
    import torch
    from paper_2412_20522_gb300 import prune, scenes
    from paper_2412_20522_gb300.autotune import GraphStep, time_step
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer

    out = {}
    p = _device_params(g, dev)
    tgt = torch.as_tensor(target).to(dev).reshape(-1)
    base = GraphStep(p, cams, RasterConfig(), tgt)
    out["graph_step_ms"] = time_step(base.replay, steps=steps)
    del base
    # the same step with tiles launched in tile-id order (no longest-first order)
    plain = GraphStep(p, cams, RasterConfig(), tgt, tile_order=False)
    out["graph_step_ms_tile_id_order"] = time_step(plain.replay, steps=steps)
    del plain
    for name, cfg in (("mask_loss_l2_lambda0.1", RasterConfig(lambda_m=0.1)),
                      ("ablation_mask_x_opacity", RasterConfig(mask_apply=1)),
                      ("ablation_ste_threshold_0.01",
                       RasterConfig(mask_mode=3, ste_logit=RasterConfig.ste_logit_of(0.01)))):
        gs = GraphStep(p, cams, cfg, tgt)
        out[name] = {"ms_per_step": time_step(gs.replay, steps=steps), "status": gs.status()}
        del gs
    torch.cuda.empty_cache()

    # pruning: converged-looking mask scores (62.4 % almost never sampled)
    pp = dict(p)
    pp["mask_logits"] = torch.as_tensor(scenes.converged_mask_logits(g.n)).to(dev)
    n = g.n
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    comp = prune.Compactor(dev)
    keep = prune.prune_sample(pp, 7, 30000, 10)
    comp.run(pp, keep)
    torch.cuda.synchronize()
    t_s, t_c = [], []
    for _ in range(steps):
        ev[0].record()
        keep = prune.prune_sample(pp, 7, 30000, 10)
        ev[1].record()
        comp.run(pp, keep)
        ev[2].record()
        torch.cuda.synchronize()
        t_s.append(ev[0].elapsed_time(ev[1]))
        t_c.append(ev[1].elapsed_time(ev[2]))
    small, _ = comp.result()
    kept = small["means"].shape[0]
    row = sum(v[0].numel() * v.element_size() for v in pp.values())      # 244 B (FP32)
    sample_bytes = n * (8 + 1)
    compact_bytes = n * (1 + 4 + 4) + 2 * kept * row
    hbm = float(peaks["hbm_gbs"])
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = sms * 128 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    ms_s, ms_c = statistics.median(t_s), statistics.median(t_c)
    out["prune"] = {
        "gaussians": n, "kept": kept, "pruned_fraction": 1 - kept / n, "draws": 10,
        "sample_ms": ms_s, "compact_ms": ms_c,
        # the sampler is bound by its arithmetic: per draw a Philox4x32-10 block
        # (98 integer ops), two uniforms (10), four correctly rounded logs (29
        # ops each, the division counted once) and the margin (3); every warp
        # runs all ten draws (it holds a Gaussian absent in every draw)
        "roofline_sample": {"bound": "alu",
                            "achieved": n * 10 * PRUNE_OPS_PER_DRAW / (ms_s * 1e-3) / 1e12,
                            "peak": alu_peak, "unit": "Tops/s",
                            "frac": n * 10 * PRUNE_OPS_PER_DRAW / (ms_s * 1e-3) / 1e12 / alu_peak,
                            "basis": f"{PRUNE_OPS_PER_DRAW} 32-bit ops per draw x 10 draws per "
                                     "lane; peak: one op per FP32 lane per clock",
                            "hbm_frac": sample_bytes / (ms_s * 1e-3) / 1e9 / hbm},
        "roofline_compact": {"bound": "hbm", "achieved": compact_bytes / (ms_c * 1e-3) / 1e9,
                             "peak": hbm, "unit": "GB/s",
                             "frac": compact_bytes / (ms_c * 1e-3) / 1e9 / hbm},
        "bytes_note": "sample: 8 B logits + 1 B flag per Gaussian; compact: flag + index "
                      "write + index read per Gaussian, one read and one write of each "
                      f"survivor's {row} B row"}

    # inference renderer (forward only, every Gaussian present) of the full
    # and of the pruned model
    W, H = cams[0].width, cams[0].height
    for name, params in (("inference_full", p), ("inference_pruned", small)):
        r = Rasterizer(dev)
        cfg = RasterConfig()
        r.forward(params, cams, cfg, check=True, inference=True)
        torch.cuda.synchronize()
        ms = time_step(lambda: r.forward(params, cams, cfg, check=False, inference=True),
                       steps=4 * steps)
        out[name] = {"gaussians": int(params["means"].shape[0]), "ms_per_frame": ms,
                     "fps": 1000.0 / ms, "mpix_per_s": W * H / 1e6 / (ms * 1e-3)}
        del r
    out["inference_speedup_pruned"] = out["inference_full"]["ms_per_frame"] / \
        out["inference_pruned"]["ms_per_frame"]
    del p, pp, small, comp
    torch.cuda.empty_cache()
    return out


def _crop_camera(cam, cw, ch):
    from paper_2412_20522_gb300 import scenes
    x0 = (cam.width - cw) // 2
    y0 = (cam.height - ch) // 2
    return scenes.Camera(cw, ch, cam.fx, cam.fy, cam.cx - x0, cam.cy - y0, cam.viewmat,
                         cam.cam_pos, cam.near)


def cpu_baseline_sample(steps=1, crop=None):
    """The oracle (FP64, all host cores through OpenMP) on a bounded sample of
    the same workload: masked forward + backward of the 1.2M-Gaussian scene
    (all Gaussians preprocessed) for the full 1557x1038 view, or for its
    centre ``crop`` (w, h)."""
    from oracle import pipeline
    from paper_2412_20522_gb300 import scenes
    w2 = scenes.workload("c2_scene")
    g, cams, target = w2.gaussians, w2.cams, w2.targets[0]
    cam, tgt = cams[0], target
    if crop is not None:
        cw, ch = crop
        cam = _crop_camera(cams[0], cw, ch)
        x0, y0 = (cams[0].width - cw) // 2, (cams[0].height - ch) // 2
        tgt = target[:, y0:y0 + ch, x0:x0 + cw]
    times = []
    for _ in range(steps):
        t = time.perf_counter()
        pipeline.forward_backward_l1(g, [cam], [tgt], pipeline.OracleConfig())
        times.append(time.perf_counter() - t)
    t = statistics.median(times)
    what = "the full 1557x1038 view" if crop is None else f"the centre {cam.width}x{cam.height} crop of the 1557x1038 view"
    return {"value": cam.width * cam.height / 1e6 / t, "unit": "Mpix/s", "cores": os.cpu_count(),
            "cpu": _cpu_model(), "kind": "oracle", "seconds_per_step": t,
            "sample": f"{what}: masked fwd+bwd of the 1.2M-Gaussian scene, all Gaussians "
                      f"preprocessed, FP64, OpenMP over tiles; median of {steps} step(s)"}


PARITY_EPS = 1e-4          # straddle band of the oracle's fragment decisions (relative)
IMG_TOL, GRAD_TOL = 2e-4, 1e-3
PARAMS = ("means", "log_scales", "quats", "opacity_logit", "sh", "mask_logits")


def error_stats(a, b):
    """a (GPU) against b (oracle), flattened: relative L2; the largest
    absolute error over the largest |b|; and, over the elements with
    |b| >= 1e-3 max|b|, the worst relative error and how many exceed 1e-2 --
    a per-tensor norm alone could hide a few badly wrong elements."""
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    d = a - b
    nb = float(np.linalg.norm(b))
    out = {"rel_l2": float(np.linalg.norm(d)) / nb if nb > 0 else float(np.linalg.norm(d))}
    mb = float(np.abs(b).max()) if b.size else 0.0
    out["max_abs_err_over_max_ref"] = float(np.abs(d).max()) / mb if mb > 0 else 0.0
    sel = np.abs(b) >= 1e-3 * mb if mb > 0 else np.zeros(b.shape, bool)
    if sel.any():
        r = np.abs(d[sel]) / np.abs(b[sel])
        out["worst_rel_elem"] = float(r.max())
        out["elems_rel_over_1e-2"] = int((r > 1e-2).sum())
        out["elems_compared"] = int(sel.sum())
    return out


def _oracle_step(g, cam, target):
    """The oracle's masked forward, L1 loss gradient (zero on straddle
    pixels) and backward of one view; returns (seconds, views, M, grads,
    per_view, dimg, straddle)."""
    from oracle import pipeline
    ocfg = pipeline.OracleConfig(eps=PARITY_EPS)
    t0 = time.perf_counter()
    views, M, minfo = pipeline.forward(g, [cam], ocfg)
    v = views[0]
    straddle = (v.out["flags"] & 11) != 0
    _, dimg = pipeline.l1_loss_grad(v.out["image"], target)
    dimg = dimg * (~straddle)[None]
    grads, per_view = pipeline.backward(g, [cam], ocfg, views, M, minfo, [dimg])
    return time.perf_counter() - t0, views, M, grads, per_view, dimg, straddle


def _gpu_vs_oracle(rast, img, out, cam, views, M, grads, per_view, straddle, lists=True):
    """Every output of a GPU step against the oracle's (one view)."""
    H, W = cam.height, cam.width
    v = views[0]
    so = rast.splat_outputs()
    d = np.abs(img.cpu().numpy().reshape(3, H, W) - v.out["image"]).max(0)
    dT = np.abs(so["final_T"].cpu().numpy().reshape(H, W) - v.out["final_T"])
    gN = so["n_contrib"].cpu().numpy().reshape(H, W)
    clean = ~straddle
    rep = {
        "image": {"pixels": H * W, "straddle_pixels": int(straddle.sum()),
                  "pixels_over_tol": int((d > IMG_TOL).sum()),
                  "pixels_over_tol_not_straddle": int(((d > IMG_TOL) & clean).sum()),
                  "max_abs_err_not_straddle": float(d[clean].max()) if clean.any() else 0.0,
                  "max_abs_err_all": float(d.max()), "tolerance": IMG_TOL},
        "final_T": {"max_abs_err_not_straddle": float(dT[clean].max()) if clean.any() else 0.0,
                    "max_abs_err_all": float(dT.max())},
        "stop_index_mismatch_not_straddle": int((gN != v.out["n_contrib"])[clean].sum()),
        "mask_mismatch": int((so["mask"].cpu().numpy() != M).sum()),
    }
    if lists:
        Ks = int(so["num_sorted"].item())
        keys = rast.sorted_keys().cpu().numpy().view(np.uint32)[:Ks]
        vals = so["sorted_vals"].cpu().numpy().view(np.uint32)[:Ks]
        rng = so["ranges"].cpu().numpy().view(np.uint32).reshape(-1, 2)
        ne = v.ranges[:, 1] > v.ranges[:, 0]
        rep["tile_lists"] = {
            "candidates_equal": int(so["num_instances"].item()) == v.K,
            "kept": Ks, "kept_equal": Ks == v.K_kept,
            "sorted_keys_equal": bool(Ks == v.K_kept and np.array_equal(
                keys.astype(np.uint64), v.sorted_keys >> np.uint64(32))),
            "sorted_values_equal": bool(Ks == v.K_kept and np.array_equal(vals, v.sorted_vals)),
            "ranges_equal": bool(np.array_equal(rng[ne], v.ranges[ne]))}
    gr = {k: error_stats(out[k].cpu().numpy(), grads[k]) for k in PARAMS}
    g2 = so["grad2d"].cpu().numpy().reshape(-1, 12)
    pv = per_view[0]
    for name, sl in (("dmean2d", slice(0, 2)), ("dconic", slice(2, 5)), ("dopacity", 5),
                     ("drgb", slice(6, 9)), ("dmask", 9)):
        gr["2d_" + name] = error_stats(g2[:, sl], pv[name])
    rep["gradients"] = gr
    rep["gradients_within_tol"] = all(e["rel_l2"] <= GRAD_TOL for e in gr.values())
    rep["grad_tolerance_rel_l2"] = GRAD_TOL
    return rep


def oracle_step_and_parity(dev, params, g, cam, target):
    """CPU-baseline leg: the oracle's step on the full benchmark view, timed,
    and the GPU step on the same inputs and upstream gradient compared with
    it output by output (the parity record of the bench line)."""
    import torch
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    secs, views, M, grads, per_view, dimg, straddle = _oracle_step(g, cam, target)
    cb = {"value": cam.width * cam.height / 1e6 / secs, "unit": "Mpix/s", "cores": os.cpu_count(),
          "cpu": _cpu_model(), "kind": "oracle", "seconds_per_step": secs,
          "sample": f"the full {cam.width}x{cam.height} view: masked fwd + L1 loss + bwd of the "
                    "1.2M-Gaussian scene, all Gaussians preprocessed, FP64, OpenMP over tiles "
                    "(straddle pixels' upstream gradient zeroed for the parity comparison); one step"}
    rast = Rasterizer(dev)
    img = rast.forward(params, [cam], RasterConfig())
    out = rast.backward(torch.as_tensor(dimg.astype(np.float32).reshape(-1)).to(dev))
    torch.cuda.synchronize()
    rep = _gpu_vs_oracle(rast, img, out, cam, views, M, grads, per_view, straddle)
    rep["upstream"] = "the oracle's L1 gradient with straddle pixels zeroed, on both sides"
    rep["straddle_band"] = PARITY_EPS
    return cb, rep


def c4_crop_workload():
    """The precision configuration (c4_precision: 3M clustered Gaussians,
    four ring views at 1957x1297): the centre crop of its error view as a
    camera, and the same crop of that view's target."""
    from paper_2412_20522_gb300 import scenes
    w4 = scenes.workload("c4_precision")
    v, n = w4.spec["error_crop"]["view"], w4.spec["error_crop"]["size"]
    full = w4.cams[v]
    cam = _crop_camera(full, n, n)
    x0, y0 = (full.width - n) // 2, (full.height - n) // 2
    tgt = w4.targets[v][:, y0:y0 + n, x0:x0 + n].copy()
    return w4.gaussians, cam, tgt


def precision_c4_error(dev):
    """Error of each output (image, final T, stop index, the six parameter
    gradients and the five 2D gradients) against the FP64 oracle on the FP32
    parameters, for BF16, FP16 and FP32 storage of log-scales, quaternions,
    opacity logits and SH, at the precision configuration's crop."""
    import torch
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    g3, cam, tgt = c4_crop_workload()
    _, views, M, grads, per_view, dimg, straddle = _oracle_step(g3, cam, tgt)
    d = torch.as_tensor(dimg.astype(np.float32).reshape(-1)).to(dev)
    res = {"gaussians": g3.n, "view": "centre 64x64 crop of view 0 of 4 at 1957x1297",
           "upstream": "the oracle's L1 gradient with straddle pixels zeroed"}
    for name, dt in (("bf16", torch.bfloat16), ("fp16", torch.float16), ("fp32", None)):
        p = _device_params(g3, dev, dt)
        rast = Rasterizer(dev)
        img = rast.forward(p, [cam], RasterConfig())
        out = rast.backward(d)
        torch.cuda.synchronize()
        res[name] = _gpu_vs_oracle(rast, img, out, cam, views, M, grads, per_view, straddle,
                                   lists=(dt is None))
        del p, rast
    torch.cuda.empty_cache()
    return res


def _cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith(("model name", "cpu model")):
                    return ln.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def tiny_workload_times(dev, steps=50):
    """The tiny configuration (10 000 Gaussians, 128x128): the GPU step, eager
    and captured (the oracle's time on it is part of the CPU baseline)."""
    import torch
    from paper_2412_20522_gb300 import scenes
    from paper_2412_20522_gb300.autotune import GraphStep, time_step
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    g, cams, tgt = scenes.tiny_workload()
    p = _device_params(g, dev)
    t = torch.as_tensor(tgt).to(dev).reshape(-1)
    rast = Rasterizer(dev)
    cfg = RasterConfig()
    rast.forward(p, cams, cfg, check=True)

    def eager():
        _, _, dimg = rast.forward_l1(p, cams, cfg, t, check=False)
        rast.backward(dimg)
    ms_eager = time_step(eager, steps=steps)
    gs = GraphStep(p, cams, cfg, t)
    ms_graph = time_step(gs.replay, steps=steps)
    return {"gaussians": g.n, "resolution": "128x128", "gpu_ms_eager": ms_eager,
            "gpu_ms_graph": ms_graph}


def tiny_workload_oracle_seconds():
    """The oracle's masked forward+backward of the tiny configuration on the
    host cores (CPU-baseline leg), and on one core (a fresh process with one
    OpenMP thread and one torch thread)."""
    from oracle import pipeline
    from paper_2412_20522_gb300 import scenes
    g, cams, tgt = scenes.tiny_workload()
    t0 = time.perf_counter()
    pipeline.forward_backward_l1(g, cams, [tgt], pipeline.OracleConfig())
    all_cores = time.perf_counter() - t0
    code = ("import sys, time; sys.path.insert(0, %r); import torch; torch.set_num_threads(1); "
            "from oracle import pipeline; from paper_2412_20522_gb300 import scenes; "
            "g, cams, tgt = scenes.tiny_workload(); t0 = time.perf_counter(); "
            "pipeline.forward_backward_l1(g, cams, [tgt], pipeline.OracleConfig()); "
            "print(time.perf_counter() - t0)" % ROOT)
    env = dict(os.environ, OMP_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    try:
        res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                             timeout=600, env=env)
        one_core = float(res.stdout.strip().splitlines()[-1])
    except (OSError, subprocess.SubprocessError, ValueError, IndexError):
        one_core = None
    return {"seconds_all_cores": all_cores, "cores": os.cpu_count(), "seconds_one_core": one_core}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    crop = (778, 519)          # a quarter of the view per step keeps K steps within minutes
    if args.warmup > 0:
        cpu_baseline_sample(steps=1, crop=crop)
    cb = cpu_baseline_sample(steps=max(args.steps, 1), crop=crop)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "Mpix/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": cb["seconds_per_step"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": cb["sample"]},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the multi-view, reduced-storage and scene-batch forms")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
