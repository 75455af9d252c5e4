#!/usr/bin/env python3
"""Benchmark of the weight-sharing kernel-prediction denoiser on one B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp8|fp32]
    python bench.py --impl reference ...      # the FP64 CPU oracle as the reference arm

One step = one full denoise (Sec. 5.1 input assembly, the ImportanceNet
convolutions, Eq. 3-5 reconstruction) of a synthetic 1920x1080 1-spp frame
(seed 2, batch 1), inputs resident in HBM.  Prints ONE JSON line.

Timing: W warm-up steps, then K steps each bracketed by CUDA events on the
launching stream; a 256 MiB buffer (> the 126 MB L2) is rewritten between
timed steps, outside the events.  Per-stage times come from the library's
own stage events (wskpn_profile_*), recorded on the same stream.  With N>1
(torchrun) every rank denoises its own frames (replicas only, no
collective on the data path); the reported time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "1080p denoise ms/frame (BF16 vs FP32 plain); p50/p99 frame latency in serving"
UNIT = "ms/frame"
H, W, SEED = 1080, 1920, 2
WIDTHS = (10, 32, 48, 64, 12)
KS = 5
KSIZES = (3, 5, 7, 9, 11, 13)
# algorithmic bytes per pixel of the reconstruction kernel: logits (12 x 4)
# + radiance (3 x 4) + albedo (3 x 4) read, output (3 x 4) written
DECODE_BYTES_PER_PX = 84
FP32_LANES_PER_SM, N_SM, SM_MAX_MHZ = 128, 148, 2032.0
# dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu capture
# of the current kernels at 1920x1080 (profiles/traffic_bf16_1080p.md); the
# reconstruction kernel reads the same bytes whatever the network's precision;
# a kernel absent here has no capture of its current version
TRAFFIC = {
    ("bf16", "prep"): 159.7e6,  # the separate assembly kernel (WSKPN_TUNE_FUSED_PREP = 0)
    ("bf16", "conv1 (10->32)"): 288.0e6,  # with the input assembly inside (the default)
    ("bf16", "conv2 (32->48)"): 604.0e6,
    ("bf16", "conv3 (48->64)"): 872.7e6,
    ("bf16", "conv4 (64->12)"): 614.7e6,
    ("bf16", "decode_fuse_fwd"): 161.8e6,
    ("fp32", "decode_fuse_fwd"): 161.8e6,
    ("fp8", "decode_fuse_fwd"): 161.8e6,
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300, help="timed steps (the paper averages 300 iterations)")
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="wskpn", choices=["wskpn", "reference"])
    p.add_argument("--precision", default="bf16", choices=["bf16", "fp8", "fp32"])
    p.add_argument("--no-fp32", action="store_true", help="skip the FP32 plain-path comparison")
    p.add_argument("--no-fp8", action="store_true", help="skip the FP8 form's timing and error (BF16 runs)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-sweep", action="store_true", help="skip the 720p / 1440p runs")
    p.add_argument("--no-variants", action="store_true", help="skip the 6-block network timing")
    p.add_argument("--train-keep", action="store_true",
                   help="with --train-only: also time the step with the activations kept")
    p.add_argument("--train-only", action="store_true",
                   help="time only the training step (16 crops of 256 x 256) and print its line")
    p.add_argument("--serve-requests", type=int, default=4096)
    p.add_argument("--serve-rate", type=float, default=240.0)
    p.add_argument("--serve-workers", type=int, default=2, help="serving workers (streams with their own context)")
    p.add_argument("--serve-sweep", type=float, nargs="*", default=[480.0, 960.0, 1920.0],
                   help="further offered rates (req/s) for the load sweep")
    p.add_argument("--serve-sweep-requests", type=int, default=2048)
    p.add_argument("--tc-split", type=int, default=None, help="BF16 activations as hi/lo pairs (1, default) or single (0)")
    p.add_argument("--fused-prep", type=int, default=None,
                   help="BF16/FP8: the first convolution assembles its input (1, default) or a separate kernel stores it (0)")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
                "source": "fallback"}


def host_upload_bytes(h: int, w: int) -> int:
    """Bytes wskpn_denoise_host uploads for one frame: every input row
    (10 float32 channels) crosses the host link once; the halo rows a band
    shares with the previous band are copied on the device."""
    return 40 * h * w


# ------------------------------------------------------- replicas (N > 1)
def replica_seed(seed: int, rank: int) -> int:
    """Each rank denoises its own frame (replicas only: no data is exchanged)."""
    return seed + 1000 * rank


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The slowest rank's value (the job ends when it does)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_metrics(ms_per_step_max: float, world: int) -> dict:
    """Whole-job numbers from the slowest rank's ms per step, with one frame
    per rank and step: ms per frame of the job and frames per second."""
    return {"ms_per_step": ms_per_step_max, "ms_per_frame": ms_per_step_max / world,
            "fps": 1e3 * world / ms_per_step_max}


def conv_flops(l, h=H, w=W):
    return 2.0 * WIDTHS[l] * WIDTHS[l + 1] * KS * KS * h * w


def tensor_peak(pk, clocks):
    """The BF16 tensor peak a timed region is compared with: the sustained
    figure of MEASURED_PEAKS.json (matmul back to back for seconds, under the
    power cap) when the region itself ran under the power cap or lasted a
    second or more, else the burst figure.  Returns (TFLOP/s, which)."""
    sustained = bool(clocks) and ("sw_power_cap" in clocks.get("reasons", [])
                                  or (clocks.get("window_ms") or 0.0) >= 1000.0)
    return (pk["bf16_tflops_sustained"], "sustained") if sustained else (pk["bf16_tflops"], "burst")


def stage_rooflines(stage_ms, precision, pk, h=H, w=W, tpeak=None, fused_prep=False):
    """Achieved throughput and fraction of the measured peak for every stage
    (algorithmic FLOPs for the convolutions, algorithmic bytes for the
    streaming kernels), from the stage times of one denoise.  fused_prep: the
    input assembly ran inside conv1 (stage 0 holds no kernel)."""
    L = len(WIDTHS) - 1
    out = {}
    prep_bytes = (40 + {"fp32": 40, "bf16": 64, "fp8": 64}[precision]) * h * w
    for i, ms in enumerate(stage_ms):
        if ms <= 0 or (i == 0 and fused_prep):  # no assembly launch: it runs inside conv1
            continue
        if i == 0 or i == L + 1:
            byts = prep_bytes if i == 0 else DECODE_BYTES_PER_PX * h * w
            gbs = byts / (ms * 1e-3) / 1e9
            out["prep" if i == 0 else "reconstruct"] = {
                "bound": "hbm", "achieved": gbs, "unit": "GB/s", "frac": gbs / pk["hbm_gbs"],
                "traffic": TRAFFIC.get((precision, "prep" if i == 0 else "decode_fuse_fwd")) if (h, w) == (H, W)
                else None}
        else:
            tf = conv_flops(i - 1, h, w) / (ms * 1e-3) / 1e12
            if precision == "fp32":
                peak, bound = N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12, "alu"
            else:
                peak = (tpeak if tpeak is not None else pk["bf16_tflops"]) * (2.0 if precision == "fp8" else 1.0)
                bound = "tensor"
            kname = f"conv{i} ({WIDTHS[i - 1]}->{WIDTHS[i]})"
            out[f"conv{i}"] = {"bound": bound, "achieved": tf, "unit": "TFLOP/s", "frac": tf / peak,
                               "traffic": TRAFFIC.get((precision, kname)) if (h, w) == (H, W) else None}
    return out


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampled every 50 ms by a reader thread; only the samples
    taken between mark_start() and mark_end() (the timed steps) are
    reported, or the last one before mark_end() when the timed region is
    shorter than the sampling period."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.lines = []  # (monotonic time, line)
        self.t0 = self.t1 = None

    def start(self, wait_s: float = 3.0):
        import threading
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                self.lines.append((time.monotonic(), line))
        threading.Thread(target=reader, daemon=True).start()
        t = time.monotonic()
        while not self.lines and time.monotonic() - t < wait_s:  # nvidia-smi is sampling
            time.sleep(0.01)

    def mark_start(self):
        self.t0 = time.monotonic()

    def mark_end(self):
        self.t1 = time.monotonic()

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        t0 = self.t0 if self.t0 is not None else -1e30
        t1 = self.t1 if self.t1 is not None else 1e30
        inside = [ln for t, ln in self.lines if t0 <= t <= t1]
        if not inside:
            before = [ln for t, ln in self.lines if t <= t1]
            inside = before[-1:]
        sm, mx, reasons = [], [], set()
        for line in inside:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons),
                "window_ms": (t1 - t0) * 1e3 if self.t0 is not None and self.t1 is not None else None}


# -------------------------------------------------------------- reference
def run_reference(args):
    """The FP64 CPU oracle, as it stands, on bounded row bands of the same
    1080p frame; each step denoises ROWS rows and is scaled to ms/frame."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import synth
    rows = 16
    f = synth.make_frame(H, W, SEED)
    wb = synth.make_weights(WIDTHS, KS, seed=SEED)
    times = []
    for i in range(args.warmup + args.steps):
        y0 = (H // 2 + 37 * i) % (H - rows)
        t0 = time.perf_counter()
        oracle.denoise(f, wb, widths=WIDTHS, ks=KS, ksizes=KSIZES, rect=(0, y0, W, y0 + rows))
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    ms_frame = statistics.mean(times) * 1e3 * H / rows
    sample = f"{args.steps} bands of {rows} x {W} px (rows near the middle) of the 1920x1080 seed-2 frame, " \
             f"each computed with its receptive-field halo, scaled x{H // rows} to a full frame"
    line = {
        "impl": "reference", "metric": METRIC, "value": ms_frame, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(times) * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_block("fp64 oracle"),
        "cpu_baseline": {"value": ms_frame, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": ms_frame, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_block(precision):
    return {"workload": "synthetic 1-spp frame 1920x1080, seed 2, batch 1 (BMFR-like stand-in)",
            "resolution": f"{W}x{H}", "batch": 1, "precision": precision,
            "network": "ImportanceNet 3 blocks 10-32-48-64 + output conv to 12, 5x5 convs",
            "kernel_sizes": list(KSIZES), "l2": "flushed between timed steps (256 MiB write)"}


def _pct(v, p):
    v = sorted(v)
    return v[min(len(v) - 1, int(p * (len(v) - 1) + 0.5))] if v else None


def serving_run(wk_serving, synth, torch, np, n_req, rate, wb, dev, n_workers=2, warm=True):
    """Serving form: n_req requests, Poisson arrivals at `rate`/s from 8
    client streams, sizes uniform over 720p / 1080p / 1440p, BF16.  Each
    request's timeline comes back with its delivery (wskpn_serve_wait_info):
    latency percentiles per resolution, batch sizes, and how long batches of
    the two workers were in flight at the same time."""
    sizes = [(720, 1280), (1080, 1920), (1440, 2560)]
    keys = ("radiance", "albedo", "normal", "depth")
    frames = []
    for i, (h, w) in enumerate(sizes):
        f = synth.make_frame(h, w, 11 + i)
        frames.append([torch.from_numpy(np.ascontiguousarray(f[k][None])).to(dev) for k in keys])
    mk = lambda: wk_serving.Server(wb, "bf16", max_hw=(1440, 2560), n_workers=n_workers, max_batch=4,
                                   mem_budget=8 << 30, batch_window_us=0)
    n_streams = 8
    outs = {(s, r): torch.empty((1, 3, *sizes[r]), device=dev) for s in range(n_streams) for r in range(3)}
    busy = {}
    g = np.random.default_rng(240)
    arrivals = np.cumsum(g.exponential(1.0 / rate, n_req))
    res = g.integers(0, 3, n_req)
    if warm:  # load every kernel once in a throw-away server
        srv = mk()
        for r in range(3):
            t = srv.submit(0, *frames[r], outs[(0, r)])
            srv.wait(t, 60000)
        srv.stop()
    srv = mk()
    for r in range(3):  # capture outside the measured stream
        t = srv.submit(0, *frames[r], outs[(0, r)])
        srv.wait(t, 60000)
    stats0 = srv.stats()
    infos = []
    t0 = time.perf_counter()
    late = 0
    for i in range(n_req):
        now = time.perf_counter() - t0
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
        sid, r = i % n_streams, int(res[i])
        prev = busy.get((sid, r))
        if prev is not None:
            s_, info = srv.wait_info(prev, 0)
            if info is None:
                late += 1
                s_, info = srv.wait_info(prev, -1)
            infos.append(info)
        busy[(sid, r)] = srv.submit(sid, *frames[r], outs[(sid, r)])
    for t in busy.values():
        infos.append(srv.wait_info(t, -1)[1])
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.stop()
    done = st["completed"] - stats0["completed"]
    per_res = {}
    for (h, w) in sizes:
        lat = [x["done_ms"] - x["submit_ms"] for x in infos if x and (x["h"], x["w"]) == (h, w)]
        per_res[f"{w}x{h}"] = {"n": len(lat), "p50_ms": _pct(lat, 0.5), "p99_ms": _pct(lat, 0.99)}
    lat_all = [x["done_ms"] - x["submit_ms"] for x in infos if x]
    # time during which batches of different workers were in flight together
    spans = {}
    for x in infos:
        if x and x["worker"] >= 0:
            spans.setdefault(x["worker"], set()).add((x["dispatch_ms"], x["done_ms"]))
    overlap = 0.0
    ws = sorted(spans)
    if len(ws) >= 2:
        ev = []
        for k in ws:
            for (a, b) in spans[k]:
                ev += [(a, 1, k), (b, -1, k)]
        ev.sort()
        live = {k: 0 for k in ws}
        last = None
        for tms, d, k in ev:
            if last is not None and sum(1 for v in live.values() if v > 0) >= 2:
                overlap += tms - last
            live[k] += d
            last = tms
    return {"requests": n_req, "rate_per_s": rate, "streams": n_streams, "workers": n_workers,
            "sizes": ["1280x720", "1920x1080", "2560x1440"], "precision": "bf16",
            "p50_ms": _pct(lat_all, 0.5), "p99_ms": _pct(lat_all, 0.99), "mean_ms": st["mean_ms"],
            "max_ms": st["max_ms"], "per_resolution": per_res,
            "fps": done / wall, "mean_batch": st["mean_batch"], "batches": st["batches"],
            "graph_launches": st["graph_launches"], "rejected": st["rejected"], "failed": st["failed"],
            "workers_in_flight_together_ms": overlap, "wall_s": wall,
            "mem_peak_gib": st["mem_peak"] / 2 ** 30, "client_waits_for_own_buffer": late,
            "note": "latency submit->delivery of the measured requests (the warm-up request of each size excluded)"}


def cpu_baseline():
    """The FP64 oracle, as it stands, on the whole 1920x1080 seed-2 frame
    (one frame, wall clock, all host cores).  Returns the baseline entry and
    the oracle's output, which the precision form's errors are taken
    against."""
    import oracle
    import synth
    f = synth.make_frame(H, W, SEED)
    wb = synth.make_weights(WIDTHS, KS, seed=SEED)
    t0 = time.perf_counter()
    ref = oracle.denoise(f, wb, widths=WIDTHS, ks=KS, ksizes=KSIZES)
    el = time.perf_counter() - t0
    return {"value": el * 1e3, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"the whole 1920x1080 seed-2 frame, once ({el:.1f} s)"}, ref


def oracle_errors(out, ref):
    """Max and mean of |x - ref| / max(|ref|, 1e-6) over every element."""
    import numpy as np
    e = np.abs(out.astype(np.float64) - ref) / np.maximum(np.abs(ref), 1e-6)
    return {"max_rel_err_vs_oracle": float(e.max()), "mean_rel_err_vs_oracle": float(e.mean())}


# --------------------------------------------------------------- our arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2202_05977_b300 as wk
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")

    def barrier():
        if world > 1:
            dist.barrier()

    dev = torch.device("cuda", local)
    f = synth.make_frame(H, W, replica_seed(SEED, rank))
    wb = synth.make_weights(WIDTHS, KS, seed=SEED)
    keys = ("radiance", "albedo", "normal", "depth")
    xin = [torch.from_numpy(np.ascontiguousarray(f[k][None])).to(dev) for k in keys]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    pk = peaks()

    def time_training(steps, warmup, keep=False):
        """The differentiation form: one training step on 16 crops of 256 x
        256 (BF16 forward, L1 loss against the mean of 256 noise draws,
        hand-written backward with the activations recomputed, Adam).  With
        keep, the forward keeps the layer inputs for the backward instead
        (WSKPN_TUNE_TRAIN_KEEP = 1)."""
        tb = synth.make_batch(16, 256, 256, seed=5)
        ttg = torch.from_numpy(synth.make_target(tb["clean"], seed=5, draws=256)).to(dev)
        tx = [torch.from_numpy(np.ascontiguousarray(tb[k])).to(dev) for k in keys]
        dt = wk.Denoiser(wb, precision="bf16", max_batch=16, max_hw=(256, 256))
        if keep:
            dt.set_tuning(11, 1)
        t_it = 1

        def train_step():
            nonlocal t_it
            o, zz = dt.forward_train(*tx)
            _, dout = dt.l1_loss(o, ttg)
            dw, _ = dt.backward(*tx, zz, dout)
            dt.adam_step(dw, t_it, lr=1e-4)
            t_it += 1

        for _ in range(warmup):
            train_step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            train_step()
        e1.record()
        torch.cuda.synchronize()
        ms_t = e0.elapsed_time(e1) / steps
        dt.close()
        return {"precision": "bf16", "activations": "kept" if keep else "recomputed", "ms_per_step": ms_t,
                "crops_per_s": 16e3 / ms_t}

    if args.train_only:
        # the differentiation form alone (for profiling its launches)
        r = time_training(args.steps, args.warmup)
        rk = time_training(args.steps, args.warmup, keep=True) if args.train_keep else None
        if rank == 0:
            line = {"metric": "training step ms (16 crops of 256 x 256, BF16, activations recomputed)",
                    "value": r["ms_per_step"], "unit": "ms/step", "steps": args.steps, "warmup": args.warmup,
                    "higher_is_better": False, "crops_per_s": r["crops_per_s"], "data": "synthetic"}
            if rk:
                line["kept_activations"] = rk
            print(json.dumps(line))
        return

    # the first layer assembles its input inside its own kernel (no prep launch)
    fused_prep_on = args.fused_prep != 0 and (args.precision == "fp8" or (args.precision == "bf16"
                                                                          and args.tc_split != 0))

    def time_path(precision, steps, warmup, hw=(H, W), frame=None, widths=WIDTHS, weights=None, ks=KS, clk=None,
                  fused_prep=None):
        h, w = hw
        xs = xin if frame is None else frame
        d = wk.Denoiser(wb if weights is None else weights, precision=precision, max_hw=(h, w), widths=widths,
                        conv_ks=ks)
        if args.tc_split is not None and precision == "bf16":
            d.set_tuning(2, args.tc_split)
        fp = fused_prep if fused_prep is not None else args.fused_prep
        if fp is not None and precision in ("bf16", "fp8"):
            d.set_tuning(12, fp)  # WSKPN_TUNE_FUSED_PREP
        if precision == "fp8":  # static activation scales from a different frame (seed 3)
            cal = synth.make_frame(h, w, SEED + 1)
            d.calibrate(*[torch.from_numpy(np.ascontiguousarray(cal[k][None])).to(dev) for k in keys])
        out = torch.empty((1, 3, h, w), device=dev)
        for _ in range(warmup):
            d.denoise(*xs, out=out)
        torch.cuda.synchronize()
        barrier()
        # the timed steps run without the per-stage events (an event between
        # two kernels would also keep the next layer from starting its set-up
        # during the previous one's tail); the stage split comes from extra
        # steps with the events on
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if clk:
            clk.mark_start()
        t_wall = time.perf_counter()
        for i in range(steps):
            flush.fill_(float(i))
            ev[i][0].record()
            d.denoise(*xs, out=out)
            ev[i][1].record()
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        if clk:
            clk.mark_end()
        barrier()
        d.profile(True)
        for i in range(max(3, steps // 2)):
            flush.fill_(float(i))
            d.denoise(*xs, out=out)
        torch.cuda.synchronize()
        d.profile(False)
        stage_ms, calls = d.profile_read()
        per = [a.elapsed_time(b) for a, b in ev]
        total = max_over_ranks(sum(per), dist if world > 1 else None, dev)
        res = {"ms_step": total / steps, "per": per, "stage_ms": [s / max(calls, 1) for s in stage_ms],
               "wall_s": t_wall, "out": out, "d": d}
        return res

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clk = ClockSampler(uuid)
    clk.start()
    main_res = time_path(args.precision, args.steps, args.warmup, clk=clk)
    clocks = clk.stop()

    fp32 = None
    fp32_720 = None
    if not args.no_fp32 and args.precision != "fp32":
        fp32 = time_path("fp32", max(3, args.steps // 4), 3)
        # the plain FP32 path on the 1280x720 seed-1 frame (its oracle is
        # timed with the CPU baseline below)
        f720p = synth.make_frame(720, 1280, replica_seed(1, rank))
        x720p = [torch.from_numpy(np.ascontiguousarray(f720p[k][None])).to(dev) for k in keys]
        r720 = time_path("fp32", max(3, args.steps // 4), 3, (720, 1280), x720p)
        fp32_720 = {"ms": r720["ms_step"], "out": r720["out"].cpu().numpy()[0], "frame": f720p}
        del r720

    # the precision form: the same frame through the BF16 and FP8 forms, each
    # output against the FP32 path's and (after the CPU baseline has run the
    # oracle on the whole frame) against the FP64 oracle's, per element
    # |x - ref| / max(|ref|, 1e-6)
    precision_form = None
    form_out = {}
    if fp32 is not None and args.precision == "bf16":
        def err_vs_fp32(out):
            ref = fp32["out"]
            e = (out - ref).abs() / ref.abs().clamp_min(1e-6)
            return {"max_rel_err_vs_fp32": float(e.max()), "mean_rel_err_vs_fp32": float(e.mean())}
        precision_form = {"bf16": {"ms_per_frame": main_res["ms_step"], **err_vs_fp32(main_res["out"])}}
        form_out = {"bf16": main_res["out"].cpu().numpy()[0], "fp32": fp32["out"].cpu().numpy()[0]}
        if not args.no_fp8:
            r8 = time_path("fp8", max(5, args.steps // 2), 3)
            precision_form["fp8"] = {"ms_per_frame": r8["ms_step"], "form": "e4m3 hi/lo activations and weights",
                                     "calibration": f"static scales from the seed-{SEED + 1} frame",
                                     "stages_ms": {k: v for k, v in zip(["prep"] + [f"conv{i + 1}" for i in range(len(WIDTHS) - 1)]
                                                                       + ["reconstruct"], r8["stage_ms"])
                                                   if not (k == "prep" and args.fused_prep != 0)},
                                     **err_vs_fp32(r8["out"])}
            form_out["fp8"] = r8["out"].cpu().numpy()[0]
            del r8

    # the same path at 720p and 1440p (seeds 1 and 3), for ms/frame, frames/s
    # and the per-stage roofline fractions at each resolution
    sweep = {}
    if not args.no_sweep:
        for (h, w), sd in (((720, 1280), 1), ((1440, 2560), 3)):
            fr = synth.make_frame(h, w, replica_seed(sd, rank))
            xs = [torch.from_numpy(np.ascontiguousarray(fr[k][None])).to(dev) for k in keys]
            r = time_path(args.precision, max(5, args.steps // 2), 3, (h, w), xs)
            sweep[f"{w}x{h}"] = {"ms_per_frame": r["ms_step"], "fps": 1e3 / r["ms_step"],
                                 "stage_rooflines": stage_rooflines(r["stage_ms"], args.precision, pk, h, w,
                                                                    fused_prep=fused_prep_on)}
            del r

    # the paper's 6-block quality variant of ImportanceNet (Sec. 4.1), widths
    # 10-32-48-64-64-64-64 + output conv to 12, at 720p (the paper's timing
    # resolution) and 1080p
    variants = {}
    if not args.no_variants and args.precision != "fp8":
        w6 = (10, 32, 48, 64, 64, 64, 64, 12)
        wb6 = synth.make_weights(w6, KS, seed=SEED)
        f720 = synth.make_frame(720, 1280, replica_seed(1, rank))
        x720 = [torch.from_numpy(np.ascontiguousarray(f720[k][None])).to(dev) for k in keys]
        six = {}
        for (h, w), xs in (((720, 1280), x720), ((H, W), None)):
            r = time_path(args.precision, max(5, args.steps // 2), 3, (h, w), xs, w6, wb6)
            six[f"{w}x{h}"] = {"ms_per_frame": r["ms_step"], "fps": 1e3 / r["ms_step"],
                               "prediction_ms": sum(r["stage_ms"][:-1]), "reconstruction_ms": r["stage_ms"][-1]}
            del r
        if not args.no_fp32 and args.precision != "fp32":
            r = time_path("fp32", 3, 2, (720, 1280), x720, w6, wb6)
            six["1280x720"]["fp32_ms_per_frame"] = r["ms_step"]
            del r
        variants["six_blocks"] = six
        # the 3x3 form of the same network (the configuration text's kernel
        # size; Sec. 4.1's 5x5 is the primary form) at 1080p
        wb3 = synth.make_weights(WIDTHS, 3, seed=SEED)
        c3 = {}
        for prec in ("bf16", "fp8"):
            r = time_path(prec, max(5, args.steps // 2), 3, (H, W), None, WIDTHS, wb3, 3)
            c3[f"{prec}_ms_per_frame"] = r["ms_step"]
            del r
        variants["conv3x3_1920x1080"] = c3
        if args.precision == "bf16":
            # the input assembly as its own kernel, its output stored in HBM
            # and read back by conv1 (the default runs it inside conv1)
            r = time_path("bf16", max(5, args.steps // 2), 3, fused_prep=0)
            variants["separate_input_assembly_1920x1080"] = {
                "ms_per_frame": r["ms_step"],
                "stages_ms": dict(zip(["prep"] + [f"conv{i + 1}" for i in range(len(WIDTHS) - 1)] + ["reconstruct"],
                                      r["stage_ms"]))}
            del r
        variants["training_step_16x256x256"] = time_training(max(5, args.steps // 4), 3)
        variants["training_step_16x256x256_kept_activations"] = time_training(max(5, args.steps // 4), 3, keep=True)
    if not args.no_variants:
        # the multi-resolution variant (U-Net, 3 levels, kernels 3 and 5, Eq. 7), FP32
        from paper_2202_05977_b300.multires import MultiResDenoiser
        from paper_2202_05977_b300.multires import n_weights as mr_n
        g = np.random.default_rng(SEED)
        wmr = (g.standard_normal(mr_n()) * 0.05).astype(np.float32)
        mres = {}
        for (h, w), sd in (((720, 1280), 1), ((H, W), SEED)):
            fr = synth.make_frame(h, w, replica_seed(sd, rank))
            xs = [torch.from_numpy(np.ascontiguousarray(fr[k][None])).to(dev) for k in keys]
            entry = {}
            for prec in ("bf16", "fp32"):
                dm = MultiResDenoiser(wmr, max_hw=(h, w), precision=prec)
                o = torch.empty((1, 3, h, w), device=dev)
                for _ in range(3):
                    dm.denoise(*xs, out=o)
                torch.cuda.synchronize()
                n_it = max(5, args.steps // 2)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                tot = 0.0
                for i in range(n_it):
                    flush.fill_(float(i))
                    e0.record()
                    dm.denoise(*xs, out=o)
                    e1.record()
                    torch.cuda.synchronize()
                    tot += e0.elapsed_time(e1)
                entry[f"{prec}_ms_per_frame"] = tot / n_it
                dm.close()
            entry["fps_bf16"] = 1e3 / entry["bf16_ms_per_frame"]
            mres[f"{w}x{h}"] = entry
        variants["multires_unet"] = mres
        # temporal accumulation (Sec. 4.3) on a 1080p moving-camera pair: one
        # step reads the frame (radiance, position, normal, motion: 44 B/px)
        # and the previous state (40 B/px) and writes the state and the
        # accumulated radiance (52 B/px)
        from paper_2202_05977_b300.temporal import TemporalAccumulator
        seq = synth.make_sequence(H, W, 2, seed=replica_seed(SEED, rank))
        tin = [{k: torch.from_numpy(np.ascontiguousarray(f[k])).to(dev)
                for k in ("radiance", "position", "normal", "motion")} for f in seq]
        ta = TemporalAccumulator(H, W)
        acc = torch.empty((3, H, W), device=dev)
        for f in tin:
            ta.step(f["radiance"], f["position"], f["normal"], f["motion"], out=acc)
        torch.cuda.synchronize()
        n_it = max(10, args.steps)
        tot = 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for i in range(n_it):
            flush.fill_(float(i))
            f = tin[1]
            e0.record()
            ta.step(f["radiance"], f["position"], f["normal"], f["motion"], out=acc)
            e1.record()
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        ms = tot / n_it
        variants["temporal_accumulation"] = {"resolution": f"{W}x{H}", "ms_per_frame": ms,
                                             "achieved_gbs": 136 * H * W / (ms * 1e-3) / 1e9,
                                             "frac_hbm": 136 * H * W / (ms * 1e-3) / 1e9 / pk["hbm_gbs"]}
        ta.close()

    # roofline of the dominant stage (stage 0 prep, 1..L convs, L+1 reconstruction)
    st = main_res["stage_ms"]
    dom = max(range(len(st)), key=lambda i: st[i])
    if 1 <= dom <= len(WIDTHS) - 1:
        l = dom - 1
        flops = conv_flops(l)
        achieved = flops / (st[dom] * 1e-3) / 1e12
        if args.precision == "fp32":
            peak = N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
            bound, psrc = "alu", "derived: 148 SMs x 128 FP32 lanes x 2 FLOP x 2032 MHz"
        else:
            tp, which = tensor_peak(pk, clocks)
            peak = tp * (2.0 if args.precision == "fp8" else 1.0)
            bound, psrc = "tensor", f"{pk['source']} bf16 {which}" + (" x2 (fp8 nominal ratio)" if args.precision == "fp8" else "")
        kname = f"conv{l + 1} ({WIDTHS[l]}->{WIDTHS[l + 1]})"
        roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": TRAFFIC.get((args.precision, kname)), "kernel": kname, "peak_source": psrc}
        if args.precision != "fp32":
            roof["frac_of_burst"] = achieved / (pk["bf16_tflops"] * (2.0 if args.precision == "fp8" else 1.0))
    else:
        name = "prep" if dom == 0 else "decode_fuse_fwd"
        byts = (40 + {"fp32": 40, "bf16": 64, "fp8": 64}[args.precision]) * H * W if dom == 0 \
            else DECODE_BYTES_PER_PX * H * W
        achieved = byts / (st[dom] * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": TRAFFIC.get((args.precision, name)), "kernel": name,
                "peak_source": pk["source"] + " copy bandwidth"}

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        d = main_res["d"]
        hin = [t.cpu().pin_memory() for t in xin]
        hout = torch.empty((1, 3, H, W), dtype=torch.float32).pin_memory()
        for _ in range(2):
            d.denoise_host(*hin, hout)
        barrier()
        ts = []
        for _ in range(max(3, args.steps // 2)):
            t0 = time.perf_counter()
            d.denoise_host(*hin, hout)
            ts.append((time.perf_counter() - t0) * 1e3)
        t_sync = statistics.mean(ts)
        # a stream of frames: each step's call returns once its copies and
        # kernels are queued (wskpn_denoise_host_async), so a frame's first
        # bands cross the host link while the previous frame's last bands
        # compute; every step still uploads its inputs and downloads its
        # result inside the timed region, which ends with a synchronisation
        cs = torch.cuda.current_stream()
        for _ in range(3):
            d.denoise_host(*hin, hout, wait=False)
        cs.synchronize()
        barrier()
        n_async = max(3, args.steps // 2)
        t0 = time.perf_counter()
        for _ in range(n_async):
            d.denoise_host(*hin, hout, wait=False)
        cs.synchronize()
        t_async = (time.perf_counter() - t0) * 1e3 / n_async
        tt = max_over_ranks(t_async, dist if world > 1 else None, dev)
        e2e = {"value": job_metrics(tt, world)["ms_per_frame"], "unit": UNIT,
               "h2d_bytes_per_step": host_upload_bytes(H, W),
               "d2h_bytes_per_step": 12 * H * W, "per_rank_ms_per_frame": tt,
               "api": "wskpn_denoise_host_async, one synchronisation after the timed steps",
               "sync_call_ms_per_frame": max_over_ranks(t_sync, dist if world > 1 else None, dev)}

    if rank == 0:
        L = len(WIDTHS) - 1
        stage_names = ["prep"] + [f"conv{l + 1}" for l in range(L)] + ["reconstruct"]
        line = {
            "metric": METRIC,
            "value": job_metrics(main_res["ms_step"], world)["ms_per_frame"],
            "unit": UNIT,
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": main_res["ms_step"],
            "higher_is_better": False,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": args.precision,
            "data": "synthetic",
            "config": config_block(args.precision),
            "fps": job_metrics(main_res["ms_step"], world)["fps"],
            "stages_ms": {k: v for k, v in zip(stage_names, main_res["stage_ms"]) if not (k == "prep" and fused_prep_on)},
            "prediction_ms": sum(main_res["stage_ms"][:L + 1]),
            "reconstruction_ms": main_res["stage_ms"][L + 1],
            "p50_step_ms": statistics.median(main_res["per"]),
            "p99_step_ms": sorted(main_res["per"])[min(len(main_res["per"]) - 1,
                                                      int(round(0.99 * (len(main_res["per"]) - 1))))],
            "roofline": roof,
            "stage_rooflines": stage_rooflines(main_res["stage_ms"], args.precision, pk,
                                               tpeak=tensor_peak(pk, clocks)[0], fused_prep=fused_prep_on),
            "input_assembly": "inside conv1 (its producer warps)" if fused_prep_on else "separate kernel",
            "gpu_launches": args.steps * (L + (1 if fused_prep_on else 2)),
            "clocks": clocks,
        }
        if sweep:
            sweep["1920x1080"] = {"ms_per_frame": main_res["ms_step"], "fps": 1e3 / main_res["ms_step"],
                                  "stage_rooflines": line["stage_rooflines"]}
            line["resolutions"] = sweep
        if variants:
            line["variants"] = variants
        # the paper's own timings (1280x720, RTX 2080 Ti, precision not stated):
        # context only, another machine and resolution
        line["paper_context"] = {"hardware": "RTX 2080 Ti", "resolution": "1280x720",
                                 "ms_per_frame": {"3_blocks": 6.58, "6_blocks": 12.89, "multires": 22.70}}
        if precision_form is not None:
            line["precision_form"] = precision_form
        if fp32 is not None:
            line["fp32_ms_per_frame"] = fp32["ms_step"] / world
            line["speedup_vs_fp32"] = fp32["ms_step"] / main_res["ms_step"]
            line["fp32_stages_ms"] = dict(zip(stage_names, fp32["stage_ms"]))
        if e2e is not None:
            line["e2e"] = e2e
        if not args.no_serving:
            import paper_2202_05977_b300.serving as wk_serving
            line["serving"] = serving_run(wk_serving, synth, torch, np, args.serve_requests, args.serve_rate, wb, dev,
                                          args.serve_workers)
            # offered load beyond the configured 240 req/s: where frames/s stops rising
            sweep = []
            for rate in args.serve_sweep:
                r_ = serving_run(wk_serving, synth, torch, np, args.serve_sweep_requests, rate, wb, dev,
                                 args.serve_workers, warm=False)
                sweep.append({k: r_[k] for k in ("rate_per_s", "requests", "fps", "mean_batch", "p50_ms", "p99_ms",
                                                 "per_resolution", "workers_in_flight_together_ms", "wall_s",
                                                 "rejected", "failed")})
            line["serving_sweep"] = sweep
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"], ref = cpu_baseline()
            if fp32_720 is not None:
                # the plain FP32 path at 1280x720 against the FP64 oracle on the
                # host cores: time per frame of each, error over every pixel
                import oracle
                wb720 = synth.make_weights(WIDTHS, KS, seed=SEED)
                t0 = time.perf_counter()
                ref720 = oracle.denoise(fp32_720["frame"], wb720, widths=WIDTHS, ks=KS, ksizes=KSIZES)
                el = time.perf_counter() - t0
                line["plain_fp32_720p"] = {"ms_per_frame": fp32_720["ms"], "oracle_ms_per_frame": el * 1e3,
                                           "oracle_cores": oracle.num_threads(),
                                           "speedup_vs_oracle": el * 1e3 / fp32_720["ms"],
                                           **oracle_errors(fp32_720["out"], ref720)}
            # every pixel of the precision forms against the FP64 oracle
            if precision_form is not None:
                for prec, o in form_out.items():
                    if prec in precision_form:
                        precision_form[prec].update(oracle_errors(o, ref))
                precision_form["fp32"] = {"ms_per_frame": fp32["ms_step"], **oracle_errors(form_out["fp32"], ref)}
                line["precision_form"] = precision_form
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
